"""Pins of the oracle's multigrid preconditioner (oracle/oracle.c, ORC_M_MG)
against facts that do not come from the oracle's own loops: the Galerkin
identity A_c = P^T A P built densely, symmetry and positivity of the cycle, the
one- and two-grid cycles written as dense matrix products, and convergence."""
import numpy as np
import pytest

import oracle
from paper_2203_13675_gb300 import synth

OMEGA, NU, CC, COARSE_SWEEPS = 2.0 / 3.0, 2, 1.5, 30


def _weights(H, W, seed, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    U = rng.uniform(0.05, 1.0, (H, W))
    V = rng.uniform(0.05, 1.0, (H, W))
    if zero_frac:
        U[rng.random((H, W)) < zero_frac] = 0.0
        V[rng.random((H, W)) < zero_frac] = 0.0
    U[:, -1] = 0.0
    V[-1, :] = 0.0
    return U, V


def _dense(U, V):
    z = np.zeros_like(U)
    return oracle.assemble(U, V, z, z)


def _prolongation(H, W):
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    P = np.zeros((H * W, Hc * Wc))
    for i in range(H):
        for j in range(W):
            P[i * W + j, (i // 2) * Wc + j // 2] = 1.0
    return P


@pytest.mark.parametrize("H,W", [(5, 7), (8, 6), (1, 9), (9, 1), (4, 4)])
def test_coarse_operator_is_galerkin(H, W):
    U, V = _weights(H, W, H * 10 + W, zero_frac=0.2)
    A = _dense(U, V).dense()
    P = _prolongation(H, W)
    Uc, Vc = oracle.mg_coarsen(U, V)
    Ac = _dense(Uc, Vc).dense()
    np.testing.assert_allclose(Ac, P.T @ A @ P, rtol=0, atol=1e-13)


def _apply(U, V, r, mask=None):
    A = _dense(U, V)
    return oracle.precond_apply(oracle.M_MG, A, r, mask=mask)


def test_cycle_is_symmetric_and_positive():
    H, W = 23, 18
    U, V = _weights(H, W, 3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((H, W))
    y = rng.standard_normal((H, W))
    Mx, My = _apply(U, V, x), _apply(U, V, y)
    a, b = np.sum(y * Mx), np.sum(x * My)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)
    for k in range(5):
        z = rng.standard_normal((H, W))
        assert np.sum(z * _apply(U, V, z)) > 0.0


def _jacobi_sweeps(A, D, b, x, nu):
    S = np.where(D > 0, OMEGA / np.where(D > 0, D, 1.0), 0.0)
    for _ in range(nu):
        x = x + S * (b - A @ x)
    return x


def test_single_grid_cycle_is_damped_jacobi():
    # at most 16 unknowns: the cycle is the coarsest-grid solve alone
    H, W = 4, 4
    U, V = _weights(H, W, 5)
    A = _dense(U, V).dense()
    D = np.diag(A)
    r = np.random.default_rng(6).standard_normal(H * W)
    ref = _jacobi_sweeps(A, D, r, np.zeros(H * W), COARSE_SWEEPS)
    np.testing.assert_allclose(_apply(U, V, r.reshape(H, W)).ravel(), ref, rtol=1e-12, atol=1e-12)


def test_two_grid_cycle_in_matrix_form():
    H, W = 8, 4  # 32 unknowns -> a 4 x 2 coarse grid (8 unknowns), two grids
    U, V = _weights(H, W, 7)
    A = _dense(U, V).dense()
    D = np.diag(A)
    P = _prolongation(H, W)
    Ac = P.T @ A @ P
    Dc = np.diag(Ac)
    b = np.random.default_rng(8).standard_normal(H * W)
    x = _jacobi_sweeps(A, D, b, np.zeros(H * W), NU)
    xc = _jacobi_sweeps(Ac, Dc, P.T @ (b - A @ x), np.zeros(Ac.shape[0]), COARSE_SWEEPS)
    x = x + CC * (P @ xc)
    x = _jacobi_sweeps(A, D, b, x, NU)
    np.testing.assert_allclose(_apply(U, V, b.reshape(H, W)).ravel(), x, rtol=1e-11, atol=1e-11)


def test_masked_pixels_get_zero():
    m = synth.phase_map(24, 30, 9, mask_frac=0.1)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros_like(m.psi), dx, dy, m.mask, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    s = oracle.precond_apply(oracle.M_MG, A, A.b, mask=m.mask)
    assert np.all(s[m.mask == 1] == 0.0) and np.any(s != 0.0)


def test_multigrid_pcg_needs_far_fewer_iterations_than_jacobi():
    m = synth.phase_map(128, 128, 3, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=0.05)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros_like(m.psi), dx, dy, m.mask, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    _, sj = oracle.pcg(A, np.zeros_like(m.psi), kind=oracle.M_JACOBI, tol=1e-6, mask=m.mask)
    phi, sm = oracle.pcg(A, np.zeros_like(m.psi), kind=oracle.M_MG, tol=1e-6, mask=m.mask)
    assert sm["status"] == oracle.OK and sm["true_relres"] < 2e-6
    assert sm["iters"] * 10 < sj["iters"], (sm["iters"], sj["iters"])
