"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Table 1), closed forms, textbook special cases, invariants of the
discrete operator, brute force on tiny grids.  A plausible slip in the oracle
(a dropped term, a wrong sign or index, a transposed operand) breaks one of
them.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2203_13675_gb300 import synth

PI = math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. (wrapped)
def test_wrap_range_and_tie_break():
    # psi in (-pi, pi]: the half-open interval puts both +pi and -pi at +pi
    assert oracle.wrap(PI) == PI
    assert oracle.wrap(-PI) == PI
    assert oracle.wrap(3 * PI) == pytest.approx(PI, abs=1e-15)
    assert oracle.wrap(0.0) == 0.0
    assert oracle.wrap(-1e-300) == -1e-300
    x = np.linspace(-20, 20, 40001)
    w = oracle.wrap(x)
    assert np.all(w > -PI) and np.all(w <= PI)
    k = (x - w) / (2 * PI)                          # x - W(x) is a multiple of 2 pi
    assert np.max(np.abs(k - np.round(k))) < 1e-13
    inside = (x > -PI) & (x <= PI)                  # identity on the principal interval
    assert np.array_equal(w[inside], x[inside])


def test_wrapped_diffs_hand_worked():
    # psi = [[0, 3, -3], [1, -2, 2]]  (2 rows, 3 columns), worked by hand:
    #   Dx row 0: W(3-0)=3, W(-3-3)=W(-6)=2pi-6, ghost 0
    #   Dx row 1: W(-2-1)=-3, W(2+2)=W(4)=4-2pi, ghost 0
    #   Dy row 0: W(1-0)=1, W(-2-3)=W(-5)=2pi-5, W(2+3)=W(5)=5-2pi; row 1 ghost 0
    psi = np.array([[0.0, 3.0, -3.0], [1.0, -2.0, 2.0]])
    dx, dy = oracle.wrapped_diffs(psi)
    np.testing.assert_allclose(dx, [[3.0, 2 * PI - 6, 0.0], [-3.0, 4 - 2 * PI, 0.0]], atol=1e-15)
    np.testing.assert_allclose(dy, [[1.0, 2 * PI - 5, 5 - 2 * PI], [0.0, 0.0, 0.0]], atol=1e-15)


def test_wrapped_diffs_recover_small_true_gradients():
    # a phase whose true differences are below pi: Delta equals the true differences
    m = synth.smooth_map(40, 50, seed=3)
    dx, dy = oracle.wrapped_diffs(m.psi)
    tx = np.diff(m.phi_true, axis=1)
    ty = np.diff(m.phi_true, axis=0)
    assert np.max(np.abs(tx)) < PI and np.max(np.abs(ty)) < PI
    np.testing.assert_allclose(dx[:, :-1], tx, atol=1e-12)
    np.testing.assert_allclose(dy[:-1, :], ty, atol=1e-12)


# ---------------------------------------------------------------- Eq. (UV)
@pytest.mark.parametrize("p", [0.0, 0.5, 1.0, 1.5])
def test_weights_half_point_and_unit_at_zero_residual(p):
    tau = 0.01
    H, W = 3, 4
    # residual e on edge (0,0)-(0,1) with |e|^(2-p) = tau gives U = 1/2 exactly
    e = tau ** (1.0 / (2.0 - p))
    phi = np.zeros((H, W))
    phi[0, 1] = e
    dx = np.zeros((H, W))
    dy = np.zeros((H, W))
    U, V = oracle.weights(phi, dx, dy, None, p, tau)
    assert U[0, 0] == pytest.approx(0.5, rel=1e-12)
    # zero residual gives weight 1 for p < 2 (tau / (0 + tau))
    assert U[2, 1] == 1.0 and V[2, 2] == 0.0 and V[1, 3] == 1.0
    # boundary edges carry zero weight (zero-flux condition)
    assert np.all(U[:, -1] == 0.0) and np.all(V[-1, :] == 0.0)
    # the sign of the residual does not matter
    phi2 = -phi
    U2, _ = oracle.weights(phi2, dx, dy, None, p, tau)
    assert U2[0, 0] == U[0, 0]


def test_weights_p2_constant_and_large_residual_limit():
    rng = np.random.default_rng(0)
    phi = rng.normal(size=(5, 6)) * 3
    dx = rng.normal(size=(5, 6))
    dy = rng.normal(size=(5, 6))
    U, V = oracle.weights(phi, dx, dy, None, 2.0, 0.01)
    assert np.all(U[:, :-1] == 0.01 / 1.01) and np.all(V[:-1, :] == 0.01 / 1.01)
    # p = 1: U |e| -> tau as |e| >> tau (IRLS weight |e|^(p-2) times tau)
    phi = np.zeros((2, 2))
    phi[0, 1] = 1e6
    U, _ = oracle.weights(phi, np.zeros((2, 2)), np.zeros((2, 2)), None, 1.0, 0.01)
    assert U[0, 0] * 1e6 == pytest.approx(0.01, rel=1e-7)


def test_weights_mask_zeroes_touching_edges():
    H, W = 4, 5
    mask = np.zeros((H, W), np.uint8)
    mask[1, 2] = 1
    U, V = oracle.weights(np.zeros((H, W)), np.zeros((H, W)), np.zeros((H, W)), mask, 1.0, 0.01)
    assert U[1, 1] == 0 and U[1, 2] == 0 and V[0, 2] == 0 and V[1, 2] == 0
    assert U[1, 0] == 1 and U[1, 3] == 1 and V[0, 1] == 1 and V[2, 2] == 1


# ---------------------------------------------------------------- Eq. (Axb)
def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_nnz.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                s, c, r, v, d = line.split()
                rows.append((int(c), int(r), int(v), float(d)))
    return rows


def test_table1_nnz_matches_paper():
    for cols, rows, variables, density in _table1():
        z = np.zeros((rows, cols))
        A = oracle.assemble(z, z, z, z)
        assert A.nnz == variables
        n = rows * cols
        assert 100.0 * A.nnz / n ** 2 == pytest.approx(density, abs=1e-3)


def _random_problem(H, W, seed, p=1.0, mask_frac=0.0):
    rng = np.random.default_rng(seed)
    psi = rng.uniform(-PI, PI, size=(H, W))
    mask = None
    if mask_frac:
        mask = (rng.uniform(size=(H, W)) < mask_frac).astype(np.uint8)
    dx, dy = oracle.wrapped_diffs(psi)
    phi = rng.normal(size=(H, W)) * 2
    U, V = oracle.weights(phi, dx, dy, mask, p, 0.01)
    return psi, mask, dx, dy, U, V


@pytest.mark.parametrize("H,W,mf", [(2, 2, 0), (5, 7, 0), (9, 4, 0.2), (16, 16, 0.05)])
def test_operator_invariants(H, W, mf):
    psi, mask, dx, dy, U, V = _random_problem(H, W, 11 + H, mask_frac=mf)
    A = oracle.assemble(U, V, dx, dy)
    Ad = A.dense()
    np.testing.assert_allclose(Ad, Ad.T, atol=0)                     # symmetric
    np.testing.assert_allclose(Ad @ np.ones(H * W), 0, atol=1e-13)     # A 1 = 0 (Neumann)
    assert abs(A.b.sum()) < 1e-12                                      # sum b = 0
    rng = np.random.default_rng(5)
    x = rng.normal(size=(H, W))
    # quadratic form as a sum over edges: x^T A x = sum U (dx x)^2 + sum V (dy x)^2
    ex = np.sum(U[:, :-1] * np.diff(x, axis=1) ** 2) + np.sum(V[:-1, :] * np.diff(x, axis=0) ** 2)
    assert x.reshape(-1) @ Ad @ x.reshape(-1) == pytest.approx(ex, rel=1e-12)
    # b^T x = sum U Dx (dx x) + sum V Dy (dy x)
    eb = (np.sum(U[:, :-1] * dx[:, :-1] * np.diff(x, axis=1))
          + np.sum(V[:-1, :] * dy[:-1, :] * np.diff(x, axis=0)))
    assert A.b.reshape(-1) @ x.reshape(-1) == pytest.approx(eb, rel=1e-11, abs=1e-12)
    # A x - b is the gradient of F(x) = 1/2 sum U (dx x - Dx)^2 + 1/2 sum V (dy x - Dy)^2
    def F(y):
        return 0.5 * (np.sum(U[:, :-1] * (np.diff(y, axis=1) - dx[:, :-1]) ** 2)
                      + np.sum(V[:-1, :] * (np.diff(y, axis=0) - dy[:-1, :]) ** 2))
    g = (Ad @ x.reshape(-1) - A.b.reshape(-1)).reshape(H, W)
    h = 1e-6
    for (i, j) in [(0, 0), (H - 1, W - 1), (H // 2, W // 2), (0, W - 1)]:
        e = np.zeros((H, W))
        e[i, j] = h
        fd = (F(x + e) - F(x - e)) / (2 * h)
        assert fd == pytest.approx(g[i, j], rel=1e-6, abs=1e-8)


def test_assemble_hand_worked_2x2():
    # U = [[u0, 0], [u1, 0]], V = [[v0, v1], [0, 0]]; unknowns k = 0:(0,0) 1:(0,1) 2:(1,0) 3:(1,1)
    u0, u1, v0, v1 = 0.3, 0.7, 0.2, 0.9
    U = np.array([[u0, 0.0], [u1, 0.0]])
    V = np.array([[v0, v1], [0.0, 0.0]])
    dx = np.array([[0.5, 0.0], [-1.0, 0.0]])
    dy = np.array([[2.0, -0.25], [0.0, 0.0]])
    A = oracle.assemble(U, V, dx, dy)
    expect = np.array([[u0 + v0, -u0, -v0, 0.0],
                       [-u0, u0 + v1, 0.0, -v1],
                       [-v0, 0.0, u1 + v0, -u1],
                       [0.0, -v1, -u1, u1 + v1]])
    np.testing.assert_allclose(A.dense(), expect, atol=1e-16)
    # b_k = Dx_{i,j-1}U_{i,j-1} - Dx_{ij}U_{ij} + Dy_{i-1,j}V_{i-1,j} - Dy_{ij}V_{ij}
    b = np.array([-0.5 * u0 - 2.0 * v0, 0.5 * u0 + 0.25 * v1,
                  1.0 * u1 + 2.0 * v0, -1.0 * u1 - 0.25 * v1])
    np.testing.assert_allclose(A.b.reshape(-1), b, atol=1e-16)


# ---------------------------------------------------------------- preconditioners
def _dense_M_from_apply(kind, A, omega=1.0, mask=None):
    n = A.H * A.W
    cols = []
    for t in range(n):
        e = np.zeros(n)
        e[t] = 1.0
        cols.append(oracle.precond_apply(kind, A, e.reshape(A.H, A.W), omega, mask).reshape(-1))
    return np.array(cols).T              # M^{-1}


def test_jacobi_closed_form():
    psi, mask, dx, dy, U, V = _random_problem(6, 5, 2, mask_frac=0.2)
    A = oracle.assemble(U, V, dx, dy)
    d = np.diag(A.dense())
    r = np.random.default_rng(1).normal(size=(6, 5))
    s = oracle.precond_apply(oracle.M_JACOBI, A, r)
    expect = np.where(d > 0, r.reshape(-1) / np.where(d > 0, d, 1), 0.0)
    np.testing.assert_allclose(s.reshape(-1), expect, rtol=1e-15)


@pytest.mark.parametrize("H,W", [(4, 5), (7, 3), (6, 6)])
def test_ilu0_ic0_reproduce_A_on_its_pattern(H, W):
    # defining property of a no-fill factorisation: (LU)_ij = a_ij on the pattern of A
    psi, mask, dx, dy, U, V = _random_problem(H, W, 3 + H)
    A = oracle.assemble(U, V, dx, dy)
    Ad = A.dense()
    pattern = Ad != 0
    np.fill_diagonal(pattern, True)
    for kind in (oracle.M_ILU0, oracle.M_IC0):
        M = np.linalg.inv(_dense_M_from_apply(kind, A))
        # the last pivot of a singular (Neumann) block is guarded; skip that row/col
        keep = pattern.copy()
        keep[-1, :] = False
        keep[:, -1] = False
        np.testing.assert_allclose(M[keep], Ad[keep], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(M, M.T, atol=1e-10)


@pytest.mark.parametrize("mf", [0.0, 0.15])
def test_ilu0_equals_ic0(mf):
    psi, mask, dx, dy, U, V = _random_problem(12, 9, 21, mask_frac=mf)
    A = oracle.assemble(U, V, dx, dy)
    r = np.random.default_rng(2).normal(size=(12, 9))
    s1 = oracle.precond_apply(oracle.M_ILU0, A, r)
    s2 = oracle.precond_apply(oracle.M_IC0, A, r)
    np.testing.assert_allclose(s1, s2, rtol=1e-13, atol=1e-13 * np.abs(s1).max())


@pytest.mark.parametrize("omega", [1.0, 1.4, 0.7])
def test_ssor_equals_symmetric_sor_sweep(omega):
    # one symmetric SOR sweep (forward then backward) from x = 0 on A x = r equals
    # omega * M_SSOR^{-1} r  (textbook relaxation, written here with dense loops)
    psi, mask, dx, dy, U, V = _random_problem(5, 6, 8)
    A = oracle.assemble(U, V, dx, dy)
    Ad = A.dense()
    n = Ad.shape[0]
    r = np.random.default_rng(3).normal(size=n)
    x = np.zeros(n)
    for i in range(n):
        sigma = Ad[i] @ x - Ad[i, i] * x[i]
        x[i] = (1 - omega) * x[i] + omega * (r[i] - sigma) / Ad[i, i]
    for i in reversed(range(n)):
        sigma = Ad[i] @ x - Ad[i, i] * x[i]
        x[i] = (1 - omega) * x[i] + omega * (r[i] - sigma) / Ad[i, i]
    s = oracle.precond_apply(oracle.M_SSOR, A, r.reshape(5, 6), omega).reshape(-1)
    np.testing.assert_allclose(omega * s, x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("H,W", [(8, 8), (6, 11), (13, 5)])
def test_dct_apply_inverts_neumann_laplacian(H, W):
    # L = kron(I_H, T_W) + kron(T_H, I_W), T_n the 1-D Neumann second difference
    def T(n):
        t = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
        t[0, 0] = t[-1, -1] = 1
        return t
    L = np.kron(np.eye(H), T(W)) + np.kron(T(H), np.eye(W))
    z = np.zeros((H, W))
    A = oracle.assemble(z, z, z, z)   # any A: the DCT preconditioner ignores it
    r = np.random.default_rng(4).normal(size=(H, W))
    s = oracle.precond_apply(oracle.M_DCT, A, r)
    np.testing.assert_allclose(L @ s.reshape(-1), (r - r.mean()).reshape(-1), atol=1e-11)
    assert abs(s.mean()) < 1e-13


# ---------------------------------------------------------------- PCG (Algorithm 1)
@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("H,W", [(4, 4), (16, 16), (11, 7)])
def test_pcg_matches_dense_direct_solve(kind, H, W):
    psi, mask, dx, dy, U, V = _random_problem(H, W, 100 + H * W, p=0.5)
    A = oracle.assemble(U, V, dx, dy)
    Ad = A.dense()
    n = H * W
    # (A + 1 1^T / n) x = b has the mean-zero solution of the consistent singular system
    Lc = np.linalg.cholesky(Ad + np.ones((n, n)) / n)
    x = np.linalg.solve(Lc.T, np.linalg.solve(Lc, A.b.reshape(-1)))
    phi, st = oracle.pcg(A, np.zeros((H, W)), kind=kind, tol=1e-14, max_inner=20 * n)
    assert st["status"] == oracle.OK
    got = phi.reshape(-1) - phi.mean()
    np.testing.assert_allclose(got, x - x.mean(), atol=1e-10 * max(1.0, np.abs(x).max()))


def test_cg_finite_termination():
    # exact arithmetic CG ends in at most (number of distinct nonzero eigenvalues) steps
    psi, mask, dx, dy, U, V = _random_problem(2, 2, 9)
    A = oracle.assemble(U, V, dx, dy)
    phi, st = oracle.pcg(A, np.zeros((2, 2)), kind=oracle.M_IDENTITY, tol=1e-13)
    assert st["iters"] <= 3 and st["status"] == oracle.OK


def _neumann_eigs(H, W):
    k = np.arange(H)[:, None]
    l = np.arange(W)[None, :]
    return (2 - 2 * np.cos(PI * k / H)) + (2 - 2 * np.cos(PI * l / W))


@pytest.mark.parametrize("kind", [oracle.M_IDENTITY, oracle.M_JACOBI, oracle.M_ILU0, oracle.M_MG])
def test_p2_pcg_equals_closed_form_dct_solution(kind):
    # p = 2: U = V = tau / (1 + tau) everywhere, A = c L; the least-squares phase is
    # the Fourier/DCT Poisson solution (Ghiglia-Romero), here through scipy's DCT
    m = synth.workload_map("c1_256") if False else synth.phase_map(48, 64, 5, noise=0.3)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros_like(m.psi), dx, dy, None, 2.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    c = 0.01 / 1.01
    bh = scipy.fft.dctn(A.b / c, type=2, norm="ortho")
    lam = _neumann_eigs(48, 64)
    lam[0, 0] = 1.0
    xh = bh / lam
    xh[0, 0] = 0.0
    x = scipy.fft.idctn(xh, type=2, norm="ortho")
    phi, st = oracle.pcg(A, np.zeros_like(m.psi), kind=kind, tol=1e-13, max_inner=20000)
    err = (phi - phi.mean()) - (x - x.mean())
    assert np.sqrt(np.mean(err ** 2)) < 1e-9


def test_p2_dct_preconditioner_converges_in_one_iteration():
    m = synth.phase_map(32, 40, 6, noise=0.4)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros_like(m.psi), dx, dy, None, 2.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    phi, st = oracle.pcg(A, np.zeros_like(m.psi), kind=oracle.M_DCT, tol=1e-10)
    assert st["iters"] == 1 and st["true_relres"] < 1e-12


def test_pcg_refresh_and_paper_stop_mode():
    psi, mask, dx, dy, U, V = _random_problem(20, 24, 77)
    A = oracle.assemble(U, V, dx, dy)
    phi1, s1 = oracle.pcg(A, np.zeros((20, 24)), kind=1, tol=1e-10)
    phi2, s2 = oracle.pcg(A, np.zeros((20, 24)), kind=1, tol=1e-10, refresh=1)
    assert abs(s1["iters"] - s2["iters"]) <= 2
    np.testing.assert_allclose(phi1 - phi1.mean(), phi2 - phi2.mean(), atol=1e-8)
    # paper criterion: delta_new <= eps^2 delta_0 with delta = r^T M^-1 r; for M = I the
    # two criteria differ only by ||r_0|| vs ||b|| which are equal from phi = 0
    _, a = oracle.pcg(A, np.zeros((20, 24)), kind=0, tol=1e-6, stop_mode=oracle.STOP_RELRES)
    _, b = oracle.pcg(A, np.zeros((20, 24)), kind=0, tol=1e-6, stop_mode=oracle.STOP_PAPER)
    assert a["iters"] == b["iters"]
    # l_max stops with the MAXITER status
    _, c = oracle.pcg(A, np.zeros((20, 24)), kind=0, tol=1e-12, max_inner=5)
    assert c["iters"] == 5 and c["status"] == oracle.MAXITER


# ---------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("p", [0.0, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5])
def test_noiseless_phase_recovered_exactly(p, kind):
    m = synth.smooth_map(24, 31, seed=9)
    phi, st = oracle.unwrap(m.psi, None, p=p, tau=0.01, kind=kind, tol=1e-12, max_outer=3,
                            max_inner=10000)
    err = (phi - phi.mean()) - (m.phi_true - m.phi_true.mean())
    assert np.max(np.abs(err)) < 1e-8
    # congruence: the output differs from psi by a constant multiple... modulo 2 pi
    w = oracle.wrap(phi - m.psi)
    assert np.max(np.abs(oracle.wrap(w - w.flat[0]))) < 1e-8


def test_congruence_post_step():
    m = synth.phase_map(40, 40, 12, noise=1.0)
    phi, _ = oracle.unwrap(m.psi, None, p=1.0, kind=1, tol=1e-8, max_outer=2)
    pc = oracle.congruence(phi, m.psi)
    np.testing.assert_allclose(oracle.wrap(pc), m.psi, atol=1e-12)


def test_solution_independent_of_preconditioner():
    # Sec. 4: every M gives the same unwrapped phase (same Q); residue-rich input
    m = synth.phase_map(32, 36, 13, noise=1.2, ramp=0.4)
    ref = None
    for kind in range(6):
        phi, st = oracle.unwrap(m.psi, None, p=1.0, kind=kind, tol=1e-11, max_outer=2,
                                max_inner=100000)
        phi = phi - phi.mean()
        if ref is None:
            ref = phi
        else:
            assert np.sqrt(np.mean((phi - ref) ** 2)) < 1e-6


def test_iteration_ordering_soft():
    # Sec. 4: ILU and IC need the fewest iterations; Jacobi beats plain CG
    m = synth.phase_map(64, 64, 14, noise=0.8, ramp=0.1, n_bumps=8)
    it = {}
    for kind in range(5):
        _, st = oracle.unwrap(m.psi, None, p=1.0, kind=kind, tol=1e-6, max_outer=1)
        it[kind] = st["inner"][0]
    assert it[2] == pytest.approx(it[3], abs=2)
    assert it[2] <= it[4] <= it[1] <= it[0]


def test_quality_q_definition():
    rng = np.random.default_rng(0)
    mu = rng.normal(size=100)
    assert oracle.quality_q(mu, mu) == 0.0
    assert oracle.quality_q(mu, -mu) == pytest.approx(1.0)
    assert oracle.quality_q(mu, np.zeros(100)) == pytest.approx(1.0)
    assert oracle.quality_q(3 * mu, 3 * (mu + 1)) == pytest.approx(oracle.quality_q(mu, mu + 1))


def test_functional_hand_case():
    # phi = 0: J = sum over interior edges of |Delta|^p
    dx = np.array([[0.5, 0.0], [-2.0, 0.0]])
    dy = np.array([[1.0, -0.25], [0.0, 0.0]])
    assert oracle.functional(np.zeros((2, 2)), dx, dy, None, 1.0) == pytest.approx(3.75)
    assert oracle.functional(np.zeros((2, 2)), dx, dy, None, 2.0) == pytest.approx(5.3125)


@pytest.mark.parametrize("p", [0.5, 1.0, 2.0])
def test_functional_invariants(p):
    # Eq. (funcional) depends on phi only through its differences, is homogeneous of
    # degree p in (phi, Delta), treats rows and columns alike, and vanishes where the
    # differences of phi equal Delta (a noiseless phase whose true gradients stay below pi)
    rng = np.random.default_rng(21)
    H, W = 7, 9
    phi = rng.normal(size=(H, W))
    dx, dy = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    J = oracle.functional(phi, dx, dy, None, p)
    assert J > 0.0
    assert oracle.functional(phi + 5.0, dx, dy, None, p) == pytest.approx(J, rel=1e-12)
    assert oracle.functional(2.0 * phi, 2.0 * dx, 2.0 * dy, None, p) == pytest.approx(2.0 ** p * J, rel=1e-14)
    assert oracle.functional(phi.T.copy(), dy.T.copy(), dx.T.copy(), None, p) == pytest.approx(J, rel=1e-14)
    m = synth.smooth_map(24, 30, seed=4)
    ex, ey = oracle.wrapped_diffs(m.psi)
    # each edge's residual is rounding (|e| < 1e-12, the wrapped differences' own pin), so J is
    # below edges x (1e-12)^p, while any misplaced term would contribute O(1) per edge
    edges = 2 * m.psi.size
    assert oracle.functional(m.phi_true, ex, ey, None, p) < edges * 1e-12 ** p
    assert oracle.functional(m.phi_true, ey, ex, None, p) > 1.0


def test_functional_ignores_masked_edges():
    # an edge with a masked end point carries no term: the value at a masked pixel is free
    rng = np.random.default_rng(22)
    phi = rng.normal(size=(6, 8))
    dx, dy = rng.normal(size=(6, 8)), rng.normal(size=(6, 8))
    mask = np.zeros((6, 8), dtype=np.uint8)
    mask[2, 3] = 1
    J = oracle.functional(phi, dx, dy, mask, 1.0)
    phi2 = phi.copy()
    phi2[2, 3] = 1e6
    assert oracle.functional(phi2, dx, dy, mask, 1.0) == J
    assert oracle.functional(phi2, dx, dy, None, 1.0) > 1e6


def test_functional_gradient_is_the_system_at_p2():
    # at p = 2 the weights are the constant c = tau / (1 + tau) (Eq. UV), so Eq. (Axb) is c times
    # the normal equations of Eq. (funcional): grad J = (2 / c) (A phi - b).  The functional and
    # the CSR assembly are separate code; a quadratic's central difference is exact up to rounding.
    rng = np.random.default_rng(23)
    H, W, tau = 5, 6, 0.01
    phi = rng.normal(size=(H, W))
    dx, dy = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    U, V = oracle.weights(phi, dx, dy, None, 2.0, tau)
    A = oracle.assemble(U, V, dx, dy)
    c = tau / (1.0 + tau)
    want = (2.0 / c) * (A.matvec(phi) - A.b)
    h = 1e-3
    got = np.empty((H, W))
    for i in range(H):
        for j in range(W):
            e = np.zeros((H, W))
            e[i, j] = h
            got[i, j] = (oracle.functional(phi + e, dx, dy, None, 2.0) -
                         oracle.functional(phi - e, dx, dy, None, 2.0)) / (2 * h)
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-7)


def test_unwrap_rejects_invalid():
    with pytest.raises(ValueError):
        oracle.unwrap(np.zeros((1, 5)))
    with pytest.raises(ValueError):
        oracle.unwrap(np.zeros((4, 5)), p=3.0)
    bad = np.zeros((4, 5))
    bad[1, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.unwrap(bad)
