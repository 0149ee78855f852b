"""Pins of the oracle's red-black (multicolour) SSOR and ILU(0): each must equal
the natural-order routine -- itself pinned in test_oracle_pins.py -- applied to
the matrix with its unknowns permuted into red-black order (red: i + j even,
first; natural order within a colour), and map back."""
import numpy as np
import pytest

import oracle
from paper_2203_13675_gb300 import synth


def _problem(H, W, seed, mask_frac=0.0):
    m = synth.phase_map(H, W, seed, noise=0.5, mask_frac=mask_frac)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, 1.0, 0.01)
    return oracle.assemble(U, V, dx, dy), m.mask


def _permuted(A):
    H, W = A.H, A.W
    n = H * W
    red = [k for k in range(n) if ((k // W) + (k % W)) % 2 == 0]
    black = [k for k in range(n) if ((k // W) + (k % W)) % 2 == 1]
    perm = np.array(red + black)          # position -> node
    pos = np.empty(n, dtype=np.int64)
    pos[perm] = np.arange(n)
    D = A.dense()[np.ix_(perm, perm)]
    indptr = np.zeros(n + 1, dtype=np.int64)
    idx, val = [], []
    for p in range(n):
        cols = np.nonzero(D[p])[0]
        if not np.any(cols == p):          # keep the diagonal in the pattern, as assemble() does
            cols = np.sort(np.append(cols, p))
        idx += list(cols)
        val += list(D[p, cols])
        indptr[p + 1] = len(idx)
    Ap = oracle.Csr(H, W, indptr, np.array(idx, dtype=np.int32), np.array(val), A.b.ravel()[perm].reshape(H, W))
    return Ap, perm, pos


@pytest.mark.parametrize("H,W,mask_frac", [(6, 7, 0.0), (9, 8, 0.1), (1, 12, 0.0), (11, 5, 0.0)])
@pytest.mark.parametrize("kinds", [(oracle.M_RBSSOR, oracle.M_SSOR), (oracle.M_RBILU, oracle.M_ILU0),
                                   (oracle.M_RBILU, oracle.M_IC0)])
def test_red_black_equals_natural_on_the_permuted_matrix(H, W, mask_frac, kinds):
    rb, nat = kinds
    A, mask = _problem(H, W, 3 + H + W, mask_frac)
    Ap, perm, pos = _permuted(A)
    r = np.random.default_rng(H * W).standard_normal((H, W))
    got = oracle.precond_apply(rb, A, r, omega=1.3 if rb == oracle.M_RBSSOR else 1.0)
    ref_p = oracle.precond_apply(nat, Ap, r.ravel()[perm].reshape(H, W),
                                 omega=1.3 if rb == oracle.M_RBSSOR else 1.0)
    ref = ref_p.ravel()[pos].reshape(H, W)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_red_black_preconditioners_are_symmetric_and_converge():
    A, mask = _problem(40, 36, 9, 0.05)
    rng = np.random.default_rng(1)
    for kind in (oracle.M_RBSSOR, oracle.M_RBILU):
        x, y = rng.standard_normal((40, 36)), rng.standard_normal((40, 36))
        a = np.sum(y * oracle.precond_apply(kind, A, x))
        b = np.sum(x * oracle.precond_apply(kind, A, y))
        assert abs(a - b) <= 1e-11 * abs(a)
    _, sj = oracle.pcg(A, np.zeros((40, 36)), kind=oracle.M_JACOBI, tol=1e-8, mask=mask)
    for kind in (oracle.M_RBSSOR, oracle.M_RBILU):
        _, st = oracle.pcg(A, np.zeros((40, 36)), kind=kind, tol=1e-8, mask=mask)
        assert st["status"] == oracle.OK and st["true_relres"] < 2e-8
        assert st["iters"] < sj["iters"], (kind, st["iters"], sj["iters"])
