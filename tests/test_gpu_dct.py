"""DCT Poisson preconditioner (tcgen05 GEMMs on split-BF16 operands, FP32 accumulation)
against the oracle's FP64 explicit-cosine apply.

Each operand is the sum of two BF16 planes (16 significant bits) and each product
keeps three of the four cross terms, so one application is within about 4e-5 of
the exact pseudo-inverse in the 2-norm (3.9e-5 in a CPU emulation of the same
rounding on the 200 x 129 case; plain BF16 operands gave 1.2e-2); the bar is
1e-4.  The solver uses it inside flexible CG, whose iteration counts then follow
the oracle's exact-M PCG within 2 (the emulation: 97 and 148 against 96 and 147).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("H,W,mask_frac", [(128, 128, 0.0), (200, 129, 0.05), (256, 384, 0.05), (64, 300, 0.0)])
def test_dct_apply_vs_oracle(H, W, mask_frac):
    m = synth.phase_map(H, W, 4, noise=0.6, mask_frac=mask_frac)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    r = A.b
    ref = oracle.precond_apply(oracle.M_DCT, A, r, mask=m.mask)
    mk = _cuda(m.mask, torch.uint8) if m.mask is not None else None
    got = native.ulp_precond_apply("dct", _cuda(U), _cuda(V), _cuda(r), mask=mk).cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err
    if m.mask is not None:
        assert np.all(got[m.mask == 1] == 0.0)


def test_dct_apply_inverts_the_laplacian_on_smooth_input():
    # a single low-frequency cosine mode is an eigenvector: s = r / lambda (to the split's rounding)
    H, W = 128, 256
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    r = np.cos(np.pi * 3 * (i + 0.5) / H) * np.cos(np.pi * 5 * (j + 0.5) / W)
    lam = (2 - 2 * np.cos(np.pi * 3 / H)) + (2 - 2 * np.cos(np.pi * 5 / W))
    z = np.zeros((H, W))
    got = native.ulp_precond_apply("dct", _cuda(z), _cuda(z), _cuda(r)).cpu().numpy()
    err = np.linalg.norm(got - r / lam) / np.linalg.norm(r / lam)
    assert err < 1e-4, err


def _rms(a, b, keep=None):
    e = a - b
    if keep is not None:
        e = e[keep]
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("H,W,p,mask_frac", [(128, 128, 1.0, 0.05), (200, 129, 0.0, 0.05), (96, 256, 2.0, 0.0)])
def test_dct_fcg_unwrap_vs_oracle(H, W, p, mask_frac):
    # the GPU runs flexible CG with the split-BF16 tensor-core M; the oracle standard PCG with the
    # exact FP64 M: same solution (1e-4 rad RMS), iteration counts within 2
    m = synth.phase_map(H, W, 21, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=mask_frac,
                        sigma_range=(5.0, 20.0))
    plan = native.Plan(H, W, outer_tol=0.0)
    mk = _cuda(m.mask, torch.uint8) if m.mask is not None else None
    phi, st = plan.unwrap(_cuda(m.psi), mk, p=p, precond="dct", tol=1e-6, max_outer=3, max_inner=2000)
    ref, rst = oracle.unwrap(m.psi, m.mask, p=p, kind=oracle.M_DCT, tol=1e-6, max_outer=3)
    keep = None if m.mask is None else (m.mask == 0)
    assert st["status"] == 0, st
    assert _rms(phi.cpu().numpy(), ref, keep) < 1e-4
    for a, b in zip(st["inner"], rst["inner"]):
        assert abs(a - b) <= 2, (st["inner"], rst["inner"])


def test_dct_fcg_p2_unmasked_few_iterations():
    # p = 2 without a mask: A = c L and M^-1 A is a projector; the exact M converges in one
    # iteration, the split-BF16 one (4e-5 off) in at most three
    m = synth.phase_map(128, 192, 8, noise=0.4)
    plan = native.Plan(128, 192, outer_tol=0.0)
    phi, st = plan.unwrap(_cuda(m.psi), None, p=2.0, precond="dct", tol=1e-6, max_outer=1, max_inner=200)
    assert st["status"] == 0 and st["inner"][0] <= 3, st


@pytest.mark.slow
def test_dct_fcg_full_size_true_residual():
    # C2 2048^2, p = 1: FP64 true residual of the first pass computed by the oracle
    m = synth.workload_map("c2_2048")
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0)
    phi, st = plan.unwrap(_cuda(m.psi), _cuda(m.mask, torch.uint8), p=1.0, precond="dct", tol=1e-6,
                          max_outer=1, max_inner=5000)
    assert st["status"] == 0, st
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    g = phi.cpu().numpy()
    res = np.linalg.norm(A.b - A.matvec(g)) / np.linalg.norm(A.b)
    assert res <= 1.1e-6, res
