"""Red-black (two-colour) SSOR and ILU(0) preconditioners on the GPU against
the oracle's red-black versions, and their flexible-CG solves against the
oracle's PCG with the same M.

One application is two passes of FP64 stencil arithmetic per pixel, a few
roundings from the oracle's CSR loops: 1e-12 relative in the 2-norm.  Flexible
CG (Polak-Ribiere beta) and PCG (Fletcher-Reeves beta) with a fixed SPD M are
the same iteration in exact arithmetic, so counts agree within 2 and the
solutions within the 1e-4 rad RMS bar.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu

KINDS = {"rbssor": oracle.M_RBSSOR, "rbilu": oracle.M_RBILU}


def _cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rms(a, b, keep=None):
    e = a - b
    if keep is not None:
        e = e[keep]
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("name,omega", [("rbssor", 1.0), ("rbssor", 1.6), ("rbilu", 1.0)])
@pytest.mark.parametrize("H,W,mask_frac", [(128, 128, 0.0), (200, 129, 0.05), (7, 300, 0.0), (257, 63, 0.05),
                                           (3, 3, 0.0), (2, 50, 0.0)])
def test_rb_apply_vs_oracle(name, omega, H, W, mask_frac):
    m = synth.phase_map(H, W, 4, noise=0.6, mask_frac=mask_frac)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    keep = 1.0 if m.mask is None else (m.mask == 0)
    r = (A.b + 0.1 * np.random.default_rng(1).standard_normal((H, W))) * keep
    ref = oracle.precond_apply(KINDS[name], A, r, omega=omega, mask=m.mask)
    got = native.ulp_precond_apply(name, _cuda(U), _cuda(V), _cuda(r), omega=omega).cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


@pytest.mark.parametrize("name,omega", [("rbssor", 1.0), ("rbssor", 1.5), ("rbilu", 1.0)])
@pytest.mark.parametrize("H,W,p,mask_frac", [(128, 128, 1.0, 0.05), (200, 129, 0.0, 0.0), (96, 257, 2.0, 0.05)])
def test_rb_fcg_unwrap_vs_oracle(name, omega, H, W, p, mask_frac):
    m = synth.phase_map(H, W, 21, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=mask_frac,
                        sigma_range=(5.0, 20.0))
    plan = native.Plan(H, W, outer_tol=0.0, omega=omega)
    mk = _cuda(m.mask, torch.uint8) if m.mask is not None else None
    phi, st = plan.unwrap(_cuda(m.psi), mk, p=p, precond=name, tol=1e-6, max_outer=3, max_inner=4000)
    ref, rst = oracle.unwrap(m.psi, m.mask, p=p, kind=KINDS[name], tol=1e-6, max_outer=3, omega=omega)
    keep = None if m.mask is None else (m.mask == 0)
    assert st["status"] == 0, st
    assert _rms(phi.cpu().numpy(), ref, keep) < 1e-4
    for a, b in zip(st["inner"], rst["inner"]):
        assert abs(a - b) <= 2, (st["inner"], rst["inner"])


@pytest.mark.parametrize("name", ["rbssor", "rbilu"])
def test_rb_pcg_entry_point(name):
    H, W = 160, 97
    m = synth.phase_map(H, W, 9, noise=0.5)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, None, 1.0, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    phi = torch.zeros((H, W), dtype=torch.float64, device="cuda")
    _, st = native.ulp_pcg(_cuda(U), _cuda(V), _cuda(A.b), phi, precond=name, tol=1e-8)
    ref, rst = oracle.pcg(A, np.zeros((H, W)), kind=KINDS[name], tol=1e-8)
    assert abs(st["inner"][0] - rst["iters"]) <= 2, (st, rst)
    assert _rms(phi.cpu().numpy(), ref) < 1e-6


def test_rb_rejects_batched_plans():
    plan = native.Plan(None, sizes=[(64, 64), (32, 48)])
    maps = [{"psi": torch.zeros(h, w, dtype=torch.float64, device="cuda"),
             "phi": torch.zeros(h, w, dtype=torch.float64, device="cuda"), "p": 1.0} for h, w in plan.sizes]
    with pytest.raises(native.UlpError) as e:
        plan.unwrap_batched(maps, precond="rbilu")
    assert e.value.status == native.ULP_ERR_UNSUPPORTED
