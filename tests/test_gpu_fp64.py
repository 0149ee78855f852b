"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Bars: bit-exact for the wrapped differences (the wrap's integer decision is
taken in FP64 by both sides from the same inputs); weights/b within a few ulp
(pow may differ by an ulp); the stencil within 1e-14 relative; whole solves
within 1e-4 rad RMS after removing the mean (the constant is free) and PCG
iteration counts within +-2 at the same relative-residual tolerance.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-4        # rad, after mean removal
ITER_TOL = 2


def iter_tol(kind, iters):
    """+-2 iterations, except plain CG (M = I): there the count is not fixed by FP64
    arithmetic to +-2 -- the oracle itself, re-run with other blockings of its own dot
    products, moves by up to 3 at 1e3-3e3 iterations on these systems -- so M = I is
    held to 1 % of the count (at least 2)."""
    if kind == "identity":
        return max(ITER_TOL, int(np.ceil(0.01 * iters)))
    return ITER_TOL


def _cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rms_mean_removed(a, b, keep=None):
    e = (a - b)
    if keep is not None:
        e = e[keep]
    e = e - e.mean()
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()


# ------------------------------------------------------------------ steps
@pytest.mark.parametrize("H,W", [(2, 2), (37, 53), (64, 64), (130, 67)])
def test_wrapped_diffs_bit_exact(H, W):
    m = synth.phase_map(H, W, 3 + H, noise=1.0)
    psi = m.psi.copy()
    psi.flat[::7] = math.pi            # ties at +-pi
    psi.flat[3::11] = -math.pi + 1e-16
    dx, dy = native.ulp_wrapped_diffs(_cuda(psi))
    ox, oy = oracle.wrapped_diffs(psi)
    assert np.array_equal(dx.cpu().numpy(), ox)
    assert np.array_equal(dy.cpu().numpy(), oy)


def test_wrapped_diffs_bit_exact_at_the_branch_cuts():
    """Differences at and a few units in the last place around the odd multiples of pi,
    where the wrap's integer decision ceil((x - pi) / (2 pi)) flips, and large ones: the
    decision and the result are the oracle's bit for bit."""
    H, W = 64, 64
    xs = []
    for n in range(-6, 7):
        c = math.pi * (2 * n + 1)
        v = c
        for _ in range(4):
            xs += [v, -v]
            v = np.nextafter(v, np.inf)
        v = c
        for _ in range(4):
            v = np.nextafter(v, -np.inf)
            xs += [v, -v]
    rng = np.random.default_rng(11)
    xs += list(rng.uniform(-1e4, 1e4, 200)) + list(rng.normal(0, 4, 200))
    x = np.resize(np.asarray(xs), (H, W // 2))
    psi = np.zeros((H, W))
    psi[:, 1::2] = x          # differences x and -x along rows, exact in FP64
    psi[1::2, :] += 0.25      # and 0.25 +- x between rows
    dx, dy = native.ulp_wrapped_diffs(_cuda(psi))
    ox, oy = oracle.wrapped_diffs(psi)
    assert np.array_equal(dx.cpu().numpy(), ox)
    assert np.array_equal(dy.cpu().numpy(), oy)


@pytest.mark.parametrize("p", [0.0, 0.5, 1.0, 2.0, 1.3])
def test_weights_and_rhs(p):
    H, W = 45, 70
    m = synth.phase_map(H, W, 5, noise=0.8, mask_frac=0.08)
    dx, dy = oracle.wrapped_diffs(m.psi)
    phi = np.random.default_rng(1).normal(size=(H, W)) * 3
    U, V, b = native.ulp_weights(_cuda(phi), _cuda(dx), _cuda(dy), _cuda(m.mask, torch.uint8), p, 0.01)
    oU, oV = oracle.weights(phi, dx, dy, m.mask, p, 0.01)
    A = oracle.assemble(oU, oV, dx, dy)
    if p in (1.0, 2.0):
        # no libm power involved: every operation is a correctly rounded +, -, *, /
        assert np.array_equal(U.cpu().numpy(), oU) and np.array_equal(V.cpu().numpy(), oV)
        assert np.array_equal(b.cpu().numpy(), A.b)
    else:
        # |e|^(2-p): the oracle calls the host libm pow (not always correctly rounded,
        # e.g. pow(x, 2) != x*x for ~0.1 % of x on glibc); within 2 ulp
        np.testing.assert_allclose(U.cpu().numpy(), oU, rtol=5e-16, atol=0)
        np.testing.assert_allclose(V.cpu().numpy(), oV, rtol=5e-16, atol=0)
        np.testing.assert_allclose(b.cpu().numpy(), A.b, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("H,W", [(2, 3), (33, 65), (100, 128), (257, 190)])
def test_matvec(H, W):
    rng = np.random.default_rng(H * W)
    U = rng.uniform(0, 1, (H, W))
    V = rng.uniform(0, 1, (H, W))
    U[:, -1] = 0
    V[-1, :] = 0
    x = rng.normal(size=(H, W))
    y = native.ulp_matvec(_cuda(U), _cuda(V), _cuda(x)).cpu().numpy()
    z = np.zeros((H, W))
    A = oracle.assemble(U, V, z, z)
    ref = A.matvec(x)
    scale = np.abs(U).max() * np.abs(x).max()
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14 * scale)


@pytest.mark.parametrize("kind", ["identity", "jacobi"])
def test_precond_apply(kind):
    H, W = 40, 77
    rng = np.random.default_rng(2)
    U = rng.uniform(0, 1, (H, W))
    V = rng.uniform(0, 1, (H, W))
    U[:, -1] = 0
    V[-1, :] = 0
    U[5, :] = 0
    V[4:6, :] = 0                      # row 5 is isolated: zero diagonal there
    r = rng.normal(size=(H, W))
    s = native.ulp_precond_apply(kind, _cuda(U), _cuda(V), _cuda(r)).cpu().numpy()
    z = np.zeros((H, W))
    A = oracle.assemble(U, V, z, z)
    ref = oracle.precond_apply(oracle.M_IDENTITY if kind == "identity" else oracle.M_JACOBI, A, r)
    np.testing.assert_allclose(s, ref, rtol=3e-16, atol=0)


# ------------------------------------------------------------------ inner PCG
@pytest.mark.parametrize("kind", ["identity", "jacobi"])
@pytest.mark.parametrize("H,W,p", [(64, 64, 1.0), (37, 53, 0.0), (200, 129, 0.5), (256, 256, 1.0)])
def test_pcg_parity(kind, H, W, p):
    m = synth.phase_map(H, W, 11 + H, noise=0.7, mask_frac=0.05, ramp=0.1)
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, p, 0.01)
    A = oracle.assemble(U, V, dx, dy)
    ok = oracle.M_IDENTITY if kind == "identity" else oracle.M_JACOBI
    ref, rs = oracle.pcg(A, np.zeros((H, W)), kind=ok, tol=1e-6)
    phi, st = native.ulp_pcg(_cuda(U), _cuda(V), _cuda(A.b), torch.zeros(H, W, dtype=torch.float64,
                                                                         device="cuda"), kind, 1e-6)
    assert st["status"] == 0
    assert abs(st["inner"][0] - rs["iters"]) <= iter_tol(kind, rs["iters"]), (st["inner"][0], rs["iters"])
    # both stop at relative residual 1e-6; a stop a few iterations apart moves phi by ~tol
    assert _rms_mean_removed(phi.cpu().numpy(), ref) < (1e-8 if kind == "jacobi" else 1e-5)


# ------------------------------------------------------------------ whole method
def _unwrap_both(m, p, kind, tol=1e-6, max_outer=5, tau=1e-2):
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0)
    mask = _cuda(m.mask, torch.uint8) if m.mask is not None else None
    phi, st = plan.unwrap(_cuda(m.psi), mask, p=p, eps=tau, precond=kind, tol=tol, max_outer=max_outer)
    ok = oracle.M_IDENTITY if kind == "identity" else oracle.M_JACOBI
    ref, rst = oracle.unwrap(m.psi, m.mask, p=p, tau=tau, kind=ok, tol=tol, max_outer=max_outer)
    return phi.cpu().numpy(), st, ref, rst


def test_config_c1_256_p1_jacobi():
    w = synth.WORKLOADS["c1_256"]
    m = synth.workload_map("c1_256")
    got, st, ref, rst = _unwrap_both(m, w["p"], "jacobi", tol=w["tol"], max_outer=w["max_outer"])
    assert st["status"] == 0 and st["outer"] == rst["outer"]
    for a, b in zip(st["inner"], rst["inner"]):
        assert abs(a - b) <= ITER_TOL, (st["inner"], rst["inner"])
    assert _rms_mean_removed(got, ref) < RMS_TOL


@pytest.mark.parametrize("p", [0.0, 1.0, 2.0])
@pytest.mark.parametrize("kind", ["identity", "jacobi"])
def test_masked_c2_style_small(p, kind):
    m = synth.phase_map(128, 96, 2, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=0.05,
                        sigma_range=(5.0, 20.0))
    got, st, ref, rst = _unwrap_both(m, p, kind, max_outer=3)
    keep = m.mask == 0
    assert st["status"] == 0
    for a, b in zip(st["inner"], rst["inner"]):
        assert abs(a - b) <= iter_tol(kind, b), (st["inner"], rst["inner"])
    assert _rms_mean_removed(got, ref, keep) < RMS_TOL
    # masked pixels keep phi^0 = 0
    assert np.all(got[~keep] == 0.0)


def test_noiseless_exact_recovery():
    m = synth.smooth_map(90, 70, seed=4)
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0)
    phi, st = plan.unwrap(_cuda(m.psi), None, p=0.5, precond="jacobi", tol=1e-12, max_outer=2)
    assert _rms_mean_removed(phi.cpu().numpy(), m.phi_true) < 1e-8


def test_degenerate_cases():
    # constant psi: b = 0, nothing to solve, phi stays 0
    plan = native.Plan(16, 16, outer_tol=0.0)
    phi, st = plan.unwrap(torch.full((16, 16), 0.3, dtype=torch.float64, device="cuda"), None, max_outer=2)
    assert st["status"] == 0 and st["inner"][0] == 0 and float(phi.abs().max()) == 0.0
    # smallest grid
    m = synth.phase_map(2, 2, 1, noise=1.0)
    got, st, ref, rst = _unwrap_both(m, 1.0, "jacobi", tol=1e-10, max_outer=2)
    assert _rms_mean_removed(got, ref) < 1e-8
    # l_max reached -> warning status, phi written
    m = synth.phase_map(64, 64, 9, noise=0.5)
    plan = native.Plan(64, 64, outer_tol=0.0)
    phi, st = plan.unwrap(_cuda(m.psi), None, precond="identity", tol=1e-12, max_outer=1, max_inner=7)
    assert st["status"] == native.ULP_WARN_MAXITER and st["inner"][0] == 7
    ref, rst = oracle.unwrap(m.psi, None, p=1.0, kind=oracle.M_IDENTITY, tol=1e-12, max_outer=1, max_inner=7)
    assert _rms_mean_removed(phi.cpu().numpy(), ref) < 1e-10


def test_non_finite_input_is_rejected():
    psi = torch.zeros(8, 8, dtype=torch.float64, device="cuda")
    psi[3, 3] = float("nan")
    plan = native.Plan(8, 8)
    with pytest.raises(native.UlpError) as e:
        plan.unwrap(psi, None)
    assert e.value.status == native.ULP_ERR_INVALID


def test_unwrap_lp_host_and_device_buffers():
    m = synth.phase_map(48, 40, 21, noise=0.5)
    host = torch.from_numpy(m.psi.copy())
    ph_h, rc = native.unwrap_lp(host, p=1.0, eps=1e-2, precond="jacobi", tol=1e-8, max_outer=2)
    ph_d, rc2 = native.unwrap_lp(host.cuda(), p=1.0, eps=1e-2, precond="jacobi", tol=1e-8, max_outer=2)
    assert rc == 0 and rc2 == 0 and not ph_h.is_cuda
    assert torch.equal(ph_h, ph_d.cpu())
    ref, _ = oracle.unwrap(m.psi, None, p=1.0, tau=1e-2, kind=oracle.M_JACOBI, tol=1e-8, max_outer=2)
    assert _rms_mean_removed(ph_h.numpy(), ref) < 1e-6


def test_plan_reuse_and_async_status():
    m = synth.phase_map(70, 70, 5, noise=0.6)
    plan = native.Plan(70, 70, outer_tol=0.0)
    psi = _cuda(m.psi)
    a, _ = plan.unwrap(psi, None, stats=False)
    rc, st = plan.last_status()
    b, st2 = plan.unwrap(psi, None)
    assert rc == 0 and torch.equal(a, b) and st["inner"] == st2["inner"]


@pytest.mark.slow
def test_full_size_c2_2048_properties():
    # 2048^2: the oracle cannot iterate at this size in seconds, so check what holds at any
    # size: the weights and the operator at full size element by element, and the true
    # residual of the GPU's first-pass solution with the oracle's own A and b.
    w = synth.WORKLOADS["c2_2048"]
    m = synth.workload_map("c2_2048")
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0)
    psi = _cuda(m.psi)
    mask = _cuda(m.mask, torch.uint8)
    phi, st = plan.unwrap(psi, mask, p=w["p"], eps=w["tau"], precond="jacobi", tol=w["tol"], max_outer=1)
    assert st["status"] == 0
    dx, dy = oracle.wrapped_diffs(m.psi)
    U, V = oracle.weights(np.zeros((H, W)), dx, dy, m.mask, w["p"], w["tau"])
    A = oracle.assemble(U, V, dx, dy)
    g = phi.cpu().numpy()
    res = np.linalg.norm(A.b - A.matvec(g)) / np.linalg.norm(A.b)
    assert res <= 1.05 * w["tol"], res
    gU, gV, gb = native.ulp_weights(torch.zeros_like(psi), _cuda(dx), _cuda(dy), mask, w["p"], w["tau"])
    assert np.array_equal(gU.cpu().numpy(), U) and np.array_equal(gb.cpu().numpy(), A.b)
    y = native.ulp_matvec(gU, gV, phi).cpu().numpy()
    np.testing.assert_allclose(y, A.matvec(g), rtol=0, atol=1e-13 * np.abs(g).max())


@pytest.mark.slow
def test_full_size_c2_2048_matches_oracle_run():
    # the oracle's own full run of this workload (tests/golden/oracle_runs.json, written by
    # tests/golden/make_oracle_runs.py): per-pass iteration counts and phase at sampled pixels
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_runs.json")))
    g = gold["c2_2048_p1_jacobi"]
    m = synth.workload_map(g["workload"])
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=g["outer_tol"])
    phi, st = plan.unwrap(_cuda(m.psi), _cuda(m.mask, torch.uint8), p=g["p"], eps=g["tau"],
                          precond=g["precond"], tol=g["tol"], max_outer=g["max_outer"])
    assert st["outer"] == g["stats"]["outer"]
    for a, b in zip(st["inner"], g["stats"]["inner"]):
        assert abs(a - b) <= ITER_TOL, (st["inner"], g["stats"]["inner"])
    got = phi.cpu().numpy()
    keep = m.mask == 0
    mean = got[keep].mean()
    ii, jj = np.array(g["sample_i"]), np.array(g["sample_j"])
    e = (got[ii, jj] - mean) - np.array(g["sample_phi_mean_removed"])
    assert np.sqrt(np.mean(e[keep[ii, jj]] ** 2)) < RMS_TOL  # unmasked samples (masked ones keep phi^0)
    rms_phi = float(np.sqrt(np.mean((got[keep] - mean) ** 2)))
    assert abs(rms_phi - g["rms_phi_mean_removed"]) < RMS_TOL
