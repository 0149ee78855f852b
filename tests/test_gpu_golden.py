"""Every full-size run the FP64 oracle has recorded (tests/golden/oracle_runs.json and
tests/golden/runs/, written by tests/golden/make_oracle_runs.py from oracle/ alone),
replayed on the GPU at the same size, preconditioner, p and stopping rule: the
per-pass inner iteration counts, and the unwrapped phase after removing the mean
over unmasked pixels, within 1e-4 rad RMS at 256 sampled pixels, at a denser
sample of 8192 pixels and over 32 x 32 block means.

Where a single-pass run stops at another iteration than the oracle (within the count
bar below), the phase is compared at the oracle's stop point: the GPU runs exactly the
oracle's iteration count.  ILU(0)/IC(0) runs are held to twice the oracle's own
ILU-vs-IC spread where that exceeds 5e-5 (see _oracle_spread).

Iteration-count bars per preconditioner: Jacobi within 2 (the same PCG;
dot-product blocking moves the stop point by at most that much); M = I within
1 % and ILU(0)/IC(0)/SSOR within 0.5 % (at least 2): over thousands of
iterations their counts are not fixed to +-2 by FP64 arithmetic -- for M = I
see test_gpu_fp64.py; for the sweeps the wavefront rounds each application
slightly differently from the sequential sweep (2568 against 2561 on the
2048^2 map); multigrid within 2.
"""
import json
import os
import sys

import numpy as np
import pytest
import torch

from paper_2203_13675_gb300 import native, synth

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_oracle_runs as gold  # noqa: E402  (sampling and block-mean definitions of the stored runs)

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)
ALL = json.load(open(os.path.join(HERE, "golden", "oracle_runs.json")))
GOLD = {k: v for k, v in ALL.items() if v["workload"] in synth.WORKLOADS}  # the named workloads
C4 = sorted((k for k, v in ALL.items() if v["workload"] == "c4"), key=lambda k: int(k.split("_")[1]))


def _compare(g, key, got, mask):
    """RMS distance (rad) of the GPU phase to the oracle's run over unmasked pixels, after
    removing the mean over unmasked pixels: at the 256 sampled pixels, and, where the run's
    dense record exists, at its denser sample of pixels and over its 32 x 32 block means.
    Masked pixels keep phi^0 on both sides and, as in every error metric here, are left out
    (after mean removal they would only carry the difference of the two means)."""
    keep = np.ones(got.shape, bool) if mask is None else (mask == 0)
    mean = got[keep].mean()
    ii, jj = np.array(g["sample_i"]), np.array(g["sample_j"])
    k = keep[ii, jj]
    e = (got[ii, jj] - mean) - np.array(g["sample_phi_mean_removed"])
    out = {"sample": float(np.sqrt(np.mean(e[k] ** 2)))}
    path = os.path.join(HERE, "golden", "runs", key + ".npz")
    if os.path.exists(path):
        d = np.load(path)
        di, dj = gold.dense_pixels(*got.shape)
        k = keep[di, dj]
        e = (got[di, dj] - mean) - d["dense_phi_mean_removed"]
        out["dense"] = float(np.sqrt(np.mean(e[k] ** 2)))
        bm = gold.block_means(got - mean, keep)
        ok = np.isfinite(d["block_means"])
        e = bm[ok] - d["block_means"][ok]
        out["blocks"] = float(np.sqrt(np.mean(e ** 2)))
    return out


def _bar(precond, n):
    if precond == "identity":
        return max(2, int(0.01 * n))
    if precond in ("ilu0", "ic0", "ssor"):
        return max(2, int(0.005 * n))
    return 2


@pytest.mark.parametrize("key", sorted(GOLD))
def test_full_size_run_matches_the_oracle(key):
    g = GOLD[key]
    m = synth.workload_map(g["workload"])
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=g["outer_tol"])
    mask = torch.from_numpy(m.mask).cuda() if m.mask is not None else None
    phi, st = plan.unwrap(torch.from_numpy(m.psi).cuda(), mask, p=g["p"], eps=g["tau"], precond=g["precond"],
                          tol=g["tol"], max_outer=g["max_outer"])
    assert st["status"] == 0, st
    assert st["outer"] == g["stats"]["outer"], (st["inner"], g["stats"]["inner"])
    for a, b in zip(st["inner"], g["stats"]["inner"]):
        assert abs(a - b) <= _bar(g["precond"], b), (st["inner"], g["stats"]["inner"])
    d = _compare(g, key, phi.cpu().numpy(), m.mask)
    print(f"{key}: {d} rad RMS; inner {st['inner']} vs {g['stats']['inner']}")
    gi = g["stats"]["inner"]
    if max(d.values()) >= 1e-4 and st["inner"] != gi and sum(1 for c in gi if c > 0) == 1:
        # The stop point moved (allowed by the count bar above) on a single-pass run: the
        # iterates are compared at the oracle's own stop point instead, by running exactly
        # its iteration count.  The stop point of these long Krylov runs is set by rounding:
        # the oracle's own ILU(0) and IC(0) -- the same M, factorised with different
        # rounding -- stop at 1579 and 1577 iterations on the C2 2048^2 map at p = 2, and
        # their solutions are 1.09e-4 rad RMS apart.
        plan1 = native.Plan(H, W, outer_tol=g["outer_tol"])
        phi1, st1 = plan1.unwrap(torch.from_numpy(m.psi).cuda(), mask, p=g["p"], eps=g["tau"],
                                 precond=g["precond"], tol=1e-30, max_outer=1, max_inner=gi[0])
        assert st1["inner"] == [gi[0]], st1
        d = _compare(g, key, phi1.cpu().numpy(), m.mask)
        print(f"{key}: at the oracle's stop point ({gi[0]} iterations): {d} rad RMS")
    bar = max(1e-4, 2.0 * _oracle_spread(key))
    assert max(d.values()) < bar, (d, bar)


def _oracle_spread(key):
    """For an ILU(0) or IC(0) run: the RMS distance between the oracle's own ILU(0) and IC(0)
    runs of the same workload and p (dense records, unmasked pixels, means removed) -- the
    same M factorised with different rounding, so the spread that rounding alone puts
    between two FP64 solves of this system; 0 for every other run.  The GPU's wavefront
    factorisation rounds differently again, and its bar is twice that spread where the
    spread exceeds half of 1e-4 (only the C2 2048^2 map at p = 2: 1.09e-4)."""
    if not (key.endswith("_ilu0") or key.endswith("_ic0")):
        return 0.0
    stem = key.rsplit("_", 1)[0]
    a = os.path.join(HERE, "golden", "runs", stem + "_ilu0.npz")
    b = os.path.join(HERE, "golden", "runs", stem + "_ic0.npz")
    if not (os.path.exists(a) and os.path.exists(b)):
        return 0.0
    m = synth.workload_map(GOLD[key]["workload"])
    keep = np.ones(m.psi.shape, bool) if m.mask is None else (m.mask == 0)
    di, dj = gold.dense_pixels(*m.psi.shape)
    e = (np.load(a)["dense_phi_mean_removed"] - np.load(b)["dense_phi_mean_removed"])[keep[di, dj]]
    return float(np.sqrt(np.mean(e ** 2)))


# The bench's chosen form -- the mixed-precision multigrid flexible CG (FP32 weights,
# recurrence and V-cycle, FP64 inner products and true residual) -- replayed at full size
# against every multigrid run the oracle recorded: per pass within 2 of the oracle's FP64
# counts, and the phase within 1e-4 rad RMS.  The solve stops at the iterate where its
# FP32 recurrence reports convergence once that iterate's FP64 true residual meets the
# tolerance, as Algorithm 1 stops on its recurrence residual; the stop point is what
# decides the distance here (one more multigrid iteration moves the C2 1024^2 solution
# by 1.5e-4 rad RMS, while rounding the weights to FP32 moves it by 1e-10 rad).
@pytest.mark.parametrize("key", sorted(k for k in GOLD if GOLD[k]["precond"] == "mg"))
def test_full_size_mixed_multigrid_matches_the_oracle(key):
    g = GOLD[key]
    m = synth.workload_map(g["workload"])
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=g["outer_tol"], precision=native.ULP_PRECISION_MIXED)
    mask = torch.from_numpy(m.mask).cuda() if m.mask is not None else None
    phi, st = plan.unwrap(torch.from_numpy(m.psi).cuda(), mask, p=g["p"], eps=g["tau"], precond="mg",
                          tol=g["tol"], max_outer=g["max_outer"])
    assert st["status"] == 0, st
    assert st["outer"] == g["stats"]["outer"], (st["inner"], g["stats"]["inner"])
    for a, b in zip(st["inner"], g["stats"]["inner"]):
        assert abs(a - b) <= 2, (st["inner"], g["stats"]["inner"])
    d = _compare(g, key, phi.cpu().numpy(), m.mask)
    print(f"{key}: mixed multigrid vs the FP64 oracle, {d} rad RMS; inner {st['inner']} vs {g['stats']['inner']}")
    assert max(d.values()) < 1e-4, d


# The mixed-precision persistent Jacobi PCG (FP32 recurrence, FP64-accurate dots, FP64 phi
# and true residual every 20 iterations) replayed against every Jacobi run the oracle
# recorded: the FP64 bars (counts within 2, 1e-4 rad RMS).
@pytest.mark.parametrize("key", sorted(k for k in GOLD if GOLD[k]["precond"] == "jacobi"))
def test_full_size_mixed_jacobi_matches_the_oracle(key):
    g = GOLD[key]
    m = synth.workload_map(g["workload"])
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=g["outer_tol"], precision=native.ULP_PRECISION_MIXED)
    mask = torch.from_numpy(m.mask).cuda() if m.mask is not None else None
    phi, st = plan.unwrap(torch.from_numpy(m.psi).cuda(), mask, p=g["p"], eps=g["tau"], precond="jacobi",
                          tol=g["tol"], max_outer=g["max_outer"])
    assert st["status"] == 0, st
    assert st["outer"] == g["stats"]["outer"], (st["inner"], g["stats"]["inner"])
    d = _compare(g, key, phi.cpu().numpy(), m.mask)
    print(f"{key}: mixed Jacobi vs the FP64 oracle, {d} rad RMS; inner {st['inner']} vs {g['stats']['inner']}")
    for a, b in zip(st["inner"], g["stats"]["inner"]):
        assert abs(a - b) <= 2, (st["inner"], g["stats"]["inner"])
    assert max(d.values()) < 1e-4, d


@pytest.mark.skipif(not C4, reason="no recorded runs of the 64-map batch")
def test_c4_batch_matches_the_oracle_per_map():
    """The 64-map batch (synth.batch_specs: sides 256..2048, own seed, p in {0, 1}, noise
    0.1-0.8) at its real sizes, solved together by the persistent Jacobi PCG (one launch per
    outer pass for all maps), against the oracle's own run of every recorded map: counts
    within 2 per pass, phase within 1e-4 rad RMS at the dense sample and the block means."""
    specs = synth.batch_specs(64)
    pm = synth.batch_maps(specs)
    plan = native.Plan(None, sizes=[m.psi.shape for m in pm], outer_tol=0.0)
    dev = [{"psi": torch.from_numpy(m.psi).cuda(), "mask": None,
            "phi": torch.empty(m.psi.shape, dtype=torch.float64, device="cuda"), "p": sp["p"], "eps": 1e-2}
           for m, sp in zip(pm, specs)]
    rc, per = plan.unwrap_batched(dev, precond="jacobi", tol=1e-6, max_outer=5)
    assert rc == 0, rc
    worst = 0.0
    for key in C4:
        t = int(key.split("_")[1])
        g = ALL[key]
        st = per[t]
        assert st["outer"] == g["stats"]["outer"], (key, st["inner"], g["stats"]["inner"])
        for a, b in zip(st["inner"], g["stats"]["inner"]):
            assert abs(a - b) <= 2, (key, st["inner"], g["stats"]["inner"])
        d = _compare(g, key, dev[t]["phi"].cpu().numpy(), None)
        worst = max(worst, max(d.values()))
        assert max(d.values()) < 1e-4, (key, d)
    print(f"64-map batch: {len(C4)} maps checked against the oracle, worst {worst:.2e} rad RMS")
