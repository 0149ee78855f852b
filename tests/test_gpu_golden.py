"""Every full-size run the FP64 oracle has recorded (tests/golden/oracle_runs.json,
written by tests/golden/make_oracle_runs.py from oracle/ alone), replayed on the
GPU at the same size, preconditioner, p and stopping rule: the per-pass inner
iteration counts, and the unwrapped phase at 256 sampled pixels after removing
the mean over unmasked pixels, within 1e-4 rad RMS.

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

import numpy as np
import pytest
import torch

from paper_2203_13675_gb300 import native, synth

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_runs.json")))


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
    got = phi.cpu().numpy()
    keep = np.ones(got.shape, bool) if m.mask is None else (m.mask == 0)
    mean = got[keep].mean()
    ii, jj = np.array(g["sample_i"]), np.array(g["sample_j"])
    e = (got[ii, jj] - mean) - np.array(g["sample_phi_mean_removed"])
    assert np.sqrt(np.mean(e ** 2)) < 1e-4, np.sqrt(np.mean(e ** 2))


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
    got = phi.cpu().numpy()
    keep = np.ones(got.shape, bool) if m.mask is None else (m.mask == 0)
    mean = got[keep].mean()
    ii, jj = np.array(g["sample_i"]), np.array(g["sample_j"])
    e = (got[ii, jj] - mean) - np.array(g["sample_phi_mean_removed"])
    rms = float(np.sqrt(np.mean(e ** 2)))
    print(f"{key}: mixed multigrid vs the FP64 oracle, {rms:.2e} rad RMS at 256 pixels; inner {st['inner']} "
          f"vs {g['stats']['inner']}")
    assert rms < 1e-4, rms
