"""The paper's experiment (Sec. 3) restated on one GB300.

For each image size of Table 1 (160x120 ... 1280x960, columns x rows) and each of
the paper's five preconditioners (Sec. 2 list), unwrap a synthetic wrapped map of
that size with the paper's stopping criteria: k_max = 500 outer passes, outer
tolerance 1e-6, Algorithm 1's inner test delta_new <= eps^2 delta_0 with
eps = 0.005, l_max = 2MN.  Records the inner iterations (the paper's Fig. 2)
and the time (Fig. 3) per size and preconditioner, and the device time spent
building the preconditioner (the set-up share the paper reports in Sec. 3).
--preconds picks the columns (default: the paper's five; "all" adds the
red-black, DCT and multigrid preconditioners).  The FP64 CPU oracle's columns of
the same study come from tests/golden/make_table1_oracle.py (test
infrastructure; this module runs the GPU library only).

The paper's 640x480 map (Fig. 1) is not available; each size uses the seeded
generator of synth.py (ramp 0.05 rad/px, 6 bumps with widths scaled to the
size, noise 0.3 rad).

usage: python -m paper_2203_13675_gb300.experiment_table1 [--out table1.json]
                                                         [--preconds identity,jacobi,...|all]
"""
import argparse
import json

import torch

from . import native, synth

SIZES = [(160, 120), (320, 240), (480, 360), (640, 480), (800, 600), (960, 720), (1120, 840), (1280, 960)]
PRECONDS = ["identity", "jacobi", "ilu0", "ic0", "ssor"]
# beyond the paper's list: red-black orderings of its SSOR and ILU(0), the DCT
# Poisson solve and the multigrid V-cycle (all in flexible CG)
EXTRA = ["rbssor", "rbilu", "dct", "mg"]


def make_map(cols, rows, seed=1):
    scale = cols / 640.0
    return synth.phase_map(rows, cols, seed, ramp=0.05, n_bumps=6, noise=0.3,
                           sigma_range=(10.0 * scale, 40.0 * scale))


def run(out, sizes=SIZES, preconds=PRECONDS, p=1.0):
    rows_out = []
    for cols, rows in sizes:
        m = make_map(cols, rows)
        psi = torch.from_numpy(m.psi).cuda()
        # profile = 1: the flexible-CG solves also time their preconditioner set-up
        plan = native.Plan(rows, cols, outer_tol=1e-6, stop_mode=native.ULP_STOP_PAPER, profile=1)
        for pc in preconds:
            plan.unwrap(psi, None, p=p, precond=pc, tol=0.005, max_outer=500, max_inner=0)  # warm-up
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            phi, st = plan.unwrap(psi, None, p=p, precond=pc, tol=0.005, max_outer=500, max_inner=0)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row = {"cols": cols, "rows": rows, "nnz": 5 * rows * cols - 2 * (rows + cols), "precond": pc,
                   "gpu_ms": ms, "outer": st["outer"], "inner_total": st["inner_total"],
                   "status": st["status"], "setup_ms": st["setup_ms"], "setup_share": st["setup_ms"] / ms}
            rows_out.append(row)
            print(json.dumps(row), flush=True)
        plan.close()
    if out:
        with open(out, "w") as f:
            json.dump(rows_out, f, indent=1)
    return rows_out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--p", type=float, default=1.0)
    ap.add_argument("--preconds", default=",".join(PRECONDS))
    a = ap.parse_args()
    pcs = PRECONDS + EXTRA if a.preconds == "all" else a.preconds.split(",")
    run(a.out, preconds=pcs, p=a.p)


if __name__ == "__main__":
    main()
