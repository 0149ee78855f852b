"""Writes table1_oracle.json: the FP64 CPU oracle's columns of the paper's Table-1 study.

Calls only oracle/ and the seeded generator.  For each Table-1 size (columns x
rows) and preconditioner, the same synthetic map as the GPU study
(paper_2203_13675_gb300/experiment_table1.py: the 256^2 workload's generator,
bump widths scaled with the size, seed 1), p = 1, tau = 0.01 and the paper's
criteria (Sec. 3): k_max = 500 outer passes, outer tolerance 1e-6, Algorithm 1's
inner test delta_new <= eps^2 delta_0 with eps = 0.005, l_max = 2MN.  Records the
outer passes, the summed inner iterations (Fig. 2), the wall time of the whole
unwrap on one core (Fig. 3) and the time spent building the preconditioner from
A in every pass, whose share of the total is what the paper reports (1-2 % for
I, Jacobi, ILU(0) and SOR; more than 90 % for its IC(0)).

usage: python tests/golden/make_table1_oracle.py [--jobs N] [--max-px N] [precond ...]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_13675_gb300 import synth  # noqa: E402

SIZES = [(160, 120), (320, 240), (480, 360), (640, 480), (800, 600), (960, 720), (1120, 840), (1280, 960)]
KINDS = {"identity": oracle.M_IDENTITY, "jacobi": oracle.M_JACOBI, "ilu0": oracle.M_ILU0, "ic0": oracle.M_IC0,
         "ssor": oracle.M_SSOR, "rbssor": oracle.M_RBSSOR, "rbilu": oracle.M_RBILU, "dct": oracle.M_DCT,
         "mg": oracle.M_MG}


def make_map(cols, rows, seed=1):
    scale = cols / 640.0
    return synth.phase_map(rows, cols, seed, ramp=0.05, n_bumps=6, noise=0.3,
                           sigma_range=(10.0 * scale, 40.0 * scale))


def run(job):
    cols, rows, pc = job
    m = make_map(cols, rows)
    t0 = time.perf_counter()
    _, st = oracle.unwrap(m.psi, None, p=1.0, tau=0.01, kind=KINDS[pc], tol=0.005, max_outer=500,
                          outer_tol=1e-6, stop_mode=oracle.STOP_PAPER)
    wall = time.perf_counter() - t0
    return {"cols": cols, "rows": rows, "precond": pc, "oracle_s": wall, "outer": st["outer"],
            "inner_total": st["inner_total"], "status": st["status"], "setup_s": st["setup_s"],
            "setup_share": st["setup_s"] / wall}


if __name__ == "__main__":
    args = sys.argv[1:]
    jobs, max_px = 1, 1280 * 960
    while args and args[0].startswith("--"):
        if args[0] == "--jobs":
            jobs, args = int(args[1]), args[2:]
        elif args[0] == "--max-px":
            max_px, args = int(args[1]), args[2:]
    pcs = args or ["identity", "jacobi", "ilu0", "ic0", "ssor"]
    todo = [(c, r, pc) for c, r in SIZES if c * r <= max_px for pc in pcs]
    path = os.path.join(HERE, "table1_oracle.json")
    with mp.get_context("spawn").Pool(jobs) as pool:
        for row in pool.imap_unordered(run, todo):
            data = json.load(open(path)) if os.path.exists(path) else []
            data = [d for d in data if (d["cols"], d["rows"], d["precond"]) != (row["cols"], row["rows"],
                                                                                row["precond"])]
            data.append(row)
            data.sort(key=lambda d: (d["cols"] * d["rows"], d["precond"]))
            with open(path, "w") as f:
                json.dump(data, f, indent=1)
            print(json.dumps(row), flush=True)
