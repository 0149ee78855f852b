"""Writes oracle_runs.json: the FP64 CPU oracle's own results on full-size workloads.

Calls only oracle/ and the seeded generator.  Records, per workload, the inner
PCG iterations and relative residuals of every outer pass, the outer errors,
the wall time, and the oracle's phase at a fixed set of sampled pixels
(mean-removed over unmasked pixels), so the GPU path can be compared at full
size without re-running the oracle.  Takes tens of minutes per 2048^2 case.

usage: python tests/golden/make_oracle_runs.py c2_2048_p1_jacobi [...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_13675_gb300 import synth  # noqa: E402

KINDS = {"identity": oracle.M_IDENTITY, "jacobi": oracle.M_JACOBI, "ilu0": oracle.M_ILU0,
         "ic0": oracle.M_IC0, "ssor": oracle.M_SSOR, "dct": oracle.M_DCT, "mg": oracle.M_MG}


def parse(name):
    # <workload>_p<p>_<precond>, e.g. c2_2048_p1_jacobi or c2_2048_p0.5_ilu0
    wl, rest = name.rsplit("_p", 1)
    p, kind = rest.split("_", 1)
    return wl, float(p), kind


def sample_pixels(H, W, n=256, seed=12345):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, H, n), rng.integers(0, W, n)


def run(name):
    wl, p, kind = parse(name)
    w = synth.WORKLOADS[wl]
    m = synth.workload_map(wl)
    t0 = time.time()
    phi, st = oracle.unwrap(m.psi, m.mask, p=p, tau=w["tau"], kind=KINDS[kind], tol=w["tol"],
                            max_outer=w["max_outer"], outer_tol=0.0)
    wall = time.time() - t0
    keep = np.ones(phi.shape, bool) if m.mask is None else (m.mask == 0)
    mean = float(phi[keep].mean())
    ii, jj = sample_pixels(*phi.shape)
    return {"workload": wl, "p": p, "precond": kind, "tau": w["tau"], "tol": w["tol"],
            "max_outer": w["max_outer"], "outer_tol": 0.0, "stats": st, "wall_s": wall,
            "sample_i": ii.tolist(), "sample_j": jj.tolist(),
            "sample_phi_mean_removed": [float(phi[i, j] - mean) for i, j in zip(ii, jj)],
            "rms_phi_mean_removed": float(np.sqrt(np.mean((phi[keep] - mean) ** 2)))}


if __name__ == "__main__":
    path = os.path.join(HERE, "oracle_runs.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    for name in sys.argv[1:]:
        data[name] = run(name)
        print(name, data[name]["stats"]["inner"], f"{data[name]['wall_s']:.1f}s", flush=True)
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
