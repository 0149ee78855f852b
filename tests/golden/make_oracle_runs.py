"""Writes oracle_runs.json (and runs/<name>.npz): the FP64 CPU oracle's own results on
full-size workloads.

Calls only oracle/ and the seeded generator.  Records, per run, the inner PCG
iterations and relative residuals of every outer pass, the outer errors, the
wall time, and the oracle's phase (mean-removed over unmasked pixels) at 256
sampled pixels in the JSON, plus, in runs/<name>.npz, the phase at a denser
fixed sample of pixels (DENSE of them, drawn from their own seed) and its means
over 32 x 32 blocks (unmasked pixels only), so that the GPU path can be compared
at full size without re-running the oracle.  Takes minutes to tens of minutes
per 2048^2 case; --jobs runs several cases at once, one process each.

Run names:
  <workload>_p<p>_<precond>   a named workload of synth.WORKLOADS, e.g. c2_2048_p1_jacobi
  c4_<t>_<precond>            map t of the 64-map batch (synth.batch_specs), its own p,
                              tau 1e-2, 5 passes, tol 1e-6, no mask

usage: python tests/golden/make_oracle_runs.py [--jobs N] c2_2048_p1_jacobi [...]
"""
import json
import multiprocessing as mp
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
DENSE = 8192
BLOCK = 32


def parse(name):
    """(workload, map, p, precond, tau, tol, max_outer) of a run name."""
    if name.startswith("c4_"):
        _, t, kind = name.split("_", 2)
        spec = synth.batch_specs(64)[int(t)]
        m = synth.batch_maps([spec])[0]
        return "c4", m, spec["p"], kind, 1e-2, 1e-6, 5
    wl, rest = name.rsplit("_p", 1)
    p, kind = rest.split("_", 1)
    w = synth.WORKLOADS[wl]
    return wl, synth.workload_map(wl), float(p), kind, w["tau"], w["tol"], w["max_outer"]


def sample_pixels(H, W, n=256, seed=12345):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, H, n), rng.integers(0, W, n)


def dense_pixels(H, W):
    return sample_pixels(H, W, DENSE, seed=67890)


def block_means(phi, keep, b=BLOCK):
    """Means of phi over b x b blocks (ragged last blocks included), unmasked pixels only
    (NaN for a block with none)."""
    H, W = phi.shape
    nb_i, nb_j = (H + b - 1) // b, (W + b - 1) // b
    s = np.zeros((nb_i, nb_j))
    c = np.zeros((nb_i, nb_j))
    ii = np.arange(H) // b
    jj = np.arange(W) // b
    np.add.at(s, (ii[:, None], jj[None, :]), np.where(keep, phi, 0.0))
    np.add.at(c, (ii[:, None], jj[None, :]), keep.astype(np.float64))
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(c > 0, s / np.maximum(c, 1), np.nan)


def run(name):
    wl, m, p, kind, tau, tol, max_outer = parse(name)
    t0 = time.time()
    phi, st = oracle.unwrap(m.psi, m.mask, p=p, tau=tau, kind=KINDS[kind], tol=tol,
                            max_outer=max_outer, outer_tol=0.0)
    wall = time.time() - t0
    keep = np.ones(phi.shape, bool) if m.mask is None else (m.mask == 0)
    mean = float(phi[keep].mean())
    ii, jj = sample_pixels(*phi.shape)
    di, dj = dense_pixels(*phi.shape)
    np.savez_compressed(os.path.join(HERE, "runs", name + ".npz"),
                        dense_phi_mean_removed=(phi[di, dj] - mean),
                        block_means=block_means(phi - mean, keep))
    return {"workload": wl, "p": p, "precond": kind, "tau": tau, "tol": tol,
            "max_outer": max_outer, "outer_tol": 0.0, "stats": st, "wall_s": wall,
            "sample_i": ii.tolist(), "sample_j": jj.tolist(),
            "sample_phi_mean_removed": [float(phi[i, j] - mean) for i, j in zip(ii, jj)],
            "rms_phi_mean_removed": float(np.sqrt(np.mean((phi[keep] - mean) ** 2))),
            "dense": DENSE, "block": BLOCK}


def _job(name):
    return name, run(name)


if __name__ == "__main__":
    args = sys.argv[1:]
    jobs = 1
    if args and args[0] == "--jobs":
        jobs, args = int(args[1]), args[2:]
    os.makedirs(os.path.join(HERE, "runs"), exist_ok=True)
    path = os.path.join(HERE, "oracle_runs.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    with mp.get_context("spawn").Pool(jobs) as pool:
        for name, res in pool.imap_unordered(_job, args):
            data = json.load(open(path)) if os.path.exists(path) else {}
            data[name] = res
            print(name, res["stats"]["inner"], f"{res['wall_s']:.1f}s", flush=True)
            with open(path, "w") as f:
                json.dump(data, f, indent=1)
