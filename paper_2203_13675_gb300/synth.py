"""Seeded synthetic wrapped-phase maps (the only module shared by the CUDA path's
callers and the oracle's tests).

It holds none of the unwrapping method's arithmetic: it draws a true phase,
forms the complex signal S exp(i phi) of the paper's signal model (Sec. 1) and
takes its angle, which is the wrapped phase psi in (-pi, pi].

Recipe (stands in for the paper's 640x480 map of Fig. 1, which is not
available): true phase = ramp along the columns + Gaussian bumps (centres
uniform in the image, sigma ~ U[10, 40] px, amplitude ~ U[-30, 30] rad) +
i.i.d. Gaussian noise; optionally a disk covering a fraction of the pixels
where the signal amplitude is zero, so its phase is uniform noise and its
pixels are masked out.  All randomness comes from numpy's PCG64(seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class PhaseMap:
    psi: np.ndarray            # wrapped phase, (H, W) float64 in (-pi, pi]
    phi_true: np.ndarray       # the phase that was wrapped, (H, W) float64
    mask: np.ndarray | None    # (H, W) uint8, 1 = pixel excluded, or None


def phase_map(H: int, W: int, seed: int, ramp: float = 0.05, n_bumps: int = 6,
              noise: float = 0.3, mask_frac: float = 0.0,
              sigma_range=(10.0, 40.0), amplitude: float = 30.0) -> PhaseMap:
    rng = np.random.Generator(np.random.PCG64(seed))
    ii = np.arange(H, dtype=np.float64)[:, None]
    jj = np.arange(W, dtype=np.float64)[None, :]
    phi = np.broadcast_to(ramp * jj, (H, W)).copy()
    for _ in range(n_bumps):
        ci = rng.uniform(0.0, H)
        cj = rng.uniform(0.0, W)
        sb = rng.uniform(*sigma_range)
        amp = rng.uniform(-amplitude, amplitude)
        gi = np.exp(-((ii - ci) ** 2) / (2.0 * sb * sb))
        gj = np.exp(-((jj - cj) ** 2) / (2.0 * sb * sb))
        phi += amp * (gi * gj)
    if noise > 0.0:
        phi += rng.normal(0.0, noise, size=(H, W))
    mask = None
    if mask_frac > 0.0:
        rad = math.sqrt(mask_frac * H * W / math.pi)
        ci = rng.uniform(rad, H - rad)
        cj = rng.uniform(rad, W - rad)
        inside = ((ii - ci) ** 2 + (jj - cj) ** 2) <= rad * rad
        phi[inside] = rng.uniform(-math.pi, math.pi, size=int(inside.sum()))
        mask = inside.astype(np.uint8)
    # phase of the complex signal exp(i phi): atan2 gives [-pi, pi]; move -pi to +pi
    psi = np.arctan2(np.sin(phi), np.cos(phi))
    psi = np.where(psi <= -math.pi, psi + 2.0 * math.pi, psi)
    return PhaseMap(np.ascontiguousarray(psi), phi, mask)


# Named workloads.  Sizes, p, tau and preconditioners follow the paper's
# experiment design (Sec. 3) scaled to the GPU's sizes.
WORKLOADS = {
    # 256x256, ramp 0.05 rad/px, 6 bumps, noise 0.3; p = 1, tau = 1e-2, 5 outer, Jacobi
    "c1_256": dict(H=256, W=256, seed=1, ramp=0.05, n_bumps=6, noise=0.3, mask_frac=0.0,
                   p=1.0, tau=1e-2, max_outer=5, tol=1e-6, precond="jacobi"),
    # 1024x1024 / 2048x2048, ramp 0.02, 12 bumps, noise 0.5, 5 % masked disk
    "c2_1024": dict(H=1024, W=1024, seed=2, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=0.05,
                    p=1.0, tau=1e-2, max_outer=5, tol=1e-6, precond="jacobi"),
    "c2_2048": dict(H=2048, W=2048, seed=3, ramp=0.02, n_bumps=12, noise=0.5, mask_frac=0.05,
                    p=1.0, tau=1e-2, max_outer=5, tol=1e-6, precond="jacobi"),
    # 4096x4096, ramp 0.02, 12 bumps, noise 0.7, p = 0.5 (mixed precision)
    "c3_4096": dict(H=4096, W=4096, seed=4, ramp=0.02, n_bumps=12, noise=0.7, mask_frac=0.0,
                    p=0.5, tau=1e-2, max_outer=5, tol=1e-6, precond="jacobi"),
    # learned-preconditioner test map: the 256x256 generator at 2048x2048 (bump widths
    # scaled by 8), p = 0.5; the network trains on the same generator at 512x512
    "c5_2048": dict(H=2048, W=2048, seed=5, ramp=0.05, n_bumps=6, noise=0.3, mask_frac=0.0,
                    p=0.5, tau=1e-2, max_outer=5, tol=1e-6, precond="jacobi", sigma_scale=8.0),
}


def workload_map(name: str) -> PhaseMap:
    w = WORKLOADS[name]
    sc = w.get("sigma_scale", 1.0)
    return phase_map(w["H"], w["W"], w["seed"], ramp=w["ramp"], n_bumps=w["n_bumps"],
                     noise=w["noise"], mask_frac=w["mask_frac"], sigma_range=(10.0 * sc, 40.0 * sc))


def batch_specs(n: int = 64, seed0: int = 100):
    """64 uneven maps: side ~ U{256, 384, 512, 768, 1024, 1536, 2048}, p ~ U{0, 1},
    noise ~ U[0.1, 0.8], ramp 0.02, 12 bumps; map t uses seed seed0 + t."""
    sides = [256, 384, 512, 768, 1024, 1536, 2048]
    specs = []
    for t in range(n):
        rng = np.random.Generator(np.random.PCG64(seed0 + t))
        side = int(sides[rng.integers(0, len(sides))])
        p = float(rng.integers(0, 2))
        noise = float(rng.uniform(0.1, 0.8))
        specs.append(dict(H=side, W=side, seed=seed0 + t + 10_000, p=p, noise=noise,
                          ramp=0.02, n_bumps=12))
    return specs


def batch_maps(specs):
    return [phase_map(s["H"], s["W"], s["seed"], ramp=s["ramp"], n_bumps=s["n_bumps"],
                      noise=s["noise"]) for s in specs]


def smooth_map(H: int, W: int, seed: int) -> PhaseMap:
    """Noiseless phase whose true gradients stay below pi (exact-recovery case)."""
    return phase_map(H, W, seed, ramp=0.05, n_bumps=4, noise=0.0, sigma_range=(6.0, 12.0),
                     amplitude=8.0)
