"""Training of the learned preconditioner, driven through the C ABI.

1. Harvest: for each training map (the 256^2 workload's generator at the
   training size: ramp 0.05 rad/px, 6 bumps of width 10-40 px scaled to the
   size, noise 0.3 rad; p = 0.5, tau = 0.01) take the IRLS weights U, V and the
   right-hand side b of Eq. (Axb) at a few outer passes of Algorithm 1, and let
   the plain Jacobi PCG produce pairs (r_l, e_l) = (b - A phi_l, phi* - phi_l)
   at a spread of iteration counts l (ulp_unet_harvest).
2. Train: Adam on the direction loss of ulp_unet_loss_grad (how much of the
   error's energy norm one exact line search along s = D^-1 r + rho N leaves),
   in minibatches of pairs drawn in a seeded random order (ulp_unet_train_step).
   The learned-preconditioner workload trains on 667 maps x 3 passes x 10
   iteration counts = 20,010 pairs of 512^2 (84 GB of FP64 planes in HBM).

Every step runs in the library's kernels; torch only holds device memory.

usage: python -m paper_2203_13675_gb300.learned --maps 667 --size 512 --epochs 2 --out unet.bin
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import native, synth

ITERS = (0, 2, 5, 10, 20, 40, 80, 160, 320, 640)


def training_map(size, seed):
    scale = size / 256.0
    return synth.phase_map(size, size, seed, ramp=0.05, n_bumps=6, noise=0.3,
                           sigma_range=(10.0 * scale, 40.0 * scale))


def harvest(n_maps, size=512, p=0.5, eps=1e-2, passes=(0, 2, 4), iters=ITERS, seed0=1000, log=None):
    """Returns dict of device tensors r [N,H,W], e [N,H,W], U [S,H,W], V [S,H,W] and sys [N] (host)."""
    S = n_maps * len(passes)
    N = S * len(iters)
    dev = torch.device("cuda")
    r = torch.empty((N, size, size), dtype=torch.float64, device=dev)
    e = torch.empty_like(r)
    U = torch.empty((S, size, size), dtype=torch.float64, device=dev)
    V = torch.empty_like(U)
    b = torch.empty((size, size), dtype=torch.float64, device=dev)
    sys_of = np.repeat(np.arange(S), len(iters))
    plan = native.Plan(size, size, outer_tol=0.0)
    t0 = time.perf_counter()
    s = 0
    for m in range(n_maps):
        psi = torch.from_numpy(training_map(size, seed0 + m).psi).to(dev)
        dx, dy = native.ulp_wrapped_diffs(psi)
        for k in passes:
            if k == 0:
                phi = torch.zeros_like(psi)
            else:
                phi, _ = plan.unwrap(psi, None, p=p, eps=eps, precond="mg", tol=1e-6, max_outer=k)
            native.ulp_weights(phi, dx, dy, None, p=p, eps=eps, U=U[s], V=V[s], b=b)
            lo = s * len(iters)
            native.ulp_unet_harvest(U[s], V[s], b, iters, precond="jacobi", tol_star=1e-10,
                                    r_out=r[lo:lo + len(iters)], e_out=e[lo:lo + len(iters)])
            s += 1
        if log:
            log(f"harvest map {m + 1}/{n_maps}  {time.perf_counter() - t0:.1f} s")
    plan.close()
    return {"r": r, "e": e, "U": U, "V": V, "sys": sys_of}


def train(net, data, epochs=4, batch=8, lr=1e-3, seed=0, log=None, loss_every=1):
    """Adam over shuffled minibatches; returns the losses of every loss_every-th step (reading a
    loss back synchronises, so the steps in between run without waiting for the GPU)."""
    rng = np.random.default_rng(seed)
    N = data["r"].shape[0]
    losses = []
    t0 = time.perf_counter()
    step = 0
    for ep in range(epochs):
        order = rng.permutation(N)
        n_ep = len(losses)
        for k in range(0, N - batch + 1, batch):
            idx = order[k:k + batch]
            want = step % loss_every == 0
            l = net.train_step(idx, data["sys"][idx], data["r"], data["e"], data["U"], data["V"], lr=lr,
                               want_loss=want)
            if want:
                losses.append(l)
            step += 1
        if log:
            log(f"epoch {ep + 1}/{epochs}  loss {np.mean(losses[n_ep:] or losses[-1:]):.4f}  "
                f"{time.perf_counter() - t0:.1f} s")
    return losses


def evaluate(net, size=2048, p=0.5, seed=5, max_outer=5, tol=1e-6, preconds=("jacobi", "dct", "learned"),
             reps=2):
    """Unwraps one held-out map (the training generator at `size`, `seed`) with each
    preconditioner: Mpixel/s (CUDA events, best of `reps` after a warm-up), inner
    iterations per pass, fallbacks, and the RMS difference to the Jacobi solution."""
    m = training_map(size, seed)
    psi = torch.from_numpy(m.psi).cuda()
    plan = native.Plan(size, size, outer_tol=0.0)
    plan.set_unet(net)
    out, ref = {}, None
    for pc in preconds:
        phi, st = plan.unwrap(psi, None, p=p, precond=pc, tol=tol, max_outer=max_outer)
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            phi, st = plan.unwrap(psi, None, p=p, precond=pc, tol=tol, max_outer=max_outer, stats=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        _, st = plan.unwrap(psi, None, p=p, precond=pc, tol=tol, max_outer=max_outer)
        a = phi.cpu().numpy()
        if ref is None:
            ref = a
        d = a - ref
        out[pc] = {"ms": best, "mpx_s": size * size / (best * 1e3), "inner": st["inner"],
                   "inner_total": st["inner_total"], "fallbacks": st["fallbacks"], "status": st["status"],
                   "rms_vs_first": float(np.sqrt(np.mean((d - d.mean()) ** 2)))}
    plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--maps", type=int, default=667)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="unet.bin")
    ap.add_argument("--report", default=None)
    ap.add_argument("--eval-size", type=int, default=0, help="also evaluate on a held-out map of this size")
    a = ap.parse_args()
    t0 = time.perf_counter()
    data = harvest(a.maps, a.size, log=print)
    t1 = time.perf_counter()
    net = native.Unet(seed=a.seed)
    losses = train(net, data, a.epochs, a.batch, a.lr, a.seed, log=print, loss_every=50)
    t2 = time.perf_counter()
    net.save(a.out)
    rep = {"pairs": int(data["r"].shape[0]), "size": a.size, "harvest_s": t1 - t0, "train_s": t2 - t1,
           "steps": len(losses), "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:]))}
    if a.eval_size:
        rep["eval"] = evaluate(net, a.eval_size)
    print(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f)


if __name__ == "__main__":
    main()
