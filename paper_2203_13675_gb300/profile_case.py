"""A bounded run of the solver for profilers (ncu): one plan, a few calls.

usage: python -m paper_2203_13675_gb300.profile_case [--workload c2_2048] [--precond jacobi]
       [--max-inner 200] [--max-outer 1] [--calls 2]

Each call runs max_outer passes with the inner PCG capped at max_inner
iterations, so a capture of the persistent solver kernel ends in seconds.
"""
import argparse

import torch

from . import native, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2_2048")
    ap.add_argument("--precond", default="jacobi")
    ap.add_argument("--precision", default="f64", choices=["f64", "mixed"])
    ap.add_argument("--max-inner", type=int, default=200)
    ap.add_argument("--max-outer", type=int, default=1)
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--eager", action="store_true", help="host-driven flexible-CG solve (every kernel a host launch, visible to ncu)")
    a = ap.parse_args()
    w = synth.WORKLOADS[a.workload]
    m = synth.workload_map(a.workload)
    psi = torch.from_numpy(m.psi).cuda()
    mask = torch.from_numpy(m.mask).cuda() if m.mask is not None else None
    H, W = m.psi.shape
    plan = native.Plan(H, W, outer_tol=0.0, profile=2 if a.eager else 0,
                       precision=native.ULP_PRECISION_MIXED if a.precision == "mixed" else 0)
    ms = []
    for _ in range(a.calls):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        phi, st = plan.unwrap(psi, mask, p=w["p"], eps=w["tau"], precond=a.precond, tol=w["tol"],
                              max_outer=a.max_outer, max_inner=a.max_inner)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    it = max(1, st["inner_total"])
    print(f"profile_case {a.workload} {a.precond} {a.precision}: inner {st['inner']} status {st['status']} "
          f"ms/call {ms} -> {1e3 * ms[-1] / it:.1f} us per inner iteration")


if __name__ == "__main__":
    main()
