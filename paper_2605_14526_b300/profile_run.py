"""Short, fixed workloads for profiler captures (a few thousand launches).

  python -m paper_2605_14526_b300.profile_run --case bar --steps 2

Runs `steps` PD steps of the named workload forward and backward once as a
warm-up and once more, so that a profiler can skip the first pass.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import binding, inputs
from .build import build

CASES = {
    "cube": lambda s: inputs.small_cube(steps=s),
    "bar": lambda s: inputs.hetero_bar(steps=s),
    "smallbar": lambda s: inputs.hetero_bar(nx=8, ny=4, nz=4, block=4, steps=s),
    # 8 uneven meshes of 1k-10k tets in one batched launch
    "batch8": lambda s: inputs.batch_meshes(n=8, tets_lo=1000, tets_hi=10000, steps=s, seed=11),
    # the full batched workload (64 meshes)
    "batch64": lambda s: inputs.batch_meshes(steps=s),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="bar", choices=sorted(CASES))
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--phases", action="store_true", help="print device phase times of the forward rollout")
    ap.add_argument("--persistent", type=int, default=1)
    args = ap.parse_args()
    build()
    sc = CASES[args.case](args.steps)
    dev = "cuda:0"
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    if isinstance(sc, list):   # a batch of instances in one launch
        scenes = sc
        sc = scenes[0]
        opt = binding.options_for(sc.solver)
        opt.persistent = args.persistent
        pd = binding.BatchContext(scenes, opt)
        x0 = t(pd.concat([s.x0 for s in scenes]).reshape(-1, 3))
        v0 = t(pd.concat([s.v0 for s in scenes]).reshape(-1, 3))
        f0 = t(pd.concat([s.f_ext[0] for s in scenes]).reshape(-1, 3))
        n_e = pd.n_e
    else:
        opt = binding.options_for(sc.solver)
        opt.persistent = args.persistent
        pd = binding.PDContext(sc, opt)
        x0, v0, f0 = t(sc.x0), t(sc.v0), t(sc.f_ext[0])
        n_e = sc.n_e
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
    dE = torch.empty(n_e, dtype=torch.float64, device=dev)
    dnu = torch.empty(getattr(pd, "n", 1), dtype=torch.float64, device=dev)
    names = ["begin", "local", "assemble+gate", "S b", "S^T y+AA dots (to reduction)", "AA solve", "update", "end+tr"]
    for r in range(args.repeat):
        if args.phases and r == args.repeat - 1 and not hasattr(pd, "n"):
            binding.pd_profile(pd.ctx, True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        binding.pd_rollout(pd.ctx, sc.steps, x0, v0, f0, 0, qT, vT)
        e1.record()
        binding.pd_backward(pd.ctx, qT, None, dq0, dv0, dE, dnu, None, 0)
        e2.record()
        torch.cuda.synchronize()
        print(f"repeat {r}: forward {e0.elapsed_time(e1):.2f} ms, backward {e1.elapsed_time(e2):.2f} ms")
    if args.phases and not hasattr(pd, "n"):
        p = binding.pd_get_profile(pd.ctx)
        print("forward phases (ms): " + ", ".join(f"{n} {p.phase_ms[i]:.3f}" for i, n in enumerate(names)))
        print("  block-0 work (ms): " + ", ".join(f"{n} {p.work_ms[i]:.3f}" for i, n in enumerate(names)))
        print("  critical-block work (ms): " + ", ".join(f"{n} {p.work_max_ms[i]:.3f}" for i, n in enumerate(names)))
        print("  to last arrival (ms): " + ", ".join(f"{n} {p.last_ms[i]:.3f}" for i, n in enumerate(names)))
    st = binding.pd_get_stats(pd.ctx)
    print(f"{args.case}: {st.iters_total} forward iterations, {st.adj_iters_total} adjoint iterations, "
          f"{st.launches} launches")
    pd.close()


if __name__ == "__main__":
    main()
