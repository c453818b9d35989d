"""Short, fixed workloads for profiler captures (a few thousand launches).

  python -m paper_2605_14526_b300.profile_run --case bar --steps 2
  python -m paper_2605_14526_b300.profile_run --case block --n 48 --repeat 3
  python -m paper_2605_14526_b300.profile_run --case mlp --repeat 3 [--n 32]

Runs `steps` PD steps of the named workload forward and backward once as a
warm-up and once more, so that a profiler can skip the first pass. The block
case factors an n^3-cell block (solve mode chosen automatically: T from
about 24^3 cells) and repeats one solve with the factor (pd_solve, one launch
per separator-tree height and sweep in mode T) and one standalone local step
(pd_local_rhs). The mlp case repeats training steps of the warm-start
network and its evaluation (pd_warm_start) on the bar, or with --n on an
n^3-cell block, on seeded data.
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


def run_block(n, repeat):
    sc = inputs.large_block(n=n, steps=1)
    pd = binding.PDContext(sc)
    st = binding.pd_get_stats(pd.ctx)
    dev = "cuda:0"
    rng = np.random.default_rng(1)
    b = torch.as_tensor(rng.standard_normal((sc.n_v, 3)), device=dev)
    q = torch.as_tensor(sc.X + 0.01 * rng.standard_normal(sc.X.shape), device=dev)
    x, out = torch.empty_like(b), torch.empty_like(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for r in range(repeat):
        ev[0].record()
        binding.pd_solve(pd.ctx, b, x)
        ev[1].record()
        binding.pd_local_rhs(pd.ctx, q, out)
        ev[2].record()
        torch.cuda.synchronize()
        print(f"repeat {r}: solve {ev[0].elapsed_time(ev[1]):.3f} ms, local step {ev[1].elapsed_time(ev[2]):.3f} ms")
    print(f"block{n}: {sc.n_e} tets, solve mode {st.solve_mode}, {st.solve_levels} heights, "
          f"{st.factor_nnz} stored entries, factor {st.factor_seconds:.1f} s")
    pd.close()


def run_mlp(repeat, n_block=0):
    dev = "cuda:0"
    rng = np.random.default_rng(3)
    n = 1 << 16
    feat = torch.as_tensor(rng.standard_normal((n, 7)).astype(np.float32), device=dev)
    targ = torch.as_tensor(1e-3 * rng.standard_normal((n, 3)).astype(np.float32), device=dev)
    net = binding.MLP(inputs.mlp_init(0), np.concatenate([np.zeros(7), np.ones(7), np.ones(3)]).astype(np.float32))
    binding.pd_mlp_fit_normalization(net.net, feat, targ, n)
    sc = inputs.large_block(n=n_block, steps=1) if n_block else inputs.hetero_bar(steps=1)
    opt = binding.options_for(sc.solver)
    pd = binding.PDContext(sc, opt)
    for r in range(repeat):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        binding.pd_mlp_train_step(net.net, feat, targ, n, 1e-3, want_loss=False)
        e1.record()
        binding.pd_mlp_load(pd.ctx, net.blob())
        xm = torch.as_tensor(sc.X, device=dev)
        xt = xm + 1e-3
        q0 = torch.empty_like(xm)
        binding.pd_set_warm_start(pd.ctx, 1)
        binding.pd_warm_start(pd.ctx, xt, xm, q0)
        e2.record()
        torch.cuda.synchronize()
        print(f"repeat {r}: train step ({n} samples) {e0.elapsed_time(e1):.3f} ms, warm start + load "
              f"{e1.elapsed_time(e2):.3f} ms")
    pd.close()
    net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="bar", choices=sorted(CASES) + ["block", "mlp"])
    ap.add_argument("--n", type=int, default=None,
                    help="cells per edge of the block (block case: default 48; mlp case: default the bar)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--phases", action="store_true", help="print device phase times of the forward rollout")
    ap.add_argument("--persistent", type=int, default=1)
    ap.add_argument("--solve-fp64", type=int, default=None,
                    help="1: FP64 products with S (the benchmark's headline), 0: double-float; default: the "
                         "workload's setting")
    args = ap.parse_args()
    build()
    if args.case == "block":
        run_block(args.n or 48, args.repeat)
        return
    if args.case == "mlp":
        run_mlp(args.repeat, args.n or 0)
        return
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
        if args.solve_fp64 is not None:
            opt.solve_fp64 = args.solve_fp64
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
