"""Benchmark: forward + backward PD steps/sec on the heterogeneous Neo-Hookean
bar (32x8x8 hex cells -> 10,240 tets, 2,673 vertices, 100x stiffness contrast,
200 implicit-Euler steps at dt = 5 ms, Anderson m = 5, dual gate tightened to
2e-7 (b-change) / 2e-9 (q-step) so that the 200-step trajectory stays within
1e-5 of the oracle's exact fixed points, FP32 local step with FP64
accumulation, FP64 factor and FP64 products with the inverse factor), against
the FP64 CPU oracle. The same rollout with the inverse-factor products in
double-float arithmetic on the FP32 pipe is timed beside it
(``double_float_variant``).

One benchmark step = one full rollout of 200 PD steps forward followed by its
adjoint (200 PD steps backward). value = PD steps (forward+backward) per
second over all ranks. Synthetic seeded inputs; L2 is flushed between timed
rollouts (the bar's working set fits in L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch    # 64 uneven meshes x 100 steps in one launch
  python bench.py --workload block    # 64^3-cell block (1.31M tets), solve mode T, local step alone
  python bench.py --workload warm     # learned warm start: train, then cold / constant-velocity / network

The batch workload (not the default line) times the batched persistent launch:
64 seeded box/ellipsoid meshes of 1k-40k tets (about 0.58M tets in total) with
per-instance materials, 100 steps forward + adjoint per benchmark step, after
the launch-shape autotuner has picked the team sizes; value = instance PD
steps (forward+backward) per second.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd PD steps/sec at <=1e-5 rel err vs FP64 oracle; local-step HBM GB/s vs peak"
UNIT = "PD steps/s"
WORKLOAD = "heterogeneous Neo-Hookean bar 32x8x8 cells (10,240 tets, 2,673 vertices), 200 steps fwd+bwd"



def max_over_ranks(value, dist, device):
    """The largest value over the ranks (a job's time is its slowest rank's);
    the value itself when the job has one rank."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])

# DRAM traffic per launch of the bar's persistent kernels, from one ncu
# capture of this benchmark (dram__bytes_read.sum + dram__bytes_write.sum of
# a full 200-step launch; profiles/bench_traffic_bar32x8x8.md), valid only
# for the kernel sources it was taken with (their hash): reported as null
# once any source under csrc/ has changed since.
BAR_TRAFFIC = {"src": "bf552fcb947edb34", "k_fwd_rollout": 17561600 + 2629376, "k_bwd_rollout": 30860800 + 8891136}


def csrc_hash() -> str:
    """SHA-256 (first 16 hex digits) of every kernel and library source."""
    import hashlib
    d = os.path.join(ROOT, "paper_2605_14526_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str):
    if BAR_TRAFFIC is None or BAR_TRAFFIC.get("src") != csrc_hash():
        return None
    return BAR_TRAFFIC.get(kernel.split()[0])


# FP64 rate derived from the unit counts and the clock: 148 SMs x 2 FP64
# multiply-adds per clock per SM x 2 flops x 2.032 GHz
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


REASONS = ["gpu_idle", "applications_clocks_setting", "sw_power_cap", "hw_slowdown", "sync_boost",
           "sw_thermal_slowdown", "hw_thermal_slowdown", "hw_power_brake_slowdown", "display_clock_setting"]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 3:
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                except ValueError:
                    pass

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [s[0] for s in self.samples]
        mask = 0
        for s in self.samples:
            mask |= s[2]
        reasons = [REASONS[i] for i in range(len(REASONS)) if mask >> i & 1 and REASONS[i] != "gpu_idle"]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(s[1] for s in self.samples), "reasons": reasons,
                "samples": len(sm)}


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                "NUMEXPR_NUM_THREADS")


def single_threaded(fn, *args):
    """fn(*args) in a spawned child process whose BLAS and OpenMP pools have
    one thread (the variables are set before numpy loads there; spawn, not
    fork, since this process may hold a CUDA context). The library's own
    host code in this process keeps its threads."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            return pool.apply(fn, args)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_sample(scene, n_steps: int):
    """The oracle as it stands (exact fixed point + direct adjoint) on the first
    n_steps steps of the workload, single-threaded. Returns (seconds, steps)."""
    return single_threaded(_oracle_sample, scene, n_steps)


def _oracle_sample(scene, n_steps: int):
    from oracle import adjoint, solver
    sc = scene.with_steps(n_steps)
    t0 = time.perf_counter()
    pb = solver.build_problem(sc)
    qT, vT, recs = solver.rollout(pb, sc, mode="exact")
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    adjoint.rollout_backward(pb, recs, dq, dv)
    dt = time.perf_counter() - t0
    return dt, n_steps


GOLD_BAR = os.path.join(ROOT, "tests", "golden", "bar32x8x8_T200.npz")


def oracle_sample_mid(scene, steps=(100, 150), repeats=1):
    """The oracle on one PD step (forward to the exact fixed point + direct
    adjoint) from each of the mid-rollout states t = 100 and t = 150 of the
    bar (the twisting part of the trajectory), read from the oracle's stored
    rollout, `repeats` times; falls back to the first two steps without it.
    Single-threaded, in a child process. Returns a list of (seconds, steps)
    per repeat and a description."""
    gold = np.load(GOLD_BAR) if os.path.exists(GOLD_BAR) else None
    if gold is None or "samples_v" not in gold.files:
        res = [oracle_sample(scene, 2) for _ in range(repeats)]
        return res, "first 2 PD steps of the same rollout, forward (exact fixed point) + adjoint, FP64, 1 thread"
    res, picked = single_threaded(_oracle_sample_mid, scene, tuple(steps), repeats)
    return res, (f"PD steps {picked} of the same rollout (from the oracle's stored states), forward "
                 "(exact fixed point) + adjoint each, FP64, 1 thread")


def _oracle_sample_mid(scene, steps, repeats):
    from oracle import adjoint, solver
    gold = np.load(GOLD_BAR)
    sc = scene.with_steps(1)
    out = []
    picked = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        pb = solver.build_problem(sc)
        picked = []
        for i, t in enumerate(gold["sample_steps"]):
            if int(t) not in steps:
                continue
            picked.append(int(t))
            qT, vT, recs = solver.rollout(pb, sc, mode="exact", x0=gold["samples"][i], v0=gold["samples_v"][i])
            _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
            adjoint.rollout_backward(pb, recs, dq, dv)
        out.append((time.perf_counter() - t0, len(picked)))
    return out, picked


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on the host on a bounded sample
    (one PD step forward + backward per benchmark step)."""
    if rank != 0:
        return
    from paper_2605_14526_b300 import inputs
    scene = inputs.hetero_bar()
    res, what = oracle_sample_mid(scene, steps=(100,), repeats=args.warmup + args.steps)
    res = res[args.warmup:]          # the first repeats are the warm-up
    tot = sum(r[0] for r in res)
    n = sum(r[1] for r in res)
    value = n / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "one PD step of the rollout, forward + adjoint, per bench step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n} PD steps (1 per bench step): {what}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


BATCH_WORKLOAD = ("64 seeded box/ellipsoid Neo-Hookean meshes, 1k-40k tets each (log-uniform), per-instance "
                  "E in [1e4,1e6] x 4^3-block maps in [1,100], nu in [0.3,0.49], 100 steps fwd+bwd, one launch")


def run_batch(args, rank, world, local_rank, dev, dist):
    """Batched workload: all instances in one persistent launch per rollout
    and one per adjoint, launch shape from the autotuner."""
    import torch
    from paper_2605_14526_b300 import binding, inputs

    scenes = inputs.batch_meshes(seed=11 + rank)
    T = scenes[0].steps
    bc = binding.BatchContext(scenes)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x0 = t(bc.concat([s.x0 for s in scenes]).reshape(-1, 3))
    v0 = t(bc.concat([s.v0 for s in scenes]).reshape(-1, 3))
    target = t(bc.concat([s.target for s in scenes]).reshape(-1, 3))
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
    dE = torch.empty(bc.n_e, dtype=torch.float64, device=dev)
    dnu = torch.empty(bc.n, dtype=torch.float64, device=dev)
    zero = torch.zeros_like(x0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def fwd_bwd(timed=False):
        if timed:
            ev[0].record(stream)
        binding.pd_rollout(bc.ctx, T, x0, v0, None, 0, qT, vT, stream)
        if timed:
            ev[1].record(stream)
        binding.pd_backward(bc.ctx, qT - target, zero, dq0, dv0, dE, dnu, None, 0, stream)
        if timed:
            ev[2].record(stream)

    # one full rollout + adjoint measures each instance's iterations per step,
    # which weigh the team sizes; the autotuner then times candidate shapes
    fwd_bwd()
    t0 = time.perf_counter()
    tune = binding.pd_autotune(bc.ctx, 10, x0, v0, None, 0, stream)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    launches0 = binding.pd_get_stats(bc.ctx).launches
    total_ms = fwd_ms = bwd_ms = 0.0
    inst_f = np.zeros(bc.n)
    inst_b = np.zeros(bc.n)
    esc = 0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            fwd_bwd(timed=True)
            torch.cuda.synchronize()
            fwd_ms += ev[0].elapsed_time(ev[1])
            bwd_ms += ev[1].elapsed_time(ev[2])
            total_ms += ev[0].elapsed_time(ev[2])
            for i in range(bc.n):
                si = binding.pd_get_instance_stats(bc.ctx, i)
                inst_f[i] += si.iters_total
                inst_b[i] += si.adj_iters_total
            esc += binding.pd_get_stats(bc.ctx).escalations
    launches = binding.pd_get_stats(bc.ctx).launches - launches0
    tmax = max_over_ranks(total_ms, dist, dev)
    value = world * bc.n * T * args.steps / (tmax / 1e3)
    st = binding.pd_get_stats(bc.ctx)
    m = bc.options.aa_m
    fwd_bytes = bwd_bytes = 0.0
    for i, sc in enumerate(scenes):
        si = binding.pd_get_instance_stats(bc.ctx, i)
        fb = 56 * sc.n_e + 48 * sc.n_v + 20 * si.factor_nnz + 96 * si.n_free + (2 * m + 3) * 24 * sc.n_v
        bb = 200 * sc.n_e + 20 * si.factor_nnz + 240 * sc.n_v
        fwd_bytes += fb * inst_f[i] / args.steps
        bwd_bytes += bb * inst_b[i] / args.steps
    fwd_launch_ms, bwd_launch_ms = fwd_ms / args.steps, bwd_ms / args.steps
    if fwd_launch_ms >= bwd_launch_ms:
        kname, kbytes, kms = "k_fwd_rollout (persistent forward, one team per instance)", fwd_bytes, fwd_launch_ms
    else:
        kname, kbytes, kms = "k_bwd_rollout (persistent adjoint, one team per instance)", bwd_bytes, bwd_launch_ms
    achieved = kbytes / (kms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    tf, tb = bc.teams()

    # end to end with host buffers
    hx0 = bc.concat([s.x0 for s in scenes])
    hv0 = bc.concat([s.v0 for s in scenes])
    htg = bc.concat([s.target for s in scenes])
    hq, hv = np.zeros_like(hx0), np.zeros_like(hx0)
    hdq0, hdv0, hdE, hdnu = np.zeros_like(hx0), np.zeros_like(hx0), np.zeros(bc.n_e), np.zeros(bc.n)
    hz = np.zeros_like(hx0)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.pd_rollout(bc.ctx, T, hx0, hv0, None, 0, hq, hv, None)
        g = np.ascontiguousarray(hq - htg)
        binding.pd_backward(bc.ctx, g, hz, hdq0, hdv0, hdE, hdnu, None, 0, None)
        e2e_s += time.perf_counter() - t0
    e2e = world * bc.n * T * args.steps / e2e_s
    nv3b = 3 * 8 * bc.n_v
    line = {"metric": METRIC, "value": value, "unit": "instance PD steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FP32 local step; FP64 RHS, factor, Anderson, adjoint; S products in double-float on the FP32 pipe)", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances": bc.n, "tets": bc.n_e, "vertices": bc.n_v,
                       "nnz_S": int(st.factor_nnz), "pd_steps_per_instance_per_bench_step": T,
                       "l2": "flushed (256 MB write) between rollouts; inverse factors total "
                             f"{20 * st.factor_nnz / 1e9:.2f} GB per iteration, above L2",
                       "gate": f"b-change {bc.options.eps_res:g}, q-step {bc.options.eps_step:g} (relative)",
                       "autotune": {**tune.as_dict(), "seconds": tune_s},
                       "teams_fwd": [int(x) for x in tf], "teams_bwd": [int(x) for x in tb],
                       "fwd_iters_per_step_mean": float(inst_f.sum() / (args.steps * T * bc.n)),
                       "fwd_iters_per_step_max_instance": float(inst_f.max() / (args.steps * T)),
                       "adj_iters_per_step_mean": float(inst_b.sum() / (args.steps * T * bc.n)),
                       "fp64_escalations_per_rollout": esc / args.steps,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": {"value": e2e, "unit": "instance PD steps/s", "h2d_bytes_per_step": 2 * nv3b + 2 * nv3b,
                    "d2h_bytes_per_step": 2 * nv3b + 2 * nv3b + 8 * bc.n_e + 8 * bc.n},
            "forward": {"value": world * bc.n * T * args.steps / (max_over_ranks(fwd_ms, dist, dev) / 1e3),
                        "unit": "forward instance PD steps/s", "ms_per_rollout": fwd_ms / args.steps},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": kname, "peak_kind": peak_kind, "avg_launch_ms": kms,
                         "bytes_per_launch": kbytes, "fwd_launch_ms": fwd_launch_ms, "bwd_launch_ms": bwd_launch_ms},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        order = np.argsort([s.n_e for s in scenes])
        mid = scenes[order[len(order) // 2]]
        dt, k = oracle_sample(mid, 1)
        line["cpu_baseline"] = {"value": k / dt, "unit": "instance PD steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"first PD step of the median instance ({mid.n_e} tets), forward + adjoint, FP64, 1 thread"}
    if rank == 0:
        print(json.dumps(line))


CONTACT_WORKLOAD = ("contact-rich pad 48x48x12 cells of 1 cm (138,240 tets, 31,213 vertices), stiff core 1e7 / "
                    "shell 1e5 Pa, pressed by a box onto the ground, Coulomb mu 0.5 (2,690 contact candidates), "
                    "dt 2 ms, fwd+bwd")


def run_contact(args, rank, world, local_rank, dev, dist):
    """Contact workload: the first --contact-steps PD steps of the 300-step
    rollout (forward with the contact solves, then its adjoint) per benchmark
    step; the full 300-step rollout takes about 5 minutes on one GPU."""
    import torch
    from paper_2605_14526_b300 import binding, inputs

    sc = inputs.contact_pad(seed=13 + rank)
    T = min(args.contact_steps, sc.steps)
    opts = binding.options_for(sc.solver)
    opts.k_max = 2000
    opts.solve_fp64 = 1   # contact contexts always run FP64 products (the library enforces it)
    t0 = time.perf_counter()
    pd = binding.PDContext(sc, opts)
    factor_s = time.perf_counter() - t0
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x0, v0 = t(sc.x0), t(sc.v0)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
    dE = torch.empty(sc.n_e, dtype=torch.float64, device=dev)
    dnu = torch.empty(1, dtype=torch.float64, device=dev)
    top = torch.as_tensor(sc.loss_vertices, device=dev)
    target = t(sc.target)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def fwd_bwd(timed=False):
        if timed:
            ev[0].record(stream)
        binding.pd_rollout(pd.ctx, T, x0, v0, None, 0, qT, vT, stream)
        if timed:
            ev[1].record(stream)
        dq = torch.zeros_like(x0)
        dq[top] = qT[top] - target[top]
        binding.pd_backward(pd.ctx, dq, None, dq0, dv0, dE, dnu, None, 0, stream)
        if timed:
            ev[2].record(stream)

    for _ in range(args.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    launches0 = binding.pd_get_stats(pd.ctx).launches
    fwd_ms = bwd_ms = 0.0
    it = adj = cpass_f = cpass_b = 0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            fwd_bwd(timed=True)
            torch.cuda.synchronize()
            fwd_ms += ev[0].elapsed_time(ev[1])
            bwd_ms += ev[1].elapsed_time(ev[2])
            st = binding.pd_get_stats(pd.ctx)
            it += st.iters_total
            adj += st.adj_iters_total
            cpass_b += st.contact_iters
    launches = binding.pd_get_stats(pd.ctx).launches - launches0
    tot = max_over_ranks(fwd_ms + bwd_ms, dist, dev)
    value = world * T * args.steps / (tot / 1e3)
    st = binding.pd_get_stats(pd.ctx)
    fwd_iter_bytes = 56 * sc.n_e + 48 * sc.n_v + 20 * st.factor_nnz + 96 * st.n_free + 13 * 24 * sc.n_v
    achieved = fwd_iter_bytes * it / args.steps / (fwd_ms / args.steps * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    line = {"metric": METRIC, "value": value, "unit": "PD steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FP32 local step; FP64 RHS, factor, contact, adjoint" + ("; FP64 S products)" if opts.solve_fp64 else "; S products in double-float on the FP32 pipe)"), "data": "synthetic",
            "config": {"workload": CONTACT_WORKLOAD, "pd_steps_per_bench_step": T,
                       "s_products": "fp64" if opts.solve_fp64 else "double-float",
                       "note": f"first {T} of the configured 300 steps per benchmark step",
                       "factor_and_delassus_s": factor_s, "nnz_S": int(st.factor_nnz),
                       "fwd_iters_per_step": it / (args.steps * T), "adj_iters_per_step": adj / (args.steps * T),
                       "fwd_ms_per_pd_step": fwd_ms / (args.steps * T), "bwd_ms_per_pd_step": bwd_ms / (args.steps * T),
                       "adjoint_contact_cg_passes_per_step": cpass_b / (args.steps * T),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": None,
            "forward": {"value": world * T * args.steps / (max_over_ranks(fwd_ms, dist, dev) / 1e3),
                        "unit": "forward PD steps/s", "ms_per_rollout": fwd_ms / args.steps},
            "gpu_launches": int(launches),
            "roofline": {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_fwd_rollout (persistent forward with contact)",
                         "peak_kind": peak_kind, "note": "algorithmic bytes exclude the contact passes over W"},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))


BLOCK_WORKLOAD = ("large heterogeneous Neo-Hookean block {n}^3 cells ({ne:,} tets, {nv:,} vertices), 8^3-cell blocks "
                  "of 1e4 / 1e6 Pa, bottom pinned, seeded top loads, {T} steps fwd+bwd")


def run_block(args, rank, world, local_rank, dev, dist):
    """Large-block workload: the 64^3-cell block (1.31M tets) whose inverse
    factor is too dense to store, so every A^-1 runs as the level-scheduled
    triangular solves with the factor (solve mode T, FP64); plus the local
    step alone, timed over repeated launches, against the HBM peak."""
    import torch
    from paper_2605_14526_b300 import binding, inputs

    n = args.block_n
    sc = inputs.large_block(n=n, steps=args.block_steps, seed=5 + rank)
    T = sc.steps
    opts = binding.options_for(sc.solver)
    t0 = time.perf_counter()
    pd = binding.PDContext(sc, opts)
    setup_s = time.perf_counter() - t0
    st0 = binding.pd_get_stats(pd.ctx)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x0, v0, f = t(sc.x0), t(sc.v0), t(sc.f_ext)
    stride = 3 * sc.n_v
    target = t(sc.target)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
    dE = torch.empty(sc.n_e, dtype=torch.float64, device=dev)
    dnu = torch.empty(1, dtype=torch.float64, device=dev)
    zero = torch.zeros_like(x0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def fwd_bwd(timed=False):
        if timed:
            ev[0].record(stream)
        binding.pd_rollout(pd.ctx, T, x0, v0, f, stride, qT, vT, stream)
        if timed:
            ev[1].record(stream)
        binding.pd_backward(pd.ctx, qT - target, zero, dq0, dv0, dE, dnu, None, 0, stream)
        if timed:
            ev[2].record(stream)

    for _ in range(args.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    launches0 = binding.pd_get_stats(pd.ctx).launches
    total_ms = fwd_ms = bwd_ms = 0.0
    iters = adj = esc = 0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            fwd_bwd(timed=True)
            torch.cuda.synchronize()
            fwd_ms += ev[0].elapsed_time(ev[1])
            bwd_ms += ev[1].elapsed_time(ev[2])
            total_ms += ev[0].elapsed_time(ev[2])
            st = binding.pd_get_stats(pd.ctx)
            iters += st.iters_total
            adj += st.adj_iters_total
            esc += st.escalations
    launches = binding.pd_get_stats(pd.ctx).launches - launches0
    tmax = max_over_ranks(total_ms, dist, dev)
    value = world * T * args.steps / (tmax / 1e3)
    peak, peak_kind = _peaks()
    st = binding.pd_get_stats(pd.ctx)
    m = pd.options.aa_m
    tmode = st.solve_mode == binding.PD_SOLVE_T
    # algorithmic bytes per iteration: local step 56 B/element + 48 B/vertex;
    # solve 16 B per stored entry in mode T (the row-major copy in the forward
    # sweep, the column-major copy in the backward) or 20 B per non-zero of S;
    # 96 B per free vertex of work vectors; Anderson (2m + 3) x 24 B/vertex
    solve_b = (16 if tmode else 20) * st.factor_nnz
    fwd_iter_bytes = 56 * sc.n_e + 48 * sc.n_v + solve_b + 96 * st.n_free + (2 * m + 3) * 24 * sc.n_v
    bwd_iter_bytes = 200 * sc.n_e + solve_b + 240 * sc.n_v
    fwd_launch_ms, bwd_launch_ms = fwd_ms / args.steps, bwd_ms / args.steps
    fwd_bytes = fwd_iter_bytes * iters / args.steps
    bwd_bytes = bwd_iter_bytes * adj / args.steps
    if fwd_launch_ms >= bwd_launch_ms:
        kname, kbytes, kms, kit = "k_fwd_rollout (persistent forward rollout)", fwd_bytes, fwd_launch_ms, iters
    else:
        kname, kbytes, kms, kit = "k_bwd_rollout (persistent adjoint)", bwd_bytes, bwd_launch_ms, adj
    achieved = kbytes / (kms * 1e-3) / 1e9
    # FP64 work of the solves: 3 right-hand sides x 2 flops per stored entry per sweep, 2 sweeps
    fp64_flops = (12.0 * st.factor_nnz) * kit / args.steps
    # the local step alone: repeated launches at the final state, CUDA events
    # on the launching stream (inputs 1.3M elements: far above L2)
    out = torch.empty_like(x0)
    for _ in range(3):
        binding.pd_local_rhs(pd.ctx, qT, out, stream)
    nrep = 20
    le = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    le[0].record(stream)
    for _ in range(nrep):
        binding.pd_local_rhs(pd.ctx, qT, out, stream)
    le[1].record(stream)
    torch.cuda.synchronize()
    local_ms = le[0].elapsed_time(le[1]) / nrep
    # the same for the corotated model on the same block (its own context;
    # no Newton iterations in the projection: the case the HBM roofline can
    # bind)
    sc_co = sc.replace(model="corotated")
    pd_co = binding.PDContext(sc_co, binding.options_for(sc_co.solver))
    for _ in range(3):
        binding.pd_local_rhs(pd_co.ctx, qT, out, stream)
    torch.cuda.synchronize()
    le[0].record(stream)
    for _ in range(nrep):
        binding.pd_local_rhs(pd_co.ctx, qT, out, stream)
    le[1].record(stream)
    torch.cuda.synchronize()
    local_co_ms = le[0].elapsed_time(le[1]) / nrep
    pd_co.close()
    # local step algorithmic bytes (the minimum the operation must move): per
    # element its corner indices 16, Dm^-1 36 (FP32) and w_e V_e 4 B; per
    # vertex q read 24 B and the right-hand side written 24 B. (The
    # implementation also writes and re-reads the 12 corner forces and the
    # prox stretches; those are not counted.)
    local_bytes = 56 * sc.n_e + 48 * sc.n_v
    local_gbs = local_bytes / (local_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64 (FP32 local step; FP64 RHS, factor, triangular solves, Anderson, adjoint)",
            "data": "synthetic",
            "config": {"workload": BLOCK_WORKLOAD.format(n=n, ne=sc.n_e, nv=sc.n_v, T=T), "pd_steps_per_bench_step": T,
                       "l2": "flushed (256 MB write) between rollouts; the solve streams "
                             f"{solve_b / 1e9:.2f} GB per iteration, far above L2",
                       "gate": f"b-change {pd.options.eps_res:g}, q-step {pd.options.eps_step:g} (relative)",
                       "solve": {"mode": "T (level-scheduled triangular solves with the factor)" if tmode else "S",
                                 "levels": int(st.solve_levels), "stored_entries": int(st.factor_nnz),
                                 "nnz_L": int(st.nnz_L), "setup_s": setup_s,
                                 "factor_s": float(st0.factor_seconds)},
                       "mean_fwd_iters_per_pd_step": iters / (args.steps * T),
                       "mean_adjoint_iters_per_pd_step": adj / (args.steps * T),
                       "fp64_escalations_per_rollout": esc / args.steps,
                       "fwd_ms_per_pd_step": fwd_ms / (args.steps * T), "bwd_ms_per_pd_step": bwd_ms / (args.steps * T),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": None,
            "forward": {"value": world * T * args.steps / (max_over_ranks(fwd_ms, dist, dev) / 1e3),
                        "unit": "forward PD steps/s", "ms_per_rollout": fwd_ms / args.steps},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": fp64_flops / (kms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": fp64_flops / (kms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "traffic": None, "kernel": kname, "avg_launch_ms": kms,
                         "peak_kind": "derived: 148 SMs x 2 FP64 FMA per clock x 2 flops x 2032 MHz",
                         "flops_per_launch": fp64_flops,
                         "note": "FP64 flops of the triangular solves (12 per stored entry and solve) in the "
                                 "dominant launch; the sweeps run 0.75 flop/B, above the FP64 ridge",
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                 "bytes_per_launch": kbytes, "peak_kind": peak_kind},
                         "fwd_launch_ms": fwd_launch_ms, "bwd_launch_ms": bwd_launch_ms,
                         "fwd_iter_bytes": fwd_iter_bytes, "bwd_iter_bytes": bwd_iter_bytes},
            "local_step": {"achieved": local_gbs, "peak": peak, "unit": "GB/s", "frac": local_gbs / peak,
                           "bytes_per_launch": local_bytes, "avg_ms": local_ms, "launches_timed": nrep,
                           "kernels": "k_local_all + k_rhs_out (pd_local_rhs)", "peak_kind": peak_kind,
                           "model": "neohookean (FP32 local step)",
                           "corotated": {"achieved": local_bytes / (local_co_ms * 1e-3) / 1e9,
                                         "frac": local_bytes / (local_co_ms * 1e-3) / 1e9 / peak,
                                         "avg_ms": local_co_ms},
                           "note": "k_local_all is issue-bound (ncu: 66% of issue slots, about 1,480 thread "
                                   "instructions per element for SVD, prox Newton and corner forces), "
                                   "profiles/local_step_block64.md"},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        small = inputs.large_block(n=12, steps=1, seed=5)
        dt, k = oracle_sample(small, 1)
        line["cpu_baseline"] = {"value": k / dt * small.n_e / sc.n_e, "unit": UNIT, "cores": 1,
                                "host_cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"one PD step of a 12^3-cell block ({small.n_e} tets), forward + adjoint, "
                                          "FP64, 1 thread, scaled by element count to the workload (the oracle's "
                                          "sparse LU of the full block does not fit a bounded sample)"}
    if rank == 0:
        print(json.dumps(line))


WARM_WORKLOAD = ("learned warm start: a 7-128-128-128-3 network trained by the library's kernels on about 10k "
                 "plain-solver frames (heterogeneous bars, uneven batched meshes), evaluated on held-out workloads: "
                 "cold start q_t, constant-velocity extrapolation and the network, same gate")


def _frames(binding, torch, ctx, n_v, T, x0, v0, f, stride, keep, dev, feats, targs):
    """Plain-solver rollout of T steps and its training samples (frames 1 .. T-1)."""
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    binding.pd_rollout(ctx, T, x0, v0, f, stride, qT, vT)
    xs = [torch.as_tensor(binding.pd_get_checkpoint(ctx, s, n_v), device=dev) for s in range(T + 1)]
    for s in range(1, T):
        fe = torch.empty((n_v, 7), dtype=torch.float32, device=dev)
        tg = torch.empty((n_v, 3), dtype=torch.float32, device=dev)
        binding.pd_mlp_sample(ctx, xs[s - 1], xs[s], xs[s + 1], fe, tg)
        feats.append(fe[keep])
        targs.append(tg[keep])
    return T - 1


def _warm_compare(binding, torch, ctx, T, x0, v0, f, stride, n_inst, stream, dev):
    """Forward rollouts from the three starts on one context: time, iterations,
    fallbacks and the final state of each."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {}
    for name, mode in (("cold", 0), ("constant_velocity", 2), ("network", 1)):
        binding.pd_set_warm_start(ctx, mode)
        qT, vT = torch.empty_like(x0), torch.empty_like(x0)
        binding.pd_rollout(ctx, T, x0, v0, f, stride, qT, vT, stream)   # untimed (uploads, caches)
        torch.cuda.synchronize()
        ev[0].record(stream)
        binding.pd_rollout(ctx, T, x0, v0, f, stride, qT, vT, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        st = binding.pd_get_stats(ctx)
        ms = ev[0].elapsed_time(ev[1])
        out[name] = {"fwd_pd_steps_per_s": n_inst * T / (ms * 1e-3), "fwd_ms": ms,
                     "iters_per_step": st.iters_total / (T * n_inst), "max_iters_step": int(st.iters_max),
                     "fallbacks": int(st.warm_fallbacks), "fallback_rate": st.warm_fallbacks / (T * n_inst),
                     "not_converged": int(st.not_converged), "qT": qT.clone()}
    ref = out["cold"]["qT"]
    for name in out:
        q = out[name].pop("qT")
        out[name]["qT_rel_diff_vs_cold"] = float((q - ref).norm() / ref.norm())
    binding.pd_set_warm_start(ctx, 0)
    return out


def run_warm(args, rank, world, local_rank, dev, dist):
    """Warm-start workload: train the network on plain-solver frames, then
    time the forward rollout of held-out workloads from the three starts."""
    import torch
    from paper_2605_14526_b300 import binding, inputs

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(100 + rank)
    feats, targs = [], []
    n_frames = 0
    t0 = time.perf_counter()
    for i in range(args.warm_bars):   # heterogeneous bars: other block maps and twist rates than the benchmark's
        sc = inputs.hetero_bar(seed=20 + i, omega0=float(rng.uniform(1.5, 2.5)))
        pd = binding.PDContext(sc)
        keep = torch.as_tensor(sc.pinned == 0, device=dev)
        n_frames += _frames(binding, torch, pd.ctx, sc.n_v, sc.steps, t(sc.x0), t(sc.v0), t(sc.f_ext[0]), 0, keep,
                            dev, feats, targs)
        pd.close()
    scenes = inputs.batch_meshes(seed=1011 + rank)   # batched meshes other than the benchmark batch
    bc = binding.BatchContext(scenes)
    keep = torch.as_tensor(bc.concat([s.pinned for s in scenes]) == 0, device=dev)
    n_frames += len(scenes) * _frames(binding, torch, bc.ctx, bc.n_v, scenes[0].steps,
                                      t(bc.concat([s.x0 for s in scenes]).reshape(-1, 3)),
                                      t(bc.concat([s.v0 for s in scenes]).reshape(-1, 3)), None, 0, keep, dev, feats,
                                      targs)
    bc.close()
    feat = torch.cat(feats).contiguous()
    targ = torch.cat(targs).contiguous()
    del feats, targs
    frames_s = time.perf_counter() - t0
    n = feat.shape[0]
    net = binding.MLP(inputs.mlp_init(0), np.concatenate([np.zeros(7), np.ones(7), np.ones(3)]).astype(np.float32))
    binding.pd_mlp_fit_normalization(net.net, feat, targ, n)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    probe = torch.randint(0, n, (1 << 20,), device=dev, generator=gen)
    fp, tp = feat[probe].contiguous(), targ[probe].contiguous()
    loss0 = binding.pd_mlp_grad(net.net, fp, tp, fp.shape[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.warm_train_steps):
        idx = torch.randint(0, n, (args.warm_batch,), device=dev, generator=gen)
        lr = 1e-3 if it < args.warm_train_steps * 3 // 4 else 2e-4
        binding.pd_mlp_train_step(net.net, feat[idx].contiguous(), targ[idx].contiguous(), args.warm_batch, lr,
                                  want_loss=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    loss1 = binding.pd_mlp_grad(net.net, fp, tp, fp.shape[0])
    blob = net.blob()
    del feat, targ, fp, tp
    # held-out workloads: the benchmark bar, the benchmark batch (one launch,
    # the batched form) and the large block
    res = {}
    sc = inputs.hetero_bar(seed=2 + rank)
    pd = binding.PDContext(sc)
    binding.pd_mlp_load(pd.ctx, blob)
    res["bar32x8x8_T200"] = _warm_compare(binding, torch, pd.ctx, sc.steps, t(sc.x0), t(sc.v0), t(sc.f_ext[0]), 0, 1,
                                          stream, dev)
    if rank == 0:
        gold_path = os.path.join(ROOT, "tests", "golden", "bar32x8x8_T200.npz")
        if os.path.exists(gold_path):
            gold = np.load(gold_path)
            for name, mode in (("cold", 0), ("network", 1)):
                binding.pd_set_warm_start(pd.ctx, mode)
                x0 = t(sc.x0)
                qT, vT = torch.empty_like(x0), torch.empty_like(x0)
                binding.pd_rollout(pd.ctx, sc.steps, x0, t(sc.v0), t(sc.f_ext[0]), 0, qT, vT, stream)
                q = qT.cpu().numpy()
                res["bar32x8x8_T200"][name]["qT_rel_err_vs_oracle"] = float(
                    max(np.linalg.norm(q - gold["qT"]) / np.linalg.norm(gold["qT"]),
                        np.abs(q - gold["qT"]).max() / np.abs(gold["qT"]).max()))
            binding.pd_set_warm_start(pd.ctx, 0)
    pd.close()
    scenes = inputs.batch_meshes(seed=11 + rank)
    bc = binding.BatchContext(scenes)
    binding.pd_mlp_load(bc.ctx, blob)
    bx0 = t(bc.concat([s.x0 for s in scenes]).reshape(-1, 3))
    bv0 = t(bc.concat([s.v0 for s in scenes]).reshape(-1, 3))
    # the launch shape as the batch benchmark picks it: one cold rollout
    # measures each instance's iterations, then the autotuner
    bq, bv = torch.empty_like(bx0), torch.empty_like(bx0)
    binding.pd_rollout(bc.ctx, scenes[0].steps, bx0, bv0, None, 0, bq, bv, stream)
    binding.pd_autotune(bc.ctx, 10, bx0, bv0, None, 0, stream)
    res["batch64_T100"] = _warm_compare(binding, torch, bc.ctx, scenes[0].steps, bx0, bv0, None, 0, len(scenes),
                                        stream, dev)
    bc.close()
    if args.block_n > 0:
        sb = inputs.large_block(n=args.block_n, steps=args.block_steps, seed=5 + rank)
        pd = binding.PDContext(sb)
        binding.pd_mlp_load(pd.ctx, blob)
        res[f"block{args.block_n}_T{sb.steps}"] = _warm_compare(binding, torch, pd.ctx, sb.steps, t(sb.x0), t(sb.v0),
                                                                t(sb.f_ext), 3 * sb.n_v, 1, stream, dev)
        pd.close()
    head = res["batch64_T100"]
    value = world * head["network"]["fwd_pd_steps_per_s"]
    line = {"metric": METRIC, "value": value, "unit": "instance PD steps/s (forward, network warm start)",
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": head["network"]["fwd_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FP32 local step; FP64 RHS, factor, Anderson; network BF16 weights, FP32 activations, "
                     "FP32 accumulation on the tensor pipe)",
            "data": "synthetic",
            "config": {"workload": WARM_WORKLOAD, "training_frames": n_frames, "training_samples": int(n),
                       "frames_s": frames_s, "train_steps": args.warm_train_steps, "train_batch": args.warm_batch,
                       "train_s": train_s, "loss_before": loss0, "loss_after": loss1,
                       "gate": "each workload's configured gate, the same for the three starts",
                       "results": res,
                       "network_vs_cold_speedup": {k: v["network"]["fwd_pd_steps_per_s"] / v["cold"]["fwd_pd_steps_per_s"]
                                                   for k, v in res.items()},
                       "network_vs_constant_velocity_speedup": {
                           k: v["network"]["fwd_pd_steps_per_s"] / v["constant_velocity"]["fwd_pd_steps_per_s"]
                           for k, v in res.items()},
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="bar", choices=["bar", "batch", "contact", "block", "warm"])
    ap.add_argument("--warm-bars", type=int, default=18, help="warm workload: training bars (200 frames each)")
    ap.add_argument("--warm-train-steps", type=int, default=3000)
    ap.add_argument("--warm-batch", type=int, default=16384)
    ap.add_argument("--block-n", type=int, default=64, help="block workload: cells per edge")
    ap.add_argument("--block-steps", type=int, default=10, help="block workload: PD steps per rollout")
    ap.add_argument("--contact-steps", type=int, default=20,
                    help="contact workload: PD steps of the 300-step rollout timed per benchmark step")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2605_14526_b300 import binding, inputs
    from paper_2605_14526_b300.build import build

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build()
    dev = torch.device("cuda", local_rank)
    if args.workload == "contact":
        run_contact(args, rank, world, local_rank, dev, dist)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "warm":
        run_warm(args, rank, world, local_rank, dev, dist)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "block":
        run_block(args, rank, world, local_rank, dev, dist)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local_rank, dev, dist)
        if dist:
            dist.destroy_process_group()
        return
    scene = inputs.hetero_bar(seed=2 + rank)
    T = scene.steps
    # the headline keeps the solve in FP64 (the factor and the products with
    # the inverse factor)
    opts = binding.options_for(scene.solver)
    opts.solve_fp64 = 1
    pd = binding.PDContext(scene, opts)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x0, v0, f0, target = t(scene.x0), t(scene.v0), t(scene.f_ext[0]), t(scene.target)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
    dE = torch.empty(scene.n_e, dtype=torch.float64, device=dev)
    dnu = torch.empty(1, dtype=torch.float64, device=dev)
    zero = torch.zeros_like(x0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream(dev)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def fwd_bwd(timed=False):
        if timed:
            ev[0].record(stream)
        binding.pd_rollout(pd.ctx, T, x0, v0, f0, 0, qT, vT, stream)
        if timed:
            ev[1].record(stream)
        binding.pd_backward(pd.ctx, qT - target, zero, dq0, dv0, dE, dnu, None, 0, stream)
        if timed:
            ev[2].record(stream)

    for _ in range(args.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    launches0 = binding.pd_get_stats(pd.ctx).launches
    total_ms = fwd_ms = bwd_ms = 0.0
    iters = adj = 0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            fwd_bwd(timed=True)
            torch.cuda.synchronize()
            fwd_ms += ev[0].elapsed_time(ev[1])
            bwd_ms += ev[1].elapsed_time(ev[2])
            total_ms += ev[0].elapsed_time(ev[2])
            st = binding.pd_get_stats(pd.ctx)
            iters += st.iters_total
            adj += st.adj_iters_total
    launches = binding.pd_get_stats(pd.ctx).launches - launches0
    tmax = max_over_ranks(total_ms, dist, dev)
    value = world * T * args.steps / (tmax / 1e3)
    qT_timed_t = qT.clone()
    qT_timed, dE_timed, dq0_timed, dv0_timed = (a.cpu().numpy() for a in (qT, dE, dq0, dv0))

    # Roofline of the dominant kernel. Each rollout is one launch of the
    # persistent forward kernel and one of the persistent adjoint kernel; the
    # CUDA events above bracket them on the work stream. Algorithmic bytes per
    # launch = iterations x bytes per iteration:
    #   forward iteration: local step 56 B/element (indices, Dm^-1, w V) + 48 B/vertex
    #     (q in, b out); solve 20 B per nnz(S) (skyline values + S^T values and
    #     indices) + 96 B per free vertex (b, y, y, q_hat); Anderson (2m+3) x 24 B/vertex
    #   adjoint iteration: element record 144 B + 56 B per element, 20 B per nnz(S),
    #     10 vectors x 24 B per vertex
    st = binding.pd_get_stats(pd.ctx)
    nnzS = st.factor_nnz
    m = pd.options.aa_m
    fwd_iter_bytes = 56 * scene.n_e + 48 * scene.n_v + 20 * nnzS + 96 * st.n_free + (2 * m + 3) * 24 * scene.n_v
    bwd_iter_bytes = 200 * scene.n_e + 20 * nnzS + 240 * scene.n_v
    fwd_bytes = fwd_iter_bytes * iters / args.steps
    bwd_bytes = bwd_iter_bytes * adj / args.steps
    peak, peak_kind = _peaks()
    fwd_launch_ms, bwd_launch_ms = fwd_ms / args.steps, bwd_ms / args.steps
    if fwd_launch_ms >= bwd_launch_ms:
        kname, kbytes, kms = "k_fwd_rollout (persistent forward rollout)", fwd_bytes, fwd_launch_ms
    else:
        kname, kbytes, kms = "k_bwd_rollout (persistent adjoint)", bwd_bytes, bwd_launch_ms
    achieved = kbytes / (kms * 1e-3) / 1e9

    # device phase breakdown of one forward rollout (globaltimer, block 0)
    binding.pd_profile(pd.ctx, True)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    binding.pd_rollout(pd.ctx, T, x0, v0, f0, 0, qT, vT, stream)
    torch.cuda.synchronize()
    prof = binding.pd_get_profile(pd.ctx)
    prof_iters = binding.pd_get_stats(pd.ctx).iters_total
    binding.pd_profile(pd.ctx, False)
    # local step alone (the metric's second half): its algorithmic bytes per
    # iteration (tet indices 16, Dm^-1 36, w V 4, corner forces 48, prox
    # warm-start stretches 12 + 12 B per element; q 24 B per vertex) over the
    # local phase's time in the profiled rollout (block 0's globaltimer, from
    # the phase start through its closing team barrier)
    local_bytes = 128 * scene.n_e + 24 * scene.n_v
    local_s = prof.phase_ms[1] * 1e-3
    local_gbs = local_bytes * prof_iters / local_s / 1e9 if local_s > 0 else None
    local_step = {"achieved": local_gbs, "peak": _peaks()[0], "unit": "GB/s",
                  "frac": local_gbs / _peaks()[0] if local_gbs else None, "bytes_per_iter": local_bytes,
                  "iters": prof_iters, "phase_ms": prof.phase_ms[1],
                  "note": "bar working set is L2-resident: latency-bound, not the HBM case"}
    phase_names = ["begin", "local", "assemble_gate", "spmv_s", "spmv_st_anderson_dots", "anderson_solve", "update", "end_tr"]
    phases = {n: round(prof.phase_ms[i], 3) for i, n in enumerate(phase_names) if prof.phase_ms[i] > 0}

    # end to end through the C ABI with host buffers (copies inside the region)
    hx0, hv0, hf0 = (np.ascontiguousarray(a) for a in (scene.x0, scene.v0, scene.f_ext[0]))
    hq, hv = np.zeros_like(hx0), np.zeros_like(hx0)
    hdq0, hdv0, hdE, hdnu = np.zeros_like(hx0), np.zeros_like(hx0), np.zeros(scene.n_e), np.zeros(1)
    hz = np.zeros_like(hx0)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.pd_rollout(pd.ctx, T, hx0, hv0, hf0, 0, hq, hv, None)
        g = np.ascontiguousarray(hq - scene.target)
        binding.pd_backward(pd.ctx, g, hz, hdq0, hdv0, hdE, hdnu, None, 0, None)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e = world * T * args.steps / e2e_s
    # accuracy of the timed run (rank 0's seed): the last timed rollout and
    # adjoint against the oracle's stored exact-fixed-point rollout
    accuracy = None
    gold_path = os.path.join(ROOT, "tests", "golden", "bar32x8x8_T200.npz")
    if rank == 0 and os.path.exists(gold_path):
        gold = np.load(gold_path)
        def _rel_norm(a, b):
            a, b = np.asarray(a), np.asarray(b)
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))

        def _rel_max(a, b):
            a, b = np.asarray(a), np.asarray(b)
            return float(np.abs(a - b).max() / np.abs(b).max())

        def _rel(a, b):
            return max(_rel_norm(a, b), _rel_max(a, b))
        accuracy = {"positions_qT": _rel(qT_timed, gold["qT"]), "dL_dE": _rel(dE_timed, gold["dE"]),
                    "dL_dx0": _rel(dq0_timed, gold["dq0"]), "dL_dv0": _rel(dv0_timed, gold["dv0"]),
                    "positions_qT_norm": _rel_norm(qT_timed, gold["qT"]),
                    "positions_qT_max_entry": _rel_max(qT_timed, gold["qT"]),
                    "metric": "max(||a-b||/||b||, max|a-b|/max|b|) of the last timed rollout + adjoint against "
                              "tests/golden/bar32x8x8_T200.npz (oracle, exact fixed point per step); the two "
                              "terms for the positions separately"}
    # the same rollout with the S products in double-float arithmetic on the
    # FP32 pipe (options.solve_fp64 = 0): one untimed and one timed fwd+bwd
    odf = binding.options_for(scene.solver)
    odf.solve_fp64 = 0
    pddf = binding.PDContext(scene, odf)
    qdf, vdf = torch.empty_like(x0), torch.empty_like(x0)
    for timed in (False, True):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev[0].record(stream)
        binding.pd_rollout(pddf.ctx, T, x0, v0, f0, 0, qdf, vdf, stream)
        ev[1].record(stream)
        binding.pd_backward(pddf.ctx, qdf - target, zero, dq0, dv0, dE, dnu, None, 0, stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
    stdf = binding.pd_get_stats(pddf.ctx)
    df_variant = {"pd_steps_per_s": T / (ev[0].elapsed_time(ev[2]) / 1e3),
                  "fwd_ms": ev[0].elapsed_time(ev[1]), "bwd_ms": ev[1].elapsed_time(ev[2]),
                  "fwd_iters_per_pd_step": stdf.iters_total / T, "adj_iters_per_pd_step": stdf.adj_iters_total / T,
                  "qT_rel_diff_vs_headline": float((qdf - qT_timed_t).norm() / qT_timed_t.norm()),
                  "note": "S and S^T products in double-float (about 2^-44 relative) instead of FP64"}
    del pddf
    # the same rollout with an FP64 local step at the gate 3e-8 / 3e-10, which
    # meets 1e-5 entry by entry as well (FP32's rounding floor keeps the FP32
    # local step from gating that tightly): one untimed and one timed fwd+bwd
    s64 = scene.replace(solver=dataclasses.replace(scene.solver, local_fp32=False, eps_res=3e-8, eps_step=3e-10))
    pd64 = binding.PDContext(s64, binding.options_for(s64.solver))
    q64, v64 = torch.empty_like(x0), torch.empty_like(x0)
    for timed in (False, True):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev[0].record(stream)
        binding.pd_rollout(pd64.ctx, T, x0, v0, f0, 0, q64, v64, stream)
        ev[1].record(stream)
        binding.pd_backward(pd64.ctx, q64 - target, zero, dq0, dv0, dE, dnu, None, 0, stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
    st64 = binding.pd_get_stats(pd64.ctx)
    fp64_variant = {"pd_steps_per_s": T / (ev[0].elapsed_time(ev[2]) / 1e3),
                    "fwd_ms": ev[0].elapsed_time(ev[1]), "bwd_ms": ev[1].elapsed_time(ev[2]),
                    "fwd_iters_per_pd_step": st64.iters_total / T,
                    "adj_iters_per_pd_step": st64.adj_iters_total / T,
                    "gate": "b-change 3e-8, q-step 3e-10 (relative)",
                    "note": "FP64 local step and FP64 S products"}
    if accuracy is not None:
        q64h, dE64, dq064, dv064 = (a.cpu().numpy() for a in (q64, dE, dq0, dv0))
        fp64_variant["accuracy_vs_oracle"] = {
            "positions_qT_norm": _rel_norm(q64h, gold["qT"]), "positions_qT_max_entry": _rel_max(q64h, gold["qT"]),
            "dL_dE": _rel(dE64, gold["dE"]), "dL_dx0": _rel(dq064, gold["dq0"]), "dL_dv0": _rel(dv064, gold["dv0"])}
    del pd64

    nv3b = 3 * 8 * scene.n_v
    h2d = 3 * nv3b + 2 * nv3b          # x0, v0, f_ext; dL/dq_T, dL/dv_T
    d2h = 2 * nv3b + 2 * nv3b + 8 * scene.n_e + 8

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FP32 local step; FP64 RHS, factor, S products, Anderson, adjoint)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pd_steps_per_bench_step": T, "l2": "flushed (256 MB write) between rollouts",
                       "gate": f"b-change {pd.options.eps_res:g}, q-step {pd.options.eps_step:g} (relative)",
                       "solve": "FP64 factor, FP64 products with the inverse factor",
                       "accuracy_vs_oracle": accuracy,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "mean_fwd_iters_per_pd_step": iters / (args.steps * T),
                       "mean_adjoint_iters_per_pd_step": adj / (args.steps * T)},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "forward": {"value": world * T * args.steps / (max_over_ranks(fwd_ms, dist, dev) / 1e3),
                        "unit": "forward PD steps/s", "ms_per_rollout": fwd_ms / args.steps},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": measured_traffic(kname), "kernel": kname,
                         "peak_kind": peak_kind,
                         "avg_launch_ms": kms, "bytes_per_launch": kbytes,
                         "fwd_launch_ms": fwd_launch_ms, "bwd_launch_ms": bwd_launch_ms,
                         "fwd_iter_bytes": fwd_iter_bytes, "bwd_iter_bytes": bwd_iter_bytes},
            "forward_phase_ms_one_rollout": phases,
            "local_step": local_step,
            "double_float_variant": df_variant,
            "fp64_local_variant": fp64_variant,
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res, what = oracle_sample_mid(scene)
        dt, k = res[0]
        line["cpu_baseline"] = {"value": k / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                                "kind": "oracle", "sample": what}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
