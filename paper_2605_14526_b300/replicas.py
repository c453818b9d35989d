"""Independent instances split across GPUs (one process per GPU): the
batched workload's only parallel axis. A single mesh does not shard (the
factor couples every DoF through the top separators), but a batch of
independent meshes does, by instance, with no exchange on the data path;
the one collective gathers the per-instance losses and gradients after the
adjoint (torch.distributed: NCCL on GPUs, gloo on CPU).

  share = shard_instances([s.n_e for s in scenes], world)[rank]
  sb = ShardedBatch(scenes, share)            # this rank's BatchContext
  out = sb.rollout_and_adjoint()              # this rank's instances
  full = gather_instances(share, out, len(scenes), dist)
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_instances(costs, world: int) -> list[list[int]]:
    """Split instances 0..n-1 over `world` ranks by predicted cost (element
    counts, or measured times): longest first, each to the rank with the
    smallest total so far (ties to the lower rank; the greedy LPT rule of
    Graham 1969, within 4/3 of the best makespan). Every rank's list is in
    ascending instance order; a rank may get none when n < world."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(costs.size), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    share = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        share[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in share]


def gather_instances(share, results: dict, n_total: int, dist=None) -> dict:
    """results: name -> list of per-instance host arrays (or scalars) in the
    order of `share`. Returns name -> list over all n_total instances in
    instance order, on every rank (one all_gather_object; without a process
    group the local results must already cover every instance)."""
    local = {"share": list(share), "results": {k: list(v) for k, v in results.items()}}
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
    else:
        parts = [local]
    names = sorted(results)
    out = {k: [None] * n_total for k in names}
    seen = np.zeros(n_total, dtype=np.int64)
    for p in parts:
        if sorted(p["results"]) != names:
            raise ValueError("ranks gathered different result names")
        for j, i in enumerate(p["share"]):
            seen[i] += 1
            for k in names:
                out[k][i] = p["results"][k][j]
    if not np.all(seen == 1):
        raise ValueError("the shares do not cover every instance exactly once")
    return out


class ShardedBatch:
    """One rank's share of a batch of independent instances, run as one
    batched context on this rank's GPU (all its instances in one persistent
    launch per rollout and per adjoint). The loss of instance i is
    0.5 ||x_T,i - x*_i||^2."""

    def __init__(self, scenes, share, options=None, device="cuda:0"):
        import torch

        from . import binding
        self.share = list(share)
        self.scenes = [scenes[i] for i in self.share]
        self.device = device
        self.bc = binding.BatchContext(self.scenes, options) if self.scenes else None
        if self.bc is None:
            return
        bc = self.bc
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
        self.x0 = t(bc.concat([s.x0 for s in self.scenes]).reshape(-1, 3))
        self.v0 = t(bc.concat([s.v0 for s in self.scenes]).reshape(-1, 3))
        self.target = t(bc.concat([s.target for s in self.scenes]).reshape(-1, 3))
        self.qT, self.vT = torch.empty_like(self.x0), torch.empty_like(self.x0)
        self.dq0, self.dv0 = torch.empty_like(self.x0), torch.empty_like(self.x0)
        self.dE = torch.empty(bc.n_e, dtype=torch.float64, device=device)
        self.dnu = torch.empty(bc.n, dtype=torch.float64, device=device)
        self.zero = torch.zeros_like(self.x0)

    def close(self):
        if self.bc is not None:
            self.bc.close()
            self.bc = None

    def rollout_and_adjoint(self, stream=None) -> dict:
        """Per instance of the share: loss, x_T, dL/dx0, dL/dv0, dL/dE,
        dL/dnu (host arrays, in share order)."""
        from . import binding
        out = {k: [] for k in ("loss", "qT", "dq0", "dv0", "dE", "dnu")}
        if self.bc is None:
            return out
        bc = self.bc
        T = self.scenes[0].steps
        binding.pd_rollout(bc.ctx, T, self.x0, self.v0, None, 0, self.qT, self.vT, stream)
        diff = (self.qT - self.target).contiguous()
        binding.pd_backward(bc.ctx, diff, self.zero, self.dq0, self.dv0, self.dE, self.dnu, None, 0, stream)
        d = diff.cpu().numpy()
        q, dq0, dv0 = self.qT.cpu().numpy(), self.dq0.cpu().numpy(), self.dv0.cpu().numpy()
        dE, dnu = self.dE.cpu().numpy(), self.dnu.cpu().numpy()
        for j in range(bc.n):
            v = slice(int(bc.v_off[j]), int(bc.v_off[j + 1]))
            e = slice(int(bc.e_off[j]), int(bc.e_off[j + 1]))
            out["loss"].append(0.5 * float(np.sum(d[v] ** 2)))
            out["qT"].append(q[v].copy())
            out["dq0"].append(dq0[v].copy())
            out["dv0"].append(dv0[v].copy())
            out["dE"].append(dE[e].copy())
            out["dnu"].append(float(dnu[j]))
        return out
