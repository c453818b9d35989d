"""Shared helpers of the GPU parity tests: run a workload through the C ABI
and through the oracle, and compare."""
import numpy as np
import torch

from oracle import adjoint, solver
from paper_2605_14526_b300 import binding
from paper_2605_14526_b300.build import build

DEV = "cuda:0"


def gpu_run(scene, options=None, backward=True, persistent=1):
    """Forward (and backward) of a workload through the library; device buffers."""
    build()
    if options is None:
        options = binding.options_for(scene.solver)
    options.persistent = persistent
    pd = binding.PDContext(scene, options)
    T = scene.steps
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    x0, v0 = t(scene.x0), t(scene.v0)
    f = t(scene.f_ext if scene.f_ext.shape[0] > 1 else scene.f_ext[0])
    stride = 3 * scene.n_v if scene.f_ext.shape[0] > 1 else 0
    qT = torch.empty_like(x0)
    vT = torch.empty_like(x0)
    binding.pd_rollout(pd.ctx, T, x0, v0, f, stride, qT, vT)
    out = {"qT": qT.cpu().numpy(), "vT": vT.cpu().numpy(), "stats": binding.pd_get_stats(pd.ctx),
           "tau": binding.pd_get_tau(pd.ctx, T), "pd": pd}
    if backward:
        mass = pd.mass()
        if scene.loss == "com_z":
            dq = np.zeros_like(out["qT"])
            dq[:, 2] = mass / mass.sum()
        else:
            dq = out["qT"] - scene.target
        dq0, dv0 = torch.empty_like(x0), torch.empty_like(x0)
        dE = torch.empty(scene.n_e, dtype=torch.float64, device=DEV)
        dnu = torch.empty(1, dtype=torch.float64, device=DEV)
        df = torch.empty((T, scene.n_v, 3) if stride else (scene.n_v, 3), dtype=torch.float64, device=DEV)
        binding.pd_backward(pd.ctx, t(dq), torch.zeros_like(x0), dq0, dv0, dE, dnu, df, stride)
        out.update(dq0=dq0.cpu().numpy(), dv0=dv0.cpu().numpy(), dE=dE.cpu().numpy(), dnu=float(dnu[0]),
                   df=df.cpu().numpy(), stats=binding.pd_get_stats(pd.ctx))
    return out


def oracle_run(scene, mode=None, backward=True):
    pb = solver.build_problem(scene)
    mode = mode or solver.mode_for(scene)
    qT, vT, recs = solver.rollout(pb, scene, mode=mode)
    out = {"qT": qT, "vT": vT, "recs": recs, "pb": pb}
    if backward:
        _, dq, dv = adjoint.loss_and_grad(scene, pb, qT, vT)
        g = adjoint.rollout_backward(pb, recs, dq, dv)
        out.update(dq0=g.dx0, dv0=g.dv0, dE=g.dE, dnu=g.dnu, df=g.df_ext)
    return out


def rel_norm(a, b):
    """Global relative error ||a - b||_2 / ||b||_2."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    """Entry-wise error against the largest entry: max |a - b| / max |b|
    (a few bad entries, e.g. on the soft half of a bar or at contact
    vertices, show here even when the global norm hides them)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


def rel(a, b):
    """The parity metric every GPU test asserts: the larger of the global
    relative error and the entry-wise error against the largest entry."""
    return max(rel_norm(a, b), rel_max(a, b))


def elem_rel(a, b, floor=1e-2):
    """Per-entry relative error max_i |a_i - b_i| / max(|b_i|, floor max|b|):
    each entry against its own size, entries smaller than floor x the largest
    against that floor (a per-element gradient near a sign change has no
    meaningful relative error of its own)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.maximum(np.abs(b), floor * max(np.abs(b).max(initial=0.0), 1e-300))
    return float((np.abs(a - b) / den).max(initial=0.0))
