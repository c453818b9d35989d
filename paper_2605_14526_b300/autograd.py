"""``torch.autograd.Function`` over pd_rollout / pd_backward.

forward(E, nu, x0, v0, f_ext) runs T implicit-Euler PD steps in the library
(checkpointing q_t per step on the device); backward calls the library's
adjoint, which recomputes the local state at each checkpoint, and returns
dL/dE, dL/dnu, dL/dx0, dL/dv0 and dL/df_ext. PyTorch only provides device
memory and the stream here. The same Function serves a batch of independent
meshes (``binding.BatchContext``): then every array is the concatenation over
instances and ``nu`` holds one Poisson ratio per instance.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, nu, x0, v0, f_ext, pd, T: int):
        E_h = E.detach().double().cpu().numpy()
        nu_h = np.atleast_1d(nu.detach().double().cpu().numpy() if isinstance(nu, torch.Tensor)
                             else np.asarray(nu, dtype=np.float64))
        pd.ensure_materials(E_h, nu_h)
        dev = x0.device
        qT = torch.empty_like(x0)
        vT = torch.empty_like(x0)
        f = f_ext.contiguous()
        stride = 0 if f.dim() == 2 else 3 * pd.n_v
        stream = torch.cuda.current_stream(dev) if dev.type == "cuda" else None
        binding.pd_rollout(pd.ctx, T, x0.contiguous(), v0.contiguous(), f, stride, qT, vT, stream)
        ctx.pd = pd
        ctx.stride = stride
        ctx.f_shape = f.shape
        ctx.nu_is_tensor = isinstance(nu, torch.Tensor)
        ctx.nu_shape = nu.shape if ctx.nu_is_tensor else None
        ctx.E_device = E.device
        return qT, vT

    @staticmethod
    def backward(ctx, gq, gv):
        pd = ctx.pd
        dev = gq.device
        dq0 = torch.empty_like(gq)
        dv0 = torch.empty_like(gq)
        dE = torch.empty(pd.n_e, dtype=torch.float64, device=dev)
        dnu = torch.empty(getattr(pd, "n", 1), dtype=torch.float64, device=dev)
        df = torch.empty(ctx.f_shape, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev) if dev.type == "cuda" else None
        gv = torch.zeros_like(gq) if gv is None else gv.contiguous()
        binding.pd_backward(pd.ctx, gq.contiguous(), gv, dq0, dv0, dE, dnu, df, ctx.stride, stream)
        dnu_out = dnu.reshape(ctx.nu_shape).to(ctx.E_device) if ctx.nu_is_tensor else None
        return (dE.to(ctx.E_device), dnu_out, dq0, dv0, df, None, None)


def rollout(E, nu, x0, v0, f_ext, pd, T: int):
    return Rollout.apply(E, nu, x0, v0, f_ext, pd, T)
