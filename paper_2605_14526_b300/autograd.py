"""``torch.autograd.Function`` over pd_rollout / pd_backward.

forward(E, nu, x0, v0, f_ext) runs T implicit-Euler PD steps in the library
(checkpointing q_t per step on the device); backward calls the library's
adjoint, which recomputes the local state at each checkpoint, and returns
dL/dE, dL/dnu, dL/dx0, dL/dv0 and dL/df_ext. PyTorch only provides device
memory and the stream here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, nu, x0, v0, f_ext, pd: binding.PDContext, T: int):
        E_h = E.detach().double().cpu().numpy()
        nu_f = float(nu.detach().cpu()) if isinstance(nu, torch.Tensor) else float(nu)
        if not (np.array_equal(E_h, pd.scene.E) and nu_f == pd.scene.nu):
            pd.set_materials(E_h, nu_f)
            pd.scene = pd.scene.replace(E=E_h.copy(), nu=nu_f)
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
        ctx.E_device = E.device
        return qT, vT

    @staticmethod
    def backward(ctx, gq, gv):
        pd = ctx.pd
        dev = gq.device
        dq0 = torch.empty_like(gq)
        dv0 = torch.empty_like(gq)
        dE = torch.empty(pd.n_e, dtype=torch.float64, device=dev)
        dnu = torch.empty(1, dtype=torch.float64, device=dev)
        df = torch.empty(ctx.f_shape, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev) if dev.type == "cuda" else None
        gv = torch.zeros_like(gq) if gv is None else gv.contiguous()
        binding.pd_backward(pd.ctx, gq.contiguous(), gv, dq0, dv0, dE, dnu, df, ctx.stride, stream)
        return (dE.to(ctx.E_device), dnu[0] if ctx.nu_is_tensor else None, dq0, dv0, df, None, None)


def rollout(E, nu, x0, v0, f_ext, pd: binding.PDContext, T: int):
    return Rollout.apply(E, nu, x0, v0, f_ext, pd, T)
