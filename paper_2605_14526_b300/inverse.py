"""Inverse problems on the library's rollout and adjoint: the paper's task
classes of Sec. 5.4 / 5.5 (system identification of per-region Young's
moduli, initial-state optimisation), driven by the library's L-BFGS
(pd_lbfgs_*, Nocedal and Wright 2006, Alg. 7.4 with a strong-Wolfe line
search). Every evaluation is one pd_rollout and one pd_backward on the
device (after pd_set_materials + pd_factor when the moduli change); this
module only moves the parameter vector between the optimiser and the
library and applies the parametrisation's chain rule.

  sysid = BlockSysID(scene, block_of_element, target_qT)
  res = lbfgs(sysid, theta0)            # theta = log10 of each block's E
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding

DEV = "cuda:0"


def lbfgs(fun, x0, options: binding.pd_lbfgs_options | None = None, callback=None):
    """Minimise fun(x) -> (f, g) (host float64 vectors) with the library's
    L-BFGS. Returns a dict: x, f, status ('converged', 'stop', 'failed'),
    iters, evals, the evaluated points and the accepted iterates."""
    x = np.array(x0, dtype=np.float64)
    f, g = fun(x)
    points, iterates = [x.copy()], [x.copy()]
    opt = binding.pd_lbfgs_create(x.size, options)
    try:
        task = binding.pd_lbfgs_next(opt, x, f, np.ascontiguousarray(g, dtype=np.float64))
        while True:
            if task == binding.PD_LBFGS_EVAL:
                f, g = fun(x)
                points.append(x.copy())
                task = binding.pd_lbfgs_next(opt, x, f, np.ascontiguousarray(g, dtype=np.float64))
            elif task == binding.PD_LBFGS_ITERATE:
                iterates.append(x.copy())
                if callback is not None:
                    callback(x, f)
                task = binding.pd_lbfgs_next(opt, x, 0.0, None)
            else:
                break
        info = binding.pd_lbfgs_info(opt)
    finally:
        binding.pd_lbfgs_destroy(opt)
    if info["iters"] > len(iterates) - 1:   # the last accepted iterate ended the run
        iterates.append(x.copy())
    return {"x": x, "f": info["f"], "status": binding.LBFGS_TASKS[task], "iters": info["iters"],
            "evals": info["evals"], "gmax": info["gmax"], "points": points, "iterates": iterates}


class _Rollout:
    """A context plus device copies of a scene's initial state and forces."""

    def __init__(self, scene, options=None):
        self.scene = scene
        self.pd = binding.PDContext(scene, options)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
        self.t = t
        self.x0, self.v0 = t(scene.x0), t(scene.v0)
        per_step = scene.f_ext.shape[0] > 1
        self.f = t(scene.f_ext if per_step else scene.f_ext[0])
        self.stride = 3 * scene.n_v if per_step else 0
        self.qT = torch.empty_like(self.x0)
        self.vT = torch.empty_like(self.x0)
        self.evals = 0

    def close(self):
        self.pd.close()

    def run(self, x0=None, v0=None):
        binding.pd_rollout(self.pd.ctx, self.scene.steps, self.x0 if x0 is None else x0,
                           self.v0 if v0 is None else v0, self.f, self.stride, self.qT, self.vT)
        self.evals += 1


class BlockSysID(_Rollout):
    """System identification of per-block Young's moduli (Sec. 5.4): theta_b
    = log10 E_b, E_e = 10^theta_{block(e)}; loss 0.5 ||x_T(theta) - x*||^2
    over all vertices (pinned ones do not move). dL/dtheta_b = sum over the
    block's elements of dL/dE_e E_e ln 10, with dL/dE from pd_backward. The
    context keeps one factor per evaluated theta (pd_set_materials +
    pd_factor whenever theta changes). Stiffness damping scales with
    mu_e / max mu, a maximum the adjoint holds fixed, so a scene for this
    task should use beta0 = 0."""

    def __init__(self, scene, block_of_element, target_qT, options=None):
        super().__init__(scene, options)
        self.block = np.ascontiguousarray(block_of_element, dtype=np.int64)
        self.n_blocks = int(self.block.max()) + 1
        self.target = self.t(target_qT)
        self.dE = torch.empty(scene.n_e, dtype=torch.float64, device=DEV)
        self.theta = None

    def moduli(self, theta):
        return np.power(10.0, np.asarray(theta, dtype=np.float64))[self.block]

    def __call__(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        E = self.moduli(theta)
        if self.theta is None or not np.array_equal(theta, self.theta):
            self.pd.set_materials(E, self.scene.nu)
            self.theta = theta.copy()
        self.run()
        diff = self.qT - self.target
        f = 0.5 * float(torch.sum(diff * diff))
        binding.pd_backward(self.pd.ctx, diff.contiguous(), None, None, None, self.dE, None, None, 0)
        dE = self.dE.cpu().numpy()
        g = np.bincount(self.block, weights=dE * E * math.log(10.0), minlength=self.n_blocks)
        return f, g


def rigid_velocity_basis(X, pinned):
    """[3 n_v, 6] basis of rigid initial velocities v_i = u + omega x (X_i - c)
    (c the centroid; columns u_x, u_y, u_z, omega_x, omega_y, omega_z), zero
    on pinned vertices: the low-dimensional initial-state parametrisation of
    the paper's inverse-design tasks (initial linear and angular velocity)."""
    X = np.asarray(X, dtype=np.float64)
    r = X - X.mean(axis=0)
    n = X.shape[0]
    B = np.zeros((n, 3, 6))
    for i in range(3):
        B[:, i, i] = 1.0
    z = np.zeros(n)
    B[:, :, 3] = np.stack([z, -r[:, 2], r[:, 1]], axis=1)
    B[:, :, 4] = np.stack([r[:, 2], z, -r[:, 0]], axis=1)
    B[:, :, 5] = np.stack([-r[:, 1], r[:, 0], z], axis=1)
    B[np.asarray(pinned) != 0] = 0.0
    return B.reshape(3 * n, 6)


class InitialVelocity(_Rollout):
    """Initial-state optimisation (Sec. 5.5): the initial velocity v0 = B p
    (B: [3 n_v, k] basis, default the identity: every coordinate free;
    pinned rows are ignored by the library) such that the rollout ends at
    x*; loss 0.5 ||x_T(v0) - x*||^2, gradient B^T dL/dv0 with dL/dv0 from
    pd_backward."""

    def __init__(self, scene, target_qT, basis=None, options=None):
        super().__init__(scene, options)
        self.target = self.t(target_qT)
        self.basis = None if basis is None else np.ascontiguousarray(basis, dtype=np.float64)
        self.dv0 = torch.empty_like(self.x0)
        self.v = torch.empty_like(self.x0)

    def __call__(self, p):
        p = np.asarray(p, dtype=np.float64)
        v0 = p if self.basis is None else self.basis @ p
        self.v.copy_(torch.as_tensor(v0.reshape(-1, 3)))
        self.run(v0=self.v)
        diff = self.qT - self.target
        f = 0.5 * float(torch.sum(diff * diff))
        binding.pd_backward(self.pd.ctx, diff.contiguous(), None, None, self.dv0, None, None, None, 0)
        g = self.dv0.cpu().numpy().reshape(-1)
        return f, (g if self.basis is None else self.basis.T @ g)
