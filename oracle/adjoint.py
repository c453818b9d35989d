"""Backward pass, FP64 (Sec. 4.3 trust region, Sec. 4.7, Alg. 2).

For one step with R(q*) = A q* - b(q*) = 0 on the free DoFs, the adjoint is
mu = (A - K)^-T q_bar with q_bar = q_bar_{t+h} + v_bar_{t+h}/h and
K = db/dq = sum_e w_e V_e G_e^T (dp_e/dF_e) G_e (eq. db_dq); dp/dF is the
trust-region-filtered prox differential (eq. tr_blend, tr_ift) for
Neo-Hookean and the polar differential for corotated.

Reading (eq. Rqq, Alg. 2): d R_q/d q = I - A^-1 K is not the identity, so the
adjoint needs (A - K)^-1, not one A^-1 application; the oracle assembles the
12x12 K_e blocks explicitly and solves the sparse system directly.

Gradient routing, derived from eq. freefall, eq. A_damped and the damping
RHS (the printed eq. dl_dq / dl_dv_dfext drop or misplace terms):
  dL/dq_t   = (1 + alpha h) M/h^2 mu + B mu / h - v_bar_{t+h}/h
  dL/dv_t   = M/h mu
  dL/df_ext = mu
  dL/dw_e   = V_e <G_e mu, p_e* - G_e q*>                         (eq. dl_dwe)
  dL/dbeta_e= -(V_e/h) <G_e mu, G_e (q* - q_t)>
  dL/d{mu_bar, lambda_bar, k_bar} through sigma*(F; means) by the same IFT,
and the chain to E_e and nu through eq. lame, the weights and the means,
with mu_ref frozen at its factor-time value (max is not differentiable).
Pinned DoFs carry zero gradient.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, prox
from .solver import Problem, local_step, logvol_ratio, rotation_share


def local_jacobian(pb: Problem, q, tau: float, unfiltered: bool = False):
    """Per-element 9x9 dp/dF at q (filtered with tau unless ``unfiltered``)."""
    _, (U, sF, V, ss) = local_step(pb, q)
    n = U.shape[0]
    if pb.model == "corotated":
        z = np.zeros((n, 3, 3))
        return prox.dp_dF_matrix(U, sF, V, ss, z, z, corot=True), 0
    if pb.model == "corotated_volume":
        # sigma* = a + (1 - a) sigma_v(sigma_F): the diagonal response is
        # (1 - a) d sigma_v/d sigma_F of the volume step; no prox Hessian to
        # filter (the trust region acts on the Neo-Hookean prox only)
        F = fem.deformation_gradient(pb.rest, pb.tets, q)
        a = rotation_share(pb)
        _, (_, _, _, _, sv, nu) = prox.corot_volume_project(F, a)
        Jd = (1.0 - a)[:, None, None] * prox.volume_sigma_jacobian(sv, nu)
        return prox.dp_dF_matrix(U, sF, V, ss, Jd, Jd, corot=False), 0
    if pb.model == "corotated_logvol":
        # sigma* = a + (1 - a) sigma_b(sigma_F): the diagonal response is
        # (1 - a) times the barrier prox's filtered IFT Jacobian (its Hessian
        # plays the part of the Neo-Hookean prox Hessian in eq. tr_blend)
        F = fem.deformation_gradient(pb.rest, pb.tets, q)
        a = rotation_share(pb)
        r = logvol_ratio(pb)
        _, (_, _, _, _, sb) = prox.corot_logvol_project(F, a, r)
        Jf, Jraw, n_indef = prox.logvol_sigma_jacobian(sb, r, tau)
        c = (1.0 - a)[:, None, None]
        Jd = Jraw if unfiltered else Jf
        return prox.dp_dF_matrix(U, sF, V, ss, c * Jd, c * Jraw, corot=False), n_indef
    Jf, Jraw, n_indef = prox.filtered_sigma_jacobian(ss, pb.mat.mu_bar, pb.mat.lam_bar, pb.mat.k_bar, tau)
    Jd = Jraw if unfiltered else Jf
    return prox.dp_dF_matrix(U, sF, V, ss, Jd, Jraw, corot=False), n_indef


def element_G(pb: Problem) -> np.ndarray:
    """[n_e,9,12] G_e (row 3i+j of vec F, column 3a+i of the corner DoFs)."""
    n = pb.tets.shape[0]
    G = np.zeros((n, 9, 12))
    for a in range(4):
        for i in range(3):
            for j in range(3):
                G[:, 3 * i + j, 3 * a + i] = pb.rest.gradN[:, a, j]
    return G


def assemble_K(pb: Problem, q, tau: float, unfiltered: bool = False) -> sp.csr_matrix:
    """K = sum_e w_e V_e G_e^T D_e G_e as a [3n_v,3n_v] sparse matrix (eq. db_dq)."""
    D, _ = local_jacobian(pb, q, tau, unfiltered)
    G = element_G(pb)
    Ke = (pb.mat.w * pb.rest.vol)[:, None, None] * np.einsum("eki,ekl,elj->eij", G, D, G)
    dof = (3 * pb.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    rows = np.repeat(dof, 12, axis=1).ravel()
    cols = np.tile(dof, (1, 12)).ravel()
    n3 = 3 * pb.n_v
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n3, n3)).tocsr()


@dataclass
class StepGrad:
    dq_t: np.ndarray
    dv_t: np.ndarray
    df_ext: np.ndarray
    dw: np.ndarray
    dbeta: np.ndarray
    dmu_bar: float
    dlam_bar: float
    dk_bar: float
    mu: np.ndarray
    n_indef: int
    dw1: np.ndarray = None   # composite: dL/dw_1 of the volume step (dw is then dL/dw_0)
    dr: float = 0.0          # barrier variant: dL/dr through sigma_b, r = mu_e/lambda_e


def adjoint_solve(pb: Problem, q_star, tau: float, qbar_free):
    """mu_f = (A_ff - K_ff)^-T qbar_f, direct sparse LU."""
    K = assemble_K(pb, q_star, tau)
    f3 = (3 * pb.free[:, None] + np.arange(3)[None, :]).ravel()
    A3 = sp.kron(pb.LA_ff, sp.identity(3), format="csr")
    Msys = (A3 - K[f3][:, f3]).T.tocsc()
    return spla.spsolve(Msys, qbar_free.ravel()).reshape(-1, 3)


def mean_sensitivities(pb: Problem, q_star, mu_full, tau: float):
    """dL/d(mu_bar, lambda_bar, k_bar) = sum_e w_e V_e <G_e mu, dp_e/d theta>."""
    if pb.model in ("corotated", "corotated_volume", "corotated_logvol"):   # no mesh means inside the projections
        return 0.0, 0.0, 0.0
    _, (U, sF, V, ss) = local_step(pb, q_star)
    Jf, _, _ = prox.filtered_sigma_jacobian(ss, pb.mat.mu_bar, pb.mat.lam_bar, pb.mat.k_bar, tau)
    Hpinv = Jf / pb.mat.k_bar                                # filtered H~^+
    lnJ = np.log(np.prod(ss, axis=1))[:, None]
    dgrad = {"k": ss - sF, "mu": ss - 1.0 / ss, "lam": lnJ / ss}
    Gmu = fem.deformation_gradient(pb.rest, pb.tets, mu_full)
    Mh = np.einsum("nki,nkl,nlj->nij", U, Gmu, V)
    diag = np.diagonal(Mh, axis1=1, axis2=2)                 # [n,3]
    coef = pb.mat.w * pb.rest.vol
    out = {}
    for key, g in dgrad.items():
        ds = -np.einsum("nij,nj->ni", Hpinv, g)
        out[key] = float(np.sum(coef * np.sum(diag * ds, axis=1)))
    return out["mu"], out["lam"], out["k"]


def ratio_sensitivity(pb: Problem, q_star, mu_full, tau: float) -> float:
    """dL/dr of the barrier variant, r_e = mu_e/lambda_e inside its prox:
    sum_e lambda_e V_e <G_e mu, U diag(d sigma_b/d r) V^T> with
    d sigma_b/d r = H~^+ (1/sigma_b) by the IFT on the stationarity
    (ln J - r)/sigma_i + sigma_i - sigma_F,i = 0 (filtered like the Jacobian)."""
    F = fem.deformation_gradient(pb.rest, pb.tets, q_star)
    r = logvol_ratio(pb)
    _, (U, _, V, _, sb) = prox.corot_logvol_project(F, rotation_share(pb), r)
    Jf, _, _ = prox.logvol_sigma_jacobian(sb, r, tau)
    ds = np.einsum("nij,nj->ni", Jf, 1.0 / sb)
    Gmu = fem.deformation_gradient(pb.rest, pb.tets, mu_full)
    Mh = np.einsum("nki,nkl,nlj->nij", U, Gmu, V)
    diag = np.diagonal(Mh, axis1=1, axis2=2)
    return float(np.sum(pb.mat.lam * pb.rest.vol * np.sum(diag * ds, axis=1)))


def backward_step(pb: Problem, q_t, q_star, tau: float, qbar_next, vbar_next) -> StepGrad:
    h = pb.h
    qbar = qbar_next + vbar_next / h
    mu_f = adjoint_solve(pb, q_star, tau, qbar[pb.free])
    mu = np.zeros_like(q_star)
    mu[pb.free] = mu_f
    return route_step(pb, q_t, q_star, tau, mu, vbar_next)


def route_step(pb: Problem, q_t, q_star, tau: float, mu, vbar_next) -> StepGrad:
    """Gradient routing of one step (eq. dl_dq, eq. dl_dv_dfext, eq. dl_dwe with
    the readings of the module docstring) for a given adjoint vector mu."""
    h = pb.h
    m = pb.rest.mass[:, None]
    dq_t = (1.0 + pb.alpha * h) * m / h ** 2 * mu + (pb.B @ mu) / h - vbar_next / h
    dv_t = m / h * mu
    df = mu.copy()
    P, (U, _, V, _) = local_step(pb, q_star)
    F = fem.deformation_gradient(pb.rest, pb.tets, q_star)
    Gmu = fem.deformation_gradient(pb.rest, pb.tets, mu)
    dw1 = None
    if pb.model == "corotated_volume":
        # b carries w_0 V G^T R + w_1 V G^T p_vol and A carries (w_0 + w_1):
        # one sensitivity per weight
        _, (_, _, _, _, sv, _) = prox.corot_volume_project(F, rotation_share(pb))
        R = np.einsum("nij,nkj->nik", U, V)
        Pv = prox.compose(U, sv, V)
        dw = pb.rest.vol * np.einsum("nij,nij->n", Gmu, R - F)
        dw1 = pb.rest.vol * np.einsum("nij,nij->n", Gmu, Pv - F)
    elif pb.model == "corotated_logvol":
        # the same two weights, with the barrier's p_b as the volume target
        _, (_, _, _, _, sb) = prox.corot_logvol_project(F, rotation_share(pb), logvol_ratio(pb))
        R = np.einsum("nij,nkj->nik", U, V)
        Pb = prox.compose(U, sb, V)
        dw = pb.rest.vol * np.einsum("nij,nij->n", Gmu, R - F)
        dw1 = pb.rest.vol * np.einsum("nij,nij->n", Gmu, Pb - F)
    else:
        dw = pb.rest.vol * np.einsum("nij,nij->n", Gmu, P - F)
    Fd = fem.deformation_gradient(pb.rest, pb.tets, q_star - q_t)
    dbeta = -pb.rest.vol / h * np.einsum("nij,nij->n", Gmu, Fd)
    dmu, dlam, dk = mean_sensitivities(pb, q_star, mu, tau)
    for arr in (dq_t, dv_t, df):
        arr[pb.fixed] = 0.0
    dr = ratio_sensitivity(pb, q_star, mu, tau) if pb.model == "corotated_logvol" else 0.0
    _, n_indef = local_jacobian(pb, q_star, tau) if pb.model in ("neohookean", "corotated_logvol") else (None, 0)
    return StepGrad(dq_t, dv_t, df, dw, dbeta, dmu, dlam, dk, mu, n_indef, dw1, dr)


def chain_material(pb: Problem, dw, dbeta, dmu_bar, dlam_bar, dk_bar, paper_literal: bool = False, dw1=None,
                   dr: float = 0.0):
    """dL/dE_e and dL/dnu from the weight, damping and mean sensitivities
    (the composite and the barrier variant: dw = dL/dw_0 with w_0 = 2 mu,
    dw1 = dL/dw_1 with w_1 = lambda; Sec. 7.2 and eq. lame; the barrier's
    dr = dL/dr with r = mu/lambda = (1 - 2 nu)/(2 nu), dr/dnu = -1/(2 nu^2))."""
    E, nu = pb.E, pb.nu
    n = E.shape[0]
    dmu_dE = 1.0 / (2.0 * (1.0 + nu)) * np.ones(n)
    dlam_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) * np.ones(n)
    dmu_dnu = -E / (2.0 * (1.0 + nu) ** 2)
    dlam_dnu = E * (1.0 + 2.0 * nu ** 2) / ((1.0 + nu) * (1.0 - 2.0 * nu)) ** 2
    if pb.model in ("corotated_volume", "corotated_logvol"):
        dw1 = np.zeros(n) if dw1 is None else dw1
        cb = pb.beta0 / pb.mat.mu_ref
        dE = 2.0 * dw * dmu_dE + dw1 * dlam_dE + dbeta * cb * dmu_dE
        dnu = float(np.sum(2.0 * dw * dmu_dnu + dw1 * dlam_dnu + dbeta * cb * dmu_dnu))
        return dE, dnu - dr / (2.0 * nu * nu)
    nh = pb.model != "corotated"
    dw_dE = 2.0 * dmu_dE + (dlam_dE if nh else 0.0)
    dw_dnu = 2.0 * dmu_dnu + (dlam_dnu if nh else 0.0)
    if paper_literal:
        return dw * dw_dE, float(np.sum(dw * dw_dnu))
    cb = pb.beta0 / pb.mat.mu_ref
    dE = dw * dw_dE + dbeta * cb * dmu_dE + (dmu_bar * dmu_dE + dlam_bar * dlam_dE + dk_bar * dw_dE) / n
    dnu = (float(np.sum(dw * dw_dnu + dbeta * cb * dmu_dnu))
           + dmu_bar * float(np.mean(dmu_dnu)) + dlam_bar * float(np.mean(dlam_dnu))
           + dk_bar * float(np.mean(dw_dnu)))
    return dE, dnu


@dataclass
class RolloutGrad:
    dx0: np.ndarray
    dv0: np.ndarray
    dE: np.ndarray
    dnu: float
    df_ext: np.ndarray     # [T,n_v,3]
    dw_total: np.ndarray


def rollout_backward(pb: Problem, records, dqT, dvT, paper_literal: bool = False) -> RolloutGrad:
    """Walk the steps backwards, carrying (dL/dq_t, dL/dv_t) (Alg. 2 per step)."""
    qbar, vbar = dqT.copy(), dvT.copy()
    qbar[pb.fixed] = 0.0
    vbar[pb.fixed] = 0.0
    n_e = pb.tets.shape[0]
    dw_tot = np.zeros(n_e)
    dw1_tot = np.zeros(n_e)
    db_tot = np.zeros(n_e)
    dmu = dlam = dk = dr = 0.0
    dfs = []
    for rec in reversed(records):
        g = backward_step(pb, rec.q_t, rec.q_next, rec.tau, qbar, vbar)
        qbar, vbar = g.dq_t, g.dv_t
        dw_tot += g.dw
        if g.dw1 is not None:
            dw1_tot += g.dw1
        db_tot += g.dbeta
        dmu += g.dmu_bar
        dlam += g.dlam_bar
        dk += g.dk_bar
        dr += g.dr
        dfs.append(g.df_ext)
    dE, dnu = chain_material(pb, dw_tot, db_tot, dmu, dlam, dk, paper_literal, dw1_tot, dr)
    return RolloutGrad(qbar, vbar, dE, dnu, np.stack(dfs[::-1]), dw_tot)


def loss_and_grad(scene, pb: Problem, qT, vT):
    """The workload's loss on the final state and dL/d(q_T, v_T)."""
    if scene.loss == "com_z":
        m = pb.rest.mass
        L = float(np.sum(m * qT[:, 2]) / np.sum(m))
        dq = np.zeros_like(qT)
        dq[:, 2] = m / np.sum(m)
        return L, dq, np.zeros_like(vT)
    d = qT - scene.target
    return 0.5 * float(np.sum(d * d)), d, np.zeros_like(vT)
