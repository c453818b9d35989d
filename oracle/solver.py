"""Forward PD step and rollout, FP64 (Sec. 3.1, 4.1, 4.3, 4.4; Alg. 1).

The result of one step is the fixed point q* of q = A^-1 b(q) on the free
DoFs (pins eliminated, held at the rest position):

  A   = (1 + alpha h) M / h^2 + sum_e (w_e + beta_e/h) V_e G_e^T G_e     (eq. A_damped)
  b(q)= M/h^2 q~ + (alpha M + B_beta)/h q_t + sum_e w_e V_e G_e^T p_e*(G_e q)
  q~  = q_t + h v_t + h^2 (g + M^-1 f_ext)                               (eq. freefall)

Reading (damping RHS): eq. A_damped adds (alpha M + B_beta)/h to A but the
paper's b (eq. A_basic, Alg. 1) never gains the matching terms; they follow
from eq. dynamics with v_{t+h} = (q - q_t)/h and are what makes a body at rest
stay at rest (A X = b(X)), so they are included.

The oracle reaches the fixed point by plain Picard iterations followed by
Newton on A q - b(q) = 0 with the exact Jacobian A - db/dq; the GPU reaches it
by Anderson acceleration with the dual gate. ``aa_reference`` restates that
accelerated loop in FP64 for iteration-count and reset checks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, prox


@dataclass
class Problem:
    X: np.ndarray
    tets: np.ndarray
    pinned: np.ndarray
    model: str
    h: float
    alpha: float
    gravity: np.ndarray
    rest: fem.Rest
    mat: fem.Material
    LA: sp.csr_matrix          # full scalar operator [n_v,n_v]
    B: sp.csr_matrix           # scalar stiffness damping [n_v,n_v]
    free: np.ndarray
    fixed: np.ndarray
    LA_ff: sp.csc_matrix
    LA_fp: sp.csr_matrix
    lu: object                  # factor of LA_ff (scalar, shared by the 3 axes)
    E: np.ndarray = field(default=None)
    nu: float = 0.0
    beta0: float = 0.0

    @property
    def n_v(self):
        return self.X.shape[0]


def build_problem(scene, E=None, nu=None, mu_ref=None) -> Problem:
    """Assemble and factor A for a scene (optionally overriding E, nu, mu_ref)."""
    E = scene.E if E is None else np.asarray(E, dtype=np.float64)
    nu = scene.nu if nu is None else float(nu)
    rest = fem.rest_shape(scene.X, scene.tets, scene.density)
    mat = fem.material(E, nu, scene.model, scene.beta0, mu_ref)
    LA = fem.assemble_LA(rest, scene.tets, mat, scene.alpha, scene.dt)
    B = fem.assemble_B(rest, scene.tets, mat)
    free = np.nonzero(scene.pinned == 0)[0]
    fixed = np.nonzero(scene.pinned != 0)[0]
    LA_ff = LA[free][:, free].tocsc()
    LA_fp = LA[free][:, fixed].tocsr()
    lu = spla.splu(LA_ff)
    return Problem(scene.X, scene.tets, scene.pinned, scene.model, scene.dt, scene.alpha,
                   np.asarray(scene.gravity, dtype=np.float64), rest, mat, LA, B, free, fixed,
                   LA_ff, LA_fp, lu, E, nu, scene.beta0)


def solve_A(pb: Problem, r_free: np.ndarray) -> np.ndarray:
    """A_ff^-1 r for r [n_f,3] (A = L_A (x) I_3: one scalar solve per axis)."""
    return np.stack([pb.lu.solve(np.ascontiguousarray(r_free[:, i])) for i in range(3)], axis=1)


def inertial_target(pb: Problem, q_t, v_t, f_ext):
    """eq. freefall with gravity as a body acceleration."""
    return q_t + pb.h * v_t + pb.h ** 2 * (pb.gravity[None, :] + f_ext / pb.rest.mass[:, None])


def rhs_const(pb: Problem, q_t, v_t, f_ext):
    """The q-independent part of b: M/h^2 q~ + (alpha M + B)/h q_t."""
    m = pb.rest.mass[:, None]
    qt = inertial_target(pb, q_t, v_t, f_ext)
    return m / pb.h ** 2 * qt + (pb.alpha * m * q_t + pb.B @ q_t) / pb.h


def local_step(pb: Problem, q):
    """p_e* for all elements (Sec. 4.1) and the SVD state."""
    F = fem.deformation_gradient(pb.rest, pb.tets, q)
    if pb.model == "corotated":
        U, sF, V = prox.svd_rv(F)
        return np.einsum("nij,nkj->nik", U, V), (U, sF, V, np.ones_like(sF))
    if pb.model == "corotated_volume":
        P, (U, sF, V, ss, _, _) = prox.corot_volume_project(F, rotation_share(pb))
        return P, (U, sF, V, ss)
    if pb.model == "corotated_logvol":
        P, (U, sF, V, ss, _) = prox.corot_logvol_project(F, rotation_share(pb), logvol_ratio(pb))
        return P, (U, sF, V, ss)
    return prox.nh_project(F, pb.mat.mu_bar, pb.mat.lam_bar, pb.mat.k_bar)


def rotation_share(pb: Problem) -> np.ndarray:
    """a_e = w_0/(w_0 + w_1) = 2 mu_e/(2 mu_e + lambda_e) of the composite
    (and of the barrier variant, whose volume weight is also lambda_e)."""
    return 2.0 * pb.mat.mu / (2.0 * pb.mat.mu + pb.mat.lam)


def logvol_ratio(pb: Problem) -> np.ndarray:
    """r_e = mu_e/lambda_e of the barrier's prox (eq. pd_log_volume)."""
    return prox.logvol_ratio(pb.mat.mu, pb.mat.lam)


def rhs(pb: Problem, b0, q):
    """b(q) = b0 + sum_e w_e V_e G_e^T p_e*(G_e q)   (eq. A_basic, Alg. 1)."""
    P, _ = local_step(pb, q)
    return b0 + fem.scatter_GT(pb.rest, pb.tets, P, pb.mat.w * pb.rest.vol, pb.n_v)


def free_rhs(pb: Problem, b_full):
    """Pinned columns moved to the right-hand side: b_f - A_fp X_p."""
    return b_full[pb.free] - pb.LA_fp @ pb.X[pb.fixed]


def apply_A_full(pb: Problem, q):
    return pb.LA @ q


def full(pb: Problem, q_free):
    q = pb.X.copy()
    q[pb.free] = q_free
    return q


def picard(pb: Problem, b0, q):
    """One local-global iteration q <- A^-1 b(q) (free DoFs)."""
    return full(pb, solve_A(pb, free_rhs(pb, rhs(pb, b0, q))))


def stationarity(pb: Problem, b0, q) -> float:
    """||A q - b(q)||_free / ||b(q)||_free."""
    r = free_rhs(pb, rhs(pb, b0, q))
    res = (pb.LA_ff @ q[pb.free]) - r
    return float(np.linalg.norm(res) / max(np.linalg.norm(r), 1e-300))


def newton_matrix(pb: Problem, q):
    """Exact Jacobian of A q - b(q) on the free DoFs: kron(L_ff, I3) - K_ff."""
    from .adjoint import assemble_K
    K = assemble_K(pb, q, tau=0.0, unfiltered=True)
    f3 = (3 * pb.free[:, None] + np.arange(3)[None, :]).ravel()
    A3 = sp.kron(pb.LA_ff, sp.identity(3), format="csr")
    return (A3 - K[f3][:, f3]).tocsc()


def fixed_point(pb: Problem, b0, q_init, tol: float = 1e-13, picard_iters: int = 30,
                newton_iters: int = 40):
    """q* with A q* = b(q*): Picard then Newton. Returns (q*, info)."""
    q = q_init.copy()
    q[pb.fixed] = pb.X[pb.fixed]
    n_pic = 0
    for _ in range(picard_iters):
        qn = picard(pb, b0, q)
        n_pic += 1
        step = np.linalg.norm(qn - q)
        q = qn
        if step <= tol * np.linalg.norm(q):
            return q, {"picard": n_pic, "newton": 0}
    n_new = 0
    for _ in range(newton_iters):
        r = free_rhs(pb, rhs(pb, b0, q))
        res = r - pb.LA_ff @ q[pb.free]
        J = newton_matrix(pb, q)
        dq = spla.spsolve(J, res.ravel()).reshape(-1, 3)
        q_try = q.copy()
        q_try[pb.free] += dq
        n_new += 1
        if not np.all(np.isfinite(q_try)):
            raise FloatingPointError("Newton produced non-finite iterate")
        q = q_try
        if np.linalg.norm(dq) <= tol * np.linalg.norm(q):
            break
    return q, {"picard": n_pic, "newton": n_new}


def phi(pb: Problem, q, q_tilde):
    """eq. primal: 1/(2h^2)||q - q~||_M^2 + sum_e V_e psi_e(F_e(q)), per-element mu_e, lambda_e."""
    d = q - q_tilde
    kin = 0.5 / pb.h ** 2 * float(np.sum(pb.rest.mass[:, None] * d * d))
    F = fem.deformation_gradient(pb.rest, pb.tets, q)
    psi = prox.nh_psi_F(F, pb.mat.mu, pb.mat.lam)
    return kin + float(np.sum(pb.rest.vol * psi))


def tr_select(pb: Problem, q_star, q_prev, q_tilde, eps_tr: float = 0.1):
    """tau* from the last PD increment (eq. tr_step, tr_decreases, tr_ratio, tr_rule).

    Returns (tau, rho). Phi = +inf at an inverted iterate gives rho non-finite
    and tau = 1 (the model is inadequate there).
    """
    dq = (q_star - q_prev)[pb.free]
    mod = 0.5 * abs(float(np.sum(dq * (pb.LA_ff @ dq))))
    if mod < 1e-12:
        rho = 1.0
    else:
        act = phi(pb, q_prev, q_tilde) - phi(pb, q_star, q_tilde)
        rho = act / mod
    tau = 0.5 if (np.isfinite(rho) and abs(rho - 1.0) <= eps_tr) else 1.0
    return tau, rho


# ------------------------------------------------------------------ Anderson

def dual_gate(dq_norm, q_norm, db_norm, b_norm, eps_step, eps_res, eps_abs):
    """eq. convergence_dual with separate step / RHS-change tolerances."""
    return dq_norm <= eps_step * q_norm + eps_abs and db_norm <= eps_res * b_norm + eps_abs


def aa_mix(hist_q, hist_g, qhat, g):
    """Type-II Anderson step from the history (eq. aa_dG, aa_dQ, aa_gamma, aa_update).

    hist_q / hist_g hold the last (q, g) pairs, oldest first, the newest being
    the current (q^k, g^k) with g^k = q_hat - q^k. Columns are successive
    differences; rho_aa = max(1e-6 ||dG||_F^2 / m_c, 1e-12) with m_c the current
    column count. Returns (q_new, reset): q_new = q_hat - (dQ + dG) gamma, or
    (q_hat, True) when ||gamma||_2 > 10 (reliability guard).
    """
    if len(hist_q) < 2:
        return qhat, False
    dG = np.stack([(hist_g[i + 1] - hist_g[i]).ravel() for i in range(len(hist_g) - 1)], axis=1)
    dQ = np.stack([(hist_q[i + 1] - hist_q[i]).ravel() for i in range(len(hist_q) - 1)], axis=1)
    mc = dG.shape[1]
    reg = max(1e-6 * float(np.sum(dG * dG)) / mc, 1e-12)
    gamma = np.linalg.solve(dG.T @ dG + reg * np.eye(mc), dG.T @ np.ravel(g))
    if np.linalg.norm(gamma) > 10.0:
        return qhat, True
    return qhat - ((dQ + dG) @ gamma).reshape(np.shape(qhat)), False


def aa_reference(pb: Problem, b0, q_t, m: int, k_max: int, eps_step, eps_res, eps_abs,
                 fixed_iters: int = 0):
    """The accelerated local-global loop of Alg. 1 in FP64.

    Readings: residual g^k = q_hat - q^k (Alg. 1); the history keeps the last
    m + 1 (q, g) pairs, i.e. m difference columns (eq. aa_dG has m columns);
    a guard trip falls back to q_hat and clears the whole history. The gate
    compares q^{k+1} with q^k and b(q^{k+1}) with b(q^k) (k >= 1), with 2-norms
    over the free DoFs. Returns (q*, q*-1, info).
    """
    q = q_t.copy()
    q[pb.fixed] = pb.X[pb.fixed]
    hist_q, hist_g = [], []
    b_prev = None
    q_prev = q.copy()
    resets = 0
    converged = False
    n_iter = 0
    for k in range(k_max + 1):
        bk = free_rhs(pb, rhs(pb, b0, q))
        if fixed_iters and k == fixed_iters:
            break
        if not fixed_iters and k >= 2:
            if dual_gate(np.linalg.norm((q - q_prev)[pb.free]), np.linalg.norm(q_prev[pb.free]),
                         np.linalg.norm(bk - b_prev), np.linalg.norm(b_prev), eps_step, eps_res, eps_abs):
                converged = True
                break
        if k == k_max:
            break
        qhat = solve_A(pb, bk)
        qf = q[pb.free]
        g = qhat - qf
        q_new = qhat
        if m > 0:
            hist_q.append(qf.copy())
            hist_g.append(g.copy())
            if len(hist_q) > m + 1:
                hist_q.pop(0)
                hist_g.pop(0)
            q_new, reset = aa_mix(hist_q, hist_g, qhat, g)
            if reset:
                resets += 1
                hist_q, hist_g = [], []
        q_prev = q.copy()
        b_prev = bk
        q = full(pb, q_new)
        n_iter += 1
    return q, q_prev, {"iters": n_iter, "converged": converged, "resets": resets}


def pd_energy(pb: Problem, q, q_t, q_tilde):
    """E_PD(q) = min_p g~(q, p): the function one local-global iteration decreases.

    g~(q,p) = 1/(2h^2)||q - q~||_M^2 + 1/(2h)(q - q_t)^T (alpha M + B)(q - q_t)
              + sum_e w_e V_e [ 1/2 ||G_e q - p_e||^2 + psi_bar(p_e)/k_bar ]
    (eq. pd_surrogate with the prox of eq. nh_prox folded into the p-minimum;
    for corotated the psi term is the indicator of SO(3)). Minimising over p
    gives the local step, over q the global step A q = b.
    """
    d = q - q_tilde
    dd = q - q_t
    m = pb.rest.mass[:, None]
    val = 0.5 / pb.h ** 2 * float(np.sum(m * d * d))
    val += 0.5 / pb.h * float(np.sum(dd * (pb.alpha * m * dd + pb.B @ dd)))
    P, (U, sF, V, ss) = local_step(pb, q)
    F = fem.deformation_gradient(pb.rest, pb.tets, q)
    if pb.model == "corotated_volume":
        # w_0/2 dist^2(F, SO(3)) + w_1/2 dist^2(F, {det = 1}), each a
        # minimum over its own projection
        w0, w1 = 2.0 * pb.mat.mu, pb.mat.lam
        _, (_, _, _, _, sv, _) = prox.corot_volume_project(F, rotation_share(pb))
        R = np.einsum("nij,nkj->nik", U, V)
        Pv = prox.compose(U, sv, V)
        el = 0.5 * (w0 * np.einsum("nij,nij->n", F - R, F - R) + w1 * np.einsum("nij,nij->n", F - Pv, F - Pv))
        return val + float(np.sum(pb.rest.vol * el))
    if pb.model == "corotated_logvol":
        # w_0/2 dist^2(F, SO(3)) + min_p [w_1/2 ||F - p||^2 + phi_log(p)],
        # w_1 = lambda_e, the second minimum attained at the barrier's prox
        w0, w1 = 2.0 * pb.mat.mu, pb.mat.lam
        r = logvol_ratio(pb)
        _, (_, _, _, _, sb) = prox.corot_logvol_project(F, rotation_share(pb), r)
        R = np.einsum("nij,nkj->nik", U, V)
        Pb = prox.compose(U, sb, V)
        el = 0.5 * (w0 * np.einsum("nij,nij->n", F - R, F - R) + w1 * np.einsum("nij,nij->n", F - Pb, F - Pb))
        el = el + w1 * prox.logvol_phi_sigma(sb, r)
        return val + float(np.sum(pb.rest.vol * el))
    el = 0.5 * np.einsum("nij,nij->n", F - P, F - P)
    if pb.model != "corotated":
        el = el + prox.nh_psi_sigma(ss, pb.mat.mu_bar, pb.mat.lam_bar) / pb.mat.k_bar
    return val + float(np.sum(pb.mat.w * pb.rest.vol * el))


# ------------------------------------------------------------------ rollout

@dataclass
class StepRecord:
    q_t: np.ndarray
    v_t: np.ndarray
    f_ext: np.ndarray
    q_next: np.ndarray
    q_prev_iter: np.ndarray
    tau: float
    rho: float
    info: dict


def step(pb: Problem, q_t, v_t, f_ext, mode: str = "exact", settings=None):
    """One implicit-Euler PD step. mode 'exact' = fixed point; 'fixed' = N plain
    iterations from q_t (no acceleration); 'aa' = the accelerated gated loop."""
    b0 = rhs_const(pb, q_t, v_t, f_ext)
    q_tilde = inertial_target(pb, q_t, v_t, f_ext)
    if mode == "fixed":
        q_prev = q_t.copy()
        q = q_t.copy()
        q[pb.fixed] = pb.X[pb.fixed]
        for _ in range(settings.fixed_iters):
            q_prev = q
            q = picard(pb, b0, q)
        info = {"iters": settings.fixed_iters}
    elif mode == "aa":
        q, q_prev, info = aa_reference(pb, b0, q_t, settings.aa_m, settings.k_max, settings.eps_step,
                                       settings.eps_res, settings.eps_abs)
    else:
        q, info = fixed_point(pb, b0, q_t)
        # no last increment at an exact fixed point: Delta Phi_mod = 0 < 1e-12
        # gives rho = 1 and tau = 1/2 by eq. tr_ratio
        q_prev = q
    if pb.model in ("neohookean", "corotated_logvol"):   # the models with a prox Hessian to filter
        tau, rho = tr_select(pb, q, q_prev, q_tilde, settings.eps_tr if settings else 0.1)
    else:
        tau, rho = 0.5, 1.0
    return q, q_prev, tau, rho, info


def rollout(pb: Problem, scene, mode: str = "exact", x0=None, v0=None, f_ext=None):
    """T steps from (x0, v0); returns (q_T, v_T, records)."""
    q = (scene.x0 if x0 is None else x0).copy()
    v = (scene.v0 if v0 is None else v0).copy()
    fe = scene.f_ext if f_ext is None else f_ext
    q[pb.fixed] = pb.X[pb.fixed]
    v[pb.fixed] = 0.0
    recs = []
    for t in range(scene.steps):
        f = fe[t if fe.shape[0] > 1 else 0]
        qn, qp, tau, rho, info = step(pb, q, v, f, mode, scene.solver)
        vn = (qn - q) / pb.h
        recs.append(StepRecord(q, v, f, qn, qp, tau, rho, info))
        q, v = qn, vn
    return q, v, recs


def mode_for(scene) -> str:
    return "fixed" if scene.solver.fixed_iters > 0 else "exact"
