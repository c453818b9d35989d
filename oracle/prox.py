"""Local step of PD and its differential, FP64 (Sec. 4.1, Sec. 4.3).

* Rotation-variant SVD: F = U diag(s) V^T with det U = det V = +1; only the
  smallest singular value may be negative (inverted element).
* Corotated local step (Sec. 4.1): p* = R = U V^T, the rotation of the polar
  decomposition.
* Neo-Hookean proximal map (eq. nh_prox, nh_prox_normal): in stretch space,
  sigma* = argmin_{sigma>0} k_bar/2 ||sigma - sigma_F||^2 + psi_bar(sigma) with
  the mesh-mean material (mu_bar, lambda_bar); p* = U diag(sigma*) V^T.
  Reading of eq. nh_hessian_stretch: its sigma^-4 is taken as a typo; the
  stretch Hessian is derived from eq. neohookean,
    d psi/d s_i      = mu (s_i - 1/s_i) + lam ln J / s_i
    d2 psi/d s_i^2   = mu (1 + 1/s_i^2) + lam (1 - ln J) / s_i^2
    d2 psi/d s_i s_j = lam / (s_i s_j)            (i != j).
  The prox is per unit volume (no V_e), matching eq. nh_prox_normal and Alg. 1.
* Log-volume barrier (eq. pd_log_volume): the opt-in volume step that
  replaces the composite's quadratic one, a stretch prox of the same kind.
* Differential of the isotropic spectral map p(F) = U diag(f(s)) V^T (the
  "SVD differential" the paper names for eq. tr_ift), with the trust-region
  blend of eq. tr_blend applied to H_prox = H_psi + k_bar I before inversion.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- SVD / polar

def svd_rv(F: np.ndarray):
    """Rotation-variant SVD of [n,3,3] -> (U [n,3,3], s [n,3], V [n,3,3])."""
    U, s, Vt = np.linalg.svd(F)
    V = np.transpose(Vt, (0, 2, 1)).copy()
    U = U.copy()
    s = s.copy()
    du = np.linalg.det(U) < 0
    U[du, :, 2] *= -1.0
    s[du, 2] *= -1.0
    dv = np.linalg.det(V) < 0
    V[dv, :, 2] *= -1.0
    s[dv, 2] *= -1.0
    return U, s, V


def compose(U, s, V):
    return np.einsum("nij,nj,nkj->nik", U, s, V)


def corotated_project(F: np.ndarray) -> np.ndarray:
    U, _, V = svd_rv(F)
    return np.einsum("nij,nkj->nik", U, V)


# ---------------------------------------------------------- Neo-Hookean energy

def nh_psi_F(F: np.ndarray, mu, lam) -> np.ndarray:
    """eq. neohookean per element; +inf where J <= 0."""
    J = np.linalg.det(F)
    out = np.full(F.shape[0], np.inf)
    ok = J > 0
    lnJ = np.log(J[ok])
    mu = np.broadcast_to(mu, J.shape)[ok]
    lam = np.broadcast_to(lam, J.shape)[ok]
    out[ok] = 0.5 * mu * (np.einsum("nij,nij->n", F[ok], F[ok]) - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2
    return out


def nh_psi_sigma(s, mu, lam):
    lnJ = np.log(np.prod(s, axis=-1))
    return 0.5 * mu * (np.sum(s * s, axis=-1) - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2


def nh_grad_sigma(s, mu, lam):
    lnJ = np.log(np.prod(s, axis=-1))[..., None]
    return mu * (s - 1.0 / s) + lam * lnJ / s


def nh_hess_sigma(s, mu, lam):
    lnJ = np.log(np.prod(s, axis=-1))
    inv = 1.0 / s
    H = lam * inv[..., :, None] * inv[..., None, :]
    d = mu * (1.0 + inv ** 2) + lam * (1.0 - lnJ[..., None]) * inv ** 2
    idx = np.arange(3)
    H[..., idx, idx] = d
    return H


def _stretch_prox(sF: np.ndarray, k: float, psi, grad, hess, tol: float = 1e-14, max_iter: int = 60):
    """Newton on f(s) = k/2||s - sF||^2 + psi(s), s > 0, in stretch space
    (eq. nh_prox_normal: the Newton-on-stretches step with backtracking and
    positivity that the Neo-Hookean prox and the log-volume barrier share).

    Start s0 = max(sF, 0.1); Newton direction if it is a descent direction of a
    positive-definite model, else the scaled gradient -g/k; step halved until
    s stays positive and either Armijo (c = 1e-4) holds or, for a Newton
    step, the gradient max-norm halves. Stops at ||g||_inf <= tol*k.
    Returns (sigma*, iterations used per element).
    """
    s = np.maximum(sF, 0.1).astype(np.float64)
    n = s.shape[0]
    active = np.ones(n, dtype=bool)
    iters = np.zeros(n, dtype=np.int64)

    def f(x, ref, rows):
        return 0.5 * k * np.sum((x - ref) ** 2, axis=-1) + psi(x, rows)

    for _ in range(max_iter):
        g = k * (s - sF) + grad(s, slice(None))
        active &= ~(np.abs(g).max(axis=1) <= tol * k)
        if not active.any():
            break
        a = np.nonzero(active)[0]
        sa, ga, ra = s[a], g[a], sF[a]
        H = k * np.eye(3) + hess(sa, a)
        pd = np.all(np.linalg.eigvalsh(H) > 0, axis=1)
        d = -np.linalg.solve(H, ga[..., None])[..., 0]
        bad = (~pd) | (np.einsum("ni,ni->n", d, ga) >= 0)
        d[bad] = -ga[bad] / k
        slope = np.einsum("ni,ni->n", d, ga)
        t = np.ones(a.shape[0])
        for _h in range(80):          # positivity
            neg = np.any(sa + t[:, None] * d <= 0, axis=1)
            if not neg.any():
                break
            t[neg] *= 0.5
        f0 = f(sa, ra, a)
        done = np.zeros(a.shape[0], dtype=bool)
        for _h in range(60):          # Armijo
            trial = sa + t[:, None] * d
            # sufficient decrease of f, or (Newton steps only) a halving of the
            # gradient's max-norm: in the quadratic-convergence regime the
            # decrease of f falls below its rounding and Armijo cannot see it
            gt = k * (trial - ra) + grad(trial, a)
            ok = (f(trial, ra, a) <= f0 + 1e-4 * t * slope) | (
                (~bad) & (np.abs(gt).max(axis=1) <= 0.5 * np.abs(ga).max(axis=1)))
            done |= ok
            if done.all():
                break
            t[~done] *= 0.5
        stalled = ~done                # no decrease representable: converged to rounding
        s[a] = np.where(done[:, None], sa + t[:, None] * d, sa)
        iters[a] += 1
        active[a[stalled]] = False
    return s, iters


def nh_prox_sigma(sF: np.ndarray, mu: float, lam: float, k: float, tol: float = 1e-14,
                  max_iter: int = 60):
    """sigma* = argmin_{sigma>0} k/2||sigma - sF||^2 + psi_bar(sigma) (eq. nh_prox,
    nh_prox_normal) with the mesh-mean Neo-Hookean energy."""
    return _stretch_prox(sF, k,
                         lambda x, rows: nh_psi_sigma(x, mu, lam),
                         lambda x, rows: nh_grad_sigma(x, mu, lam),
                         lambda x, rows: nh_hess_sigma(x, mu, lam), tol, max_iter)


def nh_project(F: np.ndarray, mu_bar: float, lam_bar: float, k_bar: float):
    """p* for every element, with the SVD pieces needed by the differential."""
    U, sF, V = svd_rv(F)
    ss, _ = nh_prox_sigma(sF, mu_bar, lam_bar, k_bar)
    return compose(U, ss, V), (U, sF, V, ss)


# ----------------------------------------------------------- volume step

def _grad_J(s):
    """Gradient of J = s_1 s_2 s_3 in stretch space."""
    return np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)


def _kkt(s, nu):
    """[[I + nu Hess J, grad J], [grad J^T, 0]] per element, [n,4,4]."""
    n = s.shape[0]
    K = np.zeros((n, 4, 4))
    K[:, :3, :3] = np.eye(3)
    for i in range(3):
        for j in range(3):
            if i != j:
                k = 3 - i - j
                K[:, i, j] += nu * s[:, k]
    g = _grad_J(s)
    K[:, :3, 3] = g
    K[:, 3, :3] = g
    return K


def _plus_root(a, nu):
    """The larger root of s^2 - a s + nu = 0 (the stationarity condition
    s - a + nu/s = 0 of one stretch on J = 1), without cancellation."""
    r = np.sqrt(np.maximum(a * a - 4.0 * nu, 0.0))
    safe = np.where(a - r != 0.0, a - r, -1.0)
    return np.where(a >= 0.0, 0.5 * (a + r), 2.0 * nu / safe)


def _volume_curve(sF, s3):
    """The stationary curve parametrized by the smallest stretch s_3: the
    multiplier nu = s_3 (sigma_F3 - s_3) (stationarity of s_3) and s_1, s_2
    the larger roots of their own stationarity quadratics at that nu.
    Returns (s [n,3], nu)."""
    nu = s3 * (sF[:, 2] - s3)
    s = np.stack([_plus_root(sF[:, 0], nu), _plus_root(sF[:, 1], nu), s3], axis=1)
    return s, nu


def volume_project_sigma(sF: np.ndarray, iters: int = 200):
    """The volume step of the corotated + volume composite (Sec. 4.1, the
    quadratic (J - 1)^2 volume step that pairs with the corotated rotation
    step; Sec. 7.2 weights w_1 = lambda): the closest point of the unit
    determinant set in stretch space,
        sigma* = argmin 1/2 ||sigma - sigma_F||^2  s.t.  sigma_1 sigma_2 sigma_3 = 1,
    on the positive sheet (sigma > 0), so that p* = U diag(sigma*) V^T is the
    closest matrix with det = 1 to F (the rotation-variant order
    sigma_F1 >= sigma_F2 >= |sigma_F3| makes the positive sheet the nearest).

    Stationarity reads s_i^2 - sigma_Fi s_i + nu = 0 for every i with one
    multiplier nu. The minimiser lies on the curve where s_1 and s_2 take the
    larger root and s_3 is free (nu = s_3 (sigma_F3 - s_3)); along it
    log(s_1 s_2 s_3) goes from -inf (s_3 -> 0) to +inf (s_3 -> inf) and
    changes sign once, so the minimiser is that sign change, found here by
    plain bisection in log s_3 over [-40, 40] (the unit-determinant set can
    have several stationary points, e.g. for a stretched element, and a
    Newton on the Lagrange system may settle on any of them; bisection on
    this curve cannot). Returns (sigma*, nu, iterations)."""
    n = sF.shape[0]
    lo = np.full(n, -40.0)
    hi = np.full(n, 40.0)
    it = 0
    for it in range(1, iters + 1):
        mid = 0.5 * (lo + hi)
        s, _ = _volume_curve(sF, np.exp(mid))
        pos = np.sum(np.log(s), axis=1) > 0.0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
        if np.all(hi - lo <= 1e-15 * np.maximum(1.0, np.abs(hi))):
            break
    s, nu = _volume_curve(sF, np.exp(0.5 * (lo + hi)))
    return s, nu, it


def volume_sigma_jacobian(s: np.ndarray, nu: np.ndarray) -> np.ndarray:
    """d sigma*/d sigma_F of the volume step, by implicit differentiation of
    its Lagrange system: the 3 x 3 leading block of the inverse KKT matrix."""
    return np.linalg.inv(_kkt(s, nu))[:, :3, :3]


def corot_volume_project(F: np.ndarray, a: np.ndarray):
    """The composite's per-element projection p = (w_0 R + w_1 p_vol)/(w_0 + w_1)
    with a = w_0/(w_0 + w_1): since R = U V^T and p_vol = U diag(sigma_v) V^T
    share the SVD of F, p = U diag(a + (1 - a) sigma_v) V^T. Returns p and
    (U, sigma_F, V, sigma*, sigma_v, nu)."""
    U, sF, V = svd_rv(F)
    sv, nu, _ = volume_project_sigma(sF)
    ss = a[:, None] + (1.0 - a[:, None]) * sv
    return compose(U, ss, V), (U, sF, V, ss, sv, nu)


# ------------------------------------------------------ log-volume barrier

def logvol_ratio(mu, lam):
    """r = mu_e / lambda_e = (1 - 2 nu)/(2 nu): the only material constant of
    the barrier's prox once it is divided by its weight w_e = lambda_e."""
    return np.asarray(mu, dtype=np.float64) / np.asarray(lam, dtype=np.float64)


def logvol_phi_sigma(s, r):
    """phi_log(sigma)/lambda_e of eq. pd_log_volume:
    -r sum_i ln sigma_i + 1/2 (sum_j ln sigma_j)^2 with r = mu_e/lambda_e."""
    ls = np.log(s)
    return -r * np.sum(ls, axis=-1) + 0.5 * np.sum(ls, axis=-1) ** 2


def logvol_grad_sigma(s, r):
    """d(phi_log/lambda)/d sigma_i = (ln J - r)/sigma_i, ln J = sum_j ln sigma_j."""
    lnJ = np.sum(np.log(s), axis=-1)
    return (lnJ - r)[..., None] / s


def logvol_hess_sigma(s, r):
    """Its Hessian: (1 + r - ln J)/sigma_i^2 on the diagonal, 1/(sigma_i sigma_j) off it."""
    lnJ = np.sum(np.log(s), axis=-1)
    inv = 1.0 / s
    H = inv[..., :, None] * inv[..., None, :]
    idx = np.arange(3)
    H[..., idx, idx] = (1.0 + r - lnJ)[..., None] * inv ** 2
    return H


def logvol_prox_sigma(sF: np.ndarray, r, tol: float = 1e-14, max_iter: int = 60):
    """The barrier's volume step (Sec. 4.1, volume-barrier surrogate, eq.
    pd_log_volume, registered with w_e = lambda_e): in stretch space
        sigma_b = argmin_{sigma>0} lambda_e/2 ||sigma - sigma_F||^2 + phi_log(sigma),
    divided by lambda_e, by the same Newton-on-stretches step as the
    Neo-Hookean prox with the barrier's own gradient and Hessian. ``r`` is a
    scalar or one value per element. Returns (sigma_b, iterations)."""
    rr = np.broadcast_to(np.asarray(r, dtype=np.float64), sF.shape[:1])
    return _stretch_prox(sF, 1.0,
                         lambda x, rows: logvol_phi_sigma(x, rr[rows]),
                         lambda x, rows: logvol_grad_sigma(x, rr[rows]),
                         lambda x, rows: logvol_hess_sigma(x, rr[rows]), tol, max_iter)


def corot_logvol_project(F: np.ndarray, a: np.ndarray, r):
    """The barrier variant's projection: the corotated rotation step (w_0 =
    2 mu) with the barrier's volume step (w_1 = lambda) in place of the
    quadratic one, p = (w_0 R + w_1 p_b)/(w_0 + w_1) = U diag(a + (1 - a)
    sigma_b) V^T. Returns p and (U, sigma_F, V, sigma*, sigma_b)."""
    U, sF, V = svd_rv(F)
    sb, _ = logvol_prox_sigma(sF, r)
    ss = a[:, None] + (1.0 - a[:, None]) * sb
    return compose(U, ss, V), (U, sF, V, ss, sb)


def logvol_sigma_jacobian(sb: np.ndarray, r, tau: float):
    """d sigma_b/d sigma_F = H~(tau)^+ with H = I + Hess(phi_log/lambda)(sigma_b)
    (eq. tr_ift with k = 1 after the division by lambda_e); (filtered,
    unfiltered, count of indefinite H)."""
    rr = np.broadcast_to(np.asarray(r, dtype=np.float64), sb.shape[:1])
    return filtered_inverse(np.eye(3) + logvol_hess_sigma(sb, rr), 1.0, tau)


# ------------------------------------------------------- trust-region filter

def tr_blend(H: np.ndarray, tau: float) -> np.ndarray:
    """eq. tr_blend: (1 - tau) H + tau |H|, |H| = Q |Lambda| Q^T, per 3x3 block."""
    lam, Q = np.linalg.eigh(H)
    lt = (1.0 - tau) * lam + tau * np.abs(lam)
    return np.einsum("nij,nj,nkj->nik", Q, lt, Q)


def filtered_inverse(H: np.ndarray, k: float, tau: float):
    """k H~(tau)^+ (eq. tr_ift) for a per-element 3x3 prox Hessian H.

    Eigen-directions of H~ with eigenvalue <= 1e-12 k get zero response (the
    pseudo-inverse: clamping a negative eigenvalue makes H~ singular).
    Also returns the unfiltered k H^-1 and the count of indefinite H.
    """
    lamH, Q = np.linalg.eigh(H)
    lt = (1.0 - tau) * lamH + tau * np.abs(lamH)
    inv = np.where(lt > 1e-12 * k, 1.0 / np.where(lt > 1e-12 * k, lt, 1.0), 0.0)
    Jf = k * np.einsum("nij,nj,nkj->nik", Q, inv, Q)
    Jraw = k * np.linalg.inv(H)
    n_indef = int(np.sum(lamH.min(axis=1) < 0))
    return Jf, Jraw, n_indef


def filtered_sigma_jacobian(ss: np.ndarray, mu: float, lam: float, k: float, tau: float):
    """d sigma*/d sigma_F = k H~(tau)^+ (eq. tr_ift) with H = H_psi(sigma*) + k I
    of the Neo-Hookean prox; (filtered, unfiltered, count of indefinite H)."""
    return filtered_inverse(k * np.eye(3) + nh_hess_sigma(ss, mu, lam), k, tau)


# ------------------------------------------------------ spectral differential

def _pair_coeffs(sF, ss, Jraw, corot: bool):
    """s_ij and t_ij for the three pairs (0,1), (0,2), (1,2)."""
    pairs = [(0, 1), (0, 2), (1, 2)]
    S = np.zeros((sF.shape[0], 3))
    T = np.zeros((sF.shape[0], 3))
    for c, (i, j) in enumerate(pairs):
        di = sF[:, i] - sF[:, j]
        sm = sF[:, i] + sF[:, j]
        if corot:
            S[:, c] = 0.0
        else:
            close = np.abs(di) <= 1e-8 * np.maximum(1.0, np.abs(sF[:, i]))
            ratio = (ss[:, i] - ss[:, j]) / np.where(close, 1.0, di)
            lim = Jraw[:, i, i] - Jraw[:, i, j]
            S[:, c] = np.where(close, lim, ratio)
        T[:, c] = (ss[:, i] + ss[:, j]) / np.where(np.abs(sm) > 1e-30, sm, 1e-30)
    return pairs, S, T


def spectral_differential(U, sF, V, ss, Jdiag, Jraw, dF, corot: bool):
    """dp for perturbations dF [n,3,3] of p = U diag(f(s)) V^T.

    With Mh = U^T dF V: diag(dp_hat) = Jdiag @ diag(Mh); for each pair i<j
      dp_hat_ij = s_ij (Mh_ij + Mh_ji)/2 + t_ij (Mh_ij - Mh_ji)/2
      dp_hat_ji = s_ij (Mh_ij + Mh_ji)/2 - t_ij (Mh_ij - Mh_ji)/2
    with s_ij = (f_i - f_j)/(s_i - s_j) (limit J_ii - J_ij at s_i = s_j) and
    t_ij = (f_i + f_j)/(s_i + s_j); dp = U dp_hat V^T. Corotated: f = 1.
    """
    Mh = np.einsum("nki,nkl,nlj->nij", U, dF, V)
    dph = np.zeros_like(Mh)
    if not corot:
        d = np.einsum("nij,nj->ni", Jdiag, np.diagonal(Mh, axis1=1, axis2=2))
        for i in range(3):
            dph[:, i, i] = d[:, i]
    pairs, S, T = _pair_coeffs(sF, ss, Jraw, corot)
    for c, (i, j) in enumerate(pairs):
        sym = 0.5 * (Mh[:, i, j] + Mh[:, j, i])
        skw = 0.5 * (Mh[:, i, j] - Mh[:, j, i])
        dph[:, i, j] = S[:, c] * sym + T[:, c] * skw
        dph[:, j, i] = S[:, c] * sym - T[:, c] * skw
    return np.einsum("nij,njk,nlk->nil", U, dph, V)


def dp_dF_matrix(U, sF, V, ss, Jdiag, Jraw, corot: bool) -> np.ndarray:
    """Explicit 9x9 dp/dF per element (row-major vec, index 3i+j)."""
    n = U.shape[0]
    D = np.zeros((n, 9, 9))
    for c in range(9):
        dF = np.zeros((n, 3, 3))
        dF[:, c // 3, c % 3] = 1.0
        D[:, :, c] = spectral_differential(U, sF, V, ss, Jdiag, Jraw, dF, corot).reshape(n, 9)
    return D
