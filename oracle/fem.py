"""FEM quantities, materials and the PD global operator (FP64, plain).

Sec. 3.1 (eq. lame, dynamics, freefall), Sec. 4.1 (eq. A_basic), Sec. 4.4
(eq. A_damped, rayleigh), Sec. 7.2 (energy-specific weights).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Rest:
    Dm_inv: np.ndarray   # [n_e,3,3]
    vol: np.ndarray      # [n_e]
    gradN: np.ndarray    # [n_e,4,3] shape-function gradients (rows)
    mass: np.ndarray     # [n_v] lumped


def rest_shape(X: np.ndarray, tets: np.ndarray, density: float) -> Rest:
    """Dm = [X1-X0, X2-X0, X3-X0]; V_e = det(Dm)/6; F = Ds Dm^-1.

    F = sum_a x_a (x) gradN_a with gradN_a = row (a-1) of Dm^-1 for a=1..3 and
    gradN_0 = -(sum of those rows). Lumped mass: density*V_e/4 to each corner.
    """
    x = X[tets]                                     # [n_e,4,3]
    Dm = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)  # columns
    det = np.linalg.det(Dm)
    if np.any(det <= 0):
        raise ValueError("rest tetrahedron with non-positive volume")
    Dm_inv = np.linalg.inv(Dm)
    vol = det / 6.0
    gradN = np.zeros((tets.shape[0], 4, 3))
    gradN[:, 1:, :] = Dm_inv
    gradN[:, 0, :] = -Dm_inv.sum(axis=1)
    mass = np.zeros(X.shape[0])
    np.add.at(mass, tets.ravel(), np.repeat(density * vol / 4.0, 4))
    return Rest(Dm_inv, vol, gradN, mass)


def deformation_gradient(rest: Rest, tets: np.ndarray, q: np.ndarray) -> np.ndarray:
    """F_e = G_e q = sum_a x_a gradN_a^T  ->  [n_e,3,3]."""
    return np.einsum("eai,eaj->eij", q[tets], rest.gradN)


def scatter_GT(rest: Rest, tets: np.ndarray, P: np.ndarray, coef: np.ndarray, n_v: int) -> np.ndarray:
    """sum_e coef_e G_e^T vec(P_e): vertex a of e receives coef_e * P_e gradN_a."""
    contrib = coef[:, None, None] * np.einsum("eij,eaj->eai", P, rest.gradN)  # [n_e,4,3]
    out = np.zeros((n_v, 3))
    np.add.at(out, tets.ravel(), contrib.reshape(-1, 3))
    return out


def lame(E: np.ndarray, nu: float):
    """eq. lame: mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu))."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


@dataclass
class Material:
    mu: np.ndarray
    lam: np.ndarray
    w: np.ndarray        # projective weight w_e
    beta: np.ndarray     # stiffness-damping coefficient beta_e
    mu_bar: float
    lam_bar: float
    k_bar: float
    mu_ref: float


def material(E: np.ndarray, nu: float, model: str, beta0: float, mu_ref: float | None = None) -> Material:
    """Weights and damping coefficients.

    eq. pd_weight / Sec. 7.2: the weight is the energy's rest tangent modulus,
    w_e = 2 mu_e for the corotated (rotation) energy and w_e = 2 mu_e + lambda_e
    for Neo-Hookean. The local prox uses the mesh-wide arithmetic means
    (eq. pd_weight_routed): mu_bar, lambda_bar and k_bar = mean(w_e).
    eq. rayleigh: beta_e = beta0 mu_e / mu_ref with mu_ref = max_e mu_e; a
    caller may pass a frozen mu_ref (the value fixed when A was factored).
    """
    mu, lam = lame(np.asarray(E, dtype=np.float64), nu)
    # corotated: rotation step only; Neo-Hookean: the single-energy weight;
    # corotated + volume composite: rotation step w_0 = 2 mu plus volume step
    # w_1 = lambda, registered together (Sec. 7.2), A carries w_0 + w_1
    w = 2.0 * mu if model == "corotated" else 2.0 * mu + lam
    if mu_ref is None:
        mu_ref = float(mu.max())
    beta = beta0 * mu / mu_ref
    return Material(mu, lam, w, beta, float(mu.mean()), float(lam.mean()), float(w.mean()), float(mu_ref))


def assemble_LA(rest: Rest, tets: np.ndarray, mat: Material, alpha: float, h: float) -> sp.csr_matrix:
    """Scalar PD operator L_A with A = L_A (x) I_3 (eq. A_damped).

    A = (1 + alpha h) M / h^2 + sum_e (w_e + beta_e/h) V_e G_e^T G_e, and
    G_e^T G_e = (N_e N_e^T) (x) I_3 with N_e the 4x3 matrix of gradN rows.
    """
    n_v = rest.mass.shape[0]
    c = (mat.w + mat.beta / h) * rest.vol
    Ke = c[:, None, None] * np.einsum("eai,ebi->eab", rest.gradN, rest.gradN)   # [n_e,4,4]
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    L = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n_v, n_v)).tocsr()
    L = L + sp.diags((1.0 + alpha * h) * rest.mass / h ** 2)
    return L.tocsr()


def assemble_B(rest: Rest, tets: np.ndarray, mat: Material) -> sp.csr_matrix:
    """Scalar stiffness-damping operator: B_beta = (sum_e beta_e V_e N_e N_e^T) (x) I_3."""
    n_v = rest.mass.shape[0]
    c = mat.beta * rest.vol
    Ke = c[:, None, None] * np.einsum("eai,ebi->eab", rest.gradN, rest.gradN)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n_v, n_v)).tocsr()


def G_matrix(rest: Rest, e: int) -> np.ndarray:
    """Explicit 9x12 G_e: vec(F) (row-major F_ij at 3i+j) from the 12 corner DoFs (3a+i)."""
    G = np.zeros((9, 12))
    for a in range(4):
        for i in range(3):
            for j in range(3):
                G[3 * i + j, 3 * a + i] = rest.gradN[e, a, j]
    return G
