"""Pins of the oracle's local step (Sec. 4.1) and trust-region filter (Sec. 4.3).

Each check compares the oracle against something other than itself: closed
forms, invariances, an independent library routine, finite differences.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import prox
from paper_2605_14526_b300.inputs import random_rotation

MU, LAM = 1.0e5, 3.0e5
K = 2 * MU + LAM


def _rand_F(rng, n, scale=0.25):
    return np.eye(3)[None] + scale * rng.standard_normal((n, 3, 3))


def test_svd_rv_reconstructs_and_is_rotation_variant():
    rng = np.random.default_rng(0)
    F = _rand_F(rng, 50, 0.8)
    U, s, V = prox.svd_rv(F)
    assert np.allclose(np.einsum("nij,nj,nkj->nik", U, s, V), F, atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0) and np.allclose(np.linalg.det(V), 1.0)
    assert np.allclose(np.einsum("nki,nkj->nij", U, U), np.eye(3), atol=1e-13)
    assert np.all(s[:, :2] > 0)
    assert np.allclose(np.sign(s[:, 2]), np.sign(np.linalg.det(F)))


def test_corotated_projection_is_scipy_polar_factor():
    rng = np.random.default_rng(1)
    F = _rand_F(rng, 20, 0.3)
    F = F[np.linalg.det(F) > 0]
    R = prox.corotated_project(F)
    for i in range(F.shape[0]):
        Rp, _ = scipy.linalg.polar(F[i])
        assert np.allclose(R[i], Rp, atol=1e-12)


def test_nh_energy_F_and_sigma_forms_agree():
    rng = np.random.default_rng(2)
    F = _rand_F(rng, 30, 0.2)
    F = F[np.linalg.det(F) > 0]
    U, s, V = prox.svd_rv(F)
    assert np.allclose(prox.nh_psi_F(F, MU, LAM), prox.nh_psi_sigma(s, MU, LAM), rtol=1e-11, atol=1e-6)


def test_nh_gradient_and_hessian_by_finite_differences():
    """Pins the reading of eq. nh_hessian_stretch (sigma^-2, not sigma^-4)."""
    rng = np.random.default_rng(3)
    s = 1.0 + 0.2 * rng.standard_normal((10, 3))
    h = 1e-6
    g = prox.nh_grad_sigma(s, MU, LAM)
    H = prox.nh_hess_sigma(s, MU, LAM)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        gfd = (prox.nh_psi_sigma(s + e, MU, LAM) - prox.nh_psi_sigma(s - e, MU, LAM)) / (2 * h)
        Hfd = (prox.nh_grad_sigma(s + e, MU, LAM) - prox.nh_grad_sigma(s - e, MU, LAM)) / (2 * h)
        assert np.allclose(g[:, i], gfd, rtol=1e-7, atol=1e-3)
        assert np.allclose(H[:, :, i], Hfd, rtol=1e-7, atol=1e-2)


def test_nh_rest_closed_forms():
    one = np.ones((1, 3))
    assert np.allclose(prox.nh_grad_sigma(one, MU, LAM), 0.0)
    assert np.allclose(prox.nh_hess_sigma(one, MU, LAM)[0], 2 * MU * np.eye(3) + LAM * np.ones((3, 3)))
    ss, _ = prox.nh_prox_sigma(one, MU, LAM, K)
    assert np.allclose(ss, 1.0, atol=1e-14)


def test_nh_prox_closed_form_when_lambda_zero():
    """With lambda = 0 the stretch problem decouples: (k+mu) s^2 - k sF s - mu = 0."""
    rng = np.random.default_rng(4)
    sF = 0.5 + rng.random((40, 3))
    sF[:5, 2] = -0.3 * rng.random(5)           # inverted inputs still give s* > 0
    mu, k = 2.0e4, 7.0e4
    ss, _ = prox.nh_prox_sigma(sF, mu, 0.0, k)
    exact = (k * sF + np.sqrt((k * sF) ** 2 + 4 * (k + mu) * mu)) / (2 * (k + mu))
    assert np.allclose(ss, exact, rtol=1e-12)


def test_nh_prox_stationary_and_minimal():
    rng = np.random.default_rng(5)
    sF = 1.0 + 0.25 * rng.standard_normal((200, 3))
    ss, _ = prox.nh_prox_sigma(sF, MU, LAM, K)
    g = K * (ss - sF) + prox.nh_grad_sigma(ss, MU, LAM)
    assert np.abs(g).max() <= 1e-12 * K

    def f(x):
        return 0.5 * K * np.sum((x - sF) ** 2, axis=1) + prox.nh_psi_sigma(x, MU, LAM)
    f0 = f(ss)
    for _ in range(20):                           # brute force: no nearby point is lower
        d = 1e-4 * rng.standard_normal(ss.shape)
        assert np.all(f(ss + d) >= f0 - 1e-9 * np.abs(f0))


@pytest.mark.parametrize("model", ["nh", "corot"])
def test_projection_rotation_invariance(model):
    rng = np.random.default_rng(6)
    F = _rand_F(rng, 30, 0.3)
    R = np.stack([random_rotation(rng) for _ in range(30)])
    Q = np.stack([random_rotation(rng) for _ in range(30)])

    def p(A):
        if model == "corot":
            return prox.corotated_project(A)
        return prox.nh_project(A, MU, LAM, K)[0]
    assert np.allclose(p(np.einsum("nij,njk->nik", R, F)), np.einsum("nij,njk->nik", R, p(F)), atol=1e-11)
    assert np.allclose(p(np.einsum("nij,njk->nik", F, Q)), np.einsum("nij,njk->nik", p(F), Q), atol=1e-11)
    assert np.allclose(p(np.eye(3)[None]), np.eye(3), atol=1e-13)


@pytest.mark.parametrize("model", ["nh", "corot"])
def test_projection_differential_by_finite_differences(model):
    rng = np.random.default_rng(7)
    n = 12
    F = _rand_F(rng, n, 0.2)
    F[0] = np.diag([1.1, 1.1, 0.95])            # repeated singular values: limit branch
    U, s, V = prox.svd_rv(F)
    corot = model == "corot"
    if corot:
        ss = np.ones_like(s)
        z = np.zeros((n, 3, 3))
        D = prox.dp_dF_matrix(U, s, V, ss, z, z, True)

        def p(A):
            return prox.corotated_project(A)
    else:
        ss, _ = prox.nh_prox_sigma(s, MU, LAM, K)
        _, Jraw, _ = prox.filtered_sigma_jacobian(ss, MU, LAM, K, 0.0)
        D = prox.dp_dF_matrix(U, s, V, ss, Jraw, Jraw, False)

        def p(A):
            return prox.nh_project(A, MU, LAM, K)[0]
    h = 1e-6
    for c in range(9):
        dF = np.zeros((n, 3, 3))
        dF[:, c // 3, c % 3] = h
        fd = ((p(F + dF) - p(F - dF)) / (2 * h)).reshape(n, 9)
        assert np.allclose(D[:, :, c], fd, atol=2e-6), (c, np.abs(D[:, :, c] - fd).max())
    assert np.allclose(D, np.transpose(D, (0, 2, 1)), atol=1e-10)     # Hessian of an envelope


def test_trust_region_blend_identities():
    """eq. tr_blend at tau = 0, 1/2, 1 equals none / clamp / abs (built independently)."""
    rng = np.random.default_rng(8)
    Q = np.stack([random_rotation(rng) for _ in range(10)])
    lam = rng.standard_normal((10, 3)) * 3.0
    H = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    assert np.allclose(prox.tr_blend(H, 0.0), H, atol=1e-12)
    assert np.allclose(prox.tr_blend(H, 0.5), np.einsum("nij,nj,nkj->nik", Q, np.maximum(lam, 0), Q), atol=1e-12)
    assert np.allclose(prox.tr_blend(H, 1.0), np.einsum("nij,nj,nkj->nik", Q, np.abs(lam), Q), atol=1e-12)


def test_filtered_jacobian_is_exact_when_definite():
    rng = np.random.default_rng(9)
    ss = 1.0 + 0.1 * rng.standard_normal((50, 3))
    for tau in (0.0, 0.5, 1.0):
        Jf, Jraw, nind = prox.filtered_sigma_jacobian(ss, MU, LAM, K, tau)
        assert nind == 0
        assert np.allclose(Jf, Jraw, rtol=1e-10, atol=1e-12)


def test_filtered_jacobian_indefinite_case():
    """Anisotropic expansion makes H_prox indefinite; clamp zeroes the negative
    direction and abs flips it (pseudo-inverse reading of eq. tr_ift)."""
    mu, lam = 1.0, 200.0
    k = 0.05
    ss = np.array([[0.3, 3.0, 3.0]])
    H = k * np.eye(3) + prox.nh_hess_sigma(ss, mu, lam)
    ev, Qe = np.linalg.eigh(H[0])
    assert ev.min() < 0
    Jc, _, nind = prox.filtered_sigma_jacobian(ss, mu, lam, k, 0.5)
    Ja, _, _ = prox.filtered_sigma_jacobian(ss, mu, lam, k, 1.0)
    assert nind == 1
    v = Qe[:, 0]
    assert np.allclose(Jc[0] @ v, 0.0, atol=1e-12)
    assert np.allclose(Ja[0] @ v, k / abs(ev[0]) * v, rtol=1e-10)
