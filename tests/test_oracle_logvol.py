"""Pins of the oracle's log-volume barrier variant (Sec. 4.1, volume-barrier
surrogate, eq. pd_log_volume, registered with w_e = lambda_e next to the
corotated rotation step) against the matrix-space definition of its prox,
closed forms at rest, finite differences and invariants."""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import fem, prox, solver
from paper_2605_14526_b300 import inputs
from paper_2605_14526_b300.inputs import random_rotation


def _matrix_prox(F, mu, lam):
    """argmin over 3x3 P with det P > 0 of lambda/2 ||P - F||^2 + phi_log(P),
    phi_log(P) = -mu ln det P + lambda/2 (ln det P)^2 (the sum of the log
    stretches of P is ln det P), by BFGS in the 9 entries of P from the
    positive-stretch reflection of F. Independent of the stretch-space
    Newton: no SVD of the iterate, no stretch formulas."""
    U, s, Vt = np.linalg.svd(F)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        U[:, 2] = -U[:, 2]
    P0 = U @ np.diag(np.maximum(s, 0.3)) @ Vt

    def f(x):   # the objective divided by lambda
        P = x.reshape(3, 3)
        d = np.linalg.det(P)
        if d <= 0:
            return 1e30, np.zeros(9)
        L = np.log(d)
        val = 0.5 * np.sum((P - F) ** 2) - mu / lam * L + 0.5 * L * L
        g = (P - F) + (L - mu / lam) * np.linalg.inv(P).T
        return val, g.ravel()

    res = scipy.optimize.minimize(f, P0.ravel(), jac=True, method="BFGS",
                                  options={"gtol": 1e-12, "maxiter": 5000})
    x = res.x
    for _ in range(6):   # polish: Newton on a central-difference Hessian of the gradient
        H = np.stack([(f(x + 1e-6 * e)[1] - f(x - 1e-6 * e)[1]) / 2e-6 for e in np.eye(9)], axis=1)
        x = x - np.linalg.solve(0.5 * (H + H.T), f(x)[1])
    assert np.abs(f(x)[1]).max() < 1e-12
    return x.reshape(3, 3), f(x)[0] * lam


def _cases():
    rng = np.random.default_rng(31)
    F = [np.eye(3) + 0.3 * rng.standard_normal((3, 3)) for _ in range(6)]
    F.append(np.diag([0.5, 0.45, 0.4]))                     # compressed
    F.append(np.diag([1.8, 1.4, 1.2]))                      # stretched
    F.append(random_rotation(rng) @ np.diag([1.1, 0.9, -0.3]))   # inverted
    return np.stack(F)


@pytest.mark.parametrize("nu", [0.3, 0.45])
def test_barrier_prox_is_the_matrix_space_minimiser(nu):
    F = _cases()
    mu, lam = fem.lame(np.full(F.shape[0], 2e5), nu)
    U, sF, V = prox.svd_rv(F)
    sb, it = prox.logvol_prox_sigma(sF, prox.logvol_ratio(mu, lam))
    assert np.all(it < 40) and np.all(sb > 0)
    Pb = prox.compose(U, sb, V)
    for i in range(F.shape[0]):
        Pm, fm = _matrix_prox(F[i], mu[i], lam[i])
        L = np.log(np.prod(sb[i]))
        fo = 0.5 * lam[i] * np.sum((Pb[i] - F[i]) ** 2) - mu[i] * L + 0.5 * lam[i] * L * L
        assert fo <= fm + 1e-12 * abs(fm)
        assert np.allclose(Pb[i], Pm, atol=1e-11)


def test_barrier_keeps_inverted_elements_positive():
    """The barrier diverges as J -> 0+: an inverted F maps to det p_b > 0."""
    rng = np.random.default_rng(2)
    s = np.stack([np.abs(rng.normal(1.0, 0.3, 40)), np.abs(rng.normal(0.8, 0.3, 40)),
                  -np.abs(rng.normal(0.3, 0.2, 40))], axis=1)
    s = -np.sort(-np.abs(s), axis=1) * np.array([1.0, 1.0, -1.0])
    sb, _ = prox.logvol_prox_sigma(s, 0.2)
    assert np.all(sb > 0)


def _rest_stretch(r):
    """The uniform stretch s of the barrier's prox at sigma_F = (1, 1, 1):
    by symmetry sigma_b = s (1, 1, 1) and the matrix-space stationarity
    lambda (s - 1) I + (3 lambda ln s - mu) I / s = 0 reads
    s (s - 1) + 3 ln s - r = 0, one root on s > 0."""
    return scipy.optimize.brentq(lambda s: s * (s - 1.0) + 3.0 * np.log(s) - r, 0.5, 2.0, xtol=1e-15)


@pytest.mark.parametrize("nu", [0.3, 0.45, 0.499])
def test_rest_stretch_closed_form(nu):
    """As printed, the barrier's gradient at sigma = 1 is -mu per stretch: its
    prox at rest is a uniform stretch s > 1 (about 1.028 at nu = 0.45),
    tending to 1 as nu -> 1/2."""
    mu, lam = fem.lame(np.array([3e5]), nu)
    r = prox.logvol_ratio(mu, lam)
    sb, _ = prox.logvol_prox_sigma(np.ones((1, 3)), r)
    s = _rest_stretch(float(r[0]))
    assert np.allclose(sb, s, rtol=1e-13)
    if nu == 0.45:
        assert abs(s - 1.028) < 5e-4
    assert s > 1.0 and (nu < 0.49 or s - 1.0 < 1e-3)


def test_rest_residual_is_the_uniform_outward_stretch():
    """At q = X every element has F = I and p = (a + (1 - a) s) I, so the
    global residual A X - b(X) is -(1 - a)(s - 1) sum_e w_e V_e G_e^T I: a body
    at rest is pushed outward by the printed barrier (the reading that keeps
    the variant opt-in)."""
    sc = inputs.tiny_block(n=2, model="corotated_logvol").replace(gravity=np.zeros(3), beta0=0.0)
    pb = solver.build_problem(sc)
    z = np.zeros_like(sc.X)
    b0 = solver.rhs_const(pb, sc.X, z, z)
    res = pb.LA_ff @ sc.X[pb.free] - solver.free_rhs(pb, solver.rhs(pb, b0, sc.X))
    a = solver.rotation_share(pb)
    s = _rest_stretch(float(solver.logvol_ratio(pb)[0]))
    P = np.tile(np.eye(3), (sc.n_e, 1, 1)) * ((1.0 - a) * (s - 1.0))[:, None, None]
    push = fem.scatter_GT(pb.rest, pb.tets, P, pb.mat.w * pb.rest.vol, pb.n_v)[pb.free]
    assert np.linalg.norm(push) > 1.0
    assert np.allclose(res, -push, atol=1e-9 * np.abs(push).max())


def test_barrier_jacobians_match_finite_differences():
    rng = np.random.default_rng(8)
    sF = np.sort(np.abs(rng.normal(1.0, 0.25, (10, 3))), axis=1)[:, ::-1].copy()
    r = 0.15
    sb, _ = prox.logvol_prox_sigma(sF, r)
    Jf, Jraw, n_indef = prox.logvol_sigma_jacobian(sb, r, 0.5)
    assert n_indef == 0 and np.allclose(Jf, Jraw, atol=1e-13)
    h = 1e-6
    for c in range(3):
        d = np.zeros_like(sF)
        d[:, c] = h
        fd = (prox.logvol_prox_sigma(sF + d, r)[0] - prox.logvol_prox_sigma(sF - d, r)[0]) / (2 * h)
        assert np.allclose(Jraw[:, :, c], fd, atol=1e-8)
    # d sigma_b / d r = H^-1 (1/sigma_b)
    fd = (prox.logvol_prox_sigma(sF, r + h)[0] - prox.logvol_prox_sigma(sF, r - h)[0]) / (2 * h)
    assert np.allclose(np.einsum("nij,nj->ni", Jraw, 1.0 / sb), fd, atol=1e-8)


def test_barrier_filter_drops_negative_curvature():
    """A strongly stretched, thin stretch triple makes I + Hess(phi_log/lambda)
    indefinite (ln J - r > sigma_min^2): tau = 1/2 answers 0 along the negative
    eigen-direction, tau = 1 uses |eigenvalue| (eq. tr_blend)."""
    sb = np.array([[3.0, 3.0, 0.5]])
    r = 0.1
    H = np.eye(3) + prox.logvol_hess_sigma(sb, np.array([r]))
    lam, Q = np.linalg.eigh(H[0])
    assert lam[0] < 0
    Jh, _, n = prox.logvol_sigma_jacobian(sb, r, 0.5)
    J1, _, _ = prox.logvol_sigma_jacobian(sb, r, 1.0)
    assert n == 1
    assert np.allclose(Jh[0] @ Q[:, 0], 0.0, atol=1e-12)
    assert np.allclose(J1[0] @ Q[:, 0], Q[:, 0] / abs(lam[0]), atol=1e-12)


def test_barrier_projection_rotation_invariant_and_reduces_to_polar():
    rng = np.random.default_rng(4)
    F = np.eye(3) + 0.3 * rng.standard_normal((20, 3, 3))
    a = np.full(20, 0.4)
    P, _ = prox.corot_logvol_project(F, a, 0.2)
    R = np.stack([random_rotation(rng) for _ in range(20)])
    P2, _ = prox.corot_logvol_project(np.einsum("nij,njk->nik", R, F), a, 0.2)
    assert np.allclose(P2, np.einsum("nij,njk->nik", R, P), atol=1e-12)
    P1, _ = prox.corot_logvol_project(F, np.ones(20), 0.2)
    for i in range(20):
        Rp, _ = scipy.linalg.polar(F[i])
        assert np.allclose(P1[i], Rp, atol=1e-12)


@pytest.mark.parametrize("a", [0.3, 0.8])
def test_barrier_composite_differential_matches_finite_differences(a):
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.25 * rng.standard_normal((8, 3, 3))
    av = np.full(8, a)
    r = 0.12
    _, (U, sF, V, ss, sb) = prox.corot_logvol_project(F, av, r)
    _, Jraw, _ = prox.logvol_sigma_jacobian(sb, r, 0.5)
    Jd = (1.0 - a) * Jraw
    D = prox.dp_dF_matrix(U, sF, V, ss, Jd, Jd, corot=False)
    h = 1e-6
    for c in range(9):
        dF = np.zeros((8, 3, 3))
        dF[:, c // 3, c % 3] = h
        fd = (prox.corot_logvol_project(F + dF, av, r)[0] - prox.corot_logvol_project(F - dF, av, r)[0]) / (2 * h)
        assert np.allclose(D[:, :, c], fd.reshape(8, 9), atol=1e-7)
