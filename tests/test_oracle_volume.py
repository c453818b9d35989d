"""Pins of the oracle's corotated + volume composite (Sec. 4.1: a corotated
rotation step with a quadratic volume step; Sec. 7.2: weights w_0 = 2 mu,
w_1 = lambda): the volume step is the closest point of the unit-determinant
set, checked against an independent constrained minimiser, closed forms and
finite differences; the composite projection against the polar factor and
rotation invariance. (Zero force at rest, rigid motions, the fixed point,
monotone PD energy and the rollout gradients by finite differences are
pinned for this model in test_oracle_solver.py and test_oracle_adjoint.py.)"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import prox
from paper_2605_14526_b300.inputs import random_rotation


def _stretches(seed, n=40, lo=0.5, hi=1.6):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, 3))


def test_volume_step_lies_on_the_set_and_is_stationary():
    sF = _stretches(0)
    s, nu, it = prox.volume_project_sigma(sF)
    assert it < 80
    assert np.allclose(np.prod(s, axis=1), 1.0, atol=1e-13)
    # first-order condition: sigma - sigma_F = -nu grad J
    g = np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)
    assert np.allclose(s - sF, -nu[:, None] * g, atol=1e-12)


def test_volume_step_matches_independent_constrained_minimiser():
    sF = _stretches(1, n=12)
    s, _, _ = prox.volume_project_sigma(sF)
    for i in range(sF.shape[0]):
        res = scipy.optimize.minimize(lambda x: 0.5 * np.sum((x - sF[i]) ** 2), np.ones(3), method="SLSQP",
                                      constraints=[{"type": "eq", "fun": lambda x: np.prod(x) - 1.0}],
                                      bounds=[(1e-3, None)] * 3, options={"ftol": 1e-15, "maxiter": 500})
        assert res.success
        assert np.allclose(s[i], res.x, atol=1e-6)
        # and it is the nearer of the two
        assert 0.5 * np.sum((s[i] - sF[i]) ** 2) <= res.fun + 1e-12


def _global_min(a):
    """Brute force: the unit-determinant positive sheet parametrized by
    (log s_1, log s_2), BFGS from a grid of 81 starts; the best value."""
    f = lambda t: (np.exp(t[0]) - a[0]) ** 2 + (np.exp(t[1]) - a[1]) ** 2 + (np.exp(-t[0] - t[1]) - a[2]) ** 2
    best = np.inf
    for t0 in np.linspace(-3, 3, 9):
        for t1 in np.linspace(-3, 3, 9):
            r = scipy.optimize.minimize(f, [t0, t1], method="BFGS", options={"gtol": 1e-12})
            best = min(best, r.fun)
    return best


@pytest.mark.parametrize("kind", ["compressed", "inverted", "stretched"])
def test_volume_step_is_the_global_closest_point(kind):
    """Where the set has several stationary points (an inverted element's
    negative stretch; a stretched element, whose symmetric stationary point
    becomes a saddle once every stretch exceeds 2 and the nearest points
    flatten one axis) the step returns the nearest one."""
    rng = np.random.default_rng({"compressed": 6, "inverted": 7, "stretched": 8}[kind])
    for _ in range(6):
        if kind == "compressed":
            a = np.sort(rng.uniform(0.2, 1.0, 3))[::-1]
        elif kind == "inverted":
            a = np.sort(rng.uniform(0.1, 2.0, 3))[::-1]
            a[2] = -rng.uniform(0.0, a[1])
        else:
            a = np.sort(rng.uniform(1.5, 4.0, 3))[::-1]
        s, _, _ = prox.volume_project_sigma(a[None, :])
        assert np.all(s > 0) and abs(np.prod(s) - 1.0) < 1e-13
        d = np.sum((s[0] - a) ** 2)
        best = _global_min(a)
        assert d <= best + 1e-10 * max(1.0, best), (a, s, d, best)
    # an isotropic stretch of 3: (1, 1, 1) is stationary but not the minimum
    s, _, _ = prox.volume_project_sigma(np.array([[3.0, 3.0, 3.0]]))
    assert np.sum((s[0] - 3.0) ** 2) < 12.0 - 1.0


def test_volume_step_closed_forms():
    # isotropic stretch -> identity; a point of the set maps to itself
    s, _, _ = prox.volume_project_sigma(np.array([[1.3, 1.3, 1.3], [0.7, 0.7, 0.7]]))
    assert np.allclose(s, 1.0, atol=1e-14)
    on = np.array([[2.0, 0.5, 1.0], [1.25, 0.8, 1.0], [1.1, 1.0, 1.0 / 1.1]])
    s, nu, _ = prox.volume_project_sigma(on)
    assert np.allclose(s, on, atol=1e-14) and np.allclose(nu, 0.0, atol=1e-14)


def test_volume_jacobian_matches_finite_differences():
    sF = _stretches(2, n=10)
    s, nu, _ = prox.volume_project_sigma(sF)
    J = prox.volume_sigma_jacobian(s, nu)
    h = 1e-6
    for c in range(3):
        d = np.zeros_like(sF)
        d[:, c] = h
        fd = (prox.volume_project_sigma(sF + d)[0] - prox.volume_project_sigma(sF - d)[0]) / (2 * h)
        assert np.allclose(J[:, :, c], fd, atol=1e-7)
    assert np.allclose(J, np.transpose(J, (0, 2, 1)), atol=1e-12)   # a projection's Jacobian is symmetric


def test_composite_projection_rotation_invariant_and_reduces_to_polar():
    rng = np.random.default_rng(4)
    F = np.eye(3) + 0.3 * rng.standard_normal((20, 3, 3))
    a = np.full(20, 0.4)
    P, _ = prox.corot_volume_project(F, a)
    R = np.stack([random_rotation(rng) for _ in range(20)])
    P2, _ = prox.corot_volume_project(np.einsum("nij,njk->nik", R, F), a)
    assert np.allclose(P2, np.einsum("nij,njk->nik", R, P), atol=1e-12)
    # a = 1: the rotation step alone, the polar factor
    P1, _ = prox.corot_volume_project(F, np.ones(20))
    for i in range(20):
        Rp, _ = scipy.linalg.polar(F[i])
        assert np.allclose(P1[i], Rp, atol=1e-12)
    # at rest the projection is the identity
    Pi, _ = prox.corot_volume_project(np.tile(np.eye(3), (3, 1, 1)), np.full(3, 0.4))
    assert np.allclose(Pi, np.eye(3), atol=1e-14)


@pytest.mark.parametrize("a", [0.3, 0.8])
def test_composite_differential_matches_finite_differences(a):
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.25 * rng.standard_normal((8, 3, 3))
    av = np.full(8, a)
    _, (U, sF, V, ss, sv, nu) = prox.corot_volume_project(F, av)
    Jd = (1.0 - a) * prox.volume_sigma_jacobian(sv, nu)
    D = prox.dp_dF_matrix(U, sF, V, ss, Jd, Jd, corot=False)
    h = 1e-6
    for c in range(9):
        dF = np.zeros((8, 3, 3))
        dF[:, c // 3, c % 3] = h
        fd = (prox.corot_volume_project(F + dF, av)[0] - prox.corot_volume_project(F - dF, av)[0]) / (2 * h)
        assert np.allclose(D[:, :, c], fd.reshape(8, 9), atol=1e-7)
