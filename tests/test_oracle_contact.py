"""Pins of the contact oracle (oracle/contact.py) against what does not come
from the oracle itself: brute-force enumeration of the LCP's complementary
bases, an independent constrained minimiser for the friction QP, closed
forms (single contact, no friction, unbounded friction), the Delassus matrix
from a dense inverse, momentum balance of a converged contact step, and
central finite differences of a contact rollout's loss for the adjoint."""
import itertools

import numpy as np
import pytest
import scipy.optimize as so

from oracle import contact, solver
from paper_2605_14526_b300 import inputs


def _spd(rng, K, cond=30.0):
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return Q @ np.diag(np.geomspace(1.0, cond, K)) @ Q.T


@pytest.mark.parametrize("seed", range(6))
def test_lcp_matches_enumeration_of_complementary_bases(seed):
    rng = np.random.default_rng(seed)
    K = 6
    M = _spd(rng, K)
    q = rng.standard_normal(K)
    sols = []
    for bits in itertools.product([0, 1], repeat=K):
        a = np.nonzero(bits)[0]
        z = np.zeros(K)
        if a.size:
            z[a] = np.linalg.solve(M[np.ix_(a, a)], -q[a])
        w = M @ z + q
        if (z >= -1e-12).all() and (w >= -1e-12).all() and abs(z @ w) <= 1e-10:
            sols.append(z)
    assert len(sols) == 1    # a positive definite M has exactly one solution
    z = contact.lcp_murty(M, q)
    assert np.allclose(z, sols[0], atol=1e-12)


def test_friction_closed_forms():
    rng = np.random.default_rng(1)
    W = _spd(rng, 4)
    s = rng.standard_normal((4, 2))
    # no friction
    assert np.array_equal(contact.tresca(W, s, np.zeros(4)), np.zeros((4, 2)))
    # disks too large to bind: the unconstrained minimiser -W^-1 s
    lam = contact.tresca(W, s, np.full(4, 1e6))
    assert np.allclose(lam, -np.linalg.solve(W, s), atol=1e-10)
    # one contact: the minimiser -s/W clipped to the disk along -s
    for rho in (0.1, 100.0):
        l1 = contact.tresca(np.array([[2.0]]), np.array([[3.0, 4.0]]), np.array([rho]))
        free = -np.array([3.0, 4.0]) / 2.0
        want = free if np.linalg.norm(free) <= rho else -rho * np.array([0.6, 0.8])
        assert np.allclose(l1[0], want, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_friction_matches_independent_constrained_minimiser(seed):
    rng = np.random.default_rng(10 + seed)
    K = 4
    W = _spd(rng, K, 10.0)
    s = rng.standard_normal((K, 2))
    rho = rng.uniform(0.1, 0.8, K)
    lam = contact.tresca(W, s, rho)

    def f(x):
        L = x.reshape(K, 2)
        return 0.5 * np.sum(L * (W @ L)) + np.sum(s * L)

    cons = [{"type": "ineq", "fun": (lambda x, c=c: rho[c] ** 2 - x[2 * c] ** 2 - x[2 * c + 1] ** 2)} for c in range(K)]
    res = so.minimize(f, np.zeros(2 * K), method="SLSQP", constraints=cons, options={"ftol": 1e-15, "maxiter": 1000})
    assert f(lam.ravel()) <= res.fun + 1e-10
    assert np.allclose(lam.ravel(), res.x, atol=1e-5)
    assert contact.tresca_kkt(W, s, rho, lam) <= 1e-9


def _tiny_pad(**kw):
    base = dict(nx=3, ny=3, nz=2, footprint=1, steps=1, box_steps=2, travel=0.002, E_core=1e5)
    base.update(kw)
    return inputs.contact_pad(**base)


def test_delassus_equals_dense_inverse():
    sc = _tiny_pad()
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    Ainv = np.linalg.inv(pb.LA_ff.toarray())
    assert np.allclose(cp.W, Ainv[np.ix_(cp.pos, cp.pos)], rtol=1e-12, atol=0)


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_contact_step_momentum_balance(mu):
    # sum over vertices of A q - b(q) is (1 + alpha h) M q / h^2 - M q~ / h^2 -
    # alpha M q_t / h (elastic and stiffness-damping forces sum to zero), and
    # it equals the total contact impulse J^T lambda
    sc = _tiny_pad()
    sc.contact.mu = mu
    rng = np.random.default_rng(4)
    v0 = 0.05 * rng.standard_normal(sc.X.shape)
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    q, lam_n, lam_f, k = contact.step(pb, cp, sc.x0, v0, sc.f_ext[0], 0, tol=1e-13)
    m = pb.rest.mass[:, None]
    qt = solver.inertial_target(pb, sc.x0, v0, sc.f_ext[0])
    lhs = (m * ((1 + pb.alpha * pb.h) * q - qt - pb.alpha * pb.h * sc.x0)).sum(0) / pb.h ** 2
    imp = np.array([lam_f[:, 0].sum(), lam_f[:, 1].sum(), (cp.normal * lam_n).sum()])
    assert np.allclose(lhs, imp, rtol=1e-7, atol=1e-9 * np.abs(imp).max())
    # complementarity on the converged positions: no penetration, no pull
    z = q[cp.verts, 2]
    gap = cp.normal * (z - cp.heights(0))
    assert gap.min() >= -1e-12
    assert np.all(lam_n >= 0) and np.abs(lam_n * gap).max() <= 1e-12 * max(lam_n.max(), 1.0)
    if mu == 0.0:
        assert np.array_equal(lam_f, np.zeros_like(lam_f))


def _loss(sc, pb, cp, v0, E=None):
    if E is not None:
        pb = solver.build_problem(sc, E=E)
        cp = contact.ContactProblem(pb, sc.contact)
    q, v = sc.x0.copy(), v0.copy()
    recs = []
    for t in range(sc.steps):
        qn, ln, lf, _ = contact.step(pb, cp, q, v, sc.f_ext[0], t, tol=1e-14)
        recs.append({"q_t": q, "v_t": v, "q_next": qn, "lam_n": ln, "lam_f": lf})
        v = (qn - q) / pb.h
        q = qn
    d = q - sc.target
    return 0.5 * float(np.sum(d * d)), q, recs


@pytest.mark.parametrize("mu", [0.0, 50.0])
def test_contact_adjoint_matches_finite_differences(mu):
    # frictionless (no friction rows) and all-stick (every friction row an
    # equality): the fixed-active-set adjoint is then the exact derivative
    sc = _tiny_pad(steps=2)
    sc.contact.mu = mu
    rng = np.random.default_rng(5)
    v0 = 0.02 * rng.standard_normal(sc.X.shape)
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    L, qT, recs = _loss(sc, pb, cp, v0)
    act, stick = contact.active_sets(cp, recs[-1]["lam_n"], recs[-1]["q_next"], recs[-1]["q_t"])
    assert act.any()
    if mu > 0:
        assert np.array_equal(act, stick)
    g = contact.rollout_backward(pb, cp, recs, qT - sc.target, np.zeros_like(qT))
    dv = rng.standard_normal(sc.X.shape)
    eps = 1e-6
    fd = (_loss(sc, pb, cp, v0 + eps * dv)[0] - _loss(sc, pb, cp, v0 - eps * dv)[0]) / (2 * eps)
    assert abs(fd - np.sum(g.dv0 * dv)) <= 1e-5 * abs(fd) + 1e-12
    dx = rng.standard_normal(sc.X.shape)
    sc2 = sc.replace(x0=sc.x0 + eps * dx)
    sc3 = sc.replace(x0=sc.x0 - eps * dx)
    fdx = (_loss(sc2, pb, cp, v0)[0] - _loss(sc3, pb, cp, v0)[0]) / (2 * eps)
    assert abs(fdx - np.sum(g.dx0 * dx)) <= 1e-5 * abs(fdx) + 1e-12
    e = int(np.argmax(np.abs(g.dE)))
    E1, E2 = sc.E.copy(), sc.E.copy()
    hE = 1e-6 * sc.E[e]
    E1[e] += hE
    E2[e] -= hE
    fde = (_loss(sc, pb, cp, v0, E1)[0] - _loss(sc, pb, cp, v0, E2)[0]) / (2 * hE)
    assert abs(fde - g.dE[e]) <= 1e-4 * abs(fde) + 1e-15


def _exact_split(cp, mu, lam_n, lam_f):
    """The active sets by the multipliers of an exact solution: normal-active
    where lam_n > 0 (Murty's pivoting leaves the non-basic lam_n exactly 0),
    sticking where the friction lies strictly inside its disk,
    |lam_f| < mu lam_n (a sliding contact's friction sits on the rim up to
    rounding, hence the relative margin 1e-9)."""
    act = lam_n > 0.0
    ratio = np.linalg.norm(lam_f, axis=1) / np.maximum(mu * lam_n, 1e-300)
    stick = act & (ratio < 1.0 - 1e-9) & (mu > 0.0)
    return act, stick


def _lift_off_velocity(sc, rng):
    v0 = 0.02 * rng.standard_normal(sc.X.shape)
    v0[:, 2] += np.where(sc.X[:, 0] > 0.5 * sc.X[:, 0].max(), 1.0, -0.2)
    return v0


@pytest.mark.parametrize("case", ["frictionless", "sliding", "sticking", "lift_off", "parity_pad"])
def test_active_set_thresholds_equal_exact_multiplier_split(case):
    # The adjoint's active sets are read with thresholds (lam_n above 1e-9 of
    # the step's total, slip at most 1e-7 of the bounding-box diagonal).
    # On the oracle's exact LCP / Tresca solutions they must be the split of
    # Sec. 4.6's complementarity itself: lam_n > 0, |lam_f| < mu lam_n.
    rng = np.random.default_rng(5)
    if case == "parity_pad":    # the pad of the GPU contact tests
        sc = inputs.contact_pad(nx=8, ny=8, nz=5, footprint=4, steps=2, box_steps=6, travel=0.004, E_core=1e6,
                                seed=27)
    else:
        sc = _tiny_pad(steps=2)
        sc.contact.mu = {"frictionless": 0.0, "sliding": 0.5, "sticking": 50.0, "lift_off": 0.5}[case]
        sc = sc.replace(v0=_lift_off_velocity(sc, rng) if case == "lift_off" else 0.02 * rng.standard_normal(sc.X.shape))
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    _, _, recs, _ = contact.rollout(pb, sc, cp)
    seen_inactive = seen_stick = seen_slide = False
    for r in recs:
        act, stick = contact.active_sets(cp, r["lam_n"], r["q_next"], r["q_t"])
        act_x, stick_x = _exact_split(cp, sc.contact.mu, r["lam_n"], r["lam_f"])
        assert np.array_equal(act, act_x)
        assert np.array_equal(stick, stick_x)
        seen_inactive |= bool((~act).any())
        seen_stick |= bool(stick.any())
        seen_slide |= bool((act & ~stick).any())
    # each case exercises the branch it is named for
    want = {"frictionless": seen_slide, "sliding": seen_stick and seen_slide, "sticking": seen_stick,
            "lift_off": seen_inactive and seen_stick and seen_slide, "parity_pad": seen_stick and seen_slide}
    assert want[case]
