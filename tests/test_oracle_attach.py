"""Pins of the contact oracle's bilateral attachment rows (Sec. 4.6: a vertex
held at a prescribed target by three equality rows with free multipliers)
against what does not come from the oracle itself: brute-force enumeration
of the mixed LCP's bases, an independent constrained minimiser for friction
with free rows, Dirichlet pinning through the factor (an attachment at the
rest position is the same constraint), the targets met at every step, and
central finite differences of a rollout's loss."""
import itertools

import numpy as np
import pytest
import scipy.optimize as so

from oracle import adjoint, contact, solver
from paper_2605_14526_b300 import inputs


def _spd(rng, K, cond=30.0):
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return Q @ np.diag(np.geomspace(1.0, cond, K)) @ Q.T


@pytest.mark.parametrize("seed", range(5))
def test_mixed_lcp_matches_enumeration(seed):
    rng = np.random.default_rng(seed)
    K = 7
    M = _spd(rng, K)
    q = rng.standard_normal(K)
    free = np.zeros(K, dtype=bool)
    free[rng.choice(K, 3, replace=False)] = True
    N = np.nonzero(~free)[0]
    sols = []
    for bits in itertools.product([0, 1], repeat=N.size):
        basic = free.copy()
        basic[N[np.array(bits, dtype=bool)]] = True
        a = np.nonzero(basic)[0]
        z = np.zeros(K)
        z[a] = np.linalg.solve(M[np.ix_(a, a)], -q[a])
        w = M @ z + q
        if (z[N] >= -1e-12).all() and (w[N] >= -1e-12).all() and abs(z[N] @ w[N]) <= 1e-10:
            sols.append(z)
    assert len(sols) == 1
    z = contact.mixed_lcp(M, q, free)
    assert np.allclose(z, sols[0], atol=1e-12)
    assert contact.mixed_lcp_kkt(M, q, z, free) <= 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_friction_with_free_rows_matches_constrained_minimiser(seed):
    rng = np.random.default_rng(10 + seed)
    K = 5
    W = _spd(rng, K, cond=10.0)
    s = rng.standard_normal((K, 2))
    rho = np.abs(rng.normal(0.3, 0.2, K))
    rho[[1, 3]] = np.inf
    lam = contact.tresca(W, s, rho)

    def f(x):
        L = x.reshape(K, 2)
        return 0.5 * np.sum(L * (W @ L)) + np.sum(s * L)

    cons = [{"type": "ineq", "fun": (lambda x, c=c: rho[c] ** 2 - x[2 * c] ** 2 - x[2 * c + 1] ** 2)}
            for c in range(K) if np.isfinite(rho[c])]
    ref = so.minimize(f, np.zeros(2 * K), constraints=cons, method="SLSQP",
                      options={"ftol": 1e-15, "maxiter": 1000}).x.reshape(K, 2)
    assert np.allclose(lam, ref, atol=1e-6)
    # a single free row alone is the unconstrained minimiser -W^-1 s
    lam1 = contact.tresca(W[:1, :1], s[:1], np.array([np.inf]))
    assert np.allclose(lam1, -s[:1] / W[0, 0], atol=1e-14)


def _pinned_bar():
    return inputs.hetero_bar(nx=4, ny=2, nz=2, block=2, steps=4, omega0=4.0)


def _attached_version(sc):
    """The same scene with its pins released and each former pin attached at
    its rest position (zero travel), no obstacle contacts."""
    P = np.nonzero(sc.pinned)[0]
    v0 = sc.v0.copy()
    v0[P] = 0.0
    spec = inputs.ContactSpec(ground=np.zeros(0, dtype=np.int64), box=np.zeros(0, dtype=np.int64), ground_z=0.0,
                              box_z0=0.0, box_travel=0.0, box_steps=1, mu=0.0, attach=P,
                              attach_p0=sc.X[P].copy(), attach_travel=np.zeros((P.size, 3)), attach_steps=1)
    att = sc.replace(pinned=np.zeros_like(sc.pinned), v0=v0)
    att.contact = spec
    return att, P


@pytest.mark.parametrize("model", ["neohookean", "corotated"])
def test_attachment_at_rest_equals_pinning(model):
    """Holding the former Dirichlet vertices by attachment rows at their rest
    positions gives the pinned rollout's positions and gradients: the pins
    act through the factor (eliminated columns), the attachments through
    multipliers on the unpinned operator."""
    sc = _pinned_bar().replace(model=model)
    att, P = _attached_version(sc)
    sc = sc.replace(v0=att.v0)
    pb = solver.build_problem(sc)
    qT, vT, recs = solver.rollout(pb, sc, mode="exact")
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    g = adjoint.rollout_backward(pb, recs, dq, dv)

    pa = solver.build_problem(att, mu_ref=pb.mat.mu_ref)
    qa, va, ra, cp = contact.rollout(pa, att)
    assert np.abs(qa - qT).max() <= 1e-10 * np.abs(qT).max()
    for t, r in enumerate(ra):
        assert np.abs(r["q_next"][P] - sc.X[P]).max() <= 1e-13
    _, dqa, dva = adjoint.loss_and_grad(att, pa, qa, va)
    ga = contact.rollout_backward(pa, cp, ra, dqa, dva)
    free = np.nonzero(sc.pinned == 0)[0]
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(ga.dE, g.dE) < 1e-7
    assert abs(ga.dnu - g.dnu) < 1e-7 * abs(g.dnu)
    assert rel(ga.dx0[free], g.dx0[free]) < 1e-7
    assert rel(ga.dv0[free], g.dv0[free]) < 1e-7


def _pad_with_attachments(mu, steps=2):
    """The tiny contact pad (ground below, box pressing its top centre) with
    two top-corner vertices attached and pulled sideways and up by 1 mm
    over the rollout."""
    sc = inputs.contact_pad(nx=3, ny=3, nz=2, footprint=1, steps=steps, box_steps=2, travel=0.002, E_core=1e5)
    X = sc.X
    top = np.nonzero(np.isclose(X[:, 2], X[:, 2].max()))[0]
    taken = set(sc.contact.ground.tolist()) | set(sc.contact.box.tolist())
    corners = [v for v in top if v not in taken and (np.isclose(X[v, 0], X[:, 0].min()) or np.isclose(X[v, 0], X[:, 0].max()))]
    A = np.array(sorted(corners)[:2], dtype=np.int64)
    sc.contact.mu = mu
    sc.contact.attach = A
    sc.contact.attach_p0 = X[A].copy()
    sc.contact.attach_travel = np.tile(np.array([0.0005, 0.0, 0.001]), (A.size, 1))
    sc.contact.attach_steps = 2
    return sc, A


def _loss(sc, pb, cp, v0, x0=None, E=None):
    if E is not None:
        pb = solver.build_problem(sc, E=E)
        cp = contact.ContactProblem(pb, sc.contact)
    q, v = (sc.x0 if x0 is None else x0).copy(), v0.copy()
    recs = []
    for t in range(sc.steps):
        qn, ln, lf, _ = contact.step(pb, cp, q, v, sc.f_ext[0], t, tol=1e-14)
        recs.append({"q_t": q, "v_t": v, "q_next": qn, "lam_n": ln, "lam_f": lf})
        v = (qn - q) / pb.h
        q = qn
    d = q - sc.target
    return 0.5 * float(np.sum(d * d)), q, recs


def test_moving_attachments_meet_their_targets():
    sc, A = _pad_with_attachments(0.5, steps=3)
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    _, _, recs = _loss(sc, pb, cp, sc.v0)
    for t, r in enumerate(recs):
        assert np.abs(r["q_next"][A] - sc.contact.attach_target(t)).max() <= 1e-12
    assert recs[-1]["lam_n"][cp.is_att].std() > 0.0     # free-sign multipliers carry load


@pytest.mark.parametrize("mu", [0.0, 50.0])
def test_attachment_adjoint_matches_finite_differences(mu):
    sc, A = _pad_with_attachments(mu)
    rng = np.random.default_rng(7)
    v0 = 0.02 * rng.standard_normal(sc.X.shape)
    pb = solver.build_problem(sc)
    cp = contact.ContactProblem(pb, sc.contact)
    L, qT, recs = _loss(sc, pb, cp, v0)
    act, stick = contact.active_sets(cp, recs[-1]["lam_n"], recs[-1]["q_next"], recs[-1]["q_t"])
    assert act[cp.is_att].all() and stick[cp.is_att].all() and act[~cp.is_att].any()
    g = contact.rollout_backward(pb, cp, recs, qT - sc.target, np.zeros_like(qT))
    eps = 1e-6
    dv = rng.standard_normal(sc.X.shape)
    fd = (_loss(sc, pb, cp, v0 + eps * dv)[0] - _loss(sc, pb, cp, v0 - eps * dv)[0]) / (2 * eps)
    assert abs(fd - np.sum(g.dv0 * dv)) <= 1e-5 * abs(fd) + 1e-12
    dx = rng.standard_normal(sc.X.shape)
    fdx = (_loss(sc, pb, cp, v0, sc.x0 + eps * dx)[0] - _loss(sc, pb, cp, v0, sc.x0 - eps * dx)[0]) / (2 * eps)
    assert abs(fdx - np.sum(g.dx0 * dx)) <= 1e-5 * abs(fdx) + 1e-12
    e = int(np.argmax(np.abs(g.dE)))
    E1, E2 = sc.E.copy(), sc.E.copy()
    hE = 1e-6 * sc.E[e]
    E1[e] += hE
    E2[e] -= hE
    fde = (_loss(sc, pb, cp, v0, E=E1)[0] - _loss(sc, pb, cp, v0, E=E2)[0]) / (2 * hE)
    assert abs(fde - g.dE[e]) <= 1e-4 * abs(fde) + 1e-15
