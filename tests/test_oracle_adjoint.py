"""Pins of the oracle's backward pass (Sec. 4.7, Alg. 2): central finite
differences of the loss through full rollouts, and db/dq against finite
differences of b(q)."""
import numpy as np
import pytest

from oracle import adjoint, fem, solver
from paper_2605_14526_b300 import inputs


def _fd_setup(model):
    sc = inputs.tiny_block(model=model)
    pb = solver.build_problem(sc)
    mu_ref = pb.mat.mu_ref

    def loss(E=None, nu=None, x0=None, v0=None, f=None):
        p = solver.build_problem(sc, E=E, nu=nu, mu_ref=mu_ref)
        qT, vT, _ = solver.rollout(p, sc, mode="exact", x0=x0, v0=v0, f_ext=f)
        return adjoint.loss_and_grad(sc, p, qT, vT)[0]

    qT, vT, recs = solver.rollout(pb, sc, mode="exact")
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    g = adjoint.rollout_backward(pb, recs, dq, dv)
    return sc, pb, loss, g, recs


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume", "corotated_logvol"])
def test_rollout_gradients_match_central_differences(model):
    sc, pb, loss, g, recs = _fd_setup(model)
    assert all(r.info["newton"] < 10 for r in recs)
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-300)
    for e in (0, 17, 33):
        h = 1e-6 * sc.E[e]
        Ep, Em = sc.E.copy(), sc.E.copy()
        Ep[e] += h
        Em[e] -= h
        assert rel(g.dE[e], (loss(E=Ep) - loss(E=Em)) / (2 * h)) < 2e-3
    h = 1e-6
    assert rel(g.dnu, (loss(nu=sc.nu + h) - loss(nu=sc.nu - h)) / (2 * h)) < 1e-3
    free = np.nonzero(sc.pinned == 0)[0]
    for v, i in ((free[0], 0), (free[-1], 2)):
        h = 1e-7
        d = np.zeros_like(sc.x0)
        d[v, i] = h
        assert rel(g.dx0[v, i], (loss(x0=sc.x0 + d) - loss(x0=sc.x0 - d)) / (2 * h)) < 1e-4
        assert rel(g.dv0[v, i], (loss(v0=sc.v0 + d) - loss(v0=sc.v0 - d)) / (2 * h)) < 1e-3
        fp, fm = sc.f_ext.copy(), sc.f_ext.copy()
        fp[1, v, i] += h
        fm[1, v, i] -= h
        assert rel(g.df_ext[1, v, i], (loss(f=fp) - loss(f=fm)) / (2 * h)) < 1e-4


def test_paper_literal_routing_misses_damping_and_mean_terms():
    """dL/dE through w_e alone (eq. dl_dwe) is farther from finite differences
    than the full routing once stiffness damping is significant."""
    sc = inputs.tiny_block(model="neohookean").replace(beta0=20.0)
    pb = solver.build_problem(sc)
    qT, vT, recs = solver.rollout(pb, sc, mode="exact")
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    full = adjoint.rollout_backward(pb, recs, dq, dv)
    lit = adjoint.rollout_backward(pb, recs, dq, dv, paper_literal=True)
    e = int(np.argmax(np.abs(full.dE)))
    h = 1e-6 * sc.E[e]

    def loss(E):
        p = solver.build_problem(sc, E=E, mu_ref=pb.mat.mu_ref)
        a, b, _ = solver.rollout(p, sc, mode="exact")
        return adjoint.loss_and_grad(sc, p, a, b)[0]
    Ep, Em = sc.E.copy(), sc.E.copy()
    Ep[e] += h
    Em[e] -= h
    fd = (loss(Ep) - loss(Em)) / (2 * h)
    assert abs(full.dE[e] - fd) < 1e-3 * abs(fd)
    assert abs(lit.dE[e] - fd) > 10 * abs(full.dE[e] - fd)


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume", "corotated_logvol"])
def test_K_is_db_dq(model):
    sc = inputs.tiny_block(model=model)
    pb = solver.build_problem(sc)
    rng = np.random.default_rng(1)
    q = sc.X + 0.002 * rng.standard_normal(sc.X.shape)
    z = np.zeros_like(q)
    b0 = solver.rhs_const(pb, sc.X, z, z)
    K = adjoint.assemble_K(pb, q, tau=0.0, unfiltered=True).toarray()
    assert np.allclose(K, K.T, atol=1e-8 * np.abs(K).max())
    d = rng.standard_normal(q.shape)
    h = 1e-7
    fd = (solver.rhs(pb, b0, q + h * d) - solver.rhs(pb, b0, q - h * d)) / (2 * h)
    assert np.allclose(K @ d.ravel(), fd.ravel(), rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_small_cube_fixed_iteration_backward_runs():
    sc = inputs.small_cube(steps=2)
    pb = solver.build_problem(sc)
    qT, vT, recs = solver.rollout(pb, sc, mode="fixed")
    assert all(r.info["iters"] == 20 for r in recs)
    L, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    g = adjoint.rollout_backward(pb, recs, dq, dv)
    assert np.all(np.isfinite(g.dE)) and np.isfinite(g.dnu)
    assert np.all(g.dx0[pb.fixed] == 0) and np.all(g.dv0[pb.fixed] == 0)
    # centre of mass height: dL/dq_T is the normalised mass on z
    assert np.isclose(dq[:, 2].sum(), 1.0)
