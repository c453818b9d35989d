"""Pins of the oracle's operator, right-hand side and fixed point (Sec. 3.1,
4.1, 4.3, 4.4; Alg. 1) against closed forms and invariants."""
import numpy as np
import pytest

from oracle import fem, solver
from paper_2605_14526_b300 import inputs
from paper_2605_14526_b300.inputs import random_rotation


def _scene(model="neohookean", n=2, **kw):
    sc = inputs.tiny_block(n=n, model=model)
    return sc.replace(**kw) if kw else sc


def test_rest_shape_closed_forms():
    sc = inputs.hetero_bar(nx=4, ny=2, nz=2, block=2)
    rest = fem.rest_shape(sc.X, sc.tets, sc.density)
    assert np.isclose(rest.vol.sum(), 4 * 2 * 2 * 0.1 ** 3, rtol=1e-12)
    assert np.isclose(rest.mass.sum(), sc.density * 4 * 2 * 2 * 0.1 ** 3, rtol=1e-12)
    assert np.allclose(rest.gradN.sum(axis=1), 0.0, atol=1e-10)
    F = fem.deformation_gradient(rest, sc.tets, sc.X)
    assert np.allclose(F, np.eye(3), atol=1e-12)
    # affine map x = A X + c gives F = A exactly
    rng = np.random.default_rng(0)
    Am = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    F2 = fem.deformation_gradient(rest, sc.tets, sc.X @ Am.T + 0.7)
    assert np.allclose(F2, Am, atol=1e-12)


def test_lame_closed_form():
    mu, lam = fem.lame(np.array([2.6e5]), 0.3)
    assert np.isclose(mu[0], 1.0e5) and np.isclose(lam[0], 1.5e5)


def test_operator_symmetric_and_row_sums():
    sc = _scene()
    pb = solver.build_problem(sc)
    LA = pb.LA.toarray()
    assert np.allclose(LA, LA.T, atol=1e-9 * np.abs(LA).max())
    # stiffness rows sum to zero (translations), leaving the damped mass term
    assert np.allclose(LA.sum(axis=1), (1 + sc.alpha * sc.dt) * pb.rest.mass / sc.dt ** 2, rtol=1e-10)
    assert np.all(np.linalg.eigvalsh(pb.LA_ff.toarray()) > 0)


def test_weights_are_energy_specific():
    E = np.array([1e5, 3e5])
    m_nh = fem.material(E, 0.3, "neohookean", 0.1)
    m_co = fem.material(E, 0.3, "corotated", 0.1)
    mu, lam = fem.lame(E, 0.3)
    assert np.allclose(m_nh.w, 2 * mu + lam) and np.allclose(m_co.w, 2 * mu)
    assert np.isclose(m_nh.k_bar, np.mean(2 * mu + lam))
    assert np.allclose(m_nh.beta, 0.1 * mu / mu.max())


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume"])
def test_zero_force_at_rest_with_damping(model):
    """A X = b(X) with Rayleigh damping on (needs the damping RHS reading)."""
    sc = _scene(model, gravity=np.zeros(3))
    pb = solver.build_problem(sc)
    z = np.zeros_like(sc.X)
    b0 = solver.rhs_const(pb, sc.X, z, z)
    r = solver.free_rhs(pb, solver.rhs(pb, b0, sc.X))
    assert np.linalg.norm(pb.LA_ff @ sc.X[pb.free] - r) <= 1e-12 * np.linalg.norm(r)
    q, _ = solver.fixed_point(pb, b0, sc.X)
    assert np.allclose(q, sc.X, atol=1e-13)


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume"])
def test_free_body_closed_form(model):
    """No pins, unstrained, uniform velocity and gravity: q = (q~ + alpha h q_t)/(1 + alpha h)."""
    sc = _scene(model, pinned=np.zeros(27, dtype=np.uint8), alpha=0.3)
    pb = solver.build_problem(sc)
    v = np.tile(np.array([0.2, -0.1, 0.4]), (sc.n_v, 1))
    z = np.zeros_like(sc.X)
    b0 = solver.rhs_const(pb, sc.X, v, z)
    q, _ = solver.fixed_point(pb, b0, sc.X)
    qt = solver.inertial_target(pb, sc.X, v, z)
    exact = (qt + sc.alpha * sc.dt * sc.X) / (1 + sc.alpha * sc.dt)
    assert np.allclose(q, exact, atol=1e-13)


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume"])
def test_rigid_rotation_has_no_elastic_force(model):
    sc = _scene(model, pinned=np.zeros(27, dtype=np.uint8), gravity=np.zeros(3))
    pb = solver.build_problem(sc)
    R = random_rotation(np.random.default_rng(3))
    qt = sc.X @ R.T + 0.05
    z = np.zeros_like(sc.X)
    b0 = solver.rhs_const(pb, qt, z, z)
    q, _ = solver.fixed_point(pb, b0, qt)
    assert np.allclose(q, qt, atol=1e-12)


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume", "corotated_logvol"])
def test_plain_iteration_decreases_pd_energy(model):
    """Local-global is block-coordinate descent on g~(q, p) (eq. pd_surrogate)."""
    sc = inputs.hetero_bar(nx=6, ny=2, nz=2, block=2, omega0=6.0).replace(model=model)
    pb = solver.build_problem(sc)
    b0 = solver.rhs_const(pb, sc.x0, sc.v0, sc.f_ext[0])
    qt = solver.inertial_target(pb, sc.x0, sc.v0, sc.f_ext[0])
    q = sc.x0.copy()
    e_prev = solver.pd_energy(pb, q, sc.x0, qt)
    for _ in range(15):
        q = solver.picard(pb, b0, q)
        e = solver.pd_energy(pb, q, sc.x0, qt)
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e


@pytest.mark.parametrize("model", ["neohookean", "corotated", "corotated_volume", "corotated_logvol"])
def test_fixed_point_is_stationary(model):
    sc = inputs.hetero_bar(nx=6, ny=2, nz=2, block=2, omega0=6.0).replace(model=model)
    pb = solver.build_problem(sc)
    b0 = solver.rhs_const(pb, sc.x0, sc.v0, sc.f_ext[0])
    q, _ = solver.fixed_point(pb, b0, sc.x0)
    assert solver.stationarity(pb, b0, q) <= 1e-12


def test_heterogeneous_path_with_equal_moduli_is_homogeneous():
    sc = inputs.hetero_bar(nx=4, ny=2, nz=2, block=2, omega0=4.0)
    homo = sc.replace(E=np.full(sc.n_e, 3e5))
    pb = solver.build_problem(homo)
    assert np.allclose(pb.mat.w, pb.mat.k_bar) and np.allclose(pb.mat.beta, sc.beta0)
    qa, _, _ = solver.rollout(pb, homo.with_steps(2))
    # standard PD: A = M/h^2(1+alpha h) + (k + beta0/h) sum V G^T G with one scalar k
    mu, lam = fem.lame(3e5, homo.nu)
    LA = fem.assemble_LA(pb.rest, homo.tets, pb.mat, homo.alpha, homo.dt)
    assert np.allclose(LA.toarray(), pb.LA.toarray())
    assert np.isclose(pb.mat.k_bar, 2 * mu + lam)
    assert np.all(np.isfinite(qa))


def test_anderson_solves_linear_map_with_full_window():
    """Type-II AA with a window covering the space is GMRES-like on a linear
    contraction (Walker & Ni 2011): it reaches the fixed point in about n + 1 steps."""
    rng = np.random.default_rng(11)
    n = 6
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Mlin = Q @ np.diag(np.linspace(0.1, 0.9, n)) @ Q.T
    c = rng.standard_normal(n)
    xs = np.linalg.solve(np.eye(n) - Mlin, c)
    x = np.zeros(n)
    hq, hg = [], []
    for k in range(n + 3):
        qhat = Mlin @ x + c
        g = qhat - x
        hq.append(x.copy())
        hg.append(g.copy())
        if len(hq) > n + 1:
            hq.pop(0)
            hg.pop(0)
        x, reset = solver.aa_mix(hq, hg, qhat, g)
        assert not reset
    assert np.linalg.norm(x - xs) <= 1e-5 * np.linalg.norm(xs)
    # plain iteration is far from converged after the same number of steps
    y = np.zeros(n)
    for _ in range(n + 3):
        y = Mlin @ y + c
    assert np.linalg.norm(y - xs) > 1e-2 * np.linalg.norm(xs)


def test_anderson_guard_trips_on_large_mixing():
    q0 = np.zeros(3)
    q1 = np.array([1.0, 0.0, 0.0])
    g0 = np.array([1.0, 0.0, 0.0])
    g1 = np.array([1.0 + 1e-3, 0.0, 0.0])     # nearly parallel residuals: gamma ~ 1e3
    qhat = q1 + g1
    out, reset = solver.aa_mix([q0, q1], [g0, g1], qhat, g1)
    assert reset and np.allclose(out, qhat)


def test_aa_reference_matches_fixed_point():
    sc = inputs.hetero_bar(nx=6, ny=2, nz=2, block=2, omega0=6.0)
    pb = solver.build_problem(sc)
    b0 = solver.rhs_const(pb, sc.x0, sc.v0, sc.f_ext[0])
    q, _ = solver.fixed_point(pb, b0, sc.x0)
    qa, qprev, info = solver.aa_reference(pb, b0, sc.x0, 5, 200, 1e-8, 1e-6, 1e-12)
    assert info["converged"]
    assert np.linalg.norm(qa - q) <= 1e-6 * np.linalg.norm(q)


def test_trust_region_ratio_rules():
    sc = inputs.hetero_bar(nx=4, ny=2, nz=2, block=2)
    pb = solver.build_problem(sc)
    tau, rho = solver.tr_select(pb, sc.X, sc.X, sc.X)
    assert rho == 1.0 and tau == 0.5                  # Delta Phi_mod < 1e-12
    # an inverted iterate: Phi = +inf, the model is inadequate
    bad = sc.X.copy()
    free = pb.free
    bad[free[0]] = bad[free[0]] + np.array([-0.5, -0.5, -0.5])
    tau, rho = solver.tr_select(pb, sc.X, bad, sc.X)
    assert tau == 1.0


# ------------------------------------------------------------------ TR ratio by hand
#
# One tetrahedron with corners 0, a e1, a e2, a e3; corners 0-2 pinned, so the
# only free vertex is the apex and every quantity of eq. primal and eq. tr_ratio
# has a closed form in its displacement u: F = I + u e3^T / a, J = 1 + u_z / a,
# tr(F^T F) = 3 + 2 u_z / a + |u|^2 / a^2, V = a^3 / 6, lumped masses rho V / 4,
# and the apex entry of the scalar operator
#   L_33 = (1 + alpha h) m / h^2 + (w + beta / h) V |grad N_3|^2,  |grad N_3| = 1 / a,
# with w = 2 mu + lambda (Neo-Hookean) and beta = beta0 (mu_ref = mu for one element).

_A, _RHO, _E, _NU, _H, _ALPHA, _BETA0 = 0.1, 1000.0, 1e5, 0.3, 0.01, 0.01, 1e-3


def _one_tet():
    X = _A * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    sc = inputs.Scene(
        name="tet", X=X, tets=np.array([[0, 1, 2, 3]], dtype=np.int32), pinned=np.array([1, 1, 1, 0], np.uint8),
        E=np.array([_E]), nu=_NU, density=_RHO, alpha=_ALPHA, beta0=_BETA0, gravity=np.zeros(3), dt=_H,
        model="neohookean", steps=1, f_ext=np.zeros((1, 4, 3)), x0=X.copy(), v0=np.zeros((4, 3)))
    return sc, solver.build_problem(sc)


def _hand_phi(u, u_tilde):
    """Phi of the one-tet problem with the apex at X3 + u and its inertial
    target at X3 + u_tilde (the pinned corners sit on their targets)."""
    mu = _E / (2 * (1 + _NU))
    lam = _E * _NU / ((1 + _NU) * (1 - 2 * _NU))
    V = _A ** 3 / 6
    m = _RHO * V / 4
    u = np.asarray(u, dtype=np.float64)
    J = 1 + u[2] / _A
    trC = 3 + 2 * u[2] / _A + u @ u / _A ** 2
    psi = mu / 2 * (trC - 3) - mu * np.log(J) + lam / 2 * np.log(J) ** 2
    d = u - np.asarray(u_tilde)
    return m / (2 * _H ** 2) * (d @ d) + V * psi


def _hand_L33():
    mu = _E / (2 * (1 + _NU))
    lam = _E * _NU / ((1 + _NU) * (1 - 2 * _NU))
    V = _A ** 3 / 6
    m = _RHO * V / 4
    return (1 + _ALPHA * _H) * m / _H ** 2 + (2 * mu + lam + _BETA0 / _H) * V / _A ** 2


def test_phi_kinetic_term_closed_form():
    # a rigid translation leaves F = I (psi = 0): Phi is the kinetic term alone,
    # 1/(2 h^2) (total mass) |t - s|^2 for positions X + t and target X + s
    sc, pb = _one_tet()
    t, s = np.array([0.01, -0.02, 0.03]), np.array([-0.005, 0.004, 0.0])
    want = _RHO * _A ** 3 / 6 / (2 * _H ** 2) * float((t - s) @ (t - s))
    assert np.isclose(solver.phi(pb, sc.X + t, sc.X + s), want, rtol=1e-13)
    # and the elastic part alone at the target: Phi = V psi
    u = np.array([0.002, -0.001, 0.003])
    q = sc.X.copy()
    q[3] += u
    assert np.isclose(solver.phi(pb, q, q), _hand_phi(u, u), rtol=1e-12)


@pytest.mark.parametrize("u_prev,u_star,u_tilde,tau_want", [
    # axial step onto the minimiser: the model's w = 2 mu + lambda matches
    # psi's axial stiffness at small strain, rho = 0.995 -> tau = 1/2
    ((0.0, 0.0, 0.001), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 0.5),
    # shear step: psi's shear stiffness is mu against the model's w, rho = 0.40 -> tau = 1
    ((0.001, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0),
    # mixed step with the target away from both iterates (the kinetic term
    # enters Delta Phi_act), rho = 0.984 -> tau = 1/2
    ((0.001, 0.0005, 0.002), (0.0003, 0.0001, 0.0008), (0.001, 0.0, 0.004), 0.5),
    # the same target, a step that overshoots the minimiser: rho = 1.26 -> tau = 1
    ((0.0, 0.0, 0.002), (0.0, 0.0, 0.0008), (0.0, 0.0, 0.004), 1.0),
])
def test_trust_region_ratio_by_hand(u_prev, u_star, u_tilde, tau_want):
    sc, pb = _one_tet()
    q_prev, q_star, q_til = sc.X.copy(), sc.X.copy(), sc.X.copy()
    q_prev[3] += u_prev
    q_star[3] += u_star
    q_til[3] += u_tilde
    du = np.subtract(u_star, u_prev)
    act = _hand_phi(u_prev, u_tilde) - _hand_phi(u_star, u_tilde)       # Phi(q*^-1) - Phi(q*)
    mod = 0.5 * abs(_hand_L33() * float(du @ du))                          # 1/2 |dq^T A dq|
    rho_want = act / mod
    assert (abs(rho_want - 1) <= 0.1) == (tau_want == 0.5)
    tau, rho = solver.tr_select(pb, q_star, q_prev, q_til, eps_tr=0.1)
    assert np.isclose(rho, rho_want, rtol=1e-9, atol=0), (rho, rho_want)
    assert tau == tau_want
