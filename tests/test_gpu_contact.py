"""GPU tests of frictional contact (vertex-ground and vertex-box contacts,
normal LCP + Tresca friction on the Delassus matrix, eq. q_update) and of
their adjoint (fixed active sets, projected CG) against the contact oracle."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, rel
from oracle import contact, solver
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu


def _pad(steps=2):
    # seed 27: every contact of both steps is well inside its active set
    # (checked on the oracle's solution in the adjoint test)
    return inputs.contact_pad(nx=8, ny=8, nz=5, footprint=4, steps=steps, box_steps=6, travel=0.004, E_core=1e6,
                              seed=27)


@pytest.fixture(scope="module")
def oracle_pad():
    sc = _pad()
    pb = solver.build_problem(sc)
    qT, vT, recs, cp = contact.rollout(pb, sc)
    return sc, qT, recs, cp


def _gpu(sc, **solver_kw):
    build()
    sc = sc.replace(solver=dataclasses.replace(sc.solver, **solver_kw)) if solver_kw else sc
    pd = binding.PDContext(sc)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    x0, v0 = t(sc.x0), t(sc.v0)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    code = binding.pd_rollout(pd.ctx, sc.steps, x0, v0, None, 0, qT, vT, check=False)
    return code, qT.cpu().numpy(), binding.pd_get_stats(pd.ctx), pd


def test_contact_rollout_fp64_matches_oracle(oracle_pad):
    sc, qT, recs, cp = oracle_pad
    code, q, st, _ = _gpu(sc, local_fp32=False, eps_res=1e-10, eps_step=1e-12, k_max=3000)
    assert binding.STATUS[code] == "PD_OK", st.not_converged
    assert st.contact_unconverged == 0
    assert rel(q, qT) <= 1e-7, rel(q, qT)


def test_contact_rollout_fp32_configured_gate_matches_oracle(oracle_pad):
    sc, qT, recs, cp = oracle_pad
    code, q, st, _ = _gpu(sc, k_max=3000)
    assert binding.STATUS[code] == "PD_OK"
    assert rel(q, qT) <= 1e-5, rel(q, qT)
    # no candidate penetrates its obstacle beyond the gate's resolution
    gap = cp.normal * (q[cp.verts, 2] - cp.heights(sc.steps - 1))
    assert gap.min() >= -1e-6 * np.abs(q[:, 2]).max()


def _active_set_margins(sc, recs, cp):
    """Smallest distance of the oracle's solution to an active-set change:
    positive normal multipliers relative to the largest, 1 - |lam_f| / (mu
    lam_n) of the sticking contacts, and the smallest slip of a sliding
    contact relative to the largest. Near zero, the fixed-active-set adjoint
    (the derivative of the rollout where the sets do not change) is not
    defined by the solution, and rounding decides which one-sided derivative
    a solver returns."""
    mu = sc.contact.mu
    out = []
    for r in recs:
        ln, lf = r["lam_n"], r["lam_f"]
        act = ln > 0
        ratio = np.linalg.norm(lf, axis=1) / np.maximum(mu * ln, 1e-300)
        stick = act & (ratio < 1 - 1e-6)
        slide = act & ~stick
        slip = np.linalg.norm(r["q_next"][cp.verts, :2] - r["q_t"][cp.verts, :2], axis=1)
        out.append((ln[act].min() / ln.max() if act.any() else 1.0,
                    1.0 - ratio[stick].max() if stick.any() else 1.0,
                    slip[slide].min() / slip[slide].max() if slide.any() else 1.0))
    return np.min(np.array(out), axis=0)


def test_contact_adjoint_fp64_matches_oracle(oracle_pad):
    sc, qT_o, recs, cp = oracle_pad
    m = _active_set_margins(sc, recs, cp)
    assert np.all(m >= [1e-3, 1e-2, 5e-2]), m
    pb = solver.build_problem(sc)
    g_o = contact.rollout_backward(pb, cp, recs, qT_o - sc.target, np.zeros_like(qT_o))
    code, q, st, pd = _gpu(sc, local_fp32=False, eps_res=1e-10, eps_step=1e-12, k_max=3000)
    assert binding.STATUS[code] == "PD_OK"
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    x = t(q - sc.target)
    dq0, dv0 = torch.empty_like(x), torch.empty_like(x)
    dE = torch.empty(sc.n_e, dtype=torch.float64, device=DEV)
    dnu = torch.empty(1, dtype=torch.float64, device=DEV)
    code = binding.pd_backward(pd.ctx, x, None, dq0, dv0, dE, dnu, None, 0, check=False)
    sb = binding.pd_get_stats(pd.ctx)
    assert binding.STATUS[code] == "PD_OK", (sb.adj_not_converged, sb.contact_unconverged)
    # the projected CG with residual update reaches its tolerance (no
    # breakdown), so the gradients follow the forward's accuracy
    assert sb.adj_not_converged == 0
    assert rel(dv0.cpu().numpy(), g_o.dv0) <= 1e-6, rel(dv0.cpu().numpy(), g_o.dv0)
    assert rel(dq0.cpu().numpy(), g_o.dx0) <= 1e-6, rel(dq0.cpu().numpy(), g_o.dx0)
    assert rel(dE.cpu().numpy(), g_o.dE) <= 1e-6, rel(dE.cpu().numpy(), g_o.dE)


def test_contact_impulses_match_oracle(oracle_pad):
    """pd_get_contact_impulses: the converged normal and friction impulses of
    every step against the oracle's exact LCP / Tresca solutions."""
    sc, qT, recs, cp = oracle_pad
    code, q, st, pd = _gpu(sc, local_fp32=False, eps_res=1e-10, eps_step=1e-12, k_max=3000)
    assert binding.STATUS[code] == "PD_OK"
    for t in range(sc.steps):
        v, ln, lf = binding.pd_get_contact_impulses(pd.ctx, t)
        o = np.argsort(v)
        assert np.array_equal(v[o], cp.verts)
        assert rel(ln[o], recs[t]["lam_n"]) <= 1e-6
        assert rel(lf[o], recs[t]["lam_f"]) <= 1e-5
        assert np.all(ln >= 0.0)


def test_full_pad_steps_are_contact_fixed_points():
    """The full pad (48x48x12 cells, 138,240 tets, 1e7 Pa core, 2,690
    contact candidates), its first 3 steps at the configured settings (FP32
    local step, gate 1e-6 / 1e-8). The oracle's contact rollout of this pad
    takes hours, so each GPU step is checked by properties the oracle
    computes at any size: the converged positions q_{t+1} and the step's
    impulses (pd_get_contact_impulses) must be a fixed point of the
    contact-corrected local-global map (eq. q_update: q = A^-1 (b(q) +
    J^T lam), with the oracle's local step, assembly and sparse solve), and
    the impulses complementary to the gaps: lam_n >= 0, no penetration
    beyond the gate's resolution, lam_n gap = 0, and |lam_f| <= mu lam_n."""
    build()
    sc = inputs.contact_pad(steps=3)
    code, qT, st, pd = _gpu(sc)
    assert binding.STATUS[code] == "PD_OK" and st.contact_unconverged == 0
    pb = solver.build_problem(sc)
    spec = sc.contact
    h = sc.dt
    q_prev = None
    for t in range(sc.steps):
        q_t = binding.pd_get_checkpoint(pd.ctx, t, sc.n_v)
        q_n = binding.pd_get_checkpoint(pd.ctx, t + 1, sc.n_v) if t + 1 < sc.steps else qT
        v_t = sc.v0 if t == 0 else (q_t - q_prev) / h
        verts, lam_n, lam_f = binding.pd_get_contact_impulses(pd.ctx, t)
        D = np.where(np.isin(verts, spec.ground), 1.0, -1.0)
        heights = np.where(D > 0, spec.ground_z, spec.box_z(t))
        # the contact-corrected map at the GPU's converged state
        b0 = solver.rhs_const(pb, q_t, v_t, sc.f_ext[0])
        q_u = solver.solve_A(pb, solver.free_rhs(pb, solver.rhs(pb, b0, q_n)))
        pos = np.searchsorted(pb.free, verts)
        r = np.zeros((pb.free.size, 3))
        r[pos, 0] = lam_f[:, 0]
        r[pos, 1] = lam_f[:, 1]
        r[pos, 2] = D * lam_n
        q_map = q_u + solver.solve_A(pb, r)
        err = rel(q_map, q_n[pb.free])
        assert err <= 2e-6, (t, err)
        # complementarity and the friction disk
        gap = D * (q_n[verts, 2] - heights)
        scale = np.abs(q_n[:, 2]).max()
        assert np.all(lam_n >= 0.0)
        assert gap.min() >= -1e-6 * scale, (t, gap.min())
        active = lam_n > 1e-9 * lam_n.sum()
        assert np.abs(gap[active]).max() <= 1e-6 * scale, (t, np.abs(gap[active]).max())
        assert np.all(np.linalg.norm(lam_f, axis=1) <= spec.mu * lam_n * (1 + 1e-6) + 1e-15)
        assert active.sum() > 100   # the box presses: many active contacts
        q_prev = q_t
    pd.close()
