"""GPU tests of bilateral attachment rows (Sec. 4.6: a vertex held at a
prescribed, moving target by three equality rows with free multipliers,
solved with the contact rows on the Delassus matrix) and of their adjoint,
against the contact oracle and against Dirichlet pinning."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, rel
from oracle import adjoint, contact, solver
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu

TIGHT = dict(local_fp32=False, eps_res=1e-10, eps_step=1e-12, k_max=3000)


def _att_pad(steps=2):
    """The contact parity pad (8x8x5 cells, ground below, box pressing the
    top centre, mu = 0.5) with its four top corners attached and lifted by
    2 mm over 4 steps. On the oracle's solution the smallest sliding slip is
    3.7x the sticking tolerance and the friction of a sticking contact stays
    2% inside its disk: the active sets are well defined."""
    sc = inputs.contact_pad(nx=8, ny=8, nz=5, footprint=4, steps=steps, box_steps=6, travel=0.004, E_core=1e6,
                            seed=27)
    X = sc.X
    top = np.nonzero(np.isclose(X[:, 2], X[:, 2].max()))[0]
    taken = set(sc.contact.ground.tolist()) | set(sc.contact.box.tolist())
    xs, ys = X[:, 0], X[:, 1]
    A = np.array(sorted(v for v in top if v not in taken
                        and (np.isclose(xs[v], xs.min()) or np.isclose(xs[v], xs.max()))
                        and (np.isclose(ys[v], ys.min()) or np.isclose(ys[v], ys.max()))), dtype=np.int64)
    assert A.size == 4
    sc.contact.attach = A
    sc.contact.attach_p0 = X[A].copy()
    sc.contact.attach_travel = np.tile(np.array([0.0, 0.0, 0.002]), (A.size, 1))
    sc.contact.attach_steps = 4
    return sc, A


@pytest.fixture(scope="module")
def oracle_att_pad():
    sc, A = _att_pad()
    pb = solver.build_problem(sc)
    qT, vT, recs, cp = contact.rollout(pb, sc)
    return sc, A, pb, qT, recs, cp


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _gpu(sc, **solver_kw):
    build()
    sc = sc.replace(solver=dataclasses.replace(sc.solver, **solver_kw)) if solver_kw else sc
    pd = binding.PDContext(sc)
    x0, v0 = _t(sc.x0), _t(sc.v0)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    code = binding.pd_rollout(pd.ctx, sc.steps, x0, v0, None, 0, qT, vT, check=False)
    return code, qT.cpu().numpy(), vT.cpu().numpy(), binding.pd_get_stats(pd.ctx), pd


def _backward(pd, dq, dv, n_e):
    dq0, dv0 = torch.empty_like(_t(dq)), torch.empty_like(_t(dq))
    dE = torch.empty(n_e, dtype=torch.float64, device=DEV)
    dnu = torch.empty(1, dtype=torch.float64, device=DEV)
    code = binding.pd_backward(pd.ctx, _t(dq), _t(dv), dq0, dv0, dE, dnu, None, 0, check=False)
    return code, dq0.cpu().numpy(), dv0.cpu().numpy(), dE.cpu().numpy(), float(dnu.cpu().numpy()[0])


def test_attachment_pad_forward_and_adjoint_match_oracle(oracle_att_pad):
    sc, A, pb, qT_o, recs, cp = oracle_att_pad
    code, q, _, st, pd = _gpu(sc, **TIGHT)
    assert binding.STATUS[code] == "PD_OK" and st.contact_unconverged == 0
    assert rel(q, qT_o) <= 1e-7, rel(q, qT_o)
    assert np.abs(q[A] - sc.contact.attach_target(sc.steps - 1)).max() <= 1e-9
    for t in range(sc.steps):   # impulses of every step, attachments included
        v, ln, lf = binding.pd_get_contact_impulses(pd.ctx, t)
        o = np.argsort(v)
        assert np.array_equal(v[o], cp.verts)
        assert rel(ln[o], recs[t]["lam_n"]) <= 1e-6
        assert rel(lf[o], recs[t]["lam_f"]) <= 1e-5
    g_o = contact.rollout_backward(pb, cp, recs, qT_o - sc.target, np.zeros_like(qT_o))
    code, dq0, dv0, dE, dnu = _backward(pd, q - sc.target, np.zeros_like(q), sc.n_e)
    sb = binding.pd_get_stats(pd.ctx)
    assert binding.STATUS[code] == "PD_OK" and sb.adj_not_converged == 0
    assert rel(dv0, g_o.dv0) <= 1e-6, rel(dv0, g_o.dv0)
    assert rel(dq0, g_o.dx0) <= 1e-6, rel(dq0, g_o.dx0)
    assert rel(dE, g_o.dE) <= 1e-6, rel(dE, g_o.dE)
    assert abs(dnu - g_o.dnu) <= 1e-6 * abs(g_o.dnu)
    pd.close()


def test_attachment_pad_fp32_configured_gate(oracle_att_pad):
    sc, A, pb, qT_o, recs, cp = oracle_att_pad
    code, q, _, st, pd = _gpu(sc, k_max=3000)
    assert binding.STATUS[code] == "PD_OK"
    assert rel(q, qT_o) <= 1e-5, rel(q, qT_o)
    assert np.abs(q[A] - sc.contact.attach_target(sc.steps - 1)).max() <= 1e-6 * np.abs(q).max()
    pd.close()


@pytest.mark.parametrize("model", ["neohookean", "corotated"])
def test_attachment_at_rest_equals_pinning(model):
    """The small heterogeneous bar with its Dirichlet vertices released and
    held by attachment rows at their rest positions reproduces the oracle's
    pinned rollout and gradients (pins act through the factor,
    attachments through multipliers on the unpinned operator)."""
    sc = inputs.hetero_bar(nx=4, ny=2, nz=2, block=2, steps=4, omega0=4.0).replace(model=model)
    P = np.nonzero(sc.pinned)[0]
    v0 = sc.v0.copy()
    v0[P] = 0.0
    sc = sc.replace(v0=v0)
    pb = solver.build_problem(sc)
    qT, vT, orecs = solver.rollout(pb, sc, mode="exact")
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    g = adjoint.rollout_backward(pb, orecs, dq, dv)
    att = sc.replace(pinned=np.zeros_like(sc.pinned))
    att.contact = inputs.ContactSpec(ground=np.zeros(0, dtype=np.int64), box=np.zeros(0, dtype=np.int64),
                                     ground_z=0.0, box_z0=0.0, box_travel=0.0, box_steps=1, mu=0.0, attach=P,
                                     attach_p0=sc.X[P].copy(), attach_travel=np.zeros((P.size, 3)), attach_steps=1)
    code, q, vq, st, pd = _gpu(att, **TIGHT)
    assert binding.STATUS[code] == "PD_OK"
    assert rel(q, qT) <= 1e-9, rel(q, qT)
    assert np.abs(q[P] - sc.X[P]).max() <= 1e-12
    _, dqg, dvg = adjoint.loss_and_grad(sc, pb, q, vq)
    code, dq0, dv0, dE, dnu = _backward(pd, dqg, dvg, sc.n_e)
    assert binding.STATUS[code] == "PD_OK"
    free = np.nonzero(sc.pinned == 0)[0]
    assert rel(dE, g.dE) <= 1e-6, rel(dE, g.dE)
    assert abs(dnu - g.dnu) <= 1e-6 * abs(g.dnu)
    assert rel(dq0[free], g.dx0[free]) <= 1e-6 and rel(dv0[free], g.dv0[free]) <= 1e-6
    pd.close()


def test_attachment_arguments_are_checked():
    build()
    sc = inputs.hetero_bar(nx=4, ny=2, nz=2, block=2, steps=1)
    pd = binding.PDContext(sc)
    P = np.nonzero(sc.pinned)[0]
    spec = inputs.ContactSpec(ground=np.zeros(0, dtype=np.int64), box=np.zeros(0, dtype=np.int64), ground_z=0.0,
                              box_z0=0.0, box_travel=0.0, box_steps=1, mu=0.0, attach=P[:1],
                              attach_p0=sc.X[P[:1]], attach_travel=np.zeros((1, 3)), attach_steps=1)
    with pytest.raises(binding.PDError) as e:   # a pinned vertex cannot be attached
        binding.pd_set_contacts(pd.ctx, spec)
    assert e.value.code == 1
    free = np.nonzero(sc.pinned == 0)[0][:1]
    spec.attach, spec.attach_p0 = free, np.array([[np.nan, 0.0, 0.0]])
    with pytest.raises(binding.PDError) as e:   # targets must be finite
        binding.pd_set_contacts(pd.ctx, spec)
    assert e.value.code == 1
    pd.close()
