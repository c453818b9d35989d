"""GPU tests of solve mode T: A^-1 applied by level-scheduled forward and
backward triangular solves with the supernodal factor (Sec. 4.5; each
separator-tree node's block column replaced by its partitioned inverse),
against the oracle's sparse LU, and the rollout and adjoint that run on it
against the oracle."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import elem_rel, gpu_run, oracle_run, rel
from oracle import solver
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _with(sc, **kw):
    return sc.replace(solver=dataclasses.replace(sc.solver, **kw))


@pytest.mark.parametrize("name", ["bar32x8x8", "tiny3", "block16"])
def test_mode_t_solve_matches_oracle_lu(name):
    build()
    sc = {"bar32x8x8": lambda: inputs.hetero_bar(steps=1),
          "tiny3": lambda: inputs.tiny_block(n=3),
          "block16": lambda: inputs.large_block(n=16, steps=1)}[name]()
    sc = _with(sc, solve_mode=binding.PD_SOLVE_T)
    pd = binding.PDContext(sc)
    st = binding.pd_get_stats(pd.ctx)
    assert st.solve_mode == binding.PD_SOLVE_T and st.solve_levels >= 2
    pb = solver.build_problem(sc)
    rng = np.random.default_rng(3)
    for _ in range(2):   # two solves in a row: the update buffer carries nothing over
        b = rng.standard_normal((sc.n_v, 3))
        x = torch.full((sc.n_v, 3), float("nan"), dtype=torch.float64, device=DEV)
        binding.pd_solve(pd.ctx, torch.as_tensor(b, device=DEV), x)
        torch.cuda.synchronize()
        xo = np.zeros_like(b)
        xo[pb.free] = solver.solve_A(pb, b[pb.free])
        got = x.cpu().numpy()
        assert np.all(got[pb.fixed] == 0.0)
        assert rel(got, xo) < 1e-13, rel(got, xo)
    pd.close()


@pytest.mark.parametrize("persistent", [1, 0])
def test_mode_t_rollout_and_adjoint_fp64_match_oracle(persistent):
    """Small heterogeneous NH bar, FP64 local step, tight gate: the rollout
    and every gradient through mode T against the oracle's exact fixed points
    and direct adjoint."""
    sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=4, steps=5)
    sc = _with(sc, local_fp32=False, eps_step=1e-11, eps_res=1e-10, k_max=400, solve_mode=binding.PD_SOLVE_T)
    g = gpu_run(sc, persistent=persistent)
    assert g["stats"].solve_mode == binding.PD_SOLVE_T
    o = oracle_run(sc)
    assert g["stats"].not_converged == 0
    assert rel(g["qT"], o["qT"]) < 1e-9, rel(g["qT"], o["qT"])
    for k in ("dq0", "dv0", "dE"):
        assert rel(g[k], o[k]) < 1e-6, (k, rel(g[k], o[k]))
    # one force array for every step: the library sums dL/df_ext over steps
    assert rel(g["df"], o["df"].sum(axis=0)) < 1e-6, rel(g["df"], o["df"].sum(axis=0))
    assert elem_rel(g["dE"], o["dE"]) < 1e-5, elem_rel(g["dE"], o["dE"])
    assert abs(g["dnu"] - o["dnu"]) < 1e-6 * abs(o["dnu"])


def test_mode_t_and_mode_s_agree_on_the_bar():
    """The benchmark bar's first 10 steps (FP32 local step, benchmark gate)
    with every A^-1 by mode T and by FP64 products with S: the same
    trajectory up to the gate's resolution, and the same iteration counts
    give or take the gate's rounding."""
    sc = inputs.hetero_bar(steps=10)
    gt = gpu_run(_with(sc, solve_mode=binding.PD_SOLVE_T), backward=True)
    gs = gpu_run(_with(sc, solve_mode=binding.PD_SOLVE_S, solve_fp64=True), backward=True)
    assert gt["stats"].solve_mode == binding.PD_SOLVE_T and gs["stats"].solve_mode == binding.PD_SOLVE_S
    assert rel(gt["qT"], gs["qT"]) < 1e-6, rel(gt["qT"], gs["qT"])
    assert rel(gt["dE"], gs["dE"]) < 1e-4, rel(gt["dE"], gs["dE"])
    assert abs(gt["stats"].iters_total - gs["stats"].iters_total) <= 0.05 * gs["stats"].iters_total


def test_mode_t_block_two_steps_against_oracle():
    """A 16^3-cell heterogeneous block (20,480 tets; bottom pinned, seeded top
    loads), FP32 local step and its configured gate, 2 steps forward and
    backward in mode T against the oracle."""
    sc = _with(inputs.large_block(n=16, steps=2), solve_mode=binding.PD_SOLVE_T)
    g = gpu_run(sc)
    o = oracle_run(sc)
    assert g["stats"].not_converged == 0
    assert rel(g["qT"], o["qT"]) < 1e-5, rel(g["qT"], o["qT"])
    for k in ("dq0", "dv0", "dE"):
        assert rel(g[k], o[k]) < 1e-4, (k, rel(g[k], o[k]))


def test_automatic_solve_mode():
    """PD_SOLVE_AUTO keeps the inverse factor on the bar (S fits in L2) and
    takes mode T on a 24^3-cell block (nnz(S) = 18M, 6x nnz(L))."""
    build()
    bar = binding.PDContext(inputs.hetero_bar(steps=1))
    assert binding.pd_get_stats(bar.ctx).solve_mode == binding.PD_SOLVE_S
    bar.close()
    blk = binding.PDContext(inputs.large_block(n=24, steps=1))
    st = binding.pd_get_stats(blk.ctx)
    assert st.solve_mode == binding.PD_SOLVE_T
    assert st.factor_nnz < 1.6 * st.nnz_L
    blk.close()


def test_mode_t_batch_matches_single_instances():
    """Three uneven instances in one persistent launch, each factored for
    mode T: every instance's rollout agrees with its own single-instance run
    (a team of fewer blocks sums the sweeps and the Anderson dots in another
    order; with the FP64 local step and a tight gate both stop within 1e-8
    of the same fixed points)."""
    build()
    scenes = inputs.batch_meshes(n=3, tets_lo=1000, tets_hi=8000, seed=5, steps=4)
    scenes = [_with(s, solve_mode=binding.PD_SOLVE_T, local_fp32=False, eps_res=1e-11, eps_step=1e-13, k_max=2000)
              for s in scenes]
    bc = binding.BatchContext(scenes)
    assert binding.pd_get_stats(bc.ctx).solve_mode == binding.PD_SOLVE_T
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    x0 = t(bc.concat([s.x0 for s in scenes]).reshape(-1, 3))
    v0 = t(bc.concat([s.v0 for s in scenes]).reshape(-1, 3))
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    binding.pd_rollout(bc.ctx, scenes[0].steps, x0, v0, None, 0, qT, vT)
    q = qT.cpu().numpy()
    off = np.cumsum([0] + [s.n_v for s in scenes])
    for i, s in enumerate(scenes):
        g = gpu_run(s, backward=False)
        assert rel(q[off[i]:off[i + 1]], g["qT"]) < 1e-8, (i, rel(q[off[i]:off[i + 1]], g["qT"]))
    bc.close()
