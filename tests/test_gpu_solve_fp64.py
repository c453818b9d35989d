"""The two representations of the products with the inverse factor S
(options.solve_fp64): plain FP64, and the default double-float pairs on the
FP32 pipe. Both against the oracle's sparse LU of the same A (eq. Ainv_STS,
two_spmv), and against each other along a converged rollout."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import gpu_run, oracle_run, rel
from oracle import solver
from paper_2605_14526_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _solve(sc, fp64):
    opts = binding.options_for(sc.solver)
    opts.solve_fp64 = 1 if fp64 else 0
    pd = binding.PDContext(sc, opts)
    pb = solver.build_problem(sc)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((sc.n_v, 3))
    x = torch.full((sc.n_v, 3), float("nan"), dtype=torch.float64, device="cuda:0")
    binding.pd_solve(pd.ctx, torch.as_tensor(b, device="cuda:0"), x)
    torch.cuda.synchronize()
    xo = np.zeros_like(b)
    xo[pb.free] = solver.solve_A(pb, b[pb.free])
    return x.cpu().numpy(), xo, pb


@pytest.mark.parametrize("shape", [(8, 4, 4, 4), (32, 8, 8, 8)])
def test_fp64_solve_matches_oracle_factor(shape):
    """FP64 products: the factor's own rounding is the only error left
    (the double-float default is held to 1e-11 in test_gpu_parity)."""
    sc = inputs.hetero_bar(nx=shape[0], ny=shape[1], nz=shape[2], block=shape[3], steps=1)
    x, xo, pb = _solve(sc, True)
    assert rel(x, xo) < 1e-13
    assert np.all(x[pb.fixed] == 0.0)
    xd, _, _ = _solve(sc, False)
    # the double-float products differ from FP64 by their 2^-44 rounding
    assert rel(xd, x) < 1e-11


def test_fp64_and_double_float_rollouts_agree():
    """FP64 local step and tight gates: both product forms converge to the
    oracle's fixed points, and to each other within the gate."""
    sc = inputs.tiny_block(model="neohookean", steps=3, cell=0.1)
    s64 = dataclasses.replace(sc.solver, solve_fp64=True)
    g64 = gpu_run(sc.replace(solver=s64))
    gdf = gpu_run(sc)
    o = oracle_run(sc)
    assert g64["stats"].not_converged == 0 and gdf["stats"].not_converged == 0
    assert rel(g64["qT"], o["qT"]) < 1e-9
    assert rel(gdf["qT"], o["qT"]) < 1e-9
    for k in ("dq0", "dv0", "dE", "df"):
        assert rel(g64[k], o[k]) < 1e-6, (k, rel(g64[k], o[k]))
    assert abs(g64["dnu"] - o["dnu"]) < 1e-6 * abs(o["dnu"])


def test_fp64_bar_fp32_config_gate():
    """Benchmark configuration (FP32 local step, gate 1e-6 / 1e-8) with FP64
    products: positions and gradients within the benchmark spec's tolerances."""
    sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=4, steps=20)
    sc = sc.replace(solver=inputs.SolverSettings(eps_res=1e-6, eps_step=1e-8, solve_fp64=True))
    g = gpu_run(sc)
    o = oracle_run(sc)
    assert g["stats"].not_converged == 0
    assert rel(g["qT"], o["qT"]) < 1e-5
    for k in ("dq0", "dv0", "dE"):
        assert rel(g[k], o[k]) < 1e-4, (k, rel(g[k], o[k]))
