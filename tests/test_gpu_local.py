"""GPU tests of the standalone local step (pd_local_rhs: per-element
projections and their scatter into the right-hand side, Sec. 4.1, eq.
A_basic; every energy: corotated, Neo-Hookean, the corotated + volume
composite and the log-volume barrier variant) against the oracle's local
step and scatter."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import rel
from oracle import solver
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _deformed(sc, seed, amp):
    rng = np.random.default_rng(seed)
    R = inputs.random_rotation(rng)
    q = sc.X @ R.T + amp * rng.standard_normal(sc.X.shape) * np.ptp(sc.X, axis=0).max()
    q[sc.pinned != 0] = sc.X[sc.pinned != 0]
    return q


@pytest.mark.parametrize("case,fp32,tol", [
    ("cube_corotated", False, 1e-12), ("cube_corotated", True, 2e-6),
    ("tiny_nh", False, 1e-12), ("tiny_nh", True, 2e-6),
    ("bar_nh", True, 2e-6), ("block16_nh", True, 2e-6),
    ("tiny_cv", False, 1e-12), ("tiny_cv", True, 2e-6), ("bar_cv", True, 2e-6),
    ("tiny_lv", False, 1e-12), ("tiny_lv", True, 2e-6), ("bar_lv", True, 2e-6)])
def test_local_rhs_matches_oracle(case, fp32, tol):
    build()
    sc = {"cube_corotated": lambda: inputs.small_cube(),
          "tiny_nh": lambda: inputs.tiny_block(n=3, cell=0.1),
          "bar_nh": lambda: inputs.hetero_bar(steps=1),
          "block16_nh": lambda: inputs.large_block(n=16, steps=1),
          "tiny_cv": lambda: inputs.tiny_block(n=3, cell=0.1, model="corotated_volume"),
          "bar_cv": lambda: inputs.hetero_bar(steps=1).replace(model="corotated_volume"),
          "tiny_lv": lambda: inputs.tiny_block(n=3, cell=0.1, model="corotated_logvol"),
          "bar_lv": lambda: inputs.hetero_bar(steps=1).replace(model="corotated_logvol")}[case]()
    sc = sc.replace(solver=dataclasses.replace(sc.solver, local_fp32=fp32))
    pd = binding.PDContext(sc)
    pb = solver.build_problem(sc)
    for seed in (1, 2):   # the second call starts each prox from the first call's stretches
        q = _deformed(sc, seed, 0.02)
        out = torch.full((sc.n_v, 3), float("nan"), dtype=torch.float64, device=DEV)
        binding.pd_local_rhs(pd.ctx, torch.as_tensor(q, device=DEV), out)
        torch.cuda.synchronize()
        want = solver.rhs(pb, np.zeros_like(q), q)
        want[pb.fixed] = 0.0
        got = out.cpu().numpy()
        assert np.all(got[pb.fixed] == 0.0)
        assert rel(got, want) < tol, (case, fp32, rel(got, want))
    pd.close()
