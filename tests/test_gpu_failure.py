"""Failure detection without a GPU fault: every team-barrier wait of the
persistent kernels is bounded (options.wait_polls). A context whose waits
give up after one poll must fail with PD_ERR_TIMEOUT, leave the device
usable, and leave the library's own state clean for the next call."""
import numpy as np
import pytest
import torch

from gpu_helpers import DEV, gpu_run, rel
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu


def _rollout(sc, opts):
    pd = binding.PDContext(sc, opts)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    x0, v0 = t(sc.x0), t(sc.v0)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    code = binding.pd_rollout(pd.ctx, sc.steps, x0, v0, t(sc.f_ext[0]), 0, qT, vT, check=False)
    return code, qT, pd


def test_barrier_wait_times_out_and_device_stays_usable():
    build()
    sc = inputs.hetero_bar(nx=16, ny=8, nz=8, block=4, steps=2)
    ref = gpu_run(sc, backward=False)["qT"]
    opts = binding.options_for(sc.solver)
    opts.wait_polls = 1   # one poll per wait: blocks arriving early give up
    code, _, pd = _rollout(sc, opts)
    assert binding.STATUS[code] == "PD_ERR_TIMEOUT"
    st = binding.pd_get_stats(pd.ctx)
    assert st.status_flags & 4
    # the same context still solves correctly (split-row counters cleared)
    x = torch.full((sc.n_v, 3), float("nan"), dtype=torch.float64, device=DEV)
    b = torch.as_tensor(np.random.default_rng(0).standard_normal((sc.n_v, 3)), device=DEV)
    binding.pd_solve(pd.ctx, b, x)
    ok = binding.PDContext(sc)
    x2 = torch.full_like(x, float("nan"))
    binding.pd_solve(ok.ctx, b, x2)
    torch.cuda.synchronize()
    assert torch.equal(x, x2)
    # and a default context on the same device reproduces the reference bitwise
    code, q, _ = _rollout(sc, binding.options_for(sc.solver))
    assert binding.STATUS[code] == "PD_OK"
    assert np.array_equal(q.cpu().numpy(), ref)
