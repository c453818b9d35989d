"""pd_solve_noalloc: the allocation-free form of pd_solve.

Some callers cannot let the library allocate device memory while they run
(stream capture, real-time loops, device memory owned by another allocator).
This checks, through the C ABI, that the allocation-free call gives pd_solve's
result on two calls in a row (the shared scratch keeps the previous call's
contents, which must not leak into the next result), and that a mesh above
the fixed scratch size is refused with a clear error. Collected last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest
import torch

from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("solve_fp64", [0, 1])
def test_noalloc_solve_matches_pd_solve_on_two_calls(solve_fp64):
    # solve_fp64 = 1 keeps the products in FP64, so the scratch holds doubles
    # where the default form keeps double-float pairs
    build()
    sc = inputs.hetero_bar(steps=1)
    opts = binding.options_for(sc.solver)
    opts.solve_fp64 = solve_fp64
    pd = binding.PDContext(sc, opts)
    rng = np.random.default_rng(11)
    for _ in range(2):
        b = torch.tensor(rng.standard_normal((sc.n_v, 3)), device="cuda:0")
        ref = torch.full_like(b, float("nan"))
        out = torch.full_like(b, float("nan"))
        binding.pd_solve(pd.ctx, b, ref)
        binding.pd_solve_noalloc(pd.ctx, b, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r)
    pd.close()


def test_noalloc_rejects_meshes_above_its_limit():
    build()
    X, tets, _ = inputs.hex_grid(41, 41, 41, 0.1)      # 68,921 vertices > 65,536
    big = inputs.hetero_bar(nx=2, ny=2, nz=2, block=2).replace(
        X=X, tets=tets, pinned=np.zeros(X.shape[0], dtype=np.uint8), E=np.full(tets.shape[0], 1e5),
        x0=X.copy(), v0=np.zeros_like(X), f_ext=np.zeros((1, X.shape[0], 3)), target=X.copy())
    pd = binding.PDContext(big, factor=False)
    x = torch.zeros((big.n_v, 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(binding.PDError) as e:
        binding.pd_solve_noalloc(pd.ctx, x, x)
    assert e.value.code == 11 and "65536" in str(e.value)
    pd.close()


def test_noalloc_solve_captures_into_a_cuda_graph():
    """After one call (which looks up the scratch's address), the call only
    enqueues kernels on the caller's stream: it can be captured into a CUDA
    graph, and replays on new right-hand sides give pd_solve's results."""
    build()
    sc = inputs.hetero_bar(steps=1)
    pd = binding.PDContext(sc)
    rng = np.random.default_rng(12)
    b = torch.tensor(rng.standard_normal((sc.n_v, 3)), device="cuda:0")
    out = torch.zeros_like(b)
    binding.pd_solve_noalloc(pd.ctx, b, out)          # warm-up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        binding.pd_solve_noalloc(pd.ctx, b, out, s)
    for _ in range(2):
        b.copy_(torch.tensor(rng.standard_normal((sc.n_v, 3)), device="cuda:0"))
        out.fill_(float("nan"))
        g.replay()
        ref = torch.full_like(b, float("nan"))
        binding.pd_solve(pd.ctx, b, ref)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r)
    del g
    pd.close()
