"""GPU tests of the learned warm start: the training kernels (forward, gradient,
Adam) and the sample kernel against the oracle, the in-rollout warm start
against the oracle, and the end-to-end claim: a network trained on the
plain solver's trajectories by the library's own kernels starts the
local-global iteration closer to the fixed point (fewer iterations than the
cold start q_t), while the converged trajectory stays that of the plain
solver."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, oracle_run, rel
from oracle import mlp as omlp
from paper_2605_14526_b300 import binding, inputs
from paper_2605_14526_b300.build import build

pytestmark = pytest.mark.gpu

H = 128


def _quantized(theta):
    """The oracle's copy of the parameters the kernels compute with: weights
    rounded to BF16, biases as they are."""
    th = np.asarray(theta, dtype=np.float32).astype(np.float64)
    parts = omlp.unpack(th, H)
    for i in (0, 2, 4, 6):
        parts[i][...] = omlp.bf16_round(parts[i].astype(np.float32)).astype(np.float64)
    return th


def _norm(rng):
    mean = rng.normal(0, 0.1, 7)
    scale = rng.uniform(0.5, 2.0, 7)
    osc = rng.uniform(1e-4, 1e-3, 3)
    return np.concatenate([mean, scale, osc]).astype(np.float32)


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def _f64(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _net_with_trained_like_biases(seed):
    theta = inputs.mlp_init(seed)
    rng = np.random.default_rng(seed + 100)
    parts = omlp.unpack(theta, H)
    for i in (1, 3, 5, 7):
        parts[i][...] = rng.normal(0, 0.1, parts[i].shape)
    return theta


def test_forward_matches_oracle():
    build()
    rng = np.random.default_rng(0)
    theta = _net_with_trained_like_biases(1)
    norm = _norm(rng)
    net = binding.MLP(theta, norm)
    n = 1000
    feat = rng.normal(0, 1, (n, 7)).astype(np.float32)
    r = torch.empty((n, 3), dtype=torch.float32, device=DEV)
    binding.pd_mlp_forward(net.net, _f32(feat), r, n)
    fn = (feat.astype(np.float64) - norm[:7]) / norm[7:14]
    want = omlp.forward(_quantized(theta), fn, H) * norm[14:]
    assert rel(r.cpu().numpy(), want) <= 1e-5


def test_gradient_and_loss_match_oracle():
    build()
    rng = np.random.default_rng(1)
    theta = _net_with_trained_like_biases(2)
    norm = _norm(rng)
    net = binding.MLP(theta, norm)
    n = 777
    feat = rng.normal(0, 1, (n, 7)).astype(np.float32)
    targ = (rng.normal(0, 1, (n, 3)) * norm[14:]).astype(np.float32)
    g = torch.empty(binding.MLP_PARAMS, dtype=torch.float32, device=DEV)
    loss = binding.pd_mlp_grad(net.net, _f32(feat), _f32(targ), n, g)
    fn = (feat.astype(np.float64) - norm[:7]) / norm[7:14]
    tn = targ.astype(np.float64) / norm[14:]
    L, gw = omlp.grad(_quantized(theta), fn, tn, H)
    assert abs(loss - L) <= 1e-5 * L
    assert rel(g.cpu().numpy(), gw) <= 1e-4
    # every layer's block separately (a transposed or mis-offset block fails here)
    gg = g.cpu().numpy().astype(np.float64)
    for a, b in zip(omlp.unpack(gg, H), omlp.unpack(gw, H)):
        assert rel(a, b) <= 1e-4


def test_adam_step_matches_oracle_on_the_same_gradient():
    build()
    rng = np.random.default_rng(2)
    theta = _net_with_trained_like_biases(3)
    norm = _norm(rng)
    net = binding.MLP(theta, norm)
    n = 300
    feat = _f32(rng.normal(0, 1, (n, 7)))
    targ = _f32(rng.normal(0, 1, (n, 3)) * norm[14:])
    g = torch.empty(binding.MLP_PARAMS, dtype=torch.float32, device=DEV)
    binding.pd_mlp_grad(net.net, feat, targ, n, g)
    lr = 1e-3
    binding.pd_mlp_train_step(net.net, feat, targ, n, lr)
    th1, _ = net.params()
    opt = omlp.Adam(binding.MLP_PARAMS, lr=lr)
    want = opt.step(theta.astype(np.float64), g.cpu().numpy().astype(np.float64))
    step_gpu = th1.astype(np.float64) - theta
    step_or = want - theta
    assert np.max(np.abs(step_gpu - step_or)) <= 1e-4 * lr + 1e-7 * np.max(np.abs(theta))


def test_sample_kernel_matches_oracle_features():
    build()
    sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=2, steps=3)
    pd = binding.PDContext(sc)
    rng = np.random.default_rng(3)
    x0 = sc.X + 1e-3 * rng.standard_normal(sc.X.shape)
    x1 = x0 + 1e-3 * rng.standard_normal(sc.X.shape)
    x2 = x1 + 1e-3 * rng.standard_normal(sc.X.shape)
    feat = torch.empty((sc.n_v, 7), dtype=torch.float32, device=DEV)
    targ = torch.empty((sc.n_v, 3), dtype=torch.float32, device=DEV)
    binding.pd_mlp_sample(pd.ctx, _f64(x0), _f64(x1), _f64(x2), feat, targ)
    torch.cuda.synchronize()
    le = omlp.vertex_log_stiffness(sc.X, sc.tets, sc.E)
    want_f = omlp.features(x1, x0, sc.X, le)
    want_t = omlp.target(x2, x1, x0)
    assert np.allclose(feat.cpu().numpy(), want_f, rtol=1e-6, atol=1e-9)
    assert np.allclose(targ.cpu().numpy(), want_t, rtol=1e-6, atol=1e-12)


def test_rollout_warm_start_matches_oracle():
    build()
    sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=2, steps=3)
    rng = np.random.default_rng(4)
    theta = _net_with_trained_like_biases(4)
    norm = _norm(rng)
    opts = binding.options_for(sc.solver)
    opts.warm_start = 1
    pd = binding.PDContext(sc, opts)
    binding.pd_mlp_load(pd.ctx, np.concatenate([theta, norm]))
    xm = sc.X + 1e-3 * rng.standard_normal(sc.X.shape)
    xt = xm + 2e-3 * rng.standard_normal(sc.X.shape)
    q0 = torch.empty((sc.n_v, 3), dtype=torch.float64, device=DEV)
    binding.pd_warm_start(pd.ctx, _f64(xt), _f64(xm), q0)
    torch.cuda.synchronize()
    le = omlp.vertex_log_stiffness(sc.X, sc.tets, sc.E)
    want = omlp.warm_start(_quantized(theta), (norm[:7].astype(np.float64), norm[7:14].astype(np.float64),
                                               norm[14:].astype(np.float64)), xt, xm, sc.X, le, sc.pinned, H)
    got = q0.cpu().numpy()
    free = sc.pinned == 0
    base = 2 * xt - xm
    assert rel(got[free] - base[free], want[free] - base[free]) <= 1e-5
    assert np.array_equal(got[~free], sc.X[~free])


def _frames(scene, ctx, T):
    """Checkpoints x_0 .. x_T of the last rollout of a context (host)."""
    return [binding.pd_get_checkpoint(ctx, t, scene.n_v) for t in range(T + 1)]


def _training_set(scenes, T):
    """Features and targets of frames t = 1 .. T-1 of plain-solver rollouts."""
    feats, targs = [], []
    for sc in scenes:
        pd = binding.PDContext(sc)
        x0, v0 = _f64(sc.x0), _f64(sc.v0)
        qT, vT = torch.empty_like(x0), torch.empty_like(x0)
        binding.pd_rollout(pd.ctx, T, x0, v0, None, 0, qT, vT)
        xs = [_f64(x) for x in _frames(sc, pd.ctx, T)]
        for t in range(1, T):
            f = torch.empty((sc.n_v, 7), dtype=torch.float32, device=DEV)
            g = torch.empty((sc.n_v, 3), dtype=torch.float32, device=DEV)
            binding.pd_mlp_sample(pd.ctx, xs[t - 1], xs[t], xs[t + 1], f, g)
            keep = torch.as_tensor(sc.pinned == 0, device=DEV)
            feats.append(f[keep])
            targs.append(g[keep])
    return torch.cat(feats).contiguous(), torch.cat(targs).contiguous()


def _train(feat, targ, steps, batch=4096, lr=1e-3, seed=0):
    net = binding.MLP(inputs.mlp_init(seed), np.concatenate([np.zeros(7), np.ones(7), np.ones(3)]))
    n = feat.shape[0]
    binding.pd_mlp_fit_normalization(net.net, feat, targ, n)
    gen = torch.Generator(device=DEV)
    gen.manual_seed(seed)
    first = binding.pd_mlp_grad(net.net, feat, targ, n)
    for _ in range(steps):
        idx = torch.randint(0, n, (batch,), device=DEV, generator=gen)
        binding.pd_mlp_train_step(net.net, feat[idx].contiguous(), targ[idx].contiguous(), batch, lr, want_loss=False)
    last = binding.pd_mlp_grad(net.net, feat, targ, n)
    return net, first, last


def _run(sc, warm, blob=None):
    opts = binding.options_for(sc.solver)
    opts.warm_start = warm
    pd = binding.PDContext(sc, opts)
    if blob is not None:
        binding.pd_mlp_load(pd.ctx, blob)
    x0, v0 = _f64(sc.x0), _f64(sc.v0)
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    binding.pd_rollout(pd.ctx, sc.steps, x0, v0, None, 0, qT, vT)
    return qT.cpu().numpy(), binding.pd_get_stats(pd.ctx)


def test_trained_warm_start_cuts_iterations_and_keeps_the_trajectory():
    build()
    T = 60

    def bar(seed, omega):
        sc = inputs.hetero_bar(nx=16, ny=4, nz=4, block=4, steps=T, seed=seed, omega0=omega)
        # FP64 local step and a tight gate, so that every start must reach the
        # oracle's trajectory (a looser gate drifts from it whatever the start)
        return sc.replace(solver=dataclasses.replace(sc.solver, eps_res=1e-8, eps_step=1e-10, local_fp32=False))

    train = [bar(s, w) for s, w in ((3, 1.5), (4, 2.5), (5, 2.0))]
    feat, targ = _training_set(train, T)
    net, first, last = _train(feat, targ, steps=400)
    assert last < 0.25 * first, (first, last)
    held = bar(6, 1.8)
    q_cold, s_cold = _run(held, 0)
    q_ext, s_ext = _run(held, 2)
    q_net, s_net = _run(held, 1, net.blob())
    print(f"iterations over {T} steps: cold {s_cold.iters_total}, constant-velocity {s_ext.iters_total}, "
          f"network {s_net.iters_total}; loss {first:.4g} -> {last:.4g}")
    assert s_net.warm_fallbacks == 0
    assert s_net.iters_total < s_cold.iters_total, (s_net.iters_total, s_ext.iters_total, s_cold.iters_total)
    # the start changes the path to the fixed point, not the fixed point
    o = oracle_run(held.with_steps(T), backward=False)
    for q in (q_cold, q_ext, q_net):
        assert rel(q, o["qT"]) <= 1e-5


def test_batch_warm_start_by_extrapolation_matches_oracle():
    build()
    scenes = inputs.batch_meshes(n=3, tets_lo=300, tets_hi=1200, steps=3, seed=9)
    opts = binding.options_for(scenes[0].solver)
    opts.warm_start = 2
    bc = binding.BatchContext(scenes, opts)
    x0 = _f64(bc.concat([s.x0 for s in scenes]).reshape(-1, 3))
    v0 = _f64(bc.concat([s.v0 for s in scenes]).reshape(-1, 3))
    qT, vT = torch.empty_like(x0), torch.empty_like(x0)
    binding.pd_rollout(bc.ctx, 3, x0, v0, None, 0, qT, vT)
    q = bc.split_v(qT.cpu().numpy())
    for i, sc in enumerate(scenes):
        o = oracle_run(sc, backward=False)
        assert rel(q[i], o["qT"]) <= 1e-5


def test_warm_start_needs_a_network():
    build()
    sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=2, steps=2)
    opts = binding.options_for(sc.solver)
    opts.warm_start = 1
    pd = binding.PDContext(sc, opts)
    x0 = _f64(sc.x0)
    code = binding.pd_rollout(pd.ctx, 2, x0, _f64(sc.v0), None, 0, torch.empty_like(x0), torch.empty_like(x0),
                              check=False)
    assert binding.STATUS[code] == "PD_ERR_ARG"
    with pytest.raises(binding.PDError):
        binding.pd_mlp_load(pd.ctx, np.zeros(10, dtype=np.float32))
