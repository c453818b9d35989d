// Batched instances (many independent meshes in one persistent launch) and
// the launch-shape autotuner.
//
// A batch context owns n single-instance contexts (mesh, factor, work
// vectors) and lays the per-rollout state of all of them out contiguously
// (control words, prox warm-start stretches, checkpoints, tau), so that one
// memset per array resets every instance. A rollout or an adjoint is ONE
// cooperative launch of the batched persistent kernel: its grid is split into
// teams, one per instance, sized by the launch shape. The per-instance Dev
// records, the prefix offsets and the block -> team maps are uploaded only
// when they change (factor, checkpoint growth, new launch shape), so an
// enqueue issues memsets and one launch: it can be captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pd_ctx.h"
#include "pd_launch.h"

using namespace pdh;

struct pd_batch {
  int n = 0;
  std::vector<pd_ctx*> kids;
  std::vector<pdk::InstOff> off;   // [n+1] prefix offsets (vertices, elements)
  Ctrl* ctrl = nullptr;            // [n] control words
  double* sstar = nullptr;         // [sum n_e][3] prox warm-start stretches
  double* ckpt = nullptr;          // instance i: [(cap_T+1)][n_v_i][3] at (cap_T+1) * 3 * off[i].v
  double* tau = nullptr;           // [n][cap_T]
  int cap_T = 0;
  Dev* d_devs = nullptr;           // [2n] device copies of the instances' Dev records: forward, then adjoint
  pdk::InstOff* d_off = nullptr;   // [n+1]
  int4* d_team[2] = {nullptr, nullptr};  // block -> {instance, index in team, team size} (forward, backward)
  int team_cap = 0;                // entries allocated per map
  int grid[2] = {0, 0};            // blocks of the current maps
  std::vector<int> tsize[2];       // team sizes of the current maps
  bool devs_dirty = true, team_dirty[2] = {true, true};
  std::vector<double> work[2];     // bytes per iteration of each instance (forward, backward)
  std::vector<double> iters[2];    // iterations per step of each instance in the last rollout / adjoint
  std::vector<double> tmeas[2];    // seconds per step of each instance's team in the last launch ...
  std::vector<int> bmeas[2];       // ... with this many blocks
  bool have_iters[2] = {false, false};
  bool freeze_iters = false;       // the autotuner's probes leave the weights alone
  std::vector<Ctrl> hctrl;
  std::vector<pd_stats> inst;
};

namespace {

// whether some instance solves in mode T (its launch requests the dynamic
// shared staging of the triangular sweeps)
bool any_tmode(const pd_batch& B) {
  for (const pd_ctx* k : B.kids)
    if (k->d.tmode) return true;
  return false;
}

// Team sizes minimise the largest predicted instance time: every instance
// gets one block, then blocks go one at a time to the instance whose
// predicted time is largest, until the co-resident grid is used up or every
// team holds ceil(n_e / min_items) blocks. Predicted time with b blocks:
// the instance's measured time in the last launch scaled by
// (measured team size / b)^gamma, or, before any measurement, iterations x
// bytes per iteration / b^gamma.
std::vector<int> team_sizes(const pd_batch& B, int dir, int G, double gamma, int min_items) {
  const int n = B.n;
  std::vector<double> base(n), ref(n);
  std::vector<int> cap(n), b(n, 1);
  const bool timed = B.tmeas[dir].size() == (size_t)n && B.bmeas[dir].size() == (size_t)n;
  for (int i = 0; i < n; ++i) {
    if (timed && B.tmeas[dir][i] > 0) {
      base[i] = B.tmeas[dir][i];
      ref[i] = std::max(B.bmeas[dir][i], 1);
    } else {
      base[i] = std::max(B.iters[dir][i], 1.0) * B.work[dir][i];
      ref[i] = 1.0;
    }
    cap[i] = std::max(1, (B.kids[i]->n_e + min_items - 1) / min_items);
  }
  auto pred = [&](int i) { return base[i] * std::pow(ref[i] / b[i], gamma); };
  int used = n;
  while (used < G) {
    int best = -1;
    double bt = -1.0;
    for (int i = 0; i < n; ++i)
      if (b[i] < cap[i] && pred(i) > bt) {
        bt = pred(i);
        best = i;
      }
    if (best < 0) break;
    ++b[best];
    ++used;
  }
  return b;
}

// team sizes that the launch shape gives now (direction dir: 0 forward, 1 adjoint)
int shape_teams(pd_ctx* c, int dir, std::vector<int>& b) {
  pd_batch& B = *c->batch;
  const bool fp32 = c->opt.local_fp32 != 0;
  const pd_tuning& tn = c->tune;
  int bps = dir ? tn.bwd_blocks_per_sm : tn.fwd_blocks_per_sm;
  if (!dir && bps == 0) bps = 2;   // a batch defaults to the narrow forward shape (more co-resident blocks)
  const int G = dir ? pdk::persistent_grid_bwd(fp32, bps) : pdk::persistent_grid(fp32, bps);
  if (G <= 0) return fail(c, PD_ERR_CUDA, "cooperative launch of the batched kernel is not available");
  if (B.n > G) return fail(c, PD_ERR_TOO_LARGE, "%d instances exceed the %d co-resident blocks", B.n, G);
  if (G > B.team_cap) return fail(c, PD_ERR_ARG, "co-resident grid %d exceeds the team map (%d)", G, B.team_cap);
  double gamma = dir ? tn.bwd_gamma : tn.fwd_gamma;
  int min_items = dir ? tn.bwd_min_items : tn.fwd_min_items;
  if (!(gamma > 0)) gamma = 1.0;
  if (min_items <= 0) min_items = 256;
  b = team_sizes(B, dir, G, gamma, min_items);
  return PD_OK;
}

// Upload what changed since the last launch (Dev records, team map of
// direction dir). Refused while the stream is being captured.
int prepare(pd_ctx* c, cudaStream_t s, int dir) {
  pd_batch& B = *c->batch;
  if ((B.devs_dirty || B.team_dirty[dir]) && capturing(s))
    return fail(c, PD_ERR_ARG, "the batch launch shape changed since the last launch: run it once before capture");
  if (B.devs_dirty) {
    std::vector<Dev> h(2 * (size_t)B.n);   // the forward's records, then the adjoint's
    for (int i = 0; i < B.n; ++i) {
      h[i] = B.kids[i]->d;
      h[B.n + i] = adjoint_dev(B.kids[i]->d);
    }
    CK(cudaMemcpyAsync(B.d_devs, h.data(), 2 * (size_t)B.n * sizeof(Dev), cudaMemcpyHostToDevice, s));
    B.devs_dirty = false;
  }
  if (B.team_dirty[dir]) {
    std::vector<int> b;
    int r = shape_teams(c, dir, b);
    if (r) return r;
    std::vector<int4> map;
    for (int i = 0; i < B.n; ++i)
      for (int k = 0; k < b[i]; ++k) map.push_back(make_int4(i, k, b[i], 0));
    CK(cudaMemcpyAsync(B.d_team[dir], map.data(), map.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    B.grid[dir] = (int)map.size();
    B.tsize[dir] = b;
    B.team_dirty[dir] = false;
  }
  return PD_OK;
}

int collect_batch(pd_ctx* c, cudaStream_t s, int which) {
  pd_batch& B = *c->batch;
  CK(cudaMemcpyAsync(B.hctrl.data(), B.ctrl, B.n * sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  pd_stats& st = c->stats;
  int status = 0, nc = 0, anc = 0;
  if (which & 1) {
    st.steps = c->last_T;
    st.iters_total = st.iters_max = st.aa_resets = st.not_converged = st.tau_half = st.tau_one = 0;
    st.escalations = 0;
    st.warm_fallbacks = 0;
    st.fwd_device_seconds = 0.0;
  }
  if (which & 2) {
    st.adj_iters_total = st.adj_iters_max = st.adj_not_converged = 0;
    st.bwd_device_seconds = 0.0;
  }
  for (int i = 0; i < B.n; ++i) {
    const Ctrl& h = B.hctrl[i];
    pd_stats& si = B.inst[i];
    if (which & 1) {
      si.steps = c->last_T;
      si.iters_total = h.iters_total;
      si.iters_max = h.iters_max;
      si.aa_resets = h.resets;
      si.not_converged = h.not_converged;
      si.tau_half = h.tau_half;
      si.tau_one = h.tau_one;
      si.last_rho = h.last_rho;
      si.escalations = h.escalations;
      si.warm_fallbacks = h.fallbacks;
      st.warm_fallbacks += h.fallbacks;
      si.fwd_device_seconds = h.elapsed_ns[0] * 1e-9;
      st.fwd_device_seconds = std::max(st.fwd_device_seconds, si.fwd_device_seconds);
      st.escalations += h.escalations;
      st.iters_total += h.iters_total;
      st.iters_max = std::max(st.iters_max, h.iters_max);
      st.aa_resets += h.resets;
      st.not_converged += h.not_converged;
      st.tau_half += h.tau_half;
      st.tau_one += h.tau_one;
      nc += h.not_converged ? 1 : 0;
      if (!B.freeze_iters) B.iters[0][i] = std::max(1.0, (double)h.iters_total / std::max(c->last_T, 1));
    }
    if (which & 2) {
      si.adj_iters_total = h.adj_iters_total;
      si.adj_iters_max = h.adj_iters_max;
      si.adj_not_converged = h.adj_not_converged;
      si.bwd_device_seconds = h.elapsed_ns[1] * 1e-9;
      st.bwd_device_seconds = std::max(st.bwd_device_seconds, si.bwd_device_seconds);
      st.adj_iters_total += h.adj_iters_total;
      st.adj_iters_max = std::max(st.adj_iters_max, h.adj_iters_max);
      st.adj_not_converged += h.adj_not_converged;
      anc += h.adj_not_converged ? 1 : 0;
      if (!B.freeze_iters) B.iters[1][i] = std::max(1.0, (double)h.adj_iters_total / std::max(c->last_T, 1));
    }
    si.status_flags = h.status;
    status |= h.status;
    if (!B.freeze_iters) {
      for (int dir = 0; dir < 2; ++dir) {
        if (!(which & (1 << dir))) continue;
        B.tmeas[dir].resize(B.n, 0.0);
        B.bmeas[dir].resize(B.n, 1);
        B.tmeas[dir][i] = (double)h.elapsed_ns[dir] * 1e-9 / std::max(c->last_T, 1);
        B.bmeas[dir][i] = B.tsize[dir].size() == (size_t)B.n ? B.tsize[dir][i] : 1;
      }
    }
  }
  if (!B.freeze_iters) {
    if (which & 1) B.have_iters[0] = true;
    if (which & 2) B.have_iters[1] = true;
  }
  st.status_flags = status;
  if (status & 4) return fail(c, PD_ERR_TIMEOUT, "a team barrier of the batched persistent launch timed out");
  if ((which & 1) && (status & 1)) return fail(c, PD_ERR_NUMERIC, "non-finite value in an instance's right-hand side");
  if ((which & 2) && (status & 2))
    return fail(c, PD_ERR_NUMERIC, "adjoint operator A - K not positive along a CG direction in an instance");
  if (nc) return fail(c, PD_ERR_NOT_CONVERGED, "%d instance(s) had steps that hit k_max", nc);
  if (anc) return fail(c, PD_ERR_NOT_CONVERGED, "%d instance(s) had adjoint solves that hit adj_max_iters", anc);
  return PD_OK;
}

void free_rollout_storage(pd_batch& B) {
  if (B.ckpt) cudaFree(B.ckpt);
  if (B.tau) cudaFree(B.tau);
  B.ckpt = nullptr;
  B.tau = nullptr;
  B.cap_T = 0;
}

}  // namespace

int batch_reserve(pd_ctx* c, int T) {
  pd_batch& B = *c->batch;
  if (B.cap_T >= T) return PD_OK;
  free_rollout_storage(B);
  const size_t nv3 = 3 * (size_t)B.off[B.n].v;
  if (cudaMalloc(&B.ckpt, (size_t)(T + 1) * nv3 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&B.tau, (size_t)B.n * T * sizeof(double)) != cudaSuccess) {
    free_rollout_storage(B);
    return fail(c, PD_ERR_OOM, "checkpoint allocation for %d steps of %d instances", T, B.n);
  }
  B.cap_T = T;
  for (int i = 0; i < B.n; ++i) {
    Dev& d = B.kids[i]->d;
    d.ckpt = B.ckpt + (size_t)(T + 1) * 3 * B.off[i].v;
    d.tau = B.tau + (size_t)i * T;
    d.phase_count = nullptr;
  }
  B.devs_dirty = true;
  return PD_OK;
}

int batch_factor(pd_ctx* c) {
  pd_batch& B = *c->batch;
  auto t0 = std::chrono::steady_clock::now();
  c->factored = false;
  std::vector<int> rc(B.n, PD_OK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < B.n; ++i) {
    if (cudaSetDevice(c->device) != cudaSuccess) {
      rc[i] = PD_ERR_CUDA;
      continue;
    }
    rc[i] = pd_factor(B.kids[i]);
  }
  int64_t nnz = 0, nnzL = 0;
  int nf = 0, smode = 0, slev = 0;
  for (int i = 0; i < B.n; ++i) {
    if (rc[i]) return fail(c, rc[i], "instance %d: %s", i, B.kids[i]->err.c_str());
    const pd_ctx* k = B.kids[i];
    const double m = k->opt.aa_m;
    // bytes per iteration (forward: local step + assembly + two SpMVs with S +
    // Anderson; backward: K apply + PCG vectors + two SpMVs)
    // (solve: 20 B per non-zero of S, or 16 B per partitioned-inverse entry
    // in mode T: one copy per sweep)
    const double solve_b = (k->tmode ? 16.0 : 20.0) * (double)k->solve_nnz;
    B.work[0][i] = 56.0 * k->n_e + 48.0 * k->n_v + solve_b + 96.0 * k->n_f + (2 * m + 3) * 24.0 * k->n_v;
    B.work[1][i] = 200.0 * k->n_e + solve_b + 240.0 * k->n_v;
    B.inst[i].factor_nnz = k->solve_nnz;
    B.inst[i].n_free = k->n_f;
    B.inst[i].factor_seconds = k->factor_seconds;
    B.inst[i].solve_mode = k->tmode ? PD_SOLVE_T : PD_SOLVE_S;
    B.inst[i].solve_levels = k->solve_levels;
    B.inst[i].nnz_L = k->fac.nnz_L;
    nnz += k->solve_nnz;
    nnzL += k->fac.nnz_L;
    smode = std::max(smode, B.inst[i].solve_mode);
    slev = std::max(slev, k->solve_levels);
    nf += k->n_f;
    // per-instance Dev records must point at the batch's contiguous state
    B.kids[i]->d.ctrl = B.ctrl + i;
    B.kids[i]->d.sstar = B.sstar + 3 * B.off[i].e;
  }
  c->factored = true;
  c->factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->stats.factor_seconds = c->factor_seconds;
  c->stats.factor_nnz = nnz;
  c->stats.n_free = nf;
  c->stats.solve_mode = smode;
  c->stats.solve_levels = slev;
  c->stats.nnz_L = nnzL;
  B.devs_dirty = true;
  B.team_dirty[0] = B.team_dirty[1] = true;
  return PD_OK;
}

int batch_rollout(pd_ctx* c, int T, const double* q0, const double* v0, const double* f_ext, int64_t f_stride,
                  double* qT, double* vT, cudaStream_t s, bool sync) {
  pd_batch& B = *c->batch;
  const size_t nv3 = 3 * (size_t)B.off[B.n].v;
  if (f_stride != 0 && f_stride != (int64_t)nv3) return fail(c, PD_ERR_ARG, "f_ext_stride must be 0 or 3 x total vertices");
  int r;
  if (B.cap_T < T) {
    if (!sync && capturing(s))
      return fail(c, PD_ERR_ARG, "checkpoint storage for %d steps is missing: call pd_reserve before capture", T);
    if ((r = batch_reserve(c, T))) return r;
  }
  const double* q0d = q0;
  const double* v0d = v0;
  const double* fd = f_ext;
  double* qTd = qT;
  double* vTd = vT;
  bool hqo = false, hvo = false;
  double *st_qo = nullptr, *st_vo = nullptr;
  if (sync) {  // host pointers are staged through one device buffer
    const bool hq = !is_device_ptr(q0), hv = !is_device_ptr(v0), hf = f_ext && !is_device_ptr(f_ext);
    hqo = qT && !is_device_ptr(qT);
    hvo = vT && !is_device_ptr(vT);
    const size_t nf_ext = f_ext ? (f_stride ? (size_t)T * nv3 : nv3) : 0;
    if ((r = ensure_stage(c, 4 * nv3 + (hf ? nf_ext : 0)))) return r;
    st_qo = c->stage + 2 * nv3;
    st_vo = c->stage + 3 * nv3;
    if (hq) { CK(cudaMemcpyAsync(c->stage, q0, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); q0d = c->stage; }
    if (hv) { CK(cudaMemcpyAsync(c->stage + nv3, v0, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); v0d = c->stage + nv3; }
    if (hf) {
      CK(cudaMemcpyAsync(c->stage + 4 * nv3, f_ext, nf_ext * sizeof(double), cudaMemcpyHostToDevice, s));
      fd = c->stage + 4 * nv3;
    }
    if (hqo) qTd = st_qo;
    if (hvo) vTd = st_vo;
  }
  if ((r = prepare(c, s, 0))) return r;
  CK(cudaMemsetAsync(B.tau, 0, (size_t)B.n * B.cap_T * sizeof(double), s));
  CK(cudaMemsetAsync(B.ctrl, 0, (size_t)B.n * sizeof(Ctrl), s));
  CK(cudaMemsetAsync(B.sstar, 0, 3 * (size_t)B.off[B.n].e * sizeof(double), s));
  pdk::BatchFwd br;
  br.T = T;
  br.q0 = q0d;
  br.v0 = v0d;
  br.fext = fd;
  br.f_stride = f_stride;
  br.qT = qTd;
  br.vT = vTd;
  CK(pdk::launch_fwd_rollout(c->opt.local_fp32 != 0, B.d_devs, B.d_team[0], B.d_off, br, B.grid[0], any_tmode(B), s));
  c->launches += 1;
  c->last_T = T;
  for (pd_ctx* k : B.kids) k->last_T = T;
  if (!sync) {
    c->pending |= 1;
    return PD_OK;
  }
  if (hqo) CK(cudaMemcpyAsync(qT, st_qo, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (hvo) CK(cudaMemcpyAsync(vT, st_vo, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  c->pending = 0;
  return collect_batch(c, s, 1);
}

int batch_backward(pd_ctx* c, const double* dqT, const double* dvT, double* dq0, double* dv0, double* dE, double* dnu,
                   double* df, int64_t df_stride, cudaStream_t s, bool sync) {
  pd_batch& B = *c->batch;
  const size_t nv3 = 3 * (size_t)B.off[B.n].v;
  const size_t ne = (size_t)B.off[B.n].e;
  const int T = c->last_T;
  if (df_stride != 0 && df_stride != (int64_t)nv3) return fail(c, PD_ERR_ARG, "df_stride must be 0 or 3 x total vertices");
  int r;
  const double* dqTd = dqT;
  const double* dvTd = dvT;
  double *dq0d = dq0, *dv0d = dv0, *dEd = dE, *dnud = dnu, *dfd = df;
  bool h_q0 = false, h_v0 = false, h_E = false, h_nu = false, h_df = false;
  const size_t ndf = df ? (df_stride ? (size_t)T * nv3 : nv3) : 0;
  double *st_q0 = nullptr, *st_v0 = nullptr, *st_E = nullptr, *st_nu = nullptr, *st_df = nullptr;
  if (sync) {
    const bool h_dq = !is_device_ptr(dqT), h_dv = dvT && !is_device_ptr(dvT);
    h_q0 = dq0 && !is_device_ptr(dq0);
    h_v0 = dv0 && !is_device_ptr(dv0);
    h_E = dE && !is_device_ptr(dE);
    h_nu = dnu && !is_device_ptr(dnu);
    h_df = df && !is_device_ptr(df);
    if ((r = ensure_stage(c, 4 * nv3 + ne + B.n + ndf))) return r;
    st_q0 = c->stage + 2 * nv3;
    st_v0 = c->stage + 3 * nv3;
    st_E = c->stage + 4 * nv3;
    st_nu = st_E + ne;
    st_df = st_nu + B.n;
    if (h_dq) { CK(cudaMemcpyAsync(c->stage, dqT, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); dqTd = c->stage; }
    if (h_dv) {
      CK(cudaMemcpyAsync(c->stage + nv3, dvT, nv3 * sizeof(double), cudaMemcpyHostToDevice, s));
      dvTd = c->stage + nv3;
    }
    if (h_q0) dq0d = st_q0;
    if (h_v0) dv0d = st_v0;
    if (h_E) dEd = st_E;
    if (h_nu) dnud = st_nu;
    if (h_df) dfd = st_df;
  }
  if ((r = prepare(c, s, 1))) return r;
  // barrier counters of every team start at zero (a timed-out launch may leave them set)
  CK(cudaMemset2DAsync(&B.ctrl[0].bar_arrive, sizeof(Ctrl), 0, sizeof(unsigned long long), B.n, s));
  if (dfd && df_stride == 0) CK(cudaMemsetAsync(dfd, 0, nv3 * sizeof(double), s));
  pdk::BatchBwd br;
  br.T = T;
  br.dqT = dqTd;
  br.dvT = dvTd;
  br.dq0 = dq0d;
  br.dv0 = dv0d;
  br.dE = dEd;
  br.dnu = dnud;
  br.df = dfd;
  br.df_stride = df_stride;
  CK(pdk::launch_bwd_rollout(c->opt.local_fp32 != 0, B.d_devs + B.n, B.d_team[1], B.d_off, br, B.grid[1], any_tmode(B),
                             s));
  c->launches += 1;
  if (!sync) {
    c->pending |= 2;
    return PD_OK;
  }
  if (h_q0) CK(cudaMemcpyAsync(dq0, st_q0, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_v0) CK(cudaMemcpyAsync(dv0, st_v0, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_E) CK(cudaMemcpyAsync(dE, st_E, ne * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_nu) CK(cudaMemcpyAsync(dnu, st_nu, B.n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_df) CK(cudaMemcpyAsync(df, st_df, ndf * sizeof(double), cudaMemcpyDeviceToHost, s));
  c->pending = 0;
  return collect_batch(c, s, 2);
}

int batch_collect(pd_ctx* c, cudaStream_t s) {
  const int which = c->pending;
  c->pending = 0;
  if (!which) {
    CK(cudaStreamSynchronize(s));
    return PD_OK;
  }
  return collect_batch(c, s, which);
}

int batch_get_mass(const pd_ctx* c, double* m) {
  const pd_batch& B = *c->batch;
  for (int i = 0; i < B.n; ++i) std::memcpy(m + B.off[i].v, B.kids[i]->mass.data(), B.kids[i]->mass.size() * sizeof(double));
  return PD_OK;
}

int batch_size(const pd_ctx* c) { return c->batch ? c->batch->n : 1; }

void batch_set_warm(pd_ctx* c, int mode) {
  pd_batch& B = *c->batch;
  for (pd_ctx* k : B.kids) {
    k->opt.warm_start = mode;
    k->d.warm = mode;
  }
  B.devs_dirty = true;
}

pd_ctx* batch_kid(const pd_ctx* c, int i, int64_t* v_off) {
  const pd_batch& B = *c->batch;
  if (v_off) *v_off = B.off[i].v;
  return B.kids[i];
}

int batch_get_checkpoint(const pd_ctx* c, int t, double* q_host) {
  const pd_batch& B = *c->batch;
  if (!q_host || t < 0 || t > c->last_T || !B.ckpt) return PD_ERR_ARG;
  for (int i = 0; i < B.n; ++i) {
    const size_t nv3 = 3 * (size_t)B.kids[i]->n_v;
    if (cudaMemcpy(q_host + 3 * B.off[i].v, B.kids[i]->d.ckpt + (size_t)t * nv3, nv3 * sizeof(double),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return PD_ERR_CUDA;
  }
  return PD_OK;
}

int batch_get_tau(const pd_ctx* c, double* tau_host, int T) {
  const pd_batch& B = *c->batch;
  if (!tau_host || T < 1 || T > c->last_T || !B.tau) return PD_ERR_ARG;
  for (int i = 0; i < B.n; ++i)
    if (cudaMemcpy(tau_host + (size_t)i * T, B.kids[i]->d.tau, T * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return PD_ERR_CUDA;
  return PD_OK;
}

int batch_mlp_load(pd_ctx* c, const void* blob, size_t bytes) {
  pd_batch& B = *c->batch;
  pdk::MlpDev m{};
  const int r = mlp_upload(c, blob, bytes, &m, c->allocs);
  if (r) return r;
  for (pd_ctx* k : B.kids) k->d.mlp = m;
  B.devs_dirty = true;
  return PD_OK;
}

bool batch_has_mlp(const pd_ctx* c) { return !c->batch->kids.empty() && c->batch->kids[0]->d.mlp.w != nullptr; }

void batch_destroy(pd_ctx* c) {
  pd_batch* B = c->batch;
  for (pd_ctx* k : B->kids) pd_destroy(k);
  free_rollout_storage(*B);
  void* bufs[] = {B->ctrl, B->sstar, B->d_devs, B->d_off, B->d_team[0], B->d_team[1]};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete B;
  c->batch = nullptr;
}

// ------------------------------------------------------------ autotuner

namespace {

std::mutex g_tune_mu;
std::map<std::string, pd_tuning> g_tune_cache;

std::string signature(const pd_ctx* c) {
  int dev = c->device;
  cudaDeviceProp p;
  std::string key;
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) key = std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
  else cudaGetLastError();
  key += "|fp32=" + std::to_string(c->opt.local_fp32) + "|m=" + std::to_string(c->opt.aa_m);
  auto one = [&](const pd_ctx* k) {
    key += "|" + std::to_string(k->model) + ":" + std::to_string(k->n_v) + ":" + std::to_string(k->n_e) + ":" +
           std::to_string(k->n_f) + ":" + std::to_string(k->nnz_S);
  };
  if (c->batch)
    for (const pd_ctx* k : c->batch->kids) one(k);
  else
    one(c);
  return key;
}

void mark_shape_changed(pd_ctx* c) {
  if (c->batch) c->batch->team_dirty[0] = c->batch->team_dirty[1] = true;
}

}  // namespace

extern "C" {

int pd_create_batch(int32_t n, const pd_mesh* meshes, const pd_material* mats, double dt, const pd_options* opt,
                    pd_ctx** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !meshes || !mats) return PD_ERR_ARG;
  pd_ctx* c = new pd_ctx();
  *out = c;
  if (opt) c->opt = *opt; else pd_default_options(&c->opt);
  c->dt = dt;
  c->batch = new pd_batch();
  pd_batch& B = *c->batch;
  B.n = n;
  B.off.assign(n + 1, pdk::InstOff{0, 0});
  for (int i = 0; i < n; ++i) {
    pd_ctx* k = nullptr;
    const int r = pd_create(&meshes[i], &mats[i], dt, &c->opt, &k);
    if (r) {
      fail(c, r, "instance %d: %s", i, k ? k->err.c_str() : "invalid arguments");
      if (k) pd_destroy(k);
      return r;
    }
    B.kids.push_back(k);
    B.off[i + 1].v = B.off[i].v + k->n_v;
    B.off[i + 1].e = B.off[i].e + k->n_e;
  }
  if (B.off[n].v > 0x7fffffffLL || B.off[n].e > 0x7fffffffLL)
    return fail(c, PD_ERR_TOO_LARGE, "total vertices / elements exceed 2^31 - 1");
  c->n_v = (int)B.off[n].v;
  c->n_e = (int)B.off[n].e;
  c->device = B.kids[0]->device;
  c->model = B.kids[0]->model;
  for (int k = 0; k < 2; ++k) {
    B.work[k].assign(n, 1.0);
    B.iters[k].assign(n, 1.0);
  }
  B.hctrl.assign(n, Ctrl{});
  B.inst.assign(n, pd_stats{});
  const bool fp32 = c->opt.local_fp32 != 0;
  B.team_cap = std::max(std::max(pdk::persistent_grid_max(fp32), pdk::persistent_grid_bwd(fp32, 0)), 1);
  CK(cudaMalloc(&B.ctrl, n * sizeof(Ctrl)));
  CK(cudaMemset(B.ctrl, 0, n * sizeof(Ctrl)));
  CK(cudaMalloc(&B.sstar, 3 * (size_t)std::max<long long>(B.off[n].e, 1) * sizeof(double)));
  CK(cudaMalloc(&B.d_devs, 2 * (size_t)n * sizeof(Dev)));
  CK(cudaMalloc(&B.d_off, (n + 1) * sizeof(pdk::InstOff)));
  CK(cudaMemcpy(B.d_off, B.off.data(), (n + 1) * sizeof(pdk::InstOff), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&B.d_team[0], B.team_cap * sizeof(int4)));
  CK(cudaMalloc(&B.d_team[1], B.team_cap * sizeof(int4)));
  for (int i = 0; i < n; ++i) {
    B.kids[i]->d.ctrl = B.ctrl + i;
    B.kids[i]->d.sstar = B.sstar + 3 * B.off[i].e;
  }
  return PD_OK;
}

int pd_batch_info(const pd_ctx* c, int32_t* n, int64_t* v_off, int64_t* e_off) {
  if (!c) return PD_ERR_ARG;
  if (!c->batch) {
    if (n) *n = 1;
    if (v_off) { v_off[0] = 0; v_off[1] = c->n_v; }
    if (e_off) { e_off[0] = 0; e_off[1] = c->n_e; }
    return PD_OK;
  }
  const pd_batch& B = *c->batch;
  if (n) *n = B.n;
  for (int i = 0; i <= B.n; ++i) {
    if (v_off) v_off[i] = B.off[i].v;
    if (e_off) e_off[i] = B.off[i].e;
  }
  return PD_OK;
}

int pd_set_materials_batch(pd_ctx* c, const double* E, const double* nu) {
  if (!c || !E || !nu) return PD_ERR_ARG;
  if (!c->batch) return pd_set_materials(c, E, nu[0]);
  pd_batch& B = *c->batch;
  for (int i = 0; i < B.n; ++i) {
    const int r = pd_set_materials(B.kids[i], E + B.off[i].e, nu[i]);
    if (r) return fail(c, r, "instance %d: %s", i, B.kids[i]->err.c_str());
  }
  c->factored = false;
  return PD_OK;
}

int pd_get_instance_stats(const pd_ctx* c, int32_t i, pd_stats* out) {
  if (!c || !out) return PD_ERR_ARG;
  if (!c->batch) {
    if (i != 0) return PD_ERR_ARG;
    return pd_get_stats(c, out);
  }
  if (i < 0 || i >= c->batch->n) return PD_ERR_ARG;
  *out = c->batch->inst[i];
  return PD_OK;
}

int pd_batch_teams(pd_ctx* c, int32_t* fwd, int32_t* bwd) {
  if (!c) return PD_ERR_ARG;
  if (!c->batch) return fail(c, PD_ERR_ARG, "pd_batch_teams needs a batch context");
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_batch_teams");
  CK(cudaSetDevice(c->device));
  pd_batch& B = *c->batch;
  int32_t* out[2] = {fwd, bwd};
  for (int dir = 0; dir < 2; ++dir) {
    if (!out[dir]) continue;
    std::vector<int> b = B.tsize[dir];
    if (B.team_dirty[dir]) {
      const int r = shape_teams(c, dir, b);
      if (r) return r;
    }
    for (int i = 0; i < B.n; ++i) out[dir][i] = b[i];
  }
  return PD_OK;
}

int pd_get_tuning(const pd_ctx* c, pd_tuning* out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = c->tune;
  return PD_OK;
}

int pd_set_tuning(pd_ctx* c, const pd_tuning* t) {
  if (!c || !t) return PD_ERR_ARG;
  if (t->fwd_blocks_per_sm < 0 || t->fwd_blocks_per_sm > 2 || t->bwd_blocks_per_sm < 0 || t->bwd_blocks_per_sm > 2 ||
      t->fwd_grid < 0 || t->bwd_grid < 0 || t->fwd_min_items < 0 || t->bwd_min_items < 0)
    return fail(c, PD_ERR_ARG, "invalid launch shape");
  c->tune = *t;
  c->tuned = true;
  mark_shape_changed(c);
  return PD_OK;
}

int pd_autotune(pd_ctx* c, int32_t T_probe, const double* q0, const double* v0, const double* f_ext, int64_t f_stride,
                pd_tuning* out, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_autotune");
  if (T_probe < 1 || !q0 || !v0) return fail(c, PD_ERR_ARG, "T_probe >= 1 and q0, v0 are required");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = signature(c);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->tune = it->second;
      c->tune.candidates = 0;
      c->tuned = true;
      mark_shape_changed(c);
      if (out) *out = c->tune;
      return PD_OK;
    }
  }
  const size_t nv3 = 3 * (size_t)c->n_v;
  double *qT = nullptr, *vT = nullptr, *g = nullptr;
  CK(cudaMalloc(&qT, nv3 * sizeof(double)));
  CK(cudaMalloc(&vT, nv3 * sizeof(double)));
  CK(cudaMalloc(&g, (2 * nv3 + c->n_e + (c->batch ? c->batch->n : 1)) * sizeof(double)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const pd_tuning saved = c->tune;
  int rc = PD_OK;
  // probe: time one enqueued rollout (dir 0) or adjoint (dir 1); a probe
  // that ends in PD_ERR_NOT_CONVERGED still counts (its time is what the
  // shape costs); any other error aborts the tuning
  auto probe = [&](int dir, double* ms) -> int {
    int r = PD_OK;
    if (cudaEventRecord(e0, s) != cudaSuccess) return fail(c, PD_ERR_CUDA, "event record");
    if (dir == 0)
      r = pd_rollout_enqueue(c, T_probe, q0, v0, f_ext, f_stride, qT, vT, s);
    else
      r = pd_backward_enqueue(c, qT, nullptr, g, g + nv3, g + 2 * nv3, g + 2 * nv3 + c->n_e, nullptr, 0, s);
    if (r) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess) return fail(c, PD_ERR_CUDA, "event record");
    r = pd_collect(c, s);
    if (r && r != PD_ERR_NOT_CONVERGED) return r;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return fail(c, PD_ERR_CUDA, "event timing");
    *ms = f;
    return PD_OK;
  };
  struct Cand {
    int bps, grid;
    double gamma;
    int min_items;
  };
  std::vector<Cand> cands;
  if (c->batch) {
    // two blocks per SM (fewer co-resident blocks never helps a batch)
    for (double gm : {0.5, 0.75, 1.0})
      for (int mi : {32, 128, 512}) cands.push_back({2, 0, gm, mi});
  } else {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const bool fp32 = c->opt.local_fp32 != 0;
    const int full = std::min(pdk::persistent_grid_max(fp32), pdk::persistent_grid_bwd(fp32, 0));
    for (int gsz : {sms / 2, sms, (3 * sms) / 2, 2 * sms})
      if (gsz >= 1 && gsz <= full) cands.push_back({0, gsz, 1.0, 256});
  }
  double best_ms[2] = {1e300, 1e300};
  Cand best[2] = {cands.empty() ? Cand{0, 0, 1.0, 256} : cands[0], cands.empty() ? Cand{0, 0, 1.0, 256} : cands[0]};
  auto apply = [&](const Cand& k) {
    pd_tuning t = saved;
    t.fwd_blocks_per_sm = t.bwd_blocks_per_sm = k.bps;
    t.fwd_grid = t.bwd_grid = k.grid;
    t.fwd_gamma = t.bwd_gamma = k.gamma;
    t.fwd_min_items = t.bwd_min_items = k.min_items;
    c->tune = t;
    mark_shape_changed(c);
  };
  // the team sizes are weighed by per-instance iterations per step: those of
  // the last full rollout / adjoint if there was one (representative of the
  // whole horizon), else of a first probe at the starting shape; the
  // candidates' probes then leave the weights unchanged
  double warm = 0;
  const bool measured = c->batch && c->batch->have_iters[0] && c->batch->have_iters[1];
  if (measured) c->batch->freeze_iters = true;
  if ((rc = probe(0, &warm)) == PD_OK) rc = probe(1, &warm);
  if (c->batch) c->batch->freeze_iters = true;
  for (int dir = 0; dir < 2 && rc == PD_OK; ++dir) {
    if (dir == 1) {  // the adjoint probes need the checkpoints of one forward
      apply(best[0]);
      if ((rc = probe(0, &warm))) break;
    }
    for (const Cand& k : cands) {
      apply(k);
      // batches are probed once per shape (long launches, little noise);
      // a single instance twice, keeping the faster
      double t1 = 0, t2 = 1e300;
      if ((rc = probe(dir, &t1))) break;
      if (!c->batch && (rc = probe(dir, &t2))) break;
      const double t = std::min(t1, t2);
      if (t < best_ms[dir]) {
        best_ms[dir] = t;
        best[dir] = k;
      }
    }
  }
  if (c->batch) c->batch->freeze_iters = false;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(qT);
  cudaFree(vT);
  cudaFree(g);
  if (rc) {
    c->tune = saved;
    mark_shape_changed(c);
    return rc;
  }
  pd_tuning t = saved;
  t.fwd_blocks_per_sm = best[0].bps;
  t.fwd_grid = best[0].grid;
  t.fwd_gamma = best[0].gamma;
  t.fwd_min_items = best[0].min_items;
  t.bwd_blocks_per_sm = best[1].bps;
  t.bwd_grid = best[1].grid;
  t.bwd_gamma = best[1].gamma;
  t.bwd_min_items = best[1].min_items;
  t.fwd_ms = best_ms[0];
  t.bwd_ms = best_ms[1];
  t.candidates = (int)cands.size();
  c->tune = t;
  c->tuned = true;
  mark_shape_changed(c);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = t;
  }
  if (out) *out = t;
  return PD_OK;
}

}  // extern "C"
