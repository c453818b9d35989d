// Persistent forward rollout: one cooperative launch runs all T steps of
// Alg. 1 (step begin, local/global iterations with Anderson mixing and the
// dual gate, step end, trust-region selection).
//
// Synchronisation: phases are separated by team barriers on a monotonic
// arrival counter (pd_grid.cuh). In a reduction every block adds all the
// team's partial rows in a fixed order (deterministic, the same bits in
// every block) and then runs the phase's scalar logic (pd_phases.cuh) on its
// own shared-memory replica of the iteration state, so all blocks take
// identical decisions without a serial chain of global-memory accesses. The grid is co-resident
// (cooperative launch) and every wait is bounded: on timeout a status bit is
// set and every block returns.
#include <cuda_runtime.h>

#include "pd_coop.h"
#include "pd_grid.cuh"
#include "pd_mlp.cuh"
#include "pd_contact.cuh"
#include "pd_launch.h"
#include "pd_phases.cuh"
#include "pd_tsolve.cuh"

namespace pdk {

// local step / assembly in the kernel's precision T, or in FP64 once an FP32
// team has escalated (the FP64 local step is a real call: it runs rarely and,
// inlined, its registers would count against every phase of the body)
__device__ __noinline__ void local_item_hi(const Dev& d, int e) { local_item<double>(d, e, d.q); }
template <typename T>
__device__ __forceinline__ void local_any(const Dev& d, int e, bool hi) {
  if constexpr (sizeof(T) == 4) {
    if (hi) local_item_hi(d, e);
    else local_item<float>(d, e, d.q, d.qhl);
  } else {
    local_item<T>(d, e, d.q);
  }
}
template <typename T>
__device__ __forceinline__ void assemble_any(const Dev& d, int v, int k, double* part, bool hi, int lane) {
  if constexpr (sizeof(T) == 4) {
    if (hi) assemble_warp<double>(d, v, k, part, lane);
    else assemble_warp<float>(d, v, k, part, lane);
  } else {
    assemble_warp<T>(d, v, k, part, lane);
  }
}

// mode T: each finished row j of q_hat (elimination order) goes to q_hat and
// to the Anderson work of its vertex (lanes 0..2, partials in shared memory)
struct FinAA {
  const Dev* d;
  AAView av;
  double* pa;    // this lane's partials (lanes 0..2)
  double* pa0;   // the warp's lane-0 partials
  __device__ __forceinline__ void operator()(int j, double a0, double a1, double a2) const {
    const int lane = threadIdx.x & 31;
    if (lane < 3) {
      const size_t o = 3 * (size_t)d->perm[j] + lane;
      const double qh = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
      d->qhat[o] = qh;
      aa_component(*d, o, qh, av, pa);
    }
  }
  // every lane with its own row: the three components each, then the warp's
  // sum of the partials into lane 0's (a fixed shuffle tree)
  __device__ __forceinline__ void lanes(bool on, int j, double a0, double a1, double a2) const {
    double part[2 * kMaxAA];
#pragma unroll
    for (int i = 0; i < 2 * kMaxAA; ++i) part[i] = 0.0;
    if (on) {
      const size_t o = 3 * (size_t)d->perm[j];
      d->qhat[o] = a0;
      d->qhat[o + 1] = a1;
      d->qhat[o + 2] = a2;
      aa_component(*d, o, a0, av, part);
      aa_component(*d, o + 1, a1, av, part);
      aa_component(*d, o + 2, a2, av, part);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 2 * kMaxAA; ++i) {
      double v = part[i];
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
      if (lane == 0) pa0[i] += v;
    }
  }
};

// the network warm start as a real call: it runs once per step and, inlined,
// its registers would count against every phase of the body
__device__ __noinline__ void warm_vertex_call(const Dev& d, int v, const double* vin, int lane) {
  warm_vertex(d, v, d.qt, nullptr, vin, d.q, d.qprev, lane, d.qhl);
}
// the network on the tensor pipe: 16 vertices per warp
__device__ __noinline__ void warm_tile_call(const Dev& d, int v0, const double* vin, int lane) {
  warm_tile(d, v0, d.qt, nullptr, vin, d.q, d.qprev, lane, d.qhl);
}

template <typename T>
__device__ __forceinline__ void fwd_rollout_body(const Dev& d, const RollArgs& a, const Team tm) {
  __shared__ FwdState S;
  __shared__ double sums[2 * kMaxAA];
  __shared__ double s_pa[kFwdWideBlock / 32][3][2 * kMaxAA];
  const int tid = threadIdx.x;
  const int gtid = tm.b * blockDim.x + tid;
  const int gthreads = tm.nb * blockDim.x;
  const int lane = tid & 31, gwarp = gtid >> 5, nwarps = gthreads >> 5;
  // a large team numbers its warps block-minor for the row-wise products:
  // consecutive rows (segments of one long row of S, rows of similar
  // length) go to different SMs, so the FP64 work of the long rows spreads
  // over the team (bar, 148 blocks: 204 -> 217.5 PD steps/s); a small team
  // keeps neighbouring rows, whose S^T rows share their ancestors' y values,
  // on one SM's L1 (64-mesh batch: 437 vs 414 instance PD steps/s)
  const int twarp = tm.nb >= kWideTeam ? (tid >> 5) * tm.nb + tm.b : gwarp;
  const size_t nv3 = 3 * (size_t)d.n_v;
  const bool writer = tm.b == 0;
  const Range re = block_range(tm, d.n_e);
  const Range rv = block_range(tm, d.n_v);
  const Range rt = block_range(tm, d.n_e + d.n_v);
  // phase timers (thread 0 only; kept in shared memory, off the registers):
  // ph block 0's phase times, wk block 0's own work, wall with d.prof every
  // block's own work per phase (from the end of the previous phase to the end
  // of its work; the largest total over the team is the critical block's),
  // lst with d.prof the time from block 0's phase start to the last block's
  // arrival at the phase's closing barrier
  __shared__ unsigned long long ph[8], wk[8], wall[8], lst[8], tmr[3];   // tmr: t0, ta, tstart
  if (tid == 0) {
    for (int i = 0; i < 8; ++i) ph[i] = wk[i] = wall[i] = lst[i] = 0;
    tmr[0] = tmr[1] = tmr[2] = 0;
  }
  auto mark = [&](int p) {
    if (tid == 0 && (writer || d.prof)) {
      const unsigned long long t1 = gtimer(), t0 = tmr[0];
      if (writer) ph[p] += t1 - t0;
      if (writer && d.prof && tm.nb > 1) {
        const unsigned long long tl = *(volatile unsigned long long*)&d.ctrl->t_last;
        if (tl > t0 && tl < t1) lst[p] += tl - t0;
      }
      tmr[0] = tmr[1] = t1;
    }
  };
  // block 0's own work of the current phase (before its barrier); all threads
  // of block 0 are done when thread 0 passes this __syncthreads
  auto work_done = [&](int p) {
    if (writer || d.prof) {
      __syncthreads();
      if (tid == 0) {
        const unsigned long long t1 = gtimer();
        if (writer) wk[p] += t1 - tmr[0];
        if (d.prof) wall[p] += t1 - tmr[1];
      }
    }
  };
  if (tid == 0) {
    S.iters_total = S.iters_max = S.resets = S.not_converged = S.tau_half = S.tau_one = S.status = 0;
    S.hi = S.escalations = S.fallbacks = 0;
    S.rot_n = S.rot_f = S.con_iters = S.con_unconverged = 0;
    S.last_rho = 0.0;
    for (int i = 0; i < kMaxAA * kMaxAA; ++i) S.gram[i] = 0.0;
    tmr[0] = tmr[1] = tmr[2] = gtimer();
  }
  // split-row counters start at zero (a launch that timed out may have left
  // some set); the first S b comes after the step's first team barrier
  {
    const Range rc = block_range(tm, d.n_slot);
    for (int i = rc.lo + tid; i < rc.hi; i += blockDim.x) d.s_cnt[i] = 0;
  }
  bool ok = true;
  for (int t = 0; t < a.T && ok; ++t) {
    const double* qin = t == 0 ? a.q0 : a.sq;
    const double* vin = t == 0 ? a.v0 : a.sv;
    const double* fst = a.fext ? a.fext + (a.f_stride ? (size_t)t * (size_t)a.f_stride : 0) : nullptr;
    if (tid == 0) ctrl_step_reset(&S, t);
    for (int v = rv.lo + tid; v < rv.hi; v += blockDim.x) step_begin_item(d, v, qin, vin, fst, a.ckpt + (size_t)t * nv3);
    if (!(ok = grid_sync(d, tm))) break;
    mark(PH_BEGIN);
    // warm start (network or constant-velocity extrapolation); a warm-started
    // step that hits k_max is run again from q_t, the plain start of Alg. 1
    const int nc0 = S.not_converged;
    bool warm_now = d.warm != 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (warm_now) {
        if (d.warm == 1)   // network: 16 vertices per warp on the tensor pipe
          for (int v0 = 16 * gwarp; v0 < d.n_v; v0 += 16 * nwarps) warm_tile_call(d, v0, vin, lane);
        else               // constant velocity: no network
          for (int v = gwarp; v < d.n_v; v += nwarps) warm_vertex_call(d, v, vin, lane);
        if (!(ok = grid_sync(d, tm))) break;
      }
      double pu[2] = {0.0, 0.0};   // step norms of the last update, reduced with the next assembly
      for (;;) {
        const int k = S.k;
        const bool hi = S.hi != 0;   // FP64 local step after an escalation
        for (int e = re.lo + tid; e < re.hi; e += blockDim.x) local_any<T>(d, e, hi);
        work_done(PH_LOCAL);
        if (!(ok = grid_sync(d, tm))) break;
        mark(PH_LOCAL);
        double p5[5] = {0.0, 0.0, 0.0, pu[0], pu[1]};
        for (int v = rv.lo + (tid >> 5); v < rv.hi; v += blockDim.x >> 5) assemble_any<T>(d, v, k, p5, hi, lane);
        work_done(PH_ASSEMBLE);
        if (!(ok = grid_reduce<5>(d, tm, p5, sums))) break;
        if (tid == 0) assemble_finish(d, &S, k, sums, true);
        __syncthreads();
        mark(PH_ASSEMBLE);
        if (S.done) break;
        // Anderson view and per-warp partials of lanes 0..2 (the Anderson work of
        // every finished row of q_hat is fused into the solve)
        const AAView av = aa_view(d, S.pairs, S.ncols, S.head);
        double* pa = &s_pa[tid >> 5][lane < 3 ? lane : 0][0];
        if (d.tmode) {
          // mode T: the two level-scheduled sweeps over the factor's
          // partitioned inverse; each finished row of q_hat goes to the
          // Anderson work as it is written
          if (lane < 3)
            for (int j = 0; j < 2 * kMaxAA; ++j) pa[j] = 0.0;
          FinAA fin{&d, av, pa, &s_pa[tid >> 5][0][0]};
          if (!(ok = tsolve_team(d, reinterpret_cast<const double*>(d.bperm), reinterpret_cast<double*>(d.y), tm,
                                 twarp, nwarps, fin)))
            break;
          mark(PH_SPMV_S);
        } else {
          for (int sg = twarp; sg < d.n_seg; sg += nwarps) spmv_s_segment(d, d.bperm, d.y, d.s_part, d.s_cnt, sg, lane);
          work_done(PH_SPMV_S);
          if (!(ok = grid_sync(d, tm))) break;
          mark(PH_SPMV_S);
          if (d.n_con > 0) {
            // contact: q_u at the candidates, normal LCP, Tresca friction, then
            // y <- y + S J^T lam so that the S^T pass below gives A^-1 (b + J^T lam)
            for (int c = gwarp; c < d.n_con; c += nwarps) contact_gather(d, c, t, lane);
            if (!(ok = grid_sync(d, tm))) break;
            if (tid == 0) fista_reset(d, &S);
            __syncthreads();
            const Range rk = block_range(tm, d.n_con);
            while (!S.f_done) {
              const int rot = S.rot_n;
              const double beta = S.f_beta;
              for (int c = rk.lo + tid; c < rk.hi; c += blockDim.x) normal_z_item(d, c, rot, beta);
              if (!(ok = grid_sync(d, tm))) break;
              double pc[3] = {0.0, 0.0, 0.0};
              for (int c = gwarp; c < d.n_con; c += nwarps) normal_row(d, c, rot, lane, pc);
              if (!(ok = grid_reduce<3>(d, tm, pc, sums))) break;
              if (tid == 0) fista_finish(d, &S, &S.rot_n, sums);
              __syncthreads();
            }
            if (!ok) break;
            const double* lam_n = con_lamn(d, S.rot_n + 1);
            if (tid == 0) fista_reset(d, &S);
            __syncthreads();
            while (!S.f_done) {
              const int rot = S.rot_f;
              const double beta = S.f_beta;
              for (int c = rk.lo + tid; c < rk.hi; c += blockDim.x) friction_z_item(d, c, rot, beta);
              if (!(ok = grid_sync(d, tm))) break;
              double pc[3] = {0.0, 0.0, 0.0};
              for (int c = gwarp; c < d.n_con; c += nwarps) friction_row(d, c, rot, lam_n, lane, pc);
              if (!(ok = grid_reduce<3>(d, tm, pc, sums))) break;
              if (tid == 0) fista_finish(d, &S, &S.rot_f, sums);
              __syncthreads();
            }
            if (!ok) break;
            const double* lam_f = con_lamf(d, S.rot_f + 1);
            for (int i = gwarp; i < d.n_f; i += nwarps) contact_y_row(d, i, lam_n, lam_f, lane);
            if (!(ok = grid_sync(d, tm))) break;
          }
          // S^T y row by row, with the Anderson work of that row's vertex fused in
          // the Anderson partials of lanes 0..2 accumulate in shared memory (in
          // registers they would stay live across the S^T loop)
          if (lane < 3)
            for (int j = 0; j < 2 * kMaxAA; ++j) pa[j] = 0.0;
          for (int j = twarp; j < d.n_f; j += nwarps) {
            double a0, a1, a2;
            spmv_st_sum(d, d.y, j, lane, a0, a1, a2);
            if (lane < 3) {
              const size_t o = 3 * (size_t)d.perm[j] + lane;
              const double qh = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
              d.qhat[o] = qh;
              aa_component(d, o, qh, av, pa);
            }
          }
        }
        work_done(PH_AA);
        __syncthreads();
        double pav = 0.0;   // the block's partial of value tid (fixed order)
        if (tid < 2 * kMaxAA)
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int l = 0; l < 3; ++l) pav += s_pa[w][l][tid];
        // every block adds the team's dots and runs the small Anderson solve
        // itself (identical sums, identical gamma): no second round trip for
        // a published result
        if (!(ok = grid_reduce_all_v<2 * kMaxAA>(d, tm, pav, sums))) break;
        mark(PH_SPMV_ST);   // S^T y + Anderson dots, through their reduction
        if (tid == 0) aa_finish(d, &S, av, sums);
        __syncthreads();
        mark(PH_AA);        // the small Anderson solve
        const int use_hat = S.use_hat, nc = S.ncols;
        pu[0] = pu[1] = 0.0;
        // one thread per free coordinate of the block's vertices
        for (int x = 3 * rv.lo + tid; x < 3 * rv.hi; x += blockDim.x)
          if (!d.pinned[x / 3]) update_comp(d, (size_t)x, use_hat, nc, S.gamma, pu);
        work_done(PH_UPDATE);
        if (!(ok = grid_sync(d, tm))) break;
        if (tid == 0) update_count(d, &S);
        __syncthreads();
        mark(PH_UPDATE);
        if (S.done) break;
      }
      if (!ok) break;
      const bool redo = warm_now && S.not_converged > nc0;
      __syncthreads();   // every thread has read S before thread 0 resets it
      if (!redo) break;
      if (tid == 0) {
        S.not_converged = nc0;
        S.fallbacks += 1;
        ctrl_step_reset(&S, t);
      }
      for (int v = rv.lo + tid; v < rv.hi; v += blockDim.x)
        for (int i = 0; i < 3; ++i) {
          const size_t o = 3 * (size_t)v + i;
          d.q[o] = d.qt[o];
          d.qhl[o] = df_split(d.qt[o]);
          d.qprev[o] = d.qt[o];
          d.gprev[o] = 0.0;
        }
      if (!(ok = grid_sync(d, tm))) break;
      warm_now = false;
    }
    if (!ok) break;
    if (d.n_con > 0 && d.con_ckpt) {
      // converged multipliers of this step (active sets of the adjoint)
      const Range rc = block_range(tm, d.n_con);
      const double* ln = con_lamn(d, S.rot_n + 1);
      const double* lf = con_lamf(d, S.rot_f + 1);
      double* ck = d.con_ckpt + (size_t)t * 3 * d.n_con;
      for (int c = rc.lo + tid; c < rc.hi; c += blockDim.x) {
        ck[c] = ln[c];
        ck[d.n_con + 2 * c] = lf[2 * c];
        ck[d.n_con + 2 * c + 1] = lf[2 * c + 1];
      }
    }
    const bool last = t == a.T - 1;
    double* qo = last && a.qT ? a.qT : a.sq;
    double* vo = last && a.vT ? a.vT : a.sv;
    if (tid == 0) step_end_ctrl(d, &S, writer);
    for (int v = rv.lo + tid; v < rv.hi; v += blockDim.x) step_end_item(d, v, qo, vo, a.ckpt + (size_t)(t + 1) * nv3);
    if (has_prox_hessian(d.model)) {
      double p4[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = rt.lo + tid; i < rt.hi; i += blockDim.x) tr_item(d, i, p4);
      if (!(ok = grid_reduce<4>(d, tm, p4, sums))) break;
      if (tid == 0) tr_finish(d, &S, sums, writer);
      __syncthreads();
    } else {
      if (!(ok = grid_sync(d, tm))) break;
    }
    mark(PH_END);
  }
  // block 0 publishes the rollout statistics
  if (writer && tid == 0) {
    Ctrl* c = d.ctrl;
    c->iters_total = S.iters_total;
    c->iters_max = S.iters_max;
    c->resets = S.resets;
    c->not_converged = S.not_converged;
    c->tau_half = S.tau_half;
    c->tau_one = S.tau_one;
    c->last_rho = S.last_rho;
    c->k = S.k;
    c->escalations = S.escalations;
    c->fallbacks = S.fallbacks;
    c->con_iters = S.con_iters;
    c->con_unconverged = S.con_unconverged;
    atomicOr(&c->status, S.status);
    for (int i = 0; i < 8; ++i) {
      c->phase_ns[i] += ph[i];
      c->work_ns[i] += wk[i];
    }
    c->elapsed_ns[0] = gtimer() - tmr[2];
  }
  if (d.prof && tid == 0)
    for (int i = 0; i < 8; ++i) {
      atomicMax(&d.ctrl->work_max_ns[i], wall[i]);
      if (writer) d.ctrl->last_ns[i] += lst[i];
    }
}

// team[blockIdx.x] = {instance, block index in its team, team size, 0}
template <typename T, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_fwd_rollout(const Dev* __restrict__ devs, const int4* __restrict__ team,
                                                             const InstOff* __restrict__ off, BatchFwd br) {
  __shared__ Dev sd;
  __shared__ RollArgs sa;
  const int4 tb = team[blockIdx.x];
  if (threadIdx.x == 0) {
    sd = devs[tb.x];
    const long long v3 = 3 * off[tb.x].v;
    RollArgs a;
    a.T = br.T;
    a.q0 = br.q0 + v3;
    a.v0 = br.v0 + v3;
    a.fext = br.fext ? br.fext + v3 : nullptr;
    a.f_stride = br.f_stride;
    a.qT = br.qT ? br.qT + v3 : nullptr;
    a.vT = br.vT ? br.vT + v3 : nullptr;
    a.ckpt = sd.ckpt;
    a.sq = sd.sq;
    a.sv = sd.sv;
    sa = a;
    team_red_count() = 0;
  }
  __syncthreads();
  fwd_rollout_body<T>(sd, sa, Team{tb.y, tb.z});
}

// ------------------------------------------------------------ launch

int coop_blocks_per_sm(const void* fn, int block, int* sms_out) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  // with the mode-T staging (the larger request), so that a grid fits either launch
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, kTStageBytes) != cudaSuccess) return 0;
  if (sms_out) *sms_out = sms;
  return per_sm < 2 ? per_sm : 2;
}

template <typename T>
static const void* fwd_fn(bool wide) {
  return wide ? (const void*)k_fwd_rollout<T, kFwdWideBlock, 1> : (const void*)k_fwd_rollout<T, kFwdNarrowBlock, 2>;
}

// blocks per SM of one forward shape that a cooperative launch can hold
static int fwd_per_sm(bool fp32, bool wide, int* sms) {
  const int per = coop_blocks_per_sm(fp32 ? fwd_fn<float>(wide) : fwd_fn<double>(wide), wide ? kFwdWideBlock : kFwdNarrowBlock, sms);
  return wide ? (per < 1 ? per : 1) : per;
}

// blocks_per_sm 2: the narrow shape at two blocks per SM; otherwise the
// wide shape at one
int persistent_grid(bool fp32, int blocks_per_sm) {
  int sms = 0;
  const bool wide = blocks_per_sm != 2;
  const int per = fwd_per_sm(fp32, wide, &sms);
  if (per < 1) return 0;
  return sms * (wide ? 1 : per);
}

int persistent_grid_max(bool fp32) {
  const int a = persistent_grid(fp32, 1), b = persistent_grid(fp32, 2);
  return a > b ? a : b;
}

// a grid of at most one block per SM takes the wide shape
cudaError_t launch_fwd_rollout(bool fp32, const Dev* devs, const int4* team, const InstOff* off, const BatchFwd& br,
                               int grid, bool tstage, cudaStream_t s) {
  const size_t sm = tstage ? kTStageBytes : 0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (grid <= sms) {
    if (fp32) return coop_launch(k_fwd_rollout<float, kFwdWideBlock, 1>, grid, kFwdWideBlock, sm, s, devs, team, off, br);
    return coop_launch(k_fwd_rollout<double, kFwdWideBlock, 1>, grid, kFwdWideBlock, sm, s, devs, team, off, br);
  }
  if (fp32) return coop_launch(k_fwd_rollout<float, kFwdNarrowBlock, 2>, grid, kFwdNarrowBlock, sm, s, devs, team, off, br);
  return coop_launch(k_fwd_rollout<double, kFwdNarrowBlock, 2>, grid, kFwdNarrowBlock, sm, s, devs, team, off, br);
}

}  // namespace pdk
