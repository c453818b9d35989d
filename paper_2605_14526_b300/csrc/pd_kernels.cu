// Per-phase CUDA kernels of the forward pass (Alg. 1) and the standalone
// solve. Each kernel runs one phase of pd_phases.cuh over its items; the
// block that completes a reduction (a "last block" ticket, no spin-waits)
// finishes the sum in a fixed order and runs the scalar logic. The
// persistent rollout kernel (pd_persistent.cu) runs the same phases in one
// launch; this path serves meshes too large for one cooperative grid.
//
// Data layout: vertex vectors are [n_v][3] float64; pinned vertices keep
// q = X and carry zeros in every difference/residual vector so that norms and
// dot products run over free DoFs only. The RHS scatter is deterministic:
// elements write their 12 corner contributions, a per-vertex gather sums them
// in FP64 together with the constant part b0.
#include <cuda_runtime.h>

#include <cstdint>

#include "pd_launch.h"
#include "pd_phases.cuh"
#include "pd_tsolve.cuh"

namespace pdk {

__global__ void k_step_begin(Dev d, const double* qt_in, const double* vt_in, const double* fext, int t,
                             double* ckpt_t) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) ctrl_step_reset(d.ctrl, t);
  if (v < d.n_v) step_begin_item(d, v, qt_in, vt_in, fext, ckpt_t);
}

template <typename T>
__global__ void __launch_bounds__(kTetBlock) k_local(Dev d, const double* x) {
  if (d.ctrl->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_e) local_item<T>(d, e, x, d.qhl);   // x is the iterate q, d.qhl its float pairs
}

// standalone local step (pd_local_rhs): the positions as float pairs first
// (FP32 step), then every element, no iteration control
__global__ void __launch_bounds__(kVtxBlock) k_split_hl(Dev d, const double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * d.n_v) d.qhl[i] = df_split(x[i]);
}

template <typename T>
__global__ void __launch_bounds__(kTetBlock) k_local_all(Dev d, const double* x) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_e) local_item<T>(d, e, x, sizeof(T) == 4 ? d.qhl : nullptr);
}

// the projection part of the right-hand side per vertex, sum_e w_e V_e G_e^T
// vec(p_e), from the elements' corner forces: one thread per vertex adds its
// incident corners in the order of the incidence list (FP64), four loads in
// flight; pinned rows get 0
template <typename T>
__global__ void __launch_bounds__(kVtxBlock) k_rhs_out(Dev d, double* out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_v) return;
  double* o = out + 3 * (size_t)v;
  if (d.pinned[v]) {
    o[0] = o[1] = o[2] = 0.0;
    return;
  }
  const T* cb = reinterpret_cast<const T*>(d.contrib);
  int p = d.inc_ptr[v];
  const int end = d.inc_ptr[v + 1];
  if constexpr (sizeof(T) == 4) {
    // FP32 corner forces summed in double-float on the FP32 pipe
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
    for (; p < end; ++p) {
      const float* f = cb + 3 * (size_t)d.inc_idx[p];
      a0 = df_add_f(a0, f[0]);
      a1 = df_add_f(a1, f[1]);
      a2 = df_add_f(a2, f[2]);
    }
    o[0] = df_join(a0);
    o[1] = df_join(a1);
    o[2] = df_join(a2);
    return;
  }
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  for (; p + 3 < end; p += 4) {
    int ic[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ic[i] = d.inc_idx[p + i];
    T f[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) f[i][j] = cb[3 * (size_t)ic[i] + j];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c0 += (double)f[i][0];
      c1 += (double)f[i][1];
      c2 += (double)f[i][2];
    }
  }
  for (; p < end; ++p) {
    const T* f = cb + 3 * (size_t)d.inc_idx[p];
    c0 += (double)f[0];
    c1 += (double)f[1];
    c2 += (double)f[2];
  }
  o[0] = c0;
  o[1] = c1;
  o[2] = c2;
}

template <typename T>
__global__ void __launch_bounds__(kVtxBlock) k_assemble(Dev d) {
  if (d.ctrl->done) return;
  const int k = d.ctrl->k;
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // warp per vertex
  double part[3] = {0.0, 0.0, 0.0};
  if (v < d.n_v) assemble_warp<T>(d, v, k, part, threadIdx.x & 31);
  block_reduce_store<3>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_ASSEMBLE]) && threadIdx.x == 0) {
    double s[3];
    for (int j = 0; j < 3; ++j) s[j] = sum_partials(d.red, gridDim.x, j);
    assemble_finish(d, d.ctrl, k, s);
  }
}

__global__ void __launch_bounds__(32 * kWarpsSpmv) k_spmv_s(Dev d, const float2* xin, float2* y, float2* part, int* cnt,
                                                             int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int sg = warp; sg < d.n_seg; sg += nwarps) spmv_s_segment(d, xin, y, part, cnt, sg, lane);
}

__global__ void __launch_bounds__(32 * kWarpsSpmv) k_spmv_st(Dev d, const float2* y, double* out, int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < d.n_f; j += nwarps) spmv_st_row(d, y, out, j, lane);
}

// solve mode T, one height of a sweep per launch (the kernel boundary is the
// barrier between heights); the backward writes its finished rows to out in
// vertex order
struct TFinOut {
  const int* perm;
  double* out;
  __device__ __forceinline__ void operator()(int j, double a0, double a1, double a2) const {
    const int lane = threadIdx.x & 31;
    if (lane < 3) out[3 * (size_t)perm[j] + lane] = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
  }
  __device__ __forceinline__ void lanes(bool on, int j, double a0, double a1, double a2) const {
    if (!on) return;
    double* o = out + 3 * (size_t)perm[j];
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
  }
};

__global__ void __launch_bounds__(kTBlock) k_tsweep_fwd(Dev d, const double* b, double* y, int h, int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  tsweep_fwd(d, b, y, h, blockIdx.x, gridDim.x, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5);
}

__global__ void __launch_bounds__(kTBlock) k_tsweep_bwd(Dev d, const double* y, double* out, int h, int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  TFinOut fin{d.perm, out};
  tsweep_bwd(d, y, h, blockIdx.x, gridDim.x, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5, fin);
}

__global__ void __launch_bounds__(kVtxBlock) k_aa(Dev d) {
  if (d.ctrl->done) return;
  const AAView a = aa_view(d, d.ctrl->pairs, d.ctrl->ncols, d.ctrl->head);
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[2 * kMaxAA] = {};
  if (v < d.n_v) aa_item(d, v, a, part);
  block_reduce_store<2 * kMaxAA>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_SPMV_T]) && threadIdx.x == 0) {
    double s[2 * kMaxAA];
    for (int j = 0; j < 2 * kMaxAA; ++j) s[j] = sum_partials(d.red, gridDim.x, j);
    aa_finish(d, d.ctrl, a, s);
  }
}

__global__ void __launch_bounds__(kVtxBlock) k_update(Dev d) {
  if (d.ctrl->done) return;
  const int use_hat = d.ctrl->use_hat;
  const int nc = d.ctrl->ncols;
  double gam[kMaxAA];
  for (int j = 0; j < nc; ++j) gam[j] = d.ctrl->gamma[j];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[2] = {0.0, 0.0};
  if (v < d.n_v) update_item(d, v, use_hat, nc, gam, part);
  block_reduce_store<2>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_UPDATE]) && threadIdx.x == 0) {
    double s[2] = {sum_partials(d.red, gridDim.x, 0), sum_partials(d.red, gridDim.x, 1)};
    update_finish(d, d.ctrl, s);
  }
}

__global__ void k_step_end(Dev d, double* qn, double* vn, double* ckpt_next) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) step_end_ctrl(d, d.ctrl, true);
  if (v < d.n_v) step_end_item(d, v, qn, vn, ckpt_next);
}

__global__ void __launch_bounds__(kVtxBlock) k_tr(Dev d) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  tr_item(d, tid, part);
  block_reduce_store<4>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_TR]) && threadIdx.x == 0) {
    double s[4];
    for (int j = 0; j < 4; ++j) s[j] = sum_partials(d.red, gridDim.x, j);
    tr_finish(d, d.ctrl, s, true);
  }
}

// ------------------------------------------------------------ standalone solve

// b (vertex order) -> elimination order in xperm (the products' input
// representation); the pinned rows of x are set to 0. The S b accumulator is
// not touched here: the first product overwrites every row of it.
__global__ void k_solve_in(Dev d, const double* b, float2* xperm, double* x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_v) return;
  if (d.pinned[v]) {
    for (int i = 0; i < 3; ++i) x[3 * (size_t)v + i] = 0.0;
    return;
  }
  const int pos = d.iperm[v];
  for (int i = 0; i < 3; ++i) store_rhs(d, xperm, 3 * (size_t)pos + i, b[3 * (size_t)v + i]);
}

// ------------------------------------------------------------ launch wrappers

static inline int nblk(int n, int b) { return (n + b - 1) / b; }

void launch_step_begin(const Dev& d, cudaStream_t s, const double* qt, const double* vt, const double* fext, int t,
                       double* ckpt_t) {
  k_step_begin<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, qt, vt, fext, t, ckpt_t);
}

int spmv_blocks(const Dev& d) {
  int b = nblk(d.n_seg, kWarpsSpmv);
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}
int spmvt_blocks(const Dev& d) {
  int b = nblk(d.n_f, kWarpsSpmv);
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

int tsweep_blocks(const Dev& d) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 2 * sms;
}

void launch_apply_inverse(const Dev& d, cudaStream_t s, const float2* xperm, float2* y, float2* part, int* cnt,
                          double* out, int check) {
  if (d.tmode) {
    const int g = tsweep_blocks(d);
    const double* b = reinterpret_cast<const double*>(xperm);
    double* yy = reinterpret_cast<double*>(y);
    for (int h = 0; h < d.t_nlev; ++h) k_tsweep_fwd<<<g, kTBlock, kTStageBytes, s>>>(d, b, yy, h, check);
    for (int h = d.t_nlev - 1; h >= 0; --h) k_tsweep_bwd<<<g, kTBlock, kTStageBytes, s>>>(d, yy, out, h, check);
    return;
  }
  k_spmv_s<<<spmv_blocks(d), 32 * kWarpsSpmv, 0, s>>>(d, xperm, y, part, cnt, check);
  k_spmv_st<<<spmvt_blocks(d), 32 * kWarpsSpmv, 0, s>>>(d, y, out, check);
}

void launch_local_rhs(const Dev& d, cudaStream_t s, const double* x, double* out) {
  if (d.local_fp32) {
    k_split_hl<<<nblk(3 * d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, x);
    k_local_all<float><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, x);
    k_rhs_out<float><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, out);
  } else {
    k_local_all<double><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, x);
    k_rhs_out<double><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, out);
  }
}

void launch_solve(const Dev& d, cudaStream_t s, const double* b, float2* xperm, float2* y, float2* part, int* cnt,
                  double* x) {
  k_solve_in<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, b, xperm, x);
  launch_apply_inverse(d, s, xperm, y, part, cnt, x, 0);
}

void launch_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  if (d.local_fp32) {
    k_local<float><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.q);
    k_assemble<float><<<nblk(32 * d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  } else {
    k_local<double><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.q);
    k_assemble<double><<<nblk(32 * d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  }
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  launch_apply_inverse(d, s, d.bperm, d.y, d.s_part, d.s_cnt, d.qhat, 1);
  if (ev) cudaEventRecord(ev[3], s);
  k_aa<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  k_update<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
}

void launch_step_end(const Dev& d, cudaStream_t s, double* qn, double* vn, double* ckpt_next, double* tau) {
  (void)tau;
  k_step_end<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, qn, vn, ckpt_next);
  if (has_prox_hessian(d.model)) k_tr<<<nblk(d.n_e + d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
}

int max_reduction_blocks(int n_v, int n_e) {
  int a = nblk(32 * n_v, kVtxBlock), b = nblk(n_e + n_v, kVtxBlock), c = nblk(n_e, kTetBlock);
  int m = a > b ? a : b;
  return m > c ? m : c;
}

}  // namespace pdk
