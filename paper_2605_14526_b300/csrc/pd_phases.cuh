// Per-item bodies of the forward phases (Alg. 1) and the scalar logic run by
// the block that completes each reduction. Shared by the per-phase kernels
// (pd_kernels.cu) and the persistent rollout kernel (pd_persistent.cu), so the
// two launch paths execute identical arithmetic. Pointers here are plain (no
// __restrict__ / read-only cache): inside the persistent kernel the same
// arrays are rewritten by other blocks between grid barriers.
#pragma once
#include "pd_common.cuh"
#include "pd_df.cuh"
#include "pd_aa_solve.cuh"
#include "pd_local.cuh"

namespace pdk {

// right-hand side entry in elimination order, in the representation the
// products read (double-float pair, or FP64 with sfp64)
__device__ __forceinline__ void store_rhs(const Dev& d, float2* xperm, size_t i, double v) {
  if (d.sfp64) reinterpret_cast<double*>(xperm)[i] = v;
  else xperm[i] = df_split(v);
}
__device__ __forceinline__ double load_y(const Dev& d, const float2* y, size_t i) {
  return d.sfp64 ? reinterpret_cast<const double*>(y)[i] : df_join(y[i]);
}
__device__ __forceinline__ void store_y(const Dev& d, float2* y, size_t i, double v) {
  if (d.sfp64) reinterpret_cast<double*>(y)[i] = v;
  else y[i] = df_split(v);
}


// ------------------------------------------------------------ step begin

// The scalar logic below is written against a state type St with the fields
// of Ctrl used here: the global control word (per-phase kernels) or the
// per-block shared replica FwdState (persistent rollout).
struct FwdState {
  int k, done, converged, pairs, ncols, head, use_hat, t, n_local, n_solve;
  int hi, since, escalations, fallbacks;
  double gmin;
  // contact inner solves (FISTA): momentum and restart of the running solve,
  // buffer rotation of the normal and the friction multipliers
  double f_t, f_beta, f_tol;
  int f_it, f_done, rot_n, rot_f, con_iters, con_unconverged;
  int iters_total, iters_max, resets, not_converged, tau_half, tau_one, status;
  double gram[kMaxAA * kMaxAA];
  double gamma[kMaxAA];
  double dq_norm2, qprev_norm2, db_norm2, bprev_norm2, last_rho;
};

template <class St>
__device__ __forceinline__ void ctrl_step_reset(St* c, int t) {
  c->k = 0; c->done = 0; c->converged = 0; c->pairs = 0; c->ncols = 0; c->head = 0; c->use_hat = 1;
  c->t = t;
  c->n_local = 0;
  c->n_solve = 0;
  c->since = 0;
  c->gmin = 1e300;
}

// q_t (pinned at X), inertial target (eq. freefall) and the constant RHS
//   b0 = M/h^2 q~ + (alpha M + B)/h q_t - A_fp X_p       (free rows)
__device__ __forceinline__ void step_begin_item(const Dev& d, int v, const double* qt_in, const double* vt_in,
                                                const double* fext, double* ckpt_t) {
  const bool pin = d.pinned[v];
  double q[3], b0[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i) q[i] = pin ? d.X[3 * v + i] : qt_in[3 * v + i];
  if (!pin) {
    const double m = d.mass[v], h = d.h;
    double bq[3] = {0.0, 0.0, 0.0};
    for (int p = d.B_ptr[v]; p < d.B_ptr[v + 1]; ++p) {
      const int u = d.B_idx[p];
      const double w = d.B_val[p];
      const bool pu = d.pinned[u];
      for (int i = 0; i < 3; ++i) bq[i] += w * (pu ? d.X[3 * u + i] : qt_in[3 * u + i]);
    }
    for (int i = 0; i < 3; ++i) {
      const double f = fext ? fext[3 * v + i] : 0.0;
      const double qtil = q[i] + h * vt_in[3 * v + i] + h * h * (d.g[i] + f / m);
      d.qtil[3 * v + i] = qtil;
      b0[i] = m / (h * h) * qtil + (d.alpha_d * m * q[i] + bq[i]) / h - d.cA[3 * v + i];
    }
  } else {
    for (int i = 0; i < 3; ++i) d.qtil[3 * v + i] = q[i] + d.h * d.h * d.g[i];
  }
  for (int i = 0; i < 3; ++i) {
    d.qt[3 * v + i] = q[i];
    d.q[3 * v + i] = q[i];
    d.qhl[3 * v + i] = df_split(q[i]);
    d.qprev[3 * v + i] = q[i];
    d.gprev[3 * v + i] = 0.0;
    d.b0[3 * v + i] = b0[i];
    if (ckpt_t) ckpt_t[3 * v + i] = q[i];
  }
}

// q^{k+1} of one coordinate of a free vertex: q_hat - sum_j gamma_j (dQ_j +
// dG_j), or q_hat when the guard rejected gamma; the history keeps the sums
// dQ_j + dG_j (dQG), the only form in which the update uses dQ
__device__ __forceinline__ double next_iterate(const Dev& d, size_t o, int use_hat, int nc, const double* gam) {
  double qn = d.qhat[o];
  if (!use_hat) {
    const size_t nv3 = 3 * (size_t)d.n_v;
#pragma unroll
    for (int j = 0; j < kMaxAA; ++j)
      if (j < nc) qn = __fma_rn(-gam[j], d.dQG[j * nv3 + o], qn);
  }
  return qn;
}

// b^k = b0 + sum of corner contributions (FP64) in vertex order and in
// elimination order (double-float); partials ||b^k - b^{k-1}||^2,
// ||b^{k-1}||^2, non-finite. One warp per vertex: lanes take the incident
// corners, a fixed shuffle tree adds them, and the lane holding component i
// finishes it.
template <typename T>
__device__ __forceinline__ void assemble_warp(const Dev& d, int v, int k, double* part, int lane) {
  if (d.pinned[v]) return;
  const T* cb = reinterpret_cast<const T*>(d.contrib);
  const int beg = d.inc_ptr[v], end = d.inc_ptr[v + 1];
  int i;
  double sum;
  if constexpr (sizeof(T) == 4) {
    // FP32 corner forces summed in double-float on the FP32 pipe (TwoSum:
    // error about 2^-44 of the sum of magnitudes, below the forces' own
    // FP32 rounding), one conversion to FP64 per component
    float2 c[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int p = beg + lane; p < end; p += 32) {
      const int ic = d.inc_idx[p];
#pragma unroll
      for (int j = 0; j < 3; ++j) c[j] = df_add_f(c[j], cb[3 * (size_t)ic + j]);
    }
    i = lane >> 3;
    float2 s3[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) s3[j] = df_warp_sum(c[j]);
    sum = i == 0 ? df_join(s3[0]) : (i == 1 ? df_join(s3[1]) : df_join(s3[2]));
  } else {
    double c[3] = {0.0, 0.0, 0.0};
    for (int p = beg + lane; p < end; p += 32) {
      const int ic = d.inc_idx[p];
#pragma unroll
      for (int j = 0; j < 3; ++j) c[j] += (double)cb[3 * (size_t)ic + j];
    }
    sum = warp_sum_scatter<3>(c, lane, i);   // component i in lanes 8i .. 8i+7
  }
  if ((lane & 7) != 0 || i >= 3) return;
  const size_t o = 3 * (size_t)v + i;
  const double acc = d.b0[o] + sum;
  const double bp = d.bprev[o];
  if (k > 0) {
    part[0] += (acc - bp) * (acc - bp);
    part[1] += bp * bp;
  }
  d.b[o] = acc;
  store_rhs(d, d.bperm, 3 * (size_t)d.iperm[v] + i, acc);
  if (!isfinite(acc)) part[2] += 1.0;
}

__device__ __forceinline__ double gate_rhs(double eps, double b2, double abs_tol) {
  return eps * eps * b2 + 2.0 * eps * abs_tol * (double)sqrtf((float)b2) + abs_tol * abs_tol;
}

// dual gate (eq. convergence_dual), iteration cap, non-finite stop.
// Precision escalation: with an FP32 local step the gate distance (the larger
// of the two squared gate ratios) must halve at least every d.escalate
// iterations; when it does not, the rounding of the FP32 projections has
// become the floor of the iteration and the local step switches to FP64 for
// the rest of the rollout.
template <class St>
__device__ __forceinline__ void assemble_finish(const Dev& d, St* c, int k, const double* s, bool carried = false) {
  c->n_local += 1;
  if (s[2] > 0.0) c->status |= 1;
  c->db_norm2 = s[0];
  c->bprev_norm2 = s[1];
  if (carried && k >= 1) {  // the previous update's step norms travel with this reduction
    c->dq_norm2 = s[3];
    c->qprev_norm2 = s[4];
  }
  if (d.fixed_iters <= 0 && k >= 2) {
    // ||a|| <= eps ||b|| + abs  <=>  a^2 <= eps^2 b^2 + 2 eps abs ||b|| + abs^2; the
    // cross term is negligible next to the others and is formed with an FP32 root
    const double rs = gate_rhs(d.eps_step, c->qprev_norm2, d.eps_abs);
    const double rr = gate_rhs(d.eps_res, s[1], d.eps_abs);
    const bool step_ok = c->dq_norm2 <= rs;
    const bool res_ok = s[0] <= rr;
    if (step_ok && res_ok) {
      c->converged = 1;
      c->done = 1;
    } else if (d.escalate > 0 && d.local_fp32 && !c->hi) {
      const double gd = fmax(c->dq_norm2 / fmax(rs, 1e-300), s[0] / fmax(rr, 1e-300));
      if (gd < 0.5 * c->gmin) {
        c->gmin = gd;
        c->since = 0;
      } else if (++c->since >= d.escalate) {
        c->hi = 1;
        c->escalations += 1;
      }
    }
  }
  if (!c->done && k >= d.k_max) {
    c->done = 1;
    c->not_converged += 1;
  }
  if (c->status & 1) c->done = 1;
}

// ------------------------------------------------------------ solve A^-1 = S^T S
//
// Both products run in double-float arithmetic (pd_df.cuh): S is stored as
// float pairs, the right-hand side b in elimination order (bperm) and the
// intermediate y = S b as float pairs, and the result S^T y is returned in
// FP64.

// FP64 forms of the two products (options.solve_fp64): the same traversal,
// FP64 multiply-adds, the same slot-ordered combination of split rows
__device__ __forceinline__ void spmv_s_segment64(const Dev& d, const double* xin, double* y, double* part, int* cnt,
                                                 int sg, int lane) {
  const int4 seg = d.s_seg[sg];
  const int row = seg.x;
  const double* sv = d.s_val64 + d.s_rowptr[row] + seg.y;
  const double* xv = xin + 3 * (size_t)(d.s_first[row] + seg.y);
  double a[4][3] = {};
  int p = lane;
  for (; p + 96 < seg.z; p += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double s = sv[p + 32 * u];
      const double* x = xv + 3 * (size_t)(p + 32 * u);
      a[u][0] += s * x[0];
      a[u][1] += s * x[1];
      a[u][2] += s * x[2];
    }
  }
  for (; p < seg.z; p += 32) {
    const double s = sv[p];
    const double* x = xv + 3 * (size_t)p;
    a[0][0] += s * x[0];
    a[0][1] += s * x[1];
    a[0][2] += s * x[2];
  }
  double r[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double v = (a[0][i] + a[1][i]) + (a[2][i] + a[3][i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    r[i] = v;
  }
  double* yr = y + 3 * (size_t)row;
  if (seg.w == 0) {
    if (lane < 3) yr[lane] = r[lane == 0 ? 0 : (lane == 1 ? 1 : 2)];
    return;
  }
  const int slot0 = seg.w - 1;
  const int ns = (row - d.s_first[row] + kSegLen) / kSegLen;
  double* pr = part + 3 * (size_t)slot0;
  int last = 0;
  if (lane == 0) {
    double* ps = pr + 3 * (size_t)(seg.y / kSegLen);
    ps[0] = r[0];
    ps[1] = r[1];
    ps[2] = r[2];
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(cnt + slot0) : "memory");
    last = old == ns - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __syncwarp();
  double t[3] = {0.0, 0.0, 0.0};
  for (int k = lane; k < ns; k += 32)
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] += __ldcg(pr + 3 * (size_t)k + i);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], o);
  if (lane < 3) yr[lane] = t[lane == 0 ? 0 : (lane == 1 ? 1 : 2)];
  if (lane == 0) cnt[slot0] = 0;
}

__device__ __forceinline__ void spmv_st_sum64(const Dev& d, const double* y, int j, int lane, double& r0, double& r1,
                                              double& r2) {
  const int64_t beg = d.st_ptr[j], end = d.st_ptr[j + 1];
  double a[4][3] = {};
  int64_t p = beg + lane;
  for (; p + 96 < end; p += 128) {
    int ix[4];
    double sv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ix[u] = d.st_idx[p + 32 * u];
      sv[u] = d.st_val64[p + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double* yv = y + 3 * (size_t)ix[u];
      a[u][0] += sv[u] * yv[0];
      a[u][1] += sv[u] * yv[1];
      a[u][2] += sv[u] * yv[2];
    }
  }
  for (; p < end; p += 32) {
    const double s = d.st_val64[p];
    const double* yv = y + 3 * (size_t)d.st_idx[p];
    a[0][0] += s * yv[0];
    a[0][1] += s * yv[1];
    a[0][2] += s * yv[2];
  }
  r0 = (a[0][0] + a[1][0]) + (a[2][0] + a[3][0]);
  r1 = (a[0][1] + a[1][1]) + (a[2][1] + a[3][1]);
  r2 = (a[0][2] + a[1][2]) + (a[2][2] + a[3][2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
}

// one segment of a skyline row of S: S[row, seg] x[seg] (3 RHS); four
// independent accumulator sets per lane keep several loads in flight. A row
// of one segment is written directly; the segments of a split row write
// their partial sums to consecutive slots and the last one to finish adds
// the slots in slot order, so the result does not depend on the schedule.
__device__ __forceinline__ void spmv_s_segment(const Dev& d, const float2* xin, float2* y, float2* part, int* cnt,
                                               int sg, int lane) {
  if (d.sfp64) {
    spmv_s_segment64(d, reinterpret_cast<const double*>(xin), reinterpret_cast<double*>(y),
                     reinterpret_cast<double*>(part), cnt, sg, lane);
    return;
  }
  const int4 seg = d.s_seg[sg];  // x = row, y = offset in row, z = length, w = 0 or 1 + first slot of a split row
  const int row = seg.x;
  const float2* sv = d.s_hl + d.s_rowptr[row] + seg.y;
  const float2* xv = xin + 3 * (size_t)(d.s_first[row] + seg.y);
  float ah[4][3], al[4][3];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int i = 0; i < 3; ++i) ah[u][i] = al[u][i] = 0.0f;
  int p = lane;
  for (; p + 96 < seg.z; p += 128) {
    float2 sa[4], xa[4][3];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sa[u] = sv[p + 32 * u];
      const float2* x = xv + 3 * (size_t)(p + 32 * u);
      xa[u][0] = x[0];
      xa[u][1] = x[1];
      xa[u][2] = x[2];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 3; ++i) df_mac(ah[u][i], al[u][i], sa[u], xa[u][i]);
  }
  for (; p < seg.z; p += 32) {
    const float2 sa = sv[p];
    const float2* x = xv + 3 * (size_t)p;
#pragma unroll
    for (int i = 0; i < 3; ++i) df_mac(ah[0][i], al[0][i], sa, x[i]);
  }
  float2 r[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    r[i] = df_warp_sum(df_add(df_add(make_float2(ah[0][i], al[0][i]), make_float2(ah[1][i], al[1][i])),
                              df_add(make_float2(ah[2][i], al[2][i]), make_float2(ah[3][i], al[3][i]))));
  float2* yr = y + 3 * (size_t)row;
  if (seg.w == 0) {
    if (lane < 3) yr[lane] = r[lane == 0 ? 0 : (lane == 1 ? 1 : 2)];
    return;
  }
  const int slot0 = seg.w - 1;
  const int ns = (row - d.s_first[row] + kSegLen) / kSegLen;   // segments of the row
  float2* pr = part + 3 * (size_t)slot0;
  int last = 0;
  if (lane == 0) {
    float2* ps = pr + 3 * (size_t)(seg.y / kSegLen);
    ps[0] = r[0];
    ps[1] = r[1];
    ps[2] = r[2];
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(cnt + slot0) : "memory");
    last = old == ns - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __syncwarp();   // lane 0's acquire orders the other lanes' loads after every segment's release
  float2 t[3] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
  for (int k = lane; k < ns; k += 32)
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = df_add(t[i], __ldcg(pr + 3 * (size_t)k + i));
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = df_warp_sum(t[i]);
  if (lane < 3) yr[lane] = t[lane == 0 ? 0 : (lane == 1 ? 1 : 2)];
  if (lane == 0) cnt[slot0] = 0;   // next use is ordered after a barrier or a kernel boundary
}

// row j of S^T: sum over the ancestors i of j of S_ij y_i, returned in FP64
// to every lane; the indices of four entries are loaded before their y values
__device__ __forceinline__ void spmv_st_sum(const Dev& d, const float2* y, int j, int lane, double& r0, double& r1,
                                            double& r2) {
  if (d.sfp64) {
    spmv_st_sum64(d, reinterpret_cast<const double*>(y), j, lane, r0, r1, r2);
    return;
  }
  const int64_t beg = d.st_ptr[j], end = d.st_ptr[j + 1];
  float ah[4][3], al[4][3];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int i = 0; i < 3; ++i) ah[u][i] = al[u][i] = 0.0f;
  int64_t p = beg + lane;
  for (; p + 96 < end; p += 128) {
    int ix[4];
    float2 sa[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ix[u] = d.st_idx[p + 32 * u];
      sa[u] = d.st_hl[p + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2* yv = y + 3 * (size_t)ix[u];
      const float2 y0 = yv[0], y1 = yv[1], y2 = yv[2];
      df_mac(ah[u][0], al[u][0], sa[u], y0);
      df_mac(ah[u][1], al[u][1], sa[u], y1);
      df_mac(ah[u][2], al[u][2], sa[u], y2);
    }
  }
  for (; p < end; p += 32) {
    const float2 sa = d.st_hl[p];
    const float2* yv = y + 3 * (size_t)d.st_idx[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) df_mac(ah[0][i], al[0][i], sa, yv[i]);
  }
  float2 r[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    r[i] = df_warp_sum(df_add(df_add(make_float2(ah[0][i], al[0][i]), make_float2(ah[1][i], al[1][i])),
                              df_add(make_float2(ah[2][i], al[2][i]), make_float2(ah[3][i], al[3][i]))));
  r0 = df_join(r[0]);
  r1 = df_join(r[1]);
  r2 = df_join(r[2]);
}

// row j of S^T written to out[perm[j]]
__device__ __forceinline__ void spmv_st_row(const Dev& d, const float2* y, double* out, int j, int lane) {
  double a0, a1, a2;
  spmv_st_sum(d, y, j, lane, a0, a1, a2);
  if (lane == 0) {
    const int v = d.perm[j];
    out[3 * v] = a0;
    out[3 * v + 1] = a1;
    out[3 * v + 2] = a2;
  }
}

// ------------------------------------------------------------ Anderson

struct AAView {
  int m, add, slot, ncols_new;
};

__device__ __forceinline__ AAView aa_view(const Dev& d, int pairs, int ncols, int head) {
  AAView a;
  a.m = d.aa_m;
  a.add = a.m > 0 && pairs >= 1;
  a.slot = head;
  a.ncols_new = a.add ? (ncols < a.m ? ncols + 1 : a.m) : ncols;
  return a;
}

// g = q_hat - q for one component o = 3v + i; with a previous pair held, the
// new difference column (q - qprev, g - gprev) goes to ring slot `slot`;
// partial dots dG_new . dG_j and dG_j . g (eq. aa_gamma)
__device__ __forceinline__ void aa_component(const Dev& d, size_t o, double qh, const AAView& a, double* part) {
  const size_t nv3 = 3 * (size_t)d.n_v;
  const double q = d.q[o];
  const double g = qh - q;
  double dg_new = 0.0;
  if (a.add) {
    dg_new = g - d.gprev[o];
    d.dG[a.slot * nv3 + o] = dg_new;
    d.dQG[a.slot * nv3 + o] = __dadd_rn(q - d.qprev[o], dg_new);
  }
  d.gprev[o] = g;
#pragma unroll
  for (int j = 0; j < kMaxAA; ++j) {   // compile-time j: the partials stay in registers
    if (j < a.ncols_new) {
      const double dgj = (a.add && j == a.slot) ? dg_new : d.dG[j * nv3 + o];
      if (a.add) part[j] += dg_new * dgj;
      part[kMaxAA + j] += dgj * g;
    }
  }
}

__device__ __forceinline__ void aa_item(const Dev& d, int v, const AAView& a, double* part) {
  if (d.pinned[v]) return;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    aa_component(d, o, d.qhat[o], a, part);
  }
}

// history bookkeeping of one Anderson step: Gram row from the reduced dots,
// window pointers; returns the columns held (0: no mixing this iteration)
template <class St>
__device__ __forceinline__ int aa_book(St* c, const AAView& a, const double* s) {
  c->n_solve += 1;
  const int m = a.m;
  c->use_hat = 1;
  if (m == 0) return 0;
  if (a.add) {
    for (int j = 0; j < a.ncols_new; ++j) {
      c->gram[a.slot * kMaxAA + j] = s[j];
      c->gram[j * kMaxAA + a.slot] = s[j];
    }
    c->ncols = a.ncols_new;
    c->head = (a.slot + 1) % m;
  }
  c->pairs = c->pairs < m + 1 ? c->pairs + 1 : m + 1;
  return c->ncols;
}

// reliability guard outcome: accept gamma, or take q_hat and clear the history
template <class St>
__device__ __forceinline__ void aa_guard(St* c, bool accept) {
  if (!accept) {
    c->resets += 1;
    c->pairs = 0;
    c->ncols = 0;
    c->head = 0;
    for (int i = 0; i < kMaxAA * kMaxAA; ++i) c->gram[i] = 0.0;
  } else {
    c->use_hat = 0;
  }
}

// Gram update, regularised normal equations, reliability guard
// ||gamma||_2 <= 10 (eq. aa_gamma); returns the guard's verdict (1 accept,
// 0 reject, -1 no solve this iteration)
template <class St>
__device__ __forceinline__ int aa_finish(const Dev& d, St* c, const AAView& a, const double* s) {
  const int nc = aa_book(c, a, s);
  if (nc < 1) return -1;
  double* gam = c->gamma;   // read only when the guard accepts it
  double gn = 0.0;
  bool ok;
  switch (nc) {
    case 1: ok = aa_solve<1>(c->gram, s + kMaxAA, gam, gn); break;
    case 2: ok = aa_solve<2>(c->gram, s + kMaxAA, gam, gn); break;
    case 3: ok = aa_solve<3>(c->gram, s + kMaxAA, gam, gn); break;
    case 4: ok = aa_solve<4>(c->gram, s + kMaxAA, gam, gn); break;
    case 5: ok = aa_solve<5>(c->gram, s + kMaxAA, gam, gn); break;
    default: ok = aa_solve_any(nc, c->gram, s + kMaxAA, gam, gn); break;
  }
  const bool accept = ok && gn <= 100.0;
  aa_guard(c, accept);
  return accept ? 1 : 0;
}

// q^{k+1} = q_hat - (dQ + dG) gamma (or q_hat); step-norm partials
__device__ __forceinline__ void update_comp(const Dev& d, size_t o, int use_hat, int nc, const double* gam,
                                            double* part) {
  const double qn = next_iterate(d, o, use_hat, nc, gam);
  const double qo = d.q[o];
  part[0] += (qn - qo) * (qn - qo);
  part[1] += qo * qo;
  d.qprev[o] = qo;
  d.q[o] = qn;
  d.qhl[o] = df_split(qn);
  d.bprev[o] = d.b[o];
}

__device__ __forceinline__ void update_item(const Dev& d, int v, int use_hat, int nc, const double* gam, double* part) {
  if (d.pinned[v]) return;
  for (int i = 0; i < 3; ++i) update_comp(d, 3 * (size_t)v + i, use_hat, nc, gam, part);
}

template <class St>
__device__ __forceinline__ void update_finish(const Dev& d, St* c, const double* s) {
  c->dq_norm2 = s[0];
  c->qprev_norm2 = s[1];
  c->k += 1;
  if (d.fixed_iters > 0 && c->k >= d.fixed_iters) c->done = 1;
}

// update bookkeeping when the step norms are carried into the next assembly
template <class St>
__device__ __forceinline__ void update_count(const Dev& d, St* c) {
  c->k += 1;
  if (d.fixed_iters > 0 && c->k >= d.fixed_iters) c->done = 1;
}

// ------------------------------------------------------------ step end

template <class St>
__device__ __forceinline__ void step_end_ctrl(const Dev& d, St* c, bool writer) {
  c->iters_total += c->k;
  if (c->k > c->iters_max) c->iters_max = c->k;
  if (writer && d.phase_count) {
    d.phase_count[2 * c->t] = c->n_local;
    d.phase_count[2 * c->t + 1] = c->n_solve;
  }
}

__device__ __forceinline__ void step_end_item(const Dev& d, int v, double* qn, double* vn, double* ckpt_next) {
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    const double q = d.q[o];
    if (qn) qn[o] = q;
    if (vn) vn[o] = d.pinned[v] ? 0.0 : (q - d.qt[o]) / d.h;
    if (ckpt_next) ckpt_next[o] = q;
  }
}

// Trust-region selection (eq. tr_step, tr_decreases, tr_ratio, tr_rule):
// elements contribute V_e (psi_e(F(q*-1)) - psi_e(F(q*))) with per-element
// mu_e, lambda_e (+inf if inverted), vertices the kinetic difference and the
// quadratic form dq^T A dq. Items [0, n_e) are elements, the rest vertices.
__device__ __forceinline__ double psi_elem(const Dev& d, const double* x, int e, bool& inverted) {
  const int4 tv = d.tets[e];
  double Bm[9];
  for (int i = 0; i < 9; ++i) Bm[i] = d.Bm64[9 * (size_t)e + i];
  double F[9];
  deform<double>(x, tv, Bm, F);
  const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
  if (!(J > 0.0)) {
    inverted = true;
    return 0.0;
  }
  double n2 = 0.0;
  for (int i = 0; i < 9; ++i) n2 += F[i] * F[i];
  const double lnJ = log(J), mu = d.mu_e[e], lam = d.lam_e[e];
  return d.vol[e] * (0.5 * mu * (n2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
}

__device__ __forceinline__ void tr_item(const Dev& d, int tid, double* part) {
  if (tid < d.n_e) {
    bool inv = false;
    const double a = psi_elem(d, d.qprev, tid, inv);
    const double b = psi_elem(d, d.q, tid, inv);
    part[0] += a - b;
    if (inv) part[3] += 1.0;
  } else if (tid < d.n_e + d.n_v) {
    const int v = tid - d.n_e;
    if (d.pinned[v]) return;
    const double m = d.mass[v];
    for (int i = 0; i < 3; ++i) {
      const size_t o = 3 * (size_t)v + i;
      const double a = d.qprev[o] - d.qtil[o], b = d.q[o] - d.qtil[o];
      part[1] += 0.5 * m / (d.h * d.h) * (a * a - b * b);
      double Adq = 0.0;
      for (int p = d.A_ptr[v]; p < d.A_ptr[v + 1]; ++p) {
        const int u = d.A_idx[p];
        Adq += d.A_val[p] * (d.q[3 * (size_t)u + i] - d.qprev[3 * (size_t)u + i]);
      }
      part[2] += (d.q[o] - d.qprev[o]) * Adq;
    }
  }
}

template <class St>
__device__ __forceinline__ void tr_finish(const Dev& d, St* c, const double* s, bool writer) {
  const double act = s[0] + s[1];
  const double mod = 0.5 * fabs(s[2]);
  const bool inverted = s[3] > 0.0;
  const double rho = mod < 1e-12 ? 1.0 : (inverted ? INFINITY : act / mod);
  double tau;
  if (d.tr_mode == 1) tau = 0.0;
  else if (d.tr_mode == 2) tau = 0.5;
  else if (d.tr_mode == 3) tau = 1.0;
  else tau = (isfinite(rho) && fabs(rho - 1.0) <= d.eps_tr) ? 0.5 : 1.0;
  if (tau == 0.5) c->tau_half += 1; else if (tau == 1.0) c->tau_one += 1;
  c->last_rho = rho;
  if (writer) d.tau[c->t] = tau;
}

}  // namespace pdk
