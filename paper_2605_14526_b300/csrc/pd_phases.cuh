// Per-item bodies of the forward phases (Alg. 1) and the scalar logic run by
// the block that completes each reduction. Shared by the per-phase kernels
// (pd_kernels.cu) and the persistent rollout kernel (pd_persistent.cu), so the
// two launch paths execute identical arithmetic. Pointers here are plain (no
// __restrict__ / read-only cache): inside the persistent kernel the same
// arrays are rewritten by other blocks between grid barriers.
#pragma once
#include "pd_common.cuh"

namespace pdk {

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
    d.qprev[3 * v + i] = q[i];
    d.gprev[3 * v + i] = 0.0;
    d.b0[3 * v + i] = b0[i];
    if (ckpt_t) ckpt_t[3 * v + i] = q[i];
  }
}

// ------------------------------------------------------------ local step

// Local step fused with the per-element part of the RHS scatter (Alg. 1,
// eq. nh_prox / corotated projection, eq. A_basic). The prox Newton starts
// from this element's sigma* of its previous local step when one is stored.
template <typename T>
__device__ __forceinline__ void local_item(const Dev& d, int e, const double* x) {
  int4 tv;
  T Bm[9], coef;
  load_elem<T>(d, e, tv, Bm, coef);
  T F[9], U[9], V[9], sF[3], ss[3], P[9], c[12];
  deform<T>(x, tv, Bm, F);
  svd3<T>(F, U, sF, V);
  if (d.model == 0) {
    ss[0] = ss[1] = ss[2] = T(1);
  } else {
    NHMean<T> m{(T)d.mu_bar, (T)d.lam_bar, (T)d.k_bar};
    float* ws = reinterpret_cast<float*>(d.sstar) + 3 * (size_t)e;
    T s0[3];
    const bool warm = ws[0] > 0.f && ws[1] > 0.f && ws[2] > 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) s0[i] = warm ? (T)ws[i] : (sF[i] > T(0.1) ? sF[i] : T(0.1));
    nh_prox_from<T>(sF, m, s0, ss);
#pragma unroll
    for (int i = 0; i < 3; ++i) ws[i] = (float)ss[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[3 * i + j] = U[3 * i] * ss[0] * V[3 * j] + U[3 * i + 1] * ss[1] * V[3 * j + 1] + U[3 * i + 2] * ss[2] * V[3 * j + 2];
  corner_forces<T>(P, Bm, coef, c);
  T* out = reinterpret_cast<T*>(d.contrib) + 12 * (size_t)e;
#pragma unroll
  for (int i = 0; i < 12; ++i) out[i] = c[i];
}

// b^k = b0 + sum of corner contributions (FP64) in vertex order and in
// elimination order; partials ||b^k - b^{k-1}||^2, ||b^{k-1}||^2, non-finite
template <typename T>
__device__ __forceinline__ void assemble_item(const Dev& d, int v, int k, double* part) {
  if (d.pinned[v]) return;
  double acc[3] = {d.b0[3 * v], d.b0[3 * v + 1], d.b0[3 * v + 2]};
  gather_contrib<T>(d, v, acc);
  const int pos = d.iperm[v];
  for (int i = 0; i < 3; ++i) {
    const double bp = d.bprev[3 * v + i];
    if (k > 0) {
      part[0] += (acc[i] - bp) * (acc[i] - bp);
      part[1] += bp * bp;
    }
    d.b[3 * v + i] = acc[i];
    d.bperm[3 * (size_t)pos + i] = acc[i];
    d.y[3 * (size_t)pos + i] = 0.0;
  }
  if (!finite3(acc[0], acc[1], acc[2])) part[2] += 1.0;
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

// one segment of a skyline row of S: y_row += S[row, seg] x[seg] (3 RHS);
// four independent accumulator sets per lane keep several loads in flight
__device__ __forceinline__ void spmv_s_segment(const Dev& d, const double* xin, double* y, int sg, int lane) {
  const int4 seg = d.s_seg[sg];  // x = row, y = offset in row, z = length, w = multi
  const int row = seg.x;
  const double* sv = d.s_val + d.s_rowptr[row] + seg.y;
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
  double a0 = (a[0][0] + a[1][0]) + (a[2][0] + a[3][0]);
  double a1 = (a[0][1] + a[1][1]) + (a[2][1] + a[3][1]);
  double a2 = (a[0][2] + a[1][2]) + (a[2][2] + a[3][2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    double* yr = y + 3 * (size_t)row;
    if (seg.w) {
      atomicAdd(yr, a0);
      atomicAdd(yr + 1, a1);
      atomicAdd(yr + 2, a2);
    } else {
      yr[0] = a0;
      yr[1] = a1;
      yr[2] = a2;
    }
  }
}

// row j of S^T: sum over the ancestors i of j of S_ij y_i, returned to every
// lane; indices of four entries are loaded before their y values
__device__ __forceinline__ void spmv_st_sum(const Dev& d, const double* y, int j, int lane, double& r0, double& r1,
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
      sv[u] = d.st_val[p + 32 * u];
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
    const double s = d.st_val[p];
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

// row j of S^T written to out[perm[j]]
__device__ __forceinline__ void spmv_st_row(const Dev& d, const double* y, double* out, int j, int lane) {
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
    d.dQ[a.slot * nv3 + o] = q - d.qprev[o];
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

// Gram update, regularised normal equations, reliability guard (eq. aa_gamma)
template <class St>
__device__ __forceinline__ void aa_finish(const Dev& d, St* c, const AAView& a, const double* s) {
  c->n_solve += 1;
  const int m = a.m;
  c->use_hat = 1;
  if (m == 0) return;
  if (a.add) {
    for (int j = 0; j < a.ncols_new; ++j) {
      c->gram[a.slot * kMaxAA + j] = s[j];
      c->gram[j * kMaxAA + a.slot] = s[j];
    }
    c->ncols = a.ncols_new;
    c->head = (a.slot + 1) % m;
  }
  c->pairs = c->pairs < m + 1 ? c->pairs + 1 : m + 1;
  const int nc = c->ncols;
  if (nc < 1) return;
  // (G + reg I) gamma = dG^T g with reg = max(1e-6 tr(G) / nc, 1e-12), solved by
  // mixed-precision iterative refinement (Wilkinson; Moler 1967): an FP32
  // Cholesky factor of the trace-normalised matrix and FP64 residuals. A
  // single-thread FP64 factorisation costs several microseconds on this part.
  const double inv_n[kMaxAA + 1] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8};
  double tr = 0.0;
  for (int j = 0; j < nc; ++j) tr += c->gram[j * kMaxAA + j];
  const double reg = fmax(1e-6 * tr * inv_n[nc], 1e-12);
  const float sc = 1.0f / (float)(tr + nc * reg);
  float L[kMaxAA * kMaxAA], ipiv[kMaxAA];
  bool ok = true;
  for (int j = 0; j < nc && ok; ++j) {
    float t = (float)(c->gram[j * kMaxAA + j] + reg) * sc;
    for (int k2 = 0; k2 < j; ++k2) t -= L[j * kMaxAA + k2] * L[j * kMaxAA + k2];
    if (!(t > 0.0f)) {
      ok = false;
      break;
    }
    const float r = sqrtf(t);
    ipiv[j] = 1.0f / r;
    for (int i = j + 1; i < nc; ++i) {
      float u = (float)c->gram[i * kMaxAA + j] * sc;
      for (int k2 = 0; k2 < j; ++k2) u -= L[i * kMaxAA + k2] * L[j * kMaxAA + k2];
      L[i * kMaxAA + j] = u * ipiv[j];
    }
    L[j * kMaxAA + j] = r;
  }
  double gam[kMaxAA];
  for (int i = 0; i < nc; ++i) gam[i] = 0.0;
  double gn = 0.0;
  if (ok) {
    for (int pass = 0; pass < 3; ++pass) {
      float y[kMaxAA];
      for (int i = 0; i < nc; ++i) {  // residual in FP64, forward solve in FP32
        double r = s[kMaxAA + i] - reg * gam[i];
        for (int j = 0; j < nc; ++j) r -= c->gram[i * kMaxAA + j] * gam[j];
        float u = (float)r * sc;
        for (int k2 = 0; k2 < i; ++k2) u -= L[i * kMaxAA + k2] * y[k2];
        y[i] = u * ipiv[i];
      }
      for (int i = nc - 1; i >= 0; --i) {
        float u = y[i];
        for (int k2 = i + 1; k2 < nc; ++k2) u -= L[k2 * kMaxAA + i] * y[k2];
        y[i] = u * ipiv[i];
      }
      for (int i = 0; i < nc; ++i) gam[i] += (double)y[i];
    }
    for (int i = 0; i < nc; ++i) gn += gam[i] * gam[i];
  }
  if (!ok || !(gn <= 100.0)) {  // reliability guard ||gamma||_2 > 10: take q_hat, clear the history
    c->resets += 1;
    c->pairs = 0;
    c->ncols = 0;
    c->head = 0;
    for (int i = 0; i < kMaxAA * kMaxAA; ++i) c->gram[i] = 0.0;
  } else {
    for (int i = 0; i < nc; ++i) c->gamma[i] = gam[i];
    c->use_hat = 0;
  }
}

// q^{k+1} = q_hat - (dQ + dG) gamma (or q_hat); step-norm partials
__device__ __forceinline__ void update_item(const Dev& d, int v, int use_hat, int nc, const double* gam, double* part) {
  if (d.pinned[v]) return;
  const size_t nv3 = 3 * (size_t)d.n_v;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    double qn = d.qhat[o];
    if (!use_hat)
#pragma unroll
      for (int j = 0; j < kMaxAA; ++j)
        if (j < nc) qn -= gam[j] * (d.dQ[j * nv3 + o] + d.dG[j * nv3 + o]);
    const double qo = d.q[o];
    part[0] += (qn - qo) * (qn - qo);
    part[1] += qo * qo;
    d.qprev[o] = qo;
    d.q[o] = qn;
    d.bprev[o] = d.b[o];
  }
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
