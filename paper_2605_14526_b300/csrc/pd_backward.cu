// Backward pass (Sec. 4.3 trust region, Sec. 4.7 adjoint, Alg. 2).
//
// Per step t (walked from T-1 down to 0) with q* = q_{t+1}:
//   setup   per element: SVD of F(q*), prox stretches sigma*, the filtered
//           stretch Jacobian J = k H~(tau)^+ (eq. tr_blend, tr_ift) and the
//           off-diagonal coefficients of the spectral differential, stored as
//           a compact record so that K = db/dq is applied matrix-free.
//   solve   (A - K) mu = q_bar by conjugate gradients preconditioned with the
//           factor of A (z = S^T S r), K applied per element (eq. db_dq).
//   route   dL/dq_t, dL/dv_t, dL/df_ext per vertex; dL/dw_e, dL/dbeta_e per
//           element (SVD and prox recomputed in FP64); mesh-mean
//           sensitivities reduced.
// After the last step, the chain to E_e and nu (eq. lame and the weights).
// Item bodies and scalar logic are shared by the per-phase kernels and the
// persistent backward kernel (one cooperative launch for all T steps).
#include <cuda_runtime.h>

#include "pd_coop.h"
#include "pd_grid.cuh"
#include "pd_launch.h"
#include "pd_contact.cuh"
#include "pd_phases.cuh"
#include "pd_tsolve.cuh"
#include "pd_bwd_elem.cuh"

namespace pdk {

struct BwdState {
  int adj_k, adj_done, status, adj_iters_total, adj_iters_max, adj_not_converged;
  double rz, rz0, alpha, beta, acc_mu, acc_lam, acc_k, dnu_acc;
  // contact projection: the masked CG on W_a, one scalar set per axis
  double cg_rr[3], cg_rr0[3], cg_alpha[3], cg_beta[3];
  int cg_done, cg_it, cg_rot, con_cg, con_cg_unconverged;
  int restart, restarts;   // contact: restarts of the outer CG from its true residual
};

// ------------------------------------------------------------ per-item bodies

__device__ __forceinline__ void bwd_begin_item(const Dev& d, int i, const double* dqT, const double* dvT) {
  if (i < d.n_e) {
    d.dw[i] = 0.0;
    d.dw1[i] = 0.0;
    d.dbeta[i] = 0.0;
  }
  if (i < d.n_v) {
    const bool pin = d.pinned[i];
    for (int a = 0; a < 3; ++a) {
      d.gq[3 * i + a] = pin ? 0.0 : dqT[3 * i + a];
      d.gv[3 * i + a] = (pin || !dvT) ? 0.0 : dvT[3 * i + a];
    }
  }
}

// q_bar = dL/dq* + dL/dv*/h; r = q_bar; mu = 0; r in elimination order
__device__ __forceinline__ void bwd_init_item(const Dev& d, int v) {
  const bool pin = d.pinned[v];
  double rv[3];
  for (int a = 0; a < 3; ++a) {
    const size_t o = 3 * (size_t)v + a;
    const double qb = pin ? 0.0 : d.gq[o] + d.gv[o] / d.h;
    rv[a] = qb;
    d.qbar[o] = qb;
    d.r[o] = qb;
    d.mu[o] = 0.0;
    d.pdir[o] = 0.0;
    d.pdir2[o] = 0.0;
    d.z[o] = 0.0;
  }
  if (!pin) {
    const int pos = d.iperm[v];
    for (int a = 0; a < 3; ++a) store_rhs(d, d.bperm, 3 * (size_t)pos + a, rv[a]);
  }
}

// p = z (first direction); partial r . z
__device__ __forceinline__ void init_z_item(const Dev& d, int v, double* part) {
  if (d.pinned[v]) return;
  for (int a = 0; a < 3; ++a) {
    const size_t o = 3 * (size_t)v + a;
    part[0] += d.r[o] * d.z[o];
    d.pdir[o] = d.z[o];
  }
}

// w = A p - K p; partial p . w
template <typename T>
__device__ __forceinline__ void pcg_w_item(const Dev& d, int v, double* part) {
  if (d.pinned[v]) return;
  double acc[3] = {0.0, 0.0, 0.0};
  gather_contrib<T>(d, v, acc);
  double ap[3] = {0.0, 0.0, 0.0};
  const int beg = d.A_ptr[v], end = d.A_ptr[v + 1];
  for (int p0 = beg; p0 < end; p0 += 8) {   // chunks of 8: overlapped loads, same order
    int uu[8];
    double av[8], pv[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uu[k] = p0 + k < end ? d.A_idx[p0 + k] : -1;
      av[k] = p0 + k < end ? d.A_val[p0 + k] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) pv[k][i] = uu[k] >= 0 ? d.pdir[3 * (size_t)uu[k] + i] : 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (uu[k] >= 0)
#pragma unroll
        for (int i = 0; i < 3; ++i) ap[i] += av[k] * pv[k][i];
  }
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    const double w = ap[i] - acc[i];
    d.w[o] = w;
    part[0] += d.pdir[o] * w;
  }
}

// persistent adjoint, one warp per vertex: p = z + beta p_old stored to
// pnew, w = A p - K p (lanes over the row of A and the incident corners, a
// fixed shuffle tree), partial p . w
template <typename T>
__device__ __forceinline__ void pcg_w_warp(const Dev& d, int v, const double* pold, double* pnew, double beta, int lane,
                                           double* part) {
  if (d.pinned[v]) return;
  const T* cb = reinterpret_cast<const T*>(d.contrib);
  double c[3] = {0.0, 0.0, 0.0};
  for (int p = d.A_ptr[v] + lane; p < d.A_ptr[v + 1]; p += 32) {
    const int u = d.A_idx[p];
    const double a = d.A_val[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] += a * p_next(d, pold, 3 * (size_t)u + i, beta);
  }
  for (int p = d.inc_ptr[v] + lane; p < d.inc_ptr[v + 1]; p += 32) {
    const int ic = d.inc_idx[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] -= (double)cb[3 * (size_t)ic + i];
  }
  int i;
  const double w = warp_sum_scatter<3>(c, lane, i);   // component i in lanes 8i .. 8i+7
  if ((lane & 7) != 0 || i >= 3) return;
  const size_t o = 3 * (size_t)v + i;
  const double pn = p_next(d, pold, o, beta);
  pnew[o] = pn;
  d.w[o] = w;
  part[0] += pn * w;
}

// true residual of the adjoint equations, one warp per vertex: r = q_bar -
// (A mu - K mu) with K mu from the corner contributions of kapply_item(mu);
// r also goes to the right-hand side of the next product with S
template <typename T>
__device__ __forceinline__ void resid_warp(const Dev& d, int v, int lane) {
  if (d.pinned[v]) return;
  const T* cb = reinterpret_cast<const T*>(d.contrib);
  double c[3] = {0.0, 0.0, 0.0};
  for (int p = d.A_ptr[v] + lane; p < d.A_ptr[v + 1]; p += 32) {
    const int u = d.A_idx[p];
    const double a = d.A_val[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] += a * d.mu[3 * (size_t)u + i];
  }
  for (int p = d.inc_ptr[v] + lane; p < d.inc_ptr[v + 1]; p += 32) {
    const int ic = d.inc_idx[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] -= (double)cb[3 * (size_t)ic + i];
  }
  int i;
  const double w = warp_sum_scatter<3>(c, lane, i);
  if ((lane & 7) != 0 || i >= 3) return;
  const size_t o = 3 * (size_t)v + i;
  const double r = d.qbar[o] - w;
  d.r[o] = r;
  store_rhs(d, d.bperm, 3 * (size_t)d.iperm[v] + i, r);
}

__device__ __forceinline__ void pcg_r_item(const Dev& d, int v, double alpha, const double* pdir = nullptr) {
  if (d.pinned[v]) return;
  const int pos = d.iperm[v];
  const double* pd = pdir ? pdir : d.pdir;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    d.mu[o] += alpha * pd[o];
    const double rn = d.r[o] - alpha * d.w[o];
    d.r[o] = rn;
    store_rhs(d, d.bperm, 3 * (size_t)pos + i, rn);
  }
}

__device__ __forceinline__ void pcg_z_item(const Dev& d, int v, double* part) {
  if (d.pinned[v]) return;
  for (int i = 0; i < 3; ++i) part[0] += d.r[3 * (size_t)v + i] * d.z[3 * (size_t)v + i];
}

__device__ __forceinline__ void pcg_p_item(const Dev& d, int v, double beta) {
  if (d.pinned[v]) return;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    d.pdir[o] = d.z[o] + beta * d.pdir[o];
  }
}

// dL/dq_t = (1 + alpha h) M/h^2 mu + B mu / h - v_bar/h, dL/dv_t = M/h mu, dL/df = mu
__device__ __forceinline__ void route_vertex_item(const Dev& d, int v, double* df, int df_acc) {
  if (d.pinned[v]) {
    for (int i = 0; i < 3; ++i) {
      d.gq[3 * v + i] = 0.0;
      d.gv[3 * v + i] = 0.0;
      if (df && !df_acc) df[3 * v + i] = 0.0;
    }
    return;
  }
  const double m = d.mass[v], h = d.h;
  double bmu[3] = {0.0, 0.0, 0.0};
  for (int p = d.B_ptr[v]; p < d.B_ptr[v + 1]; ++p) {
    const int u = d.B_idx[p];
    const double b = d.B_val[p];
    for (int i = 0; i < 3; ++i) bmu[i] += b * d.mu[3 * (size_t)u + i];
  }
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    const double mu = d.mu[o];
    const double gv_next = d.gv[o];
    d.gq[o] = (1.0 + d.alpha_d * h) * m / (h * h) * mu + bmu[i] / h - gv_next / h;
    d.gv[o] = m / h * mu;
    if (df) df[o] = df_acc ? df[o] + mu : mu;
  }
}

// per element, in FP64: dL/dw_e = V_e <G mu, p* - F>, dL/dbeta_e, and the
// mean-sensitivity partials; p* - F = U diag(s* - s_F) V^T is a small
// difference of O(1) quantities, so the SVD and prox are recomputed in double
__device__ __forceinline__ void route_elem_item(const Dev& d, int e, const double* qstar, const double* qt, double tau,
                                                double* part) {
  const int4 tv = d.tets[e];
  double Bm[9];
  for (int i = 0; i < 9; ++i) Bm[i] = d.Bm64[9 * (size_t)e + i];
  double Gm[9], Fs[9], Ft[9];
  deform<double>(d.mu, tv, Bm, Gm);
  deform<double>(qstar, tv, Bm, Fs);
  deform<double>(qt, tv, Bm, Ft);
  double gb = 0.0;
  for (int i = 0; i < 9; ++i) gb += Gm[i] * (Fs[i] - Ft[i]);
  double U[9], V[9], sf[3], ss[3], sv[3] = {1.0, 1.0, 1.0};
  svd3<double>(Fs, U, sf, V);
  NHMean<double> m{d.mu_bar, d.lam_bar, d.k_bar};
  const NHMean<double> mb = barrier_prox_energy<double>(d);
  if (d.model == 1) {
    nh_prox<double>(sf, m, ss);
  } else {
    // corotated, and the rotation weight of models 2 and 3: p = R; their
    // volume weight takes p_vol = U diag(sigma_v) V^T below (sigma_v: the
    // volume step, or the barrier's prox)
    ss[0] = ss[1] = ss[2] = 1.0;
    if (d.model == 2) {
      double nu;
      vol_project<double>(sf, sv, nu);
    } else if (d.model == 3) {
      nh_prox<double>(sf, mb, sv);
    }
  }
  double Md[3];  // diagonal of U^T (G mu) V
  for (int i = 0; i < 3; ++i) {
    double acc = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) acc += U[3 * k + i] * Gm[3 * k + l] * V[3 * l + i];
    Md[i] = acc;
  }
  double dw = 0.0;
  for (int i = 0; i < 3; ++i) dw += (ss[i] - sf[i]) * Md[i];
  d.dw[e] += d.vol[e] * dw;
  if (d.model == 2 || d.model == 3) {   // b carries w_0 V G^T R + w_1 V G^T p_vol, A carries w_0 + w_1
    double dw1 = 0.0;
    for (int i = 0; i < 3; ++i) dw1 += (sv[i] - sf[i]) * Md[i];
    d.dw1[e] += d.vol[e] * dw1;
  }
  d.dbeta[e] += -d.vol[e] / d.h * gb;
  if (d.model == 3) {
    // dL/dr of the barrier (r = mu/lambda inside its prox) into the first
    // mean slot: lambda_e V_e <G mu, U diag(d sigma_b/d r) V^T> with
    // d sigma_b/d r = H~^+ (1/sigma_b) (the IFT on the stationarity
    // (ln J - r)/sigma_i + sigma_i - sigma_F,i = 0, filtered like K)
    double Jm[9];
    filtered_jacobian<double>(sv, mb, tau, Jm);
    const double lam_e = d.E[e] * d.nu / ((1.0 + d.nu) * (1.0 - 2.0 * d.nu));
    const double coef = lam_e * d.vol[e];
    for (int i = 0; i < 3; ++i) {
      double ds = 0.0;
      for (int j = 0; j < 3; ++j) ds += Jm[3 * i + j] / sv[j];
      part[0] += coef * Md[i] * ds;
    }
  }
  if (d.model == 1) {
    double Jm[9];
    filtered_jacobian<double>(ss, m, tau, Jm);
    const double lnJ = log(ss[0] * ss[1] * ss[2]);
    const double k = d.k_bar, coef = d.coef64[e];
    double gk[3], gm[3], gl[3];
    for (int i = 0; i < 3; ++i) {
      gk[i] = ss[i] - sf[i];
      gm[i] = ss[i] - 1.0 / ss[i];
      gl[i] = lnJ / ss[i];
    }
    for (int i = 0; i < 3; ++i) {
      double sk = 0.0, sm = 0.0, sl = 0.0;
      for (int j = 0; j < 3; ++j) {
        sk += Jm[3 * i + j] * gk[j];
        sm += Jm[3 * i + j] * gm[j];
        sl += Jm[3 * i + j] * gl[j];
      }
      part[0] += -coef * Md[i] * sm / k;
      part[1] += -coef * Md[i] * sl / k;
      part[2] += -coef * Md[i] * sk / k;
    }
  }
}

// dL/dE_e from dL/dw_e, dL/dbeta_e and the mean sensitivities; nu partials
__device__ __forceinline__ void chain_item(const Dev& d, int e, double* dE, double am, double al, double ak,
                                           double* part) {
  const double nu = d.nu, E = d.E[e];
  const bool nh = d.model == 1;
  const double dmu_dE = 1.0 / (2.0 * (1.0 + nu));
  const double dlam_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double dmu_dnu = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
  const double den = (1.0 + nu) * (1.0 - 2.0 * nu);
  const double dlam_dnu = E * (1.0 + 2.0 * nu * nu) / (den * den);
  const double dw_dE = 2.0 * dmu_dE + (nh ? dlam_dE : 0.0);
  const double dw_dnu = 2.0 * dmu_dnu + (nh ? dlam_dnu : 0.0);
  const double cb = d.mu_ref > 0.0 ? d.beta0 / d.mu_ref : 0.0;
  const double inv_n = 1.0 / d.n_e;
  // the two weights of models 2 and 3: w_0 = 2 mu (dw), w_1 = lambda (dw1)
  const bool two = d.model == 2 || d.model == 3;
  const double v1E = two ? d.dw1[e] * dlam_dE : 0.0;
  const double v1nu = two ? d.dw1[e] * dlam_dnu : 0.0;
  // the mesh means enter only the Neo-Hookean prox (model 3 keeps dL/dr in am)
  const double mE = nh ? (am * dmu_dE + al * dlam_dE + ak * dw_dE) * inv_n : 0.0;
  if (dE) dE[e] = d.dw[e] * dw_dE + v1E + d.dbeta[e] * cb * dmu_dE + mE;
  part[0] += d.dw[e] * dw_dnu + v1nu + d.dbeta[e] * cb * dmu_dnu;
  part[1] += dmu_dnu;
  part[2] += dlam_dnu;
  part[3] += dw_dnu;
}

// ------------------------------------------------------------ scalar logic

template <class St>
__device__ __forceinline__ void init_z_finish(St* c, const double* s) {
  c->rz = s[0];
  c->rz0 = s[0];
  c->adj_k = 0;
  c->adj_done = s[0] > 0.0 ? 0 : 1;
}

template <class St>
__device__ __forceinline__ void pcg_w_finish(St* c, const double* s) {
  const double pw = s[0];
  if (!(pw > 0.0) || !isfinite(pw)) {  // (A - K) not positive along p
    c->status |= 2;
    c->adj_done = 1;
    c->alpha = 0.0;
  } else {
    c->alpha = c->rz / pw;
  }
}

template <class St>
__device__ __forceinline__ void pcg_z_finish(const Dev& d, St* c, const double* s) {
  const double rz = s[0];
  c->beta = rz / c->rz;
  c->rz = rz;
  c->adj_k += 1;
  // also ends when r . z stops being positive: with contact constraints the
  // projected preconditioner is positive only up to the consistency of W with
  // the device's A^-1, and r . z falls through zero once the residual reaches
  // that level (the accuracy the projection allows)
  if (!(rz > d.adj_tol * d.adj_tol * c->rz0)) {
    c->adj_done = 1;
  } else if (c->adj_k >= d.adj_max_iters) {
    c->adj_done = 1;
    c->adj_not_converged += 1;
  }
}

template <class St>
__device__ __forceinline__ void route_finish(St* c, const double* s) {
  c->acc_mu += s[0];
  c->acc_lam += s[1];
  c->acc_k += s[2];
  c->adj_iters_total += c->adj_k;
  if (c->adj_k > c->adj_iters_max) c->adj_iters_max = c->adj_k;
}

__device__ __forceinline__ double chain_nu(const Dev& d, double am, double al, double ak, const double* s) {
  if (d.model == 3) return s[0] - am / (2.0 * d.nu * d.nu);   // dL/dr dr/dnu, r = (1 - 2 nu)/(2 nu)
  const double inv_n = 1.0 / d.n_e;
  return s[0] + (am * s[1] + al * s[2] + ak * s[3]) * inv_n;
}

// ------------------------------------------------------------ per-phase kernels

__global__ void k_bwd_begin(Dev d, const double* dqT, const double* dvT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    Ctrl* c = d.ctrl;
    c->acc_mu = c->acc_lam = c->acc_k = 0.0;
    c->adj_iters_total = c->adj_iters_max = c->adj_not_converged = 0;
  }
  bwd_begin_item(d, i, dqT, dvT);
}

template <typename T>
__global__ void __launch_bounds__(kTetBlock) k_bwd_setup(Dev d, const double* qstar, const double* tau_t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_e) bwd_setup_item<T>(d, e, qstar, *tau_t);
}

template <typename T>
__global__ void __launch_bounds__(kTetBlock) k_kapply(Dev d, const double* pv) {
  if (d.ctrl->adj_done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_e) kapply_item<T>(d, e, pv);
}

__global__ void k_bwd_init(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) {
    d.ctrl->adj_k = 0;
    d.ctrl->adj_done = 0;
  }
  if (v < d.n_v) bwd_init_item(d, v);
}

__global__ void __launch_bounds__(kVtxBlock) k_pcg_init_z(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (v < d.n_v) init_z_item(d, v, part);
  block_reduce_store<1>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_PCG_INIT]) && threadIdx.x == 0) {
    double s[1] = {sum_partials(d.red, gridDim.x, 0)};
    init_z_finish(d.ctrl, s);
  }
}

template <typename T>
__global__ void __launch_bounds__(kVtxBlock) k_pcg_w(Dev d) {
  if (d.ctrl->adj_done) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (v < d.n_v) pcg_w_item<T>(d, v, part);
  block_reduce_store<1>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_PCG_W]) && threadIdx.x == 0) {
    double s[1] = {sum_partials(d.red, gridDim.x, 0)};
    pcg_w_finish(d.ctrl, s);
  }
}

__global__ void __launch_bounds__(kVtxBlock) k_pcg_r(Dev d) {
  if (d.ctrl->adj_done) return;
  const double alpha = d.ctrl->alpha;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n_v) pcg_r_item(d, v, alpha);
}

__global__ void __launch_bounds__(kVtxBlock) k_pcg_z(Dev d) {
  if (d.ctrl->adj_done) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (v < d.n_v) pcg_z_item(d, v, part);
  block_reduce_store<1>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_PCG_Z]) && threadIdx.x == 0) {
    double s[1] = {sum_partials(d.red, gridDim.x, 0)};
    pcg_z_finish(d, d.ctrl, s);
  }
}

__global__ void __launch_bounds__(kVtxBlock) k_pcg_p(Dev d) {
  if (d.ctrl->adj_done) return;
  const double beta = d.ctrl->beta;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n_v) pcg_p_item(d, v, beta);
}

__global__ void __launch_bounds__(kVtxBlock) k_route(Dev d, const double* qstar, const double* qt, const double* tau_t,
                                                     double* df, int df_acc) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double part[3] = {0.0, 0.0, 0.0};
  if (tid < d.n_v) route_vertex_item(d, tid, df, df_acc);
  else if (tid < d.n_v + d.n_e) route_elem_item(d, tid - d.n_v, qstar, qt, *tau_t, part);
  block_reduce_store<3>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_ROUTE]) && threadIdx.x == 0) {
    double s[3];
    for (int j = 0; j < 3; ++j) s[j] = sum_partials(d.red, gridDim.x, j);
    route_finish(d.ctrl, s);
  }
}

__global__ void __launch_bounds__(kVtxBlock) k_chain(Dev d, double* dE, double* dnu) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  const Ctrl* c = d.ctrl;
  if (e < d.n_e) chain_item(d, e, dE, c->acc_mu, c->acc_lam, c->acc_k, part);
  block_reduce_store<4>(part, d.red, blockIdx.x);
  if (last_block(&d.ctrl->ticket[TK_CHAIN]) && threadIdx.x == 0) {
    double s[4];
    for (int j = 0; j < 4; ++j) s[j] = sum_partials(d.red, gridDim.x, j);
    const double v = chain_nu(d, c->acc_mu, c->acc_lam, c->acc_k, s);
    if (dnu) *dnu = v;
    d.ctrl->dnu_acc = v;
  }
}

__global__ void k_bwd_finish(Dev d, double* dq0, double* dv0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * d.n_v) return;
  if (dq0) dq0[i] = d.gq[i];
  if (dv0) dv0[i] = d.gv[i];
}

// ------------------------------------------------------------ persistent backward

// mode T: each finished row j of z = A^-1 r (elimination order) goes to z
// and to this thread's partial of r . z (lanes 0..2)
struct FinRZ {
  const Dev* d;
  double acc;
  __device__ __forceinline__ void operator()(int j, double a0, double a1, double a2) {
    const int lane = threadIdx.x & 31;
    if (lane < 3) {
      const size_t o = 3 * (size_t)d->perm[j] + lane;
      const double zv = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
      d->z[o] = zv;
      acc += d->r[o] * zv;
    }
  }
  __device__ __forceinline__ void lanes(bool on, int j, double a0, double a1, double a2) {
    if (!on) return;
    const size_t o = 3 * (size_t)d->perm[j];
    d->z[o] = a0;
    d->z[o + 1] = a1;
    d->z[o + 2] = a2;
    acc += d->r[o] * a0 + d->r[o + 1] * a1 + d->r[o + 2] * a2;
  }
};

template <typename T>
__device__ __forceinline__ void bwd_rollout_body(const Dev& d, const BwdArgs& a, const Team tm) {
  __shared__ BwdState S;
  __shared__ double sums[4];
  const int tid = threadIdx.x;
  const int gtid = tm.b * blockDim.x + tid;
  const int gthreads = tm.nb * blockDim.x;
  const int lane = tid & 31, gwarp = gtid >> 5, nwarps = gthreads >> 5;
  const int twarp = tm.nb >= kWideTeam ? (tid >> 5) * tm.nb + tm.b : gwarp;   // as in the forward rollout
  const size_t nv3 = 3 * (size_t)d.n_v;
  const bool writer = tm.b == 0;
  const Range re = block_range(tm, d.n_e);
  const Range rv = block_range(tm, d.n_v);
  const Range rb = block_range(tm, d.n_v > d.n_e ? d.n_v : d.n_e);
  const Range rt = block_range(tm, d.n_v + d.n_e);
  const unsigned long long tstart = gtimer();
  const Range rcn = block_range(tm, d.n_con);
  if (tid == 0) {
    S.adj_k = S.adj_done = S.status = S.adj_iters_total = S.adj_iters_max = S.adj_not_converged = 0;
    S.rz = S.rz0 = S.alpha = S.beta = S.acc_mu = S.acc_lam = S.acc_k = S.dnu_acc = 0.0;
    S.con_cg = S.con_cg_unconverged = 0;
  }
  // contact: after y = S r, project the preconditioned residual onto null(G):
  // w = W_a^-1 G A^-1 r by CG on the active rows (per axis), then
  // y <- y - S G^T w, so that the S^T pass gives A^-1 (r - G^T w), and
  // r <- r - G^T w, nu <- nu + w (residual update; reset: nu <- w)
  auto project = [&](const double* ck, bool reset) -> bool {
    double pu[3] = {0.0, 0.0, 0.0};
    for (int c = gwarp; c < d.n_con; c += nwarps) proj_gather(d, c, lane, pu);
    if (!grid_reduce<3>(d, tm, pu, sums)) return false;
    if (tid == 0) {
      for (int k = 0; k < 3; ++k) S.cg_rr[k] = S.cg_rr0[k] = sums[k];
      S.cg_rot = 0;
      S.cg_it = 0;
      S.cg_done = (sums[0] == 0.0 && sums[1] == 0.0 && sums[2] == 0.0) ? 1 : 0;
    }
    __syncthreads();
    while (!S.cg_done) {
      const int rot = S.cg_rot;
      double pa[3] = {0.0, 0.0, 0.0};
      for (int c = gwarp; c < d.n_con; c += nwarps) proj_ap_row(d, c, rot, lane, pa);
      if (!grid_reduce<3>(d, tm, pa, sums)) return false;
      if (tid == 0)
        for (int k = 0; k < 3; ++k) S.cg_alpha[k] = (S.cg_rr[k] > 0.0 && sums[k] > 0.0) ? S.cg_rr[k] / sums[k] : 0.0;
      __syncthreads();
      const double al[3] = {S.cg_alpha[0], S.cg_alpha[1], S.cg_alpha[2]};
      double pr[3] = {0.0, 0.0, 0.0};
      for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x) proj_update(d, c, rot, al, pr);
      if (!grid_reduce<3>(d, tm, pr, sums)) return false;
      if (tid == 0) {
        bool all = true;
        for (int k = 0; k < 3; ++k) {
          S.cg_beta[k] = S.cg_rr[k] > 0.0 ? sums[k] / S.cg_rr[k] : 0.0;
          S.cg_rr[k] = sums[k];
          if (!(sums[k] <= 1e-26 * S.cg_rr0[k])) all = false;
        }
        S.cg_it += 1;
        S.con_cg += 1;
        if (all) S.cg_done = 1;
        else if (S.cg_it >= d.con_max_iters) {
          S.cg_done = 1;
          S.con_cg_unconverged += 1;
        }
      }
      __syncthreads();
      if (S.cg_done) break;
      const double be[3] = {S.cg_beta[0], S.cg_beta[1], S.cg_beta[2]};
      for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x) proj_dir(d, c, rot, be);
      if (tid == 0) S.cg_rot = rot + 1;
      if (!grid_sync(d, tm)) return false;
    }
    for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x) proj_impulse(d, c, reset);
    if (!grid_sync(d, tm)) return false;
    for (int i = gwarp; i < d.n_f; i += nwarps) contact_y_row(d, i, cb_nz(d), cb_nxy(d), lane);
    return grid_sync(d, tm);
  };
  for (int i = rb.lo + tid; i < rb.hi; i += blockDim.x) bwd_begin_item(d, i, a.dqT, a.dvT);
  {   // split-row counters start at zero (a launch that timed out may have left some set)
    const Range rc = block_range(tm, d.n_slot);
    for (int i = rc.lo + tid; i < rc.hi; i += blockDim.x) d.s_cnt[i] = 0;
  }
  bool ok = grid_sync(d, tm);
  for (int t = a.T - 1; t >= 0 && ok; --t) {
    const double* qstar = a.ckpt + (size_t)(t + 1) * nv3;
    const double* qt = a.ckpt + (size_t)t * nv3;
    const double tau = __ldcg(&d.tau[t]);
    const double* ck = (d.n_con > 0 && d.con_ckpt) ? d.con_ckpt + (size_t)t * 3 * d.n_con : nullptr;
    if (ck) {   // the step's total normal impulse sets the normal-active threshold
      double ps[1] = {0.0};
      for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x)
        if (!con_is_att(d, c)) ps[0] += ck[c];   // attachments carry free-sign multipliers
      if (!(ok = grid_reduce<1>(d, tm, ps, sums))) break;
      const double thr = 1e-9 * sums[0];
      for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x) contact_flag_item(d, ck, thr, qstar, qt, c);
    }
    for (int e = re.lo + tid; e < re.hi; e += blockDim.x) bwd_setup_item<T>(d, e, qstar, tau);
    for (int v = rv.lo + tid; v < rv.hi; v += blockDim.x) bwd_init_item(d, v);
    if (!(ok = grid_sync(d, tm))) break;
    // z = A^-1 r (r in elimination order in bperm) with the partial r . z of
    // each finished row fused in: S b, the contact projection, then S^T y row
    // by row; or, in mode T, the two level sweeps over the factor's
    // partitioned inverse (first direction p = z: beta = 0 and p_old = 0 on
    // the first iteration)
    auto apply_rz = [&](double* prz, bool first) -> bool {
      if (d.tmode) {
        FinRZ fin{&d, 0.0};
        const bool r = tsolve_team(d, reinterpret_cast<const double*>(d.bperm), reinterpret_cast<double*>(d.y), tm,
                                   twarp, nwarps, fin);
        prz[0] += fin.acc;
        return r;
      }
      for (int sg = twarp; sg < d.n_seg; sg += nwarps) spmv_s_segment(d, d.bperm, d.y, d.s_part, d.s_cnt, sg, lane);
      if (!grid_sync(d, tm)) return false;
      if (ck && !project(ck, first)) return false;
      for (int j = twarp; j < d.n_f; j += nwarps) {
        double a0, a1, a2;
        spmv_st_sum(d, d.y, j, lane, a0, a1, a2);
        if (lane < 3) {
          const size_t o = 3 * (size_t)d.perm[j] + lane;
          const double zv = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
          d.z[o] = zv;
          prz[0] += d.r[o] * zv;
        }
      }
      return true;
    };
    double p1[1] = {0.0};
    if (!(ok = apply_rz(p1, true))) break;
    if (!(ok = grid_reduce<1>(d, tm, p1, sums))) break;
    if (tid == 0) {
      init_z_finish(&S, sums);
      S.beta = 0.0;
      S.restart = S.restarts = 0;
    }
    __syncthreads();
    // one CG iteration: K p (elements, p formed on the fly) | p stored, w = A p
    // - K p, p . w | r, mu, b | S b | S^T y, r . z; the directions alternate
    // between two buffers so that the owners can store p while the
    // neighbours still read p_old
    for (int it = 0; !S.adj_done; ++it) {
      if (S.restart) {
        // contact (a guard: with the residual update r . z is not expected
        // to fall through zero): r . z fell below zero while the residual
        // was still above the target; start again from the true residual
        // q_bar - (A - K) mu, whose projection resets nu
        for (int e = re.lo + tid; e < re.hi; e += blockDim.x) kapply_item<T>(d, e, d.mu);
        if (!(ok = grid_sync(d, tm))) break;
        for (int v = rv.lo + (tid >> 5); v < rv.hi; v += blockDim.x >> 5) resid_warp<T>(d, v, lane);
        if (!(ok = grid_sync(d, tm))) break;
        double prz0[1] = {0.0};
        if (!(ok = apply_rz(prz0, true))) break;
        if (!(ok = grid_reduce<1>(d, tm, prz0, sums))) break;
        if (tid == 0) {
          S.rz = sums[0];
          S.beta = 0.0;
          S.restart = 0;
          if (!(S.rz > d.adj_tol * d.adj_tol * S.rz0)) S.adj_done = 1;
        }
        __syncthreads();
        if (S.adj_done) break;
      }
      const double beta = S.beta;
      const double* pold = (it & 1) ? d.pdir2 : d.pdir;
      double* pnew = (it & 1) ? d.pdir : d.pdir2;
      for (int e = re.lo + tid; e < re.hi; e += blockDim.x) kapply_item<T>(d, e, nullptr, pold, beta);
      if (!(ok = grid_sync(d, tm))) break;
      double pw[1] = {0.0};
      for (int v = rv.lo + (tid >> 5); v < rv.hi; v += blockDim.x >> 5) pcg_w_warp<T>(d, v, pold, pnew, beta, lane, pw);
      if (!(ok = grid_reduce<1>(d, tm, pw, sums))) break;
      if (tid == 0) pcg_w_finish(&S, sums);
      __syncthreads();
      if (S.adj_done) break;
      const double alpha = S.alpha;
      for (int v = rv.lo + tid; v < rv.hi; v += blockDim.x) pcg_r_item(d, v, alpha, pnew);
      if (!(ok = grid_sync(d, tm))) break;
      double prz[1] = {0.0};
      if (!(ok = apply_rz(prz, false))) break;
      if (!(ok = grid_reduce<1>(d, tm, prz, sums))) break;
      if (tid == 0) {
        pcg_z_finish(d, &S, sums);
        // contact: a negative r . z above the projection's floor (1e-16 of
        // the first r . z, i.e. a relative residual of about 1e-8) is a
        // breakdown, not convergence: restart (at most 4 times a step)
        if (ck && S.adj_done && S.rz < -1e-16 * S.rz0 && S.restarts < 4 && S.adj_k < d.adj_max_iters) {
          S.adj_done = 0;
          S.restart = 1;
          S.restarts += 1;
        }
      }
      __syncthreads();
    }
    if (!ok) break;
    double* df_t = a.df ? (a.df_stride ? a.df + (size_t)t * nv3 : a.df) : nullptr;
    double p3[3] = {0.0, 0.0, 0.0};
    for (int i = rt.lo + tid; i < rt.hi; i += blockDim.x) {
      if (i < d.n_v) route_vertex_item(d, i, df_t, a.df_stride == 0 ? 1 : 0);
      else route_elem_item(d, i - d.n_v, qstar, qt, tau, p3);
    }
    if (!(ok = grid_reduce<3>(d, tm, p3, sums))) break;
    if (tid == 0) route_finish(&S, sums);
    __syncthreads();
    if (ck) {
      // sticking contacts: the constraint q_xy = q_t,xy routes nu_S to dL/dq_t
      // (attachments hold their vertices at prescribed targets instead)
      for (int c = rcn.lo + tid; c < rcn.hi; c += blockDim.x)
        if (con_stick(d, c) && !con_is_att(d, c)) {
          const int v = d.con_v[c];
          d.gq[3 * (size_t)v] += cb_nu(d)[3 * c];
          d.gq[3 * (size_t)v + 1] += cb_nu(d)[3 * c + 1];
        }
      if (!(ok = grid_sync(d, tm))) break;
    }
  }
  if (ok) {
    double p4[4] = {0.0, 0.0, 0.0, 0.0};
    const double am = S.acc_mu, al = S.acc_lam, ak = S.acc_k;
    for (int e = re.lo + tid; e < re.hi; e += blockDim.x) chain_item(d, e, a.dE, am, al, ak, p4);
    ok = grid_reduce<4>(d, tm, p4, sums);
    if (ok && writer && tid == 0) {
      const double v = chain_nu(d, am, al, ak, sums);
      if (a.dnu) *a.dnu = v;
      d.ctrl->dnu_acc = v;
    }
    for (int i = rv.lo + tid; i < rv.hi; i += blockDim.x)
      for (int c = 0; c < 3; ++c) {
        if (a.dq0) a.dq0[3 * (size_t)i + c] = d.gq[3 * (size_t)i + c];
        if (a.dv0) a.dv0[3 * (size_t)i + c] = d.gv[3 * (size_t)i + c];
      }
  }
  if (writer && tid == 0) {
    Ctrl* c = d.ctrl;
    c->adj_iters_total = S.adj_iters_total;
    c->adj_iters_max = S.adj_iters_max;
    c->adj_not_converged = S.adj_not_converged;
    c->acc_mu = S.acc_mu;
    c->acc_lam = S.acc_lam;
    c->acc_k = S.acc_k;
    c->elapsed_ns[1] = gtimer() - tstart;
    c->con_iters += S.con_cg;
    c->con_unconverged += S.con_cg_unconverged;
    atomicOr(&c->status, S.status);
  }
}

// team[blockIdx.x] = {instance, block index in its team, team size, 0}
template <typename T>
__global__ void __launch_bounds__(kBwdBlock, kBwdMinBlocks) k_bwd_rollout(const Dev* __restrict__ devs, const int4* __restrict__ team,
                                                                const InstOff* __restrict__ off, BatchBwd br) {
  __shared__ Dev sd;
  __shared__ BwdArgs sa;
  const int4 tb = team[blockIdx.x];
  if (threadIdx.x == 0) {
    sd = devs[tb.x];
    const long long v3 = 3 * off[tb.x].v;
    BwdArgs a;
    a.T = br.T;
    a.dqT = br.dqT + v3;
    a.dvT = br.dvT ? br.dvT + v3 : nullptr;
    a.dq0 = br.dq0 ? br.dq0 + v3 : nullptr;
    a.dv0 = br.dv0 ? br.dv0 + v3 : nullptr;
    a.dE = br.dE ? br.dE + off[tb.x].e : nullptr;
    a.dnu = br.dnu ? br.dnu + tb.x : nullptr;
    a.df = br.df ? br.df + v3 : nullptr;
    a.df_stride = br.df_stride;
    a.ckpt = sd.ckpt;
    sa = a;
    team_red_count() = 0;
  }
  __syncthreads();
  bwd_rollout_body<T>(sd, sa, Team{tb.y, tb.z});
}

// ------------------------------------------------------------ wrappers

static inline int nblk(int n, int b) { return (n + b - 1) / b; }

void launch_bwd_begin(const Dev& d, cudaStream_t s, const double* dqT, const double* dvT) {
  const int n = d.n_v > d.n_e ? d.n_v : d.n_e;
  k_bwd_begin<<<nblk(n, kVtxBlock), kVtxBlock, 0, s>>>(d, dqT, dvT);
}

void launch_bwd_setup(const Dev& d, cudaStream_t s, const double* qstar, const double* tau_t) {
  if (d.local_fp32)
    k_bwd_setup<float><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, qstar, tau_t);
  else
    k_bwd_setup<double><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, qstar, tau_t);
}

void launch_bwd_init(const Dev& d, cudaStream_t s) {
  k_bwd_init<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  launch_apply_inverse(d, s, d.bperm, d.y, d.s_part, d.s_cnt, d.z, 0);
  k_pcg_init_z<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
}

void launch_pcg_iteration(const Dev& d, cudaStream_t s) {
  if (d.local_fp32) {
    k_kapply<float><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.pdir);
    k_pcg_w<float><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  } else {
    k_kapply<double><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.pdir);
    k_pcg_w<double><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  }
  k_pcg_r<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  launch_apply_inverse(d, s, d.bperm, d.y, d.s_part, d.s_cnt, d.z, 2);
  k_pcg_z<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  k_pcg_p<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
}

void launch_route(const Dev& d, cudaStream_t s, const double* qstar, const double* qt, const double* tau_t,
                  double* df_out, int df_acc) {
  k_route<<<nblk(d.n_v + d.n_e, kVtxBlock), kVtxBlock, 0, s>>>(d, qstar, qt, tau_t, df_out, df_acc);
}

void launch_chain(const Dev& d, cudaStream_t s, double* dE, double* dnu) {
  k_chain<<<nblk(d.n_e, kVtxBlock), kVtxBlock, 0, s>>>(d, dE, dnu);
}

void launch_bwd_finish(const Dev& d, cudaStream_t s, double* dq0, double* dv0) {
  k_bwd_finish<<<nblk(3 * d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, dq0, dv0);
}

static const void* bwd_fn(bool fp32) {
  return fp32 ? (const void*)k_bwd_rollout<float> : (const void*)k_bwd_rollout<double>;
}

int persistent_grid_bwd(bool fp32, int blocks_per_sm) {
  int sms = 0;
  const int per = coop_blocks_per_sm(bwd_fn(fp32), kBwdBlock, &sms);
  if (per < 1) return 0;
  return sms * (blocks_per_sm >= 1 && blocks_per_sm < per ? blocks_per_sm : per);
}

cudaError_t launch_bwd_rollout(bool fp32, const Dev* devs, const int4* team, const InstOff* off, const BatchBwd& br,
                               int grid, bool tstage, cudaStream_t s) {
  const size_t sm = tstage ? kTStageBytes : 0;
  if (fp32) return coop_launch(k_bwd_rollout<float>, grid, kBwdBlock, sm, s, devs, team, off, br);
  return coop_launch(k_bwd_rollout<double>, grid, kBwdBlock, sm, s, devs, team, off, br);
}

}  // namespace pdk
