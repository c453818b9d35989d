// Per-element bodies of the adjoint (Sec. 4.3, Sec. 4.7): the record of the
// local step's differential at q* and the matrix-free product K p it gives.
// Their own header so that the same source also builds as host C++ for the
// CPU tests.
#pragma once
#include "pd_local.cuh"

namespace pdk {

// record layout: U[9] V[9] sF[3] ss[3] J[6] (00 11 22 01 02 12) S[3] T[3] (pairs 01 02 12)
enum { R_U = 0, R_V = 9, R_SF = 18, R_SS = 21, R_J = 24, R_S = 30, R_T = 33 };

template <typename T>
__device__ __forceinline__ void bwd_setup_item(const Dev& d, int e, const double* qstar, double tau) {
  int4 tv;
  T Bm[9], coef;
  load_elem<T>(d, e, tv, Bm, coef);
  T F[9], U[9], V[9], sF[3], ss[3];
  deform<T>(qstar, tv, Bm, F);
  svd3<T>(F, U, sF, V);
  T J[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T Sp[3], Tp[3];
  const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
  if (has_prox_hessian(d.model)) {
    // Neo-Hookean prox, or the log-volume barrier's (model 3: sigma* = a +
    // (1 - a) sigma_b, its differential (1 - a) times the barrier prox's)
    const bool bar = d.model == 3;
    const NHMean<T> m = bar ? barrier_prox_energy<T>(d) : NHMean<T>{(T)d.mu_bar, (T)d.lam_bar, (T)d.k_bar};
    nh_prox<T>(sF, m, ss);
    filtered_jacobian<T>(ss, m, (T)tau, J);
    // (s*_i - s*_j)/(s_i - s_j) = k / (k + mu dv + (mu - lam ln J*)/(s*_i s*_j)),
    // exact at the prox stationarity and free of cancellation near s_i = s_j
    const T lnJ = dlog(ss[0] * ss[1] * ss[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) Sp[c] = m.k / (m.k + m.mu * m.dv + (m.mu - m.lam * lnJ) / (ss[pi[c]] * ss[pj[c]]));
    if (bar) {
      const T a = (T)d.rot_share;
#pragma unroll
      for (int i = 0; i < 9; ++i) J[i] *= T(1) - a;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ss[i] = a + (T(1) - a) * ss[i];
        Sp[i] *= T(1) - a;
      }
    }
  } else if (d.model == 2) {
    // composite: sigma* = a + (1 - a) sigma_v; d sigma*/d sigma_F = (1 - a)
    // d sigma_v/d sigma_F (no prox Hessian, nothing to filter); with
    // sigma_F,i = sigma_v,i + nu / sigma_v,i at the volume step's stationarity,
    // (sigma*_i - sigma*_j)/(sigma_F,i - sigma_F,j) = (1 - a)/(1 - nu/(sigma_v,i sigma_v,j))
    // exactly, free of cancellation near sigma_F,i = sigma_F,j
    T sv[3], nu;
    vol_project<T>(sF, sv, nu);
    vol_jacobian<T>(sv, nu, J);
    const T a = (T)d.rot_share;
#pragma unroll
    for (int i = 0; i < 9; ++i) J[i] *= T(1) - a;
#pragma unroll
    for (int i = 0; i < 3; ++i) ss[i] = a + (T(1) - a) * sv[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) Sp[c] = (T(1) - a) / (T(1) - nu / (sv[pi[c]] * sv[pj[c]]));
  } else {
    ss[0] = ss[1] = ss[2] = T(1);
#pragma unroll
    for (int c = 0; c < 3; ++c) Sp[c] = T(0);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T sm = sF[pi[c]] + sF[pj[c]];
    if (dabs(sm) < T(1e-20)) sm = T(1e-20);
    Tp[c] = (ss[pi[c]] + ss[pj[c]]) / sm;
  }
  T* r = reinterpret_cast<T*>(d.jac) + kJacRec * (size_t)e;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    r[R_U + i] = U[i];
    r[R_V + i] = V[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[R_SF + i] = sF[i];
    r[R_SS + i] = ss[i];
    r[R_S + i] = Sp[i];
    r[R_T + i] = Tp[i];
  }
  r[R_J + 0] = J[0]; r[R_J + 1] = J[4]; r[R_J + 2] = J[8];
  r[R_J + 3] = J[1]; r[R_J + 4] = J[2]; r[R_J + 5] = J[5];
}

// the CG direction of this iteration at one coordinate: z + beta p_old
// (p_old = 0, beta = 0 on the first iteration); the element and the vertex
// phases of the persistent adjoint both read it through this function
__device__ __forceinline__ double p_next(const Dev& d, const double* pold, size_t o, double beta) {
  return __fma_rn(beta, pold[o], d.z[o]);
}

// corner contributions of K p for one element: coef * G^T (dp/dF) G p
template <typename T>
__device__ __forceinline__ void kapply_item(const Dev& d, int e, const double* pv, const double* pold = nullptr,
                                            double beta = 0.0) {
  int4 tv;
  T Bm[9], coef;
  load_elem<T>(d, e, tv, Bm, coef);
  const T* r = reinterpret_cast<const T*>(d.jac) + kJacRec * (size_t)e;
  T U[9], V[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    U[i] = r[R_U + i];
    V[i] = r[R_V + i];
  }
  T dF[9];
  if (pold) {   // direction formed on the fly (pinned rows of z and p_old are 0)
    const int id[4] = {tv.x, tv.y, tv.z, tv.w};
    double xv[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) xv[a][i] = p_next(d, pold, 3 * (size_t)id[a] + i, beta);
    deform_x<T>(xv, Bm, dF);
  } else {
    deform<T>(pv, tv, Bm, dF);
  }
  T W[9], Mh[9];  // Mh = U^T dF V
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) W[3 * i + j] = dF[3 * i] * V[j] + dF[3 * i + 1] * V[3 + j] + dF[3 * i + 2] * V[6 + j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Mh[3 * i + j] = U[i] * W[j] + U[3 + i] * W[3 + j] + U[6 + i] * W[6 + j];
  T D[9];
  const T J00 = r[R_J], J11 = r[R_J + 1], J22 = r[R_J + 2], J01 = r[R_J + 3], J02 = r[R_J + 4], J12 = r[R_J + 5];
  D[0] = J00 * Mh[0] + J01 * Mh[4] + J02 * Mh[8];
  D[4] = J01 * Mh[0] + J11 * Mh[4] + J12 * Mh[8];
  D[8] = J02 * Mh[0] + J12 * Mh[4] + J22 * Mh[8];
  const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int i = pi[c], j = pj[c];
    const T sym = T(0.5) * (Mh[3 * i + j] + Mh[3 * j + i]);
    const T skw = T(0.5) * (Mh[3 * i + j] - Mh[3 * j + i]);
    D[3 * i + j] = r[R_S + c] * sym + r[R_T + c] * skw;
    D[3 * j + i] = r[R_S + c] * sym - r[R_T + c] * skw;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) W[3 * i + j] = U[3 * i] * D[j] + U[3 * i + 1] * D[3 + j] + U[3 * i + 2] * D[6 + j];
  T dp[9];  // dp = U D V^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) dp[3 * i + j] = W[3 * i] * V[3 * j] + W[3 * i + 1] * V[3 * j + 1] + W[3 * i + 2] * V[3 * j + 2];
  T c12[12];
  corner_forces<T>(dp, Bm, coef, c12);
  T* out = reinterpret_cast<T*>(d.contrib) + 12 * (size_t)e;
#pragma unroll
  for (int i = 0; i < 12; ++i) out[i] = c12[i];
}

}  // namespace pdk
