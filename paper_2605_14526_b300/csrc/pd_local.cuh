// The local step of one element (Alg. 1, Sec. 4.1): its own header so that
// the same source also builds as host C++ for the CPU tests.
#pragma once
#include "pd_common.cuh"

namespace pdk {

// Local step fused with the per-element part of the RHS scatter (Alg. 1,
// eq. nh_prox / corotated projection, eq. A_basic). The prox Newton starts
// from this element's sigma* of its previous local step when one is stored.
// The FP32 step reads the positions as float pairs xhl when given (the
// iterate's copy kept by its writers), else the FP64 positions x.
template <typename T>
__device__ __forceinline__ void local_item(const Dev& d, int e, const double* x, const float2* xhl = nullptr) {
  int4 tv;
  T Bm[9], coef;
  load_elem<T>(d, e, tv, Bm, coef);
  T F[9], U[9], V[9], sF[3], ss[3], P[9], c[12];
  if constexpr (sizeof(T) == 4) {
    if (xhl) deform_hl(xhl, tv, Bm, F);
    else deform<T>(x, tv, Bm, F);
  } else {
    deform<T>(x, tv, Bm, F);
  }
  svd3<T>(F, U, sF, V);
  if (d.model == 0) {
    ss[0] = ss[1] = ss[2] = T(1);
  } else if (d.model == 2) {
    // corotated + volume composite: p = (w_0 R + w_1 p_vol)/(w_0 + w_1) =
    // U diag(a + (1 - a) sigma_v) V^T with a = w_0/(w_0 + w_1)
    T sv[3], nu;
    vol_project<T>(sF, sv, nu);
    const T a = (T)d.rot_share;
#pragma unroll
    for (int i = 0; i < 3; ++i) ss[i] = a + (T(1) - a) * sv[i];
  } else {
    // Neo-Hookean prox (model 1), or the log-volume barrier's prox (model 3,
    // eq. pd_log_volume) mixed with the rotation step like the composite:
    // p = U diag(a + (1 - a) sigma_b) V^T; both warm-start from the
    // element's previous prox stretches
    const bool bar = d.model == 3;
    const NHMean<T> m = bar ? barrier_prox_energy<T>(d) : NHMean<T>{(T)d.mu_bar, (T)d.lam_bar, (T)d.k_bar};
    float* ws = reinterpret_cast<float*>(d.sstar) + 3 * (size_t)e;
    T s0[3];
    const bool warm = ws[0] > 0.f && ws[1] > 0.f && ws[2] > 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) s0[i] = warm ? (T)ws[i] : (sF[i] > T(0.1) ? sF[i] : T(0.1));
    nh_prox_from<T>(sF, m, s0, ss);
#pragma unroll
    for (int i = 0; i < 3; ++i) ws[i] = (float)ss[i];
    if (bar) {
      const T a = (T)d.rot_share;
#pragma unroll
      for (int i = 0; i < 3; ++i) ss[i] = a + (T(1) - a) * ss[i];
    }
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

}  // namespace pdk
