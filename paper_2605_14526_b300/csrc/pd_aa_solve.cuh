// The small solve of type-II Anderson acceleration (Sec. 4.2, eq. aa_gamma):
// the regularised normal equations of the least-squares problem on the
// difference columns, for one thread. Kept apart from the phase code so that
// the same source also builds as host C++ for the CPU tests.
#pragma once
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pdk {

// (G + reg I) gamma = rhs for NC columns, reg = max(1e-6 tr(G) / NC, 1e-12),
// by mixed-precision iterative refinement (Wilkinson; Moler 1967): an FP32
// Cholesky factor of the trace-normalised matrix and three passes with FP64
// residuals. Sizes are compile-time, so every array lives in registers
// (one thread runs this; a dependent chain through local memory, or an FP64
// factorisation at this part's FP64 rate, costs several microseconds).
// Returns false on a non-positive pivot; gn = ||gamma||^2.
template <int NC>
__device__ __forceinline__ bool aa_solve(const double* G, const double* rhs, double* gam, double& gn) {
  static_assert(NC >= 1 && NC <= kMaxAA, "window");
  double tr = 0.0;
#pragma unroll
  for (int j = 0; j < NC; ++j) tr += G[j * kMaxAA + j];
  const double reg = fmax(1e-6 * tr * (1.0 / NC), 1e-12);
  const float sc = 1.0f / (float)(tr + NC * reg);
  float L[NC][NC], ipiv[NC];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    float t = (float)(G[j * kMaxAA + j] + reg) * sc;
#pragma unroll
    for (int k = 0; k < j; ++k) t -= L[j][k] * L[j][k];
    ok = ok && t > 0.0f;
    const float r = sqrtf(fmaxf(t, 1e-30f));
    ipiv[j] = 1.0f / r;
#pragma unroll
    for (int i = j + 1; i < NC; ++i) {
      float u = (float)G[i * kMaxAA + j] * sc;
#pragma unroll
      for (int k = 0; k < j; ++k) u -= L[i][k] * L[j][k];
      L[i][j] = u * ipiv[j];
    }
    L[j][j] = r;
  }
  double g[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) g[i] = 0.0;
  if (!ok) return false;
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    double res[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {   // residual in FP64 (rows independent)
      double r = rhs[i] - reg * g[i];
#pragma unroll
      for (int j = 0; j < NC; ++j) r -= G[i * kMaxAA + j] * g[j];
      res[i] = r;
    }
    float y[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {   // forward solve in FP32
      float u = (float)res[i] * sc;
#pragma unroll
      for (int k = 0; k < i; ++k) u -= L[i][k] * y[k];
      y[i] = u * ipiv[i];
    }
#pragma unroll
    for (int i = NC - 1; i >= 0; --i) {   // backward solve
      float u = y[i];
#pragma unroll
      for (int k = i + 1; k < NC; ++k) u -= L[k][i] * y[k];
      y[i] = u * ipiv[i];
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) g[i] += (double)y[i];
  }
  gn = 0.0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    gn += g[i] * g[i];
    gam[i] = g[i];
  }
  return true;
}

// the same solve for a window size known only at run time (NC > 5: unrolled
// copies of those sizes would not fit the persistent kernels' registers)
__device__ __forceinline__ bool aa_solve_any(int nc, const double* G, const double* rhs, double* gam, double& gn) {
  double tr = 0.0;
  for (int j = 0; j < nc; ++j) tr += G[j * kMaxAA + j];
  const double reg = fmax(1e-6 * tr / nc, 1e-12);
  const float sc = 1.0f / (float)(tr + nc * reg);
  float L[kMaxAA * kMaxAA], ipiv[kMaxAA];
  for (int j = 0; j < nc; ++j) {
    float t = (float)(G[j * kMaxAA + j] + reg) * sc;
    for (int k = 0; k < j; ++k) t -= L[j * kMaxAA + k] * L[j * kMaxAA + k];
    if (!(t > 0.0f)) return false;
    const float r = sqrtf(t);
    ipiv[j] = 1.0f / r;
    for (int i = j + 1; i < nc; ++i) {
      float u = (float)G[i * kMaxAA + j] * sc;
      for (int k = 0; k < j; ++k) u -= L[i * kMaxAA + k] * L[j * kMaxAA + k];
      L[i * kMaxAA + j] = u * ipiv[j];
    }
    L[j * kMaxAA + j] = r;
  }
  for (int i = 0; i < nc; ++i) gam[i] = 0.0;
  for (int pass = 0; pass < 3; ++pass) {
    float y[kMaxAA];
    for (int i = 0; i < nc; ++i) {
      double r = rhs[i] - reg * gam[i];
      for (int j = 0; j < nc; ++j) r -= G[i * kMaxAA + j] * gam[j];
      float u = (float)r * sc;
      for (int k = 0; k < i; ++k) u -= L[i * kMaxAA + k] * y[k];
      y[i] = u * ipiv[i];
    }
    for (int i = nc - 1; i >= 0; --i) {
      float u = y[i];
      for (int k = i + 1; k < nc; ++k) u -= L[k * kMaxAA + i] * y[k];
      y[i] = u * ipiv[i];
    }
    for (int i = 0; i < nc; ++i) gam[i] += (double)y[i];
  }
  gn = 0.0;
  for (int i = 0; i < nc; ++i) gn += gam[i] * gam[i];
  return true;
}

}  // namespace pdk
