// Learned warm start, device side: per-vertex features and the 7 -> 128 ->
// 128 -> 128 -> 3 ReLU network evaluated by one warp per vertex (each lane
// owns 4 of the 128 hidden units; inputs are broadcast by shuffles; BF16
// weights read as 8-byte rows of 4, FP32 arithmetic). The step then starts
// from q0 = 2 x_t - x_{t-1} + oscale * net((f - fmean) / fscale) instead of
// q_t (Alg. 1); the network is not part of the paper's method.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pd_internal.h"

namespace pdk {

__device__ __forceinline__ void bf16x4(const uint16_t* p, float* w) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  w[0] = __uint_as_float(v.x << 16);
  w[1] = __uint_as_float(v.x & 0xffff0000u);
  w[2] = __uint_as_float(v.y << 16);
  w[3] = __uint_as_float(v.y & 0xffff0000u);
}

// one hidden layer: g = relu(b + W^T h) with the 128 inputs spread over the
// warp (lane l holds inputs 4l .. 4l+3) and outputs 4 lane .. 4 lane + 3
__device__ __forceinline__ void mlp_hidden(const uint16_t* Wt, const float* b, float* h, int lane) {
  const float4 bb = *reinterpret_cast<const float4*>(b + 4 * lane);
  float g[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll 4
  for (int kk = 0; kk < 32; ++kk) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float x = __shfl_sync(0xffffffffu, h[c], kk);
      float w[4];
      bf16x4(Wt + (size_t)(4 * kk + c) * kMlpH + 4 * lane, w);
#pragma unroll
      for (int o = 0; o < 4; ++o) g[o] = fmaf(w[o], x, g[o]);
    }
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) h[o] = fmaxf(g[o], 0.f);
}

// network output (normalised units) for normalised features f[7], the same
// on every lane of the warp
__device__ __forceinline__ void mlp_eval_warp(const MlpDev& m, const float* f, float* out, int lane) {
  const uint16_t* W1 = m.w;
  const uint16_t* W2 = W1 + kMlpIn * kMlpH;
  const uint16_t* W3 = W2 + kMlpH * kMlpH;
  const uint16_t* W4 = W3 + kMlpH * kMlpH;
  const float* b1 = m.b;
  const float* b2 = b1 + kMlpH;
  const float* b3 = b2 + kMlpH;
  const float* b4 = b3 + kMlpH;
  const float4 bb = *reinterpret_cast<const float4*>(b1 + 4 * lane);
  float h[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) {
    float w[4];
    bf16x4(W1 + k * kMlpH + 4 * lane, w);
#pragma unroll
    for (int o = 0; o < 4; ++o) h[o] = fmaf(w[o], f[k], h[o]);
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) h[o] = fmaxf(h[o], 0.f);
  mlp_hidden(W2, b2, h, lane);
  mlp_hidden(W3, b3, h, lane);
  // output layer: lane partial sums over its 4 inputs, then a fixed tree to
  // lane 0, broadcast (every lane returns lane 0's bits)
  float w4[12];
  bf16x4(W4 + 12 * lane, w4);
  bf16x4(W4 + 12 * lane + 4, w4 + 4);
  bf16x4(W4 + 12 * lane + 8, w4 + 8);
  float p[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) p[o] = h[0] * w4[o] + h[1] * w4[3 + o] + h[2] * w4[6 + o] + h[3] * w4[9 + o];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1)
#pragma unroll
    for (int o = 0; o < 3; ++o) p[o] += __shfl_down_sync(0xffffffffu, p[o], s);
#pragma unroll
  for (int o = 0; o < 3; ++o) out[o] = __shfl_sync(0xffffffffu, p[o], 0) + b4[o];
}

// Warm start of vertex v (the whole warp): q0 = 2 x_t - x_{t-1} + r with
// x_{t-1} = xtm1 if given, else x_t - h v_t; r from the network (warm = 1)
// or 0 (warm = 2, constant-velocity extrapolation). A non-finite network
// output leaves the vertex at x_t. Pinned vertices are not written.
__device__ __forceinline__ void warm_vertex(const Dev& d, int v, const double* xt, const double* xtm1, const double* vt,
                                            double* out1, double* out2, int lane) {
  if (d.pinned[v]) return;
  double x[3], xm[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    x[i] = xt[3 * (size_t)v + i];
    xm[i] = xtm1 ? xtm1[3 * (size_t)v + i] : x[i] - d.h * vt[3 * (size_t)v + i];
  }
  float r[3] = {0.f, 0.f, 0.f};
  if (d.warm == 1) {
    float f[kMlpIn];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f[i] = (float)(((x[i] - xm[i]) - (double)d.mlp.fmean[i]) / (double)d.mlp.fscale[i]);
      f[3 + i] = (float)(((x[i] - d.X[3 * (size_t)v + i]) - (double)d.mlp.fmean[3 + i]) / (double)d.mlp.fscale[3 + i]);
    }
    f[6] = (d.logE[v] - d.mlp.fmean[6]) / d.mlp.fscale[6];
    float y[3];
    mlp_eval_warp(d.mlp, f, y, lane);
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = y[i] * d.mlp.oscale[i];
  }
  const bool ok = isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (lane == i) {
      const double q0 = ok ? 2.0 * x[i] - xm[i] + (double)r[i] : x[i];
      out1[3 * (size_t)v + i] = q0;
      if (out2) out2[3 * (size_t)v + i] = q0;
    }
}

}  // namespace pdk
