// Learned warm start, device side: per-vertex features and the 7 -> 128 ->
// 128 -> 128 -> 3 ReLU network, evaluated on the tensor pipe for 16
// vertices per warp (warm_tile, below), or by one warp per vertex on the
// FP32 pipe (each lane owns 4 of the 128 hidden units; inputs are broadcast
// by shuffles; BF16 weights read as 8-byte rows of 4). The step then starts
// from q0 = 2 x_t - x_{t-1} + oscale * net((f - fmean) / fscale) instead of
// q_t (Alg. 1); the network is not part of the paper's method.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pd_df.cuh"
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

// ------------------------------------------------------------ tensor cores
//
// The same network on the tensor pipe: a warp evaluates 16 vertices at once
// with mma.sync m16n8k16 (BF16 x BF16, FP32 accumulation). Weights are the
// BF16 values (fragment-packed, MlpDev::wf); each FP32 activation enters as
// the sum of three BF16 values hi + mid + lo (x - hi and the next remainder
// are exact in FP32), so the products are those of the FP32 activations
// with the BF16 weights, as in the one-warp-per-vertex form above. Between
// layers the accumulators stay in registers: the C fragments of n-tiles 2j
// and 2j + 1 are the A fragment of k-step j of the next layer.

__device__ __forceinline__ uint32_t bf16_rn_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}

// (x0, x1) -> three packed BF16 pairs with x_i = hi_i + mid_i + lo_i
__device__ __forceinline__ void split3_pair(float x0, float x1, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  const uint32_t h0 = bf16_rn_bits(x0), h1 = bf16_rn_bits(x1);
  const float r0 = x0 - __uint_as_float(h0 << 16), r1 = x1 - __uint_as_float(h1 << 16);
  const uint32_t m0 = bf16_rn_bits(r0), m1 = bf16_rn_bits(r1);
  const float s0 = r0 - __uint_as_float(m0 << 16), s1 = r1 - __uint_as_float(m1 << 16);
  hi = h0 | (h1 << 16);
  mid = m0 | (m1 << 16);
  lo = bf16_rn_bits(s0) | (bf16_rn_bits(s1) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// acc[nt] += A (one k-step, given as its FP32 pairs p[0..3]) x W (n-tiles
// 0..NT-1 of that k-step), lo, mid and hi parts in that order
template <int NT>
__device__ __forceinline__ void mma_kstep(float (&acc)[NT][4], const float (&p)[8], const uint2* wf_ks, int lane) {
  uint32_t ah[4], am[4], al[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split3_pair(p[2 * i], p[2 * i + 1], ah[i], am[i], al[i]);
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const uint2 b = __ldg(wf_ks + nt * 32 + lane);
    mma_bf16_16816(acc[nt], al, b);
    mma_bf16_16816(acc[nt], am, b);
    mma_bf16_16816(acc[nt], ah, b);
  }
}

// one hidden layer on the warp's 16 rows: h <- relu(b + h W), 128 -> 128
__device__ __forceinline__ void mma_hidden(const uint2* wf, const float* b, float (&h)[16][4], int lane) {
  const int t = lane & 3;
  float acc[16][4];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const float2 bb = *reinterpret_cast<const float2*>(b + 8 * nt + 2 * t);
    acc[nt][0] = acc[nt][2] = bb.x;
    acc[nt][1] = acc[nt][3] = bb.y;
  }
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
    const float p[8] = {h[2 * ks][0], h[2 * ks][1], h[2 * ks][2], h[2 * ks][3],
                        h[2 * ks + 1][0], h[2 * ks + 1][1], h[2 * ks + 1][2], h[2 * ks + 1][3]};
    mma_kstep<16>(acc, p, wf + ks * 16 * 32, lane);
  }
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) h[nt][i] = fmaxf(acc[nt][i], 0.f);
}

// network outputs (normalised units) of 16 rows of normalised features:
// lane r < 16 passes its row's features f[7] and gets its row's y[3]
__device__ __forceinline__ void mlp_eval_tile(const MlpDev& m, const float* f, float* y, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const uint2* wf1 = m.wf;
  const uint2* wf2 = wf1 + kMlpFrag1;
  const uint2* wf3 = wf2 + kMlpFragH;
  const uint2* wf4 = wf3 + kMlpFragH;
  const float* b1 = m.b;
  const float* b2 = b1 + kMlpH;
  const float* b3 = b2 + kMlpH;
  const float* b4 = b3 + kMlpH;
  // layer 1: the features in A-fragment order (rows g, g + 8; columns 2t,
  // 2t + 1; columns 7 .. 15 are zero padding)
  float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < kMlpIn; ++c) {
    const float vg = __shfl_sync(0xffffffffu, f[c], g);
    const float vg8 = __shfl_sync(0xffffffffu, f[c], g + 8);
    if (c == 2 * t) {
      p[0] = vg;
      p[2] = vg8;
    }
    if (c == 2 * t + 1) {
      p[1] = vg;
      p[3] = vg8;
    }
  }
  float h[16][4];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const float2 bb = *reinterpret_cast<const float2*>(b1 + 8 * nt + 2 * t);
    h[nt][0] = h[nt][2] = bb.x;
    h[nt][1] = h[nt][3] = bb.y;
  }
  mma_kstep<16>(h, p, wf1, lane);
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) h[nt][i] = fmaxf(h[nt][i], 0.f);
  mma_hidden(wf2, b2, h, lane);
  mma_hidden(wf3, b3, h, lane);
  // output layer: one n-tile (columns 0..2 used)
  float o[1][4];
  o[0][0] = o[0][2] = 2 * t < kMlpOut ? b4[2 * t] : 0.f;
  o[0][1] = o[0][3] = 2 * t + 1 < kMlpOut ? b4[2 * t + 1] : 0.f;
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
    const float q[8] = {h[2 * ks][0], h[2 * ks][1], h[2 * ks][2], h[2 * ks][3],
                        h[2 * ks + 1][0], h[2 * ks + 1][1], h[2 * ks + 1][2], h[2 * ks + 1][3]};
    mma_kstep<1>(o, q, wf4 + ks * 32, lane);
  }
  // row r's outputs: columns 0, 1 at lane 4 (r mod 8), column 2 at the next
  // lane; rows 8..15 in the fragment's lower half
  const int src = 4 * (lane & 7);
  const float y00 = __shfl_sync(0xffffffffu, o[0][0], src), y01 = __shfl_sync(0xffffffffu, o[0][1], src);
  const float y02 = __shfl_sync(0xffffffffu, o[0][0], src + 1);
  const float y10 = __shfl_sync(0xffffffffu, o[0][2], src), y11 = __shfl_sync(0xffffffffu, o[0][3], src);
  const float y12 = __shfl_sync(0xffffffffu, o[0][2], src + 1);
  const bool upper = (lane & 15) < 8;
  y[0] = upper ? y00 : y10;
  y[1] = upper ? y01 : y11;
  y[2] = upper ? y02 : y12;
}

// Warm start of the 16 vertices v0 .. v0 + 15 (the whole warp; lane r < 16
// owns vertex v0 + r): q0 = 2 x_t - x_{t-1} + r as in warm_vertex, the
// network on the tensor pipe.
__device__ __forceinline__ void warm_tile(const Dev& d, int v0, const double* xt, const double* xtm1, const double* vt,
                                          double* out1, double* out2, int lane, float2* out1_hl = nullptr) {
  const int v = v0 + (lane & 15);
  const bool mine = lane < 16 && v < d.n_v && !d.pinned[v];
  double x[3] = {0.0, 0.0, 0.0}, xm[3] = {0.0, 0.0, 0.0};
  float f[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) f[i] = 0.f;
  if (mine) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = xt[3 * (size_t)v + i];
      xm[i] = xtm1 ? xtm1[3 * (size_t)v + i] : x[i] - d.h * vt[3 * (size_t)v + i];
      f[i] = (float)(((x[i] - xm[i]) - (double)d.mlp.fmean[i]) / (double)d.mlp.fscale[i]);
      f[3 + i] = (float)(((x[i] - d.X[3 * (size_t)v + i]) - (double)d.mlp.fmean[3 + i]) / (double)d.mlp.fscale[3 + i]);
    }
    f[6] = (d.logE[v] - d.mlp.fmean[6]) / d.mlp.fscale[6];
  }
  float y[3];
  mlp_eval_tile(d.mlp, f, y, lane);
  if (!mine) return;
  float r[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) r[i] = y[i] * d.mlp.oscale[i];
  const bool ok = isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double q0 = ok ? 2.0 * x[i] - xm[i] + (double)r[i] : x[i];
    out1[3 * (size_t)v + i] = q0;
    if (out1_hl) out1_hl[3 * (size_t)v + i] = df_split(q0);
    if (out2) out2[3 * (size_t)v + i] = q0;
  }
}

// Warm start of vertex v (the whole warp): q0 = 2 x_t - x_{t-1} + r with
// x_{t-1} = xtm1 if given, else x_t - h v_t; r from the network (warm = 1)
// or 0 (warm = 2, constant-velocity extrapolation). A non-finite network
// output leaves the vertex at x_t. Pinned vertices are not written.
__device__ __forceinline__ void warm_vertex(const Dev& d, int v, const double* xt, const double* xtm1, const double* vt,
                                            double* out1, double* out2, int lane, float2* out1_hl = nullptr) {
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
      if (out1_hl) out1_hl[3 * (size_t)v + i] = df_split(q0);
      if (out2) out2[3 * (size_t)v + i] = q0;
    }
}

}  // namespace pdk
