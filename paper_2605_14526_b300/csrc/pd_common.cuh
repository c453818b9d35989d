// Device helpers shared by the forward and backward kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pd_internal.h"
#include "pd_math.cuh"

namespace pdk {

// ------------------------------------------------------------ models

// the log-volume barrier's prox (eq. pd_log_volume) divided by its weight
// lambda_e, as the stretch prox of pd_math.cuh: mu = r, lam = k = 1, no
// deviatoric term
template <typename T>
__device__ __forceinline__ NHMean<T> barrier_prox_energy(const Dev& d) {
  NHMean<T> m{(T)d.bar_r, T(1), T(1)};
  m.dv = T(0);
  return m;
}

// ------------------------------------------------------------ reductions

__host__ __device__ constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }

// Warp sum of v[NV] by recursive halving: at each of the first log2(P)
// levels (P = NV rounded up to a power of two, at most 32) a lane keeps one
// half of its values and adds its partner's copy of that half, so all NV
// sums take P - 1 + 5 - log2(P) shuffles instead of 5 NV. Returns this
// lane's sum, of value index *idx (the same sum in the 32 / P lanes that
// share idx); the order of the additions is fixed.
template <int NV>
__device__ __forceinline__ double warp_sum_scatter(const double (&v)[NV], int lane, int& idx) {
  constexpr int P = pow2_ceil(NV);
  static_assert(P <= 32, "at most 32 values");
  double w[P];
#pragma unroll
  for (int j = 0; j < P; ++j) w[j] = j < NV ? v[j] : 0.0;
  int base = 0;
#pragma unroll
  for (int h = P / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double send = up ? w[k] : w[k + h];
      const double keep = up ? w[k + h] : w[k];
      w[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (up) base += h;
  }
  double x = w[0];
#pragma unroll
  for (int o = 16 / P; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  idx = base;
  return x;
}

// block-wide sum of v[NV] (warp sums in a fixed order, then the warps in
// order) into sh_out[NV] (shared), read by threads < NV. Only threads below
// `nactive` hold values (the others hold zeros): the warps past them skip
// their FP64 shuffle tree and the final sum, which leaves the result
// unchanged (each FP64 instruction costs a scheduler about 64 cycles here)
template <int NV>
__device__ __forceinline__ double block_sum_lane(double (&v)[NV], int nactive = 1 << 30) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = ((nactive < (int)blockDim.x ? nactive : (int)blockDim.x) + 31) >> 5;
  constexpr int P = pow2_ceil(NV);
  if (wid < nw) {
    int idx;
    const double x = warp_sum_scatter<NV>(v, lane, idx);
    if ((lane & (32 / P - 1)) == 0 && idx < NV) sh[wid][idx] = x;
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < NV)
    for (int w = 0; w < nw; ++w) s += sh[w][threadIdx.x];
  return s;
}

// block-wide sum of v[NV] stored to row `row` of the reduction scratch
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* red, int row) {
  const double s = block_sum_lane<NV>(v);
  if (threadIdx.x < NV) red[(size_t)row * kRed + threadIdx.x] = s;
}

// block-wide sum of v[NV] into out[NV] (shared), visible to the whole block
// on return
template <int NV>
__device__ __forceinline__ void block_reduce_to(double (&v)[NV], double* out, int nactive = 1 << 30) {
  const double s = block_sum_lane<NV>(v, nactive);
  if (threadIdx.x < NV) out[threadIdx.x] = s;
  __syncthreads();
}

// returns true in every thread of the last block to finish; its partials
// are then visible. Resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int v = atomicAdd(ticket, 1u);
    is_last = (v == gridDim.x - 1);
    if (is_last) *ticket = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

__device__ __forceinline__ double sum_partials(const double* red, int nblocks, int j) {
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += red[(size_t)b * kRed + j];
  return s;
}

__device__ __forceinline__ bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// ------------------------------------------------------------ local step

template <typename T>
__device__ __forceinline__ void load_elem(const Dev& d, int e, int4& tv, T* Bm, T& coef);

template <>
__device__ __forceinline__ void load_elem<float>(const Dev& d, int e, int4& tv, float* Bm, float& coef) {
  tv = d.tets[e];
#pragma unroll
  for (int i = 0; i < 9; ++i) Bm[i] = d.Bm32[9 * (size_t)e + i];
  coef = d.coef32[e];
}
template <>
__device__ __forceinline__ void load_elem<double>(const Dev& d, int e, int4& tv, double* Bm, double& coef) {
  tv = d.tets[e];
#pragma unroll
  for (int i = 0; i < 9; ++i) Bm[i] = d.Bm64[9 * (size_t)e + i];
  coef = d.coef64[e];
}

// F = sum_{a=1..3} (x_a - x_0) gradN_a^T, differences taken in FP64
template <typename T>
__device__ __forceinline__ void deform(const double* __restrict__ x, int4 tv, const T* Bm, T* F) {
  const int id[4] = {tv.x, tv.y, tv.z, tv.w};
  T D[9];  // D[3*i + a-1] = (x_a - x_0)_i
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) D[3 * i + a - 1] = (T)(x[3 * id[a] + i] - x[3 * id[0] + i]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = D[3 * i] * Bm[j] + D[3 * i + 1] * Bm[3 + j] + D[3 * i + 2] * Bm[6 + j];
}

// F from positions held as float pairs x = hi + lo (the FP32 local step):
// the edge vectors (hi_a - hi_0) + (lo_a - lo_0) on the FP32 pipe. The high
// parts of nearby vertices differ by an exactly representable amount
// (Sterbenz), so each edge vector is the FP64 difference rounded to FP32, as
// in deform(), without FP64 arithmetic in the element loop.
__device__ __forceinline__ void deform_hl(const float2* __restrict__ xhl, int4 tv, const float* Bm, float* F) {
  const int id[4] = {tv.x, tv.y, tv.z, tv.w};
  float2 x0[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) x0[i] = xhl[3 * id[0] + i];
  float D[9];
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float2 xa = xhl[3 * id[a] + i];
      D[3 * i + a - 1] = __fadd_rn(__fsub_rn(xa.x, x0[i].x), __fsub_rn(xa.y, x0[i].y));
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = D[3 * i] * Bm[j] + D[3 * i + 1] * Bm[3 + j] + D[3 * i + 2] * Bm[6 + j];
}

// the same from the four vertex positions already loaded
template <typename T>
__device__ __forceinline__ void deform_x(const double (&xv)[4][3], const T* Bm, T* F) {
  T D[9];
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) D[3 * i + a - 1] = (T)(xv[a][i] - xv[0][i]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = D[3 * i] * Bm[j] + D[3 * i + 1] * Bm[3 + j] + D[3 * i + 2] * Bm[6 + j];
}

// c_a = coef * P gradN_a for a = 1..3, c_0 = -(c_1 + c_2 + c_3)
template <typename T>
__device__ __forceinline__ void corner_forces(const T* P, const T* Bm, T coef, T* out12) {
  T s[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T v = coef * (P[3 * i] * Bm[3 * (a - 1)] + P[3 * i + 1] * Bm[3 * (a - 1) + 1] + P[3 * i + 2] * Bm[3 * (a - 1) + 2]);
      out12[3 * a + i] = v;
      s[i] += v;
    }
#pragma unroll
  for (int i = 0; i < 3; ++i) out12[i] = -s[i];
}

// acc += the corner contributions of vertex v, in incidence order. Indices
// and values are loaded in chunks of 8 before they are added, so the
// dependent index -> value loads of a chunk overlap instead of running one
// incidence at a time (same summation order, same bits).
template <typename T>
__device__ __forceinline__ void gather_contrib(const Dev& d, int v, double* acc) {
  const T* cb = reinterpret_cast<const T*>(d.contrib);
  const int beg = d.inc_ptr[v], end = d.inc_ptr[v + 1];
  for (int p0 = beg; p0 < end; p0 += 8) {
    int ic[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) ic[u] = p0 + u < end ? d.inc_idx[p0 + u] : -1;
    T val[8][3];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < 3; ++i) val[u][i] = ic[u] >= 0 ? cb[3 * (size_t)ic[u] + i] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (ic[u] >= 0)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += (double)val[u][i];
  }
}


}  // namespace pdk
