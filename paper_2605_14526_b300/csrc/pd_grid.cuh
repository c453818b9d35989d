// Grid-wide synchronisation of the persistent kernels (cooperative launch).
// Barrier: acq_rel arrival counter + release/acquire generation word; every
// wait is bounded (status bit 4 on timeout, the caller returns). Reduction
// barrier: the last block to arrive adds the per-block partials in a fixed
// order and publishes the sums to every block (deterministic).
#pragma once
#include "pd_common.cuh"

namespace pdk {

constexpr unsigned int kSpinLimit = 1u << 22;   // polls (~0.4 us each with the sleep): ~2 s per wait at most
constexpr int kStatusTimeout = 4;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The blocks of a persistent launch form teams: team-local block index `b`
// of `nb` blocks; one team works on one problem instance (the whole grid in
// a single-instance launch). Barriers and reductions span one team.
struct Team {
  int b, nb;
};

// Team barrier; with NV > 0 also a sum over the team's blocks of NV partial
// values per block, returned in `sums` (shared) to every block. Returns false
// in every thread of the block if the wait timed out. A one-block team needs
// no global memory traffic at all.
template <int NV>
__device__ __forceinline__ bool grid_reduce(const Dev& d, Team tm, double (&part)[NV > 0 ? NV : 1], double* sums) {
  __shared__ int s_last, s_fail;
  __shared__ unsigned long long s_tarr;
  if (tm.nb == 1) {
    if constexpr (NV > 0) block_reduce_to<NV>(part, sums);
    else __syncthreads();
    return true;
  }
  if constexpr (NV > 0) block_reduce_store<NV>(part, d.red, tm.b);
  __syncthreads();
  Ctrl* c = d.ctrl;
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(&c->bar_gen);
    const unsigned int arrived = atom_add_acq_rel(&c->bar_count, 1u);
    s_last = arrived == (unsigned int)tm.nb - 1;
    if (d.prof && s_last) s_tarr = gtimer();
    s_fail = 0;
    if (!s_last) {
      unsigned int it = 0;
      while (ld_acquire(&c->bar_gen) == g) {
        if (++it > kSpinLimit) {
          atomicOr(&c->status, kStatusTimeout);
          s_fail = 1;
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
  double* pub = d.red + (size_t)(kRedRows - 1) * kRed;   // published sums
  if (s_last) {
    if constexpr (NV > 0) {
      // thread t adds the partials of blocks t, t + blockDim.x, ... (all NV
      // values of a block loaded at once, independent loads), then a fixed
      // shuffle/shared-memory tree: deterministic, ~2 L2 round trips
      double acc[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] = 0.0;
#pragma unroll 4
      for (int b = threadIdx.x; b < tm.nb; b += blockDim.x) {
        double v[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldcg(&d.red[(size_t)b * kRed + j]);
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += v[j];
      }
      block_reduce_to<NV>(acc, sums);
      if (threadIdx.x < NV) pub[threadIdx.x] = sums[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (d.prof) c->t_last = s_tarr;
      st_relaxed(&c->bar_count, 0u);
      red_release(&c->bar_gen, 1u);
    }
  } else if constexpr (NV > 0) {
    if (threadIdx.x < NV) sums[threadIdx.x] = __ldcg(&pub[threadIdx.x]);
  }
  __syncthreads();
  return !s_fail;
}

__device__ __forceinline__ bool grid_sync(const Dev& d, Team tm) {
  double none[1] = {0.0};
  return grid_reduce<0>(d, tm, none, nullptr);
}

// contiguous range of n items owned by this block of the team
struct Range {
  int lo, hi;
};
__device__ __forceinline__ Range block_range(Team tm, int n) {
  const int chunk = (n + tm.nb - 1) / tm.nb;
  const int lo = min(n, tm.b * chunk);
  return {lo, min(n, lo + chunk)};
}

}  // namespace pdk
