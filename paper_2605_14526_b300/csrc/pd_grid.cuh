// Team-wide synchronisation of the persistent kernels (cooperative launch).
// Barrier: a monotonic arrival counter (release RMW per block, acquire
// polling); every wait is bounded (status bit 4 on timeout, the caller
// returns). Reduction: every block stores its partials, passes the barrier
// and adds all the team's partials itself in a fixed order (deterministic,
// the same sums in every block).
#pragma once
#include "pd_common.cuh"

namespace pdk {

constexpr int kStatusTimeout = 4;

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

__device__ __forceinline__ unsigned long long atom_add_release64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Arrival and wait of thread 0 at a team barrier: the arrival counter only
// grows, so arrival number n belongs to the barrier n / nb, which opens when
// the counter reaches (n / nb + 1) nb. Each arrival is a release RMW and the
// wait an acquire load that reads the last of them, so the waiter sees every
// write the team made before arriving. Bounded: status bit 4 on timeout.
__device__ __forceinline__ bool team_arrive_wait(const Dev& d, Team tm) {
  Ctrl* c = d.ctrl;
  const unsigned long long n = atom_add_release64(&c->bar_arrive, 1ull);
  const unsigned long long open = (n / (unsigned long long)tm.nb + 1ull) * (unsigned long long)tm.nb;
  if (d.prof && n + 1 == open) c->t_last = gtimer();   // profiling: the last arrival
  unsigned int it = 0;
  while (ld_acquire64(&c->bar_arrive) < open) {
    if (++it > d.spin_limit) {
      atomicOr(&c->status, kStatusTimeout);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// reduction count of this block (one shared word for every reduction of the
// kernel); thread 0 sets it to 0 at kernel start
__device__ __forceinline__ int& team_red_count() {
  __shared__ int n;
  return n;
}

// Team barrier; with NV > 0 also a sum over the team's blocks of NV partial
// values per block, returned in `sums` (shared) to every block, identical in
// every block (fixed order). Returns false in every thread of the block if a
// wait timed out. A one-block team needs no global memory traffic at all.
// Each block stores its row of partials in kRedRep copies, passes the
// barrier and adds all the team's rows itself (copy b mod kRedRep): no
// second round trip for a published result. Partial rows live in buffer
// `parity`, which alternates between consecutive reductions, so a block
// already at the next reduction cannot overwrite rows that a slower block is
// still reading.

// Every block adds all the team's rows itself: thread t < NV holds the
// block's value t in v on entry (NV = 0: a plain barrier).
template <int NV>
__device__ __forceinline__ bool grid_reduce_all_v(const Dev& d, Team tm, double v, double* sums) {
  static_assert(NV <= kRedTeam, "values per team reduction");
  __shared__ int s_fail;
  int& s_parity = team_red_count();
  if (tm.nb == 1) {
    if (NV > 0 && threadIdx.x < NV) sums[threadIdx.x] = v;
    __syncthreads();
    return true;
  }
  const int par = s_parity & 1;
  if (NV > 0 && threadIdx.x < NV)
#pragma unroll
    for (int r = 0; r < kRedRep; ++r)
      d.red[((size_t)(par * kRedRep + r) * kRedRows + tm.b) * kRedTeam + threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_fail = team_arrive_wait(d, tm) ? 0 : 1;
    if (NV > 0) s_parity += 1;   // every thread read `par` before the __syncthreads above
  }
  __syncthreads();
  if constexpr (NV > 0) {
    const double* rows = d.red + (size_t)(par * kRedRep + tm.b % kRedRep) * kRedRows * kRedTeam;
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.0;
#pragma unroll 2
    for (int b = threadIdx.x; b < tm.nb; b += blockDim.x) {
      double w[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) w[j] = __ldcg(&rows[(size_t)b * kRedTeam + j]);
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] += w[j];
    }
    block_reduce_to<NV>(acc, sums, tm.nb);   // threads >= tm.nb hold no row
  }
  return !s_fail;
}

template <int NV>
__device__ __forceinline__ bool grid_reduce(const Dev& d, Team tm, double (&part)[NV > 0 ? NV : 1], double* sums) {
  static_assert(NV <= kRedTeam, "values per team reduction");
  if constexpr (NV > 0) {
    return grid_reduce_all_v<NV>(d, tm, block_sum_lane<NV>(part), sums);
  } else {
    return grid_reduce_all_v<0>(d, tm, 0.0, sums);
  }
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
