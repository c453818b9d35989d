// Solve mode T: A^-1 b by the two level-scheduled sweeps over the
// partitioned inverse of the supernodal factor (tsolve.h): the forward sweep
// L y = P b from the leaves of the node tree up, the backward sweep
// L^T x = y from the root down, one pass per height of the node tree, FP64.
//
// Node s of height h, columns [c0, c0 + nc), nb rows below:
//   forward   r = b_s - (children's updates at the node's columns)
//             [y_s; U_s] = [Linv_s; M_s] r + [0; children's updates below]
//   backward  x_s = [Linv_s^T, M_s^T] [y_s; -x_below]
// A node of more than kWarpNodeCols columns is cut into work units that the
// blocks of the team take round-robin (the forward: kUnitRows rows of
// [Linv; M], one warp per row with the lanes along it, r staged in shared
// memory; the backward: kUnitCols columns, one warp per column with the lanes
// down it, the right-hand side staged in shared memory in chunks). A smaller
// node is one warp's work (the forward: a lane per row, walking the
// column-major copy; the backward: a lane per column, walking the row-major
// copy). All reads of the stored entries are contiguous across the lanes.
//
// Work units are assigned to blocks (and warp nodes to warps) by index, so a
// given launch shape always sums in the same order: results are
// deterministic. Callers separate consecutive heights by a team barrier (or
// a kernel boundary).
#pragma once
#include "pd_common.cuh"
#include "pd_grid.cuh"

namespace pdk {

constexpr int kTStage = 1024;      // entries of the shared staging vector (3 doubles each); = largest node
                                   // (the host's kNodeMaxCols and kStageRows)

__device__ __forceinline__ int64_t t_rowoff(int nc, int o) {   // row o of the packed row-major copy
  return o < nc ? (int64_t)o * (o + 1) / 2 : (int64_t)nc * (nc + 1) / 2 + (int64_t)(o - nc) * nc;
}
__device__ __forceinline__ int64_t t_coloff(int nc, int nb, int k) {   // column k of the column-major copy
  return (int64_t)k * (nc + nb) - (int64_t)k * (k - 1) / 2;
}

// sum of the children's updates that feed position g (global position index)
__device__ __forceinline__ void t_gather(const Dev& d, int64_t g, double& a0, double& a1, double& a2) {
  a0 = a1 = a2 = 0.0;
  const int p1 = d.t_gptr[g + 1];
  for (int p = d.t_gptr[g]; p < p1; ++p) {
    const double* u = d.t_U + 3 * (size_t)d.t_gsrc[p];
    a0 += u[0];
    a1 += u[1];
    a2 += u[2];
  }
}

// the shared staging vector of both sweeps (one per block; a function-scope
// shared array is a single object per kernel)
// the staging vector lives in dynamic shared memory, which only launches
// that may run mode T request (kTStageBytes): a mode-S launch keeps the L1
// share of the SM's unified L1 / shared memory for its gathers
__device__ __forceinline__ double* t_stage() {
  extern __shared__ double t_stage_dyn[];
  return t_stage_dyn;
}

__device__ __forceinline__ double t_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// forward sweep, nodes of height h: b (elimination order, [n_f][3]) -> y
// (elimination order), U
static __device__ __noinline__ void tsweep_fwd(const Dev& d, const double* b, double* y, int h, int blk, int nblk, int gwarp,
                                              int nwarps) {
  double* sr = t_stage();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, bwarps = blockDim.x >> 5;
  for (int u = d.t_lev_f[h] + blk; u < d.t_lev_f[h + 1]; u += nblk) {
    const int4 un = d.t_unit_f[u];
    const int s = un.x, row0 = un.y, rows = un.z;
    const int c0 = d.t_c0[s], nc = d.t_nc[s];
    const int64_t g0 = d.t_goff[s];
    __syncthreads();   // the previous unit's rows are done with sr
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      double a0, a1, a2;
      t_gather(d, g0 + k, a0, a1, a2);
      const double* bk = b + 3 * (size_t)(c0 + k);
      sr[3 * k] = bk[0] - a0;
      sr[3 * k + 1] = bk[1] - a1;
      sr[3 * k + 2] = bk[2] - a2;
    }
    __syncthreads();
    if (un.w) {
      // a node of 33..256 columns: a lane per row, 32 rows per warp, walking
      // the column-major copy (column k holds rows k..; lanes read
      // consecutive rows) with r_k broadcast from shared memory
      const int nb = d.t_nb[s];
      const double* Pc = d.t_pcol + d.t_poff[s];
      for (int g = row0 + 32 * warp; g < row0 + rows; g += 32 * bwarps) {
        const int o = g + lane;
        const bool valid = o < row0 + rows;
        const int kend = valid ? (o < nc ? o + 1 : nc) : 0;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        int k = 0;
        for (; k + 3 < kend; k += 4) {
          double p[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) p[i] = Pc[t_coloff(nc, nb, k + i) + (o - k - i)];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double* rk = sr + 3 * (k + i);
            a0 += p[i] * rk[0];
            a1 += p[i] * rk[1];
            a2 += p[i] * rk[2];
          }
        }
        for (; k < kend; ++k) {
          const double p = Pc[t_coloff(nc, nb, k) + (o - k)];
          const double* rk = sr + 3 * k;
          a0 += p * rk[0];
          a1 += p * rk[1];
          a2 += p * rk[2];
        }
        if (!valid) continue;
        if (o < nc) {
          double* yo = y + 3 * (size_t)(c0 + o);
          yo[0] = a0;
          yo[1] = a1;
          yo[2] = a2;
        } else {
          double g0a, g1a, g2a;
          t_gather(d, g0 + o, g0a, g1a, g2a);
          double* uo = d.t_U + 3 * (size_t)(d.t_boff[s] + o - nc);
          uo[0] = a0 + g0a;
          uo[1] = a1 + g1a;
          uo[2] = a2 + g2a;
        }
      }
      continue;
    }
    const double* P = d.t_prow + d.t_poff[s];
    for (int o = row0 + warp; o < row0 + rows; o += bwarps) {
      const int len = o < nc ? o + 1 : nc;
      const double* pr = P + t_rowoff(nc, o);
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, c0a = 0.0, c1a = 0.0, c2a = 0.0;
      int k = lane;
      for (; k + 32 < len; k += 64) {
        const double p = pr[k], q = pr[k + 32];
        a0 += p * sr[3 * k];
        a1 += p * sr[3 * k + 1];
        a2 += p * sr[3 * k + 2];
        c0a += q * sr[3 * (k + 32)];
        c1a += q * sr[3 * (k + 32) + 1];
        c2a += q * sr[3 * (k + 32) + 2];
      }
      if (k < len) {
        const double p = pr[k];
        a0 += p * sr[3 * k];
        a1 += p * sr[3 * k + 1];
        a2 += p * sr[3 * k + 2];
      }
      a0 = t_warp_sum(a0 + c0a);
      a1 = t_warp_sum(a1 + c1a);
      a2 = t_warp_sum(a2 + c2a);
      if (lane == 0) {
        if (o < nc) {
          double* yo = y + 3 * (size_t)(c0 + o);
          yo[0] = a0;
          yo[1] = a1;
          yo[2] = a2;
        } else {
          double g0a, g1a, g2a;
          t_gather(d, g0 + o, g0a, g1a, g2a);
          double* uo = d.t_U + 3 * (size_t)(d.t_boff[s] + o - nc);
          uo[0] = a0 + g0a;
          uo[1] = a1 + g1a;
          uo[2] = a2 + g2a;
        }
      }
    }
  }
  // nodes of at most 32 columns: one warp item per 32 rows; lane k forms
  // r_k from the gathers, lane o computes row o (walking the column-major
  // copy: rows are contiguous)
  for (int w = d.t_lev_wf[h] + gwarp; w < d.t_lev_wf[h + 1]; w += nwarps) {
    const int2 it = d.t_wnode_f[w];
    const int s = it.x, o0 = it.y;
    const int c0 = d.t_c0[s], nc = d.t_nc[s], nb = d.t_nb[s];
    const int64_t g0 = d.t_goff[s];
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    if (lane < nc) {
      double a0, a1, a2;
      t_gather(d, g0 + lane, a0, a1, a2);
      const double* bk = b + 3 * (size_t)(c0 + lane);
      r0 = bk[0] - a0;
      r1 = bk[1] - a1;
      r2 = bk[2] - a2;
    }
    const double* P = d.t_pcol + d.t_poff[s];
    {
      const int o = o0 + lane;
      const bool valid = o < nc + nb;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      int k = 0;
      // four columns per pass (their loads in flight together); column k of
      // the column-major copy starts at t_coloff(k) and holds rows k..
      for (; k + 3 < nc; k += 4) {
        double p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          p[i] = (valid && o >= k + i) ? P[t_coloff(nc, nb, k + i) + (o - k - i)] : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double x0 = __shfl_sync(0xffffffffu, r0, k + i);
          const double x1 = __shfl_sync(0xffffffffu, r1, k + i);
          const double x2 = __shfl_sync(0xffffffffu, r2, k + i);
          a0 += p[i] * x0;
          a1 += p[i] * x1;
          a2 += p[i] * x2;
        }
      }
      for (; k < nc; ++k) {
        const double x0 = __shfl_sync(0xffffffffu, r0, k);
        const double x1 = __shfl_sync(0xffffffffu, r1, k);
        const double x2 = __shfl_sync(0xffffffffu, r2, k);
        if (valid && o >= k) {
          const double p = P[t_coloff(nc, nb, k) + (o - k)];
          a0 += p * x0;
          a1 += p * x1;
          a2 += p * x2;
        }
      }
      if (!valid) continue;
      if (o < nc) {
        double* yo = y + 3 * (size_t)(c0 + o);
        yo[0] = a0;
        yo[1] = a1;
        yo[2] = a2;
      } else {
        double g0a, g1a, g2a;
        t_gather(d, g0 + o, g0a, g1a, g2a);
        double* uo = d.t_U + 3 * (size_t)(d.t_boff[s] + o - nc);
        uo[0] = a0 + g0a;
        uo[1] = a1 + g1a;
        uo[2] = a2 + g2a;
      }
    }
  }
}

// backward sweep, nodes of height h: y -> x (elimination order, t_x). Each
// finished row j is handed on: fin(j, x0, x1, x2) from a block-mode unit,
// called by every lane of a warp with the same values (lanes 0..2 take
// component lane); fin.lanes(on, j, x0, x1, x2) from a warp-mode node, called
// by every lane at once, each lane with its own row (on: the lane has one).
template <class Fin>
__device__ __forceinline__ void tsweep_bwd(const Dev& d, const double* y, int h, int blk, int nblk, int gwarp, int nwarps,
                                           Fin& fin) {
  double* sz = t_stage();
  double* x = d.t_x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, bwarps = blockDim.x >> 5;
  auto stage_z = [&](int c0, int nc, const int* bl, int r, double* dst) {
    if (r < nc) {
      const double* yr = y + 3 * (size_t)(c0 + r);
      dst[0] = yr[0];
      dst[1] = yr[1];
      dst[2] = yr[2];
    } else {
      const double* xr = x + 3 * (size_t)bl[r - nc];
      dst[0] = -xr[0];
      dst[1] = -xr[1];
      dst[2] = -xr[2];
    }
  };
  for (int u = d.t_lev_b[h] + blk; u < d.t_lev_b[h + 1]; u += nblk) {
    const int4 un = d.t_unit_b[u];
    const int s = un.x, k0 = un.y, ncols = un.z;
    const int c0 = d.t_c0[s], nc = d.t_nc[s], nb = d.t_nb[s];
    const int R = nc + nb;
    const int* bl = d.t_below + d.t_boff[s];
    const double* P = d.t_pcol + d.t_poff[s];
    if (R <= kTStage) {
      // the right-hand side [y_s; -x_below] staged once; warps take the
      // unit's columns in turn
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) stage_z(c0, nc, bl, r, sz + 3 * r);
      __syncthreads();
      for (int kk = warp; kk < ncols; kk += bwarps) {
        const int k = k0 + kk;
        const double* pc = P + t_coloff(nc, nb, k) - k;   // pc[r]: row r of column k
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
        int r = k + lane;
        for (; r + 32 < R; r += 64) {
          const double p = pc[r], q = pc[r + 32];
          const double* zr = sz + 3 * r;
          const double* zq = zr + 96;
          a0 += p * zr[0];
          a1 += p * zr[1];
          a2 += p * zr[2];
          e0 += q * zq[0];
          e1 += q * zq[1];
          e2 += q * zq[2];
        }
        if (r < R) {
          const double p = pc[r];
          const double* zr = sz + 3 * r;
          a0 += p * zr[0];
          a1 += p * zr[1];
          a2 += p * zr[2];
        }
        a0 = t_warp_sum(a0 + e0);
        a1 = t_warp_sum(a1 + e1);
        a2 = t_warp_sum(a2 + e2);
        if (lane == 0) {
          double* xk = x + 3 * (size_t)(c0 + k);
          xk[0] = a0;
          xk[1] = a1;
          xk[2] = a2;
        }
        fin(c0 + k, a0, a1, a2);
      }
      continue;
    }
    // a long right-hand side: staged in chunks, one column per warp
    const int k = k0 + warp;
    const bool mine = warp < ncols;
    const double* pc = P + (mine ? t_coloff(nc, nb, k) - k : 0);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int z0 = 0; z0 < R; z0 += kTStage) {
      const int z1 = min(R, z0 + kTStage);
      __syncthreads();
      for (int r = z0 + (int)threadIdx.x; r < z1; r += blockDim.x) stage_z(c0, nc, bl, r, sz + 3 * (r - z0));
      __syncthreads();
      if (mine)
        for (int r = max(k, z0) + lane; r < z1; r += 32) {
          const double p = pc[r];
          const double* zr = sz + 3 * (r - z0);
          a0 += p * zr[0];
          a1 += p * zr[1];
          a2 += p * zr[2];
        }
    }
    if (mine) {
      a0 = t_warp_sum(a0);
      a1 = t_warp_sum(a1);
      a2 = t_warp_sum(a2);
      if (lane == 0) {
        double* xk = x + 3 * (size_t)(c0 + k);
        xk[0] = a0;
        xk[1] = a1;
        xk[2] = a2;
      }
      fin(c0 + k, a0, a1, a2);
    }
  }
  __syncthreads();   // the block-mode units are done with the staging buffer
  // nodes of at most 32 columns: one warp each, lane k accumulates column k
  // over the rows (walking the row-major copy: a row's columns are
  // contiguous); the rows' right-hand side goes through the warp's slice of
  // the staging buffer in chunks
  const int cap = kTStage / bwarps;
  double* zw = sz + 3 * (size_t)warp * cap;
  for (int w = d.t_lev_wb[h] + gwarp; w < d.t_lev_wb[h + 1]; w += nwarps) {
    const int s = d.t_wnode_b[w];
    const int c0 = d.t_c0[s], nc = d.t_nc[s], nb = d.t_nb[s];
    const int R = nc + nb;
    const double* P = d.t_prow + d.t_poff[s];
    const int* bl = d.t_below + d.t_boff[s];
    const bool on = lane < nc;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int r0 = 0; r0 < R; r0 += cap) {
      const int r1 = min(R, r0 + cap);
      __syncwarp();
      for (int r = r0 + lane; r < r1; r += 32) stage_z(c0, nc, bl, r, zw + 3 * (r - r0));
      __syncwarp();
      int r = r0;
      // rows of Linv (row r holds columns 0..r)
      for (; r < min(r1, nc); ++r) {
        if (on && lane <= r) {
          const double p = P[(int64_t)r * (r + 1) / 2 + lane];
          const double* zr = zw + 3 * (r - r0);
          a0 += p * zr[0];
          a1 += p * zr[1];
          a2 += p * zr[2];
        }
      }
      // rows of M (nc columns each), four rows per pass for loads in flight
      const double* pm = P + (int64_t)nc * (nc + 1) / 2 - (int64_t)nc * nc;   // pm[r * nc]: row r >= nc
      for (; r + 3 < r1; r += 4) {
        if (on) {
          double p[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) p[i] = pm[(int64_t)(r + i) * nc + lane];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double* zr = zw + 3 * (r + i - r0);
            a0 += p[i] * zr[0];
            a1 += p[i] * zr[1];
            a2 += p[i] * zr[2];
          }
        }
      }
      for (; r < r1; ++r) {
        if (on) {
          const double p = pm[(int64_t)r * nc + lane];
          const double* zr = zw + 3 * (r - r0);
          a0 += p * zr[0];
          a1 += p * zr[1];
          a2 += p * zr[2];
        }
      }
    }
    if (on) {
      double* xk = x + 3 * (size_t)(c0 + lane);
      xk[0] = a0;
      xk[1] = a1;
      xk[2] = a2;
    }
    fin.lanes(on, c0 + lane, a0, a1, a2);
  }
}

}  // namespace pdk

namespace pdk {

// A^-1 b for one team: both sweeps with a team barrier between heights (none
// after the last backward height: the caller's reduction or barrier follows).
// A real call: inlined, its registers would count against every phase of the
// persistent kernels that use the products with S instead.
template <class Fin>
__device__ __noinline__ bool tsolve_team(const Dev& d, const double* b, double* y, Team tm, int gwarp, int nwarps,
                                         Fin& fin) {
  for (int h = 0; h < d.t_nlev; ++h) {
    tsweep_fwd(d, b, y, h, tm.b, tm.nb, gwarp, nwarps);
    if (!grid_sync(d, tm)) return false;
  }
  for (int h = d.t_nlev - 1; h >= 0; --h) {
    tsweep_bwd(d, y, h, tm.b, tm.nb, gwarp, nwarps, fin);
    if (h > 0 && !grid_sync(d, tm)) return false;
  }
  return true;
}

}  // namespace pdk
