// CUDA kernels of the PD hot path (forward: Alg. 1; backward: Alg. 2).
//
// Data layout: vertex vectors are [n_v][3] float64 (row per vertex); pinned
// vertices keep q = X and carry zeros in every difference/residual vector so
// that norms and dot products run over free DoFs only. Per-element data are
// arrays of structures indexed by element (Dm^-1 as 9 values, w_e V_e).
// The RHS scatter is deterministic: each element writes its 12 corner
// contributions, and a per-vertex gather (vertex -> incident corners, CSR)
// sums them in FP64 together with the constant part b0.
// Reductions use block partials plus a "last block" that finishes the sum in
// a fixed order (no spin-waits); the last block also runs the scalar logic
// (dual gate, Anderson coefficients, trust-region ratio, PCG scalars).
#include <cuda_runtime.h>

#include <cstdint>

#include "pd_common.cuh"
#include "pd_launch.h"

namespace pdk {

// ------------------------------------------------------------ step begin

// q_t (pinned at X), inertial target (eq. freefall) and the constant RHS
//   b0 = M/h^2 q~ + (alpha M + B)/h q_t - A_fp X_p       (free rows)
__global__ void k_step_begin(Dev d, const double* __restrict__ qt_in, const double* __restrict__ vt_in,
                             const double* __restrict__ fext, int t, double* __restrict__ ckpt_t) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) {
    Ctrl* c = d.ctrl;
    c->k = 0; c->done = 0; c->converged = 0; c->pairs = 0; c->ncols = 0; c->head = 0; c->use_hat = 1;
    c->t = t;
    c->n_local = 0;
    c->n_solve = 0;
  }
  if (v >= d.n_v) return;
  const bool pin = d.pinned[v];
  double q[3], b0[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i) q[i] = pin ? d.X[3 * v + i] : qt_in[3 * v + i];
  if (!pin) {
    const double m = d.mass[v], h = d.h;
    double bq[3] = {0.0, 0.0, 0.0};
    for (int p = d.B_ptr[v]; p < d.B_ptr[v + 1]; ++p) {
      const int u = d.B_idx[p];
      const double w = d.B_val[p];
      const bool pu = d.pinned[u];
      for (int i = 0; i < 3; ++i) bq[i] += w * (pu ? d.X[3 * u + i] : qt_in[3 * u + i]);
    }
    for (int i = 0; i < 3; ++i) {
      const double f = fext ? fext[3 * v + i] : 0.0;
      const double qtil = q[i] + h * vt_in[3 * v + i] + h * h * (d.g[i] + f / m);
      d.qtil[3 * v + i] = qtil;
      b0[i] = m / (h * h) * qtil + (d.alpha_d * m * q[i] + bq[i]) / h - d.cA[3 * v + i];
    }
  } else {
    for (int i = 0; i < 3; ++i) d.qtil[3 * v + i] = q[i] + d.h * d.h * d.g[i];
  }
  for (int i = 0; i < 3; ++i) {
    d.qt[3 * v + i] = q[i];
    d.q[3 * v + i] = q[i];
    d.qprev[3 * v + i] = q[i];
    d.gprev[3 * v + i] = 0.0;
    d.b0[3 * v + i] = b0[i];
    if (ckpt_t) ckpt_t[3 * v + i] = q[i];
  }
}

// Local step fused with the per-element part of the RHS scatter (Alg. 1,
// eq. nh_prox / corotated projection, eq. A_basic).
template <typename T>
__global__ void __launch_bounds__(kTetBlock) k_local(Dev d, const double* __restrict__ x) {
  if (d.ctrl->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_e) return;
  int4 tv;
  T Bm[9], coef;
  load_elem<T>(d, e, tv, Bm, coef);
  T F[9], P[9], U[9], V[9], sF[3], ss[3], c[12];
  deform<T>(x, tv, Bm, F);
  project<T>(d, F, P, U, sF, V, ss);
  corner_forces<T>(P, Bm, coef, c);
  T* out = reinterpret_cast<T*>(d.contrib) + 12 * (size_t)e;
#pragma unroll
  for (int i = 0; i < 12; ++i) out[i] = c[i];
}

// b^k = b0 + sum of corner contributions (FP64); writes b in vertex order and
// in elimination order; dual gate on (q^k, q^{k-1}, b^k, b^{k-1}) (eq. convergence_dual).
template <typename T>
__global__ void __launch_bounds__(kVtxBlock) k_assemble(Dev d) {
  if (d.ctrl->done) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[3] = {0.0, 0.0, 0.0};  // ||b - bprev||^2, ||bprev||^2, non-finite count
  const int k = d.ctrl->k;
  if (v < d.n_v && !d.pinned[v]) {
    double acc[3] = {d.b0[3 * v], d.b0[3 * v + 1], d.b0[3 * v + 2]};
    gather_contrib<T>(d, v, acc);
    const int pos = d.iperm[v];
    for (int i = 0; i < 3; ++i) {
      const double bp = d.bprev[3 * v + i];
      if (k > 0) {
        part[0] += (acc[i] - bp) * (acc[i] - bp);
        part[1] += bp * bp;
      }
      d.b[3 * v + i] = acc[i];
      d.bperm[3 * (size_t)pos + i] = acc[i];
      d.y[3 * (size_t)pos + i] = 0.0;
    }
    if (!finite3(acc[0], acc[1], acc[2])) part[2] += 1.0;
  }
  block_reduce_store<3>(part, d.red);
  if (last_block(&d.ctrl->ticket[TK_ASSEMBLE])) {
    if (threadIdx.x == 0) {
      Ctrl* c = d.ctrl;
      const double db2 = sum_partials(d.red, gridDim.x, 0);
      const double bp2 = sum_partials(d.red, gridDim.x, 1);
      c->n_local += 1;
      if (sum_partials(d.red, gridDim.x, 2) > 0.0) c->status |= 1;
      c->db_norm2 = db2;
      c->bprev_norm2 = bp2;
      if (d.fixed_iters <= 0 && k >= 2) {
        const bool step_ok = sqrt(c->dq_norm2) <= d.eps_step * sqrt(c->qprev_norm2) + d.eps_abs;
        const bool res_ok = sqrt(db2) <= d.eps_res * sqrt(bp2) + d.eps_abs;
        if (step_ok && res_ok) {
          c->converged = 1;
          c->done = 1;
        }
      }
      if (!c->done && k >= d.k_max) {
        c->done = 1;
        c->not_converged += 1;
      }
      if (c->status & 1) c->done = 1;
    }
  }
}

// ------------------------------------------------------------ solve A^-1 = S^T S

// y_i = sum_{j in [first_i, i]} S_ij x_j for 3 right-hand sides; one warp per
// segment of at most a few hundred entries of one skyline row; rows split
// into several segments accumulate with atomics into y (zeroed beforehand).
__global__ void __launch_bounds__(32 * kWarpsSpmv) k_spmv_s(Dev d, const double* __restrict__ xin,
                                                            double* __restrict__ y, int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int sg = warp; sg < d.n_seg; sg += nwarps) {
    const int4 seg = d.s_seg[sg];  // x = row, y = offset in row, z = length, w = multi
    const int row = seg.x;
    const int64_t base = d.s_rowptr[row] + seg.y;
    const int col0 = d.s_first[row] + seg.y;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int p = lane; p < seg.z; p += 32) {
      const double s = d.s_val[base + p];
      const double* xv = xin + 3 * (size_t)(col0 + p);
      a0 += s * xv[0];
      a1 += s * xv[1];
      a2 += s * xv[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      double* yr = y + 3 * (size_t)row;
      if (seg.w) {
        atomicAdd(yr, a0);
        atomicAdd(yr + 1, a1);
        atomicAdd(yr + 2, a2);
      } else {
        yr[0] = a0;
        yr[1] = a1;
        yr[2] = a2;
      }
    }
  }
}

// out[perm[j]] = sum over the ancestors i of j of S_ij y_i (row j of S^T);
// one warp per row.
__global__ void __launch_bounds__(32 * kWarpsSpmv) k_spmv_st(Dev d, const double* __restrict__ y,
                                                             double* __restrict__ out, int check_done) {
  if (check_done == 1 && d.ctrl->done) return;
  if (check_done == 2 && d.ctrl->adj_done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < d.n_f; j += nwarps) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t p = d.st_ptr[j] + lane; p < d.st_ptr[j + 1]; p += 32) {
      const double s = d.st_val[p];
      const double* yv = y + 3 * (size_t)d.st_idx[p];
      a0 += s * yv[0];
      a1 += s * yv[1];
      a2 += s * yv[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      const int v = d.perm[j];
      out[3 * v] = a0;
      out[3 * v + 1] = a1;
      out[3 * v + 2] = a2;
    }
  }
}

// ------------------------------------------------------------ Anderson

// g = q_hat - q; with a previous pair in the history, the new difference
// column (q - qprev, g - gprev) goes to the ring slot `head`; partial dots
// dG_new . dG_j (all held columns) and dG_j . g (eq. aa_gamma).
__global__ void __launch_bounds__(kVtxBlock) k_aa(Dev d) {
  if (d.ctrl->done) return;
  const Ctrl* c = d.ctrl;
  const int m = d.aa_m;
  const bool add = m > 0 && c->pairs >= 1;
  const int slot = c->head;
  const int ncols_new = add ? (c->ncols < m ? c->ncols + 1 : m) : c->ncols;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double part[2 * kMaxAA] = {};
  const size_t nv3 = 3 * (size_t)d.n_v;
  if (v < d.n_v && !d.pinned[v]) {
    for (int i = 0; i < 3; ++i) {
      const size_t o = 3 * (size_t)v + i;
      const double g = d.qhat[o] - d.q[o];
      if (add) {
        const double dg = g - d.gprev[o];
        d.dG[slot * nv3 + o] = dg;
        d.dQ[slot * nv3 + o] = d.q[o] - d.qprev[o];
      }
      d.gprev[o] = g;
      for (int j = 0; j < ncols_new; ++j) {
        const double dgj = d.dG[j * nv3 + o];
        if (add) part[j] += d.dG[slot * nv3 + o] * dgj;
        part[kMaxAA + j] += dgj * g;
      }
    }
  }
  block_reduce_store<2 * kMaxAA>(part, d.red);
  if (last_block(&d.ctrl->ticket[TK_SPMV_T])) {
    if (threadIdx.x == 0) {
      Ctrl* cc = d.ctrl;
      cc->n_solve += 1;
      if (m == 0) {
        cc->use_hat = 1;
      } else {
        if (add) {
          for (int j = 0; j < ncols_new; ++j) {
            const double gj = sum_partials(d.red, gridDim.x, j);
            cc->gram[slot * kMaxAA + j] = gj;
            cc->gram[j * kMaxAA + slot] = gj;
          }
          cc->ncols = ncols_new;
          cc->head = (slot + 1) % m;
        }
        cc->pairs = cc->pairs < m + 1 ? cc->pairs + 1 : m + 1;
        const int nc = cc->ncols;
        cc->use_hat = 1;
        if (nc >= 1) {
          // (dG^T dG + reg I) gamma = dG^T g, reg = max(1e-6 ||dG||_F^2 / nc, 1e-12)
          double A[kMaxAA * kMaxAA], rhs[kMaxAA];
          double tr = 0.0;
          for (int j = 0; j < nc; ++j) tr += cc->gram[j * kMaxAA + j];
          const double reg = fmax(1e-6 * tr / nc, 1e-12);
          for (int i = 0; i < nc; ++i) {
            rhs[i] = sum_partials(d.red, gridDim.x, kMaxAA + i);
            for (int j = 0; j < nc; ++j) A[i * nc + j] = cc->gram[i * kMaxAA + j] + (i == j ? reg : 0.0);
          }
          // Cholesky solve (SPD by the regularisation)
          bool ok = true;
          for (int j = 0; j < nc && ok; ++j) {
            double s = A[j * nc + j];
            for (int k2 = 0; k2 < j; ++k2) s -= A[j * nc + k2] * A[j * nc + k2];
            if (!(s > 0.0)) { ok = false; break; }
            const double r = sqrt(s);
            A[j * nc + j] = r;
            for (int i = j + 1; i < nc; ++i) {
              double t = A[i * nc + j];
              for (int k2 = 0; k2 < j; ++k2) t -= A[i * nc + k2] * A[j * nc + k2];
              A[i * nc + j] = t / r;
            }
          }
          double gam[kMaxAA];
          double gn = 0.0;
          if (ok) {
            for (int i = 0; i < nc; ++i) {
              double t = rhs[i];
              for (int k2 = 0; k2 < i; ++k2) t -= A[i * nc + k2] * gam[k2];
              gam[i] = t / A[i * nc + i];
            }
            for (int i = nc - 1; i >= 0; --i) {
              double t = gam[i];
              for (int k2 = i + 1; k2 < nc; ++k2) t -= A[k2 * nc + i] * gam[k2];
              gam[i] = t / A[i * nc + i];
            }
            for (int i = 0; i < nc; ++i) gn += gam[i] * gam[i];
          }
          if (!ok || !(sqrt(gn) <= 10.0)) {
            // reliability guard: take q_hat and clear the history
            cc->resets += 1;
            cc->pairs = 0;
            cc->ncols = 0;
            cc->head = 0;
            for (int i = 0; i < kMaxAA * kMaxAA; ++i) cc->gram[i] = 0.0;
          } else {
            for (int i = 0; i < nc; ++i) cc->gamma[i] = gam[i];
            cc->use_hat = 0;
          }
        }
      }
    }
  }
}

// q^{k+1} = q_hat - (dQ + dG) gamma (or q_hat); step norms for the gate.
__global__ void __launch_bounds__(kVtxBlock) k_update(Dev d) {
  if (d.ctrl->done) return;
  const Ctrl* c = d.ctrl;
  const int use_hat = c->use_hat;
  const int nc = c->ncols;
  double gam[kMaxAA];
  for (int j = 0; j < nc; ++j) gam[j] = c->gamma[j];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nv3 = 3 * (size_t)d.n_v;
  double part[2] = {0.0, 0.0};
  if (v < d.n_v && !d.pinned[v]) {
    for (int i = 0; i < 3; ++i) {
      const size_t o = 3 * (size_t)v + i;
      double qn = d.qhat[o];
      if (!use_hat)
        for (int j = 0; j < nc; ++j) qn -= gam[j] * (d.dQ[j * nv3 + o] + d.dG[j * nv3 + o]);
      const double qo = d.q[o];
      part[0] += (qn - qo) * (qn - qo);
      part[1] += qo * qo;
      d.qprev[o] = qo;
      d.q[o] = qn;
      d.bprev[o] = d.b[o];
    }
  }
  block_reduce_store<2>(part, d.red);
  if (last_block(&d.ctrl->ticket[TK_UPDATE])) {
    if (threadIdx.x == 0) {
      Ctrl* cc = d.ctrl;
      cc->dq_norm2 = sum_partials(d.red, gridDim.x, 0);
      cc->qprev_norm2 = sum_partials(d.red, gridDim.x, 1);
      cc->k += 1;
      if (d.fixed_iters > 0 && cc->k >= d.fixed_iters) cc->done = 1;
    }
  }
}

// ------------------------------------------------------------ step end

__global__ void k_step_end(Dev d, double* __restrict__ qn, double* __restrict__ vn, double* __restrict__ ckpt_next) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) {
    Ctrl* c = d.ctrl;
    c->iters_total += c->k;
    if (c->k > c->iters_max) c->iters_max = c->k;
    if (d.phase_count) {
      d.phase_count[2 * c->t] = c->n_local;
      d.phase_count[2 * c->t + 1] = c->n_solve;
    }
  }
  if (v >= d.n_v) return;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    const double q = d.q[o];
    if (qn) qn[o] = q;
    if (vn) vn[o] = d.pinned[v] ? 0.0 : (q - d.qt[o]) / d.h;
    if (ckpt_next) ckpt_next[o] = q;
  }
}

// Trust-region selection (eq. tr_step, tr_decreases, tr_ratio, tr_rule):
// Delta Phi_act = Phi(q*-1) - Phi(q*), Delta Phi_mod = 1/2 |dq^T A dq| with the
// assembled operator; elements contribute V_e (psi_e(F(q*-1)) - psi_e(F(q*)))
// with per-element mu_e, lambda_e (+inf if inverted), vertices the kinetic
// difference and the quadratic form. Threads [0, n_e) take elements, the
// rest vertices.
__device__ __forceinline__ double psi_elem(const Dev& d, const double* x, int e, bool& inverted) {
  const int4 tv = d.tets[e];
  double Bm[9];
  for (int i = 0; i < 9; ++i) Bm[i] = d.Bm64[9 * (size_t)e + i];
  double F[9];
  deform<double>(x, tv, Bm, F);
  const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
  if (!(J > 0.0)) {
    inverted = true;
    return 0.0;
  }
  double n2 = 0.0;
  for (int i = 0; i < 9; ++i) n2 += F[i] * F[i];
  const double lnJ = log(J), mu = d.mu_e[e], lam = d.lam_e[e];
  return d.vol[e] * (0.5 * mu * (n2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
}

__global__ void __launch_bounds__(kVtxBlock) k_tr(Dev d, double* tau_out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double part[4] = {0.0, 0.0, 0.0, 0.0};  // elastic diff, kinetic diff, quad form, inverted count
  if (tid < d.n_e) {
    bool inv = false;
    const double a = psi_elem(d, d.qprev, tid, inv);
    const double b = psi_elem(d, d.q, tid, inv);
    part[0] = a - b;
    if (inv) part[3] = 1.0;
  } else if (tid < d.n_e + d.n_v) {
    const int v = tid - d.n_e;
    if (!d.pinned[v]) {
      const double m = d.mass[v];
      for (int i = 0; i < 3; ++i) {
        const size_t o = 3 * (size_t)v + i;
        const double a = d.qprev[o] - d.qtil[o], b = d.q[o] - d.qtil[o];
        part[1] += 0.5 * m / (d.h * d.h) * (a * a - b * b);
        double Adq = 0.0;
        for (int p = d.A_ptr[v]; p < d.A_ptr[v + 1]; ++p) {
          const int u = d.A_idx[p];
          Adq += d.A_val[p] * (d.q[3 * (size_t)u + i] - d.qprev[3 * (size_t)u + i]);
        }
        part[2] += (d.q[o] - d.qprev[o]) * Adq;
      }
    }
  }
  block_reduce_store<4>(part, d.red);
  if (last_block(&d.ctrl->ticket[TK_TR])) {
    if (threadIdx.x == 0) {
      Ctrl* c = d.ctrl;
      const double act = sum_partials(d.red, gridDim.x, 0) + sum_partials(d.red, gridDim.x, 1);
      const double mod = 0.5 * fabs(sum_partials(d.red, gridDim.x, 2));
      const bool inverted = sum_partials(d.red, gridDim.x, 3) > 0.0;
      double rho = mod < 1e-12 ? 1.0 : (inverted ? INFINITY : act / mod);
      double tau;
      if (d.tr_mode == 1) tau = 0.0;
      else if (d.tr_mode == 2) tau = 0.5;
      else if (d.tr_mode == 3) tau = 1.0;
      else tau = (isfinite(rho) && fabs(rho - 1.0) <= d.eps_tr) ? 0.5 : 1.0;
      if (tau == 0.5) c->tau_half += 1; else if (tau == 1.0) c->tau_one += 1;
      c->last_rho = rho;
      tau_out[c->t] = tau;
    }
  }
}

// ------------------------------------------------------------ standalone solve

// b (vertex order) -> elimination order in xperm; zero the S b accumulator
// rows and the pinned rows of x
__global__ void k_solve_in(Dev d, const double* __restrict__ b, double* __restrict__ xperm, double* __restrict__ y,
                           double* __restrict__ x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_v) return;
  if (d.pinned[v]) {
    for (int i = 0; i < 3; ++i) x[3 * (size_t)v + i] = 0.0;
    return;
  }
  const int pos = d.iperm[v];
  for (int i = 0; i < 3; ++i) {
    xperm[3 * (size_t)pos + i] = b[3 * (size_t)v + i];
    y[3 * (size_t)pos + i] = 0.0;
  }
}

// ------------------------------------------------------------ launch wrappers

static inline int nblk(int n, int b) { return (n + b - 1) / b; }

void launch_step_begin(const Dev& d, cudaStream_t s, const double* qt, const double* vt, const double* fext, int t,
                       double* ckpt_t) {
  k_step_begin<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, qt, vt, fext, t, ckpt_t);
}

int spmv_blocks(const Dev& d) {
  int b = nblk(d.n_seg, kWarpsSpmv);
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}
int spmvt_blocks(const Dev& d) {
  int b = nblk(d.n_f, kWarpsSpmv);
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

void launch_apply_inverse(const Dev& d, cudaStream_t s, const double* xperm, double* y, double* out, int check) {
  k_spmv_s<<<spmv_blocks(d), 32 * kWarpsSpmv, 0, s>>>(d, xperm, y, check);
  k_spmv_st<<<spmvt_blocks(d), 32 * kWarpsSpmv, 0, s>>>(d, y, out, check);
}

void launch_solve(const Dev& d, cudaStream_t s, const double* b, double* xperm, double* y, double* x) {
  k_solve_in<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, b, xperm, y, x);
  launch_apply_inverse(d, s, xperm, y, x, 0);
}

void launch_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  if (d.local_fp32) {
    k_local<float><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.q);
    k_assemble<float><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  } else {
    k_local<double><<<nblk(d.n_e, kTetBlock), kTetBlock, 0, s>>>(d, d.q);
    k_assemble<double><<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  }
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  launch_apply_inverse(d, s, d.bperm, d.y, d.qhat, 1);
  if (ev) cudaEventRecord(ev[3], s);
  k_aa<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
  k_update<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d);
}

void launch_step_end(const Dev& d, cudaStream_t s, double* qn, double* vn, double* ckpt_next, double* tau) {
  k_step_end<<<nblk(d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, qn, vn, ckpt_next);
  if (d.model == 1) k_tr<<<nblk(d.n_e + d.n_v, kVtxBlock), kVtxBlock, 0, s>>>(d, tau);
}

int max_reduction_blocks(int n_v, int n_e) {
  int a = nblk(n_v, kVtxBlock), b = nblk(n_e + n_v, kVtxBlock), c = nblk(n_e, kTetBlock);
  int m = a > b ? a : b;
  return m > c ? m : c;
}

}  // namespace pdk
