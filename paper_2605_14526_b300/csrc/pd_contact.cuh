// Frictional contact inside the local-global iteration (Sec. 4.6, eq. fb_n,
// eq. contact_system, eq. q_update), with the factor of A kept fixed.
//
// Contacts are vertex-ground (z >= z_g, normal +z) and vertex-box-bottom
// (z <= z_box(t), normal -z); A = L_A (x) I_3 and the normals are +-z, so the
// normal and the tangential subproblems decouple by axis and share the scalar
// Delassus matrix W = (L_A^-1)_CC of the candidates C. Per iteration:
//   q_u,C  = rows C of S^T (S b)                    (the plain global step at C)
//   normal 0 <= lam_n _|_ D W D lam_n + g >= 0,   g_c = n_c (q_u,z - z_c)
//   Tresca lam_f = argmin 1/2 sum_axes lam^T W lam + s^T lam over |lam_f,c| <= mu lam_n,c,
//          s_c = q_u,xy - q_t,xy
//   y     <- S b + S J^T lam;  q = S^T y = A^-1 (b + J^T lam)
// Both subproblems are strictly convex QPs; each is solved by FISTA (Beck &
// Teboulle 2009) with gradient-based adaptive restart (O'Donoghue & Candes
// 2015), step 1 / lambda_max(W), warm-started from the previous iteration's
// multipliers, one team-parallel row pass over W per inner iteration. The
// paper solves the linearised FB system by dense LDL^T each inner iteration;
// on this part's FP64 rate that costs K^3/3 per refactorisation, while the
// FISTA pass costs K^2.
#pragma once
#include "pd_phases.cuh"

namespace pdk {

__device__ __forceinline__ double con_height(const Dev& d, int c, int t) {
  if (d.con_n[c] > 0.0) return d.con_zg;
  const int k = min(t + 1, d.con_steps);
  return d.con_zb0 - d.con_travel * (double)k / (double)d.con_steps;
}

// bilateral attachments: three equality rows with free multipliers that
// hold the vertex at its target p(t) = p0 + travel min(t + 1, steps)/steps
__device__ __forceinline__ bool con_is_att(const Dev& d, int c) { return d.con_att && d.con_att[c]; }
__device__ __forceinline__ double con_target(const Dev& d, int c, int t, int k) {
  const double s = (double)min(t + 1, d.con_att_steps) / (double)d.con_att_steps;
  return d.con_tgt[6 * (size_t)c + k] + s * d.con_tgt[6 * (size_t)c + 3 + k];
}

// work buffer layout: lam_n [3][K] (rotating prev / cur / next), lam_f [3][K][2],
// gap [K], slip [K][2]
__device__ __forceinline__ double* con_lamn(const Dev& d, int r) { return d.con_buf + (size_t)(r % 3) * d.n_con; }
__device__ __forceinline__ double* con_lamf(const Dev& d, int r) {
  return d.con_buf + 3 * (size_t)d.n_con + (size_t)(r % 3) * 2 * d.n_con;
}
__device__ __forceinline__ double* con_gap(const Dev& d) { return d.con_buf + 9 * (size_t)d.n_con; }
__device__ __forceinline__ double* con_slip(const Dev& d) { return d.con_buf + 10 * (size_t)d.n_con; }
// the pass's extrapolated multipliers z = cur + beta (cur - prev): n_c z_c for
// the normal pass, (z_x, z_y) for the friction pass
__device__ __forceinline__ double* con_z(const Dev& d) { return d.con_buf + 12 * (size_t)d.n_con; }

// warp per candidate: q_u at the candidate (row pos_c of S^T y), its gap and
// its slip since q_t (an attachment: its residuals to the target)
__device__ __forceinline__ void contact_gather(const Dev& d, int c, int t, int lane) {
  double a0, a1, a2;
  spmv_st_sum(d, d.y, d.con_pos[c], lane, a0, a1, a2);
  if (lane == 0) {
    const int v = d.con_v[c];
    if (con_is_att(d, c)) {   // residuals to the target on all three rows
      con_gap(d)[c] = a2 - con_target(d, c, t, 2);
      con_slip(d)[2 * c] = a0 - con_target(d, c, t, 0);
      con_slip(d)[2 * c + 1] = a1 - con_target(d, c, t, 1);
    } else {
      con_gap(d)[c] = d.con_n[c] * (a2 - con_height(d, c, t));
      con_slip(d)[2 * c] = a0 - d.qt[3 * (size_t)v];
      con_slip(d)[2 * c + 1] = a1 - d.qt[3 * (size_t)v + 1];
    }
  }
}

// FISTA state (one instance per subproblem, in the team's shared state).
// The inner tolerance follows the outer iteration: 1e-2 x the relative
// b-change of the last local step, clamped to [con_tol, 1e-4], so early outer
// iterations take cheap inexact inner solves and the converged step an
// inner solve at con_tol (the fixed point does not depend on the path).
template <class St>
__device__ __forceinline__ void fista_reset(const Dev& d, St* S) {
  const double rel = S->bprev_norm2 > 0.0 ? sqrt(S->db_norm2 / S->bprev_norm2) : 1.0;
  S->f_tol = fmax(d.con_tol, fmin(1e-4, 1e-2 * rel));
  S->f_t = 1.0;
  S->f_beta = 0.0;   // the first pass starts from the warm multipliers (no momentum)
  S->f_it = 0;
  S->f_done = 0;
}

// after a pass: sums = {||next - cur||^2, ||next||^2, restart indicator};
// rot is the rotation index of the subproblem's multipliers
template <class St>
__device__ __forceinline__ void fista_finish(const Dev& d, St* S, int* rot, const double* sums) {
  *rot += 1;         // next becomes cur
  S->f_it += 1;
  S->con_iters += 1;
  const bool conv = sums[0] <= S->f_tol * S->f_tol * sums[1] + 1e-300;
  if (conv) {
    S->f_done = 1;
  } else if (S->f_it >= d.con_max_iters) {
    S->f_done = 1;
    S->con_unconverged += 1;
  } else if (sums[2] > 0.0) {   // the step went against the momentum: restart
    S->f_t = 1.0;
    S->f_beta = 0.0;
  } else {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * S->f_t * S->f_t));
    S->f_beta = (S->f_t - 1.0) / tn;
    S->f_t = tn;
  }
}

// extrapolation of a pass, item c (block range over the candidates); the
// rows below read it after a team barrier, so each W entry costs one FMA
__device__ __forceinline__ void normal_z_item(const Dev& d, int c, int rot, double beta) {
  const double* prev = con_lamn(d, rot);
  const double* cur = con_lamn(d, rot + 1);
  con_z(d)[c] = d.con_n[c] * (cur[c] + beta * (cur[c] - prev[c]));
}
__device__ __forceinline__ void friction_z_item(const Dev& d, int c, int rot, double beta) {
  const double* prev = con_lamf(d, rot);
  const double* cur = con_lamf(d, rot + 1);
  for (int k = 0; k < 2; ++k) con_z(d)[2 * c + k] = cur[2 * c + k] + beta * (cur[2 * c + k] - prev[2 * c + k]);
}

// normal LCP pass, warp per row c: next_c = max(0, z_c - ((D W D z)_c + g_c) / L)
// with D z from the extrapolation buffer (an attachment's row: no max, the
// mixed LCP's free variable)
__device__ __forceinline__ void normal_row(const Dev& d, int c, int rot, int lane, double* part) {
  const int K = d.n_con;
  const double* cur = con_lamn(d, rot + 1);
  double* nxt = con_lamn(d, rot + 2);
  const double* Wr = d.con_W + (size_t)c * K;
  const double* z = con_z(d);
  double acc = 0.0;
  for (int j = lane; j < K; j += 32) acc += Wr[j] * z[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double zc = d.con_n[c] * z[c];   // n_c = +-1
    const double grad = d.con_n[c] * acc + con_gap(d)[c];
    const double nv = con_is_att(d, c) ? zc - grad / d.con_L : fmax(0.0, zc - grad / d.con_L);   // attachment: free
    nxt[c] = nv;
    const double dl = nv - cur[c];
    part[0] += dl * dl;
    part[1] += nv * nv;
    part[2] += (zc - nv) * dl;
  }
}

// Tresca pass, warp per row c: two components, disk radius mu * lam_n,c (an
// attachment's rows: no disk)
__device__ __forceinline__ void friction_row(const Dev& d, int c, int rot, const double* lam_n, int lane,
                                             double* part) {
  const int K = d.n_con;
  const double* cur = con_lamf(d, rot + 1);
  double* nxt = con_lamf(d, rot + 2);
  const double* Wr = d.con_W + (size_t)c * K;
  const double2* z = reinterpret_cast<const double2*>(con_z(d));
  double sx = 0.0, sy = 0.0;
  for (int j = lane; j < K; j += 32) {
    const double w = Wr[j];
    const double2 zz = z[j];
    sx += w * zz.x;
    sy += w * zz.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    const double zx = z[c].x, zy = z[c].y;
    double nx = zx - (sx + con_slip(d)[2 * c]) / d.con_L;
    double ny = zy - (sy + con_slip(d)[2 * c + 1]) / d.con_L;
    const double rho = d.con_mu * lam_n[c];
    const double r = sqrt(nx * nx + ny * ny);
    if (r > rho && !con_is_att(d, c)) {   // an attachment has no disk
      const double s = r > 0.0 ? rho / r : 0.0;
      nx *= s;
      ny *= s;
    }
    nxt[2 * c] = nx;
    nxt[2 * c + 1] = ny;
    const double dx = nx - cur[2 * c], dy = ny - cur[2 * c + 1];
    part[0] += dx * dx + dy * dy;
    part[1] += nx * nx + ny * ny;
    part[2] += (zx - nx) * dx + (zy - ny) * dy;
  }
}

// y_i += sum over candidates c with pos_c in [first_desc(i), i] of
// S[i, pos_c] (lam_f,c, n_c lam_n,c): the contact impulse J^T lam pushed
// through the first product with S (warp per row i; candidates sorted by
// position, found by binary search)
__device__ __forceinline__ void contact_y_row(const Dev& d, int i, const double* lam_n, const double* lam_f, int lane) {
  const int lo = d.s_first[i];
  int a = 0, b = d.n_con;   // first candidate with pos >= lo
  while (a < b) {
    const int m = (a + b) >> 1;
    if (d.con_pos[m] < lo) a = m + 1;
    else b = m;
  }
  const float2* srow = d.s_hl + d.s_rowptr[i];
  const double* srow64 = d.sfp64 ? d.s_val64 + d.s_rowptr[i] : nullptr;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  for (int c = a + lane; c < d.n_con; c += 32) {
    const int p = d.con_pos[c];
    if (p > i) break;
    const double s = srow64 ? srow64[p - lo] : df_join(srow[p - lo]);
    r0 += s * lam_f[2 * c];
    r1 += s * lam_f[2 * c + 1];
    r2 += s * d.con_n[c] * lam_n[c];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if (lane == 0) {
    const size_t o = 3 * (size_t)i;
    store_y(d, d.y, o, load_y(d, d.y, o) + r0);
    store_y(d, d.y, o + 1, load_y(d, d.y, o + 1) + r1);
    store_y(d, d.y, o + 2, load_y(d, d.y, o + 2) + r2);
  }
}

// ---------------------------------------------------------------- adjoint
//
// With the active sets of step t held fixed (normal-active: lam_n > 0;
// sticking: no slip, see contact_flag_item), the adjoint solves
//   (A - K) a + G^T nu = q_bar,  G a = 0
// by the same preconditioned CG with the preconditioner projected
// A-orthogonally onto null(G): z = A^-1 (r - G^T w), w = W_a^-1 G A^-1 r,
// W_a = G A^-1 G^T (the Delassus matrix on the active rows, per axis).
// Every projection also takes its share G^T w out of the residual,
// r <- r - G^T w, and adds w to nu (the residual update of Gould, Hribar and
// Nocedal 2001): r keeps no part that the projection removes, so r . z is no
// longer the small difference of the projected preconditioner's two large
// terms, and the CG reaches its tolerance instead of breaking down at the
// rounding level of W_a. On exit (A - K) a + G^T nu = q_bar - r; the
// sticking rows of nu enter dL/dq_t (the constraint q_xy = q_t,xy of a
// sticking contact depends on q_t; an attachment's rows, whose constraint is
// its prescribed target, do not).

// active sets of the step, one flag per candidate (bit 0 normal-active,
// bit 1 sticking), formed at the step's start by contact_flag_item
__device__ __forceinline__ double* cb_flag(const Dev& d) { return d.con_bwd + 19 * (size_t)d.n_con; }   // [K]
__device__ __forceinline__ bool con_act(const Dev& d, int c) { return ((int)cb_flag(d)[c] & 1) != 0; }
__device__ __forceinline__ bool con_stick(const Dev& d, int c) { return ((int)cb_flag(d)[c] & 2) != 0; }

// normal-active: lam_n above thr = 1e-9 x the step's total normal impulse (an
// inactive contact's inner iterate can keep a rounding-level lam_n);
// sticking: active, with friction, and a tangential slip over the step of at
// most con_slip_tol (an exact solution does not slip where the friction is
// strictly inside its disk; the positions are determined far better than the
// multipliers in the ill-conditioned directions of W)
__device__ __forceinline__ void contact_flag_item(const Dev& d, const double* ck, double thr, const double* qnext,
                                                  const double* qt, int c) {
  if (con_is_att(d, c)) {   // attachments: equality rows on all three axes at every step
    cb_flag(d)[c] = 3.0;
    return;
  }
  const bool act = ck[c] > thr;
  const size_t v = 3 * (size_t)d.con_v[c];
  const double sx = qnext[v] - qt[v], sy = qnext[v + 1] - qt[v + 1];
  const bool stick = act && d.con_mu > 0.0 && sqrt(sx * sx + sy * sy) <= d.con_slip_tol;
  cb_flag(d)[c] = (double)((act ? 1 : 0) | (stick ? 2 : 0));
}
// adjoint work buffers ([K][3] each unless noted)
__device__ __forceinline__ double* cb_x(const Dev& d) { return d.con_bwd; }
__device__ __forceinline__ double* cb_r(const Dev& d) { return d.con_bwd + 3 * (size_t)d.n_con; }
__device__ __forceinline__ double* cb_p(const Dev& d, int r) { return d.con_bwd + (6 + 3 * (r & 1)) * (size_t)d.n_con; }
__device__ __forceinline__ double* cb_ap(const Dev& d) { return d.con_bwd + 12 * (size_t)d.n_con; }
__device__ __forceinline__ double* cb_nz(const Dev& d) { return d.con_bwd + 15 * (size_t)d.n_con; }    // [K]
__device__ __forceinline__ double* cb_nxy(const Dev& d) { return d.con_bwd + 16 * (size_t)d.n_con; }   // [K][2]
// n_c p_z of the current CG direction (the W rows then cost three FMAs per entry)
__device__ __forceinline__ double* cb_pz(const Dev& d) { return d.con_bwd + 18 * (size_t)d.n_con; }   // [K]
// nu: the sum of the step's projection multipliers w (since its last restart)
__device__ __forceinline__ double* cb_nu(const Dev& d) { return d.con_bwd + 20 * (size_t)d.n_con; }

// warp per candidate: u = G A^-1 r (masked rows of S^T y) as the CG
// residual; w = 0; p = u; partial |u|^2 per axis
__device__ __forceinline__ void proj_gather(const Dev& d, int c, int lane, double* part) {
  double a0, a1, a2;
  spmv_st_sum(d, d.y, d.con_pos[c], lane, a0, a1, a2);
  if (lane == 0) {
    const bool st = con_stick(d, c), ac = con_act(d, c);
    const double u[3] = {st ? a0 : 0.0, st ? a1 : 0.0, ac ? d.con_n[c] * a2 : 0.0};
    for (int k = 0; k < 3; ++k) {
      cb_x(d)[3 * c + k] = 0.0;
      cb_r(d)[3 * c + k] = u[k];
      cb_p(d, 0)[3 * c + k] = u[k];
      part[k] += u[k] * u[k];
    }
    cb_pz(d)[c] = d.con_n[c] * u[2];
  }
}

// warp per row: W_a p (axis 2 with the normal signs), partial p . W_a p
__device__ __forceinline__ void proj_ap_row(const Dev& d, int c, int rot, int lane, double* part) {
  const int K = d.n_con;
  const double* p = cb_p(d, rot);
  const double* pz = cb_pz(d);
  const double* Wr = d.con_W + (size_t)c * K;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int j = lane; j < K; j += 32) {
    const double w = Wr[j];
    s0 += w * p[3 * j];
    s1 += w * p[3 * j + 1];
    s2 += w * pz[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    const bool st = con_stick(d, c), ac = con_act(d, c);
    const double ap[3] = {st ? s0 : 0.0, st ? s1 : 0.0, ac ? d.con_n[c] * s2 : 0.0};
    for (int k = 0; k < 3; ++k) {
      cb_ap(d)[3 * c + k] = ap[k];
      part[k] += p[3 * c + k] * ap[k];
    }
  }
}

// thread per candidate: w += alpha p, r -= alpha W_a p; partial |r|^2 per axis
__device__ __forceinline__ void proj_update(const Dev& d, int c, int rot, const double* alpha, double* part) {
  const double* p = cb_p(d, rot);
  for (int k = 0; k < 3; ++k) {
    const size_t o = 3 * (size_t)c + k;
    cb_x(d)[o] += alpha[k] * p[o];
    const double r = cb_r(d)[o] - alpha[k] * cb_ap(d)[o];
    cb_r(d)[o] = r;
    part[k] += r * r;
  }
}

// thread per candidate: next direction p' = r + beta p (other buffer)
__device__ __forceinline__ void proj_dir(const Dev& d, int c, int rot, const double* beta) {
  const double* p = cb_p(d, rot);
  double* pn = cb_p(d, rot + 1);
  for (int k = 0; k < 3; ++k) pn[3 * c + k] = cb_r(d)[3 * c + k] + beta[k] * p[3 * c + k];
  cb_pz(d)[c] = d.con_n[c] * pn[3 * c + 2];
}

// thread per candidate: the impulse parts of -G^T w for the y correction;
// residual update r <- r - G^T w at the candidate's vertex (every vertex is
// at most one candidate) and nu <- w (reset: the step's first projection or
// a restart) or nu + w. Masked rows have w = 0 and change nothing.
__device__ __forceinline__ void proj_impulse(const Dev& d, int c, bool reset) {
  const double wx = cb_x(d)[3 * c], wy = cb_x(d)[3 * c + 1], wz = cb_x(d)[3 * c + 2];
  cb_nxy(d)[2 * c] = -wx;
  cb_nxy(d)[2 * c + 1] = -wy;
  cb_nz(d)[c] = -wz;
  const size_t o = 3 * (size_t)d.con_v[c];
  d.r[o] -= wx;
  d.r[o + 1] -= wy;
  d.r[o + 2] -= d.con_n[c] * wz;
  double* nu = cb_nu(d) + 3 * (size_t)c;
  nu[0] = reset ? wx : nu[0] + wx;
  nu[1] = reset ? wy : nu[1] + wy;
  nu[2] = reset ? wz : nu[2] + wz;
}

}  // namespace pdk
