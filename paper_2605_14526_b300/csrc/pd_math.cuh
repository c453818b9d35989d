// Per-element math of the PD local step, templated on the arithmetic type
// (float for the FP32 local step, double for FP64).
//
//  * svd3: rotation-variant SVD F = U diag(s) V^T with U, V in SO(3). V comes
//    from cyclic Jacobi on F^T F (exact Givens angles), sorted by decreasing
//    eigenvalue; U and s come from a Givens QR of B = F V, whose diagonal is
//    the signed singular values (only the last may be negative). This is the
//    scheme of McAdams et al. 2011 (Jacobi eigenanalysis + QR), written with
//    exact rotations instead of their approximate quaternion ones.
//  * nh_prox: Newton on the Neo-Hookean stretch-space prox (Sec. 4.1,
//    eq. nh_prox_normal) with positivity and a sufficient-decrease test; the
//    same Newton solves the log-volume barrier's prox (eq. pd_log_volume).
//  * filtered_jacobian: the prox's stretch Jacobian through the
//    trust-region blend of its Hessian (Sec. 4.3, eq. tr_blend, tr_ift).
#pragma once
#include <cuda_runtime.h>

namespace pdk {

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T dlog(T x);
template <> __device__ __forceinline__ float dlog<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double dlog<double>(double x) { return log(x); }
template <typename T> __device__ __forceinline__ T dabs(T x) { return x < T(0) ? -x : x; }
template <typename T> __device__ __forceinline__ T dcbrt(T x);
template <> __device__ __forceinline__ float dcbrt<float>(float x) { return cbrtf(x); }
template <> __device__ __forceinline__ double dcbrt<double>(double x) { return cbrt(x); }
template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }

// symmetric Jacobi rotation zeroing S[p][q]; S and V row-major 3x3
template <typename T>
__device__ __forceinline__ void jacobi_pq(T* S, T* V, int p, int q) {
  const T apq = S[3 * p + q];
  if (apq == T(0)) return;
  const T app = S[3 * p + p], aqq = S[3 * q + q];
  const T theta = (aqq - app) / (T(2) * apq);
  const T at = dabs(theta);
  T t = T(1) / (at + dsqrt(at * at + T(1)));
  if (theta < T(0)) t = -t;
  const T c = T(1) / dsqrt(t * t + T(1));
  const T s = t * c;
  const int r = 3 - p - q;
  const T arp = S[3 * r + p], arq = S[3 * r + q];
  const T nrp = c * arp - s * arq, nrq = c * arq + s * arp;
  S[3 * r + p] = nrp; S[3 * p + r] = nrp;
  S[3 * r + q] = nrq; S[3 * q + r] = nrq;
  S[3 * p + p] = app - t * apq;
  S[3 * q + q] = aqq + t * apq;
  S[3 * p + q] = T(0); S[3 * q + p] = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T vp = V[3 * k + p], vq = V[3 * k + q];
    V[3 * k + p] = c * vp - s * vq;
    V[3 * k + q] = s * vp + c * vq;
  }
}

template <typename T>
__device__ __forceinline__ void swap_cols_neg(T* V, T* lam, int i, int j) {
  T tl = lam[i]; lam[i] = lam[j]; lam[j] = tl;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T a = V[3 * k + i];
    V[3 * k + i] = V[3 * k + j];
    V[3 * k + j] = -a;
  }
}

// Givens on rows p,q of B zeroing B[q][col]; U accumulates U * G^T
template <typename T>
__device__ __forceinline__ void qr_givens(T* B, T* U, int p, int q, int col) {
  const T a = B[3 * p + col], b = B[3 * q + col];
  const T r2 = a * a + b * b;
  T c = T(1), s = T(0);
  if (r2 > T(0)) {
    const T ir = T(1) / dsqrt(r2);
    c = a * ir;
    s = b * ir;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T bp = B[3 * p + k], bq = B[3 * q + k];
    B[3 * p + k] = c * bp + s * bq;
    B[3 * q + k] = -s * bp + c * bq;
    const T up = U[3 * k + p], uq = U[3 * k + q];
    U[3 * k + p] = c * up + s * uq;
    U[3 * k + q] = -s * up + c * uq;
  }
}

template <typename T>
__device__ __forceinline__ void svd3(const T* F, T* U, T* s, T* V) {
  T S[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      S[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? T(1) : T(0);
  const T eps = sizeof(T) == 4 ? T(1e-14) : T(1e-30);
  for (int sweep = 0; sweep < 8; ++sweep) {
    const T off = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
    const T dia = S[0] * S[0] + S[4] * S[4] + S[8] * S[8];
    if (off <= eps * dia) break;
    jacobi_pq(S, V, 0, 1);
    jacobi_pq(S, V, 0, 2);
    jacobi_pq(S, V, 1, 2);
  }
  T lam[3] = {S[0], S[4], S[8]};
  if (lam[0] < lam[1]) swap_cols_neg(V, lam, 0, 1);
  if (lam[0] < lam[2]) swap_cols_neg(V, lam, 0, 2);
  if (lam[1] < lam[2]) swap_cols_neg(V, lam, 1, 2);
  T B[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      B[3 * i + j] = F[3 * i] * V[j] + F[3 * i + 1] * V[3 + j] + F[3 * i + 2] * V[6 + j];
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? T(1) : T(0);
  qr_givens(B, U, 0, 1, 0);
  qr_givens(B, U, 0, 2, 0);
  qr_givens(B, U, 1, 2, 1);
  s[0] = B[0];
  s[1] = B[4];
  s[2] = B[8];
}

// ------------------------------------------------------------ Neo-Hookean

// The stretch-space prox energy k/2 ||s - sF||^2 + mu dv/2 (sum s^2 - 3)
// - mu ln J + lam/2 (ln J)^2. dv = 1: the Neo-Hookean prox with the mesh
// means (eq. nh_prox_normal). dv = 0: the log-volume barrier of eq.
// pd_log_volume divided by its weight lambda_e (mu = r = mu_e/lambda_e,
// lam = k = 1), whose Hessian is the Neo-Hookean one without the
// deviatoric term. dv multiplies exactly, so the Neo-Hookean arithmetic is
// unchanged by it.
template <typename T>
struct NHMean {
  T mu, lam, k;
  T dv = T(1);
};

template <typename T>
__device__ __forceinline__ void nh_grad(const T* s, const NHMean<T>& m, const T* sF, T* g, T& lnJ) {
  lnJ = dlog(s[0] * s[1] * s[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T inv = T(1) / s[i];
    g[i] = m.k * (s[i] - sF[i]) + m.mu * (m.dv * s[i] - inv) + m.lam * lnJ * inv;
  }
}

// H = k I + H_psi(s) (symmetric, stored as full 3x3)
template <typename T>
__device__ __forceinline__ void nh_hess(const T* s, const NHMean<T>& m, T lnJ, T* H) {
  T inv[3] = {T(1) / s[0], T(1) / s[1], T(1) / s[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[3 * i + j] = (i == j) ? m.k + m.mu * (m.dv + inv[i] * inv[i]) + m.lam * (T(1) - lnJ) * inv[i] * inv[i]
                              : m.lam * inv[i] * inv[j];
}

template <typename T>
__device__ __forceinline__ T nh_obj(const T* s, const NHMean<T>& m, const T* sF) {
  const T lnJ = dlog(s[0] * s[1] * s[2]);
  T d2 = T(0), s2 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d2 += (s[i] - sF[i]) * (s[i] - sF[i]);
    s2 += s[i] * s[i];
  }
  return T(0.5) * m.k * d2 + T(0.5) * m.mu * (m.dv * (s2 - T(3))) - m.mu * lnJ + T(0.5) * m.lam * lnJ * lnJ;
}

// inverse of symmetric 3x3 by cofactors; returns false unless positive definite
template <typename T>
__device__ __forceinline__ bool spd_inv3(const T* H, T* Hi) {
  const T c00 = H[4] * H[8] - H[5] * H[7];
  const T c01 = H[5] * H[6] - H[3] * H[8];
  const T c02 = H[3] * H[7] - H[4] * H[6];
  const T det = H[0] * c00 + H[1] * c01 + H[2] * c02;
  const T m2 = H[0] * H[4] - H[1] * H[3];
  if (!(H[0] > T(0) && m2 > T(0) && det > T(0))) return false;
  const T id = T(1) / det;
  Hi[0] = c00 * id;
  Hi[1] = (H[2] * H[7] - H[1] * H[8]) * id;
  Hi[2] = (H[1] * H[5] - H[2] * H[4]) * id;
  Hi[3] = c01 * id;
  Hi[4] = (H[0] * H[8] - H[2] * H[6]) * id;
  Hi[5] = (H[2] * H[3] - H[0] * H[5]) * id;
  Hi[6] = c02 * id;
  Hi[7] = (H[1] * H[6] - H[0] * H[7]) * id;
  Hi[8] = m2 * id;
  return true;
}

// sigma* = argmin k/2||s - sF||^2 + psi_bar(s), s > 0, Newton from s0 (> 0).
// Returns iterations.
template <typename T>
__device__ __forceinline__ int nh_prox_from(const T* sF, const NHMean<T>& m, const T* s0, T* s) {
  const bool f32 = sizeof(T) == 4;
  const T tol = f32 ? T(2e-7) : T(1e-13);
  const T loose = f32 ? T(1e-5) : T(1e-11);
#pragma unroll
  for (int i = 0; i < 3; ++i) s[i] = s0[i];
  T g[3], lnJ;   // gradient at s (the accepted trial's gradient after the first iteration)
  nh_grad(s, m, sF, g, lnJ);
  int it = 0;
  for (; it < 40; ++it) {
    const T gmax = fmax(fmax(dabs(g[0]), dabs(g[1])), dabs(g[2]));
    if (!(gmax > tol * m.k)) break;     // converged (also exits on NaN)
    T H[9], Hi[9], d[3];
    nh_hess(s, m, lnJ, H);
    bool newton = spd_inv3(H, Hi);
    if (newton) {
#pragma unroll
      for (int i = 0; i < 3; ++i) d[i] = -(Hi[3 * i] * g[0] + Hi[3 * i + 1] * g[1] + Hi[3 * i + 2] * g[2]);
      if (d[0] * g[0] + d[1] * g[1] + d[2] * g[2] >= T(0)) newton = false;
    }
    if (!newton) {
#pragma unroll
      for (int i = 0; i < 3; ++i) d[i] = -g[i] / m.k;
    }
    const T slope = d[0] * g[0] + d[1] * g[1] + d[2] * g[2];
    T t = T(1);
    for (int hh = 0; hh < 60; ++hh) {
      if (s[0] + t * d[0] > T(0) && s[1] + t * d[1] > T(0) && s[2] + t * d[2] > T(0)) break;
      t *= T(0.5);
    }
    bool ok = false;
    T trial[3];
    T f0 = T(0);
    bool have_f0 = false;
    T gt[3], lt = T(0);
    for (int hh = 0; hh < 40; ++hh) {
#pragma unroll
      for (int i = 0; i < 3; ++i) trial[i] = s[i] + t * d[i];
      nh_grad(trial, m, sF, gt, lt);
      const T gtmax = fmax(fmax(dabs(gt[0]), dabs(gt[1])), dabs(gt[2]));
      if (newton && gtmax <= T(0.5) * gmax) {
        ok = true;
        break;
      }
      if (!have_f0) {
        f0 = nh_obj(s, m, sF);
        have_f0 = true;
      }
      if (nh_obj(trial, m, sF) <= f0 + T(1e-4) * t * slope) {
        ok = true;
        break;
      }
      if (gmax <= loose * m.k) break;   // at the rounding floor of this precision
      t *= T(0.5);
    }
    if (!ok) break;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      s[i] = trial[i];
      g[i] = gt[i];
    }
    lnJ = lt;
  }
  return it;
}

// ------------------------------------------------------------ volume step
//
// The volume step of the corotated + volume composite (Sec. 4.1, with the
// corotated rotation step; Sec. 7.2 weights w_0 = 2 mu, w_1 = lambda): the
// closest point of the unit-determinant set in stretch space,
//   sigma_v = argmin 1/2 ||sigma - sigma_F||^2 s.t. sigma_1 sigma_2 sigma_3 = 1,
// on the positive sheet. Stationarity is s_i^2 - sigma_Fi s_i + nu = 0 with
// one multiplier nu; the minimiser lies on the curve where s_1 and s_2 take
// the larger root and s_3 is free (nu = s_3 (sigma_F3 - s_3)), at the one
// point of it where log(s_1 s_2 s_3) changes sign. That point is found by
// Newton in log s_3 inside a bracket that every iterate tightens, with
// geometric bisection (or bracket expansion by 4x) whenever the Newton step
// leaves the bracket or the curve's slope is not clearly positive.

// x = K^-1 r for a 4 x 4 system, Gaussian elimination with partial pivoting
template <typename T>
__device__ __forceinline__ void solve4(T (&K)[4][4], T (&r)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int p = c;
#pragma unroll
    for (int i = c + 1; i < 4; ++i)
      if (dabs(K[i][c]) > dabs(K[p][c])) p = i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T t = K[c][j];
      K[c][j] = K[p][j];
      K[p][j] = t;
    }
    const T t = r[c];
    r[c] = r[p];
    r[p] = t;
    const T inv = T(1) / K[c][c];
#pragma unroll
    for (int i = c + 1; i < 4; ++i) {
      const T f = K[i][c] * inv;
#pragma unroll
      for (int j = c; j < 4; ++j) K[i][j] -= f * K[c][j];
      r[i] -= f * r[c];
    }
  }
#pragma unroll
  for (int c = 3; c >= 0; --c) {
    T acc = r[c];
#pragma unroll
    for (int j = c + 1; j < 4; ++j) acc -= K[c][j] * r[j];
    r[c] = acc / K[c][c];
  }
}

// the Lagrange system's matrix [[I + nu Hess J, grad J], [grad J^T, 0]]
template <typename T>
__device__ __forceinline__ void vol_kkt(const T* s, T nu, T (&K)[4][4]) {
  const T g[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) K[i][j] = i == j ? T(1) : nu * s[3 - i - j];
    K[i][3] = g[i];
    K[3][i] = g[i];
  }
  K[3][3] = T(0);
}

// the larger root of s^2 - a s + nu = 0, without cancellation
template <typename T>
__device__ __forceinline__ T vol_root(T a, T nu) {
  const T q = a * a - T(4) * nu;
  const T r = dsqrt(q > T(0) ? q : T(0));
  return a >= T(0) ? T(0.5) * (a + r) : T(2) * nu / (a - r);
}

// sigma_v and its multiplier; returns iterations
template <typename T>
__device__ __forceinline__ int vol_project(const T* sF, T* s, T& nu) {
  const T tol = sizeof(T) == 4 ? T(3e-7) : T(1e-15);      // on log J
  const T btol = sizeof(T) == 4 ? T(1e-6) : T(4e-16);     // relative bracket width
  T m[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) m[i] = sF[i] > T(1e-3) ? sF[i] : T(1e-3);
  T s3 = m[2] / dcbrt(m[0] * m[1] * m[2]);   // sigma_F scaled onto J = 1
  T lo = T(0), hi = T(0);                    // log J(lo) < 0 < log J(hi); 0: not found yet
  int it = 0;
  for (; it < 60; ++it) {
    nu = s3 * (sF[2] - s3);
    s[0] = vol_root<T>(sF[0], nu);
    s[1] = vol_root<T>(sF[1], nu);
    s[2] = s3;
    const T L = dlog(s[0] * s[1] * s3);
    if (L > T(0)) hi = s3;
    else lo = s3;
    if (dabs(L) <= tol || (lo > T(0) && hi > T(0) && hi - lo <= btol * hi)) break;
    // d log J / d log s_3 along the curve (2 s_i - sigma_Fi = sqrt(sigma_Fi^2 - 4 nu))
    const T D = T(1) + s3 * (T(2) * s3 - sF[2]) *
                           (T(1) / (s[0] * (T(2) * s[0] - sF[0])) + T(1) / (s[1] * (T(2) * s[1] - sF[1])));
    T next = D > T(0.1) ? s3 * dexp(-L / D) : T(0);
    if (!(next > lo && (hi == T(0) || next < hi)))
      next = (lo > T(0) && hi > T(0)) ? dsqrt(lo * hi) : (L > T(0) ? T(0.25) * s3 : T(4) * s3);
    s3 = next;
  }
  return it;
}

// d sigma_v / d sigma_F: the leading 3 x 3 block of the inverse Lagrange
// matrix (symmetric), row-major
template <typename T>
__device__ __forceinline__ void vol_jacobian(const T* s, T nu, T* J) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T K[4][4];
    vol_kkt<T>(s, nu, K);
    T r[4] = {T(0), T(0), T(0), T(0)};
    r[c] = T(1);
    solve4<T>(K, r);
#pragma unroll
    for (int i = 0; i < 3; ++i) J[3 * i + c] = r[i];
  }
}

// same, from s0 = max(sF, 0.1)
template <typename T>
__device__ __forceinline__ int nh_prox(const T* sF, const NHMean<T>& m, T* s) {
  T s0[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) s0[i] = sF[i] > T(0.1) ? sF[i] : T(0.1);
  return nh_prox_from<T>(sF, m, s0, s);
}

// d sigma* / d sigma_F of the prox (eq. tr_ift): k H~^+ with H = k I +
// H_psi(sigma*) and H~ = (1 - tau) H + tau |H| (eq. tr_blend), as a full 3x3
// matrix. A definite H is its own blend and is inverted directly; otherwise
// H is diagonalised by Jacobi sweeps, the eigenvalues are blended, and
// directions whose blended eigenvalue is at most 1e-6 k (FP32) or 1e-12 k
// (FP64) respond with 0 (the pseudo-inverse: clamping a negative eigenvalue
// to 0 makes H~ singular).
template <typename T>
__device__ __forceinline__ void filtered_jacobian(const T* ss, const NHMean<T>& m, T tau, T* J) {
  const T lnJ = dlog(ss[0] * ss[1] * ss[2]);
  T H[9], Hi[9];
  nh_hess(ss, m, lnJ, H);
  if (spd_inv3(H, Hi)) {  // definite: every blend of eq. tr_blend is H itself
#pragma unroll
    for (int i = 0; i < 9; ++i) J[i] = m.k * Hi[i];
    return;
  }
  T S[9], Q[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    S[i] = H[i];
    Q[i] = (i % 4 == 0) ? T(1) : T(0);
  }
  for (int sweep = 0; sweep < 10; ++sweep) {
    jacobi_pq(S, Q, 0, 1);
    jacobi_pq(S, Q, 0, 2);
    jacobi_pq(S, Q, 1, 2);
  }
  const T thr = (sizeof(T) == 4 ? T(1e-6) : T(1e-12)) * m.k;
  T inv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T lam = S[4 * i];
    const T lt = (T(1) - tau) * lam + tau * dabs(lam);
    inv[i] = lt > thr ? T(1) / lt : T(0);  // pseudo-inverse: clamped directions respond with 0
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      J[3 * i + j] = m.k * (Q[3 * i] * inv[0] * Q[3 * j] + Q[3 * i + 1] * inv[1] * Q[3 * j + 1] + Q[3 * i + 2] * inv[2] * Q[3 * j + 2]);
}

}  // namespace pdk
