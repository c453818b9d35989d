// The library's per-element math (pd_math.cuh: rotation-variant 3x3 SVD,
// Neo-Hookean stretch prox and the log-volume barrier's, 3x3 SPD inverse,
// the prox's filtered stretch Jacobian) compiled as host C++ so that the CPU tests can check it against
// numpy, scipy and the oracle. __device__ and __forceinline__ are defined
// away; everything else is the header as the GPU build compiles it.
#define __device__
#define __forceinline__ inline
#include "../../paper_2605_14526_b300/csrc/pd_math.cuh"

using namespace pdk;

template <typename T>
static void svd_n(int n, const T* F, T* U, T* s, T* V) {
  for (int i = 0; i < n; ++i) svd3<T>(F + 9 * i, U + 9 * i, s + 3 * i, V + 9 * i);
}

template <typename T>
static void prox_n(int n, const T* sF, T mu, T lam, T k, T* s, int* iters) {
  const NHMean<T> m{mu, lam, k};
  for (int i = 0; i < n; ++i) iters[i] = nh_prox<T>(sF + 3 * i, m, s + 3 * i);
}

extern "C" {
void svd3_f32(int n, const float* F, float* U, float* s, float* V) { svd_n<float>(n, F, U, s, V); }
void svd3_f64(int n, const double* F, double* U, double* s, double* V) { svd_n<double>(n, F, U, s, V); }
void nh_prox_f32(int n, const float* sF, float mu, float lam, float k, float* s, int* it) {
  prox_n<float>(n, sF, mu, lam, k, s, it);
}
void nh_prox_f64(int n, const double* sF, double mu, double lam, double k, double* s, int* it) {
  prox_n<double>(n, sF, mu, lam, k, s, it);
}
// the log-volume barrier's prox divided by its weight: mu = r, lam = k = 1,
// no deviatoric term (dv = 0), solved by the same Newton
void barrier_prox_f32(int n, const float* sF, float r, float* s, int* it) {
  NHMean<float> m{r, 1.0f, 1.0f};
  m.dv = 0.0f;
  for (int i = 0; i < n; ++i) it[i] = nh_prox<float>(sF + 3 * i, m, s + 3 * i);
}
void barrier_prox_f64(int n, const double* sF, double r, double* s, int* it) {
  NHMean<double> m{r, 1.0, 1.0};
  m.dv = 0.0;
  for (int i = 0; i < n; ++i) it[i] = nh_prox<double>(sF + 3 * i, m, s + 3 * i);
}
void barrier_jacobian_f64(int n, const double* ss, double r, double tau, double* J) {
  NHMean<double> m{r, 1.0, 1.0};
  m.dv = 0.0;
  for (int i = 0; i < n; ++i) filtered_jacobian<double>(ss + 3 * i, m, tau, J + 9 * i);
}
int spd_inv3_f64(const double* H, double* Hi) { return spd_inv3<double>(H, Hi) ? 1 : 0; }
void filtered_jacobian_f64(int n, const double* ss, double mu, double lam, double k, double tau, double* J) {
  const NHMean<double> m{mu, lam, k};
  for (int i = 0; i < n; ++i) filtered_jacobian<double>(ss + 3 * i, m, tau, J + 9 * i);
}
void filtered_jacobian_f32(int n, const float* ss, float mu, float lam, float k, float tau, float* J) {
  const NHMean<float> m{mu, lam, k};
  for (int i = 0; i < n; ++i) filtered_jacobian<float>(ss + 3 * i, m, tau, J + 9 * i);
}
}
