// The adjoint's per-element bodies (pd_bwd_elem.cuh: the differential record
// of the local step at q* and the matrix-free K p) compiled as host C++ and
// run over a whole mesh from a host-side Dev record, for the CPU parity test
// against the oracle's assembled K.
#define __device__
#define __forceinline__ inline
#include <vector>

#include "../../paper_2605_14526_b300/csrc/pd_bwd_elem.cuh"

using namespace pdk;

template <typename T>
static void run(Dev& d, int n_e, const double* qstar, double tau, const double* p, double* out) {
  std::vector<T> jac((size_t)kJacRec * n_e), c(12 * (size_t)n_e);
  d.jac = jac.data();
  d.contrib = c.data();
  for (int e = 0; e < n_e; ++e) bwd_setup_item<T>(d, e, qstar, tau);
  for (int e = 0; e < n_e; ++e) kapply_item<T>(d, e, p);
  for (size_t i = 0; i < c.size(); ++i) out[i] = (double)c[i];
}

extern "C" {
// tets [n_e][4]; Bm [n_e][9] (Dm^-1 row-major); coef [n_e] (w_e V_e);
// qstar, p [n_v][3]; out [n_e][12]: the corner contributions of K p
void kapply_host(int fp64, int model, int n_e, const int* tets, const double* Bm, const double* coef, double mu_bar,
                 double lam_bar, double k_bar, double rot_share, double bar_r, const double* qstar, double tau, const double* p,
                 double* out) {
  std::vector<float> Bm32(9 * (size_t)n_e), coef32(n_e);
  for (size_t i = 0; i < Bm32.size(); ++i) Bm32[i] = (float)Bm[i];
  for (int e = 0; e < n_e; ++e) coef32[e] = (float)coef[e];
  Dev d{};
  d.n_e = n_e;
  d.model = model;
  d.mu_bar = mu_bar;
  d.lam_bar = lam_bar;
  d.k_bar = k_bar;
  d.rot_share = rot_share;
  d.bar_r = bar_r;
  d.tets = reinterpret_cast<const int4*>(tets);
  d.Bm32 = Bm32.data();
  d.Bm64 = Bm;
  d.coef32 = coef32.data();
  d.coef64 = coef;
  if (fp64) run<double>(d, n_e, qstar, tau, p, out);
  else run<float>(d, n_e, qstar, tau, p, out);
}
}
