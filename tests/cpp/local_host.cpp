// The library's local step (pd_local.cuh: per element F, SVD, corotated or
// Neo-Hookean projection, the composite's or the barrier's, corner forces) compiled as host C++ and run over a
// whole mesh from a host-side Dev record, for the CPU parity test against the
// oracle's local step and scatter.
#define __device__
#define __forceinline__ inline
#include <vector>

#include "../../paper_2605_14526_b300/csrc/pd_local.cuh"

using namespace pdk;

extern "C" {
// tets [n_e][4]; Bm [n_e][9] (Dm^-1 row-major); coef [n_e] (w_e V_e); x
// [n_v][3]; out [n_e][12] corner forces in FP64; fp64 selects the local
// step's precision; rot_share is a = 2 mu/(2 mu + lambda) of models 2 and 3,
// bar_r = mu/lambda inside the log-volume barrier's prox (model 3).
// Every element starts cold (no stored sigma*).
void local_step_host(int fp64, int model, int n_e, const int* tets, const double* Bm, const double* coef,
                     double mu_bar, double lam_bar, double k_bar, double rot_share, double bar_r, const double* x, double* out) {
  std::vector<float> Bm32(9 * (size_t)n_e), coef32(n_e), sstar(6 * (size_t)n_e, 0.0f), c32(12 * (size_t)n_e);
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
  d.sstar = sstar.data();
  if (fp64) {
    d.contrib = out;
    for (int e = 0; e < n_e; ++e) local_item<double>(d, e, x);
  } else {
    // the FP32 step reads the positions as float pairs (hi, lo), as the
    // iterate's writers keep them on the device
    int n_v = 0;
    for (int i = 0; i < 4 * n_e; ++i) n_v = tets[i] + 1 > n_v ? tets[i] + 1 : n_v;
    std::vector<float2> xhl(3 * (size_t)n_v);
    for (size_t i = 0; i < xhl.size(); ++i) {
      const float h = (float)x[i];
      xhl[i] = make_float2(h, (float)(x[i] - (double)h));
    }
    d.contrib = c32.data();
    for (int e = 0; e < n_e; ++e) local_item<float>(d, e, x, xhl.data());
    for (size_t i = 0; i < c32.size(); ++i) out[i] = c32[i];
  }
}
}
