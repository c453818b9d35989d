// C ABI of the PD hot path: context, assembly + factorization (host, FP64),
// and the launch drivers of the forward rollout and its adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/pd_b300.h"
#include "factor.h"
#include "tsolve.h"
#include "pd_ctx.h"
#include "pd_internal.h"
#include "pd_launch.h"
#include "pd_noalloc.h"

namespace {

using namespace pdh;

const char* kVersion = "pd_b300 1.0 (sm_103a)";

struct ScalarCSR {
  std::vector<int> ptr, idx;
  std::vector<double> val;
};

// scalar PD operator pieces from per-element coefficients c_e (N N^T blocks)
void assemble_scalar(const pd_ctx* c, const std::vector<double>& ce, const std::vector<double>& diag,
                     std::vector<std::map<int, double>>& rows) {
  rows.assign(c->n_v, {});
  for (int e = 0; e < c->n_e; ++e) {
    const double* gN = &c->Bm[9 * (size_t)e];
    double G[4][3];
    for (int j = 0; j < 3; ++j) {
      G[1][j] = gN[j];
      G[2][j] = gN[3 + j];
      G[3][j] = gN[6 + j];
      G[0][j] = -(G[1][j] + G[2][j] + G[3][j]);
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const double v = ce[e] * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
        rows[c->tets[4 * e + a]][c->tets[4 * e + b]] += v;
      }
  }
  for (int v = 0; v < c->n_v; ++v)
    if (!diag.empty()) rows[v][v] += diag[v];
}

int run_until(pd_ctx* c, cudaStream_t s, const int* d_flag, int max_iter, int chunk,
              const std::function<void()>& one) {
  int launched = 0, slot = 0;
  bool pending = false;
  int prev = 0;
  while (launched < max_iter) {
    for (int i = 0; i < chunk && launched < max_iter; ++i, ++launched) one();
    CK(cudaMemcpyAsync(&c->h_flag[slot], d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev[slot], s));
    if (chunk == 1) {  // synchronous check: nothing launched past the last iteration
      CK(cudaEventSynchronize(c->ev[slot]));
      if (c->h_flag[slot]) return PD_OK;
      continue;
    }
    if (pending) {
      CK(cudaEventSynchronize(c->ev[prev]));
      if (c->h_flag[prev]) return PD_OK;
    }
    pending = true;
    prev = slot;
    slot ^= 1;
  }
  if (pending) CK(cudaEventSynchronize(c->ev[prev]));
  return PD_OK;
}

cudaEvent_t prof_event(pd_ctx* c) {
  if (c->prof_used == c->prof_ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof_ev.push_back(e);
  }
  return c->prof_ev[c->prof_used++];
}

// harvest the recorded pairs (stream already synchronised)
void prof_harvest(pd_ctx* c, int T) {
  std::vector<int> cnt(2 * (size_t)T, 0);
  if (cudaMemcpy(cnt.data(), c->phase_count, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    cudaGetLastError();
  for (size_t p = 0; 2 * p + 1 < c->prof_used; ++p) {
    const int kind = c->prof_kind[p], t = c->prof_step[p], it = c->prof_iter[p];
    if (t < 0 || t >= T || it >= cnt[2 * (size_t)t + kind]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[2 * p], c->prof_ev[2 * p + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (kind == 0) {
      c->prof.local_ms += ms;
      c->prof.local_launches++;
    } else {
      c->prof.solve_ms += ms;
      c->prof.solve_launches++;
    }
  }
  c->prof_used = 0;
  c->prof_kind.clear();
  c->prof_step.clear();
  c->prof_iter.clear();
}

}  // namespace

extern "C" {

const char* pd_version(void) { return kVersion; }

void pd_default_options(pd_options* o) {
  if (!o) return;
  o->aa_m = 5;
  o->k_max = 200;
  o->fixed_iters = 0;
  o->local_fp32 = 1;
  o->tr_mode = PD_TR_ADAPT;
  o->adj_max_iters = 1000;
  o->persistent = 1;
  o->eps_step = 1e-8;
  o->eps_res = 1e-6;
  o->eps_abs = 1e-12;
  o->eps_tr = 0.1;
  o->adj_tol = 1e-9;
  o->escalate_window = 100;
  o->warm_start = 0;
  o->solve_fp64 = 0;
  o->wait_polls = 0;
  o->solve_mode = PD_SOLVE_AUTO;
}

const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pd_create(const pd_mesh* mesh, const pd_material* mat, double dt, const pd_options* opt, pd_ctx** out) {
  pd_ctx* c = nullptr;
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (!mesh || !mat || !mesh->X || !mesh->tets || !mat->E) return PD_ERR_ARG;
  if (mesh->n_v < 4 || mesh->n_e < 1 || !(dt > 0)) return PD_ERR_ARG;
  if (!(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->density > 0)) return PD_ERR_ARG;
  if (mat->model != PD_COROTATED && mat->model != PD_NEOHOOKEAN && mat->model != PD_COROT_VOLUME &&
      mat->model != PD_COROT_LOGVOL)
    return PD_ERR_ARG;
  if (mat->model == PD_COROT_LOGVOL && !(mat->nu > 0.0)) return PD_ERR_ARG;   // the barrier's weight lambda_e > 0
  c = new pd_ctx();
  c->n_v = mesh->n_v;
  c->n_e = mesh->n_e;
  c->X.assign(mesh->X, mesh->X + 3 * (size_t)mesh->n_v);
  c->tets.assign(mesh->tets, mesh->tets + 4 * (size_t)mesh->n_e);
  c->pinned.assign(mesh->n_v, 0);
  if (mesh->pinned)
    for (int v = 0; v < mesh->n_v; ++v) c->pinned[v] = mesh->pinned[v] ? 1 : 0;
  c->E.assign(mat->E, mat->E + mesh->n_e);
  c->nu = mat->nu;
  c->density = mat->density;
  c->alpha = mat->alpha;
  c->beta0 = mat->beta0;
  for (int i = 0; i < 3; ++i) c->g[i] = mat->gravity[i];
  c->model = mat->model;
  c->dt = dt;
  if (opt) c->opt = *opt; else pd_default_options(&c->opt);
  *out = c;
  if (c->opt.aa_m < 0 || c->opt.aa_m > pdk::kMaxAA) return fail(c, PD_ERR_ARG, "aa_m must be in [0, %d]", pdk::kMaxAA);
  if (c->opt.k_max < 1 || c->opt.adj_max_iters < 1) return fail(c, PD_ERR_ARG, "k_max and adj_max_iters must be >= 1");
  if (c->opt.solve_mode < PD_SOLVE_AUTO || c->opt.solve_mode > PD_SOLVE_T)
    return fail(c, PD_ERR_ARG, "solve_mode must be PD_SOLVE_AUTO, PD_SOLVE_S or PD_SOLVE_T");
  for (size_t i = 0; i < c->tets.size(); ++i)
    if (c->tets[i] < 0 || c->tets[i] >= c->n_v) return fail(c, PD_ERR_ARG, "tet index out of range at %zu", i);
  for (int e = 0; e < c->n_e; ++e)
    if (!(c->E[e] > 0)) return fail(c, PD_ERR_ARG, "E[%d] must be > 0", e);
  c->n_f = 0;
  for (int v = 0; v < c->n_v; ++v) c->n_f += c->pinned[v] ? 0 : 1;
  if (c->n_f == 0) return fail(c, PD_ERR_ARG, "every vertex is pinned");

  // rest shape: Dm = [X1-X0, X2-X0, X3-X0], V = det/6, Bm = Dm^-1, lumped mass
  c->Bm.assign(9 * (size_t)c->n_e, 0.0);
  c->vol.assign(c->n_e, 0.0);
  c->mass.assign(c->n_v, 0.0);
  for (int e = 0; e < c->n_e; ++e) {
    const int* t = &c->tets[4 * e];
    double D[9];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) D[3 * i + a] = c->X[3 * t[a + 1] + i] - c->X[3 * t[0] + i];
    const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                       D[2] * (D[3] * D[7] - D[4] * D[6]);
    if (!(det > 0)) return fail(c, PD_ERR_MESH, "element %d has non-positive rest volume", e);
    const double id = 1.0 / det;
    double* B = &c->Bm[9 * (size_t)e];
    B[0] = (D[4] * D[8] - D[5] * D[7]) * id;
    B[1] = (D[2] * D[7] - D[1] * D[8]) * id;
    B[2] = (D[1] * D[5] - D[2] * D[4]) * id;
    B[3] = (D[5] * D[6] - D[3] * D[8]) * id;
    B[4] = (D[0] * D[8] - D[2] * D[6]) * id;
    B[5] = (D[2] * D[3] - D[0] * D[5]) * id;
    B[6] = (D[3] * D[7] - D[4] * D[6]) * id;
    B[7] = (D[1] * D[6] - D[0] * D[7]) * id;
    B[8] = (D[0] * D[4] - D[1] * D[3]) * id;
    c->vol[e] = det / 6.0;
    for (int a = 0; a < 4; ++a) c->mass[t[a]] += c->density * c->vol[e] / 4.0;
  }
  // vertex -> incident corners
  std::vector<int> inc_ptr(c->n_v + 1, 0), inc_idx(4 * (size_t)c->n_e);
  for (int e = 0; e < c->n_e; ++e)
    for (int a = 0; a < 4; ++a) inc_ptr[c->tets[4 * e + a] + 1]++;
  for (int v = 0; v < c->n_v; ++v) inc_ptr[v + 1] += inc_ptr[v];
  {
    std::vector<int> fillp(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int e = 0; e < c->n_e; ++e)
      for (int a = 0; a < 4; ++a) inc_idx[fillp[c->tets[4 * e + a]]++] = 4 * e + a;
  }

  CK(cudaGetDevice(&c->device));
  Dev& d = c->d;
  d.n_v = c->n_v;
  d.n_e = c->n_e;
  d.n_f = c->n_f;
  d.model = c->model;
  std::vector<int4> t4(c->n_e);
  for (int e = 0; e < c->n_e; ++e) t4[e] = make_int4(c->tets[4 * e], c->tets[4 * e + 1], c->tets[4 * e + 2], c->tets[4 * e + 3]);
  std::vector<float> Bm32(c->Bm.begin(), c->Bm.end());
  std::vector<uint8_t> pin = c->pinned;
  int r;
  int4* tets_d; float* bm32; double* bm64; double* vol_d; double* X_d; double* mass_d; uint8_t* pin_d;
  int* ip; int* ii;
  if ((r = upload(c, &tets_d, t4)) || (r = upload(c, &bm32, Bm32)) || (r = upload(c, &bm64, c->Bm)) ||
      (r = upload(c, &vol_d, c->vol)) || (r = upload(c, &X_d, c->X)) || (r = upload(c, &mass_d, c->mass)) ||
      (r = upload(c, &pin_d, pin)) || (r = upload(c, &ip, inc_ptr)) || (r = upload(c, &ii, inc_idx)))
    return r;
  d.tets = tets_d; d.Bm32 = bm32; d.Bm64 = bm64; d.vol = vol_d; d.X = X_d; d.mass = mass_d; d.pinned = pin_d;
  d.inc_ptr = ip; d.inc_idx = ii;
  const size_t nv3 = 3 * (size_t)c->n_v;
  double** vecs[] = {&d.q, &d.qprev, &d.qhat, &d.gprev, &d.qt, &d.qtil, &d.b0, &d.b, &d.bprev, &d.mu, &d.r,
                     &d.z, &d.pdir, &d.pdir2, &d.w, &d.qbar, &d.gq, &d.gv, &c->sq, &c->sv};
  for (double** p : vecs)
    if ((r = dalloc(c, p, nv3))) return r;
  if ((r = dalloc(c, &d.bperm, 3 * (size_t)c->n_f)) || (r = dalloc(c, &d.y, 3 * (size_t)c->n_f))) return r;  // float2
  if ((r = dalloc(c, &d.qhl, nv3))) return r;
  d.sq = c->sq;
  d.sv = c->sv;
  const int m = std::max(c->opt.aa_m, 1);
  if ((r = dalloc(c, &d.dQG, (size_t)m * nv3)) || (r = dalloc(c, &d.dG, (size_t)m * nv3))) return r;
  double* contrib;
  double* jac;
  double* sstar;
  if ((r = dalloc(c, &contrib, 12 * (size_t)c->n_e)) || (r = dalloc(c, &jac, (size_t)pdk::kJacRec * c->n_e)) ||
      (r = dalloc(c, &sstar, 3 * (size_t)c->n_e)))
    return r;
  d.contrib = contrib;
  d.jac = jac;
  d.sstar = sstar;
  if ((r = dalloc(c, &d.red, std::max((size_t)pdk::max_reduction_blocks(c->n_v, c->n_e) * pdk::kRed,
                                      (size_t)2 * pdk::kRedRep * pdk::kRedRows * pdk::kRedTeam))))
    return r;
  if ((r = dalloc(c, &d.dw, c->n_e)) || (r = dalloc(c, &d.dw1, c->n_e)) || (r = dalloc(c, &d.dbeta, c->n_e))) return r;
  if ((r = dalloc(c, &d.ctrl, 1))) return r;
  CK(cudaMemset(d.ctrl, 0, sizeof(Ctrl)));
  CK(cudaMemset(d.dQG, 0, sizeof(double) * m * nv3));
  CK(cudaMemset(d.dG, 0, sizeof(double) * m * nv3));
  CK(cudaHostAlloc(&c->h_flag, 2 * sizeof(int), cudaHostAllocDefault));
  CK(cudaEventCreateWithFlags(&c->ev[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev[1], cudaEventDisableTiming));
  return PD_OK;
}

int pd_set_contacts(pd_ctx* c, const pd_contact_desc* desc) {
  if (!c) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "pd_set_contacts is single-instance only");
  c->con_ground.clear();
  c->con_box.clear();
  c->con_att.clear();
  c->con_att_p0.clear();
  c->con_att_tr.clear();
  c->con = pd_contact_desc{};
  c->factored = false;
  if (!desc || desc->n_ground + desc->n_box + desc->n_attach == 0) return PD_OK;
  if (desc->n_ground < 0 || desc->n_box < 0 || desc->n_attach < 0 || (desc->n_ground && !desc->ground) ||
      (desc->n_box && !desc->box) || (desc->n_attach && (!desc->attach || !desc->attach_target)))
    return fail(c, PD_ERR_ARG, "contact candidate arrays");
  if (desc->n_box > 0 && desc->box_steps < 1) return fail(c, PD_ERR_ARG, "box_steps must be >= 1");
  if (desc->n_attach > 0 && desc->attach_travel && desc->attach_steps < 1)
    return fail(c, PD_ERR_ARG, "attach_steps must be >= 1");
  if (!(desc->mu >= 0)) return fail(c, PD_ERR_ARG, "mu must be >= 0");
  std::vector<char> seen(c->n_v, 0);
  auto take = [&](const int32_t* p, int n, std::vector<int>& out) -> int {
    for (int i = 0; i < n; ++i) {
      const int v = p[i];
      if (v < 0 || v >= c->n_v) return fail(c, PD_ERR_ARG, "contact vertex %d out of range", v);
      if (c->pinned[v]) return fail(c, PD_ERR_ARG, "contact vertex %d is pinned", v);
      if (seen[v]) return fail(c, PD_ERR_ARG, "contact vertex %d listed twice", v);
      seen[v] = 1;
      out.push_back(v);
    }
    return PD_OK;
  };
  int r;
  if ((r = take(desc->ground, desc->n_ground, c->con_ground)) || (r = take(desc->box, desc->n_box, c->con_box)) ||
      (r = take(desc->attach, desc->n_attach, c->con_att))) {
    c->con_ground.clear();
    c->con_box.clear();
    c->con_att.clear();
    return r;
  }
  for (int i = 0; i < 3 * desc->n_attach; ++i) {
    const double p = desc->attach_target[i], tr = desc->attach_travel ? desc->attach_travel[i] : 0.0;
    if (!std::isfinite(p) || !std::isfinite(tr)) {
      c->con_ground.clear();
      c->con_box.clear();
      c->con_att.clear();
      return fail(c, PD_ERR_ARG, "attachment target %d is not finite", i / 3);
    }
    c->con_att_p0.push_back(p);
    c->con_att_tr.push_back(tr);
  }
  c->con = *desc;
  c->con.ground = nullptr;
  c->con.box = nullptr;
  c->con.attach = nullptr;
  c->con.attach_target = nullptr;
  c->con.attach_travel = nullptr;
  if (c->con.attach_steps < 1) c->con.attach_steps = 1;
  if (!(c->con.tol > 0)) c->con.tol = 1e-12;
  if (c->con.max_iters <= 0) c->con.max_iters = 2000;
  return PD_OK;
}

int pd_set_materials(pd_ctx* c, const double* E, double nu) {
  if (!c || !E) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "a batch context takes pd_set_materials_batch");
  if (!(nu > -1.0 && nu < 0.5)) return fail(c, PD_ERR_ARG, "nu must be in (-1, 0.5)");
  if (c->model == PD_COROT_LOGVOL && !(nu > 0.0)) return fail(c, PD_ERR_ARG, "the log-volume barrier needs nu > 0");
  for (int e = 0; e < c->n_e; ++e)
    if (!(E[e] > 0)) return fail(c, PD_ERR_ARG, "E[%d] must be > 0", e);
  c->E.assign(E, E + c->n_e);
  c->nu = nu;
  c->factored = false;
  return PD_OK;
}

int pd_factor(pd_ctx* c) {
  if (!c) return PD_ERR_ARG;
  if (c->batch) return batch_factor(c);
  auto t0 = std::chrono::steady_clock::now();
  CK(cudaSetDevice(c->device));
  for (void* p : c->factor_allocs) cudaFree(p);
  c->factor_allocs.clear();
  c->factored = false;
  const int n_v = c->n_v, n_e = c->n_e;
  const double h = c->dt;
  // materials (eq. lame, pd_weight, rayleigh; Sec. 7.2)
  std::vector<double> mu(n_e), lam(n_e), w(n_e), beta(n_e), coef(n_e), ce(n_e), cb(n_e);
  double mu_ref = 0, mu_bar = 0, lam_bar = 0, k_bar = 0;
  for (int e = 0; e < n_e; ++e) {
    mu[e] = c->E[e] / (2.0 * (1.0 + c->nu));
    lam[e] = c->E[e] * c->nu / ((1.0 + c->nu) * (1.0 - 2.0 * c->nu));
    w[e] = 2.0 * mu[e] + (c->model != PD_COROTATED ? lam[e] : 0.0);   // composite: w_0 + w_1 = 2 mu + lambda
    mu_ref = std::max(mu_ref, mu[e]);
    mu_bar += mu[e];
    lam_bar += lam[e];
    k_bar += w[e];
  }
  mu_bar /= n_e;
  lam_bar /= n_e;
  k_bar /= n_e;
  for (int e = 0; e < n_e; ++e) {
    beta[e] = c->beta0 * mu[e] / mu_ref;
    coef[e] = w[e] * c->vol[e];
    ce[e] = (w[e] + beta[e] / h) * c->vol[e];
    cb[e] = beta[e] * c->vol[e];
  }
  std::vector<double> diag(n_v);
  for (int v = 0; v < n_v; ++v) diag[v] = (1.0 + c->alpha * h) * c->mass[v] / (h * h);
  std::vector<std::map<int, double>> Arows, Brows;
  assemble_scalar(c, ce, diag, Arows);
  assemble_scalar(c, cb, {}, Brows);
  // free-local numbering
  std::vector<int> f2v, v2f(n_v, -1);
  for (int v = 0; v < n_v; ++v)
    if (!c->pinned[v]) {
      v2f[v] = (int)f2v.size();
      f2v.push_back(v);
    }
  const int nf = (int)f2v.size();
  pdf::SymCSR Aff;
  Aff.n = nf;
  Aff.ptr.assign(nf + 1, 0);
  std::vector<double> cA(3 * (size_t)n_v, 0.0);
  ScalarCSR Ad, Bd;
  Ad.ptr.assign(n_v + 1, 0);
  Bd.ptr.assign(n_v + 1, 0);
  for (int v = 0; v < n_v; ++v) {
    if (!c->pinned[v]) {
      for (auto& kv : Arows[v]) {
        if (c->pinned[kv.first]) {
          for (int i = 0; i < 3; ++i) cA[3 * v + i] += kv.second * c->X[3 * kv.first + i];
        } else {
          Aff.idx.push_back(v2f[kv.first]);
          Aff.val.push_back(kv.second);
          Ad.idx.push_back(kv.first);
          Ad.val.push_back(kv.second);
        }
      }
      for (auto& kv : Brows[v]) {
        Bd.idx.push_back(kv.first);
        Bd.val.push_back(kv.second);
      }
      Aff.ptr[v2f[v] + 1] = (int64_t)Aff.idx.size();
    }
    Ad.ptr[v + 1] = (int)Ad.idx.size();
    Bd.ptr[v + 1] = (int)Bd.idx.size();
  }
  // ordering (geometry-only, cached) + symbolic + numeric
  if (!c->have_order) {
    std::vector<double> xyz(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f)
      for (int i = 0; i < 3; ++i) xyz[3 * f + i] = c->X[3 * f2v[f] + i];
    c->order_perm = pdf::nested_dissection(nf, Aff.ptr, Aff.idx, xyz.data(), 32);
    c->have_order = true;
  }
  pdf::symbolic(c->fac, Aff, c->order_perm);
  int64_t bad = pdf::numeric(c->fac, Aff);
  if (bad) return fail(c, PD_ERR_NOT_SPD, "non-positive pivot at elimination position %lld", (long long)(bad - 1));
  // self-check of the factor on one right-hand side
  {
    std::vector<double> b(nf), x(nf), ax(nf, 0.0);
    for (int i = 0; i < nf; ++i) b[i] = std::sin(0.37 * i + 1.0);
    pdf::solve_host(c->fac, b.data(), x.data());
    double rn = 0, bn = 0;
    for (int i = 0; i < nf; ++i) {
      for (int64_t p = Aff.ptr[i]; p < Aff.ptr[i + 1]; ++p) ax[i] += Aff.val[p] * x[Aff.idx[p]];
      rn += (ax[i] - b[i]) * (ax[i] - b[i]);
      bn += b[i] * b[i];
    }
    if (!(std::sqrt(rn) <= 1e-8 * std::sqrt(bn))) return fail(c, PD_ERR_NOT_SPD, "factor residual %g", std::sqrt(rn / bn));
  }
  c->nnz_S = pdf::inverse_factor_nnz(c->fac);
  // solve mode: products with S, or level-scheduled solves with L (mode T)
  const bool has_con = !c->con_ground.empty() || !c->con_box.empty() || !c->con_att.empty();
  int mode = c->opt.solve_mode;
  if (mode == PD_SOLVE_T && has_con) return fail(c, PD_ERR_ARG, "solve mode T does not support contacts");
  // automatic choice: S while its stream stays near the L2 size (2 barriers
  // per solve, latency-bound meshes), T once S is both large (more than 8M
  // entries, 160 MB a solve) and several times the factor
  if (mode == PD_SOLVE_AUTO)
    mode = !has_con && ((c->nnz_S > 8000000 && c->nnz_S > 4 * c->fac.nnz_L) || c->nnz_S > (int64_t)2147483647)
               ? PD_SOLVE_T
               : PD_SOLVE_S;
  const bool tmode = mode == PD_SOLVE_T;
  if (!tmode && c->nnz_S > (int64_t)2147483647)
    return fail(c, PD_ERR_TOO_LARGE, "nnz(S) = %lld exceeds 2^31-1 (solve mode T does not store S)", (long long)c->nnz_S);
  std::vector<int64_t> s_rowptr, st_ptr;
  std::vector<double> s_val, st_val;
  std::vector<int> st_idx;
  pdf::TSolve ts;
  if (tmode) {
    pdf::build_tsolve(c->fac, ts);
    // host check of the sweeps against the factor's own solve (3 right-hand sides)
    std::vector<double> b3(3 * (size_t)nf), x3(3 * (size_t)nf), b1(nf), x1(nf);
    for (size_t i = 0; i < b3.size(); ++i) b3[i] = std::cos(0.731 * (double)i + 0.2);
    pdf::tsolve_host(ts, b3.data(), x3.data());   // positions in, positions out
    double en = 0, xn = 0;
    for (int a = 0; a < 3; ++a) {
      for (int k = 0; k < nf; ++k) b1[c->fac.perm[k]] = b3[3 * (size_t)k + a];
      pdf::solve_host(c->fac, b1.data(), x1.data());
      for (int k = 0; k < nf; ++k) {
        const double dx = x3[3 * (size_t)k + a] - x1[c->fac.perm[k]];
        en += dx * dx;
        xn += x1[c->fac.perm[k]] * x1[c->fac.perm[k]];
      }
    }
    if (!(std::sqrt(en) <= 1e-10 * std::sqrt(xn)))
      return fail(c, PD_ERR_NUMERIC, "mode T host check: relative difference %g from the factor's solve", std::sqrt(en / xn));
  } else {
    pdf::inverse_factor(c->fac, s_rowptr, s_val, st_ptr, st_idx, st_val);
  }
  // skyline segments of at most kSegLen entries, one warp each; the segments
  // of a split row own consecutive partial slots
  std::vector<int4> seg;
  int n_slot = 0;
  for (int i = 0; i < nf && !tmode; ++i) {
    const int len = i - c->fac.first_desc[i] + 1;
    const int ns = (len + pdk::kSegLen - 1) / pdk::kSegLen;
    for (int s = 0; s < ns; ++s)
      seg.push_back(make_int4(i, s * pdk::kSegLen, std::min(pdk::kSegLen, len - s * pdk::kSegLen), ns > 1 ? 1 + n_slot : 0));
    if (ns > 1) n_slot += ns;
  }
  // S and S^T as double-float pairs for the device products
  auto split = [](const std::vector<double>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float h = (float)v[i];
      o[i] = make_float2(h, (float)(v[i] - (double)h));
    }
    return o;
  };
  const std::vector<float2> s_hl = split(s_val), st_hl = split(st_val);
  double *sv64 = nullptr, *stv64 = nullptr;
  // contact contexts keep the products in FP64: W is formed from the FP64
  // factor, and the adjoint's projection needs the device's A^-1 to agree
  // with it (with double-float products its projected CG does not settle)
  const bool s64 = c->opt.solve_fp64 || has_con;
  if (s64 && !tmode) {
    int r0;
    if ((r0 = upload(c, &sv64, s_val, true)) || (r0 = upload(c, &stv64, st_val, true))) return r0;
  }
  std::vector<double>().swap(s_val);
  std::vector<double>().swap(st_val);
  std::vector<int> iperm_v(n_v, -1), perm_v(nf);
  for (int k = 0; k < nf; ++k) {
    perm_v[k] = f2v[c->fac.perm[k]];
    iperm_v[perm_v[k]] = k;
  }
  Dev& d = c->d;
  int r;
  std::vector<float> coef32(coef.begin(), coef.end());
  float* c32; double *c64, *mu_d, *lam_d, *E_d, *cA_d, *Av, *Bv;
  float2 *sv, *stv, *spart, *spart_na;
  int *scnt, *scnt_na;
  int *iperm_d, *perm_d, *sfirst, *sti, *Ap, *Ai, *Bp, *Bi;
  int64_t *srp, *stp;
  int4* seg_d;
  if ((r = upload(c, &c32, coef32, true)) || (r = upload(c, &c64, coef, true)) || (r = upload(c, &mu_d, mu, true)) ||
      (r = upload(c, &lam_d, lam, true)) || (r = upload(c, &E_d, c->E, true)) || (r = upload(c, &cA_d, cA, true)) ||
      (r = upload(c, &iperm_d, iperm_v, true)) || (r = upload(c, &perm_d, perm_v, true)) ||
      (r = upload(c, &srp, s_rowptr, true)) || (r = upload(c, &sfirst, c->fac.first_desc, true)) ||
      (r = upload(c, &sv, s_hl, true)) || (r = upload(c, &seg_d, seg, true)) || (r = upload(c, &stp, st_ptr, true)) ||
      (r = upload(c, &sti, st_idx, true)) || (r = upload(c, &stv, st_hl, true)) || (r = upload(c, &Ap, Ad.ptr, true)) ||
      (r = upload(c, &Ai, Ad.idx, true)) || (r = upload(c, &Av, Ad.val, true)) || (r = upload(c, &Bp, Bd.ptr, true)) ||
      (r = upload(c, &Bi, Bd.idx, true)) || (r = upload(c, &Bv, Bd.val, true)) ||
      (r = dalloc(c, &spart, 3 * (size_t)n_slot, true)) || (r = dalloc(c, &spart_na, 3 * (size_t)n_slot, true)) ||
      (r = upload(c, &scnt, std::vector<int>(std::max(n_slot, 1), 0), true)) ||
      (r = upload(c, &scnt_na, std::vector<int>(std::max(n_slot, 1), 0), true)))
    return r;
  // warm-start feature: log10 of the volume-weighted mean E around each vertex
  {
    std::vector<double> num(n_v, 0.0), den(n_v, 0.0);
    for (int e = 0; e < n_e; ++e)
      for (int a = 0; a < 4; ++a) {
        num[c->tets[4 * e + a]] += c->vol[e] * c->E[e];
        den[c->tets[4 * e + a]] += c->vol[e];
      }
    std::vector<float> le(n_v, 0.f);
    for (int v = 0; v < n_v; ++v) le[v] = den[v] > 0 ? (float)std::log10(num[v] / den[v] / 1e5) : 0.f;
    float* le_d;
    if ((r = upload(c, &le_d, le, true))) return r;
    d.logE = le_d;
  }
  d.coef32 = c32; d.coef64 = c64; d.mu_e = mu_d; d.lam_e = lam_d; d.E = E_d; d.cA = cA_d;
  d.iperm = iperm_d; d.perm = perm_d; d.s_rowptr = srp; d.s_first = sfirst; d.s_hl = sv; d.s_seg = seg_d;
  d.sfp64 = (s64 || tmode) ? 1 : 0; d.s_val64 = sv64; d.st_val64 = stv64;
  d.tmode = tmode ? 1 : 0;
  d.t_nlev = 0;
  if (tmode) {
    auto units = [](const std::vector<int>& u) {
      std::vector<int4> o(u.size() / 4);
      for (size_t i = 0; i < o.size(); ++i) o[i] = make_int4(u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3]);
      return o;
    };
    const std::vector<int4> uf = units(ts.unit_f), ub = units(ts.unit_b);
    std::vector<int2> wf(ts.wnode_f.size() / 2);
    for (size_t i = 0; i < wf.size(); ++i) wf[i] = make_int2(ts.wnode_f[2 * i], ts.wnode_f[2 * i + 1]);
    int *c0d, *ncd, *nbd, *bld, *gpd, *gsd, *lfd, *lbd, *lwfd, *lwbd, *wbd;
    int2* wfd;
    int64_t *bod, *pod, *god;
    double *prd, *pcd, *Ud, *xd;
    int4 *ufd, *ubd;
    if ((r = upload(c, &c0d, ts.c0, true)) || (r = upload(c, &ncd, ts.nc, true)) || (r = upload(c, &nbd, ts.nb, true)) ||
        (r = upload(c, &bod, ts.boff, true)) || (r = upload(c, &bld, ts.below, true)) ||
        (r = upload(c, &pod, ts.poff, true)) || (r = upload(c, &prd, ts.prow, true)) ||
        (r = upload(c, &pcd, ts.pcol, true)) || (r = upload(c, &god, ts.goff, true)) ||
        (r = upload(c, &gpd, ts.gptr, true)) || (r = upload(c, &gsd, ts.gsrc, true)) ||
        (r = upload(c, &lfd, ts.lev_f, true)) || (r = upload(c, &lbd, ts.lev_b, true)) ||
        (r = upload(c, &lwfd, ts.lev_wf, true)) || (r = upload(c, &lwbd, ts.lev_wb, true)) ||
        (r = upload(c, &ufd, uf, true)) || (r = upload(c, &ubd, ub, true)) || (r = upload(c, &wfd, wf, true)) ||
        (r = upload(c, &wbd, ts.wnode_b, true)) || (r = dalloc(c, &Ud, 3 * (size_t)ts.u_rows, true)) ||
        (r = dalloc(c, &xd, 3 * (size_t)nf, true)))
      return r;
    d.t_nlev = ts.n_level;
    d.t_c0 = c0d; d.t_nc = ncd; d.t_nb = nbd; d.t_boff = bod; d.t_below = bld; d.t_poff = pod;
    d.t_prow = prd; d.t_pcol = pcd; d.t_goff = god; d.t_gptr = gpd; d.t_gsrc = gsd;
    d.t_lev_f = lfd; d.t_lev_b = lbd; d.t_lev_wf = lwfd; d.t_lev_wb = lwbd; d.t_unit_f = ufd; d.t_unit_b = ubd;
    d.t_wnode_f = wfd; d.t_wnode_b = wbd;
    d.t_U = Ud; d.t_x = xd;
  }
  c->tmode = tmode;
  c->solve_nnz = tmode ? ts.entries : c->nnz_S;
  c->solve_levels = tmode ? ts.n_level : 0;
  c->tsolve_seconds = tmode ? ts.build_seconds : 0.0;
  d.spin_limit = c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : (1u << 22);
  d.n_seg = (int)seg.size(); d.st_ptr = stp; d.st_idx = sti; d.st_hl = stv;
  d.n_slot = n_slot; d.s_part = spart; d.s_cnt = scnt; d.s_part_na = spart_na; d.s_cnt_na = scnt_na;
  d.A_ptr = Ap; d.A_idx = Ai; d.A_val = Av; d.B_ptr = Bp; d.B_idx = Bi; d.B_val = Bv;
  d.n_f = nf;
  d.local_fp32 = c->opt.local_fp32 ? 1 : 0;
  d.aa_m = c->opt.aa_m; d.k_max = c->opt.k_max; d.fixed_iters = c->opt.fixed_iters; d.tr_mode = c->opt.tr_mode;
  d.adj_max_iters = c->opt.adj_max_iters;
  d.escalate = c->opt.escalate_window;
  d.warm = c->opt.warm_start;
  d.h = h; d.alpha_d = c->alpha; d.eps_step = c->opt.eps_step; d.eps_res = c->opt.eps_res; d.eps_abs = c->opt.eps_abs;
  d.eps_tr = c->opt.eps_tr; d.adj_tol = c->opt.adj_tol;
  for (int i = 0; i < 3; ++i) d.g[i] = c->g[i];
  d.mu_bar = mu_bar; d.lam_bar = lam_bar; d.k_bar = k_bar; d.mu_ref = mu_ref; d.beta0 = c->beta0; d.nu = c->nu;
  d.rot_share = (1.0 - 2.0 * c->nu) / (1.0 - c->nu);   // 2 mu / (2 mu + lambda) for any E
  d.bar_r = (1.0 - 2.0 * c->nu) / (2.0 * c->nu);      // mu / lambda for any E
  // contacts: candidates in elimination order, W = (L_A^-1)_CC by host solves
  d.n_con = 0;
  if (!c->con_ground.empty() || !c->con_box.empty() || !c->con_att.empty()) {
    std::vector<std::pair<int, int>> cand;  // (position, index into ground+box+attach)
    std::vector<int> all(c->con_ground);
    all.insert(all.end(), c->con_box.begin(), c->con_box.end());
    all.insert(all.end(), c->con_att.begin(), c->con_att.end());
    for (size_t i = 0; i < all.size(); ++i) cand.push_back({iperm_v[all[i]], (int)i});
    std::sort(cand.begin(), cand.end());
    const int K = (int)cand.size();
    const int n_gb = (int)(c->con_ground.size() + c->con_box.size());
    std::vector<int> cv(K), cp(K), cf(K), ca(K, 0);
    std::vector<double> cn(K), W((size_t)K * K), ct((size_t)6 * K, 0.0);
    for (int k = 0; k < K; ++k) {
      const int src = cand[k].second;
      cv[k] = all[src];
      cp[k] = cand[k].first;
      cn[k] = src < (int)c->con_ground.size() || src >= n_gb ? 1.0 : -1.0;   // attachments: +z rows
      cf[k] = v2f[cv[k]];
      if (src >= n_gb) {   // attachment: its target and the target's travel
        ca[k] = 1;
        for (int j = 0; j < 3; ++j) {
          ct[6 * (size_t)k + j] = c->con_att_p0[3 * (size_t)(src - n_gb) + j];
          ct[6 * (size_t)k + 3 + j] = c->con_att_tr[3 * (size_t)(src - n_gb) + j];
        }
      }
    }
#pragma omp parallel
    {
      std::vector<double> e(nf, 0.0), x(nf);
#pragma omp for schedule(dynamic, 4)
      for (int j = 0; j < K; ++j) {
        e[cf[j]] = 1.0;
        pdf::solve_host(c->fac, e.data(), x.data());
        e[cf[j]] = 0.0;
        for (int i = 0; i < K; ++i) W[(size_t)i * K + j] = x[cf[i]];
      }
    }
    for (int i = 0; i < K; ++i)   // symmetric part (W is symmetric up to rounding)
      for (int j = i + 1; j < K; ++j) {
        const double a = 0.5 * (W[(size_t)i * K + j] + W[(size_t)j * K + i]);
        W[(size_t)i * K + j] = W[(size_t)j * K + i] = a;
      }
    // largest eigenvalue by power iteration (the FISTA step is 1 / lambda_max)
    std::vector<double> u(K, 1.0), w(K);
    double lmax = 0.0;
    for (int it = 0; it < 300; ++it) {
      double nn = 0.0;
      for (int i = 0; i < K; ++i) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += W[(size_t)i * K + j] * u[j];
        w[i] = s;
        nn += s * s;
      }
      nn = std::sqrt(nn);
      double un = 0.0;
      for (int i = 0; i < K; ++i) un += u[i] * u[i];
      lmax = nn / std::sqrt(un);
      for (int i = 0; i < K; ++i) u[i] = w[i] / nn;
    }
    int *cv_d, *cp_d, *ca_d = nullptr;
    double *cn_d, *W_d, *buf_d, *ct_d = nullptr;
    if ((r = upload(c, &cv_d, cv, true)) || (r = upload(c, &cp_d, cp, true)) || (r = upload(c, &cn_d, cn, true)) ||
        (r = upload(c, &W_d, W, true)) || (r = dalloc(c, &buf_d, 14 * (size_t)K, true)))
      return r;
    if (!c->con_att.empty() && ((r = upload(c, &ca_d, ca, true)) || (r = upload(c, &ct_d, ct, true)))) return r;
    double* bwd_d;
    if ((r = dalloc(c, &bwd_d, 23 * (size_t)K, true))) return r;
    d.con_bwd = bwd_d;
    if (c->con_ckpt) cudaFree(c->con_ckpt);   // sized with the checkpoints (reserve)
    c->con_ckpt = nullptr;
    d.con_ckpt = nullptr;
    c->con_ckpt_cap = 0;
    d.n_con = K;
    d.con_v = cv_d;
    d.con_pos = cp_d;
    d.con_n = cn_d;
    d.con_att = ca_d;
    d.con_tgt = ct_d;
    d.con_att_steps = c->con.attach_steps > 0 ? c->con.attach_steps : 1;
    d.con_W = W_d;
    d.con_buf = buf_d;
    d.con_L = 1.001 * lmax;   // a little above lambda_max: the step stays below 1 / L
    {   // sticking slip tolerance: 1e-7 of the rest mesh's bounding-box diagonal
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int v = 0; v < c->n_v; ++v)
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], c->X[3 * v + k]);
          hi[k] = std::max(hi[k], c->X[3 * v + k]);
        }
      d.con_slip_tol = 1e-7 * std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                        (hi[2] - lo[2]) * (hi[2] - lo[2]));
    }
    d.con_mu = c->con.mu;
    d.con_zg = c->con.ground_z;
    d.con_zb0 = c->con.box_z0;
    d.con_travel = c->con.box_travel;
    d.con_steps = c->con.box_steps > 0 ? c->con.box_steps : 1;
    d.con_tol = c->con.tol;
    d.con_max_iters = c->con.max_iters;
  }
  c->factored = true;
  c->factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->stats.factor_seconds = c->factor_seconds;
  c->stats.factor_nnz = c->solve_nnz;
  c->stats.n_free = nf;
  c->stats.solve_mode = tmode ? PD_SOLVE_T : PD_SOLVE_S;
  c->stats.solve_levels = c->solve_levels;
  c->stats.nnz_L = c->fac.nnz_L;
  return PD_OK;
}

}  // extern "C"

namespace {

int reserve_contact(pd_ctx* c, int T) {
  if (c->d.n_con == 0 || c->con_ckpt_cap >= T) return PD_OK;
  if (c->con_ckpt) cudaFree(c->con_ckpt);
  c->con_ckpt = nullptr;
  c->con_ckpt_cap = 0;
  if (cudaMalloc(&c->con_ckpt, (size_t)T * 3 * c->d.n_con * sizeof(double)) != cudaSuccess)
    return fail(c, PD_ERR_OOM, "contact checkpoint allocation for %d steps", T);
  c->con_ckpt_cap = T;
  c->d.con_ckpt = c->con_ckpt;
  return PD_OK;
}

int reserve_single(pd_ctx* c, int T) {
  if (int r = reserve_contact(c, T)) return r;
  if (c->ckpt_cap >= T) return PD_OK;
  if (c->ckpt) cudaFree(c->ckpt);
  if (c->tau) cudaFree(c->tau);
  if (c->phase_count) cudaFree(c->phase_count);
  c->ckpt = nullptr;
  c->tau = nullptr;
  c->phase_count = nullptr;
  c->ckpt_cap = 0;
  const size_t nv3 = 3 * (size_t)c->n_v;
  if (cudaMalloc(&c->ckpt, (size_t)(T + 1) * nv3 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->tau, (size_t)T * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->phase_count, 2 * (size_t)T * sizeof(int)) != cudaSuccess)
    return fail(c, PD_ERR_OOM, "checkpoint allocation for %d steps", T);
  c->ckpt_cap = T;
  return PD_OK;
}

// reserve for an enqueue: allocation is refused while the stream is captured
int reserve_enqueue(pd_ctx* c, int T, cudaStream_t s) {
  if (c->ckpt_cap >= T && (c->d.n_con == 0 || c->con_ckpt_cap >= T)) return PD_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(c, PD_ERR_ARG, "checkpoint storage for %d steps is missing: call pd_reserve before capture", T);
  return reserve_single(c, T);
}

// co-resident grid of a persistent launch: the tuned grid if one is set, else
// SMs x blocks per SM; 0 if cooperative launch is unavailable
int grid_of(pd_ctx* c, bool bwd, int* grid) {
  const bool fp32 = c->opt.local_fp32 != 0;
  const int full = bwd ? pdk::persistent_grid_bwd(fp32, 0) : pdk::persistent_grid_max(fp32);
  *grid = 0;
  if (full <= 0) return PD_OK;
  const int want = bwd ? c->tune.bwd_grid : c->tune.fwd_grid;
  const int bps = bwd ? c->tune.bwd_blocks_per_sm : c->tune.fwd_blocks_per_sm;
  if (want > 0) {
    if (want > full) return fail(c, PD_ERR_ARG, "tuned grid %d exceeds the %d co-resident blocks", want, full);
    *grid = want;
  } else {
    *grid = bwd ? pdk::persistent_grid_bwd(fp32, bps) : pdk::persistent_grid(fp32, bps);
  }
  return PD_OK;
}

// device state of a single-instance persistent launch: the Dev record when
// it changed, the team map of direction dir when the grid changed; refused
// while the stream is captured (run once before capture)
int prepare_single(pd_ctx* c, cudaStream_t s, int dir, int grid) {
  const bool cap = capturing(s);
  const bool same_d = c->d_valid && std::memcmp(&c->d_uploaded, &c->d, sizeof(Dev)) == 0;
  if ((!c->d_dev || !same_d || c->team_grid[dir] != grid) && cap)
    return fail(c, PD_ERR_ARG, "the launch state changed since the last launch: run it once before capture");
  if (!c->d_dev) {
    const bool fp32 = c->opt.local_fp32 != 0;
    c->team_cap = std::max(std::max(pdk::persistent_grid_max(fp32), pdk::persistent_grid_bwd(fp32, 0)), 1);
    int r;
    if ((r = dalloc(c, &c->d_dev, 2)) || (r = dalloc(c, &c->d_off, 2)) || (r = dalloc(c, &c->d_team[0], c->team_cap)) ||
        (r = dalloc(c, &c->d_team[1], c->team_cap)))
      return r;
    const pdk::InstOff off[2] = {{0, 0}, {c->n_v, c->n_e}};
    CK(cudaMemcpy(c->d_off, off, sizeof(off), cudaMemcpyHostToDevice));
  }
  if (grid > c->team_cap) return fail(c, PD_ERR_ARG, "grid %d exceeds the team map (%d)", grid, c->team_cap);
  if (!same_d) {
    c->d_uploaded = c->d;
    c->d_adjoint = adjoint_dev(c->d);   // record 1: the persistent adjoint's
    CK(cudaMemcpyAsync(c->d_dev, &c->d_uploaded, sizeof(Dev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_dev + 1, &c->d_adjoint, sizeof(Dev), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    c->d_valid = true;
  }
  if (c->team_grid[dir] != grid) {
    std::vector<int4> map(grid);
    for (int b = 0; b < grid; ++b) map[b] = make_int4(0, b, grid, 0);
    CK(cudaMemcpyAsync(c->d_team[dir], map.data(), grid * sizeof(int4), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    c->team_grid[dir] = grid;
  }
  return PD_OK;
}

// memsets + the persistent forward launch (no host synchronisation)
int enqueue_fwd_single(pd_ctx* c, int T, const double* q0d, const double* v0d, const double* fd, int64_t f_stride,
                       double* qTd, double* vTd, cudaStream_t s, int grid) {
  Dev& d = c->d;
  d.ckpt = c->ckpt;
  d.tau = c->tau;
  d.phase_count = nullptr;
  d.T = 0;
  int r;
  if ((r = prepare_single(c, s, 0, grid))) return r;
  CK(cudaMemsetAsync(c->tau, 0, (size_t)T * sizeof(double), s));
  CK(cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), s));  // per-rollout statistics and flags
  CK(cudaMemsetAsync(d.sstar, 0, 3 * sizeof(double) * (size_t)c->n_e, s));  // no prox warm start across rollouts
  if (d.n_con > 0) CK(cudaMemsetAsync(d.con_buf, 0, 14 * sizeof(double) * (size_t)d.n_con, s));
  pdk::BatchFwd br;
  br.T = T;
  br.q0 = q0d;
  br.v0 = v0d;
  br.fext = fd;
  br.f_stride = f_stride;
  br.qT = qTd;
  br.vT = vTd;
  CK(pdk::launch_fwd_rollout(d.local_fp32 != 0, c->d_dev, c->d_team[0], c->d_off, br, grid, d.tmode != 0, s));
  c->launches += 1;
  c->last_T = T;
  return PD_OK;
}

int enqueue_bwd_single(pd_ctx* c, const double* dqTd, const double* dvTd, double* dq0d, double* dv0d, double* dEd,
                       double* dnud, double* dfd, int64_t df_stride, cudaStream_t s, int grid) {
  Dev& d = c->d;
  int r;
  if ((r = prepare_single(c, s, 1, grid))) return r;
  if (dfd && df_stride == 0) CK(cudaMemsetAsync(dfd, 0, 3 * (size_t)c->n_v * sizeof(double), s));
  pdk::BatchBwd br;
  br.T = c->last_T;
  br.dqT = dqTd;
  br.dvT = dvTd;
  br.dq0 = dq0d;
  br.dv0 = dv0d;
  br.dE = dEd;
  br.dnu = dnud;
  br.df = dfd;
  br.df_stride = df_stride;
  CK(cudaMemsetAsync(&d.ctrl->bar_arrive, 0, sizeof(unsigned long long), s));
  CK(pdk::launch_bwd_rollout(d.local_fp32 != 0, c->d_dev + 1, c->d_team[1], c->d_off, br, grid, d.tmode != 0, s));
  c->launches += 1;
  return PD_OK;
}

// fold a control word into the statistics; returns the status of `which`
// (bit 0 forward, bit 1 backward)
int stats_from_ctrl(pd_ctx* c, const Ctrl& hc, int which) {
  pd_stats& st = c->stats;
  int rc = PD_OK;
  if (which & 1) {
    st.steps = c->last_T;
    st.iters_total = hc.iters_total;
    st.iters_max = hc.iters_max;
    st.aa_resets = hc.resets;
    st.not_converged = hc.not_converged;
    st.tau_half = hc.tau_half;
    st.tau_one = hc.tau_one;
    st.last_rho = hc.last_rho;
    st.escalations = hc.escalations;
    st.warm_fallbacks = hc.fallbacks;
    st.fwd_device_seconds = hc.elapsed_ns[0] * 1e-9;
    st.contact_iters = hc.con_iters;
    st.contact_unconverged = hc.con_unconverged;
  }
  if (which & 2) {
    st.adj_iters_total = hc.adj_iters_total;
    st.adj_iters_max = hc.adj_iters_max;
    st.adj_not_converged = hc.adj_not_converged;
    st.bwd_device_seconds = hc.elapsed_ns[1] * 1e-9;
    if (!(which & 1)) {
      st.contact_iters = hc.con_iters;
      st.contact_unconverged = hc.con_unconverged;
    }
  }
  st.status_flags = hc.status;
  if (hc.status & 4) {
    // blocks that gave up may have left split-row counters set: clear them
    // for pd_solve (persistent launches clear them at their start)
    if (c->d.s_cnt && c->d.n_slot > 0) cudaMemset(c->d.s_cnt, 0, sizeof(int) * (size_t)c->d.n_slot);
    return fail(c, PD_ERR_TIMEOUT, "a grid barrier of a persistent launch timed out");
  }
  if ((which & 1) && (hc.status & 1)) return fail(c, PD_ERR_NUMERIC, "non-finite value in the right-hand side");
  if ((which & 2) && (hc.status & 2))
    return fail(c, PD_ERR_NUMERIC, "adjoint operator A - K not positive along a CG direction");
  if ((which & 1) && hc.not_converged) rc = fail(c, PD_ERR_NOT_CONVERGED, "%d step(s) hit k_max", hc.not_converged);
  if ((which & 2) && hc.adj_not_converged)
    rc = fail(c, PD_ERR_NOT_CONVERGED, "%d adjoint solve(s) hit adj_max_iters", hc.adj_not_converged);
  return rc;
}

int collect_single(pd_ctx* c, cudaStream_t s, int which) {
  Ctrl hc;
  CK(cudaMemcpyAsync(&hc, c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c->profiling && (which & 1)) {
    prof_harvest(c, c->last_T);
    for (int i = 0; i < 8; ++i) {
      c->prof.phase_ms[i] += hc.phase_ns[i] * 1e-6;
      c->prof.work_ms[i] += hc.work_ns[i] * 1e-6;
      c->prof.work_max_ms[i] += hc.work_max_ns[i] * 1e-6;
      c->prof.last_ms[i] += hc.last_ns[i] * 1e-6;
    }
  }
  return stats_from_ctrl(c, hc, which);
}

}  // namespace

extern "C" {

int pd_reserve(pd_ctx* c, int32_t T) {
  if (!c || T < 1) return PD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  if (c->batch) return batch_reserve(c, T);
  return reserve_single(c, T);
}

int pd_rollout(pd_ctx* c, int32_t T, const double* q0, const double* v0, const double* f_ext, int64_t f_stride,
               double* qT, double* vT, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_rollout");
  if (T < 1 || !q0 || !v0) return fail(c, PD_ERR_ARG, "T >= 1 and q0, v0 are required");
  if (c->opt.warm_start < 0 || c->opt.warm_start > 2) return fail(c, PD_ERR_ARG, "warm_start must be 0, 1 or 2");
  if (c->opt.warm_start && !c->opt.persistent) return fail(c, PD_ERR_ARG, "the warm start needs persistent launches");
  if (!c->batch && c->d.n_con > 0 && !c->opt.persistent) return fail(c, PD_ERR_ARG, "contact needs persistent launches");
  if (c->opt.warm_start == 1 && !(c->batch ? batch_has_mlp(c) : c->d.mlp.w != nullptr))
    return fail(c, PD_ERR_ARG, "warm_start = 1 needs a network (pd_mlp_load)");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->batch) return batch_rollout(c, T, q0, v0, f_ext, f_stride, qT, vT, s, true);
  const size_t nv3 = 3 * (size_t)c->n_v;
  if (f_stride != 0 && f_stride != (int64_t)nv3) return fail(c, PD_ERR_ARG, "f_ext_stride must be 0 or 3*n_v");
  Dev& d = c->d;
  int r;
  if ((r = reserve_single(c, T))) return r;
  // host pointers are staged through one device buffer
  const bool hq = !is_device_ptr(q0), hv = !is_device_ptr(v0), hf = f_ext && !is_device_ptr(f_ext);
  const bool hqo = qT && !is_device_ptr(qT), hvo = vT && !is_device_ptr(vT);
  const size_t nf_ext = f_ext ? (f_stride ? (size_t)T * nv3 : nv3) : 0;
  if ((r = ensure_stage(c, 4 * nv3 + (hf ? nf_ext : 0)))) return r;
  double* st_q = c->stage;
  double* st_v = c->stage + nv3;
  double* st_qo = c->stage + 2 * nv3;
  double* st_vo = c->stage + 3 * nv3;
  double* st_f = c->stage + 4 * nv3;
  const double* q0d = q0;
  const double* v0d = v0;
  const double* fd = f_ext;
  if (hq) { CK(cudaMemcpyAsync(st_q, q0, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); q0d = st_q; }
  if (hv) { CK(cudaMemcpyAsync(st_v, v0, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); v0d = st_v; }
  if (hf) { CK(cudaMemcpyAsync(st_f, f_ext, nf_ext * sizeof(double), cudaMemcpyHostToDevice, s)); fd = st_f; }
  double* qTd = qT ? (hqo ? st_qo : qT) : nullptr;
  double* vTd = vT ? (hvo ? st_vo : vT) : nullptr;
  int pgrid = 0;
  if (c->opt.persistent && (r = grid_of(c, false, &pgrid))) return r;
  if (pgrid > 0) {
    // one cooperative launch for all T steps
    if ((r = enqueue_fwd_single(c, T, q0d, v0d, fd, f_stride, qTd, vTd, s, pgrid))) return r;
  } else {
    // per-phase kernels: no precision escalation (its kernels are compiled for one precision)
    const int escalate = d.escalate;
    d.escalate = 0;
    d.ckpt = c->ckpt;
    d.tau = c->tau;
    d.phase_count = c->phase_count;
    d.T = T;
    CK(cudaMemsetAsync(c->tau, 0, (size_t)T * sizeof(double), s));
    CK(cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), s));
    CK(cudaMemsetAsync(d.sstar, 0, 3 * sizeof(double) * (size_t)c->n_e, s));
    const int max_iter = c->opt.fixed_iters > 0 ? c->opt.fixed_iters : c->opt.k_max + 1;
    const int* done_flag = &d.ctrl->done;
    for (int t = 0; t < T; ++t) {
      const double* qin = t == 0 ? q0d : c->sq;
      const double* vin = t == 0 ? v0d : c->sv;
      const double* fstep = fd ? fd + (f_stride ? (size_t)t * nv3 : 0) : nullptr;
      pdk::launch_step_begin(d, s, qin, vin, fstep, t, c->ckpt + (size_t)t * nv3);
      c->launches += 1;
      CK(cudaGetLastError());
      int it_idx = 0;
      r = run_until(c, s, done_flag, max_iter, 4, [&]() {
        c->launches += 6;
        if (c->profiling) {
          cudaEvent_t ev[4];
          for (int i = 0; i < 4; ++i) ev[i] = prof_event(c);
          for (int kind = 0; kind < 2; ++kind) {
            c->prof_kind.push_back(kind);
            c->prof_step.push_back(t);
            c->prof_iter.push_back(it_idx);
          }
          pdk::launch_iteration(d, s, ev);
        } else {
          pdk::launch_iteration(d, s, nullptr);
        }
        ++it_idx;
      });
      if (r) return r;
      CK(cudaGetLastError());
      const bool last = t == T - 1;
      double* qo = last && qTd ? qTd : c->sq;
      double* vo = last && vTd ? vTd : c->sv;
      pdk::launch_step_end(d, s, qo, vo, c->ckpt + (size_t)(t + 1) * nv3, c->tau);
      c->launches += pdk::has_prox_hessian(c->model) ? 2 : 1;
      CK(cudaGetLastError());
    }
    d.escalate = escalate;
    c->last_T = T;
  }
  if (hqo) CK(cudaMemcpyAsync(qT, st_qo, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (hvo) CK(cudaMemcpyAsync(vT, st_vo, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  c->pending = 0;
  return collect_single(c, s, 1);
}

int pd_rollout_enqueue(pd_ctx* c, int32_t T, const double* q0, const double* v0, const double* f_ext,
                       int64_t f_stride, double* qT, double* vT, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_rollout_enqueue");
  if (T < 1 || !q0 || !v0) return fail(c, PD_ERR_ARG, "T >= 1 and q0, v0 are required");
  if (c->opt.warm_start < 0 || c->opt.warm_start > 2) return fail(c, PD_ERR_ARG, "warm_start must be 0, 1 or 2");
  if (c->opt.warm_start == 1 && !(c->batch ? batch_has_mlp(c) : c->d.mlp.w != nullptr))
    return fail(c, PD_ERR_ARG, "warm_start = 1 needs a network (pd_mlp_load)");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->batch) return batch_rollout(c, T, q0, v0, f_ext, f_stride, qT, vT, s, false);
  if (f_stride != 0 && f_stride != 3 * (int64_t)c->n_v) return fail(c, PD_ERR_ARG, "f_ext_stride must be 0 or 3*n_v");
  int r, grid = 0;
  if (!c->opt.persistent) return fail(c, PD_ERR_ARG, "pd_rollout_enqueue needs options.persistent = 1");
  if ((r = grid_of(c, false, &grid))) return r;
  if (grid <= 0) return fail(c, PD_ERR_ARG, "no co-resident grid for the persistent rollout");
  if ((r = reserve_enqueue(c, T, s))) return r;
  if ((r = enqueue_fwd_single(c, T, q0, v0, f_ext, f_stride, qT, vT, s, grid))) return r;
  c->pending |= 1;
  return PD_OK;
}

int pd_step(pd_ctx* c, const double* q_t, const double* v_t, const double* f_ext, double* q_next, double* v_next,
            void* stream) {
  return pd_rollout(c, 1, q_t, v_t, f_ext, 0, q_next, v_next, stream);
}

int pd_backward(pd_ctx* c, const double* dqT, const double* dvT, double* dq0, double* dv0, double* dE, double* dnu,
                double* df_ext, int64_t df_stride, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_backward");
  if (c->last_T < 1) return fail(c, PD_ERR_NO_CHECKPOINT, "no recorded rollout");
  if (!dqT) return fail(c, PD_ERR_ARG, "dqT is required");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->batch) return batch_backward(c, dqT, dvT, dq0, dv0, dE, dnu, df_ext, df_stride, s, true);
  const size_t nv3 = 3 * (size_t)c->n_v;
  if (df_stride != 0 && df_stride != (int64_t)nv3) return fail(c, PD_ERR_ARG, "df_stride must be 0 or 3*n_v");
  Dev& d = c->d;
  const int T = c->last_T;
  int r;
  const size_t ndf = df_ext ? (df_stride ? (size_t)T * nv3 : nv3) : 0;
  const bool h_dq = !is_device_ptr(dqT), h_dv = dvT && !is_device_ptr(dvT);
  const bool h_q0 = dq0 && !is_device_ptr(dq0), h_v0 = dv0 && !is_device_ptr(dv0);
  const bool h_E = dE && !is_device_ptr(dE), h_nu = dnu && !is_device_ptr(dnu), h_df = df_ext && !is_device_ptr(df_ext);
  if ((r = ensure_stage(c, 4 * nv3 + c->n_e + 1 + ndf))) return r;
  double* st_dq = c->stage;
  double* st_dv = c->stage + nv3;
  double* st_q0 = c->stage + 2 * nv3;
  double* st_v0 = c->stage + 3 * nv3;
  double* st_E = c->stage + 4 * nv3;
  double* st_nu = st_E + c->n_e;
  double* st_df = st_nu + 1;
  const double* dqTd = dqT;
  const double* dvTd = dvT;
  if (h_dq) { CK(cudaMemcpyAsync(st_dq, dqT, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); dqTd = st_dq; }
  if (h_dv) { CK(cudaMemcpyAsync(st_dv, dvT, nv3 * sizeof(double), cudaMemcpyHostToDevice, s)); dvTd = st_dv; }
  double* dq0d = h_q0 ? st_q0 : dq0;
  double* dv0d = h_v0 ? st_v0 : dv0;
  double* dEd = h_E ? st_E : dE;
  double* dnud = h_nu ? st_nu : dnu;
  double* dfd = h_df ? st_df : df_ext;
  int pgrid = 0;
  if (c->opt.persistent && (r = grid_of(c, true, &pgrid))) return r;
  if (pgrid > 0) {
    // one cooperative launch for the adjoint of all T steps
    if ((r = enqueue_bwd_single(c, dqTd, dvTd, dq0d, dv0d, dEd, dnud, dfd, df_stride, s, pgrid))) return r;
  } else {
    if (dfd && df_stride == 0) CK(cudaMemsetAsync(dfd, 0, nv3 * sizeof(double), s));
    pdk::launch_bwd_begin(d, s, dqTd, dvTd);
    c->launches += 1;
    CK(cudaGetLastError());
    const int* done_flag = &d.ctrl->adj_done;
    for (int t = T - 1; t >= 0; --t) {
      const double* qstar = c->ckpt + (size_t)(t + 1) * nv3;
      const double* qt = c->ckpt + (size_t)t * nv3;
      pdk::launch_bwd_setup(d, s, qstar, c->tau + t);
      pdk::launch_bwd_init(d, s);
      c->launches += 5;
      CK(cudaGetLastError());
      r = run_until(c, s, done_flag, c->opt.adj_max_iters, 4, [&]() {
        c->launches += 7;
        pdk::launch_pcg_iteration(d, s);
      });
      if (r) return r;
      double* df_t = dfd ? (df_stride ? dfd + (size_t)t * nv3 : dfd) : nullptr;
      pdk::launch_route(d, s, qstar, qt, c->tau + t, df_t, df_stride == 0 ? 1 : 0);
      c->launches += 1;
      CK(cudaGetLastError());
    }
    pdk::launch_chain(d, s, dEd, dnud);
    pdk::launch_bwd_finish(d, s, dq0d, dv0d);
    c->launches += 2;
    CK(cudaGetLastError());
  }
  if (h_q0) CK(cudaMemcpyAsync(dq0, st_q0, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_v0) CK(cudaMemcpyAsync(dv0, st_v0, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_E) CK(cudaMemcpyAsync(dE, st_E, c->n_e * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_nu) CK(cudaMemcpyAsync(dnu, st_nu, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h_df) CK(cudaMemcpyAsync(df_ext, st_df, ndf * sizeof(double), cudaMemcpyDeviceToHost, s));
  c->pending = 0;
  return collect_single(c, s, 2);
}

int pd_backward_enqueue(pd_ctx* c, const double* dqT, const double* dvT, double* dq0, double* dv0, double* dE,
                        double* dnu, double* df_ext, int64_t df_stride, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_backward_enqueue");
  if (c->last_T < 1) return fail(c, PD_ERR_NO_CHECKPOINT, "no recorded or enqueued rollout");
  if (!dqT) return fail(c, PD_ERR_ARG, "dqT is required");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->batch) return batch_backward(c, dqT, dvT, dq0, dv0, dE, dnu, df_ext, df_stride, s, false);
  if (df_stride != 0 && df_stride != 3 * (int64_t)c->n_v) return fail(c, PD_ERR_ARG, "df_stride must be 0 or 3*n_v");
  int r, grid = 0;
  if (!c->opt.persistent) return fail(c, PD_ERR_ARG, "pd_backward_enqueue needs options.persistent = 1");
  if ((r = grid_of(c, true, &grid))) return r;
  if (grid <= 0) return fail(c, PD_ERR_ARG, "no co-resident grid for the persistent adjoint");
  if ((r = enqueue_bwd_single(c, dqT, dvT, dq0, dv0, dE, dnu, df_ext, df_stride, s, grid))) return r;
  c->pending |= 2;
  return PD_OK;
}

int pd_collect(pd_ctx* c, void* stream) {
  if (!c) return PD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->batch) return batch_collect(c, s);
  const int which = c->pending;
  c->pending = 0;
  if (!which) {
    CK(cudaStreamSynchronize(s));
    return PD_OK;
  }
  return collect_single(c, s, which);
}

int pd_mlp_load(pd_ctx* c, const void* weights, size_t bytes) {
  if (!c || !weights) return PD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  if (c->batch) return batch_mlp_load(c, weights, bytes);
  return mlp_upload(c, weights, bytes, &c->d.mlp, c->allocs);
}

int pd_solve(pd_ctx* c, const double* b, double* x, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "pd_solve is single-instance only");
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_solve");
  if (!b || !x) return fail(c, PD_ERR_ARG, "b and x are required");
  CK(cudaSetDevice(c->device));
  pdk::launch_solve(c->d, (cudaStream_t)stream, b, c->d.bperm, c->d.y, c->d.s_part, c->d.s_cnt, x);
  c->launches += 3;
  CK(cudaGetLastError());
  return PD_OK;
}

int pd_local_rhs(pd_ctx* c, const double* q, double* out, void* stream) {
  if (!c) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "pd_local_rhs is single-instance only");
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_local_rhs");
  if (!q || !out) return fail(c, PD_ERR_ARG, "q and out are required");
  if (!is_device_ptr(q) || !is_device_ptr(out)) return fail(c, PD_ERR_ARG, "q and out must be device pointers");
  CK(cudaSetDevice(c->device));
  pdk::launch_local_rhs(c->d, (cudaStream_t)stream, q, out);
  c->launches += c->d.local_fp32 ? 3 : 2;
  CK(cudaGetLastError());
  return PD_OK;
}

int pd_profile(pd_ctx* c, int32_t enable) {
  if (!c) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "pd_profile is single-instance only");
  c->profiling = enable != 0;
  c->d.prof = c->profiling ? 1 : 0;
  c->prof = pd_profile_out{};
  c->prof_used = 0;
  c->prof_kind.clear();
  c->prof_step.clear();
  c->prof_iter.clear();
  return PD_OK;
}

int pd_get_profile(const pd_ctx* c, pd_profile_out* out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = c->prof;
  return PD_OK;
}

int pd_get_mass(const pd_ctx* c, double* m) {
  if (!c || !m) return PD_ERR_ARG;
  if (c->batch) return batch_get_mass(c, m);
  std::memcpy(m, c->mass.data(), c->mass.size() * sizeof(double));
  return PD_OK;
}

int pd_get_checkpoint(const pd_ctx* c, int32_t t, double* q_host) {
  if (c && c->batch) return batch_get_checkpoint(c, t, q_host);
  if (!c || !q_host || t < 0 || t > c->last_T || !c->ckpt) return PD_ERR_ARG;
  const size_t nv3 = 3 * (size_t)c->n_v;
  if (cudaMemcpy(q_host, c->ckpt + (size_t)t * nv3, nv3 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PD_ERR_CUDA;
  return PD_OK;
}

int pd_get_tau(const pd_ctx* c, double* tau_host, int32_t T) {
  if (c && c->batch) return batch_get_tau(c, tau_host, T);
  if (!c || !tau_host || T < 1 || T > c->last_T || !c->tau) return PD_ERR_ARG;
  if (cudaMemcpy(tau_host, c->tau, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return PD_ERR_CUDA;
  return PD_OK;
}

int pd_get_contact_impulses(const pd_ctx* c, int32_t t, int32_t* n_out, int32_t* vertex, double* lam_n,
                            double* lam_f) {
  if (!c || !n_out || c->batch) return PD_ERR_ARG;
  const int K = c->d.n_con;
  *n_out = K;
  if (K == 0 || (!vertex && !lam_n && !lam_f)) return PD_OK;
  if (!c->d.con_ckpt || t < 0 || t >= c->last_T) return PD_ERR_ARG;
  std::vector<double> ck(3 * (size_t)K);
  if (cudaMemcpy(ck.data(), c->d.con_ckpt + (size_t)t * 3 * K, ck.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return PD_ERR_CUDA;
  if (vertex && cudaMemcpy(vertex, c->d.con_v, (size_t)K * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PD_ERR_CUDA;
  for (int i = 0; i < K; ++i) {
    if (lam_n) lam_n[i] = ck[i];
    if (lam_f) {
      lam_f[2 * i] = ck[K + 2 * i];
      lam_f[2 * i + 1] = ck[K + 2 * i + 1];
    }
  }
  return PD_OK;
}

int pd_get_stats(const pd_ctx* c, pd_stats* out) {
  if (!c || !out) return PD_ERR_ARG;
  *out = c->stats;
  out->launches = c->launches;
  return PD_OK;
}

void pd_destroy(pd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->batch) batch_destroy(c);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->factor_allocs) cudaFree(p);
  if (c->ckpt) cudaFree(c->ckpt);
  if (c->tau) cudaFree(c->tau);
  if (c->phase_count) cudaFree(c->phase_count);
  if (c->con_ckpt) cudaFree(c->con_ckpt);
  if (c->stage) cudaFree(c->stage);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  for (auto& e : c->prof_ev) cudaEventDestroy(e);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"

void pd_internal_state(pd_ctx* c, const pdk::Dev** d, int* device, int* factored) {
  *d = c->batch ? nullptr : &c->d;
  *device = c->device;
  *factored = c->factored ? 1 : 0;
}

void pd_internal_set_error(pd_ctx* c, const char* msg) { c->err = msg; }
