// Private definition of the library context (pd_ctx) and the small host
// helpers shared by the single-instance and batched drivers.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/pd_b300.h"
#include "factor.h"
#include "pd_internal.h"

using pdk::Ctrl;
using pdk::Dev;

struct pd_batch;  // batched-instance state (pd_batch.cpp)

struct pd_ctx {
  // host copies
  int n_v = 0, n_e = 0, n_f = 0;
  std::vector<double> X;
  std::vector<int32_t> tets;
  std::vector<uint8_t> pinned;
  std::vector<double> E;
  double nu = 0.3, density = 1000.0, alpha = 0.0, beta0 = 0.0, g[3] = {0, 0, 0};
  int model = PD_NEOHOOKEAN;
  double dt = 0.01;
  pd_options opt{};
  // rest shape
  std::vector<double> Bm, vol, mass;
  // factor state
  bool factored = false;
  bool have_order = false;
  std::vector<int> order_perm;  // free-local elimination order (geometry only)
  pdf::Factor fac;
  int64_t nnz_S = 0;
  double factor_seconds = 0;
  // solve mode chosen by pd_factor: T (level-scheduled partitioned-inverse
  // triangular solves) or S (products with the inverse factor)
  bool tmode = false;
  int64_t solve_nnz = 0;        // stored entries the solve streams per sweep (S: nnz(S); T: one copy)
  int solve_levels = 0;         // mode T: heights of the separator tree
  double tsolve_seconds = 0;    // mode T: host time of the partitioned inverse
  // device
  int device = 0;
  Dev d{};
  std::vector<void*> allocs;        // context-lifetime device buffers
  std::vector<void*> factor_allocs; // freed on refactor
  double* ckpt = nullptr;
  int ckpt_cap = 0;
  double* tau = nullptr;
  double *sq = nullptr, *sv = nullptr;   // rollout state
  double* stage = nullptr;               // host-pointer staging
  size_t stage_cap = 0;
  int* h_flag = nullptr;                 // pinned host flags
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int last_T = 0;
  pd_stats stats{};
  // phase timers: event pairs with the step and iteration they bracket; pairs
  // of iterations that exited early (launched after convergence) are dropped
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind, prof_step, prof_iter;  // per pair
  size_t prof_used = 0;                              // events in use
  pd_profile_out prof{};
  int* phase_count = nullptr;                        // device [T][2]
  int64_t launches = 0;
  std::string err;
  // launch shape (autotuner): blocks per SM and explicit grid sizes (0 = default)
  pd_tuning tune{};
  bool tuned = false;
  // batch of independent instances (null for a single-instance context)
  pd_batch* batch = nullptr;
  // last asynchronous operation awaiting pd_collect: 0 none, 1 rollout, 2 backward
  int pending = 0;
  // persistent launches of a single instance run the batched kernel with one
  // team: device copy of d (re-uploaded when d changes), prefix offsets and
  // the block -> team maps of the forward and the adjoint grid
  Dev* d_dev = nullptr;
  pdk::InstOff* d_off = nullptr;
  int4* d_team[2] = {nullptr, nullptr};
  int team_cap = 0;
  int team_grid[2] = {0, 0};
  Dev d_uploaded{};
  Dev d_adjoint{};           // host copy of the adjoint's record (d_dev[1])
  bool d_valid = false;
  // frictional contacts (pd_set_contacts)
  std::vector<int> con_ground, con_box, con_att;
  std::vector<double> con_att_p0, con_att_tr;   // [n_attach][3] targets and their travel
  pd_contact_desc con{};
  double* con_ckpt = nullptr;   // [T][3K] converged multipliers per step
  int con_ckpt_cap = 0;
};

// batched instances (pd_batch.cpp)
int batch_rollout(pd_ctx* c, int T, const double* q0, const double* v0, const double* f_ext, int64_t f_stride,
                  double* qT, double* vT, cudaStream_t s, bool sync);
int batch_backward(pd_ctx* c, const double* dqT, const double* dvT, double* dq0, double* dv0, double* dE,
                   double* dnu, double* df, int64_t df_stride, cudaStream_t s, bool sync);
int batch_collect(pd_ctx* c, cudaStream_t s);
int batch_reserve(pd_ctx* c, int T);
int batch_factor(pd_ctx* c);
int batch_get_mass(const pd_ctx* c, double* m);
int batch_get_checkpoint(const pd_ctx* c, int t, double* q_host);
int batch_size(const pd_ctx* c);                            // instances (1 without a batch)
void batch_set_warm(pd_ctx* c, int mode);                   // warm_start of every instance
pd_ctx* batch_kid(const pd_ctx* c, int i, int64_t* v_off);  // instance i and its first vertex
int batch_get_tau(const pd_ctx* c, double* tau_host, int T);
void batch_destroy(pd_ctx* c);
// warm-start network blob -> device layout (pd_mlp.cu); buffers appended to owner
int mlp_upload(pd_ctx* c, const void* blob, size_t bytes, pdk::MlpDev* out, std::vector<void*>& owner);
int batch_mlp_load(pd_ctx* c, const void* blob, size_t bytes);
bool batch_has_mlp(const pd_ctx* c);

namespace pdh {


inline int fail(pd_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(c, PD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
inline int dalloc(pd_ctx* c, T** p, size_t n, bool factor_scope = false) {
  void* q = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) return fail(c, PD_ERR_OOM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  (factor_scope ? c->factor_allocs : c->allocs).push_back(q);
  *p = reinterpret_cast<T*>(q);
  return PD_OK;
}

template <typename T>
inline int upload(pd_ctx* c, T** p, const std::vector<T>& h, bool factor_scope = false) {
  int r = dalloc(c, p, h.size(), factor_scope);
  if (r) return r;
  if (!h.empty()) CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PD_OK;
}

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The Dev record of the persistent adjoint: without contacts, in mode S,
// the products with S that precondition its conjugate gradients run in
// double-float (the pairs are always uploaded) even where the forward uses
// FP64 products; the CG's residuals and stopping test stay FP64.
inline Dev adjoint_dev(const Dev& d) {
  Dev b = d;
  if (b.sfp64 && !b.tmode && b.n_con == 0) b.sfp64 = 0;
  return b;
}

inline bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

inline int ensure_stage(pd_ctx* c, size_t n) {
  if (n <= c->stage_cap) return PD_OK;
  if (c->stage) cudaFree(c->stage);
  c->stage = nullptr;
  c->stage_cap = 0;
  cudaError_t e = cudaMalloc(&c->stage, n * sizeof(double));
  if (e != cudaSuccess) return fail(c, PD_ERR_OOM, "staging allocation: %s", cudaGetErrorString(e));
  c->stage_cap = n;
  return PD_OK;
}

}  // namespace pdh
