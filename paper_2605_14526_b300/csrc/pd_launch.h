// Host-side launch wrappers of the PD kernels (defined in pd_kernels.cu and
// pd_backward.cu).
#pragma once
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pdk {

int max_reduction_blocks(int n_v, int n_e);

// forward (Alg. 1)
void launch_step_begin(const Dev& d, cudaStream_t s, const double* qt, const double* vt, const double* fext, int t,
                       double* ckpt_t);
// ev: optional 4 events bracketing (local step + assembly) and (two SpMVs)
void launch_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev);
void launch_step_end(const Dev& d, cudaStream_t s, double* qn, double* vn, double* ckpt_next, double* tau);
// A^-1 x for x given in elimination order (check: 0 none, 1 forward done flag, 2 backward done flag)
void launch_apply_inverse(const Dev& d, cudaStream_t s, const float2* xperm, float2* y, float2* part, int* cnt,
                          double* out, int check);

// the local step of every element at positions x and the projection part of
// the right-hand side, out[v] = sum_e w_e V_e G_e^T vec(p_e*) (two launches)
void launch_local_rhs(const Dev& d, cudaStream_t s, const double* x, double* out);

// x = A^-1 b for b, x in vertex order; xperm and y are [n_f][3] work buffers
void launch_solve(const Dev& d, cudaStream_t s, const double* b, float2* xperm, float2* y, float2* part, int* cnt,
                  double* x);

// co-resident blocks per SM of a persistent kernel (at most 2; 0 if
// cooperative launch is unavailable); *sms gets the SM count
int coop_blocks_per_sm(const void* fn, int block, int* sms);

// Persistent rollout / adjoint of one or many instances (one team of blocks
// per instance): co-resident grid size (0 if cooperative launch is not
// available; at most blocks_per_sm blocks per SM when that is >= 1) and the
// launch. devs and off are device arrays with one entry per instance (off:
// n + 1 prefix offsets), team[grid] maps each block to {instance, index in
// its team, team size, 0}.
int persistent_grid(bool fp32, int blocks_per_sm);
int persistent_grid_max(bool fp32);   // the larger grid of the two forward shapes
// tstage: some instance of the launch solves in mode T (its dynamic shared
// staging is requested)
cudaError_t launch_fwd_rollout(bool fp32, const Dev* devs, const int4* team, const InstOff* off, const BatchFwd& br,
                               int grid, bool tstage, cudaStream_t s);
int persistent_grid_bwd(bool fp32, int blocks_per_sm);
cudaError_t launch_bwd_rollout(bool fp32, const Dev* devs, const int4* team, const InstOff* off, const BatchBwd& br,
                               int grid, bool tstage, cudaStream_t s);

// backward (Alg. 2)
void launch_bwd_setup(const Dev& d, cudaStream_t s, const double* qstar, const double* tau_t);
void launch_bwd_init(const Dev& d, cudaStream_t s);
void launch_pcg_iteration(const Dev& d, cudaStream_t s);
void launch_route(const Dev& d, cudaStream_t s, const double* qstar, const double* qt, const double* tau_t,
                  double* df_out, int df_accumulate);
void launch_chain(const Dev& d, cudaStream_t s, double* dE, double* dnu);
void launch_bwd_begin(const Dev& d, cudaStream_t s, const double* dqT, const double* dvT);
void launch_bwd_finish(const Dev& d, cudaStream_t s, double* dq0, double* dv0);

}  // namespace pdk
