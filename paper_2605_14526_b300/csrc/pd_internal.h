// Internal device-side state of a pd_ctx, shared by the host API and kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pdk {

constexpr int kMaxAA = 8;        // largest Anderson window
constexpr size_t kTStageBytes = 1024 * 3 * sizeof(double);   // dynamic shared staging of mode T (kTStage rows)
constexpr int kWideTeam = 64;    // teams of at least this many blocks number warps block-minor for row-wise products
constexpr int kRed = 24;         // doubles per block in the reduction scratch
constexpr int kVtxBlock = 256;   // threads per block, vertex kernels
constexpr int kTetBlock = 128;   // threads per block, element kernels
constexpr int kWarpsSpmv = 8;    // warps per block, skyline SpMV
constexpr int kSegLen = 512;     // entries per segment of a skyline row of S (one warp each)
constexpr int kJacRec = 36;      // values per element in the backward Jacobian record
// persistent kernels: threads per block and the resident blocks per SM the
// register budget is sized for. The forward comes in two shapes: one wide
// block per SM (its registers hold the local step, the S products and the
// Anderson solve without spilling; used when the grid needs at most one
// block per SM) and two narrow blocks per SM (more co-resident blocks, for
// batches of many instances). The adjoint uses two blocks of 256.
constexpr int kFwdWideBlock = 384;
constexpr int kFwdNarrowBlock = 256;
constexpr int kBwdBlock = 256;
constexpr int kBwdMinBlocks = 2;
constexpr int kRedRows = 2048;   // rows of the reduction scratch (>= any grid used)
constexpr int kRedRep = 4;       // copies of each block's partials in the team reductions
constexpr int kRedTeam = 16;     // values per row in the team reductions (>= 2 kMaxAA)
constexpr int kTBlock = 256;     // threads per block, per-height kernels of solve mode T

// Device-resident control word of the iteration (one per context).
struct Ctrl {
  int k;             // local-global iteration index within the step
  int done;          // step finished (kernels of later iterations exit at once)
  int converged;     // dual gate passed
  int pairs;         // Anderson history pairs held (0 .. m+1)
  int ncols;         // difference columns held (0 .. m)
  int head;          // ring slot the next difference column goes to
  int use_hat;       // 1: this iteration takes q_hat (no mixing / guard trip)
  int t;             // step index in the rollout
  int n_local, n_solve;  // phases that ran in this step (launches after done exit at once)
  double gram[kMaxAA * kMaxAA];
  double gamma[kMaxAA];
  double dgg[kMaxAA];
  double dq_norm2, qprev_norm2;   // ||q^{k+1} - q^k||^2, ||q^k||^2 from the last update
  double db_norm2, bprev_norm2;   // ||b^k - b^{k-1}||^2, ||b^{k-1}||^2
  // precision escalation of the FP32 local step (persistent rollouts)
  int fallbacks;     // warm-started steps that hit k_max and were re-run from q_t
  int hi;            // 1: the local step runs in FP64 for the rest of the rollout
  int since;         // iterations since the gate distance last halved
  int escalations;   // switches to FP64 (at most one per rollout)
  double gmin;       // smallest gate distance of this step
  // statistics (accumulated over a rollout)
  int iters_total, iters_max, resets, not_converged, tau_half, tau_one;
  int adj_iters_total, adj_iters_max, adj_not_converged;
  int status;        // bit 0: non-finite value; bit 1: PCG breakdown
  double last_rho;
  // backward (PCG) scalars
  int adj_k, adj_done;
  double rz, rz0, alpha, beta;
  double acc_mu, acc_lam, acc_k;  // mesh-mean sensitivities accumulated over steps
  double dnu_acc;
  unsigned int ticket[16];        // last-block-done counters, one per kernel kind
  unsigned long long bar_arrive;  // team barrier of the persistent kernels: arrivals so far (monotonic)
  unsigned long long phase_ns[8];  // persistent kernels: time per phase (globaltimer, block 0)
  unsigned long long work_ns[8];   // ... of which block 0's own work before the phase's barrier
  unsigned long long elapsed_ns[2]; // persistent launches: wall time of the forward / adjoint (team block 0)
  unsigned long long work_max_ns[8]; // profiling: largest per-block total work per phase
  unsigned long long last_ns[8];     // profiling: phase start to the last block's arrival at its barrier
  unsigned long long t_last;         // profiling: arrival time of the last block at the latest team barrier
  int con_iters, con_unconverged;   // contact: inner (FISTA) iterations, inner solves that hit their cap
};

// phases timed inside the persistent rollout
enum Phase { PH_BEGIN = 0, PH_LOCAL = 1, PH_ASSEMBLE = 2, PH_SPMV_S = 3, PH_SPMV_ST = 4, PH_AA = 5, PH_UPDATE = 6, PH_END = 7 };

enum Ticket {
  TK_ASSEMBLE = 0, TK_SPMV_T = 1, TK_UPDATE = 2, TK_TR = 3, TK_PCG_W = 4, TK_PCG_Z = 5,
  TK_ROUTE = 6, TK_CHAIN = 7, TK_PCG_INIT = 8
};

// Warm-start network (7 -> 128 -> 128 -> 128 -> 3, ReLU) as the kernels read
// it: BF16 weights (bit patterns) in input-major order W1t [7][128],
// W2t [128][128], W3t [128][128], W4t [128][3]; FP32 biases b1, b2, b3 [128],
// b4 [3]; normalisation of the features and scale of the output.
constexpr int kMlpIn = 7, kMlpH = 128, kMlpOut = 3;
constexpr int kMlpWeights = kMlpIn * kMlpH + 2 * kMlpH * kMlpH + kMlpH * kMlpOut;
constexpr int kMlpBiases = 3 * kMlpH + kMlpOut;
// The same weights packed in the B-fragment order of mma.sync m16n8k16
// (BF16): for layer l, k-step ks (16 inputs), n-tile nt (8 outputs) and lane,
// one uint2 {W[16ks+2t, n] | W[16ks+2t+1, n] << 16, W[16ks+2t+8, n] | ...}
// with t = lane % 4, n = 8 nt + lane / 4, zero beyond the layer's sizes;
// layers padded to 16 x 128, 128 x 128, 128 x 128, 128 x 8.
constexpr int kMlpFrag1 = 1 * 16 * 32, kMlpFragH = 8 * 16 * 32, kMlpFrag4 = 8 * 1 * 32;
constexpr int kMlpFrags = kMlpFrag1 + 2 * kMlpFragH + kMlpFrag4;
struct MlpDev {
  const uint16_t* w;   // [kMlpWeights]
  const uint2* wf;     // [kMlpFrags] fragment-packed weights (tensor-core path)
  const float* b;      // [kMlpBiases]
  float fmean[kMlpIn], fscale[kMlpIn], oscale[kMlpOut];
};

// the models whose local step is a stretch prox with a Hessian to filter
// (Sec. 4.3): Neo-Hookean and the log-volume barrier; they select tau per step
__host__ __device__ constexpr bool has_prox_hessian(int model) { return model == 1 || model == 3; }

// Everything the kernels need, passed by value.
struct Dev {
  int n_v, n_e, n_f;
  int model;          // 0 corotated, 1 Neo-Hookean, 2 corotated + volume composite, 3 corotated + log-volume barrier
  double rot_share;   // models 2, 3: a = w_0/(w_0 + w_1) = 2 mu/(2 mu + lambda) (the same for every element)
  double bar_r;       // model 3: r = mu/lambda = (1 - 2 nu)/(2 nu) inside the barrier's prox (the same for every element)
  int local_fp32;
  int aa_m, k_max, fixed_iters, tr_mode, adj_max_iters;
  int escalate;       // FP32 local step: switch to FP64 after this many iterations without progress (0 = never)
  int warm;           // start of each step: 0 q_t, 1 network warm start, 2 constant-velocity extrapolation
  int prof;           // 1: every block times its own work per phase (pd_profile)
  double h, alpha_d, eps_step, eps_res, eps_abs, eps_tr, adj_tol;
  double g[3];
  double mu_bar, lam_bar, k_bar, mu_ref, beta0, nu;

  // mesh
  const int4* tets;        // [n_e]
  const float* Bm32;       // [n_e][9] Dm^-1 row-major
  const double* Bm64;      // [n_e][9]
  const float* coef32;     // [n_e] w_e V_e
  const double* coef64;
  const double* vol;       // [n_e]
  const double* mu_e;      // [n_e]
  const double* lam_e;     // [n_e]
  const double* E;         // [n_e]
  const double* X;         // [n_v][3]
  const float* logE;       // [n_v] log10(E_v / 1e5), E_v the volume-weighted mean E around v
  MlpDev mlp;
  const double* mass;      // [n_v]
  const uint8_t* pinned;   // [n_v]
  const int* inc_ptr;      // [n_v+1] vertex -> incident (element*4 + corner)
  const int* inc_idx;
  // operators (rows indexed by vertex, pinned rows empty)
  const int* B_ptr; const int* B_idx; const double* B_val;   // scalar stiffness damping, all columns
  const int* A_ptr; const int* A_idx; const double* A_val;   // scalar L_A, free columns only
  const double* cA;        // [n_v][3] constant pinned-column term  A_fp X_p
  // inverse factor
  const int* iperm;        // [n_v] elimination position of free vertex (-1 if pinned)
  const int* perm;         // [n_f] vertex at elimination position
  const int64_t* s_rowptr; // skyline rows of S
  const int* s_first;      // first_desc per row
  int sfp64;               // 1: the S products in FP64 (s_val64, st_val64; b, y as doubles)
  unsigned int spin_limit; // polls of a team-barrier wait before it gives up
  const double* s_val64;   // S entries in FP64 (sfp64 only)
  const double* st_val64;  // S^T entries in FP64 (sfp64 only)
  const float2* s_hl;      // S entries as double-float pairs (hi, lo)
  const int4* s_seg;       // segments {row, offset, length, 0 or 1 + first partial slot of a split row}
  int n_seg;
  int n_slot;              // partial slots of the split rows
  float2* s_part;          // [n_slot][3] partial sums of split rows
  int* s_cnt;              // [n_slot] finished segments of a split row (at its first slot)
  float2* s_part_na;       // the same two buffers for pd_solve_noalloc, which shares no work
  int* s_cnt_na;           // buffer with the rollouts of its context
  const int64_t* st_ptr;   // S^T CSR (rows = positions)
  const int* st_idx;
  const float2* st_hl;
  // solve mode T (tsolve.h, pd_tsolve.cuh): A^-1 by the two level-scheduled
  // sweeps over the partitioned inverse of the factor instead of S^T S (the
  // products run in FP64: sfp64 = 1, b and y as doubles)
  int tmode;               // 1: mode T
  int t_nlev;              // heights of the node tree
  const int* t_c0;         // [nodes] first column (elimination position)
  const int* t_nc;         // [nodes] columns
  const int* t_nb;         // [nodes] rows below the node
  const int64_t* t_boff;   // [nodes + 1] offset of a node's below rows / U rows
  const int* t_below;      // below rows (positions)
  const int64_t* t_poff;   // [nodes + 1] offset of a node's [Linv; M] entries
  const double* t_prow;    // [Linv; M] row-major packed
  const double* t_pcol;    // [Linv; M] column-major packed
  const int64_t* t_goff;   // [nodes + 1] offset of a node's positions in t_gptr
  const int* t_gptr;       // gather lists per (node, position) into t_gsrc
  const int* t_gsrc;       // U rows of the children
  const int* t_lev_f;      // [heights + 1] forward block units per height
  const int* t_lev_b;      // [heights + 1] backward block units per height
  const int* t_lev_wf;     // [heights + 1] forward warp items per height
  const int* t_lev_wb;     // [heights + 1] backward warp nodes per height
  const int4* t_unit_f;    // {node, first row, rows, 1: a lane per row}
  const int4* t_unit_b;    // {node, first column, columns, 0}
  const int2* t_wnode_f;   // {node, first row}: 32 rows of a node of at most 32 columns
  const int* t_wnode_b;    // nodes of at most 32 columns and 160 rows
  double* t_U;             // [sum nb][3] updates passed up the node tree
  double* t_x;             // [n_f][3] result of the backward sweep (elimination order)

  // work vectors [n_v][3] unless noted
  double* q;        // current iterate q^k
  float2* qhl;      // [n_v][3] the same as float pairs hi + lo (read by the FP32 local step; kept by q's writers)
  double* qprev;    // q^{k-1}
  double* qhat;
  double* gprev;
  double* qt;       // q_t of the current step (pinned at X)
  double* qtil;     // inertial target
  double* b0;       // q-independent RHS
  double* b;        // b^k   (two buffers, swapped by parity of k)
  double* bprev;
  float2* bperm;    // [n_f][3] b in elimination order (double-float)
  float2* y;        // [n_f][3] S b (double-float)
  double* dQG;      // [kMaxAA][n_v][3] history sums dQ_j + dG_j
  double* dG;
  void* contrib;    // [n_e][12] float or double
  void* sstar;      // [n_e][3] float: last prox stretches (Newton warm start; <= 0 = none)
  double* red;      // [blocks][kRed]
  Ctrl* ctrl;

  // frictional contacts (vertex-ground, vertex-box) and bilateral
  // attachments (Sec. 4.6): candidates
  // sorted by elimination position, dense scalar Delassus W = (L_A^-1)_CC
  int n_con;               // 0: no contact
  const int* con_v;        // [K] vertex
  const int* con_pos;      // [K] elimination position (ascending)
  const double* con_n;     // [K] normal sign: +1 ground (z >= z_g), -1 box (z <= z_box(t)), +1 attachment
  const int* con_att;      // [K] 1: bilateral attachment (free multipliers, target con_tgt), else 0; null: none
  const double* con_tgt;   // [K][6] attachment target at the start of its motion and the motion's travel
  int con_att_steps;       // steps over which the attachment targets move
  const double* con_W;     // [K][K]
  double con_L;            // largest eigenvalue of W (FISTA step 1/L)
  double con_mu, con_zg, con_zb0, con_travel, con_tol;
  double con_slip_tol;     // adjoint: slip over a step at most this counts as sticking
  int con_steps, con_max_iters;
  double* con_buf;         // work: lam_n [3][K], lam_f [3][2K], gap [K], slip [2K], z [2K]
  double* con_ckpt;        // [T][3K]: converged lam_n [K], lam_f [K][2] of each step (adjoint)
  double* con_bwd;         // adjoint work [20K]: w, r, p (2 buffers), W p [K][3]; -G^T w parts

  // rollout storage
  double* sq;       // [n_v][3] state carried between steps of a rollout
  double* sv;
  double* ckpt;     // [(T+1)][n_v][3]
  double* tau;      // [T]
  int* phase_count; // [T][2] local / solve phases run per step
  int T;

  // backward
  void* jac;        // [n_e][kJacRec] float or double
  double* mu;       // adjoint solution
  double* r;        // residual
  double* z;        // preconditioned residual
  double* pdir;     // search direction
  double* pdir2;    // second buffer of the direction (persistent adjoint: old / new alternate)
  double* w;        // (A - K) p
  double* qbar;     // gradient on q*
  double* gq;       // running dL/dq_t
  double* gv;       // running dL/dv_t
  double* dw;       // [n_e] accumulated dL/dw_e (composite: of the rotation weight w_0)
  double* dw1;      // [n_e] composite: accumulated dL/dw_1 of the volume weight
  double* dbeta;    // [n_e]
};

// Arguments of the persistent forward rollout.
struct RollArgs {
  int T;
  const double* q0;
  const double* v0;
  const double* fext;
  long long f_stride;   // 0: one force array for all steps; else 3 n_v
  double* qT;
  double* vT;
  double* ckpt;         // [(T+1)][n_v][3]
  double* sq;           // state between steps
  double* sv;
};

// Arguments of the persistent backward rollout.
struct BwdArgs {
  int T;
  const double* dqT;
  const double* dvT;    // may be null
  double* dq0;          // outputs, each may be null
  double* dv0;
  double* dE;
  double* dnu;
  double* df;
  long long df_stride;  // 0: summed into one [n_v][3]; else 3 n_v per step
  const double* ckpt;   // [(T+1)][n_v][3]
};

// Batched launches: one descriptor for all instances; instance i reads its
// slice of each concatenated array at its prefix offsets.
struct InstOff {
  long long v, e;       // first vertex / element of the instance in the concatenation
};
struct BatchFwd {
  int T;
  const double* q0;
  const double* v0;
  const double* fext;
  long long f_stride;   // 0, or 3 x (total vertices) per step
  double* qT;
  double* vT;
};
struct BatchBwd {
  int T;
  const double* dqT;
  const double* dvT;
  double* dq0;
  double* dv0;
  double* dE;
  double* dnu;          // [instances]
  double* df;
  long long df_stride;  // 0, or 3 x (total vertices) per step
};

}  // namespace pdk
