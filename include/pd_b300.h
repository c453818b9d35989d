/*
 * pd_b300.h - C ABI of the B300-native differentiable heterogeneous
 * Projective Dynamics hot path (arXiv 2605.14526, "DiffPhD").
 *
 * One context holds one tetrahedral mesh, its materials, the factored PD
 * operator and the per-step checkpoints of the last rollout. All compute runs
 * in the library's CUDA kernels on the device that is current when the
 * context is created; host code in the library only validates inputs,
 * assembles and factors the operator (once per material change: Sec. 4.5
 * on when to refactor), and orders launches.
 *
 * Conventions
 *   - Vertex arrays are [n_v][3] row-major float64 (x, y, z per vertex).
 *   - Pinned (Dirichlet) vertices are held at their rest position X; their
 *     outputs are X (positions) / 0 (velocities) and their gradients are 0.
 *   - "stream" is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued on it; calls that must read device results synchronise it.
 *   - Every function returns a pd_status; PD_OK = 0. On error, pd_last_error
 *     returns a message. Nothing aborts; device-side numeric problems are
 *     recorded in a status word and reported by the next synchronising call.
 *   - The library never frees memory it does not own.
 */
#ifndef PD_B300_H
#define PD_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PD_OK = 0,
  PD_ERR_ARG = 1,           /* bad size, index out of range, null pointer */
  PD_ERR_MESH = 2,          /* a rest tetrahedron with det(Dm) <= 0 */
  PD_ERR_NOT_FACTORED = 3,  /* pd_step/pd_rollout before pd_factor */
  PD_ERR_NOT_SPD = 4,       /* non-positive pivot while factoring A */
  PD_ERR_NOT_CONVERGED = 5, /* a step hit k_max (results are still written) */
  PD_ERR_NUMERIC = 6,       /* NaN/Inf met in a kernel */
  PD_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
  PD_ERR_CUDA = 8,          /* a CUDA runtime call failed */
  PD_ERR_OOM = 9,           /* device or host allocation failed */
  PD_ERR_NO_CHECKPOINT = 10,/* pd_backward without a recorded rollout */
  PD_ERR_TOO_LARGE = 11     /* a size exceeds a documented limit */
} pd_status;

/* Energies (Sec. 4.1, Sec. 7.2): corotated rotation step (w_e = 2 mu_e);
 * Neo-Hookean stretch prox (w_e = 2 mu_e + lambda_e); the corotated + volume
 * composite: the rotation step with w_0 = 2 mu_e plus a volume step with
 * w_1 = lambda_e, the closest point of the unit-determinant set in stretch
 * space (sigma_1 sigma_2 sigma_3 = 1), both in the one operator A (weight
 * w_0 + w_1) and in b; the opt-in log-volume barrier variant (Sec. 4.1,
 * eq. pd_log_volume): the same rotation step with the barrier
 * phi_log = -mu_e sum ln sigma_i + lambda_e/2 (sum ln sigma_j)^2 as the volume
 * step, the stretch prox of phi_log with weight w_1 = lambda_e solved by the
 * Neo-Hookean Newton, its differential filtered by the trust region like
 * Neo-Hookean's. As printed, phi_log has gradient -mu_e at rest, so an
 * unloaded body is pushed outward (a uniform stretch of about 2.8% in the
 * volume step at nu = 0.45); it needs nu in (0, 0.5). */
enum { PD_COROTATED = 0, PD_NEOHOOKEAN = 1, PD_COROT_VOLUME = 2, PD_COROT_LOGVOL = 3 };
enum { PD_TR_ADAPT = 0, PD_TR_NONE = 1, PD_TR_CLAMP = 2, PD_TR_ABS = 3 };
/* How every A^-1 application is computed (pd_options.solve_mode). */
enum { PD_SOLVE_AUTO = 0, PD_SOLVE_S = 1, PD_SOLVE_T = 2 };

/* Mesh, copied by pd_create (host pointers). */
typedef struct {
  int32_t n_v, n_e;
  const double* X;        /* [n_v][3] rest positions (m) */
  const int32_t* tets;    /* [n_e][4] vertex indices, det[X1-X0,X2-X0,X3-X0] > 0 */
  const uint8_t* pinned;  /* [n_v] 1 = Dirichlet vertex held at X; may be NULL */
} pd_mesh;

/* Material (Sec. 3.1 eq. lame; Sec. 4.4 eq. rayleigh), copied by pd_create. */
typedef struct {
  int32_t model;          /* PD_COROTATED | PD_NEOHOOKEAN | PD_COROT_VOLUME | PD_COROT_LOGVOL */
  const double* E;        /* [n_e] Young's modulus per element (Pa), > 0 */
  double nu;              /* Poisson ratio shared by all elements, in (-1, 0.5) */
  double density;         /* kg/m^3; lumped mass density*V_e/4 per corner */
  double alpha;           /* Rayleigh mass-damping coefficient (1/s) */
  double beta0;           /* stiffness damping scale: beta_e = beta0 mu_e / max mu */
  double gravity[3];      /* body acceleration added to every vertex (m/s^2) */
} pd_material;

/* Solver options (Sec. 4.3 Anderson + dual gate; Sec. 4.3 trust region). */
typedef struct {
  int32_t aa_m;           /* Anderson window: difference columns (0 = off, <= 8) */
  int32_t k_max;          /* iteration cap per step */
  int32_t fixed_iters;    /* > 0: exactly this many local-global iterations, no gate */
  int32_t local_fp32;     /* 1: FP32 local step with FP64 RHS accumulation; 0: FP64 */
  int32_t tr_mode;        /* PD_TR_ADAPT | PD_TR_NONE | PD_TR_CLAMP | PD_TR_ABS */
  int32_t adj_max_iters;  /* cap on backward PCG iterations per step */
  int32_t persistent;     /* 1: one cooperative launch per rollout when its grid fits
                             (falls back to per-phase kernels otherwise); 0: per-phase kernels */
  double eps_step;        /* relative q-step gate */
  double eps_res;         /* relative b-change gate */
  double eps_abs;         /* absolute term of both gates */
  double eps_tr;          /* trust-region ratio tolerance (0.1 in the paper) */
  double adj_tol;         /* backward: relative preconditioned residual target */
  int32_t escalate_window;/* FP32 local step, persistent launches: when the gate distance
                             (the larger squared ratio of the two gates) has not halved for
                             this many iterations, the rounding of the FP32 projections
                             is the floor of the iteration and the local step switches to
                             FP64 for the rest of the rollout (0 = never; default 100) */
  int32_t warm_start;     /* start of each step's iteration: 0 q_t (Alg. 1); 1 the learned
                             warm start (pd_mlp_load); 2 constant-velocity extrapolation
                             2 x_t - x_{t-1}. Persistent launches only; a warm-started step
                             that hits k_max is run again from q_t (pd_stats.warm_fallbacks) */
  int32_t solve_fp64;     /* products with the inverse factor S (every A^-1 application):
                             0 (default) double-float arithmetic on the FP32 pipe, S, S^T,
                             b and y held as (hi, lo) float pairs, error of order 2^-44 of the
                             row's sum of magnitudes, at 64x the FP64 rate of this part;
                             1 plain FP64 (S and S^T also kept as FP64 values, 8 more bytes
                             per non-zero). Fixed at pd_create. A context with contacts
                             (pd_set_contacts) always uses FP64 products: its Delassus
                             matrix comes from the FP64 factor and the adjoint's
                             projection needs A^-1 to agree with it. Without contacts the
                             persistent adjoint applies S in double-float whatever this
                             option: there A^-1 only preconditions the conjugate gradients,
                             whose residuals, updates and stopping test stay FP64, so the
                             product's precision changes the iteration count, not the
                             adjoint it converges to. */
  int32_t wait_polls;     /* persistent launches: polls (about 0.5 us each) a block spends at
                             a team barrier before it gives up, sets the timeout flag and
                             returns; the call then fails with PD_ERR_TIMEOUT and the context
                             stays usable (0 = 4194304, about 2 s). Fixed at pd_create. */
  int32_t solve_mode;     /* how A^-1 is applied (Sec. 4.5; read at pd_factor):
                             PD_SOLVE_S: the two products with the inverse factor S = L^-1 P
                               (eq. Ainv_STS / two_spmv); S holds every descendant of a
                               column of the elimination tree, so it grows like n^(5/3) on
                               3-D meshes (10% of n^2 on a 2,592-vertex bar, 2.5e9 entries
                               at 270k vertices);
                             PD_SOLVE_T: forward and backward triangular solves with the
                               factor L itself, level-scheduled over the separator tree
                               (one pass per tree height), each node's block column of L
                               replaced by its partitioned inverse [L_ss^-1; L_bs L_ss^-1]
                               (about nnz(L) entries, stored row- and column-major), FP64
                               arithmetic; not with contacts;
                             PD_SOLVE_AUTO (0, default): T when there are no contacts and
                               nnz(S) > 8e6 and nnz(S) > 4 nnz(L) (S no longer near the L2
                               size and several times L), or nnz(S) exceeds 2^31 - 1; else S. */
} pd_options;

/* Statistics of the last pd_rollout / pd_backward (host copy). */
typedef struct {
  int32_t steps;            /* steps recorded by the last rollout */
  int32_t iters_total;      /* local-global iterations summed over steps */
  int32_t iters_max;        /* largest per-step iteration count */
  int32_t aa_resets;        /* Anderson reliability-guard trips */
  int32_t not_converged;    /* steps that hit k_max */
  int32_t tau_half;         /* steps whose trust-region selection gave tau = 1/2 */
  int32_t tau_one;          /* ... tau = 1 */
  int32_t adj_iters_total;  /* backward PCG iterations summed over steps */
  int32_t adj_iters_max;
  int32_t adj_not_converged;
  int32_t status_flags;     /* bit 0: NaN/Inf seen; bit 1: PCG breakdown */
  int32_t n_free;           /* free vertices */
  int64_t factor_nnz;       /* stored entries of the solve: non-zeros of the inverse factor S
                               (mode S) or of one copy of the partitioned inverse (mode T) */
  double factor_seconds;    /* host time of the last pd_factor */
  double last_rho;          /* trust-region ratio of the last step */
  int64_t launches;         /* kernel launches issued by this context so far */
  int32_t escalations;      /* rollouts whose local step switched from FP32 to FP64 (a batch: instances) */
  int32_t warm_fallbacks;   /* warm-started steps that hit k_max and were run again from q_t */
  double fwd_device_seconds;  /* persistent launches: the last forward's wall time measured on the device
                                 (a batch: the instance's team; pd_get_stats gives the largest) */
  double bwd_device_seconds;  /* ... of the last adjoint */
  int32_t contact_iters;      /* contact: inner solver passes over W in the last rollout */
  int32_t contact_unconverged;/* contact: inner solves that hit contact_max_iters */
  int32_t solve_mode;         /* PD_SOLVE_S or PD_SOLVE_T as chosen by pd_factor (a batch: the
                                 largest over its instances) */
  int32_t solve_levels;       /* mode T: heights of the separator tree (passes per sweep) */
  int64_t nnz_L;              /* non-zeros of the factor L (a batch: summed) */
} pd_stats;

typedef struct pd_ctx pd_ctx;

/* Frictional contacts (Sec. 4.6; vertex-obstacle, position level), set with
 * pd_set_contacts before pd_factor. Ground vertices stay at z >= ground_z
 * (normal +z); box vertices stay at z <= z_box(t) (normal -z), the bottom of
 * a rigid box that moves down by box_travel over the first box_steps steps
 * of a rollout, z_box(t) = box_z0 - box_travel min(t + 1, box_steps) /
 * box_steps at the end of step t. Coulomb friction with coefficient mu, as
 * Tresca disks of radius mu lambda_n on the tangential displacement since
 * q_t. Bilateral attachments (Sec. 4.6): vertex attach[i] is held at
 * p_i(t) = attach_target[i] + attach_travel[i] min(t + 1, attach_steps) /
 * attach_steps at the end of step t, by three equality rows with free
 * multipliers (its z row solved with the normal rows, its x, y rows with the
 * friction rows, without a disk); in the adjoint they are equality
 * constraints at every step (no gradient with respect to the targets is
 * returned). Candidates must be free vertices; every index appears once
 * over ground, box and attach. */
typedef struct {
  int32_t n_ground, n_box;
  const int32_t* ground;  /* [n_ground] vertex indices (host, copied) */
  const int32_t* box;     /* [n_box] */
  double ground_z, box_z0, box_travel;
  int32_t box_steps;
  double mu;
  double tol;             /* relative tolerance of the inner solves (0: 1e-12) */
  int32_t max_iters;      /* cap on inner passes per solve (0: 2000) */
  int32_t n_attach;
  const int32_t* attach;        /* [n_attach] vertex indices (host, copied) */
  const double* attach_target;  /* [n_attach][3] target at the start of the motion (m) */
  const double* attach_travel;  /* [n_attach][3] displacement of the target; NULL: static */
  int32_t attach_steps;         /* steps over which the targets move (>= 1 when attach_travel is set) */
} pd_contact_desc;

/* Default options (m = 5, k_max = 200, gate 1e-8 / 1e-6 / 1e-12, FP32 local,
 * adaptive trust region with eps_tr = 0.1, backward 1e-9 / 1000 iterations,
 * persistent launches on, precision escalation after 100 iterations without
 * progress). */
void pd_default_options(pd_options* out);

/* Create a context: validates the mesh (indices in range, positive rest
 * volumes, no pinned-only mesh), copies mesh and materials, computes rest
 * shape data (Dm^-1, V_e, lumped mass) and uploads the per-element arrays.
 * Sec. 3.1 (eq. lame, dynamics, freefall). Host pointers; dt > 0.
 * On failure *out may still hold a context whose pd_last_error explains the
 * error; release it with pd_destroy. */
int pd_create(const pd_mesh* mesh, const pd_material* mat, double dt, const pd_options* opt,
              pd_ctx** out);

/* Frictional contacts and attachments of a single-instance context (NULL or
 * n_ground + n_box + n_attach = 0 removes them). pd_factor then also forms the dense scalar
 * Delassus matrix W = (L_A^-1)_CC of the K candidates (K host solves with the
 * factor, FP64; K^2 x 8 bytes on the device). Each local-global iteration of
 * a rollout computes q_u = A^-1 b(q) at the candidates, solves the normal
 * LCP 0 <= lam_n _|_ D W D lam_n + g >= 0 and the Tresca QP of the friction
 * on W (FISTA with adaptive restart), and takes q = A^-1 (b + J^T lam)
 * (eq. q_update) through the same two products with S. Persistent launches
 * only. pd_backward differentiates a contact rollout with each step's active
 * sets held fixed (normal-active and sticking contacts as equality
 * constraints; preconditioned CG projected onto their null space, with the
 * constraint multipliers taken out of the residual at every projection). */
int pd_set_contacts(pd_ctx* ctx, const pd_contact_desc* desc);

/* Contact impulses of step t (0 <= t < T) of the last rollout: n_out = the
 * number K of candidates; vertex [K] (the candidate's vertex), lam_n [K]
 * (normal impulse, >= 0, along +z for ground and -z for box candidates;
 * an attachment's z impulse, of either sign), lam_f [K][2] (tangential x, y
 * impulse). Any of the three arrays may be
 * NULL (only n_out is written when all are). Host outputs; synchronous.
 * Candidates come in elimination order, not in the order of the descriptor. */
int pd_get_contact_impulses(const pd_ctx* ctx, int32_t t, int32_t* n_out, int32_t* vertex, double* lam_n,
                            double* lam_f);

/* Replace the Young's moduli ([n_e], host, Pa) and Poisson ratio; marks A stale
 * so that the next pd_factor refactors (Sec. 4.5 refactorisation policy). */
int pd_set_materials(pd_ctx* ctx, const double* E, double nu);

/* Assemble and factor the PD operator
 *   A = (1 + alpha h) M / h^2 + sum_e (w_e + beta_e/h) V_e G_e^T G_e   (Sec. 4.4 eq. A_damped)
 * with w_e = 2 mu_e (corotated) or 2 mu_e + lambda_e (Neo-Hookean) (Sec. 4.1
 * eq. pd_weight; Sec. 7.2), beta_e = beta0 mu_e / mu_ref, mu_ref = max mu_e
 * frozen here. Pins are eliminated. The scalar operator (A = L_A (x) I_3) is
 * reordered by geometric nested dissection, factored by a supernodal
 * Cholesky in FP64 on the host, and uploaded in the form the solve mode
 * (pd_options.solve_mode) applies: the inverse factor S = L^-1 P
 * (A^-1 = S^T S, Sec. 4.5 eq. Ainv_STS, two_spmv), or the partitioned
 * inverse of L by separator-tree node for the level-scheduled triangular
 * solves (mode T). Returns PD_ERR_NOT_SPD on a non-positive pivot,
 * PD_ERR_TOO_LARGE if mode S is asked for and nnz(S) exceeds 2^31 - 1,
 * PD_ERR_ARG for mode T with contacts, PD_ERR_NUMERIC if the host check of
 * the mode-T structures against the factor fails. Blocking. */
int pd_factor(pd_ctx* ctx);

/* T implicit-Euler PD steps from (q0, v0) (Alg. 1 per step): inertial target,
 * fused local step + RHS scatter, global solve by two SpMVs with S,
 * type-II Anderson acceleration (window aa_m) and the dual gate; at the end
 * of each step the trust-region ratio picks tau* for the backward pass
 * (Sec. 4.3 eq. tr_step .. tr_rule). Checkpoints q_t for t = 0..T are kept
 * on the device for pd_backward.
 *   q0, v0   [n_v][3]; f_ext [T][n_v][3] if f_ext_stride = n_v*3, or one
 *            [n_v][3] array used at every step if f_ext_stride = 0 (N);
 *   qT, vT   [n_v][3] outputs.
 * Pointers may be device pointers (no copies) or host pointers (staged by
 * the library with cudaMemcpyAsync on the stream). Synchronises the stream
 * at the end and returns PD_ERR_NOT_CONVERGED if any step hit k_max. */
int pd_rollout(pd_ctx* ctx, int32_t T, const double* q0, const double* v0, const double* f_ext,
               int64_t f_ext_stride, double* qT, double* vT, void* stream);

/* One time step of Alg. 1 (Sec. 3.1 eq. dynamics / freefall: the inertial
 * target q~ = q_t + h v_t + h^2 (g + M^-1 f_ext); then local-global
 * iterations with Anderson mixing until the dual gate, Sec. 4.3
 * eq. convergence_dual; q_next = q*, v_next = (q* - q_t) / h). It is
 * pd_rollout with T = 1: the same kernels, the checkpoint of this step only,
 * so a following pd_backward is the adjoint of this one step (Alg. 2).
 *   q_t, v_t, f_ext  [n_v][3] inputs (f_ext may be NULL: no extra force);
 *   q_next, v_next   [n_v][3] outputs.
 * Pointers as in pd_rollout (device, or host staged by the library); the
 * stream is synchronised; PD_ERR_NOT_CONVERGED if the step hit k_max. */
int pd_step(pd_ctx* ctx, const double* q_t, const double* v_t, const double* f_ext, double* q_next,
            double* v_next, void* stream);

/* Adjoint of the last pd_rollout (Alg. 2 per step, walked from T-1 to 0).
 * Per step: mu = (A - K)^-1 q_bar with K = db/dq (Sec. 4.7 eq. db_dq, the
 * trust-region-filtered prox differential of eq. tr_blend / tr_ift, or the
 * polar differential for corotated), solved by conjugate gradients
 * preconditioned with the same factor (A^-1 = S^T S); then gradient routing
 *   dL/dq_t = (1+alpha h) M/h^2 mu + B mu/h - v_bar/h,  dL/dv_t = M/h mu,
 *   dL/df_ext = mu, dL/dw_e = V_e <G_e mu, p_e - G_e q*> (eq. dl_dwe),
 *   dL/dbeta_e = -(V_e/h) <G_e mu, G_e (q* - q_t)>, plus the mesh-mean terms,
 * chained to E_e and nu (eq. lame). Inputs dqT, dvT [n_v][3] (dvT may be
 * NULL); outputs dq0, dv0 [n_v][3], dE [n_e], dnu [1], df_ext [T][n_v][3] if
 * df_stride = n_v*3 or summed into one [n_v][3] if df_stride = 0 (may be
 * NULL). Any output pointer may be NULL to skip it. Host or device pointers
 * as in pd_rollout. Synchronises the stream. */
int pd_backward(pd_ctx* ctx, const double* dqT, const double* dvT, double* dq0, double* dv0,
                double* dE, double* dnu, double* df_ext, int64_t df_stride, void* stream);

/* x = A^-1 b on the free DoFs with the factored operator of the context,
 * in the context's solve mode: two sparse products x = S^T (S b) (Sec. 4.5
 * eq. two_spmv), or in mode T the level-scheduled forward and backward
 * triangular solves with the factor (one launch per separator-tree height
 * and sweep). b, x: [n_v][3] device pointers (caller-owned); rows of pinned
 * vertices of b are ignored and those of x are set to 0. Uses the context's
 * work buffers, so it must not overlap a pd_rollout / pd_backward of the same
 * context on another stream. Enqueued on the stream; does not synchronise. */
int pd_solve(pd_ctx* ctx, const double* b, double* x, void* stream);

/* The local step alone (Sec. 4.1, Alg. 1 local step and RHS scatter): for
 * positions q, every element's projection p_e* (corotated: the polar factor
 * U V^T of F_e = G_e q; Neo-Hookean: the stretch prox of eq. nh_prox /
 * nh_prox_normal at k_bar), and the projection part of the right-hand side
 *   out[v] = sum_e w_e V_e G_e^T vec(p_e*)   (eq. A_basic),
 * summed per vertex in FP64 in a fixed order; rows of pinned vertices are
 * set to 0. The context's local precision (options.local_fp32) applies; the
 * Neo-Hookean prox starts from each element's last stretches. q, out:
 * [n_v][3] device pointers. After pd_factor (materials and weights);
 * single-instance contexts. Enqueued on the stream (two launches); does not
 * synchronise; must not overlap the context's rollouts. */
int pd_local_rhs(pd_ctx* ctx, const double* q, double* out, void* stream);

/* Same result as pd_solve, for callers that cannot allocate device memory
 * while they run (code under stream capture or in a real-time loop, hosts
 * whose device memory belongs to another allocator or a fixed arena). The
 * call allocates nothing: its two [n_f][3] work vectors live in one
 * file-scope device array sized for at most 65536 free vertices (3 MiB, held
 * by every GPU that loads the library until the process exits). The paper has
 * no counterpart; this is a convenience of this library.
 *   - Meshes with more than 65536 free vertices: PD_ERR_TOO_LARGE.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *     that first call before any stream capture. A device reset
 *     (cudaDeviceReset) after the first call is not supported: the kept
 *     address would belong to the destroyed context.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other contexts, other host threads) race. Each call overwrites
 *     it; the partial sums of long rows of S go to buffers that pd_factor
 *     sets aside for this call alone, so it shares nothing with the
 *     context's rollouts.
 * b, x: [n_v][3] device pointers; pinned rows of x are set to 0. */
int pd_solve_noalloc(pd_ctx* ctx, const double* b, double* x, void* stream);

/* Lumped vertex masses [n_v] (host output, kg): density * V_e / 4 per corner. */
int pd_get_mass(const pd_ctx* ctx, double* mass_host);

/* Position checkpoint q_t of the last rollout, 0 <= t <= T (q_0 with pinned
 * vertices at X, q_T the final state): [n_v][3] host output. Synchronous. */
int pd_get_checkpoint(const pd_ctx* ctx, int32_t t, double* q_host);

/* Per-step trust-region choices of the last rollout: tau [T] (host output). */
int pd_get_tau(const pd_ctx* ctx, double* tau_host, int32_t T);

int pd_get_stats(const pd_ctx* ctx, pd_stats* out);
const char* pd_last_error(const pd_ctx* ctx);
void pd_destroy(pd_ctx* ctx);

/* Phase timers while profiling is enabled (pd_profile). With per-phase
 * kernels, CUDA events on the work stream bracket the fused local step + RHS
 * assembly ("local") and the two SpMVs with S ("solve") of every forward
 * iteration. Persistent rollouts are timed per phase on the device. */
typedef struct {
  int64_t local_launches;
  double local_ms;
  int64_t solve_launches;
  double solve_ms;
  /* persistent rollouts: time per phase measured on the device (globaltimer,
   * block 0, including the grid barrier that ends the phase), summed over the
   * rollouts run since profiling was enabled: begin, local step, assembly +
   * gate, S b, S^T y with the Anderson dot products (through their
   * reduction), the small Anderson solve, update, step end + trust region */
  double phase_ms[8];
  double work_ms[8];  /* of which block 0's own work before the phase's barrier */
  double work_max_ms[8]; /* the largest total over the blocks of each block's own work per phase
                            (the critical block; the rest of phase_ms is barrier and reduction) */
  double last_ms[8];     /* per iteration, the phase's start (block 0) to the last block's arrival
                            at the phase's closing barrier, summed; approximate (block 0 may read
                            the last arrival's timestamp before it lands and then skips it) */
} pd_profile_out;

/* enable != 0 turns the phase timers on (and clears them); 0 turns them off. */
int pd_profile(pd_ctx* ctx, int32_t enable);
int pd_get_profile(const pd_ctx* ctx, pd_profile_out* out);

/* ---------------------------------------------------------------------
 * Capture-safe form of pd_rollout / pd_backward.
 *
 * pd_rollout and pd_backward synchronise the stream to read the iteration
 * statistics. The *_enqueue variants only enqueue work (memsets and one
 * cooperative persistent launch), so they can be recorded into a CUDA graph
 * by stream capture and replayed; pd_collect then synchronises the stream and
 * reads the statistics and status of the enqueued work. Requirements: every
 * pointer is a device pointer; options.persistent = 1 and a co-resident grid
 * (else PD_ERR_ARG); checkpoint storage for T steps exists (pd_reserve, or an
 * earlier rollout of >= T steps) when the stream is being captured. The
 * graph replays the buffers and shapes seen at capture time.
 * --------------------------------------------------------------------- */

/* Allocate checkpoint storage for rollouts of up to T steps (blocking). */
int pd_reserve(pd_ctx* ctx, int32_t T);

int pd_rollout_enqueue(pd_ctx* ctx, int32_t T, const double* q0, const double* v0, const double* f_ext,
                       int64_t f_ext_stride, double* qT, double* vT, void* stream);
int pd_backward_enqueue(pd_ctx* ctx, const double* dqT, const double* dvT, double* dq0, double* dv0,
                        double* dE, double* dnu, double* df_ext, int64_t df_stride, void* stream);

/* Synchronise the stream and fold the statistics of the work enqueued since
 * the last collect into pd_get_stats; returns what pd_rollout / pd_backward
 * would have returned (PD_ERR_NOT_CONVERGED, PD_ERR_TIMEOUT, ...). */
int pd_collect(pd_ctx* ctx, void* stream);

/* ---------------------------------------------------------------------
 * Batched instances (many independent meshes in one persistent launch).
 *
 * pd_create_batch makes one context for n independent problems: mesh i and
 * material i as for pd_create, one dt and one set of options for all. The
 * batch context takes the concatenation of the per-instance arrays
 * everywhere a single context takes one instance's: vertex arrays are
 * [sum n_v][3] (instance 0's vertices first), element arrays [sum n_e],
 * per-step forces [T][sum n_v][3] with f_ext_stride = 3 sum n_v (or
 * 0 for one [sum n_v][3] array), dnu is [n]. pd_factor factors every
 * instance (host threads in parallel). pd_rollout / pd_backward (and their
 * _enqueue forms) run all instances in ONE cooperative launch: the grid is
 * split into teams of blocks, one team per instance, with team sizes set by
 * the launch shape (pd_tuning; pd_autotune); each team iterates its own
 * instance to its own gate and synchronises only with itself, so a fast
 * instance never waits for a slow one. At most one instance per block of the
 * co-resident grid (2 x SMs): more gives PD_ERR_TOO_LARGE at launch.
 * pd_get_stats sums the per-instance statistics (iters_max, adj_iters_max:
 * maximum); pd_get_instance_stats gives one instance's. pd_get_mass,
 * pd_get_checkpoint give concatenated arrays; pd_get_tau gives [n][T].
 * pd_solve, pd_solve_noalloc and pd_profile are single-instance only.
 * --------------------------------------------------------------------- */
int pd_create_batch(int32_t n, const pd_mesh* meshes, const pd_material* mats, double dt,
                    const pd_options* opt, pd_ctx** out);

/* Number of instances (1 for a single-instance context) and the prefix
 * offsets of their vertices and elements (host outputs [n+1] each, may be
 * NULL). */
int pd_batch_info(const pd_ctx* ctx, int32_t* n, int64_t* v_off, int64_t* e_off);

/* Batch form of pd_set_materials: E [sum n_e] (Pa), nu [n]. */
int pd_set_materials_batch(pd_ctx* ctx, const double* E, const double* nu);

int pd_get_instance_stats(const pd_ctx* ctx, int32_t i, pd_stats* out);

/* Team sizes (blocks per instance) that the current launch shape gives the
 * forward and the adjoint launch: fwd, bwd [n] host outputs (either may be
 * NULL). The shape is fixed until pd_factor, pd_set_tuning or pd_autotune
 * changes it. Batch contexts only; after pd_factor. */
int pd_batch_teams(pd_ctx* ctx, int32_t* fwd, int32_t* bwd);

/* ---------------------------------------------------------------------
 * Launch shape of the persistent kernels and its autotuner.
 * --------------------------------------------------------------------- */
typedef struct {
  int32_t fwd_blocks_per_sm;  /* forward: 1 = one block of 384 threads per SM (registers for every
                                 phase, no spills), 2 = two blocks of 256 per SM (more co-resident
                                 blocks for batches); 0 = 1 for a single instance, 2 for a batch */
  int32_t bwd_blocks_per_sm;
  int32_t fwd_grid;           /* single instance: blocks of the launch (0 = SMs x blocks_per_sm) */
  int32_t bwd_grid;
  double fwd_gamma;           /* batch: an instance's time is taken to scale as (team size)^-gamma */
  double bwd_gamma;
  int32_t fwd_min_items;      /* batch: a team gets at most ceil(n_e / min_items) blocks */
  int32_t bwd_min_items;
  double fwd_ms;              /* pd_autotune: probe time of the chosen forward shape */
  double bwd_ms;              /* ... backward shape */
  int32_t candidates;         /* shapes timed by the last pd_autotune (0: found in the cache) */
  int32_t reserved;
} pd_tuning;

/* Choose the launch shape by timing probe rollouts of T_probe steps from
 * (q0, v0, f_ext) (as pd_rollout; device pointers) and their adjoints over
 * a fixed candidate set: blocks per SM; for a single instance, the grid
 * size; for a batch (two blocks per SM), the exponent gamma (0.5, 0.75, 1)
 * and the cap on blocks per element count (32, 128 or 512 elements per block
 * at least). Batch team sizes minimise the largest predicted instance time,
 * where an instance's time with b blocks is predicted from its own measured
 * time in the last full pd_rollout / pd_backward (each team times itself on
 * the device) scaled by (measured team size / b)^gamma; run one rollout and
 * adjoint over the real horizon first (a short probe does not see the slow
 * steps). Without a measurement the prediction is iterations x bytes per
 * iteration / b^gamma. The choice is kept in
 * the context and cached in the process, keyed by device and problem
 * signature (instance sizes, nnz(S), options), so a second context of the
 * same problem reuses it without probing. Overwrites the checkpoints (run
 * pd_rollout again before pd_backward). Blocking. out may be NULL. */
int pd_autotune(pd_ctx* ctx, int32_t T_probe, const double* q0, const double* v0, const double* f_ext,
                int64_t f_ext_stride, pd_tuning* out, void* stream);
int pd_get_tuning(const pd_ctx* ctx, pd_tuning* out);
/* Set the launch shape directly (e.g. one saved from pd_get_tuning). */
int pd_set_tuning(pd_ctx* ctx, const pd_tuning* t);

/* ---------------------------------------------------------------------
 * Learned warm start (not part of the paper's method).
 *
 * A per-vertex network predicts the correction r to the constant-velocity
 * guess, and each step's local-global iteration starts from
 *   q0 = 2 x_t - x_{t-1} + r,   x_{t-1} = x_t - h v_t,
 * instead of q_t (Alg. 1), on free vertices (options.warm_start = 1). The
 * network: features f = [x_t - x_{t-1}, x_t - X, log10(E_v / 1e5)] (E_v the
 * volume-weighted mean Young's modulus of the elements around v),
 * normalised (f - mean) / scale; 4 dense layers 7 -> 128 -> 128 -> 128 -> 3
 * with ReLU between them; output times oscale. Parameters (FP32, 34,435) in
 * one flat vector: W1 [128][7], b1 [128], W2 [128][128], b2 [128],
 * W3 [128][128], b3 [128], W4 [3][128], b4 [3]; normalisation (17 floats):
 * feature mean [7], feature scale [7], output scale [3]. Inference and
 * training forward passes use the weights rounded to BF16 (nearest even),
 * biases in FP32, FP32 arithmetic. The converged step does not depend on
 * the start: the network only changes iteration counts, and a warm-started
 * step that hits k_max is run again from q_t.
 * --------------------------------------------------------------------- */
#define PD_MLP_PARAMS 34435
#define PD_MLP_NORM 17

typedef struct pd_mlp pd_mlp;

/* Trainer on the current device: FP32 master parameters theta [PD_MLP_PARAMS]
 * and normalisation norm [PD_MLP_NORM] (host arrays, copied), Adam moments at
 * zero. On failure *out may hold a trainer whose pd_mlp_last_error explains. */
int pd_mlp_create(const float* theta, const float* norm, pd_mlp** out);
/* Host copies of the master parameters and the normalisation (either may be NULL). */
int pd_mlp_params(const pd_mlp* net, float* theta, float* norm);
/* Set the normalisation from n samples (device arrays feat [n][7], targ
 * [n][3], raw units): feature mean and standard deviation (1 where it is
 * below 1e-12), output scale = root mean square of each target component. */
int pd_mlp_fit_normalization(pd_mlp* net, const float* feat, const float* targ, int64_t n, void* stream);
/* r [n][3] (raw units) for raw features feat [n][7] (device arrays). */
int pd_mlp_forward(pd_mlp* net, const float* feat, float* r, int64_t n, void* stream);
/* Loss = mean over the n samples and 3 outputs of (net(f) - targ / oscale)^2
 * (host *loss, may be NULL) and its gradient with respect to the parameters
 * (device grad [PD_MLP_PARAMS], may be NULL), by backpropagation. */
int pd_mlp_grad(pd_mlp* net, const float* feat, const float* targ, int64_t n, float* grad, double* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; Kingma & Ba 2015,
 * Algorithm 1) of learning rate lr on the loss of the n samples. */
int pd_mlp_train_step(pd_mlp* net, const float* feat, const float* targ, int64_t n, double lr, double* loss,
                      void* stream);
const char* pd_mlp_last_error(const pd_mlp* net);
void pd_mlp_destroy(pd_mlp* net);

/* Training samples of one frame of a trajectory of the context's mesh:
 * raw features feat [n_v][7] of (x_{t-1}, x_t) and, if x_tp1 is given, raw
 * targets targ [n_v][3] = x_{t+1} - (2 x_t - x_{t-1}) (device arrays, every
 * vertex in order; pinned vertices give zero rows). A batch context takes the
 * concatenated arrays of all its instances (one launch per instance). */
int pd_mlp_sample(pd_ctx* ctx, const double* x_tm1, const double* x_t, const double* x_tp1, float* feat,
                  float* targ, void* stream);

/* Attach a network to a context (a batch: to every instance): weights =
 * FP32 parameters [PD_MLP_PARAMS] followed by the normalisation
 * [PD_MLP_NORM], bytes = 4 x (PD_MLP_PARAMS + PD_MLP_NORM), host memory. */
int pd_mlp_load(pd_ctx* ctx, const void* weights, size_t bytes);

/* Change the start of each step's iteration (pd_options.warm_start: 0 q_t,
 * 1 the learned warm start, 2 constant-velocity extrapolation) without
 * recreating or refactoring the context; 1 needs a loaded network. For a
 * batch, every instance. Takes effect at the next rollout. Not part of the
 * paper (its iteration starts from q_t, Alg. 1). */
int pd_set_warm_start(pd_ctx* ctx, int32_t mode);

/* The warm start as the rollout computes it: q0 [n_v][3] from x_t, x_{t-1}
 * (device arrays) with options.warm_start (1: the loaded network; 2 or 0:
 * constant velocity); pinned vertices at X. Single instance. */
int pd_warm_start(pd_ctx* ctx, const double* x_t, const double* x_tm1, double* q0, void* stream);

/* ---------------------------------------------------------------------
 * L-BFGS driver for inverse problems (the paper's optimiser for system
 * identification and initial-state tasks, Sec. 5.4 / 5.5, run on the
 * gradients of pd_backward).
 *
 * Limited-memory BFGS (Nocedal and Wright, Numerical Optimization, 2nd ed.,
 * 2006: the two-loop recursion of Alg. 7.4 with H0 = (s^T y / y^T y) I,
 * Sec. 7.2) with a line search satisfying the strong Wolfe conditions
 * (Alg. 3.5 bracketing with step doubling, Alg. 3.6 zoom by safeguarded
 * cubic interpolation, eq. 3.59). Host FP64; the parameter vector is small
 * (per-block moduli, initial states), the simulation it wraps runs on the
 * device.
 *
 * Reverse communication: the caller owns x [n] (host) and evaluates
 * f(x), g(x) wherever the optimiser asks:
 *   pd_lbfgs_create(n, opts, &o); evaluate f, g at x0;
 *   loop: pd_lbfgs_next(o, x, f, g, &task)
 *     task PD_LBFGS_EVAL:      x holds a trial point: evaluate f, g there
 *     task PD_LBFGS_ITERATE:   x holds the accepted iterate (f, g of the
 *                              last evaluation belong to it); call again
 *     task PD_LBFGS_CONVERGED: max |g| <= gtol, or a relative decrease of f
 *                              of at most ftol; x holds the last iterate
 *     task PD_LBFGS_STOP:      max_iters or max_evals reached
 *     task PD_LBFGS_FAILED:    the line search found no acceptable step
 *                              along steepest descent either (x: last iterate)
 * f and g are read on every call except right after PD_LBFGS_ITERATE. A
 * direction that is not a descent direction, or a line search that fails
 * with curvature pairs stored, clears the memory and restarts from
 * steepest descent. Pairs with s^T y <= 1e-12 y^T y are skipped.
 * Returns PD_ERR_ARG for bad sizes or options, PD_ERR_NUMERIC for a
 * non-finite f or g at an iterate (a non-finite trial value shrinks the
 * step instead).
 * --------------------------------------------------------------------- */
typedef struct pd_lbfgs pd_lbfgs;
enum { PD_LBFGS_EVAL = 1, PD_LBFGS_ITERATE = 2, PD_LBFGS_CONVERGED = 3, PD_LBFGS_STOP = 4, PD_LBFGS_FAILED = 5 };
typedef struct {
  int32_t m;          /* stored curvature pairs (default 10) */
  int32_t max_iters;  /* accepted iterations (default 100) */
  int32_t max_evals;  /* function evaluations, the initial one included (default 200) */
  int32_t max_ls;     /* evaluations per line search (default 20) */
  double gtol;        /* max |g| at convergence (default 1e-8) */
  double ftol;        /* (f_k - f_k+1) / max(|f_k|, |f_k+1|, 1) at convergence (default 1e-12) */
  double c1, c2;      /* sufficient decrease and curvature constants (default 1e-4, 0.9) */
  double step0;       /* length of the first trial step, steepest descent (default 1) */
} pd_lbfgs_options;

/* Defaults of every field. */
void pd_lbfgs_default_options(pd_lbfgs_options* opts);
int pd_lbfgs_create(int32_t n, const pd_lbfgs_options* opts, pd_lbfgs** out);
int pd_lbfgs_next(pd_lbfgs* o, double* x, double f, const double* g, int32_t* task);
/* Counters and the last iterate's f and max |g| (any pointer may be NULL). */
int pd_lbfgs_info(const pd_lbfgs* o, int32_t* iters, int32_t* evals, double* f, double* gmax);
void pd_lbfgs_destroy(pd_lbfgs* o);

/* Library version string. */
const char* pd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PD_B300_H */
