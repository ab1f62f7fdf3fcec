/*
 * ddfd.h -- C ABI of the GB300 (sm_103a) hot path of the adaptive domain
 * decomposition FE/FD method for the stabilized time-dependent Maxwell
 * system in conductive media (Kyhn, Lindstrom, Beilina, arXiv 2508.07780).
 *
 * The library time-steps the model problem of Sec. 5 (eq. model1; the same
 * equation as eq. forward_prob of Sec. 2)
 *
 *     eps d_tt E + sigma d_t E - Lap E - grad div((eps - 1) E) = 0
 *
 * forward for the state E, backward for the adjoint lambda of eq.
 * adjoint_prob (Sec. 3), driven by the detector residuals E - Eobs, and
 * accumulates the gradient of the Tikhonov functional (eq.
 * tikhonov_functional) with respect to eps and sigma (eq. gradeps, Sec. 4).
 *
 * Discretisation (all of it computed on the GPU):
 *   - grid: n^3 nodes on [0,1]^3, h = 1/(n-1), node id i + n*(j + n*k),
 *     x fastest, k = depth, top (incident, observed) face k = n-1;
 *   - outer region: finite differences on the hexahedral grid (7-point
 *     Laplacian, ghost-node Neumann closure, lumped trapezoid masses);
 *   - inner FEM cube: node box [a,b]^3, a = (n - fem_n)/2 (integer division),
 *     b = a + fem_n - 1, P1 elements on the six Kuhn tetrahedra of each cube,
 *     lumped mass; FEM rows for nodes strictly inside the box;
 *   - free (coefficient) nodes: [a+2, b-2]^3, listed x fastest; every other
 *     node has eps = 1, sigma = 0 (eq. epsilon_sigma_constraint);
 *   - explicit central time stepping, tau = cfl * h, E(0) = d_t E(0) = 0;
 *   - boundary: Neumann flux P on the top face for steps n <= n1 (n1 =
 *     floor(t1/tau + 1e-9)), first-order absorbing d_n E = -d_t E on the top
 *     face afterwards and on the bottom face always, d_n E = 0 on the sides
 *     (eq. model1); the absorbing set is configurable.
 *
 * Conventions:
 *   - every call returns a ddfd_status; nothing is thrown across the ABI;
 *   - on error, outputs are untouched and ddfd_last_error() holds a message
 *     (one stated exception: ddfd_cg_run hands back the records and the
 *     iterate of a run that failed part-way);
 *   - the caller owns every buffer it passes; host inputs are copied before
 *     the call returns; device pointers must stay valid until the call
 *     returns (the library synchronises its stream before returning from
 *     every call that takes a caller buffer);
 *   - one handle per thread; handles are independent;
 *   - no CPU fallback: without a usable CUDA device ddfd_create fails with
 *     DDFD_E_CUDA.
 */
#ifndef DDFD_H
#define DDFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddfd_problem ddfd_problem; /* opaque; owns all its device memory */
typedef struct ddfd_batch ddfd_batch;     /* opaque; a set of problems stepped together */

typedef enum {
  DDFD_OK = 0,
  DDFD_E_ARG = -1,       /* invalid argument or configuration */
  DDFD_E_CFL = -2,       /* tau above the stability bound of the current coefficients */
  DDFD_E_STATE = -3,     /* call out of order (adjoint before forward, ...) */
  DDFD_E_CUDA = -4,      /* CUDA runtime error (message has the CUDA text) */
  DDFD_E_OOM = -5,       /* device memory (or the configured budget) exhausted */
  DDFD_E_NONFINITE = -6, /* a non-finite value appeared in a trace or gradient */
  DDFD_E_TIMEOUT = -7,   /* a bounded device wait gave up */
  DDFD_E_COEFF = -8      /* coefficient outside [1, eps_max] x [0, sig_max] or non-finite */
} ddfd_status;

enum { DDFD_FP64 = 0, DDFD_FP32 = 1 };           /* field precision; reductions are FP64 */
enum { DDFD_SRC_GAUSS = 0, DDFD_SRC_SINE = 1 };  /* pulse shape, see ddfd_config */
/* FEM apply: Kuhn block stencil / element gather over the Kuhn split /
 * element gather over an explicit, locally refined mesh (mesh_* fields) */
enum { DDFD_FEM_STENCIL = 0, DDFD_FEM_EBE = 1, DDFD_FEM_MESH = 2 };
enum { DDFD_GRAD_EXACT = 0, DDFD_GRAD_LITERAL = 1 };  /* gradient form, see ddfd_config */
enum {
  DDFD_ABS_BOTTOM = 1, DDFD_ABS_TOP = 2, /* top: only after the source phase */
  DDFD_ABS_X0 = 4, DDFD_ABS_X1 = 8, DDFD_ABS_Y0 = 16, DDFD_ABS_Y1 = 32
};

typedef struct {
  int32_t n;             /* grid nodes per axis, 7 <= n <= 1024 */
  int32_t fem_n;         /* FEM cube nodes per axis, 5 <= fem_n <= n - 2 */
  int32_t n_steps;       /* Nt >= 1 time steps */
  double cfl;            /* tau = cfl * h; 0 < cfl */
  int32_t precision;     /* DDFD_FP64 or DDFD_FP32 */
  int32_t fem_kind;      /* DDFD_FEM_STENCIL (default), DDFD_FEM_EBE or DDFD_FEM_MESH */
  int32_t n_src;         /* incident plane waves, >= 1; J and g sum over them */
  const double *src_dir; /* [n_src][3] propagation directions k (k_z < 0), or NULL
                            for normal incidence k = (0,0,-1); copied */
  int32_t source_kind;   /* DDFD_SRC_GAUSS: P(t) = sin(2 pi f (t-t0)) exp(-((t-t0)/w)^2);
                            DDFD_SRC_SINE: the paper's eq. f, sin(2 pi f t) on (0, 1/f) */
  double freq, t0, width;/* f, t0, w of the pulse */
  double t1;             /* end of the source phase; < 0: pulse end (t0 + 3w, or 1/f)
                            plus the largest oblique delay */
  int32_t n_det;         /* detectors, >= 0 */
  const int32_t *det_ij; /* [n_det][2] top-face node indices (i, j); copied */
  uint32_t absorbing_faces; /* DDFD_ABS_* bits; default BOTTOM|TOP */
  double gamma_eps, gamma_sig; /* Tikhonov regularisation parameters (>= 0) */
  double z_delta_frac;   /* observation taper z_delta: 1 up to T - d, cosine to 0 at T,
                            d = frac * T; 0 disables it */
  double eps_max, sig_max; /* coefficient bounds checked by ddfd_set_coeffs */
  int32_t n_snapshots;   /* 0: keep E on the free nodes for every step in device memory;
                            1..n_steps: checkpointing -- the forward keeps the state
                            (E^n, E^{n-1}) at the starts of n_snapshots equal segments
                            and the adjoint replays each segment's forward steps from its
                            snapshot into a one-segment history (one extra forward sweep;
                            results are bitwise those of the full history) */
  int32_t cfl_check;     /* nonzero: estimate the stability bound by power iteration
                            at ddfd_set_coeffs and fail with DDFD_E_CFL above it */
  int64_t mem_budget;    /* device bytes the handle may allocate; 0 = no limit */
  int32_t tile_kz;       /* z planes per thread block of the full step kernel (FP32 tiles
                            holding FEM-cube or free nodes; every FP64 tile); tuning:
                            0 = library default (16 for n >= 128, else 8), else 2..n */
  int32_t forward_only;  /* nonzero: keep neither the E history nor snapshots (for
                            data generation); ddfd_adjoint then fails with DDFD_E_STATE */
  /* fem_kind = DDFD_FEM_MESH: the tetrahedra of the FEM cube [a, b]^3, a locally
     refined mesh (Sec. 4, the adaptive refinement that eq. meshref marks).  Node
     ids: grid node i + n (j + n k) (inside [a, b]^3), new node e = n^3 + e, the
     midpoint of its two parents mesh_parents[e] (ids below n^3 + e).  New nodes
     must lie in the free box [a+2, b-2]^3 and are free nodes: the coefficient
     arrays list the grid's free nodes (x fastest), then the new nodes.  Rows of
     the grid nodes strictly inside the cube and of the new nodes are P1 rows
     over these tetrahedra (lumped masses); the time step must suit the smallest
     elements.  Not combined with n_snapshots or cfl_check.  Copied. */
  int32_t mesh_n_new;
  const int32_t *mesh_parents;   /* [mesh_n_new][2] */
  int64_t mesh_n_tets;
  const int32_t *mesh_tets;      /* [mesh_n_tets][4] */
  void *stream;          /* cudaStream_t for all work, or NULL for the default stream */
  int32_t grad_variant;  /* DDFD_GRAD_EXACT (default): g is the exact derivative of the
                            discrete J; DDFD_GRAD_LITERAL: eq. gradeps as printed in Sec. 4,
                            with div(eps_bar E) ~ eps_bar div E (the Gauss-law term becomes
                            sum_K |K|/4 (div E)_K (div mu)_K around each free node).  The
                            literal variant keeps E on every FEM-updated node for every step
                            and takes neither n_snapshots, forward_only, fem_kind other than
                            DDFD_FEM_STENCIL, nor batches. */
  int32_t tile_kz_lean;  /* z planes per thread block of the lean FP32 step kernel (the
                            finite-difference-only tiles, run beside the full kernel);
                            tuning: 0 = library default (16 for n >= 128, else 8), else 2..64 */
} ddfd_config;

/* Fill *cfg with defaults: cfl 0.3, FP64, stencil FEM, 1 normal-incidence
 * source, Gaussian pulse f = 2, t0 = 0.75, w = 0.25, t1 auto, absorbing
 * bottom|top, gammas 0, z_delta_frac 0.1, eps_max 100, sig_max 100, no
 * snapshots (full history), cfl_check 0, no budget, default stream.  n,
 * fem_n, n_steps and the detectors are left zero. */
void ddfd_config_default(ddfd_config *cfg);

/* Validate *cfg and allocate a handle with vacuum coefficients (eps = 1,
 * sigma = 0).  Errors: DDFD_E_ARG (bad sizes, detector off the grid,
 * direction with k_z >= 0), DDFD_E_OOM, DDFD_E_CUDA.  *out is set only on
 * success. */
int ddfd_create(const ddfd_config *cfg, ddfd_problem **out);

/* Release the handle and all its device memory.  NULL is allowed. */
void ddfd_destroy(ddfd_problem *p);

/* Message of the last failing call on this handle ("" if none).  Valid until
 * the next call on the handle. */
const char *ddfd_last_error(const ddfd_problem *p);

/* Message of the last ddfd_create failure in this thread. */
const char *ddfd_create_error(void);

/* Nodal coefficients on the free nodes (eq. epsilon_sigma_constraint;
 * the unknowns of the inverse problem, eq. inverse_problem), in free-node
 * order (x fastest over [a+2, b-2]^3), (fem_n - 4)^3 doubles each, host
 * memory.  eps0/sig0 are the regularisation centres of eq.
 * tikhonov_functional; NULL means eps0 = 1, sig0 = 0.  Checks
 * 1 <= eps <= eps_max and 0 <= sigma <= sig_max (DDFD_E_COEFF).  Builds the
 * per-node step coefficients on the device and invalidates any forward or
 * adjoint state.  With cfl_check, fails with DDFD_E_CFL if tau exceeds
 * 2/sqrt(lambda_max(M_eps^-1 K)). */
int ddfd_set_coeffs(ddfd_problem *p, const double *eps, const double *sig,
                    const double *eps0, const double *sig0);
/* Same, with device pointers (same layout; eps0/sig0 may be NULL). */
int ddfd_set_coeffs_dev(ddfd_problem *p, const double *eps, const double *sig,
                        const double *eps0, const double *sig0);

/* Forward solve for every source (eq. model1, Sec. 5): E^0 = E^-1 = 0, then
 * Nt explicit steps.  Records the detector trace and keeps what the adjoint
 * needs (E on the free nodes, or checkpoints).  trace_out, if not NULL,
 * receives [n_src][n_steps + 1][n_det][3] doubles (host), E at the detector
 * nodes for t_0 .. t_Nt.  Errors: DDFD_E_NONFINITE if the trace holds a
 * non-finite value, DDFD_E_CUDA. */
int ddfd_forward(ddfd_problem *p, double *trace_out);
/* Same; trace_out (may be NULL) is a device pointer. */
int ddfd_forward_dev(ddfd_problem *p, double *trace_out);

/* Tikhonov functional (eq. tikhonov_functional) of the last forward run:
 * J = tau/2 sum_{s, n=1..Nt} z(t_n) sum_d |E^n_d - Eobs^n_d|^2
 *   + gamma_eps/2 sum_i m_i (eps_i - eps0_i)^2 + gamma_sig/2 sum_i m_i (sig_i - sig0_i)^2,
 * reduced in FP64.  eobs has the trace layout (host).  Requires a forward
 * run (DDFD_E_STATE). */
int ddfd_functional(ddfd_problem *p, const double *eobs, double *J);
/* Same; eobs is a device pointer, *J a host double. */
int ddfd_functional_dev(ddfd_problem *p, const double *eobs, double *J);

/* Adjoint solve for every source (eq. adjoint_prob, Sec. 3, as the exact
 * transpose of the discrete forward recursion), backward from t_Nt with zero
 * terminal data, driven by j^k = tau z(t_k) (E^k - Eobs^k) at the detectors.
 * The gradient time integrals are accumulated in the same kernels.  eobs:
 * trace layout, host.  Requires a forward run (DDFD_E_STATE). */
int ddfd_adjoint(ddfd_problem *p, const double *eobs);
/* Same; eobs is a device pointer. */
int ddfd_adjoint_dev(ddfd_problem *p, const double *eobs);

/* Gradient of the discrete J with respect to the free-node eps and sigma
 * (eq. gradeps, Sec. 4, taken as the exact derivative of the discrete
 * functional), summed over sources, FP64, free-node order, host.  Requires
 * an adjoint run (DDFD_E_STATE).  DDFD_E_NONFINITE if non-finite. */
int ddfd_gradient(ddfd_problem *p, double *g_eps, double *g_sig);
/* Same; outputs are device pointers. */
int ddfd_gradient_dev(ddfd_problem *p, double *g_eps, double *g_sig);

/* Sizes and bookkeeping of a handle. */
typedef struct {
  int32_t n, fem_n, n_free, n_det, n_src, n_steps;
  int32_t a, b, switch_step;   /* FEM box [a,b]; last source step n1 (per source 0) */
  double h, tau;
  int64_t device_bytes;        /* bytes allocated by the handle */
  int64_t kernel_launches;     /* kernels launched by the handle so far */
  int64_t forward_steps;       /* forward steps executed so far (replays included) */
  int64_t generation;          /* incremented by every ddfd_set_coeffs and every forward run
                                  (single or batched); a caller that keeps results of a run can
                                  compare it to tell whether the handle's state is still theirs */
} ddfd_info;
int ddfd_get_info(const ddfd_problem *p, ddfd_info *info);

/* Device time of the last forward / adjoint sequences, measured with CUDA
 * events recorded on the handle's stream around each (all sources, with the
 * forward replays of checkpointing in the adjoint sequence), and the number
 * of step kernels each launched.  loop_ms / kernels is the average step-kernel
 * time including the small per-source set-up.  Zero before a run. */
typedef struct {
  double forward_loop_ms, adjoint_loop_ms;
  int64_t forward_step_kernels, adjoint_step_kernels;
} ddfd_timing;
int ddfd_get_timing(const ddfd_problem *p, ddfd_timing *t);

/* Capture full fields for testing: before ddfd_forward / ddfd_adjoint, name
 * up to 16 step indices; the forward then keeps E^n and the adjoint mu^n
 * (the multiplier of the step equations; lambda ~ mu / tau) of source 0 at
 * those steps.  ddfd_get_capture copies capture idx of kind 0 (E) or 1 (mu)
 * as 3 * n^3 doubles (component-major, node order) to host memory. */
int ddfd_set_capture(ddfd_problem *p, int32_t count, const int32_t *steps);
int ddfd_get_capture(ddfd_problem *p, int32_t kind, int32_t idx, double *out);

/* Device time of one step's element-apply launches (fem_kind DDFD_FEM_EBE or
 * DDFD_FEM_MESH): the element gather, and for refined meshes the rows taken
 * from the block stencil, run `reps` >= 1 times in the forward form and in
 * the adjoint form on the handle's current fields, timed with CUDA events on
 * its stream.  *fwd_ms, *adj_ms (may be NULL) receive the average per step
 * (adj_ms 0 for forward_only handles); *fwd_bytes, *adj_bytes (may be NULL)
 * the algorithmic bytes of those launches: each gathered tet's four node ids
 * and twelve gradient values, each of its nodes' values once (field and s
 * forward, field adjoint), each row's outputs (R forward; R and q adjoint),
 * and for stencil rows their own node values and outputs.  The launches only
 * overwrite the gather's row scratch, so the handle's state is unchanged.
 * Errors: DDFD_E_ARG (no element gather, reps < 1), DDFD_E_TIMEOUT,
 * DDFD_E_CUDA.  The paper has no counterpart (a measurement aid). */
int ddfd_time_gather(ddfd_problem *p, int32_t reps, double *fwd_ms, double *adj_ms, int64_t *fwd_bytes,
                     int64_t *adj_bytes);

/* Failure-detection test hook (not for production runs; the paper has no
 * counterpart).  fault = 1: the first thread block of the element gather
 * never starts the bulk copy of its first block of rows, so the mbarrier it
 * waits on is never completed; its bounded wait gives up after spin_limit
 * polls (0: the default 1 << 22), it records the timeout and returns, and the
 * ddfd_forward / ddfd_adjoint that ran it fails with DDFD_E_TIMEOUT.  No copy
 * is left in flight and no fault is raised, so the handle stays usable.
 * fault = 0 restores normal operation.  Needs fem_kind DDFD_FEM_EBE or
 * DDFD_FEM_MESH (DDFD_E_ARG otherwise). */
int ddfd_test_gather_timeout(ddfd_problem *p, int32_t fault, uint32_t spin_limit);

/* Host-only inspection of the step kernels' dispatch order (no device call,
 * no handle; the paper has no counterpart).  Builds the item list of one step
 * launch over nprob problems of n^3 nodes (precision DDFD_FP32 or DDFD_FP64)
 * whose FEM cube spans nodes [a, b] and free box [f0, f0 + nf) on each axis,
 * boxes[4 q .. 4 q + 3] = (a, b, f0, nf) for problem q, with z depths kz (full
 * kernel, FP64 kernel) and kz_lean (lean FP32 kernel).  Each item packs tile x
 * (bits 0-4, 32 nodes a tile), tile y (bits 5-11; 16 rows FP32, 8 FP64), the
 * first plane z0 (bits 12-21), the plane count minus one (bits 22-27) and the
 * problem (bits 28-31); the first *n_full items run on the full kernel.  Up to
 * cap items are written to items (may be NULL with cap = 0); *n_items gets
 * the count.  DDFD_E_ARG: n outside [7, 1024], nprob outside [1, 16], a depth
 * outside [1, 64], a box outside the grid, or cap too small (with *n_items
 * set). */
int ddfd_test_step_items(int32_t n, int32_t precision, int32_t nprob, const int32_t *boxes, int32_t kz,
                         int32_t kz_lean, uint32_t *items, int64_t cap, int64_t *n_items, int64_t *n_full);

/* Tile autotuner for the step kernels of one handle.  Times `steps` forward
 * and `steps` adjoint steps (CUDA events on the handle's stream) for each
 * candidate z depth of the full kernel's thread-block tiles (4, 6, 8, 12, 16,
 * 24, 32, up to n), the lean kernel's depth held, and keeps the fastest; in
 * FP32 it then does the same for the lean kernel's depth.  *tile_kz_out (may
 * be NULL) receives the full kernel's depth (ddfd_batch_get_info reports
 * both for a batch).  The trial steps overwrite the fields, so forward
 * and adjoint state are invalidated (run ddfd_forward again).  1 <= steps
 * <= n_steps.  The paper has no counterpart (a GPU tuning aid). */
int ddfd_autotune(ddfd_problem *p, int32_t steps, int32_t *tile_kz_out);

/* Batched heterogeneous problems.  count (1..256) problems with the same n,
 * n_steps, cfl and precision, each with its own FEM cube size fem_n, FEM
 * apply (fem_kind; element members add their own gather and new-node
 * launches around the batched step), detectors, absorbing faces,
 * regularisation, n_snapshots and one incident plane wave (n_src = 1, src_dir may differ;
 * several waves on one model are several members with the same
 * coefficients).  The members' fields are stacked in one allocation and
 * every time step of the whole batch is one kernel launch per group of 16
 * members, the whole forward (adjoint) sequence one CUDA graph.  Members
 * that checkpoint (n_snapshots > 0) must share the segment length
 * ceil(n_steps / n_snapshots).  Stream: cfgs[0].stream for all work.
 * The paper solves its measurements one by one; batching is a GPU
 * throughput device and changes no result: a member's trace, J and
 * gradient are bitwise those of the same problem run alone.
 * Errors: DDFD_E_ARG (mismatched members), DDFD_E_OOM, DDFD_E_CUDA; the
 * message is ddfd_create_error(). */
int ddfd_create_batch(const ddfd_config *cfgs, int32_t count, ddfd_batch **out);
void ddfd_destroy_batch(ddfd_batch *b);  /* NULL allowed; destroys the members too */
const char *ddfd_batch_last_error(const ddfd_batch *b);

/* Member i as a problem handle, owned by the batch (ddfd_destroy ignores
 * it).  Every single-problem call works on it: ddfd_set_coeffs,
 * ddfd_functional, ddfd_gradient after a batch run, and also ddfd_forward /
 * ddfd_adjoint, which run that member alone. */
int ddfd_batch_member(ddfd_batch *b, int32_t i, ddfd_problem **out);

/* Forward solve of every member in the batched launches.  trace_out may be
 * NULL; else trace_out[i] (may be NULL) receives member i's trace (host,
 * layout of ddfd_forward).  Afterwards every member is in the forward state. */
int ddfd_batch_forward(ddfd_batch *b, double *const *trace_out);
/* Same; trace_out[i] are device pointers. */
int ddfd_batch_forward_dev(ddfd_batch *b, double *const *trace_out);

/* Adjoint solve of every member in the batched launches; eobs[i] is member
 * i's observed trace (host, layout of ddfd_adjoint).  Requires every member
 * in the forward state (DDFD_E_STATE).  Afterwards ddfd_gradient(member)
 * returns each member's gradient. */
int ddfd_batch_adjoint(ddfd_batch *b, const double *const *eobs);
/* Same; eobs[i] are device pointers. */
int ddfd_batch_adjoint_dev(ddfd_batch *b, const double *const *eobs);

/* The tile autotuner of ddfd_autotune, timing the batched launches; it
 * invalidates every member's forward and adjoint state. */
int ddfd_batch_autotune(ddfd_batch *b, int32_t steps, int32_t *tile_kz_out);

/* Bookkeeping of a batch: timing of the last batched forward / adjoint
 * sequences (device time, CUDA events on the batch stream; the step-kernel
 * counts count one per batched step of a group of up to 16 members, which
 * runs one kernel, or in FP32 the full and the lean kernel side by side),
 * kernels launched, device bytes of the batch and its members, and the tile
 * depths in use (full kernel, lean kernel). */
typedef struct {
  int32_t count, tile_kz;
  double forward_loop_ms, adjoint_loop_ms;
  int64_t forward_step_kernels, adjoint_step_kernels;
  int64_t kernel_launches;
  int64_t device_bytes;
  int32_t tile_kz_lean;
} ddfd_batch_info;
int ddfd_batch_get_info(const ddfd_batch *b, ddfd_batch_info *info);

/* Conjugate gradient reconstruction (Sec. 4, the CGA): iterations m = 0, 1, ...
 * of  1) E^m, lambda^m and g^m at (eps^m, sig^m) for every member of the batch
 * (the members are the measurements -- incident waves -- of one model: same
 * fem_n, and gamma_eps = gamma_sig = 0 in their configurations, the CG
 * supplies the regularisation);  2)-3) Fletcher-Reeves directions
 * d^m = -g^m + beta^m d^{m-1}, beta^m = ||g^m||^2 / ||g^{m-1}||^2, d^0 = -g^0, and
 * updates eps^{m+1} = eps^m + alpha_eps^m d_eps^m (sigma likewise), clamped to
 * [1, eps_max] x [0, sig_max];  4) alpha^{m+1} = -(g^m, d^m) / (gamma^m (d^m, d^m));
 * 5) gamma^{m+1} = gamma^0 / (m+1)^p;  6) stop when (||eps^{m+1} - eps^m|| < eta1_eps
 * or ||sig^{m+1} - sig^m|| < eta1_sig) and (||g_eps^m|| < eta2_eps or ||g_sig^m|| <
 * eta2_sig), or after max_iter iterations.
 * g^m is the L2(Omega) representative of the derivative of the discrete
 * functional (the summed member gradients divided by the lumped mass h^3)
 * plus gamma^m (eps^m - eps^0); (u, v) = h^3 sum over the free nodes; the
 * initial guess eps^0, sig^0 is the regularisation centre (eq.
 * tikhonov_functional).  Inner products, norms and step sizes are FP64;
 * every vector operation runs on the GPU, the scalar rules on the host. */
typedef struct {
  int32_t max_iter;                 /* M >= 1 */
  double gamma_eps0, gamma_sig0;    /* gamma^0 >= 0 */
  double alpha_eps0, alpha_sig0;    /* alpha^0 */
  double p;                         /* gamma schedule exponent, 0 <= p < 1 */
  double eta1_eps, eta1_sig, eta2_eps, eta2_sig;  /* stopping tolerances (0: never) */
  double eps_max, sig_max;          /* admissible box */
  int32_t restart;                  /* nonzero (not in the paper): a direction with
                                       (g^m, d^m) >= 0 is replaced by -g^m */
} ddfd_cg_params;

/* One iteration's record. */
typedef struct {
  int32_t iter, stop;
  double J, J_data;                 /* functional with gamma^m, and its data part */
  double gnorm_eps, gnorm_sig;      /* ||g^m|| */
  double alpha_eps, alpha_sig, beta_eps, beta_sig, gamma_eps, gamma_sig;  /* used at m */
  double step_eps, step_sig;        /* ||eps^{m+1} - eps^m||, ||sig^{m+1} - sig^m|| */
  double ms;                        /* device time of the iteration (CUDA events) */
} ddfd_cg_iter;

/* Defaults: max_iter 20, gammas 1, alphas 1, p 0.5, tolerances 0, box 100, no restart. */
void ddfd_cg_params_default(ddfd_cg_params *prm);

/* Run the CGA on batch b.  eobs[i]: member i's observed trace (host, the
 * layout of ddfd_adjoint).  eps, sig (host, free-node order): the initial
 * guess on entry, the last iterate eps^{m+1} on return.  log (host, may be
 * NULL): room for max_iter records; *iters (may be NULL): iterations done;
 * eps_iters, sig_iters (host, may be NULL): [max_iter][n_free], iterate
 * m+1 after iteration m.  The box must lie inside every member's eps_max,
 * sig_max.  Errors: DDFD_E_ARG (members differ in fem_n or carry gammas, bad
 * parameters), DDFD_E_COEFF (initial guess outside the box), the errors of
 * the forward/adjoint calls; message in ddfd_batch_last_error.  When an
 * iteration m fails (e.g. DDFD_E_NONFINITE: the stabilized operator with a
 * rough iterate has growing modes), *iters = m, log[0..m) and eps_iters /
 * sig_iters rows [0..m) are filled, and eps, sig hold the iterate eps^m,
 * sig^m whose evaluation failed. */
int ddfd_cg_run(ddfd_batch *b, const double *const *eobs, const ddfd_cg_params *prm, double *eps,
                double *sig, ddfd_cg_iter *log, int32_t *iters, double *eps_iters, double *sig_iters);

/* Allocation-free data misfit, without a handle.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory (a strict device-memory budget, a host framework that owns
 * every allocation through its own arena, a real-time loop that cannot
 * afford cudaMalloc's latency and implicit synchronisation).  Such callers
 * cannot use ddfd_create, which allocates the field buffers.
 *
 * Writes to *J the data part of the functional that ddfd_functional
 * returns with both regularisation weights at zero: half the time step tau
 * times the sum, over sources s and steps n = 1..n_steps, of the taper
 * z(t_n) times the squared distance between trace and eobs at step n (all
 * detectors, all three components); t_n = n tau, and z is the taper of
 * ddfd_config.z_delta_frac with horizon T = n_steps tau.
 *   trace, eobs: device pointers, [n_src][n_steps + 1][n_det][3] doubles,
 *                owned by the caller (may be NULL when n_det = 0);
 *   J:           device pointer to one double, owned by the caller;
 *   stream:      cudaStream_t (NULL: default stream).  The call is
 *                asynchronous on `stream`: read *J after synchronising it.
 * Scratch: a fixed 512 KB array in the library's device image (one FP64
 * partial per (source, step) row); it requires 1 <= n_src * (n_steps + 1)
 * <= 65536, else DDFD_E_ARG with a message, and nothing is launched.  The
 * call allocates and frees nothing.  The array's device address is looked
 * up (cudaGetSymbolAddress) with the device current on the first call in
 * each device context -- the first call on a device, and again after that
 * device's context was reset; make that first call before any stream
 * capture.  Every call in the process shares the array and it keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong results.
 * Errors: DDFD_E_ARG, DDFD_E_CUDA; the message is ddfd_create_error(). */
int ddfd_misfit_noalloc(const double *trace, const double *eobs, int32_t n_src, int32_t n_steps,
                        int32_t n_det, double tau, double z_delta_frac, double *J, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DDFD_H */
