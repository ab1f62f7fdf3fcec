// Internal declarations shared by the host driver and the kernels of the
// ddfd library (GB300 / sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ddfd.h"

namespace ddfd {

// Kuhn P1 div-div blocks for an interior node at h = 1:
// (D^T D)_{i,i+o} = h * B[o], B[-o] = B[o]; index 0 = offset 0, 1..7 = the
// offsets (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,0,1) (0,1,1) (1,1,1).
struct KuhnBlocks {
  double B[8][9];
  double mass;      // lumped mass of an interior node at h = 1 (must be 1)
  double lap[8];    // Laplacian row coefficients for the same offsets (7-point check)
};

// Builds the blocks by assembling the 24 Kuhn tetrahedra around a node;
// returns false (with a message) if the FE rows do not match the FD rows.
bool build_kuhn_blocks(KuhnBlocks *out, std::string *msg);

// Inverse of a 4x4 matrix (Gauss-Jordan, partial pivoting); false if singular.
bool invert4(const double A[4][4], double X[4][4]);

// Checks the assembled blocks against the table compiled into the step
// kernels (cudaErrorInvalidValue if they differ).
cudaError_t check_kuhn_blocks(const KuhnBlocks &kb, cudaStream_t s);

// Step-kernel tiling: a CTA of 256 computing threads owns a STEP_TX x TY
// (x, y) tile of one z chunk: FP64 one node per thread (TY = 8), FP32 two
// x-adjacent nodes per thread (TY = 16).
constexpr int STEP_TX = 32;
template <typename T>
struct StepTile {
  static constexpr int TY = 8;
};
template <>
struct StepTile<float> {
  static constexpr int TY = 16;
};

// FP32 gradient accumulation: the adjoint steps of each block of GRAD_BLOCK
// consecutive time steps are summed in FP32 (per free node) and the block sum
// is added to the FP64 accumulators; gmode tells a launch where it sits.
constexpr int GRAD_BLOCK = 16;
enum { GM_FIRST = 1, GM_FOLD = 2 };

// Geometry and per-step scalars common to the forward and adjoint steps.
// Fields are component-major with x pitch px: offset i + px (j + n k).
template <typename T>
struct StepParams {
  int n;                 // nodes per axis
  int px;                // x pitch of the padded layout (multiple of 8)
  int a, b;              // FEM box [a,b]
  int f0, nf;            // free box origin and side
  int kz;                // z planes per CTA
  long long cs;          // component stride (px n^2)
  const T *cur;          // E^n (forward) or mu^k (adjoint): detector gather only
  T *old;                // written: E^{n+1} (forward) or mu^{k-1} (adjoint)
  T r2;                  // (tau/h)^2
  T cb;                  // tau/h: damping of one absorbing face, divided form
  T inv_tab[4];          // 1 / (1 + f tau/h) for f = 0..3 absorbing faces at a node
  uint32_t abs_now;      // forward: absorbing faces at step n; adjoint: at step k-1
  uint32_t abs_next;     // adjoint: absorbing faces at step k+1
  // top-face source (forward only)
  int src_on;            // 1 while n <= n1
  int oblique;           // 0: normal incidence, value src_y on the y component
  T src_y;               // 2 tau^2 / h * P(t_n) (normal incidence)
  const double *delay;   // oblique: delay of each top node, n^2 (i + n j)
  double pol[3];         // oblique: polarisation
  double t_n;            // time of the step
  double src_scale;      // 2 tau^2 / h
  int pulse_kind;
  double freq, t0, width;
  // detectors
  int n_det;
  const int *det_node;   // forward gather: padded offset of each detector node
  double *trace_n;       // forward: trace[n] base ([n_det][3]), gathered from cur
  const int *det_ptr;    // adjoint: CSR over top-plane nodes (i + n j; n^2 + 1)
  const int *det_list;
  const double *res_k;   // adjoint: residual tau z (E^k - Eobs^k), [n_det][3]
  const int *det_slot;   // FP32 adjoint: detector-node index u of each top node (i + n j), or -1
  const float *src_k;    // FP32 adjoint: step k's detector sources, [u][3] (k_det_sources)
  double inv_h3;         // 1 / h^3
  double tau2;           // tau^2
  // history of E on the free nodes
  T *hist_w;             // forward: hist[n+1] ([3][n_free]); null: not kept
  const T *hist_r;       // adjoint: hist[k]
  long long n_free;
  double *gacc_e;        // adjoint: gradient accumulators (FP64)
  double *gacc_s;
  // element-by-element FEM rows (fem_kind = DDFD_FEM_EBE): when ebe_r is set,
  // nodes strictly inside the FEM cube take R = h^2 M^-1 (K E) (and, in the
  // adjoint, q = h^2 M^-1 (D^T D mu)) from these arrays, row index
  // (x-a-1) + (fem_n-2) ((y-a-1) + (fem_n-2) (k-a-1)), instead of the stencil
  const T *ebe_r;
  const T *ebe_q;
  int ebe_rows;
  int *err;              // bit 4: a bounded mbarrier wait gave up
  uint32_t spin_limit;   // polls per bounded wait
  int chan;              // first channel of this problem in the launch's tensor maps:
                         // fields at chan..chan+2, coefficients (s, q1, q2) likewise
  float *gpart;          // FP32 adjoint: (g_eps, g_sig) block sums per free node
  int gmode;             // FP32 adjoint: GM_FIRST (block starts: no partial to read),
                         // GM_FOLD (block ends: add to the FP64 accumulators)
};

// One step launch over NB_MAX problems at most, all with the same grid size
// and z chunking: the TMA descriptors span the stacked fields (channel axis
// 3 x problems) of the current level (halo box), the previous level (centre
// box), s (halo box, one channel) and (q1, q2) (centre box, two channels);
// CTA z index = z chunk + zchunks x problem.
constexpr int BATCH_MAX = 16;
template <typename T, int NB>
struct StepLaunch {
  CUtensorMap cur, old, s, q;
  int nprob;
  int zchunks;
  // optional dispatch order: block b of a 1-D grid of n_items blocks takes
  // the item items[b] (a tile, a z range and a problem, pack_step_item);
  // NULL: a 3-D grid of (tile x, tile y, z chunk + zchunks x problem), z
  // chunks of kz planes
  const uint32_t *items;
  int n_items;
  // FP32 with a dispatch order: items[0, n_full) hold FEM-cube or free nodes
  // and run on the full step kernel; the rest are finite-difference z ranges
  // only and run on the lean one (concurrently, on StepFork's side stream)
  int n_full;
  StepParams<T> p[NB];
};

// Side stream and fork/join events of a step whose FP32 tiles are split
// between the full and the lean kernel: the lean launch runs on `side`,
// ordered after the work queued before the step (ev_fork) and before the work
// queued after it (ev_join), so that both kernels of one step run side by side,
// also inside a captured graph.
struct StepFork {
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Tiles per axis of the step kernels' launch grid (FP32: 32 x 16 tiles,
// with n = 32 m + 1 covered by m x tiles; FP64: 32 x 8 tiles).
int step_tiles_x(int n, bool fp32);
int step_tiles_y(int n, bool fp32);
// One dispatch item: tile x (< 32), tile y (< 128), first plane z0 (< 1024),
// plane count nz (1..64), problem of the launch (< 16).
__host__ __device__ inline uint32_t pack_step_item(int tx, int ty, int z0, int nz, int prob) {
  return (uint32_t)tx | ((uint32_t)ty << 5) | ((uint32_t)z0 << 12) | ((uint32_t)(nz - 1) << 22) |
         ((uint32_t)prob << 28);
}
constexpr int ITEM_MAX_NZ = 64;

// Sets the dynamic shared-memory limit of every step-kernel instance (once,
// before any launch or capture).
cudaError_t prepare_step_kernels();

// One step: returns the number of kernels launched (1, or 2 when the FP32
// tiles are split; the lean launch goes to fk->side when fk has one, else to s).
template <typename T, int NB>
int launch_forward_step(const StepLaunch<T, NB> &L, cudaStream_t s, const StepFork *fk = nullptr);
template <typename T, int NB>
int launch_adjoint_step(const StepLaunch<T, NB> &L, cudaStream_t s, const StepFork *fk = nullptr);

// Element-by-element FEM apply over an explicit tetrahedral mesh, staged in
// shared memory block by block.  A block holds up to EBE_RB rows (nearby
// nodes), every tet incident to them and every node of those tets; one CTA
// copies the block's tets into shared memory, gathers its nodes' values, and
// then sums each row over its incident tets from shared memory only.
constexpr int EBE_RB = 128;                  // rows per block
constexpr int EBE_TPR = 8;                   // threads per row
constexpr int EBE_THREADS = EBE_TPR * EBE_RB;
constexpr int EBE_SMEM_BUDGET = 100 * 1024;  // per block (one of two pipeline stages)
constexpr uint16_t EBE_PAD = 0xFFFF;         // unused incidence slot

// The kernel is persistent (one CTA per SM) and double-buffered: while it
// sums one block, the next block's blob arrives by bulk copy and its nodes by
// per-thread asynchronous copies.
//
// One block.  Its blob (16-byte aligned, a multiple of 16 bytes) holds, for
// its nt tets (nt even; a padding tet has zero gradients), sqrt|K| times the
// P1 gradients [nt][4][3] (element type T), the tets' local node ids
// [nt][4] (uint16), and the rows' incidences [maxinc][EBE_RB] (uint16:
// local tet << 2 | the row's vertex in it, EBE_PAD where a row has fewer).
struct EbeBlock {
  long long blob;  // byte offset of the blob
  int bytes;       // blob size
  int nt;          // tets
  int nn;          // nodes (their padded offsets at nodes[node0 ..])
  int maxinc;      // incidences of the block's busiest row
  int nrows;       // rows (their indices at rows[row0 ..])
  int node0, row0;
};

// Host packer: rows in brick order of their positions, cut greedily into
// blocks under EBE_RB rows and EBE_SMEM_BUDGET bytes of shared memory.
// tnode: [ntet][4] padded node offsets; tgrad: [ntet][12] sqrt|K| g (FP64);
// rptr / itet / iloc: each row's incidences; rpos: [n_rows][3] node
// positions in units of h; esz: sizeof(T) of the kernel.
struct EbePack {
  std::vector<EbeBlock> blocks;
  std::vector<unsigned char> blob;
  std::vector<int> nodes, rows;
  int smem = 0;  // dynamic shared memory of the largest block
};
bool pack_ebe_blocks(long long n_rows, long long ntet, const int *tnode, const double *tgrad, const int *rptr,
                     const int *itet, const int *iloc, const double *rpos, int esz, EbePack *out, std::string *err,
                     const unsigned char *use = nullptr);
// use (may be NULL: every row): rows with use[r] = 0 are left out of the blocks.

// Marks the grid rows (the first n_grid_rows rows) whose incident tets are
// exactly the 24 tets of the uniform Kuhn split around the node: 24 incident
// tets, all four vertices grid nodes (ids below n^3, id = i + n (j + n k)), each
// a path o, o + e_p0, o + e_p0 + e_p1, o + (1,1,1).  Such a row equals the
// 15-point Kuhn block stencil row.
void kuhn_stencil_rows(long long n_grid_rows, int n, const int *rptr, const int *itet, const int *tet_ids,
                       std::vector<unsigned char> *is_stencil);

// Explicit-mesh rows that are Kuhn stencil rows: R (and, in the adjoint, q)
// from the 15-point block stencil instead of the element gather.
template <typename T>
struct KuhnRowParams {
  int n_list;
  const int *list;          // row indices
  const int *row_node;      // padded offset of each row's node
  const T *field;           // E^n or mu^k, padded, 3 components
  const T *s;               // eps - 1, padded
  long long cs;             // component stride
  int px, n;                // x pitch, nodes per axis
  T *out_r, *out_q;         // [3][n_rows]
  int n_rows;
  T B[8][9];                // (D^T D)_{i,i+o} / h, offsets 0, (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,0,1) (0,1,1) (1,1,1)
};
template <typename T>
void launch_kuhn_rows(const KuhnRowParams<T> &P, bool adj, cudaStream_t s);
// Shared-memory bytes of a block with nt tets, nn nodes, maxinc incidences.
long long ebe_block_smem(long long nt, long long nn, long long maxinc, int esz);

template <typename T>
struct EbeParams {
  int n_rows;               // FEM-updated nodes
  const int *row_node;      // padded offset of each row's node
  const double *scale;      // h^2 / m of each row (lumped P1 mass)
  int n_blocks;
  const EbeBlock *blocks;
  const unsigned char *blob;
  const int *blk_nodes;     // padded node offsets of the blocks' nodes
  const int *blk_rows;      // row indices of the blocks' rows
  int stage_bytes;          // shared memory of one pipeline stage (>= every block's)
  int *err;                 // bit 8: a bounded wait for a block's copy gave up
  uint32_t spin_limit;      // polls per bounded wait
  int test_skip_copy;       // failure-detection test: CTA 0 never starts its first block's copy
  const T *field;           // E^n (forward) or mu^k (adjoint), padded, 3 components
  const T *s;               // eps - 1, padded (coefficient channel 0)
  long long cs;             // component stride
  T *out_r;                 // [3][n_rows] h^2 M^-1 (K E) or (K^T mu)
  T *out_q;                 // [3][n_rows] adjoint: h^2 M^-1 (D^T D mu)
  // refined meshes: a node offset >= cs names new node (offset - cs), whose
  // field and s are xfield[c * n_new + e], xs[e]
  const T *xfield;
  const T *xs;
  int n_new;
};
// Sets the shared-memory limit of the gather kernels (once, before any launch).
cudaError_t prepare_ebe_kernels();

// Paper-literal gradient (grad_variant = DDFD_GRAD_LITERAL).  copy: E on the
// FEM-updated nodes (a, b)^3 into dst [3][(b-a-1)^3] (x fastest).  literal:
// adds, for every free node i, r2/6 sum_{K ni i} (div mu)_K ((div E)_K / 4 -
// grad phi_i . E_i) (Kuhn tets, divergences with unit gradients, r2 = tau^2/h^2)
// to the eps accumulator gacc[i]: the literal Gauss-law term replaces the exact
// one in the units the step kernels accumulate in.
template <typename T>
void launch_copy_fem_nodes(const T *E, T *dst, int n, int px, long long cs, int a, int b, cudaStream_t s);
template <typename T>
void launch_grad_literal(const T *Efem, const T *mu, double *gacc, int n, int px, long long cs, int a, int b,
                         double r2, cudaStream_t s);
template <typename T>
void launch_ebe(const EbeParams<T> &P, bool adj, cudaStream_t s);

// Update of the new nodes of a refined FEM mesh (their rows are FEM rows
// computed by k_ebe; interior nodes: no boundary or source terms), with the
// history writes (forward) or the gradient accumulation (adjoint) of the
// step kernels.
template <typename T>
struct NewStepParams {
  int n_new;
  int row0;              // row of new node 0 in ebe_r / ebe_q
  int ebe_rows;          // component stride of ebe_r / ebe_q
  const T *ebe_r, *ebe_q;
  const T *cur;          // [3][n_new] E^n (forward) or mu^k (adjoint)
  T *old;                // [3][n_new] in: E^{n-1} / mu^{k+1}, out: E^{n+1} / mu^{k-1}
  const T *xcoef;        // [3][n_new] (s, q1, q2)
  T r2;
  long long n_free;      // history / accumulator stride
  long long f0;          // free-node index of new node 0
  T *hist_w;
  const T *hist_r;
  double *gacc_e, *gacc_s;
  float *gpart;
  int gmode;
};
template <typename T>
void launch_new_step(const NewStepParams<T> &P, bool adj, cudaStream_t s);

// Small kernels.
void launch_gather_trace(const void *E, int fp32, long long cs, int n_det, const int *det_node,
                         double *trace_n, cudaStream_t s);
// (s, q1, q2) of the free nodes into the padded full-grid coefficient field;
// launch_coef_vacuum sets every node to the vacuum values (0, 1, 1) first.
void launch_expand_coeffs(int fp32, const double *coef_free, int nf, int f0, int n, int px,
                          long long cs, double tau, void *coef, cudaStream_t s, long long stride = -1);
// (s, q1, q2) of the new nodes of a refined mesh: free entries first .. first+n_new-1
// of the coefficient array (stride n_free between eps and sigma) into xcoef [3][n_new]
void launch_expand_new(int fp32, const double *coef_free, long long stride, long long first, int n_new,
                       double tau, void *xcoef, cudaStream_t s);
void launch_coef_vacuum(int fp32, long long cs, void *coef, cudaStream_t s);
// x[0, n) = v on the device (the default regularisation references).
void launch_fill(double *x, long long n, double v, cudaStream_t s);
void launch_check_coeffs(const double *coef_free, int n_free, double eps_max, double sig_max,
                         int *flag, cudaStream_t s);
// residual r = tau z (trace - eobs) for n >= 1 (r[0] = 0); partial sums of
// z |trace - eobs|^2 per block into part[] (deterministic two-pass sum).
// Adjoint sources of the FP32 step kernel, per detector node u (the distinct
// top nodes that carry detectors) and step: tau^2 / (h^3 m_u) times the sum of
// the residuals of u's detectors, summed in FP64 in detector order and rounded
// to FP32 (m_u: lumped mass of the top node, h^3 w_x w_y / 2).
// res: [n_src][n_steps+1][n_det][3]; out: [n_src][n_steps+1][n_unode][3];
// uptr/ulist: CSR of each node's detectors; uij: (i, j) of each node.
void launch_det_sources(const double *res, int n_steps, int n_det, int n_src, int n_unode, const int *uptr,
                        const int *ulist, const int *uij, int n, double tau2, double inv_h3, float *out,
                        cudaStream_t s);
void launch_residual(const double *trace, const double *eobs, const double *z, int n_steps,
                     int n_det, int n_src, double tau, double *res, double *part, int n_part,
                     cudaStream_t s);
void launch_regulariser(const double *coef_free, int n_free, double *part, int n_part,
                        cudaStream_t s, const double *mass = nullptr);
void launch_sum(const double *part, int n_part, double *out, cudaStream_t s);
void launch_grad_finalize(const double *coef_free, int n_free, const double *gacc_e,
                          const double *gacc_s, double ge_scale, double gs_scale, double m,
                          double gamma_e, double gamma_s, double *g_eps, double *g_sig,
                          cudaStream_t s, const double *mass = nullptr);
void launch_nonfinite(const double *x, long long count, int *flag, cudaStream_t s);
// power iteration helpers (FP64): y = M_eps^-1 K x, and the squared norm.
void launch_apply_op(const double *x, double *y, int n, int px, int a, int b, const void *coef_s, int fp32,
                     cudaStream_t s);
void launch_norm2(const double *x, long long count, double *part, int n_part, cudaStream_t s);
void launch_scale(double *x, long long count, const double *norm2, cudaStream_t s);

// Conjugate gradient vector kernels (csrc/ddfd_cg.cu), FP64 over the free
// nodes; part holds CG_BLOCKS x 6 partial sums, out the 4 or 6 sums.
constexpr int CG_BLOCKS = 256;
void launch_cg_accum(double *ge, double *gs, const double *te, const double *ts, long long n, cudaStream_t s);
void launch_cg_grad(const double *Ge, const double *Gs, const double *eps, const double *sig, const double *re,
                    const double *rs, double inv_m, double gam_e, double gam_s, double *gte, double *gts,
                    const double *dpe, const double *dps, int use_d, long long n, double *part, double *out,
                    cudaStream_t s, const double *mass = nullptr);
void launch_cg_update(const double *gte, const double *gts, double *de, double *ds, double beta_e, double beta_s,
                      double alpha_e, double alpha_s, const double *eps, const double *sig, double *eps_new,
                      double *sig_new, double eps_max, double sig_max, int first, long long n, double *part,
                      double *out, cudaStream_t s, const double *mass = nullptr);

}  // namespace ddfd
