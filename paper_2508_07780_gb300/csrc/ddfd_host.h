// Host-side state and helpers of the ddfd library shared by its host
// translation units (ddfd_api.cu: single problems; ddfd_batch.cu: batches;
// ddfd_autotune.cu: the tile autotuner; ddfd_fem_setup.cu: explicit FEM
// meshes; ddfd_cg_host.cu: the conjugate gradient loop).  Not part of the
// public ABI.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ddfd_internal.h"

namespace ddfd {

// Message of the last failing handle-less call in this thread (read back by
// ddfd_create_error).
void set_thread_error(const std::string &msg);

namespace host {

constexpr int kMaxCapture = 16;
constexpr double kPi = 3.141592653589793;

// Call-order state of a handle.
enum { ST_READY = 0, ST_FORWARD = 1, ST_ADJOINT = 2 };

// The six descriptors of `problems` stacked problems: fields E[q], Mu[q]
// (3 channels each per problem) and the coefficients (s, q1, q2).
struct FieldMaps {
  CUtensorMap E_halo[2], E_ctr[2], M_halo[2], M_ctr[2], S, Q;
};

// Dispatch orders of a batch's step launches over one member list: per group
// of BATCH_MAX members, the device table and its count of leading items for
// the full FP32 step kernel.
struct ItemTables {
  std::vector<uint32_t *> d;
  std::vector<int> n_items, n_full;
};

// Creates (destroys) the side stream and the two events of a StepFork.
int make_fork(ddfd::StepFork *f);
void drop_fork(ddfd::StepFork *f);

}  // namespace host
}  // namespace ddfd

struct ddfd_problem {
  ddfd_config cfg{};
  std::vector<double> src_dir;
  std::vector<int32_t> det_ij;
  std::string err;
  int n = 0, fem_n = 0, a = 0, b = 0, f0 = 0, nf = 0, Nt = 0, n_src = 0, n_det = 0;
  int px = 0;                 // x pitch of the padded field layout
  long long n_free = 0, nn = 0, cs = 0;  // cs = px n^2, the component stride
  double h = 0, tau = 0;
  int fp32 = 0;
  size_t esz = 8;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  std::vector<size_t> alloc_bytes;  // size of each allocation, in the order of allocs
  int64_t bytes = 0;
  void *E[2] = {nullptr, nullptr}, *Mu[2] = {nullptr, nullptr};
  void *kcoef = nullptr;      // padded full-grid (s, q1, q2), 3 channels
  void *hist = nullptr;       // E on the free nodes: every step, or one replayed segment
  void *hist_fem = nullptr;   // literal gradient: E on the FEM-updated nodes, every step
  // checkpointing (n_snapshots > 0): state snapshots (E^n, E^{n-1}) at the
  // starts of segments of seg steps; the adjoint replays each segment
  int nsnap = 0, seg = 0;
  void *snap = nullptr;
  // element-by-element FEM rows (fem_kind = DDFD_FEM_EBE): explicit mesh
  int ebe_rows = 0;
  int *ebe_row_node = nullptr, *ebe_blk_nodes = nullptr, *ebe_blk_rows = nullptr;
  ddfd::EbeBlock *ebe_blocks = nullptr;
  unsigned char *ebe_blob = nullptr;
  int ebe_nblocks = 0, ebe_smem = 0;
  // algorithmic bytes of one step's element-apply launches (forward, adjoint):
  // each gathered tet's node ids and gradients, each of its nodes' values once,
  // each row's outputs; stencil rows their own node values and outputs
  int64_t ebe_bytes_fwd = 0, ebe_bytes_adj = 0;
  int test_fault = 0;          // ddfd_test_gather_timeout
  uint32_t test_spin = 0;
  int *kuhn_list = nullptr;   // explicit-mesh rows taken from the Kuhn block stencil
  int kuhn_n = 0;
  double kuhn_B[8][9] = {};   // (D^T D)_{i,i+o} / h of the uniform Kuhn split
  void *ebe_out_r = nullptr, *ebe_out_q = nullptr;
  double *ebe_scale = nullptr;
  double *trace = nullptr, *res = nullptr, *eobs_stage = nullptr, *gacc = nullptr;
  float *gpart = nullptr;     // FP32: per free node (g_eps, g_sig) sums of the current step block
  double *coef = nullptr, *coef_stage = nullptr, *z = nullptr, *part = nullptr, *scal = nullptr;
  double *gout = nullptr, *delay = nullptr, *pw[2] = {nullptr, nullptr};
  int *det_node = nullptr, *det_ptr = nullptr, *det_list = nullptr, *flag = nullptr;
  // FP32 adjoint sources per detector node (distinct top nodes with detectors):
  // slot of each top node (-1: none), CSR of its detectors into det_list, its
  // (i, j), and the scaled residual sums [n_src][Nt+1][n_unode][3]
  int *det_slot = nullptr, *uptr = nullptr, *uij = nullptr;
  int n_unode = 0;
  float *rsrc = nullptr;
  int *errflag = nullptr;     // kernel-side error bits (bounded waits)

  // TMA descriptors: [buffer] halo-box (current level) and centre-box (old level)
  CUtensorMap mE_halo[2], mE_ctr[2], mM_halo[2], mM_ctr[2], mS, mQ;
  std::vector<double> ptab;  // [n_src][Nt] pulse value P(t_n) (normal incidence), 0 after n1
  std::vector<int> n1, oblique;
  std::vector<double> pol;   // [n_src][3]
  std::vector<int> cap_steps;
  void *capE = nullptr, *capMu = nullptr;
  int state = ddfd::host::ST_READY;
  int64_t generation = 0;     // +1 whenever the coefficients or the forward state change
  int64_t launches = 0, fwd_steps = 0;
  int kz = 16;                // z depth of the full step kernel's items (and of the FP64 kernel's)
  int kz_lean = 16;           // z depth of the lean FP32 step kernel's items
  uint32_t *items = nullptr;  // dispatch order of the step launches (heaviest slabs first), for items_kz
  int items_kz = 0, n_items = 0;
  int items_nfull = 0;        // FP32: leading items for the full step kernel, the rest lean
  ddfd::StepFork fork;        // side stream of the lean step launches
  int n_part = 256;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double fwd_ms = 0.0, adj_ms = 0.0;
  int64_t fwd_kernels = 0, adj_kernels = 0;
  // The forward and adjoint sequences (all sources) are captured once into
  // CUDA graphs on cap_stream and replayed on the caller's stream.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gfwd = nullptr, gadj = nullptr;
  int64_t gfwd_launches = 0, gadj_launches = 0;
  // batch member: E, Mu and the coefficient field are slot `slot` of the
  // batch's stacked slabs (not owned); the batch destroys its members
  ddfd_batch *batch = nullptr;
  int slot = 0;
  bool fonly = false;         // forward_only: no history, no snapshots, no adjoint
  // explicit refined FEM mesh (fem_kind = DDFD_FEM_MESH): new nodes keep their
  // fields and (s, q1, q2) in arrays of their own, [3][n_new]
  int n_new = 0;
  long long n_free_grid = 0;  // free grid nodes; new node e is free node n_free_grid + e
  std::vector<int32_t> mesh_parents, mesh_tets;
  void *X[2] = {nullptr, nullptr}, *XMu[2] = {nullptr, nullptr}, *xcoef = nullptr;
  double *mass_free = nullptr;  // lumped mass of every free node (refined meshes)
};

struct ddfd_batch {
  std::vector<ddfd_problem *> m;
  std::string err;
  int n = 0, Nt = 0, px = 0, fp32 = 0, kz = 16, kz_lean = 16, seg = 0;
  long long cs = 0;
  size_t esz = 8;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  void *E[2] = {nullptr, nullptr}, *Mu[2] = {nullptr, nullptr}, *kcoef = nullptr;
  std::vector<void *> allocs;
  int64_t bytes = 0, launches = 0;
  ddfd::host::FieldMaps maps;
  int *errflag = nullptr;
  cudaGraphExec_t gfwd = nullptr, gadj = nullptr;
  int64_t gfwd_launches = 0, gadj_launches = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double fwd_ms = 0.0, adj_ms = 0.0;
  int64_t fwd_kernels = 0, adj_kernels = 0;
  // dispatch orders of the batched step launches (heaviest tiles first), for
  // items_kz: one table per group of BATCH_MAX members of all members, and of
  // the checkpointing members (their replays)
  ddfd::host::ItemTables items_all, items_ck;
  int items_kz = 0;
  ddfd::StepFork fork;        // side stream of the lean step launches
  // conjugate gradient work space (FP64, free nodes): 14 vectors, partial
  // sums, the 6 reduced scalars
  double *cg = nullptr;
  long long cg_n = 0;
};

namespace ddfd {
namespace host {

// Stacked field storage of a batch member: slot of E[0], E[1], Mu[0], Mu[1]
// and the coefficient field.
struct MemberSlot {
  void *E[2], *Mu[2], *kcoef;
  ddfd_batch *batch;
  int slot;
};

// Message of the last failing handle-less call in this thread.
const std::string &thread_error();

// Problem and batch error reporting: store the message, return the code.
int fail(ddfd_problem *p, int code, const std::string &m);
int bfail(ddfd_batch *b, int code, const std::string &m);

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(p, DDFD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(b, DDFD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

// Device allocation against the handle's budget (freed with the handle);
// dfree releases one such allocation early.
int dalloc(ddfd_problem *p, size_t bytes, void **out);
void dfree(ddfd_problem *p, void *ptr);

// Dispatch order of one step launch over the problems `ps` (stacked in that
// order), in z slabs (one problem's z range over a set of its tile columns,
// in grid order within the slab).  Full-kernel items first (their count in
// *n_full).  FP64: every column in z chunks of kz, the slabs sorted by an
// estimate of their work, heaviest first (node count, plus twice the FEM rows
// and once the free nodes they hold), ties in order of creation.  FP32: the
// columns that meet the FEM cube's interior or the free box, over the z range
// of those boxes, in chunks of kz; then the lean-kernel items in chunks of
// kz_lean from z = 0: every other column, and the FEM columns' planes outside
// their full range.  Both FP32 kernels take the problems in the same order
// (by their full-kernel work, heaviest first) and each problem's slabs in
// ascending z, so that they stay near each other in time and share halos.
std::vector<uint32_t> step_item_order(const std::vector<const ddfd_problem *> &ps, int kz, int kz_lean,
                                      int *n_full);
// (Re)builds p->items for p->kz and p->kz_lean.
int build_items(ddfd_problem *p);
// (Re)builds the batch's tables for b->kz.
int build_batch_items(ddfd_batch *b);
template <typename X>
int dalloc_t(ddfd_problem *p, size_t count, X **out) {
  void *v = nullptr;
  int st = dalloc(p, count * sizeof(X), &v);
  *out = (X *)v;
  return st;
}

// FP32: the adjoint's detector sources from p->res (after launch_residual);
// returns the number of kernels launched (0 or 1).
int enqueue_det_sources(ddfd_problem *p, cudaStream_t s);

// Absorbing faces of source s at step `step` (the top face only after its source phase).
uint32_t faces_at(const ddfd_problem *p, int s, long long step);
int validate(const ddfd_config *c, std::string *m);
int grad_mode(int k, int k_first);

// Single-problem operations (ddfd_api.cu).
int create_impl(const ddfd_config *cfg, const MemberSlot *ext, ddfd_problem **out);
void destroy_problem(ddfd_problem *p);
void drop_graphs(ddfd_problem *p);
int sync_check(ddfd_problem *p);
int check_err(ddfd_problem *p);
int set_coeffs_impl(ddfd_problem *p, const double *eps, const double *sig, const double *eps0,
                    const double *sig0, cudaMemcpyKind kind);
int functional_impl(ddfd_problem *p, const double *eobs, double *J, bool host);
int gradient_impl(ddfd_problem *p, double *g_eps, double *g_sig, bool host);
int encode_field_maps(std::string *err, FieldMaps *fm, void *const E[2], void *const Mu[2], void *coef, int n,
                      int px, int fp32, int problems);

// Explicit FEM meshes (ddfd_fem_setup.cu).
int build_ebe(ddfd_problem *p);
int build_mesh(ddfd_problem *p);

// Batches (ddfd_batch.cu).
std::vector<int> all_members(const ddfd_batch *b);
void drop_batch_graphs(ddfd_batch *b);
int batch_check_err(ddfd_batch *b);
int batch_forward_impl(ddfd_batch *b, double *const *trace_out, cudaMemcpyKind kind);
int batch_adjoint_impl(ddfd_batch *b, const double *const *eobs, bool host);

// Step-launch parameters and enqueueing, shared by the single-problem, batch
// and autotuner sequences.
template <typename T>
StepParams<T> base_params(const ddfd_problem *p) {
  StepParams<T> P;
  std::memset(&P, 0, sizeof(P));
  P.n = p->n;
  P.px = p->px;
  P.a = p->a;
  P.b = p->b;
  P.f0 = p->f0;
  P.nf = p->nf;
  P.kz = p->kz;
  P.cs = p->cs;
  P.err = p->errflag;
  P.ebe_r = (const T *)p->ebe_out_r;
  P.ebe_q = (const T *)p->ebe_out_q;
  P.ebe_rows = p->ebe_rows;

  P.spin_limit = 1u << 22;
  P.r2 = (T)((p->tau / p->h) * (p->tau / p->h));
  P.cb = (T)(p->tau / p->h);
  for (int f = 0; f < 4; ++f) P.inv_tab[f] = (T)(1.0 / (1.0 + f * (p->tau / p->h)));
  P.src_scale = 2.0 * p->tau * p->tau / p->h;
  P.pulse_kind = p->cfg.source_kind;
  P.freq = p->cfg.freq;
  P.t0 = p->cfg.t0;
  P.width = p->cfg.width;
  P.n_det = p->n_det;
  P.det_node = p->det_node;
  P.det_ptr = p->det_ptr;
  P.det_list = p->det_list;
  P.det_slot = p->det_slot;
  P.inv_h3 = 1.0 / (p->h * p->h * p->h);
  P.tau2 = p->tau * p->tau;
  P.n_free = p->n_free;
  P.gacc_e = p->gacc;
  P.gacc_s = p->gacc + p->n_free;
  P.gpart = p->gpart;
  return P;
}

template <typename T>
void set_source(StepParams<T> &P, const ddfd_problem *p, int s) {
  P.delay = p->delay ? p->delay + (size_t)s * p->n * p->n : nullptr;
  P.oblique = p->oblique[s];
  for (int q = 0; q < 3; ++q) P.pol[q] = p->pol[3 * s + q];
}

// Per-step scalars of forward step st (E^st -> E^{st+1}) of source s.
template <typename T>
void set_forward_step(StepParams<T> &P, const ddfd_problem *p, int s, int st, const void *cur, void *old,
                      T *hist_w) {
  P.cur = (const T *)cur;
  P.old = (T *)old;
  P.abs_now = faces_at(p, s, st);
  P.src_on = st <= p->n1[s] ? 1 : 0;
  P.t_n = st * p->tau;
  P.src_y = (T)(P.src_scale * p->ptab[(size_t)s * p->Nt + st]);
  P.trace_n = p->trace + ((size_t)s * (p->Nt + 1) + st) * p->n_det * 3;
  P.hist_w = hist_w;
}

// Per-step scalars of adjoint step k (mu^k -> mu^{k-1}) of source s.
template <typename T>
void set_adjoint_step(StepParams<T> &P, const ddfd_problem *p, int s, int k, const void *cur, void *old,
                      const T *hist_r, int k_first) {
  P.gmode = grad_mode(k, k_first);
  P.cur = (const T *)cur;
  P.old = (T *)old;
  P.abs_now = faces_at(p, s, k - 1);
  P.abs_next = faces_at(p, s, k + 1);
  P.res_k = p->res + ((size_t)s * (p->Nt + 1) + k) * p->n_det * 3;
  P.src_k = p->rsrc ? p->rsrc + ((size_t)s * (p->Nt + 1) + k) * p->n_unode * 3 : nullptr;
  P.hist_r = hist_r;
}

template <typename T>
StepLaunch<T, 1> single_launch(const StepParams<T> &P, const CUtensorMap &cur, const CUtensorMap &old,
                               const ddfd_problem *p) {
  StepLaunch<T, 1> L;
  L.cur = cur;
  L.old = old;
  L.s = p->mS;
  L.q = p->mQ;
  L.nprob = 1;
  L.zchunks = (p->n + P.kz - 1) / P.kz;
  L.items = P.kz == p->items_kz ? p->items : nullptr;
  L.n_items = p->n_items;
  L.n_full = p->items_nfull;
  L.p[0] = P;
  return L;
}

// The element-by-element rows of the current level (fem_kind = DDFD_FEM_EBE).
template <typename T>
void enqueue_ebe(ddfd_problem *p, const void *field, bool adj, cudaStream_t sm, int64_t *nk,
                 const void *xfield = nullptr, int *err = nullptr) {
  if (!p->ebe_rows) return;
  EbeParams<T> E;
  E.n_rows = p->ebe_rows;
  E.row_node = p->ebe_row_node;
  E.scale = p->ebe_scale;
  E.n_blocks = p->ebe_nblocks;
  E.blocks = p->ebe_blocks;
  E.blob = p->ebe_blob;
  E.blk_nodes = p->ebe_blk_nodes;
  E.blk_rows = p->ebe_blk_rows;
  E.stage_bytes = p->ebe_smem;
  E.err = err ? err : p->errflag;
  E.spin_limit = p->test_spin ? p->test_spin : 1u << 22;
  E.test_skip_copy = p->test_fault;
  if (p->kuhn_n) {
    KuhnRowParams<T> K;
    K.n_list = p->kuhn_n;
    K.list = p->kuhn_list;
    K.row_node = p->ebe_row_node;
    K.field = (const T *)field;
    K.s = (const T *)p->kcoef;
    K.cs = p->cs;
    K.px = p->px;
    K.n = p->n;
    K.out_r = (T *)p->ebe_out_r;
    K.out_q = (T *)p->ebe_out_q;
    K.n_rows = p->ebe_rows;
    for (int o = 0; o < 8; ++o)
      for (int e = 0; e < 9; ++e) K.B[o][e] = (T)p->kuhn_B[o][e];
    launch_kuhn_rows<T>(K, adj, sm);
    ++*nk;
  }
  E.field = (const T *)field;
  E.s = (const T *)p->kcoef;
  E.cs = p->cs;
  E.out_r = (T *)p->ebe_out_r;
  E.out_q = (T *)p->ebe_out_q;
  E.xfield = (const T *)xfield;
  E.xs = (const T *)p->xcoef;
  E.n_new = p->n_new;
  if (p->ebe_nblocks > 0) {
    launch_ebe<T>(E, adj, sm);
    ++*nk;
  }
}

// The new nodes of a refined mesh, one step (after the rows of enqueue_ebe).
template <typename T>
void enqueue_new_step(ddfd_problem *p, const void *cur, void *old, bool adj, const StepParams<T> &S,
                      cudaStream_t sm, int64_t *nk) {
  if (!p->n_new) return;
  NewStepParams<T> N;
  N.n_new = p->n_new;
  N.row0 = p->ebe_rows - p->n_new;
  N.ebe_rows = p->ebe_rows;
  N.ebe_r = (const T *)p->ebe_out_r;
  N.ebe_q = (const T *)p->ebe_out_q;
  N.cur = (const T *)cur;
  N.old = (T *)old;
  N.xcoef = (const T *)p->xcoef;
  N.r2 = S.r2;
  N.n_free = p->n_free;
  N.f0 = p->n_free_grid;
  N.hist_w = S.hist_w;
  N.hist_r = S.hist_r;
  N.gacc_e = S.gacc_e;
  N.gacc_s = S.gacc_s;
  N.gpart = S.gpart;
  N.gmode = S.gmode;
  launch_new_step<T>(N, adj, sm);
  ++*nk;
}

// One batched step launch per group of BATCH_MAX members; fill(P, p) sets the
// per-step scalars of member p; tables (may be NULL): the groups' dispatch
// orders, used when built for the batch's current kz.
template <typename T, typename Fill>
void launch_groups(ddfd_batch *b, bool adj, const std::vector<int> &idx, const CUtensorMap &cur,
                   const CUtensorMap &old, Fill fill, cudaStream_t sm, int64_t *nk,
                   const ItemTables *tables = nullptr) {
  for (size_t g0 = 0; g0 < idx.size(); g0 += BATCH_MAX) {
    StepLaunch<T, BATCH_MAX> L;
    std::memset(&L, 0, sizeof(L));
    L.cur = cur;
    L.old = old;
    L.s = b->maps.S;
    L.q = b->maps.Q;
    L.nprob = (int)std::min<size_t>(BATCH_MAX, idx.size() - g0);
    L.zchunks = (b->n + b->kz - 1) / b->kz;
    const size_t gi = g0 / BATCH_MAX;
    const bool tab = tables && b->kz == b->items_kz && gi < tables->d.size();
    L.items = tab ? tables->d[gi] : nullptr;
    L.n_items = tab ? tables->n_items[gi] : 0;
    L.n_full = tab ? tables->n_full[gi] : 0;
    for (int g = 0; g < L.nprob; ++g) {
      ddfd_problem *p = b->m[idx[g0 + g]];
      StepParams<T> P = base_params<T>(p);
      set_source(P, p, 0);
      P.kz = b->kz;
      P.chan = 3 * p->slot;
      P.err = b->errflag;
      fill(P, p);
      L.p[g] = P;
    }
    *nk += adj ? launch_adjoint_step(L, sm, &b->fork) : launch_forward_step(L, sm, &b->fork);
  }
}

}  // namespace host
}  // namespace ddfd
