// Host driver of the ddfd C ABI (include/ddfd.h): configuration checks, the
// call-order state machine, device memory, the incident-source setup and the
// enqueueing of the step kernels.  All arithmetic of the method runs in the
// kernels of ddfd_step.cu and ddfd_aux.cu; the host only prepares per-step
// scalars (pulse value, absorbing-face set) and small tables.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ddfd_internal.h"

using namespace ddfd;

namespace {
thread_local std::string g_create_err;
constexpr int kMaxCapture = 16;
constexpr double kPi = 3.141592653589793;

enum { ST_READY = 0, ST_FORWARD = 1, ST_ADJOINT = 2 };

double pulse_host(int kind, double f, double t0, double w, double t) {
  if (kind == DDFD_SRC_GAUSS) {
    const double s = t - t0, q = s / w;
    return std::sin(2.0 * kPi * f * s) * std::exp(-q * q);
  }
  return (t > 0.0 && t < 1.0 / f) ? std::sin(2.0 * kPi * f * t) : 0.0;
}
}  // namespace

namespace ddfd {
// Message of the last failing handle-less call in this thread.
void set_thread_error(const std::string &msg) { g_create_err = msg; }
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
  EbeBlock *ebe_blocks = nullptr;
  unsigned char *ebe_blob = nullptr;
  int ebe_nblocks = 0, ebe_smem = 0;
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
  int *errflag = nullptr;     // kernel-side error bits (bounded waits)

  // TMA descriptors: [buffer] halo-box (current level) and centre-box (old level)
  CUtensorMap mE_halo[2], mE_ctr[2], mM_halo[2], mM_ctr[2], mS, mQ;
  std::vector<double> ptab;  // [n_src][Nt] pulse value P(t_n) (normal incidence), 0 after n1
  std::vector<int> n1, oblique;
  std::vector<double> pol;   // [n_src][3]
  std::vector<int> cap_steps;
  void *capE = nullptr, *capMu = nullptr;
  int state = ST_READY;
  int64_t generation = 0;     // +1 whenever the coefficients or the forward state change
  int64_t launches = 0, fwd_steps = 0;
  int kz = 16;
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

namespace {

void destroy_problem(ddfd_problem *p);

int fail(ddfd_problem *p, int code, const std::string &m) {
  p->err = m;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(p, DDFD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

int dalloc(ddfd_problem *p, size_t bytes, void **out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  if (p->cfg.mem_budget > 0 && p->bytes + (int64_t)bytes > p->cfg.mem_budget)
    return fail(p, DDFD_E_OOM, "device memory budget exceeded (" + std::to_string(p->bytes + bytes) +
                                   " > " + std::to_string(p->cfg.mem_budget) + " bytes)");
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(p, DDFD_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  p->allocs.push_back(*out);
  p->bytes += (int64_t)bytes;
  return DDFD_OK;
}

template <typename X>
int dalloc_t(ddfd_problem *p, size_t count, X **out) {
  void *v = nullptr;
  int st = dalloc(p, count * sizeof(X), &v);
  *out = (X *)v;
  return st;
}

uint32_t faces_at(const ddfd_problem *p, int s, long long step) {
  uint32_t m = p->cfg.absorbing_faces & ~(uint32_t)DDFD_ABS_TOP;
  if ((p->cfg.absorbing_faces & DDFD_ABS_TOP) && step > p->n1[s]) m |= DDFD_ABS_TOP;
  return m;
}

int validate(const ddfd_config *c, std::string *m) {
  if (c->n < 7 || c->n > 1024) return *m = "n must be in [7, 1024]", DDFD_E_ARG;
  if (c->fem_n < 5 || c->fem_n > c->n - 2) return *m = "fem_n must be in [5, n-2]", DDFD_E_ARG;
  if (c->n_steps < 1) return *m = "n_steps must be >= 1", DDFD_E_ARG;
  if (!(c->cfl > 0.0) || !std::isfinite(c->cfl)) return *m = "cfl must be positive", DDFD_E_ARG;
  if (c->precision != DDFD_FP64 && c->precision != DDFD_FP32) return *m = "bad precision", DDFD_E_ARG;
  if (c->fem_kind != DDFD_FEM_STENCIL && c->fem_kind != DDFD_FEM_EBE && c->fem_kind != DDFD_FEM_MESH)
    return *m = "bad fem_kind", DDFD_E_ARG;
  if (c->grad_variant != DDFD_GRAD_EXACT && c->grad_variant != DDFD_GRAD_LITERAL)
    return *m = "bad grad_variant", DDFD_E_ARG;
  if (c->grad_variant == DDFD_GRAD_LITERAL &&
      (c->fem_kind != DDFD_FEM_STENCIL || c->n_snapshots > 0 || c->forward_only))
    return *m = "grad_variant DDFD_GRAD_LITERAL takes the stencil FEM, the full history and an adjoint", DDFD_E_ARG;
  if (c->fem_kind == DDFD_FEM_MESH) {
    if (c->mesh_n_new < 0 || c->mesh_n_tets < 1 || !c->mesh_tets || (c->mesh_n_new > 0 && !c->mesh_parents))
      return *m = "fem_kind DDFD_FEM_MESH needs mesh_tets (and mesh_parents for new nodes)", DDFD_E_ARG;
    if (c->n_snapshots > 0 || c->cfl_check)
      return *m = "refined meshes take neither n_snapshots nor cfl_check", DDFD_E_ARG;
    const long long n3 = (long long)c->n * c->n * c->n;
    for (int e = 0; e < c->mesh_n_new; ++e)
      for (int q = 0; q < 2; ++q) {
        const long long v = c->mesh_parents[2 * e + q];
        if (v < 0 || v >= n3 + e) return *m = "mesh_parents: a parent must be a grid node or an earlier new node", DDFD_E_ARG;
      }
    for (long long t = 0; t < 4 * c->mesh_n_tets; ++t)
      if (c->mesh_tets[t] < 0 || c->mesh_tets[t] >= n3 + c->mesh_n_new) return *m = "mesh_tets: node id out of range", DDFD_E_ARG;
  }
  if (c->n_src < 1) return *m = "n_src must be >= 1", DDFD_E_ARG;
  if (c->source_kind != DDFD_SRC_GAUSS && c->source_kind != DDFD_SRC_SINE) return *m = "bad source_kind", DDFD_E_ARG;
  if (!(c->freq > 0.0) || (c->source_kind == DDFD_SRC_GAUSS && !(c->width > 0.0)))
    return *m = "pulse frequency and width must be positive", DDFD_E_ARG;
  if (c->n_det < 0 || (c->n_det > 0 && !c->det_ij)) return *m = "bad detector list", DDFD_E_ARG;
  for (int d = 0; d < c->n_det; ++d) {
    const int i = c->det_ij[2 * d], j = c->det_ij[2 * d + 1];
    if (i < 0 || j < 0 || i >= c->n || j >= c->n) return *m = "detector off the top face", DDFD_E_ARG;
  }
  if (c->absorbing_faces > 63u) return *m = "bad absorbing_faces mask", DDFD_E_ARG;
  if (c->gamma_eps < 0 || c->gamma_sig < 0) return *m = "gammas must be >= 0", DDFD_E_ARG;
  if (!(c->z_delta_frac >= 0.0 && c->z_delta_frac < 1.0)) return *m = "z_delta_frac must be in [0,1)", DDFD_E_ARG;
  if (!(c->eps_max >= 1.0) || !(c->sig_max >= 0.0)) return *m = "bad coefficient bounds", DDFD_E_ARG;
  if (c->n_snapshots < 0 || c->n_snapshots > c->n_steps) return *m = "n_snapshots must be in [0, n_steps]", DDFD_E_ARG;
  if (c->mem_budget < 0) return *m = "mem_budget must be >= 0", DDFD_E_ARG;
  if (c->tile_kz != 0 && (c->tile_kz < 2 || c->tile_kz > c->n)) return *m = "tile_kz must be 0 or in [2, n]", DDFD_E_ARG;
  if (c->src_dir)
    for (int s = 0; s < c->n_src; ++s) {
      const double *k = c->src_dir + 3 * s;
      const double nrm = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
      if (!(nrm > 0.0) || !(k[2] / nrm < -1e-6)) return *m = "source directions need k_z < 0", DDFD_E_ARG;
    }
  return DDFD_OK;
}

// Incidence geometry of each source: polarisation, delays over the top face,
// switch step, pulse table.  A plane wave with direction k reaches top node x
// after k.(x - x_c) + Delta (x_c the face centre, Delta making the smallest
// delay zero); the flux is p P(t - delay), p = normalise(y - (y.k) k).
int setup_sources(ddfd_problem *p, std::vector<double> *delay_host) {
  const int n = p->n, Nt = p->Nt;
  const ddfd_config &c = p->cfg;
  p->n1.assign(p->n_src, 0);
  p->oblique.assign(p->n_src, 0);
  p->pol.assign(3 * p->n_src, 0.0);
  p->ptab.assign((size_t)p->n_src * Nt, 0.0);
  delay_host->assign((size_t)p->n_src * n * n, 0.0);
  for (int s = 0; s < p->n_src; ++s) {
    double k[3] = {0.0, 0.0, -1.0};
    if (!p->src_dir.empty()) {
      const double *d = p->src_dir.data() + 3 * s;
      const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int q = 0; q < 3; ++q) k[q] = d[q] / nrm;
    }
    double pv[3] = {-k[1] * k[0], 1.0 - k[1] * k[1], -k[1] * k[2]};
    double pn = std::sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
    if (pn < 1e-12) {
      pv[0] = 1.0 - k[0] * k[0];
      pv[1] = -k[0] * k[1];
      pv[2] = -k[0] * k[2];
      pn = std::sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
    }
    for (int q = 0; q < 3; ++q) p->pol[3 * s + q] = pv[q] / pn;
    double *dl = delay_host->data() + (size_t)s * n * n;
    double dmax = -1e300;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double proj = k[0] * (i * p->h - 0.5) + k[1] * (j * p->h - 0.5) + k[2] * 0.0;
        dl[i + n * j] = proj;
        dmax = std::max(dmax, -proj);
      }
    bool any = false;
    double dbig = 0.0;
    for (int q = 0; q < n * n; ++q) {
      dl[q] += dmax;
      if (dl[q] != 0.0) any = true;
      dbig = std::max(dbig, dl[q]);
    }
    const bool ypol = p->pol[3 * s] == 0.0 && p->pol[3 * s + 1] == 1.0 && p->pol[3 * s + 2] == 0.0;
    p->oblique[s] = (any || !ypol) ? 1 : 0;
    const double pend = c.source_kind == DDFD_SRC_GAUSS ? c.t0 + 3.0 * c.width : 1.0 / c.freq;
    const double t1 = c.t1 >= 0.0 ? c.t1 : pend + dbig;
    const double q = std::floor(t1 / p->tau + 1e-9);
    p->n1[s] = q > 2e9 ? 2000000000 : (int)q;
    for (int st = 0; st < Nt; ++st)
      p->ptab[(size_t)s * Nt + st] =
          st <= p->n1[s] ? pulse_host(c.source_kind, c.freq, c.t0, c.width, st * p->tau) : 0.0;
  }
  return DDFD_OK;
}

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
  P.inv_h3 = 1.0 / (p->h * p->h * p->h);
  P.tau2 = p->tau * p->tau;
  P.n_free = p->n_free;
  P.gacc_e = p->gacc;
  P.gacc_s = p->gacc + p->n_free;
  P.gpart = p->gpart;
  return P;
}

// Where adjoint step k sits in its block of GRAD_BLOCK steps (blocks end at
// k = 1, GRAD_BLOCK + 1, ...); k_first is the first step of the sequence.
int grad_mode(int k, int k_first) {
  const int phase = (k - 1) % GRAD_BLOCK;
  return ((k == k_first || phase == GRAD_BLOCK - 1) ? GM_FIRST : 0) | (phase == 0 ? GM_FOLD : 0);
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
  L.p[0] = P;
  return L;
}

int capture_slot(const ddfd_problem *p, int step) {
  for (size_t q = 0; q < p->cap_steps.size(); ++q)
    if (p->cap_steps[q] == step) return (int)q;
  return -1;
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

// Enqueue the whole forward sequence (every source) on stream `st`; returns
// the number of kernels enqueued in *nk.
template <typename T>
int enqueue_forward(ddfd_problem *p, cudaStream_t sm, int64_t *nk) {
  const size_t fbytes = 3 * (size_t)p->cs * sizeof(T);
  const int Nt = p->Nt;
  *nk = 0;
  for (int s = 0; s < p->n_src; ++s) {
    CK(cudaMemsetAsync(p->E[0], 0, fbytes, sm));
    CK(cudaMemsetAsync(p->E[1], 0, fbytes, sm));
    if (p->n_new) {
      CK(cudaMemsetAsync(p->X[0], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
      CK(cudaMemsetAsync(p->X[1], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
    }
    if (s == 0) {
      const int sl = capture_slot(p, 0);
      if (sl >= 0) CK(cudaMemsetAsync((char *)p->capE + sl * fbytes, 0, fbytes, sm));
    }
    int ic = 1, io = 0;  // buffer holding E^n, and E^{n-1}
    StepParams<T> P = base_params<T>(p);
    set_source(P, p, s);
    for (int st = 0; st < Nt; ++st) {
      if (p->nsnap && st % p->seg == 0) {  // snapshot the state (E^st, E^{st-1})
        char *sn = (char *)p->snap + ((size_t)s * p->nsnap + st / p->seg) * 2 * fbytes;
        CK(cudaMemcpyAsync(sn, p->E[ic], fbytes, cudaMemcpyDeviceToDevice, sm));
        CK(cudaMemcpyAsync(sn + fbytes, p->E[io], fbytes, cudaMemcpyDeviceToDevice, sm));
      }
      set_forward_step(P, p, s, st, p->E[ic], p->E[io],
                       (p->nsnap || p->fonly) ? nullptr
                                              : (T *)p->hist + ((size_t)s * (Nt + 1) + st + 1) * 3 * p->n_free);
      enqueue_ebe<T>(p, p->E[ic], false, sm, nk, p->X[ic]);
      launch_forward_step(single_launch(P, p->mE_halo[ic], p->mE_ctr[io], p), sm);
      enqueue_new_step<T>(p, p->X[ic], p->X[io], false, P, sm, nk);
      ++*nk;
      std::swap(ic, io);
      if (p->hist_fem) {  // E^{st+1} on the FEM-updated nodes, for the literal gradient
        const size_t nfu = (size_t)(p->b - p->a - 1) * (p->b - p->a - 1) * (p->b - p->a - 1);
        launch_copy_fem_nodes<T>((const T *)p->E[ic], (T *)p->hist_fem + ((size_t)s * (Nt + 1) + st + 1) * 3 * nfu,
                                 p->n, p->px, p->cs, p->a, p->b, sm);
        ++*nk;
      }
      if (s == 0) {
        const int sl = capture_slot(p, st + 1);
        if (sl >= 0)
          CK(cudaMemcpyAsync((char *)p->capE + sl * fbytes, p->E[ic], fbytes, cudaMemcpyDeviceToDevice, sm));
      }
    }
    CK(cudaGetLastError());
    launch_gather_trace(p->E[ic], p->fp32, p->cs, p->n_det, p->det_node,
                        p->trace + ((size_t)s * (Nt + 1) + Nt) * p->n_det * 3, sm);
    if (p->n_det > 0) ++*nk;
  }
  CK(cudaGetLastError());
  return DDFD_OK;
}

template <typename T>
int enqueue_adjoint(ddfd_problem *p, cudaStream_t sm, int64_t *nk) {
  const size_t fbytes = 3 * (size_t)p->cs * sizeof(T);
  const int Nt = p->Nt;
  *nk = 0;
  CK(cudaMemsetAsync(p->gacc, 0, 2 * (size_t)p->n_free * sizeof(double), sm));
  for (int s = 0; s < p->n_src; ++s) {
    CK(cudaMemsetAsync(p->Mu[0], 0, fbytes, sm));
    CK(cudaMemsetAsync(p->Mu[1], 0, fbytes, sm));
    if (p->n_new) {
      CK(cudaMemsetAsync(p->XMu[0], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
      CK(cudaMemsetAsync(p->XMu[1], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
    }
    int ic = 1, io = 0;  // buffers holding mu^k and mu^{k+1}
    StepParams<T> P = base_params<T>(p);
    // segments [n0, n1): all of [0, Nt) at once when the whole history is
    // kept, else the checkpoint segments from the last to the first
    const int nseg = p->nsnap ? (Nt + p->seg - 1) / p->seg : 1;
    for (int j = nseg - 1; j >= 0; --j) {
      const int n0 = p->nsnap ? j * p->seg : 0;
      const int n1 = p->nsnap ? std::min(n0 + p->seg, Nt) : Nt;
      const T *hbase;  // E^k of this segment at hbase + (k - n0) * 3 n_free
      if (p->nsnap) {
        // restore the snapshot of step n0 and replay the segment's forward
        // steps, keeping E on the free nodes for the adjoint steps below
        const char *sn = (const char *)p->snap + ((size_t)s * p->nsnap + j) * 2 * fbytes;
        CK(cudaMemcpyAsync(p->E[1], sn, fbytes, cudaMemcpyDeviceToDevice, sm));
        CK(cudaMemcpyAsync(p->E[0], sn + fbytes, fbytes, cudaMemcpyDeviceToDevice, sm));
        int fc = 1, fo = 0;
        StepParams<T> F = base_params<T>(p);
        set_source(F, p, s);
        for (int st = n0; st < n1; ++st) {
          // (the trace is written again with the same values)
          set_forward_step(F, p, s, st, p->E[fc], p->E[fo], (T *)p->hist + (size_t)(st + 1 - n0) * 3 * p->n_free);
          enqueue_ebe<T>(p, p->E[fc], false, sm, nk);
          launch_forward_step(single_launch(F, p->mE_halo[fc], p->mE_ctr[fo], p), sm);
          ++*nk;
          std::swap(fc, fo);
        }
        hbase = (const T *)p->hist;
      } else {
        hbase = (const T *)p->hist + (size_t)s * (Nt + 1) * 3 * p->n_free;
      }
      for (int k = n1; k >= n0 + 1; --k) {
        set_adjoint_step(P, p, s, k, p->Mu[ic], p->Mu[io], hbase + (size_t)(k - n0) * 3 * p->n_free, Nt);
        enqueue_ebe<T>(p, p->Mu[ic], true, sm, nk, p->XMu[ic]);
        launch_adjoint_step(single_launch(P, p->mM_halo[ic], p->mM_ctr[io], p), sm);
        enqueue_new_step<T>(p, p->XMu[ic], p->XMu[io], true, P, sm, nk);
        ++*nk;
        if (p->hist_fem) {  // literal gradient: swap the Gauss-law term of step k (mu^k is still in Mu[ic])
          const size_t nfu = (size_t)(p->b - p->a - 1) * (p->b - p->a - 1) * (p->b - p->a - 1);
          launch_grad_literal<T>((const T *)p->hist_fem + ((size_t)s * (Nt + 1) + k) * 3 * nfu, (const T *)p->Mu[ic],
                                 p->gacc, p->n, p->px, p->cs, p->a, p->b, p->tau * p->tau / (p->h * p->h), sm);
          ++*nk;
        }
        std::swap(ic, io);
        if (s == 0) {
          const int sl = capture_slot(p, k - 1);
          if (sl >= 0)
            CK(cudaMemcpyAsync((char *)p->capMu + sl * fbytes, p->Mu[ic], fbytes, cudaMemcpyDeviceToDevice, sm));
        }
      }
    }
    CK(cudaGetLastError());
  }
  return DDFD_OK;
}

void drop_graphs(ddfd_problem *p) {
  if (p->gfwd) cudaGraphExecDestroy(p->gfwd);
  if (p->gadj) cudaGraphExecDestroy(p->gadj);
  p->gfwd = p->gadj = nullptr;
}

// Capture `adj ? adjoint : forward` into a graph (once), replay it on the
// caller's stream between two timing events.
int run_sequence(ddfd_problem *p, bool adj) {
  cudaGraphExec_t *ge = adj ? &p->gadj : &p->gfwd;
  int64_t *gl = adj ? &p->gadj_launches : &p->gfwd_launches;
  if (!*ge) {
    CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    int64_t nk = 0;
    int st;
    if (adj)
      st = p->fp32 ? enqueue_adjoint<float>(p, p->cap_stream, &nk) : enqueue_adjoint<double>(p, p->cap_stream, &nk);
    else
      st = p->fp32 ? enqueue_forward<float>(p, p->cap_stream, &nk) : enqueue_forward<double>(p, p->cap_stream, &nk);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    CK(ec);
    const cudaError_t ei = cudaGraphInstantiate(ge, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    *gl = nk;
  }
  cudaEvent_t e0 = p->ev[adj ? 2 : 0], e1 = p->ev[adj ? 3 : 1];
  CK(cudaEventRecord(e0, p->stream));
  CK(cudaGraphLaunch(*ge, p->stream));
  CK(cudaEventRecord(e1, p->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  p->launches += *gl;
  if (adj) {
    p->adj_ms = ms;
    p->adj_kernels = (int64_t)p->Nt * p->n_src * (p->nsnap ? 2 : 1);
    if (p->nsnap) p->fwd_steps += (int64_t)p->Nt * p->n_src;  // replayed forward steps
  } else {
    p->fwd_ms = ms;
    p->fwd_kernels = (int64_t)p->Nt * p->n_src;
    p->fwd_steps += (int64_t)p->Nt * p->n_src;
  }
  return DDFD_OK;
}

int sync_check(ddfd_problem *p) {
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return DDFD_OK;
}

int read_flag(ddfd_problem *p, int *out) {
  CK(cudaMemcpyAsync(out, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return DDFD_OK;
}

// Power iteration for lambda_max of M_eps^-1 K (units 1/h^2 folded in).
int cfl_check(ddfd_problem *p) {
  const long long cnt = 3 * p->nn;
  for (int q = 0; q < 2; ++q)
    if (!p->pw[q]) {
      int st = dalloc_t(p, (size_t)cnt, &p->pw[q]);
      if (st) return st;
    }
  std::vector<double> x0((size_t)cnt);
  uint64_t r = 0x9E3779B97F4A7C15ull;
  for (long long q = 0; q < cnt; ++q) {
    r ^= r << 13;
    r ^= r >> 7;
    r ^= r << 17;
    x0[q] = (double)(r >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  CK(cudaMemcpyAsync(p->pw[0], x0.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  launch_norm2(p->pw[0], cnt, p->part, p->n_part, p->stream);
  launch_sum(p->part, p->n_part, p->scal, p->stream);
  launch_scale(p->pw[0], cnt, p->scal, p->stream);
  p->launches += 3;
  const int iters = 120;
  for (int it = 0; it < iters; ++it) {
    launch_apply_op(p->pw[0], p->pw[1], p->n, p->px, p->a, p->b, p->kcoef, p->fp32, p->stream);
    launch_norm2(p->pw[1], cnt, p->part, p->n_part, p->stream);
    launch_sum(p->part, p->n_part, p->scal, p->stream);
    launch_scale(p->pw[1], cnt, p->scal, p->stream);
    p->launches += 4;
    std::swap(p->pw[0], p->pw[1]);
  }
  double nrm2 = 0.0;
  CK(cudaMemcpyAsync(&nrm2, p->scal, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const double lam = std::sqrt(nrm2) / (p->h * p->h);
  if (!(p->tau * p->tau * lam < 4.0 * 0.98))
    return fail(p, DDFD_E_CFL, "tau = " + std::to_string(p->tau) + " exceeds the stability bound 2/sqrt(" +
                                   std::to_string(lam) + ")");
  return DDFD_OK;
}

// TMA descriptors of one padded field: a 4-D tensor (x, y, z, channel) with
// row stride px, plane stride px n, channel stride px n^2; the halo box is
// (32 + 2 hx) x (TY + 2) x 1 x ch starting hx elements (16 bytes) left of
// the tile, the centre box 32 x TY x 1 x ch.  Out-of-range elements read as
// zero.
int encode_map(std::string *err, CUtensorMap *m, void *base, int n, int px, int fp32, int channels,
               int box_channels, bool halo) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return *err = "cuTensorMapEncodeTiled is not available from the driver", DDFD_E_CUDA;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t esz = fp32 ? 4 : 8;
  const cuuint64_t cs = (cuuint64_t)px * n * n;
  const cuuint64_t dims[4] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)channels};
  const cuuint64_t strides[3] = {(cuuint64_t)px * esz, (cuuint64_t)px * n * esz, cs * esz};
  const cuuint32_t hx = (cuuint32_t)(16 / esz);
  const cuuint32_t ty = fp32 ? StepTile<float>::TY : StepTile<double>::TY;
  const cuuint32_t box[4] = {halo ? (cuuint32_t)STEP_TX + 2 * hx : (cuuint32_t)STEP_TX, halo ? ty + 2 : ty, 1,
                             (cuuint32_t)box_channels};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                            base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return *err = "cuTensorMapEncodeTiled failed: " + std::to_string((int)r), DDFD_E_CUDA;
  return DDFD_OK;
}

// The six descriptors of `problems` stacked problems: fields E[q], Mu[q]
// (3 channels each per problem) and the coefficients (s, q1, q2).
struct FieldMaps {
  CUtensorMap E_halo[2], E_ctr[2], M_halo[2], M_ctr[2], S, Q;
};
int encode_field_maps(std::string *err, FieldMaps *fm, void *const E[2], void *const Mu[2], void *coef, int n,
                      int px, int fp32, int problems) {
  const int ch = 3 * problems;
  int st;
  for (int q = 0; q < 2; ++q)
    if ((st = encode_map(err, &fm->E_halo[q], E[q], n, px, fp32, ch, 3, true)) ||
        (st = encode_map(err, &fm->E_ctr[q], E[q], n, px, fp32, ch, 3, false)) ||
        (Mu[q] && (st = encode_map(err, &fm->M_halo[q], Mu[q], n, px, fp32, ch, 3, true))) ||
        (Mu[q] && (st = encode_map(err, &fm->M_ctr[q], Mu[q], n, px, fp32, ch, 3, false))))
      return st;
  if ((st = encode_map(err, &fm->S, coef, n, px, fp32, ch, 1, true))) return st;
  return encode_map(err, &fm->Q, coef, n, px, fp32, ch, 2, false);
}

// Explicit P1 mesh of the FEM cube for the element-by-element path: the six
// Kuhn tetrahedra of every cube of [a, b]^3 as a tet list with per-tet
// sqrt|K| g (from the inverse of [1 x] in FP64), the incidences of the nodes
// strictly inside the cube (the rows the FEM updates) and their lumped masses.
// Packs the element-by-element rows into shared-memory blocks and uploads
// them with the rows' node offsets and mass scales (both mesh kinds).
int upload_ebe(ddfd_problem *p, long long rows, long long ntet, const std::vector<int> &tnode,
               const std::vector<double> &tgrad, const std::vector<int> &rptr, const std::vector<int> &itet,
               const std::vector<int> &iloc, const std::vector<int> &rnode, const std::vector<double> &scale,
               const std::vector<double> &rpos, const std::vector<unsigned char> *stencil = nullptr) {
  // rows marked in *stencil take the Kuhn block stencil; the others are gathered
  std::vector<unsigned char> use;
  std::vector<int> klist;
  if (stencil) {
    use.assign((size_t)rows, 1);
    for (size_t r = 0; r < stencil->size(); ++r)
      if ((*stencil)[r]) {
        use[r] = 0;
        klist.push_back((int)r);
      }
  }
  EbePack pk;
  std::string m;
  if (!pack_ebe_blocks(rows, ntet, tnode.data(), tgrad.data(), rptr.data(), itet.data(), iloc.data(), rpos.data(),
                       (int)p->esz, &pk, &m, stencil ? use.data() : nullptr))
    return fail(p, DDFD_E_ARG, m);
  if (!klist.empty()) {
    int st;
    if ((st = dalloc_t(p, klist.size(), &p->kuhn_list))) return st;
    CK(cudaMemcpy(p->kuhn_list, klist.data(), klist.size() * sizeof(int), cudaMemcpyHostToDevice));
    p->kuhn_n = (int)klist.size();
  }
  int st;
  const size_t es = p->esz;
  if ((st = dalloc_t(p, (size_t)rows, &p->ebe_row_node)) || (st = dalloc_t(p, (size_t)rows, &p->ebe_scale)) ||
      (st = dalloc_t(p, pk.blocks.size(), &p->ebe_blocks)) || (st = dalloc_t(p, pk.blob.size(), &p->ebe_blob)) ||
      (st = dalloc_t(p, pk.nodes.size(), &p->ebe_blk_nodes)) || (st = dalloc_t(p, pk.rows.size(), &p->ebe_blk_rows)) ||
      (st = dalloc(p, 3 * (size_t)rows * es, &p->ebe_out_r)) || (st = dalloc(p, 3 * (size_t)rows * es, &p->ebe_out_q)))
    return st;
  CK(cudaMemcpy(p->ebe_row_node, rnode.data(), rows * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_scale, scale.data(), rows * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blocks, pk.blocks.data(), pk.blocks.size() * sizeof(EbeBlock), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blob, pk.blob.data(), pk.blob.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blk_nodes, pk.nodes.data(), pk.nodes.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blk_rows, pk.rows.data(), pk.rows.size() * sizeof(int), cudaMemcpyHostToDevice));
  p->ebe_nblocks = (int)pk.blocks.size();
  p->ebe_smem = (pk.smem + 127) & ~127;  // one pipeline stage
  p->ebe_rows = (int)rows;
  return DDFD_OK;
}

int build_ebe(ddfd_problem *p) {
  const int a = p->a, b = p->b, n = p->n;
  const int fm = b - a - 1;  // rows per axis
  const long long rows = (long long)fm * fm * fm;
  const long long cubes = (long long)(b - a) * (b - a) * (b - a);
  const long long ntet = 6 * cubes;
  if (ntet > (1LL << 31) / 4) return fail(p, DDFD_E_ARG, "FEM mesh too large for the element path");
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  std::vector<int> tnode((size_t)ntet * 4);
  std::vector<double> tgrad((size_t)ntet * 12);
  std::vector<int> rptr((size_t)rows + 1, 0);
  std::vector<double> mass((size_t)rows, 0.0);
  auto off = [&](int i, int j, int k) { return (int)(i + (long long)p->px * (j + (long long)n * k)); };
  auto rowof = [&](int i, int j, int k) -> long long {
    if (i <= a || i >= b || j <= a || j >= b || k <= a || k >= b) return -1;
    return (i - a - 1) + (long long)fm * ((j - a - 1) + (long long)fm * (k - a - 1));
  };
  long long t = 0;
  for (int k = a; k < b; ++k)
    for (int j = a; j < b; ++j)
      for (int i = a; i < b; ++i)
        for (const auto &pm : perms) {
          int v[4][3] = {{i, j, k}};
          for (int q = 0; q < 3; ++q) {
            for (int d = 0; d < 3; ++d) v[q + 1][d] = v[q][d];
            v[q + 1][pm[q]] += 1;
          }
          double A[4][4], C[4][4];
          for (int q = 0; q < 4; ++q) {
            A[q][0] = 1.0;
            for (int d = 0; d < 3; ++d) A[q][d + 1] = v[q][d] * p->h;
          }
          if (!invert4(A, C)) return fail(p, DDFD_E_ARG, "degenerate tetrahedron in the FEM mesh");
          double e1[3], e2[3], e3[3];
          for (int d = 0; d < 3; ++d) {
            e1[d] = A[1][d + 1] - A[0][d + 1];
            e2[d] = A[2][d + 1] - A[0][d + 1];
            e3[d] = A[3][d + 1] - A[0][d + 1];
          }
          const double vol = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                                       e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
          const double sv = std::sqrt(vol);
          for (int q = 0; q < 4; ++q) {
            tnode[t * 4 + q] = off(v[q][0], v[q][1], v[q][2]);
            for (int d = 0; d < 3; ++d) tgrad[t * 12 + q * 3 + d] = sv * C[d + 1][q];
            const long long r = rowof(v[q][0], v[q][1], v[q][2]);
            if (r >= 0) {
              rptr[r + 1]++;
              mass[r] += vol / 4.0;
            }
          }
          ++t;
        }
  for (long long r = 0; r < rows; ++r) rptr[r + 1] += rptr[r];
  const long long ninc = rptr[rows];
  std::vector<int> itet((size_t)ninc), iloc((size_t)ninc), fillp(rptr.begin(), rptr.end() - 1), rnode((size_t)rows);
  std::vector<double> scale((size_t)rows);
  for (t = 0; t < ntet; ++t)
    for (int q = 0; q < 4; ++q) {
      const int o = tnode[t * 4 + q];
      const int i = (int)(o % p->px), j = (int)((o / p->px) % n), k = (int)(o / ((long long)p->px * n));
      const long long r = rowof(i, j, k);
      if (r >= 0) {
        itet[fillp[r]] = (int)t;
        iloc[fillp[r]++] = q;
      }
    }
  for (int k = a + 1; k < b; ++k)
    for (int j = a + 1; j < b; ++j)
      for (int i = a + 1; i < b; ++i) {
        const long long r = rowof(i, j, k);
        rnode[r] = off(i, j, k);
        scale[r] = p->h * p->h / mass[r];
      }
  std::vector<double> rpos((size_t)rows * 3);
  for (int k = a + 1; k < b; ++k)
    for (int j = a + 1; j < b; ++j)
      for (int i = a + 1; i < b; ++i) {
        const long long r = rowof(i, j, k);
        rpos[3 * r] = i;
        rpos[3 * r + 1] = j;
        rpos[3 * r + 2] = k;
      }
  return upload_ebe(p, rows, ntet, tnode, tgrad, rptr, itet, iloc, rnode, scale, rpos);
}

// Explicit refined FEM mesh (fem_kind = DDFD_FEM_MESH): node coordinates
// (new nodes as midpoints of their parents, in FP64), per-tet sqrt|K| g,
// the incidences of the FEM rows -- the grid nodes strictly inside the cube in
// the order of build_ebe, then the new nodes -- with their lumped masses, the
// masses of every free node, and the new nodes' field and coefficient arrays.
int build_mesh(ddfd_problem *p) {
  const int a = p->a, b = p->b, n = p->n;
  const long long n3 = (long long)n * n * n;
  const int fm = b - a - 1;
  const long long grid_rows = (long long)fm * fm * fm;
  const long long rows = grid_rows + p->n_new;
  const long long ntet = (long long)p->mesh_tets.size() / 4;
  if (p->cs + (long long)p->n_new >= (1LL << 31) || 4 * ntet >= (1LL << 31))
    return fail(p, DDFD_E_ARG, "refined mesh too large for 32-bit node offsets");
  std::vector<double> X((size_t)p->n_new * 3);
  auto xyz = [&](long long v, double out[3]) {
    if (v < n3) {
      out[0] = (double)(v % n) * p->h;
      out[1] = (double)((v / n) % n) * p->h;
      out[2] = (double)(v / ((long long)n * n)) * p->h;
    } else {
      for (int d = 0; d < 3; ++d) out[d] = X[(size_t)(v - n3) * 3 + d];
    }
  };
  const double lo = (p->f0 - 1e-9) * p->h, hi = (p->f0 + p->nf - 1 + 1e-9) * p->h;
  for (int e = 0; e < p->n_new; ++e) {
    double u[3], w[3];
    xyz(p->mesh_parents[2 * e], u);
    xyz(p->mesh_parents[2 * e + 1], w);
    for (int d = 0; d < 3; ++d) {
      X[(size_t)e * 3 + d] = 0.5 * (u[d] + w[d]);
      if (!(X[(size_t)e * 3 + d] >= lo && X[(size_t)e * 3 + d] <= hi))
        return fail(p, DDFD_E_ARG, "mesh: new node " + std::to_string(e) + " outside the free box");
    }
  }
  auto in_cube = [&](long long v) {
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    return i >= a && i <= b && j >= a && j <= b && k >= a && k <= b;
  };
  auto rowof = [&](long long v) -> long long {
    if (v >= n3) return grid_rows + (v - n3);
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    if (i <= a || i >= b || j <= a || j >= b || k <= a || k >= b) return -1;
    return (i - a - 1) + (long long)fm * ((j - a - 1) + (long long)fm * (k - a - 1));
  };
  auto off = [&](long long v) -> int {
    if (v >= n3) return (int)(p->cs + (v - n3));
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    return (int)(i + (long long)p->px * (j + (long long)n * k));
  };
  std::vector<int> tnode((size_t)ntet * 4), rptr((size_t)rows + 1, 0);
  std::vector<double> tgrad((size_t)ntet * 12), mass((size_t)rows, 0.0);
  double vol_sum = 0.0;
  for (long long t = 0; t < ntet; ++t) {
    double A[4][4], C[4][4];
    for (int q = 0; q < 4; ++q) {
      const long long v = p->mesh_tets[t * 4 + q];
      if (v < n3 && !in_cube(v)) return fail(p, DDFD_E_ARG, "mesh: a grid node outside the FEM cube");
      double x[3];
      xyz(v, x);
      A[q][0] = 1.0;
      for (int d = 0; d < 3; ++d) A[q][d + 1] = x[d];
    }
    if (!invert4(A, C)) return fail(p, DDFD_E_ARG, "mesh: degenerate tetrahedron");
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = A[1][d + 1] - A[0][d + 1];
      e2[d] = A[2][d + 1] - A[0][d + 1];
      e3[d] = A[3][d + 1] - A[0][d + 1];
    }
    const double vol = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                                 e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
    vol_sum += vol;
    const double sv = std::sqrt(vol);
    for (int q = 0; q < 4; ++q) {
      const long long v = p->mesh_tets[t * 4 + q];
      tnode[t * 4 + q] = off(v);
      for (int d = 0; d < 3; ++d) tgrad[t * 12 + q * 3 + d] = sv * C[d + 1][q];
      const long long r = rowof(v);
      if (r >= 0) {
        rptr[r + 1]++;
        mass[r] += vol / 4.0;
      }
    }
  }
  const double cube = std::pow((b - a) * p->h, 3);
  if (std::fabs(vol_sum - cube) > 1e-9 * cube)
    return fail(p, DDFD_E_ARG, "mesh: the tetrahedra do not fill the FEM cube");
  for (long long r = 0; r < rows; ++r) {
    if (!(mass[r] > 0.0)) return fail(p, DDFD_E_ARG, "mesh: a FEM row without elements");
    rptr[r + 1] += rptr[r];
  }
  const long long ninc = rptr[rows];
  std::vector<int> itet((size_t)ninc), iloc((size_t)ninc), fillp(rptr.begin(), rptr.end() - 1), rnode((size_t)rows);
  std::vector<double> scale((size_t)rows);
  for (long long t = 0; t < ntet; ++t)
    for (int q = 0; q < 4; ++q) {
      const long long r = rowof(p->mesh_tets[t * 4 + q]);
      if (r >= 0) {
        itet[fillp[r]] = (int)t;
        iloc[fillp[r]++] = q;
      }
    }
  for (long long k = a + 1; k < b; ++k)
    for (long long j = a + 1; j < b; ++j)
      for (long long i = a + 1; i < b; ++i) {
        const long long v = i + n * (j + n * k);
        rnode[rowof(v)] = off(v);
      }
  for (int e = 0; e < p->n_new; ++e) rnode[grid_rows + e] = off(n3 + e);
  for (long long r = 0; r < rows; ++r) scale[r] = p->h * p->h / mass[r];
  // lumped masses of the free nodes: grid free nodes, then the new nodes
  std::vector<double> mfree((size_t)p->n_free);
  for (long long f = 0; f < p->n_free_grid; ++f) {
    const long long li = f % p->nf, lj = (f / p->nf) % p->nf, lk = f / ((long long)p->nf * p->nf);
    mfree[f] = mass[rowof((p->f0 + li) + n * ((p->f0 + lj) + (long long)n * (p->f0 + lk)))];
  }
  for (int e = 0; e < p->n_new; ++e) mfree[p->n_free_grid + e] = mass[grid_rows + e];
  std::vector<double> rpos((size_t)rows * 3);
  for (long long k = a + 1; k < b; ++k)
    for (long long j = a + 1; j < b; ++j)
      for (long long i = a + 1; i < b; ++i) {
        const long long r = rowof(i + n * (j + n * k));
        rpos[3 * r] = (double)i;
        rpos[3 * r + 1] = (double)j;
        rpos[3 * r + 2] = (double)k;
      }
  for (int e = 0; e < p->n_new; ++e)
    for (int d = 0; d < 3; ++d) rpos[3 * (grid_rows + e) + d] = X[(size_t)e * 3 + d] / p->h;
  // grid rows whose elements are the 24 untouched Kuhn tets take the block stencil
  std::vector<unsigned char> stencil;
  kuhn_stencil_rows(grid_rows, n, rptr.data(), itet.data(), p->mesh_tets.data(), &stencil);
  int st;
  if ((st = upload_ebe(p, rows, ntet, tnode, tgrad, rptr, itet, iloc, rnode, scale, rpos, &stencil))) return st;
  const size_t es = p->esz, xb = 3 * (size_t)std::max(p->n_new, 1) * es;
  if ((st = dalloc_t(p, (size_t)p->n_free, &p->mass_free)) || (st = dalloc(p, xb, &p->X[0])) ||
      (st = dalloc(p, xb, &p->X[1])) || (st = dalloc(p, xb, &p->xcoef)) ||
      (!p->fonly && ((st = dalloc(p, xb, &p->XMu[0])) || (st = dalloc(p, xb, &p->XMu[1])))))
    return st;
  CK(cudaMemcpy(p->mass_free, mfree.data(), p->n_free * sizeof(double), cudaMemcpyHostToDevice));
  for (int q = 0; q < 2; ++q) {
    CK(cudaMemset(p->X[q], 0, xb));
    if (p->XMu[q]) CK(cudaMemset(p->XMu[q], 0, xb));
  }
  CK(cudaMemset(p->xcoef, 0, xb));
  return DDFD_OK;
}

int build_maps(ddfd_problem *p) {
  FieldMaps fm;
  const int st = encode_field_maps(&p->err, &fm, p->E, p->Mu, p->kcoef, p->n, p->px, p->fp32, 1);
  if (st) return st;
  for (int q = 0; q < 2; ++q) {
    p->mE_halo[q] = fm.E_halo[q];
    p->mE_ctr[q] = fm.E_ctr[q];
    p->mM_halo[q] = fm.M_halo[q];
    p->mM_ctr[q] = fm.M_ctr[q];
  }
  p->mS = fm.S;
  p->mQ = fm.Q;
  return DDFD_OK;
}

int check_err(ddfd_problem *p) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, p->errflag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (e) {
    CK(cudaMemsetAsync(p->errflag, 0, sizeof(int), p->stream));
    return fail(p, DDFD_E_TIMEOUT, "a kernel gave up a bounded wait on its TMA copies");
  }
  return DDFD_OK;
}

int set_coeffs_impl(ddfd_problem *p, const double *eps, const double *sig, const double *eps0,
                    const double *sig0, cudaMemcpyKind kind) {
  if (!eps || !sig) return fail(p, DDFD_E_ARG, "eps and sigma are required");
  const size_t nfb = (size_t)p->n_free * sizeof(double);
  CK(cudaMemcpyAsync(p->coef_stage, eps, nfb, kind, p->stream));
  CK(cudaMemcpyAsync(p->coef_stage + p->n_free, sig, nfb, kind, p->stream));
  std::vector<double> fill;
  if (!eps0 || !sig0) fill.assign((size_t)p->n_free, 0.0);
  if (eps0) {
    CK(cudaMemcpyAsync(p->coef_stage + 2 * p->n_free, eps0, nfb, kind, p->stream));
  } else {
    std::vector<double> ones((size_t)p->n_free, 1.0);
    CK(cudaMemcpyAsync(p->coef_stage + 2 * p->n_free, ones.data(), nfb, cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  if (sig0)
    CK(cudaMemcpyAsync(p->coef_stage + 3 * p->n_free, sig0, nfb, kind, p->stream));
  else
    CK(cudaMemcpyAsync(p->coef_stage + 3 * p->n_free, fill.data(), nfb, cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream));
  launch_check_coeffs(p->coef_stage, (int)p->n_free, p->cfg.eps_max, p->cfg.sig_max, p->flag, p->stream);
  ++p->launches;
  int flag = 0;
  int st = read_flag(p, &flag);
  if (st) return st;
  if (flag) return fail(p, DDFD_E_COEFF, "coefficient outside [1, eps_max] x [0, sig_max] or non-finite");
  CK(cudaMemcpyAsync(p->coef, p->coef_stage, 4 * nfb, cudaMemcpyDeviceToDevice, p->stream));
  launch_expand_coeffs(p->fp32, p->coef, p->nf, p->f0, p->n, p->px, p->cs, p->tau, p->kcoef, p->stream,
                       p->n_free);
  ++p->launches;
  if (p->n_new) {
    launch_expand_new(p->fp32, p->coef, p->n_free, p->n_free_grid, p->n_new, p->tau, p->xcoef, p->stream);
    ++p->launches;
  }
  p->state = ST_READY;
  ++p->generation;
  if (p->cfg.cfl_check) {
    st = cfl_check(p);
    if (st) return st;
  }
  return sync_check(p);
}

int forward_impl(ddfd_problem *p, double *trace_out, cudaMemcpyKind kind) {
  // the run overwrites the trace and the E history: until it has completed,
  // no earlier forward or adjoint state may be used
  p->state = ST_READY;
  ++p->generation;
  int st = run_sequence(p, false);
  if (st) return st;
  if ((st = check_err(p))) return st;
  const long long cnt = (long long)p->n_src * (p->Nt + 1) * p->n_det * 3;
  CK(cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream));
  launch_nonfinite(p->trace, cnt, p->flag, p->stream);
  if (cnt > 0) ++p->launches;
  int flag = 0;
  int s2 = read_flag(p, &flag);
  if (s2) return s2;
  p->state = ST_FORWARD;
  if (flag) return fail(p, DDFD_E_NONFINITE, "non-finite value in the forward trace");
  if (trace_out && cnt > 0)
    CK(cudaMemcpyAsync(trace_out, p->trace, cnt * sizeof(double), kind, p->stream));
  return sync_check(p);
}

int functional_impl(ddfd_problem *p, const double *eobs, double *J, bool host) {
  if (p->state < ST_FORWARD) return fail(p, DDFD_E_STATE, "ddfd_functional needs a forward run");
  if (!J || (!eobs && p->n_det > 0)) return fail(p, DDFD_E_ARG, "eobs and J are required");
  const long long cnt = (long long)p->n_src * (p->Nt + 1) * p->n_det * 3;
  const double *e = eobs;
  if (host && cnt > 0) {
    CK(cudaMemcpyAsync(p->eobs_stage, eobs, cnt * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    e = p->eobs_stage;
  }
  launch_residual(p->trace, e, p->z, p->Nt, p->n_det, p->n_src, p->tau, p->res, p->part, p->n_part, p->stream);
  launch_sum(p->part, p->n_part, p->scal, p->stream);
  launch_regulariser(p->coef, (int)p->n_free, p->part, p->n_part, p->stream, p->mass_free);
  launch_sum(p->part, p->n_part, p->scal + 1, p->stream);
  launch_sum(p->part + p->n_part, p->n_part, p->scal + 2, p->stream);
  p->launches += 5;
  double v[3];
  CK(cudaMemcpyAsync(v, p->scal, sizeof(v), cudaMemcpyDeviceToHost, p->stream));
  int st = sync_check(p);
  if (st) return st;
  const double m = p->mass_free ? 1.0 : p->h * p->h * p->h;  // with per-node masses the sums carry them
  const double Jv = 0.5 * p->tau * v[0] + 0.5 * p->cfg.gamma_eps * m * v[1] + 0.5 * p->cfg.gamma_sig * m * v[2];
  if (!std::isfinite(Jv)) return fail(p, DDFD_E_NONFINITE, "non-finite functional");
  *J = Jv;
  return DDFD_OK;
}

int adjoint_impl(ddfd_problem *p, const double *eobs, bool host) {
  if (p->fonly) return fail(p, DDFD_E_STATE, "the handle was created forward_only");
  if (p->state < ST_FORWARD) return fail(p, DDFD_E_STATE, "ddfd_adjoint needs a forward run");
  if (!eobs && p->n_det > 0) return fail(p, DDFD_E_ARG, "eobs is required");
  const long long cnt = (long long)p->n_src * (p->Nt + 1) * p->n_det * 3;
  const double *e = eobs;
  if (host && cnt > 0) {
    CK(cudaMemcpyAsync(p->eobs_stage, eobs, cnt * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    e = p->eobs_stage;
  }
  launch_residual(p->trace, e, p->z, p->Nt, p->n_det, p->n_src, p->tau, p->res, p->part, p->n_part, p->stream);
  ++p->launches;
  p->state = ST_FORWARD;  // the accumulators are overwritten: no earlier gradient survives a failed run
  int st = run_sequence(p, true);
  if (st) return st;
  if ((st = check_err(p))) return st;
  const int s2 = sync_check(p);
  if (s2) return s2;
  p->state = ST_ADJOINT;
  return DDFD_OK;
}

int gradient_impl(ddfd_problem *p, double *g_eps, double *g_sig, bool host) {
  if (p->state < ST_ADJOINT) return fail(p, DDFD_E_STATE, "ddfd_gradient needs an adjoint run");
  if (!g_eps || !g_sig) return fail(p, DDFD_E_ARG, "gradient outputs are required");
  const double m = p->h * p->h * p->h;
  double *ge = host ? p->gout : g_eps;
  double *gs = host ? p->gout + p->n_free : g_sig;
  if (p->mass_free)
    launch_grad_finalize(p->coef, (int)p->n_free, p->gacc, p->gacc + p->n_free, 1.0 / (p->tau * p->tau),
                         1.0 / (2.0 * p->tau), m, p->cfg.gamma_eps, p->cfg.gamma_sig, ge, gs, p->stream,
                         p->mass_free);
  else
    launch_grad_finalize(p->coef, (int)p->n_free, p->gacc, p->gacc + p->n_free, m / (p->tau * p->tau),
                         m / (2.0 * p->tau), m, p->cfg.gamma_eps, p->cfg.gamma_sig, ge, gs, p->stream);
  CK(cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream));
  launch_nonfinite(ge, p->n_free, p->flag, p->stream);
  launch_nonfinite(gs, p->n_free, p->flag, p->stream);
  p->launches += 3;
  int flag = 0;
  int st = read_flag(p, &flag);
  if (st) return st;
  if (flag) return fail(p, DDFD_E_NONFINITE, "non-finite gradient");
  if (host) {
    CK(cudaMemcpyAsync(g_eps, ge, p->n_free * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(g_sig, gs, p->n_free * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  }
  return sync_check(p);
}

}  // namespace

extern "C" {

void ddfd_config_default(ddfd_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->cfl = 0.3;
  c->precision = DDFD_FP64;
  c->fem_kind = DDFD_FEM_STENCIL;
  c->n_src = 1;
  c->source_kind = DDFD_SRC_GAUSS;
  c->freq = 2.0;
  c->t0 = 0.75;
  c->width = 0.25;
  c->t1 = -1.0;
  c->absorbing_faces = DDFD_ABS_BOTTOM | DDFD_ABS_TOP;
  c->z_delta_frac = 0.1;
  c->eps_max = 100.0;
  c->sig_max = 100.0;
}

const char *ddfd_create_error(void) { return g_create_err.c_str(); }

}  // extern "C"

namespace {
// Stacked field storage of a batch member: slot of E[0], E[1], Mu[0], Mu[1]
// and the coefficient field.
struct MemberSlot {
  void *E[2], *Mu[2], *kcoef;
  ddfd_batch *batch;
  int slot;
};

int create_impl(const ddfd_config *cfg, const MemberSlot *ext, ddfd_problem **out);
}  // namespace

extern "C" {

int ddfd_create(const ddfd_config *cfg, ddfd_problem **out) { return create_impl(cfg, nullptr, out); }

}  // extern "C"

namespace {
int create_impl(const ddfd_config *cfg, const MemberSlot *ext, ddfd_problem **out) {
  g_create_err.clear();
  if (!cfg || !out) {
    g_create_err = "NULL argument";
    return DDFD_E_ARG;
  }
  std::string m;
  int st = validate(cfg, &m);
  if (st) {
    g_create_err = m;
    return st;
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_create_err = std::string("no usable CUDA device: ") + cudaGetErrorString(ce);
    return DDFD_E_CUDA;
  }
  ddfd_problem *p = new ddfd_problem();
  p->cfg = *cfg;
  if (cfg->src_dir) p->src_dir.assign(cfg->src_dir, cfg->src_dir + 3 * cfg->n_src);
  if (cfg->fem_kind == DDFD_FEM_MESH) {
    p->mesh_parents.assign(cfg->mesh_parents, cfg->mesh_parents + 2 * (size_t)cfg->mesh_n_new);
    p->mesh_tets.assign(cfg->mesh_tets, cfg->mesh_tets + 4 * (size_t)cfg->mesh_n_tets);
    p->n_new = cfg->mesh_n_new;
  }
  p->cfg.mesh_parents = nullptr;
  p->cfg.mesh_tets = nullptr;
  if (cfg->n_det > 0) p->det_ij.assign(cfg->det_ij, cfg->det_ij + 2 * cfg->n_det);
  p->cfg.src_dir = nullptr;
  p->cfg.det_ij = nullptr;
  p->n = cfg->n;
  p->fem_n = cfg->fem_n;
  p->a = (cfg->n - cfg->fem_n) / 2;
  p->b = p->a + cfg->fem_n - 1;
  p->f0 = p->a + 2;
  p->nf = cfg->fem_n - 4;
  p->n_free_grid = (long long)p->nf * p->nf * p->nf;
  p->n_free = p->n_free_grid + p->n_new;
  p->nn = (long long)p->n * p->n * p->n;
  p->px = (p->n + 7) / 8 * 8;
  p->cs = (long long)p->px * p->n * p->n;
  p->Nt = cfg->n_steps;
  p->n_src = cfg->n_src;
  p->n_det = cfg->n_det;
  p->h = 1.0 / (p->n - 1);
  p->tau = cfg->cfl * p->h;
  p->fp32 = cfg->precision == DDFD_FP32;
  p->esz = p->fp32 ? 4 : 8;
  p->stream = (cudaStream_t)cfg->stream;
  p->kz = cfg->tile_kz ? cfg->tile_kz : (p->n >= 128 ? 16 : 8);

  auto bail = [&](int code) {
    g_create_err = p->err;
    destroy_problem(p);
    return code;
  };
  for (int q = 0; q < 4; ++q)
    if (cudaEventCreate(&p->ev[q]) != cudaSuccess) {
      p->err = "cudaEventCreate failed";
      return bail(DDFD_E_CUDA);
    }
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      prepare_step_kernels() != cudaSuccess || prepare_ebe_kernels() != cudaSuccess) {
    p->err = "stream creation or kernel attribute setup failed";
    return bail(DDFD_E_CUDA);
  }
  KuhnBlocks kb;
  if (!build_kuhn_blocks(&kb, &m)) {
    p->err = m;
    return bail(DDFD_E_ARG);
  }
  if ((ce = check_kuhn_blocks(kb, p->stream)) != cudaSuccess) {
    p->err = "the Kuhn blocks assembled from the tetrahedra differ from the compiled-in table";
    return bail(DDFD_E_CUDA);
  }
  std::memcpy(p->kuhn_B, kb.B, sizeof(p->kuhn_B));
  std::vector<double> delay_host;
  setup_sources(p, &delay_host);
  const size_t fbytes = 3 * (size_t)p->cs * p->esz;
  const size_t trn = (size_t)p->n_src * (p->Nt + 1) * p->n_det * 3;
  p->fonly = cfg->forward_only != 0;
  if (cfg->n_snapshots > 0 && !p->fonly) {
    p->seg = (p->Nt + cfg->n_snapshots - 1) / cfg->n_snapshots;
    p->nsnap = (p->Nt + p->seg - 1) / p->seg;
  }
  const size_t histn = p->fonly ? 0
                       : p->nsnap ? (size_t)(p->seg + 1) * 3 * p->n_free
                                  : (size_t)p->n_src * (p->Nt + 1) * 3 * p->n_free;
  if (ext) {
    for (int q = 0; q < 2; ++q) {
      p->E[q] = ext->E[q];
      p->Mu[q] = ext->Mu[q];
    }
    p->kcoef = ext->kcoef;
    p->batch = ext->batch;
    p->slot = ext->slot;
  } else if ((st = dalloc(p, fbytes, &p->E[0])) || (st = dalloc(p, fbytes, &p->E[1])) ||
             (!p->fonly && ((st = dalloc(p, fbytes, &p->Mu[0])) || (st = dalloc(p, fbytes, &p->Mu[1])))) ||
             (st = dalloc(p, 3 * (size_t)p->cs * p->esz, &p->kcoef))) {
    return bail(st);
  }
  if ((st = dalloc_t(p, 1, &p->errflag)) ||
      (st = dalloc(p, histn * p->esz, &p->hist)) || (st = dalloc_t(p, trn, &p->trace)) ||
      (st = dalloc_t(p, trn, &p->res)) || (st = dalloc_t(p, trn, &p->eobs_stage)) ||
      (st = dalloc_t(p, 2 * (size_t)p->n_free, &p->gacc)) || (st = dalloc_t(p, 4 * (size_t)p->n_free, &p->coef)) ||
      (st = dalloc_t(p, 4 * (size_t)p->n_free, &p->coef_stage)) ||
      (st = dalloc_t(p, 2 * (size_t)p->n_free, &p->gout)) || (st = dalloc_t(p, (size_t)p->Nt + 1, &p->z)) ||
      (st = dalloc_t(p, 2 * (size_t)p->n_part, &p->part)) || (st = dalloc_t(p, 4, &p->scal)) ||
      (st = dalloc_t(p, 1, &p->flag)) || (st = dalloc_t(p, (size_t)std::max(p->n_det, 1), &p->det_node)) ||
      (st = dalloc_t(p, (size_t)p->n * p->n + 1, &p->det_ptr)) ||
      (st = dalloc_t(p, (size_t)std::max(p->n_det, 1), &p->det_list)) ||
      (p->fp32 && (st = dalloc_t(p, 2 * (size_t)p->n_free, &p->gpart))))
    return bail(st);
  if (p->nsnap && (st = dalloc(p, (size_t)p->n_src * p->nsnap * 2 * fbytes, &p->snap))) return bail(st);
  if (cfg->grad_variant == DDFD_GRAD_LITERAL) {
    const size_t nfu = (size_t)(p->b - p->a - 1) * (p->b - p->a - 1) * (p->b - p->a - 1);
    const size_t hb = (size_t)p->n_src * (p->Nt + 1) * 3 * nfu * p->esz;
    if ((st = dalloc(p, hb, &p->hist_fem))) return bail(st);
    if (cudaMemsetAsync(p->hist_fem, 0, hb, p->stream) != cudaSuccess) {
      p->err = "cudaMemsetAsync of the FEM-node history failed";
      return bail(DDFD_E_CUDA);
    }
  }
  bool any_oblique = false;
  for (int s = 0; s < p->n_src; ++s) any_oblique |= p->oblique[s] != 0;
  if (any_oblique && (st = dalloc_t(p, delay_host.size(), &p->delay))) return bail(st);

  // tables
  std::vector<double> zt((size_t)p->Nt + 1);
  const double T = p->Nt * p->tau, dl = cfg->z_delta_frac * T;
  for (int q = 0; q <= p->Nt; ++q) {
    const double t = q * p->tau;
    zt[q] = (dl <= 0.0 || t <= T - dl) ? 1.0 : 0.5 * (1.0 + std::cos(kPi * (t - T + dl) / dl));
  }
  std::vector<int> dnode((size_t)std::max(p->n_det, 1), 0), dptr((size_t)p->n * p->n + 1, 0),
      dlist((size_t)std::max(p->n_det, 1), 0);
  for (int d = 0; d < p->n_det; ++d) {
    const int i = p->det_ij[2 * d], j = p->det_ij[2 * d + 1];
    dnode[d] = (int)(i + (long long)p->px * (j + (long long)p->n * (p->n - 1)));
    dptr[i + p->n * j + 1]++;
  }
  for (int q = 0; q < p->n * p->n; ++q) dptr[q + 1] += dptr[q];
  {
    std::vector<int> fillp(dptr.begin(), dptr.end() - 1);
    for (int d = 0; d < p->n_det; ++d) {
      const int i = p->det_ij[2 * d], j = p->det_ij[2 * d + 1];
      dlist[fillp[i + p->n * j]++] = d;
    }
  }
  auto h2d = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->stream);
  };
  if (h2d(p->z, zt.data(), zt.size() * sizeof(double)) || h2d(p->det_node, dnode.data(), dnode.size() * sizeof(int)) ||
      h2d(p->det_ptr, dptr.data(), dptr.size() * sizeof(int)) ||
      h2d(p->det_list, dlist.data(), dlist.size() * sizeof(int)) ||
      (p->delay && h2d(p->delay, delay_host.data(), delay_host.size() * sizeof(double)))) {
    p->err = "table upload failed";
    return bail(DDFD_E_CUDA);
  }
  launch_coef_vacuum(p->fp32, p->cs, p->kcoef, p->stream);
  ++p->launches;
  if (cudaMemsetAsync(p->errflag, 0, sizeof(int), p->stream) ||
 cudaMemsetAsync(p->E[0], 0, fbytes, p->stream) ||
      cudaMemsetAsync(p->E[1], 0, fbytes, p->stream) ||
      (p->Mu[0] && cudaMemsetAsync(p->Mu[0], 0, fbytes, p->stream)) ||
      (p->Mu[1] && cudaMemsetAsync(p->Mu[1], 0, fbytes, p->stream))) {
    p->err = "memset failed";
    return bail(DDFD_E_CUDA);
  }
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
    p->err = std::string("create: ") + cudaGetErrorString(cudaGetLastError());
    return bail(DDFD_E_CUDA);
  }
  if ((st = build_maps(p))) return bail(st);
  if (cfg->fem_kind == DDFD_FEM_EBE && (st = build_ebe(p))) return bail(st);
  if (cfg->fem_kind == DDFD_FEM_MESH && (st = build_mesh(p))) return bail(st);
  // vacuum coefficients
  std::vector<double> one((size_t)p->n_free, 1.0), zero((size_t)p->n_free, 0.0);
  const bool chk = p->cfg.cfl_check != 0;
  p->cfg.cfl_check = 0;
  st = set_coeffs_impl(p, one.data(), zero.data(), nullptr, nullptr, cudaMemcpyHostToDevice);
  p->cfg.cfl_check = chk;
  if (st) return bail(st);
  *out = p;
  return DDFD_OK;
}
}  // namespace

extern "C" {

void ddfd_destroy(ddfd_problem *p) {
  if (!p || p->batch) return;  // batch members go with their batch
  destroy_problem(p);
}

}  // extern "C"

namespace {
void destroy_problem(ddfd_problem *p) {
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  for (void *v : p->allocs) cudaFree(v);
  for (int q = 0; q < 4; ++q)
    if (p->ev[q]) cudaEventDestroy(p->ev[q]);
  drop_graphs(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}
}  // namespace

extern "C" {

const char *ddfd_last_error(const ddfd_problem *p) { return p ? p->err.c_str() : "NULL handle"; }

int ddfd_set_coeffs(ddfd_problem *p, const double *eps, const double *sig, const double *eps0,
                    const double *sig0) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return set_coeffs_impl(p, eps, sig, eps0, sig0, cudaMemcpyHostToDevice);
}

int ddfd_set_coeffs_dev(ddfd_problem *p, const double *eps, const double *sig, const double *eps0,
                        const double *sig0) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return set_coeffs_impl(p, eps, sig, eps0, sig0, cudaMemcpyDeviceToDevice);
}

int ddfd_forward(ddfd_problem *p, double *trace_out) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return forward_impl(p, trace_out, cudaMemcpyDeviceToHost);
}

int ddfd_forward_dev(ddfd_problem *p, double *trace_out) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return forward_impl(p, trace_out, cudaMemcpyDeviceToDevice);
}

int ddfd_functional(ddfd_problem *p, const double *eobs, double *J) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return functional_impl(p, eobs, J, true);
}

int ddfd_functional_dev(ddfd_problem *p, const double *eobs, double *J) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return functional_impl(p, eobs, J, false);
}

int ddfd_adjoint(ddfd_problem *p, const double *eobs) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return adjoint_impl(p, eobs, true);
}

int ddfd_adjoint_dev(ddfd_problem *p, const double *eobs) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return adjoint_impl(p, eobs, false);
}

int ddfd_gradient(ddfd_problem *p, double *g_eps, double *g_sig) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return gradient_impl(p, g_eps, g_sig, true);
}

int ddfd_gradient_dev(ddfd_problem *p, double *g_eps, double *g_sig) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  return gradient_impl(p, g_eps, g_sig, false);
}

int ddfd_get_info(const ddfd_problem *p, ddfd_info *info) {
  if (!p || !info) return DDFD_E_ARG;
  info->n = p->n;
  info->fem_n = p->fem_n;
  info->n_free = (int32_t)p->n_free;
  info->n_det = p->n_det;
  info->n_src = p->n_src;
  info->n_steps = p->Nt;
  info->a = p->a;
  info->b = p->b;
  info->switch_step = p->n1.empty() ? 0 : p->n1[0];
  info->h = p->h;
  info->tau = p->tau;
  info->device_bytes = p->bytes;
  info->kernel_launches = p->launches;
  info->forward_steps = p->fwd_steps;
  info->generation = p->generation;
  return DDFD_OK;
}

int ddfd_get_timing(const ddfd_problem *p, ddfd_timing *t) {
  if (!p || !t) return DDFD_E_ARG;
  t->forward_loop_ms = p->fwd_ms;
  t->adjoint_loop_ms = p->adj_ms;
  t->forward_step_kernels = p->fwd_kernels;
  t->adjoint_step_kernels = p->adj_kernels;
  return DDFD_OK;
}

int ddfd_test_gather_timeout(ddfd_problem *p, int32_t fault, uint32_t spin_limit) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  if (!p->ebe_rows || p->ebe_nblocks <= 0)
    return fail(p, DDFD_E_ARG, "the timeout test needs an element gather (fem_kind DDFD_FEM_EBE or DDFD_FEM_MESH)");
  if (fault != 0 && fault != 1) return fail(p, DDFD_E_ARG, "fault must be 0 or 1");
  p->test_fault = fault;
  p->test_spin = spin_limit;
  drop_graphs(p);  // the captured sequences hold the old kernel parameters
  return DDFD_OK;
}

int ddfd_set_capture(ddfd_problem *p, int32_t count, const int32_t *steps) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  if (count < 0 || count > kMaxCapture || (count > 0 && !steps))
    return fail(p, DDFD_E_ARG, "capture count must be in [0, 16]");
  for (int q = 0; q < count; ++q)
    if (steps[q] < 0 || steps[q] > p->Nt) return fail(p, DDFD_E_ARG, "capture step out of range");
  const size_t fbytes = 3 * (size_t)p->cs * p->esz;
  if (count > (int)p->cap_steps.size() || !p->capE) {
    // grow: allocate fresh buffers for count slots
    int st;
    if ((st = dalloc(p, fbytes * std::max(count, 1), &p->capE)) ||
        (st = dalloc(p, fbytes * std::max(count, 1), &p->capMu)))
      return st;
  }
  p->cap_steps.assign(steps, steps + count);
  drop_graphs(p);  // the captured sequences copy fields at the capture steps
  return DDFD_OK;
}

int ddfd_get_capture(ddfd_problem *p, int32_t kind, int32_t idx, double *out) {
  if (!p || !out) return DDFD_E_ARG;
  p->err.clear();
  if (idx < 0 || idx >= (int)p->cap_steps.size() || (kind != 0 && kind != 1))
    return fail(p, DDFD_E_ARG, "bad capture index or kind");
  const size_t cnt = 3 * (size_t)p->cs;
  const char *src = (const char *)(kind == 0 ? p->capE : p->capMu) + idx * cnt * p->esz;
  CK(cudaStreamSynchronize(p->stream));
  std::vector<double> tmp(cnt);
  if (p->fp32) {
    std::vector<float> tf(cnt);
    CK(cudaMemcpy(tf.data(), src, cnt * 4, cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < cnt; ++q) tmp[q] = tf[q];
  } else {
    CK(cudaMemcpy(tmp.data(), src, cnt * 8, cudaMemcpyDeviceToHost));
  }
  const int n = p->n;
  for (int c = 0; c < 3; ++c)
    for (long long kj = 0; kj < (long long)n * n; ++kj)
      for (int i = 0; i < n; ++i)
        out[(size_t)c * p->nn + kj * n + i] = tmp[(size_t)c * p->cs + kj * p->px + i];
  return DDFD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tile autotuner and batched problems
// ---------------------------------------------------------------------------

struct ddfd_batch {
  std::vector<ddfd_problem *> m;
  std::string err;
  int n = 0, Nt = 0, px = 0, fp32 = 0, kz = 16, seg = 0;
  long long cs = 0;
  size_t esz = 8;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  void *E[2] = {nullptr, nullptr}, *Mu[2] = {nullptr, nullptr}, *kcoef = nullptr;
  std::vector<void *> allocs;
  int64_t bytes = 0, launches = 0;
  FieldMaps maps;
  int *errflag = nullptr;
  cudaGraphExec_t gfwd = nullptr, gadj = nullptr;
  int64_t gfwd_launches = 0, gadj_launches = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double fwd_ms = 0.0, adj_ms = 0.0;
  int64_t fwd_kernels = 0, adj_kernels = 0;
  // conjugate gradient work space (FP64, free nodes): 14 vectors, partial
  // sums, the 6 reduced scalars
  double *cg = nullptr;
  long long cg_n = 0;
};

namespace {

int bfail(ddfd_batch *b, int code, const std::string &m) {
  b->err = m;
  return code;
}

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(b, DDFD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

const int kTileKz[] = {4, 6, 8, 12, 16, 24, 32};

// Runs trial(kz, &ms) for every candidate z depth (after one untimed warm-up
// trial) and returns the fastest in *best.
template <typename Trial>
int autotune_kz(int n, Trial trial, int *best) {
  int st;
  float ms = 0.0f;
  if ((st = trial(kTileKz[0] <= n ? kTileKz[0] : n, &ms))) return st;
  float best_ms = 3.4e38f;
  *best = 0;
  for (int kz : kTileKz) {
    if (kz > n) break;
    if ((st = trial(kz, &ms))) return st;
    if (ms < best_ms) {
      best_ms = ms;
      *best = kz;
    }
  }
  return DDFD_OK;
}

// E^n on the free nodes for trial step st (any valid slot of the history).
long long trial_hist_index(const ddfd_problem *p, int st) {
  return p->nsnap ? (long long)(st % p->seg) + 1 : (long long)st + 1;
}

template <typename T>
int single_trial(ddfd_problem *p, int steps, int kz, float *ms) {
  const size_t fbytes = 3 * (size_t)p->cs * sizeof(T);
  const size_t trn = (size_t)p->n_src * (p->Nt + 1) * p->n_det * 3;
  cudaStream_t sm = p->stream;
  p->kz = kz;
  for (int q = 0; q < 2; ++q) {
    CK(cudaMemsetAsync(p->E[q], 0, fbytes, sm));
    if (p->Mu[q]) CK(cudaMemsetAsync(p->Mu[q], 0, fbytes, sm));
  }
  if (trn) CK(cudaMemsetAsync(p->res, 0, trn * sizeof(double), sm));
  CK(cudaEventRecord(p->ev[0], sm));
  int64_t nk = 0;
  StepParams<T> P = base_params<T>(p);
  set_source(P, p, 0);
  int ic = 1, io = 0;
  for (int st = 0; st < steps; ++st) {
    set_forward_step(P, p, 0, st, p->E[ic], p->E[io],
                     p->fonly ? nullptr : (T *)p->hist + trial_hist_index(p, st) * 3 * p->n_free);
    enqueue_ebe<T>(p, p->E[ic], false, sm, &nk, p->X[ic]);
    launch_forward_step(single_launch(P, p->mE_halo[ic], p->mE_ctr[io], p), sm);
    std::swap(ic, io);
  }
  ic = 1, io = 0;
  for (int k = p->fonly ? 0 : steps; k >= 1; --k) {  // forward_only handles time the forward alone
    set_adjoint_step(P, p, 0, k, p->Mu[ic], p->Mu[io], (const T *)p->hist + trial_hist_index(p, k - 1) * 3 * p->n_free,
                     steps);
    enqueue_ebe<T>(p, p->Mu[ic], true, sm, &nk, p->XMu[ic]);
    launch_adjoint_step(single_launch(P, p->mM_halo[ic], p->mM_ctr[io], p), sm);
    std::swap(ic, io);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(p->ev[1], sm));
  CK(cudaEventSynchronize(p->ev[1]));
  CK(cudaEventElapsedTime(ms, p->ev[0], p->ev[1]));
  p->launches += 2 * steps + nk;
  return DDFD_OK;
}

// One batched step launch per group of BATCH_MAX members; fill(P, p) sets the
// per-step scalars of member p.
template <typename T, typename Fill>
void launch_groups(ddfd_batch *b, bool adj, const std::vector<int> &idx, const CUtensorMap &cur,
                   const CUtensorMap &old, Fill fill, cudaStream_t sm, int64_t *nk) {
  for (size_t g0 = 0; g0 < idx.size(); g0 += BATCH_MAX) {
    StepLaunch<T, BATCH_MAX> L;
    std::memset(&L, 0, sizeof(L));
    L.cur = cur;
    L.old = old;
    L.s = b->maps.S;
    L.q = b->maps.Q;
    L.nprob = (int)std::min<size_t>(BATCH_MAX, idx.size() - g0);
    L.zchunks = (b->n + b->kz - 1) / b->kz;
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
    if (adj)
      launch_adjoint_step(L, sm);
    else
      launch_forward_step(L, sm);
    ++*nk;
  }
}

std::vector<int> all_members(const ddfd_batch *b) {
  std::vector<int> v(b->m.size());
  for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
  return v;
}

template <typename T>
int enqueue_batch_forward(ddfd_batch *b, cudaStream_t sm, int64_t *nk) {
  const size_t fbytes = 3 * (size_t)b->cs * sizeof(T);
  const size_t slab = fbytes * b->m.size();
  const int Nt = b->Nt;
  *nk = 0;
  BCK(cudaMemsetAsync(b->E[0], 0, slab, sm));
  BCK(cudaMemsetAsync(b->E[1], 0, slab, sm));
  for (ddfd_problem *p : b->m)
    if (p->n_new) {
      BCK(cudaMemsetAsync(p->X[0], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
      BCK(cudaMemsetAsync(p->X[1], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
    }
  const std::vector<int> all = all_members(b);
  int ic = 1, io = 0;
  for (int st = 0; st < Nt; ++st) {
    for (ddfd_problem *p : b->m)
      if (p->nsnap && st % p->seg == 0) {
        char *sn = (char *)p->snap + (size_t)(st / p->seg) * 2 * fbytes;
        BCK(cudaMemcpyAsync(sn, p->E[ic], fbytes, cudaMemcpyDeviceToDevice, sm));
        BCK(cudaMemcpyAsync(sn + fbytes, p->E[io], fbytes, cudaMemcpyDeviceToDevice, sm));
      }
    auto fill = [&](StepParams<T> &P, ddfd_problem *p) {
      set_forward_step(P, p, 0, st, p->E[ic], p->E[io],
                       (p->nsnap || p->fonly) ? nullptr : (T *)p->hist + (size_t)(st + 1) * 3 * p->n_free);
    };
    // element-by-element members: their FEM rows of this level first
    for (ddfd_problem *p : b->m) enqueue_ebe<T>(p, p->E[ic], false, sm, nk, p->X[ic], b->errflag);
    launch_groups<T>(b, false, all, b->maps.E_halo[ic], b->maps.E_ctr[io], fill, sm, nk);
    for (ddfd_problem *p : b->m)
      if (p->n_new) {
        StepParams<T> P = base_params<T>(p);
        fill(P, p);
        enqueue_new_step<T>(p, p->X[ic], p->X[io], false, P, sm, nk);
      }
    std::swap(ic, io);
  }
  BCK(cudaGetLastError());
  for (ddfd_problem *p : b->m) {
    launch_gather_trace(p->E[ic], p->fp32, p->cs, p->n_det, p->det_node, p->trace + (size_t)Nt * p->n_det * 3, sm);
    if (p->n_det > 0) ++*nk;
  }
  BCK(cudaGetLastError());
  return DDFD_OK;
}

template <typename T>
int enqueue_batch_adjoint(ddfd_batch *b, cudaStream_t sm, int64_t *nk) {
  const size_t fbytes = 3 * (size_t)b->cs * sizeof(T);
  const size_t slab = fbytes * b->m.size();
  const int Nt = b->Nt;
  *nk = 0;
  for (ddfd_problem *p : b->m) BCK(cudaMemsetAsync(p->gacc, 0, 2 * (size_t)p->n_free * sizeof(double), sm));
  BCK(cudaMemsetAsync(b->Mu[0], 0, slab, sm));
  BCK(cudaMemsetAsync(b->Mu[1], 0, slab, sm));
  for (ddfd_problem *p : b->m)
    if (p->n_new) {
      BCK(cudaMemsetAsync(p->XMu[0], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
      BCK(cudaMemsetAsync(p->XMu[1], 0, 3 * (size_t)p->n_new * sizeof(T), sm));
    }
  const std::vector<int> all = all_members(b);
  std::vector<int> ck;  // checkpointing members: replayed segment by segment
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i]->nsnap) ck.push_back((int)i);
  const int seg = b->seg;
  const int nseg = seg ? (Nt + seg - 1) / seg : 1;
  int ic = 1, io = 0;
  for (int j = nseg - 1; j >= 0; --j) {
    const int n0 = seg ? j * seg : 0;
    const int n1 = seg ? std::min(n0 + seg, Nt) : Nt;
    if (!ck.empty()) {
      for (int i : ck) {
        ddfd_problem *p = b->m[i];
        const char *sn = (const char *)p->snap + (size_t)j * 2 * fbytes;
        BCK(cudaMemcpyAsync(p->E[1], sn, fbytes, cudaMemcpyDeviceToDevice, sm));
        BCK(cudaMemcpyAsync(p->E[0], sn + fbytes, fbytes, cudaMemcpyDeviceToDevice, sm));
      }
      int fc = 1, fo = 0;
      for (int st = n0; st < n1; ++st) {
        for (int i : ck) enqueue_ebe<T>(b->m[i], b->m[i]->E[fc], false, sm, nk, b->m[i]->X[fc], b->errflag);
        launch_groups<T>(
            b, false, ck, b->maps.E_halo[fc], b->maps.E_ctr[fo],
            [&](StepParams<T> &P, ddfd_problem *p) {
              set_forward_step(P, p, 0, st, p->E[fc], p->E[fo], (T *)p->hist + (size_t)(st + 1 - n0) * 3 * p->n_free);
            },
            sm, nk);
        std::swap(fc, fo);
      }
    }
    for (int k = n1; k >= n0 + 1; --k) {
      auto fill = [&](StepParams<T> &P, ddfd_problem *p) {
        const long long hk = p->nsnap ? k - n0 : k;
        set_adjoint_step(P, p, 0, k, p->Mu[ic], p->Mu[io], (const T *)p->hist + (size_t)hk * 3 * p->n_free, Nt);
      };
      for (ddfd_problem *p : b->m) enqueue_ebe<T>(p, p->Mu[ic], true, sm, nk, p->XMu[ic], b->errflag);
      launch_groups<T>(b, true, all, b->maps.M_halo[ic], b->maps.M_ctr[io], fill, sm, nk);
      for (ddfd_problem *p : b->m)
        if (p->n_new) {
          StepParams<T> P = base_params<T>(p);
          fill(P, p);
          enqueue_new_step<T>(p, p->XMu[ic], p->XMu[io], true, P, sm, nk);
        }
      std::swap(ic, io);
    }
  }
  BCK(cudaGetLastError());
  return DDFD_OK;
}

void drop_batch_graphs(ddfd_batch *b) {
  if (b->gfwd) cudaGraphExecDestroy(b->gfwd);
  if (b->gadj) cudaGraphExecDestroy(b->gadj);
  b->gfwd = b->gadj = nullptr;
}

int run_batch_sequence(ddfd_batch *b, bool adj) {
  cudaGraphExec_t *ge = adj ? &b->gadj : &b->gfwd;
  int64_t *gl = adj ? &b->gadj_launches : &b->gfwd_launches;
  if (!*ge) {
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
    int64_t nk = 0;
    int st;
    if (adj)
      st = b->fp32 ? enqueue_batch_adjoint<float>(b, b->cap_stream, &nk)
                   : enqueue_batch_adjoint<double>(b, b->cap_stream, &nk);
    else
      st = b->fp32 ? enqueue_batch_forward<float>(b, b->cap_stream, &nk)
                   : enqueue_batch_forward<double>(b, b->cap_stream, &nk);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    BCK(ec);
    const cudaError_t ei = cudaGraphInstantiate(ge, g, 0);
    cudaGraphDestroy(g);
    BCK(ei);
    *gl = nk;
  }
  cudaEvent_t e0 = b->ev[adj ? 2 : 0], e1 = b->ev[adj ? 3 : 1];
  BCK(cudaEventRecord(e0, b->stream));
  BCK(cudaGraphLaunch(*ge, b->stream));
  BCK(cudaEventRecord(e1, b->stream));
  BCK(cudaEventSynchronize(e1));
  float ms = 0.0f;
  BCK(cudaEventElapsedTime(&ms, e0, e1));
  b->launches += *gl;
  const int64_t groups = ((int64_t)b->m.size() + BATCH_MAX - 1) / BATCH_MAX;
  if (adj) {
    b->adj_ms = ms;
    int64_t ckg = 0;
    for (ddfd_problem *p : b->m) ckg += p->nsnap ? 1 : 0;
    ckg = (ckg + BATCH_MAX - 1) / BATCH_MAX;
    b->adj_kernels = (int64_t)b->Nt * (groups + ckg);
    for (ddfd_problem *p : b->m)
      if (p->nsnap) p->fwd_steps += b->Nt;
  } else {
    b->fwd_ms = ms;
    b->fwd_kernels = (int64_t)b->Nt * groups;
    for (ddfd_problem *p : b->m) p->fwd_steps += b->Nt;
  }
  return DDFD_OK;
}

int batch_check_err(ddfd_batch *b) {
  int e = 0;
  BCK(cudaMemcpyAsync(&e, b->errflag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (e) {
    BCK(cudaMemsetAsync(b->errflag, 0, sizeof(int), b->stream));
    return bfail(b, DDFD_E_TIMEOUT, "a kernel gave up a bounded wait on its TMA copies");
  }
  return DDFD_OK;
}

template <typename T>
int batch_trial(ddfd_batch *b, int steps, int kz, float *ms) {
  const size_t fbytes = 3 * (size_t)b->cs * sizeof(T);
  const size_t slab = fbytes * b->m.size();
  cudaStream_t sm = b->stream;
  b->kz = kz;
  for (int q = 0; q < 2; ++q) {
    BCK(cudaMemsetAsync(b->E[q], 0, slab, sm));
    if (b->Mu[q]) BCK(cudaMemsetAsync(b->Mu[q], 0, slab, sm));
  }
  for (ddfd_problem *p : b->m) {
    const size_t trn = (size_t)(p->Nt + 1) * p->n_det * 3;
    if (trn) BCK(cudaMemsetAsync(p->res, 0, trn * sizeof(double), sm));
  }
  const std::vector<int> all = all_members(b);
  int64_t nk = 0;
  BCK(cudaEventRecord(b->ev[0], sm));
  int ic = 1, io = 0;
  for (int st = 0; st < steps; ++st) {
    launch_groups<T>(
        b, false, all, b->maps.E_halo[ic], b->maps.E_ctr[io],
        [&](StepParams<T> &P, ddfd_problem *p) {
          set_forward_step(P, p, 0, st, p->E[ic], p->E[io],
                           p->fonly ? nullptr : (T *)p->hist + trial_hist_index(p, st) * 3 * p->n_free);
        },
        sm, &nk);
    std::swap(ic, io);
  }
  bool any_fonly = false;
  for (ddfd_problem *p : b->m) any_fonly |= p->fonly;
  ic = 1, io = 0;
  for (int k = any_fonly ? 0 : steps; k >= 1; --k) {  // forward_only members: forward trials only
    launch_groups<T>(
        b, true, all, b->maps.M_halo[ic], b->maps.M_ctr[io],
        [&](StepParams<T> &P, ddfd_problem *p) {
          set_adjoint_step(P, p, 0, k, p->Mu[ic], p->Mu[io],
                           (const T *)p->hist + trial_hist_index(p, k - 1) * 3 * p->n_free, steps);
        },
        sm, &nk);
    std::swap(ic, io);
  }
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(b->ev[1], sm));
  BCK(cudaEventSynchronize(b->ev[1]));
  BCK(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
  b->launches += nk;
  return DDFD_OK;
}

int batch_forward_impl(ddfd_batch *b, double *const *trace_out, cudaMemcpyKind kind) {
  for (ddfd_problem *p : b->m) {
    p->state = ST_READY;
    ++p->generation;
  }
  int st = run_batch_sequence(b, false);
  if (st) return st;
  if ((st = batch_check_err(b))) return st;
  for (size_t i = 0; i < b->m.size(); ++i) {
    ddfd_problem *p = b->m[i];
    const long long cnt = (long long)(p->Nt + 1) * p->n_det * 3;
    BCK(cudaMemsetAsync(p->flag, 0, sizeof(int), b->stream));
    if (cnt > 0) {
      launch_nonfinite(p->trace, cnt, p->flag, b->stream);
      ++b->launches;
    }
    int flag = 0;
    BCK(cudaMemcpyAsync(&flag, p->flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    p->state = ST_FORWARD;
    if (flag) return bfail(b, DDFD_E_NONFINITE, "non-finite value in the forward trace of member " + std::to_string(i));
    if (trace_out && trace_out[i] && cnt > 0)
      BCK(cudaMemcpyAsync(trace_out[i], p->trace, cnt * sizeof(double), kind, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  return DDFD_OK;
}

int batch_adjoint_impl(ddfd_batch *b, const double *const *eobs, bool host) {
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i]->fonly) return bfail(b, DDFD_E_STATE, "member " + std::to_string(i) + " was created forward_only");
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i]->state < ST_FORWARD)
      return bfail(b, DDFD_E_STATE, "member " + std::to_string(i) + " has no forward run");
  for (size_t i = 0; i < b->m.size(); ++i) {
    ddfd_problem *p = b->m[i];
    const long long cnt = (long long)(p->Nt + 1) * p->n_det * 3;
    if (cnt > 0 && (!eobs || !eobs[i])) return bfail(b, DDFD_E_ARG, "eobs of member " + std::to_string(i) + " is missing");
    const double *e = cnt > 0 ? eobs[i] : nullptr;
    if (host && cnt > 0) {
      BCK(cudaMemcpyAsync(p->eobs_stage, e, cnt * sizeof(double), cudaMemcpyHostToDevice, b->stream));
      e = p->eobs_stage;
    }
    launch_residual(p->trace, e, p->z, p->Nt, p->n_det, 1, p->tau, p->res, p->part, p->n_part, b->stream);
    ++b->launches;
  }
  for (ddfd_problem *p : b->m) p->state = ST_FORWARD;
  int st = run_batch_sequence(b, true);
  if (st) return st;
  if ((st = batch_check_err(b))) return st;
  BCK(cudaStreamSynchronize(b->stream));
  for (ddfd_problem *p : b->m) p->state = ST_ADJOINT;
  return DDFD_OK;
}

// The CGA of Sec. 4 over the batch's members (see ddfd_cg_run in ddfd.h).
int cg_run_impl(ddfd_batch *b, const double *const *eobs, const ddfd_cg_params *prm, double *eps_h,
                double *sig_h, ddfd_cg_iter *log, int32_t *iters, double *eps_it, double *sig_it) {
  if (iters) *iters = 0;
  if (!prm || !eps_h || !sig_h) return bfail(b, DDFD_E_ARG, "parameters, eps and sigma are required");
  if (prm->max_iter < 1 || !(prm->gamma_eps0 >= 0) || !(prm->gamma_sig0 >= 0) || !(prm->p >= 0 && prm->p < 1) ||
      !(prm->eps_max >= 1) || !(prm->sig_max >= 0) || !std::isfinite(prm->alpha_eps0) || !std::isfinite(prm->alpha_sig0))
    return bfail(b, DDFD_E_ARG, "bad CG parameters");
  ddfd_problem *p0 = b->m[0];
  for (size_t i = 0; i < b->m.size(); ++i) {
    const ddfd_problem *p = b->m[i];
    if (p->fem_n != p0->fem_n || p->n_free != p0->n_free || p->n_new != p0->n_new)
      return bfail(b, DDFD_E_ARG, "CG members must share fem_n (and their refined mesh)");
    if (p->cfg.gamma_eps != 0.0 || p->cfg.gamma_sig != 0.0)
      return bfail(b, DDFD_E_ARG, "CG members must have gamma_eps = gamma_sig = 0 (the CG regularises)");
    if (p->fonly) return bfail(b, DDFD_E_ARG, "CG members cannot be forward_only");
    const long long cnt = (long long)(p->Nt + 1) * p->n_det * 3;
    if (cnt > 0 && (!eobs || !eobs[i])) return bfail(b, DDFD_E_ARG, "eobs of member " + std::to_string(i) + " is missing");
  }
  const long long n = p0->n_free;
  cudaStream_t sm = b->stream;
  if (!b->cg || b->cg_n != n) {
    if (b->cg) {
      cudaFree(b->cg);
      b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), (void *)b->cg));
    }
    const size_t bytes = (14 * (size_t)n + 6 * CG_BLOCKS + 8) * sizeof(double);
    if (cudaMalloc((void **)&b->cg, bytes) != cudaSuccess) {
      cudaGetLastError();
      b->cg = nullptr;
      return bfail(b, DDFD_E_OOM, "cudaMalloc of the CG work space failed");
    }
    b->allocs.push_back(b->cg);
    b->bytes += (int64_t)bytes;
    b->cg_n = n;
  }
  double *v[14];
  for (int q = 0; q < 14; ++q) v[q] = b->cg + (size_t)q * n;
  double *eps = v[0], *sig = v[1], *eps_n = v[2], *sig_n = v[3], *re = v[4], *rs = v[5];
  double *Ge = v[6], *Gs = v[7], *Te = v[8], *Ts = v[9], *gte = v[10], *gts = v[11], *de = v[12], *ds = v[13];
  double *part = b->cg + 14 * (size_t)n, *out = part + 6 * CG_BLOCKS;
  const size_t nb = (size_t)n * sizeof(double);
  BCK(cudaMemcpyAsync(eps, eps_h, nb, cudaMemcpyHostToDevice, sm));
  BCK(cudaMemcpyAsync(sig, sig_h, nb, cudaMemcpyHostToDevice, sm));
  BCK(cudaMemcpyAsync(re, eps, nb, cudaMemcpyDeviceToDevice, sm));
  BCK(cudaMemcpyAsync(rs, sig, nb, cudaMemcpyDeviceToDevice, sm));
  std::vector<const double *> eobs_dev(b->m.size(), nullptr);
  for (size_t i = 0; i < b->m.size(); ++i) {
    ddfd_problem *p = b->m[i];
    const long long cnt = (long long)(p->Nt + 1) * p->n_det * 3;
    if (cnt > 0) BCK(cudaMemcpyAsync(p->eobs_stage, eobs[i], cnt * sizeof(double), cudaMemcpyHostToDevice, sm));
    eobs_dev[i] = p->eobs_stage;
  }
  // lumped mass of a free node (uniform mesh), or per-node masses carried by
  // the reductions themselves (refined mesh: m = 1 on the host)
  const double *mass = p0->mass_free;
  const double hm = p0->h * p0->h * p0->h;
  const double m = mass ? 1.0 : hm;
  double gam_e = prm->gamma_eps0, gam_s = prm->gamma_sig0;
  double alp_e = prm->alpha_eps0, alp_s = prm->alpha_sig0;
  double gg_e_prev = 0.0, gg_s_prev = 0.0;
  int done = 0;
  // an iteration that fails (typically DDFD_E_NONFINITE) keeps the records of
  // the iterations before it and hands back the iterate it was evaluating
  auto failed = [&](int st) {
    if (iters) *iters = done;
    cudaMemcpyAsync(eps_h, eps, nb, cudaMemcpyDeviceToHost, sm);
    cudaMemcpyAsync(sig_h, sig, nb, cudaMemcpyDeviceToHost, sm);
    cudaStreamSynchronize(sm);
    return st;
  };
  for (int it = 0; it < prm->max_iter; ++it) {
    BCK(cudaEventRecord(b->ev[0], sm));
    // 1. E^m, lambda^m, g^m
    int st;
    for (ddfd_problem *p : b->m)
      if ((st = set_coeffs_impl(p, eps, sig, nullptr, nullptr, cudaMemcpyDeviceToDevice)))
        return failed(bfail(b, st, p->err));
    if ((st = batch_forward_impl(b, nullptr, cudaMemcpyDeviceToDevice))) return failed(st);
    double J_data = 0.0;
    for (size_t i = 0; i < b->m.size(); ++i) {
      double Ji = 0.0;
      if ((st = functional_impl(b->m[i], eobs_dev[i], &Ji, false))) return failed(bfail(b, st, b->m[i]->err));
      J_data += Ji;
    }
    if ((st = batch_adjoint_impl(b, eobs_dev.data(), false))) return failed(st);
    for (size_t i = 0; i < b->m.size(); ++i) {
      const bool first = i == 0;
      if ((st = gradient_impl(b->m[i], first ? Ge : Te, first ? Gs : Ts, false)))
        return failed(bfail(b, st, b->m[i]->err));
      if (!first) launch_cg_accum(Ge, Gs, Te, Ts, n, sm);
    }
    launch_cg_grad(Ge, Gs, eps, sig, re, rs, 1.0 / hm, gam_e, gam_s, gte, gts, de, ds, it > 0, n, part, out, sm,
                   mass);
    double r4[6];
    BCK(cudaMemcpyAsync(r4, out, sizeof(r4), cudaMemcpyDeviceToHost, sm));
    BCK(cudaStreamSynchronize(sm));
    const double gg_e = m * r4[0], gg_s = m * r4[1];
    const double J = J_data + 0.5 * gam_e * m * r4[2] + 0.5 * gam_s * m * r4[3];
    // 2.-3. Fletcher-Reeves directions and clamped updates; with restart, a
    // direction that is not a descent one, (g, -g + beta d) >= 0, becomes -g
    double beta_e = (it > 0 && gg_e_prev > 0) ? gg_e / gg_e_prev : 0.0;
    double beta_s = (it > 0 && gg_s_prev > 0) ? gg_s / gg_s_prev : 0.0;
    if (prm->restart && it > 0 && -gg_e + beta_e * m * r4[4] >= 0.0) beta_e = 0.0;
    if (prm->restart && it > 0 && -gg_s + beta_s * m * r4[5] >= 0.0) beta_s = 0.0;
    launch_cg_update(gte, gts, de, ds, beta_e, beta_s, alp_e, alp_s, eps, sig, eps_n, sig_n, prm->eps_max,
                     prm->sig_max, it == 0, n, part, out, sm, mass);
    double r6[6];
    BCK(cudaMemcpyAsync(r6, out, sizeof(r6), cudaMemcpyDeviceToHost, sm));
    BCK(cudaEventRecord(b->ev[1], sm));
    BCK(cudaEventSynchronize(b->ev[1]));
    float ms = 0.0f;
    BCK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    b->launches += 4 + (int64_t)b->m.size();
    // 4. step sizes, 5. regularisation schedule, 6. stopping rule
    const double gd_e = m * r6[0], dd_e = m * r6[1], gd_s = m * r6[3], dd_s = m * r6[4];
    const double step_e = std::sqrt(m * r6[2]), step_s = std::sqrt(m * r6[5]);
    const double alp_e_next = (gam_e > 0 && dd_e > 0) ? -gd_e / (gam_e * dd_e) : alp_e;
    const double alp_s_next = (gam_s > 0 && dd_s > 0) ? -gd_s / (gam_s * dd_s) : alp_s;
    const bool stop = (step_e < prm->eta1_eps || step_s < prm->eta1_sig) &&
                      (std::sqrt(gg_e) < prm->eta2_eps || std::sqrt(gg_s) < prm->eta2_sig);
    if (log) {
      ddfd_cg_iter &L = log[it];
      L.iter = it;
      L.stop = stop ? 1 : 0;
      L.J = J;
      L.J_data = J_data;
      L.gnorm_eps = std::sqrt(gg_e);
      L.gnorm_sig = std::sqrt(gg_s);
      L.alpha_eps = alp_e;
      L.alpha_sig = alp_s;
      L.beta_eps = beta_e;
      L.beta_sig = beta_s;
      L.gamma_eps = gam_e;
      L.gamma_sig = gam_s;
      L.step_eps = step_e;
      L.step_sig = step_s;
      L.ms = ms;
    }
    if (eps_it) BCK(cudaMemcpyAsync(eps_it + (size_t)it * n, eps_n, nb, cudaMemcpyDeviceToHost, sm));
    if (sig_it) BCK(cudaMemcpyAsync(sig_it + (size_t)it * n, sig_n, nb, cudaMemcpyDeviceToHost, sm));
    std::swap(eps, eps_n);
    std::swap(sig, sig_n);
    alp_e = alp_e_next;
    alp_s = alp_s_next;
    gam_e = prm->gamma_eps0 / std::pow((double)(it + 1), prm->p);
    gam_s = prm->gamma_sig0 / std::pow((double)(it + 1), prm->p);
    gg_e_prev = gg_e;
    gg_s_prev = gg_s;
    done = it + 1;
    if (stop) break;
  }
  BCK(cudaMemcpyAsync(eps_h, eps, nb, cudaMemcpyDeviceToHost, sm));
  BCK(cudaMemcpyAsync(sig_h, sig, nb, cudaMemcpyDeviceToHost, sm));
  BCK(cudaStreamSynchronize(sm));
  if (iters) *iters = done;
  return DDFD_OK;
}

void destroy_batch(ddfd_batch *b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (ddfd_problem *p : b->m) destroy_problem(p);
  for (void *v : b->allocs) cudaFree(v);
  for (int q = 0; q < 4; ++q)
    if (b->ev[q]) cudaEventDestroy(b->ev[q]);
  drop_batch_graphs(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // namespace

extern "C" {

int ddfd_autotune(ddfd_problem *p, int32_t steps, int32_t *tile_kz_out) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  if (steps < 1 || steps > p->Nt) return fail(p, DDFD_E_ARG, "steps must be in [1, n_steps]");
  int best = 0;
  int st = autotune_kz(
      p->n,
      [&](int kz, float *ms) { return p->fp32 ? single_trial<float>(p, steps, kz, ms) : single_trial<double>(p, steps, kz, ms); },
      &best);
  if (!st && (st = check_err(p))) best = 0;
  p->kz = best ? best : p->kz;
  p->state = ST_READY;
  drop_graphs(p);
  const size_t fbytes = 3 * (size_t)p->cs * p->esz;
  for (int q = 0; q < 2; ++q) {
    CK(cudaMemsetAsync(p->E[q], 0, fbytes, p->stream));
    if (p->Mu[q]) CK(cudaMemsetAsync(p->Mu[q], 0, fbytes, p->stream));
  }
  if (st) return st;
  if (tile_kz_out) *tile_kz_out = p->kz;
  return sync_check(p);
}

int ddfd_create_batch(const ddfd_config *cfgs, int32_t count, ddfd_batch **out) {
  g_create_err.clear();
  if (!cfgs || !out || count < 1 || count > 256) {
    g_create_err = "need 1..256 configurations and an output pointer";
    return DDFD_E_ARG;
  }
  int seg = 0;
  for (int i = 0; i < count; ++i) {
    const ddfd_config &c = cfgs[i];
    std::string m;
    int st = validate(&c, &m);
    if (st) {
      g_create_err = "member " + std::to_string(i) + ": " + m;
      return st;
    }
    if (c.grad_variant != DDFD_GRAD_EXACT) {
      g_create_err = "member " + std::to_string(i) + ": batches compute the exact gradient only";
      return DDFD_E_ARG;
    }
    if (c.n != cfgs[0].n || c.n_steps != cfgs[0].n_steps || c.cfl != cfgs[0].cfl ||
        c.precision != cfgs[0].precision) {
      g_create_err = "member " + std::to_string(i) + ": n, n_steps, cfl and precision must match member 0";
      return DDFD_E_ARG;
    }
    if (c.n_src != 1) {
      g_create_err = "member " + std::to_string(i) + ": batch members take one source";
      return DDFD_E_ARG;
    }
    if (c.n_snapshots > 0) {
      const int sg = (c.n_steps + c.n_snapshots - 1) / c.n_snapshots;
      if (seg && sg != seg) {
        g_create_err = "member " + std::to_string(i) + ": checkpointing members must share the segment length";
        return DDFD_E_ARG;
      }
      seg = sg;
    }
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_create_err = std::string("no usable CUDA device: ") + cudaGetErrorString(ce);
    return DDFD_E_CUDA;
  }
  ddfd_batch *b = new ddfd_batch();
  b->n = cfgs[0].n;
  b->Nt = cfgs[0].n_steps;
  b->px = (b->n + 7) / 8 * 8;
  b->cs = (long long)b->px * b->n * b->n;
  b->fp32 = cfgs[0].precision == DDFD_FP32;
  b->esz = b->fp32 ? 4 : 8;
  b->seg = seg;
  b->stream = (cudaStream_t)cfgs[0].stream;
  b->kz = cfgs[0].tile_kz ? cfgs[0].tile_kz : (b->n >= 128 ? 16 : 8);
  auto bail = [&](int code, const std::string &m) {
    g_create_err = m;
    destroy_batch(b);
    return code;
  };
  for (int q = 0; q < 4; ++q)
    if (cudaEventCreate(&b->ev[q]) != cudaSuccess) return bail(DDFD_E_CUDA, "cudaEventCreate failed");
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(DDFD_E_CUDA, "stream creation failed");
  const size_t slab = 3 * (size_t)b->cs * b->esz * count;
  bool all_fonly = true;
  for (int i = 0; i < count; ++i) all_fonly &= cfgs[i].forward_only != 0;
  void **bufs[5] = {&b->E[0], &b->E[1], &b->kcoef, &b->Mu[0], &b->Mu[1]};
  for (void **v : bufs) {
    if (all_fonly && (v == &b->Mu[0] || v == &b->Mu[1])) continue;  // no adjoint fields
    if (cudaMalloc(v, slab) != cudaSuccess) {
      cudaGetLastError();
      *v = nullptr;
      return bail(DDFD_E_OOM, "cudaMalloc of a " + std::to_string(slab) + "-byte field slab failed");
    }
    b->allocs.push_back(*v);
    b->bytes += (int64_t)slab;
  }
  if (cudaMalloc((void **)&b->errflag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return bail(DDFD_E_OOM, "cudaMalloc of the error flag failed");
  }
  b->allocs.push_back(b->errflag);
  if (cudaMemset(b->errflag, 0, sizeof(int)) != cudaSuccess) return bail(DDFD_E_CUDA, "memset failed");
  std::string m;
  if (encode_field_maps(&m, &b->maps, b->E, b->Mu, b->kcoef, b->n, b->px, b->fp32, count))
    return bail(DDFD_E_CUDA, m);
  const size_t fb = 3 * (size_t)b->cs * b->esz;
  for (int i = 0; i < count; ++i) {
    ddfd_config c = cfgs[i];
    c.stream = cfgs[0].stream;
    c.tile_kz = b->kz;
    MemberSlot ms;
    for (int q = 0; q < 2; ++q) {
      ms.E[q] = (char *)b->E[q] + i * fb;
      ms.Mu[q] = b->Mu[q] ? (char *)b->Mu[q] + i * fb : nullptr;
    }
    ms.kcoef = (char *)b->kcoef + i * fb;
    ms.batch = b;
    ms.slot = i;
    ddfd_problem *p = nullptr;
    const int st = create_impl(&c, &ms, &p);
    if (st) return bail(st, "member " + std::to_string(i) + ": " + g_create_err);
    b->m.push_back(p);
  }
  *out = b;
  return DDFD_OK;
}

void ddfd_destroy_batch(ddfd_batch *b) {
  if (b) destroy_batch(b);
}

const char *ddfd_batch_last_error(const ddfd_batch *b) { return b ? b->err.c_str() : "NULL handle"; }

int ddfd_batch_member(ddfd_batch *b, int32_t i, ddfd_problem **out) {
  if (!b || !out) return DDFD_E_ARG;
  b->err.clear();
  if (i < 0 || i >= (int)b->m.size()) return bfail(b, DDFD_E_ARG, "member index out of range");
  *out = b->m[i];
  return DDFD_OK;
}

int ddfd_batch_forward(ddfd_batch *b, double *const *trace_out) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  return batch_forward_impl(b, trace_out, cudaMemcpyDeviceToHost);
}

int ddfd_batch_forward_dev(ddfd_batch *b, double *const *trace_out) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  return batch_forward_impl(b, trace_out, cudaMemcpyDeviceToDevice);
}

int ddfd_batch_adjoint(ddfd_batch *b, const double *const *eobs) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  return batch_adjoint_impl(b, eobs, true);
}

int ddfd_batch_adjoint_dev(ddfd_batch *b, const double *const *eobs) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  return batch_adjoint_impl(b, eobs, false);
}

int ddfd_batch_autotune(ddfd_batch *b, int32_t steps, int32_t *tile_kz_out) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  if (steps < 1 || steps > b->Nt) return bfail(b, DDFD_E_ARG, "steps must be in [1, n_steps]");
  int best = 0;
  int st = autotune_kz(
      b->n,
      [&](int kz, float *ms) { return b->fp32 ? batch_trial<float>(b, steps, kz, ms) : batch_trial<double>(b, steps, kz, ms); },
      &best);
  if (!st && (st = batch_check_err(b))) best = 0;
  b->kz = best ? best : b->kz;
  drop_batch_graphs(b);
  for (ddfd_problem *p : b->m) {
    p->kz = b->kz;
    p->state = ST_READY;
    drop_graphs(p);
  }
  const size_t slab = 3 * (size_t)b->cs * b->esz * b->m.size();
  for (int q = 0; q < 2; ++q) {
    BCK(cudaMemsetAsync(b->E[q], 0, slab, b->stream));
    if (b->Mu[q]) BCK(cudaMemsetAsync(b->Mu[q], 0, slab, b->stream));
  }
  if (st) return st;
  if (tile_kz_out) *tile_kz_out = b->kz;
  BCK(cudaStreamSynchronize(b->stream));
  return DDFD_OK;
}

void ddfd_cg_params_default(ddfd_cg_params *prm) {
  if (!prm) return;
  std::memset(prm, 0, sizeof(*prm));
  prm->max_iter = 20;
  prm->gamma_eps0 = prm->gamma_sig0 = 1.0;
  prm->alpha_eps0 = prm->alpha_sig0 = 1.0;
  prm->p = 0.5;
  prm->eps_max = prm->sig_max = 100.0;
}

int ddfd_cg_run(ddfd_batch *b, const double *const *eobs, const ddfd_cg_params *prm, double *eps, double *sig,
                ddfd_cg_iter *log, int32_t *iters, double *eps_iters, double *sig_iters) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  return cg_run_impl(b, eobs, prm, eps, sig, log, iters, eps_iters, sig_iters);
}

int ddfd_batch_get_info(const ddfd_batch *b, ddfd_batch_info *info) {
  if (!b || !info) return DDFD_E_ARG;
  info->count = (int32_t)b->m.size();
  info->tile_kz = b->kz;
  info->forward_loop_ms = b->fwd_ms;
  info->adjoint_loop_ms = b->adj_ms;
  info->forward_step_kernels = b->fwd_kernels;
  info->adjoint_step_kernels = b->adj_kernels;
  int64_t l = b->launches, bytes = b->bytes;
  for (const ddfd_problem *p : b->m) {
    l += p->launches;
    bytes += p->bytes;
  }
  info->kernel_launches = l;
  info->device_bytes = bytes;
  return DDFD_OK;
}

}  // extern "C"
