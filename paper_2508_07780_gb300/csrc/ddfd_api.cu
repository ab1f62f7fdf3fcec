// Host driver of the ddfd C ABI (include/ddfd.h) for single problems:
// configuration checks, the call-order state machine, device memory, the
// incident-source setup, the TMA descriptors and the enqueueing of the step
// kernels into CUDA graphs.  All arithmetic of the method runs in the kernels
// of ddfd_step.cu and ddfd_aux.cu; the host only prepares per-step scalars
// (pulse value, absorbing-face set) and small tables.  Batches, the tile
// autotuner, explicit FEM meshes and the conjugate gradient loop have host
// units of their own (ddfd_batch.cu, ddfd_autotune.cu, ddfd_fem_setup.cu,
// ddfd_cg_host.cu).
#include "ddfd_host.h"

using namespace ddfd;
using namespace ddfd::host;

namespace {
thread_local std::string g_create_err;

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

namespace host {

const std::string &thread_error() { return g_create_err; }

int fail(ddfd_problem *p, int code, const std::string &m) {
  p->err = m;
  return code;
}

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
  p->alloc_bytes.push_back(bytes);
  p->bytes += (int64_t)bytes;
  return DDFD_OK;
}

void dfree(ddfd_problem *p, void *ptr) {
  for (size_t q = 0; q < p->allocs.size(); ++q)
    if (p->allocs[q] == ptr) {
      cudaFree(ptr);
      p->bytes -= (int64_t)p->alloc_bytes[q];
      p->allocs.erase(p->allocs.begin() + q);
      p->alloc_bytes.erase(p->alloc_bytes.begin() + q);
      return;
    }
}

std::vector<uint32_t> step_item_order(const std::vector<const ddfd_problem *> &ps, int kz, int kz_lean,
                                      int *n_full) {
  const int n = ps[0]->n;
  const bool f32 = ps[0]->fp32 != 0;
  const int gx = step_tiles_x(n, f32), gy = step_tiles_y(n, f32);
  const int ty_rows = f32 ? StepTile<float>::TY : StepTile<double>::TY;
  // A slab is one problem's z range [z0, z1) over a set of its tile columns:
  // the items of a slab are dispatched together, so that tiles that share
  // halos run side by side.
  struct Slab {
    long long cost;
    int q, z0, z1;
    bool fem;  // FP32: the columns that meet the FEM cube or the free box
  };
  auto ov = [](int lo, int hi, int first, int last) {  // nodes of [lo, hi) inside [first, last]
    return (long long)std::max(0, std::min(hi, last + 1) - std::max(lo, first));
  };
  // does tile column (tx, ty) meet [lo, hi]^2 in x and y (the x tail column
  // n - 1 is never a FEM or free node)
  auto meets = [&](int tx, int ty, int lo, int hi) {
    const int x0 = tx * STEP_TX, y0 = ty * ty_rows;
    return lo <= hi && x0 <= hi && x0 + STEP_TX - 1 >= lo && y0 <= hi && y0 + ty_rows - 1 >= lo;
  };
  std::vector<Slab> full, lean;
  std::vector<std::vector<char>> colfem(ps.size());
  for (size_t q = 0; q < ps.size(); ++q) {
    const ddfd_problem *p = ps[q];
    const long long fem2 = (long long)(p->b - p->a - 1) * (p->b - p->a - 1), fre2 = (long long)p->nf * p->nf;
    auto cost = [&](int z0, int z1) {
      return (long long)n * n * (z1 - z0) + 2 * fem2 * ov(z0, z1, p->a + 1, p->b - 1) +
             fre2 * ov(z0, z1, p->f0, p->f0 + p->nf - 1);
    };
    colfem[q].assign((size_t)gx * gy, 0);
    // FP32: the z range [zf0, zf1) of the FEM columns that holds FEM-cube or
    // free nodes (the hull of the two boxes' z ranges)
    int zf0 = n, zf1 = 0;
    if (f32) {
      for (int ty = 0; ty < gy; ++ty)
        for (int tx = 0; tx < gx; ++tx) {
          const bool c1 = meets(tx, ty, p->a + 1, p->b - 1), c2 = p->nf > 0 && meets(tx, ty, p->f0, p->f0 + p->nf - 1);
          colfem[q][(size_t)tx + (size_t)gx * ty] = c1 || c2;
          if (c1) zf0 = std::min(zf0, p->a + 1), zf1 = std::max(zf1, p->b);
          if (c2) zf0 = std::min(zf0, p->f0), zf1 = std::max(zf1, p->f0 + p->nf);
        }
    }
    if (zf0 >= zf1) {  // FP64, or no FEM columns: every column in chunks of kz on the full kernel
      for (int z0 = 0; z0 < n; z0 += kz) full.push_back({cost(z0, std::min(z0 + kz, n)), (int)q, z0, std::min(z0 + kz, n), false});
      continue;
    }
    // FEM columns: [zf0, zf1) in chunks of kz on the full kernel; the rest of
    // them and every other column on the lean one (below)
    for (int z0 = zf0; z0 < zf1; z0 += kz) full.push_back({cost(z0, std::min(z0 + kz, zf1)), (int)q, z0, std::min(z0 + kz, zf1), true});
    lean.push_back({0, (int)q, zf0, zf1, true});
  }
  auto heavy_first = [](const Slab &l, const Slab &r) { return l.cost > r.cost; };
  if (lean.empty()) {
    std::stable_sort(full.begin(), full.end(), heavy_first);
  } else {
    // problems by FEM work, heaviest first; both kernels take them in that order, z ascending
    std::vector<long long> pc(ps.size(), 0);
    for (const Slab &sl : full) pc[sl.q] += sl.cost;
    std::vector<int> rank(ps.size());
    std::vector<int> ord(ps.size());
    for (size_t q = 0; q < ps.size(); ++q) ord[q] = (int)q;
    std::stable_sort(ord.begin(), ord.end(), [&](int l, int r) { return pc[l] > pc[r]; });
    for (size_t i = 0; i < ord.size(); ++i) rank[ord[i]] = (int)i;
    auto by_problem = [&](const Slab &l, const Slab &r) {
      return rank[l.q] != rank[r.q] ? rank[l.q] < rank[r.q] : l.z0 < r.z0;
    };
    std::stable_sort(full.begin(), full.end(), by_problem);
    std::stable_sort(lean.begin(), lean.end(), by_problem);
  }
  std::vector<uint32_t> out;
  for (const Slab &sl : full)
    for (int ty = 0; ty < gy; ++ty)
      for (int tx = 0; tx < gx; ++tx) {
        // full slabs of FP64 / FEM-free problems hold every column, the others
        // only the FEM columns
        if (sl.fem && !colfem[sl.q][(size_t)tx + (size_t)gx * ty]) continue;
        out.push_back(pack_step_item(tx, ty, sl.z0, sl.z1 - sl.z0, sl.q));
      }
  *n_full = (int)out.size();
  // lean items: every node's work is the same, so they go by problem and z
  // chunk (chunks of kz_lean from z = 0), all the chunk's columns together,
  // which keeps the planes that neighbouring items share (x, y and z halos)
  // in L2 between their reads; a FEM column contributes the parts of the chunk
  // outside its full range [zf0, zf1)
  for (const Slab &sl : lean) {
    const int zf0 = sl.z0, zf1 = sl.z1;
    for (int z0 = 0; z0 < n; z0 += kz_lean) {
      const int z1 = std::min(z0 + kz_lean, n);
      for (int ty = 0; ty < gy; ++ty)
        for (int tx = 0; tx < gx; ++tx) {
          if (!colfem[sl.q][(size_t)tx + (size_t)gx * ty]) {
            out.push_back(pack_step_item(tx, ty, z0, z1 - z0, sl.q));
            continue;
          }
          if (z0 < zf0) out.push_back(pack_step_item(tx, ty, z0, std::min(z1, zf0) - z0, sl.q));
          if (z1 > zf1) {
            const int lo = std::max(z0, zf1);
            out.push_back(pack_step_item(tx, ty, lo, z1 - lo, sl.q));
          }
        }
    }
  }
  return out;
}

// Dispatch items fit the packing (n < 1024, z ranges of at most ITEM_MAX_NZ planes).
static bool items_fit(int n, int kz, int kz_lean) {
  return n <= 1024 && kz >= 1 && kz <= ITEM_MAX_NZ && kz_lean >= 1 && kz_lean <= ITEM_MAX_NZ;
}

int build_items(ddfd_problem *p) {
  if (p->items) {
    dfree(p, p->items);
    p->items = nullptr;
    p->items_kz = 0;
  }
  if (!items_fit(p->n, p->kz, p->kz_lean)) return DDFD_OK;  // beyond the item packing: grid order
  int n_full = 0;
  const std::vector<uint32_t> it = step_item_order({p}, p->kz, p->kz_lean, &n_full);
  int st = dalloc_t(p, it.size(), &p->items);
  if (st) return st;
  CK(cudaMemcpy(p->items, it.data(), it.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  p->items_kz = p->kz;
  p->n_items = (int)it.size();
  p->items_nfull = n_full;
  return DDFD_OK;
}

int enqueue_det_sources(ddfd_problem *p, cudaStream_t s) {
  if (!p->rsrc) return 0;
  launch_det_sources(p->res, p->Nt, p->n_det, p->n_src, p->n_unode, p->uptr, p->det_list, p->uij, p->n,
                     p->tau * p->tau, 1.0 / (p->h * p->h * p->h), p->rsrc, s);
  return 1;
}

int make_fork(StepFork *f) {
  if (cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    drop_fork(f);
    return DDFD_E_CUDA;
  }
  return DDFD_OK;
}

void drop_fork(StepFork *f) {
  if (f->ev_fork) cudaEventDestroy(f->ev_fork);
  if (f->ev_join) cudaEventDestroy(f->ev_join);
  if (f->side) cudaStreamDestroy(f->side);
  *f = StepFork();
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
  if (c->tile_kz_lean != 0 && (c->tile_kz_lean < 2 || c->tile_kz_lean > ITEM_MAX_NZ))
    return *m = "tile_kz_lean must be 0 or in [2, 64]", DDFD_E_ARG;
  if (c->src_dir)
    for (int s = 0; s < c->n_src; ++s) {
      const double *k = c->src_dir + 3 * s;
      const double nrm = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
      if (!(nrm > 0.0) || !(k[2] / nrm < -1e-6)) return *m = "source directions need k_z < 0", DDFD_E_ARG;
    }
  return DDFD_OK;
}

// Where adjoint step k sits in its block of GRAD_BLOCK steps (blocks end at
// k = 1, GRAD_BLOCK + 1, ...); k_first is the first step of the sequence.
int grad_mode(int k, int k_first) {
  const int phase = (k - 1) % GRAD_BLOCK;
  return ((k == k_first || phase == GRAD_BLOCK - 1) ? GM_FIRST : 0) | (phase == 0 ? GM_FOLD : 0);
}

}  // namespace host
}  // namespace ddfd

namespace {

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

int capture_slot(const ddfd_problem *p, int step) {
  for (size_t q = 0; q < p->cap_steps.size(); ++q)
    if (p->cap_steps[q] == step) return (int)q;
  return -1;
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
      *nk += launch_forward_step(single_launch(P, p->mE_halo[ic], p->mE_ctr[io], p), sm, &p->fork);
      enqueue_new_step<T>(p, p->X[ic], p->X[io], false, P, sm, nk);
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
          *nk += launch_forward_step(single_launch(F, p->mE_halo[fc], p->mE_ctr[fo], p), sm, &p->fork);
          std::swap(fc, fo);
        }
        hbase = (const T *)p->hist;
      } else {
        hbase = (const T *)p->hist + (size_t)s * (Nt + 1) * 3 * p->n_free;
      }
      for (int k = n1; k >= n0 + 1; --k) {
        set_adjoint_step(P, p, s, k, p->Mu[ic], p->Mu[io], hbase + (size_t)(k - n0) * 3 * p->n_free, Nt);
        enqueue_ebe<T>(p, p->Mu[ic], true, sm, nk, p->XMu[ic]);
        *nk += launch_adjoint_step(single_launch(P, p->mM_halo[ic], p->mM_ctr[io], p), sm, &p->fork);
        enqueue_new_step<T>(p, p->XMu[ic], p->XMu[io], true, P, sm, nk);
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

}  // namespace

namespace ddfd {
namespace host {

void drop_graphs(ddfd_problem *p) {
  if (p->gfwd) cudaGraphExecDestroy(p->gfwd);
  if (p->gadj) cudaGraphExecDestroy(p->gadj);
  p->gfwd = p->gadj = nullptr;
}

}  // namespace host
}  // namespace ddfd

namespace {

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

}  // namespace

namespace ddfd {
namespace host {

int sync_check(ddfd_problem *p) {
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return DDFD_OK;
}

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

}  // namespace host
}  // namespace ddfd

namespace {

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

}  // namespace

namespace ddfd {
namespace host {

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
  // default references eps0 = 1, sig0 = 0, filled on the device
  if (eps0) {
    CK(cudaMemcpyAsync(p->coef_stage + 2 * p->n_free, eps0, nfb, kind, p->stream));
  } else {
    launch_fill(p->coef_stage + 2 * p->n_free, p->n_free, 1.0, p->stream);
    ++p->launches;
  }
  if (sig0)
    CK(cudaMemcpyAsync(p->coef_stage + 3 * p->n_free, sig0, nfb, kind, p->stream));
  else
    CK(cudaMemsetAsync(p->coef_stage + 3 * p->n_free, 0, nfb, p->stream));
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
  p->launches += enqueue_det_sources(p, p->stream);
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

}  // namespace host
}  // namespace ddfd

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

int ddfd_create(const ddfd_config *cfg, ddfd_problem **out) { return create_impl(cfg, nullptr, out); }

void ddfd_destroy(ddfd_problem *p) {
  if (!p || p->batch) return;  // batch members go with their batch
  destroy_problem(p);
}

}  // extern "C"

namespace ddfd {
namespace host {

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
  p->kz_lean = cfg->tile_kz_lean ? cfg->tile_kz_lean : (p->n >= 128 ? 16 : 8);

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
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess || make_fork(&p->fork) ||
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
  // detector nodes: the distinct top nodes that carry detectors, in node order
  std::vector<int> dslot((size_t)p->n * p->n, -1), uptr(1, 0), uij;
  {
    std::vector<int> cnt((size_t)p->n * p->n, 0);
    for (int d = 0; d < p->n_det; ++d) cnt[p->det_ij[2 * d] + (size_t)p->n * p->det_ij[2 * d + 1]]++;
    for (int q = 0; q < p->n * p->n; ++q)
      if (cnt[q]) {
        dslot[q] = (int)uij.size() / 2;
        uij.push_back(q % p->n);
        uij.push_back(q / p->n);
        uptr.push_back(uptr.back() + cnt[q]);
      }
    p->n_unode = (int)uij.size() / 2;
  }
  if (p->fp32 && !p->fonly && p->n_unode > 0 &&
      ((st = dalloc_t(p, dslot.size(), &p->det_slot)) || (st = dalloc_t(p, uptr.size(), &p->uptr)) ||
       (st = dalloc_t(p, uij.size(), &p->uij)) ||
       (st = dalloc_t(p, (size_t)p->n_src * (p->Nt + 1) * p->n_unode * 3, &p->rsrc))))
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
      (p->det_slot && (h2d(p->det_slot, dslot.data(), dslot.size() * sizeof(int)) ||
                       h2d(p->uptr, uptr.data(), uptr.size() * sizeof(int)) ||
                       h2d(p->uij, uij.data(), uij.size() * sizeof(int)))) ||
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
  if ((st = build_maps(p)) || (st = build_items(p))) return bail(st);
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

void destroy_problem(ddfd_problem *p) {
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  for (void *v : p->allocs) cudaFree(v);
  for (int q = 0; q < 4; ++q)
    if (p->ev[q]) cudaEventDestroy(p->ev[q]);
  drop_graphs(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  drop_fork(&p->fork);
  delete p;
}

}  // namespace host
}  // namespace ddfd

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

int ddfd_time_gather(ddfd_problem *p, int32_t reps, double *fwd_ms, double *adj_ms, int64_t *fwd_bytes,
                     int64_t *adj_bytes) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  if (!p->ebe_rows) return fail(p, DDFD_E_ARG, "the handle has no element gather (fem_kind DDFD_FEM_EBE or DDFD_FEM_MESH)");
  if (reps < 1) return fail(p, DDFD_E_ARG, "reps must be >= 1");
  float ms[2] = {0.0f, 0.0f};
  for (int adj = 0; adj < 2; ++adj) {
    if (adj && !p->Mu[1]) break;  // forward_only: no adjoint fields
    int64_t nk = 0;
    const void *f = adj ? p->Mu[1] : p->E[1];
    const void *xf = adj ? p->XMu[1] : p->X[1];
    CK(cudaEventRecord(p->ev[0], p->stream));
    for (int r = 0; r < reps; ++r) {
      if (p->fp32)
        enqueue_ebe<float>(p, f, adj != 0, p->stream, &nk, xf);
      else
        enqueue_ebe<double>(p, f, adj != 0, p->stream, &nk, xf);
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->ev[1], p->stream));
    CK(cudaEventSynchronize(p->ev[1]));
    CK(cudaEventElapsedTime(&ms[adj], p->ev[0], p->ev[1]));
    p->launches += nk;
  }
  const int st = check_err(p);
  if (st) return st;
  if (fwd_ms) *fwd_ms = ms[0] / reps;
  if (adj_ms) *adj_ms = ms[1] / reps;
  if (fwd_bytes) *fwd_bytes = p->ebe_bytes_fwd;
  if (adj_bytes) *adj_bytes = p->ebe_bytes_adj;
  return DDFD_OK;
}

int ddfd_test_step_items(int32_t n, int32_t precision, int32_t nprob, const int32_t *boxes, int32_t kz,
                         int32_t kz_lean, uint32_t *items, int64_t cap, int64_t *n_items, int64_t *n_full) {
  if (n < 7 || n > 1024 || nprob < 1 || nprob > BATCH_MAX || !boxes || !n_items || !n_full || kz < 1 ||
      kz > ITEM_MAX_NZ || kz_lean < 1 || kz_lean > ITEM_MAX_NZ || cap < 0 || (cap > 0 && !items) ||
      (precision != DDFD_FP32 && precision != DDFD_FP64))
    return DDFD_E_ARG;
  std::vector<ddfd_problem> pv((size_t)nprob);
  std::vector<const ddfd_problem *> ps;
  for (int q = 0; q < nprob; ++q) {
    ddfd_problem &p = pv[(size_t)q];
    p.n = n;
    p.fp32 = precision == DDFD_FP32;
    p.a = boxes[4 * q];
    p.b = boxes[4 * q + 1];
    p.f0 = boxes[4 * q + 2];
    p.nf = boxes[4 * q + 3];
    if (p.a < 0 || p.b >= n || p.a > p.b || p.nf < 0 || (p.nf > 0 && (p.f0 < 0 || p.f0 + p.nf > n)))
      return DDFD_E_ARG;
    ps.push_back(&p);
  }
  int nf = 0;
  const std::vector<uint32_t> it = step_item_order(ps, kz, kz_lean, &nf);
  *n_items = (int64_t)it.size();
  *n_full = nf;
  if ((int64_t)it.size() > cap) return cap == 0 && !items ? DDFD_OK : DDFD_E_ARG;
  std::copy(it.begin(), it.end(), items);
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
