// Host driver of batched heterogeneous problems (ddfd_create_batch and the
// ddfd_batch_* calls of include/ddfd.h): members share the grid, step count
// and precision; their fields are stacked in one slab per level so that one
// step launch per group of BATCH_MAX members advances all of them, and the
// whole forward (adjoint) sequence is one CUDA graph.
#include "ddfd_host.h"

using namespace ddfd;
using namespace ddfd::host;

namespace ddfd {
namespace host {

int bfail(ddfd_batch *b, int code, const std::string &m) {
  b->err = m;
  return code;
}

std::vector<int> all_members(const ddfd_batch *b) {
  std::vector<int> v(b->m.size());
  for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
  return v;
}

int build_batch_items(ddfd_batch *b) {
  for (ItemTables *v : {&b->items_all, &b->items_ck}) {
    for (uint32_t *t : v->d) {
      cudaFree(t);
      b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), (void *)t));
    }
    *v = ItemTables();
  }
  b->items_kz = 0;
  if (b->n > 1024 || b->kz > ITEM_MAX_NZ || b->kz_lean > ITEM_MAX_NZ) return DDFD_OK;  // grid order
  std::vector<int> ck;
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i]->nsnap) ck.push_back((int)i);
  const std::vector<int> all = all_members(b);
  const std::pair<const std::vector<int> *, ItemTables *> lists[2] = {{&all, &b->items_all}, {&ck, &b->items_ck}};
  for (const auto &lt : lists)
    for (size_t g0 = 0; g0 < lt.first->size(); g0 += BATCH_MAX) {
      std::vector<const ddfd_problem *> ps;
      for (size_t g = g0; g < std::min(g0 + BATCH_MAX, lt.first->size()); ++g) ps.push_back(b->m[(*lt.first)[g]]);
      int n_full = 0;
      const std::vector<uint32_t> it = step_item_order(ps, b->kz, b->kz_lean, &n_full);
      uint32_t *d = nullptr;
      if (cudaMalloc((void **)&d, it.size() * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, DDFD_E_OOM, "cudaMalloc of a dispatch table failed");
      }
      b->allocs.push_back(d);
      lt.second->d.push_back(d);
      lt.second->n_items.push_back((int)it.size());
      lt.second->n_full.push_back(n_full);
      BCK(cudaMemcpy(d, it.data(), it.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
  b->items_kz = b->kz;
  return DDFD_OK;
}

}  // namespace host
}  // namespace ddfd

namespace {

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
    launch_groups<T>(b, false, all, b->maps.E_halo[ic], b->maps.E_ctr[io], fill, sm, nk, &b->items_all);
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
            sm, nk, &b->items_ck);
        std::swap(fc, fo);
      }
    }
    for (int k = n1; k >= n0 + 1; --k) {
      auto fill = [&](StepParams<T> &P, ddfd_problem *p) {
        const long long hk = p->nsnap ? k - n0 : k;
        set_adjoint_step(P, p, 0, k, p->Mu[ic], p->Mu[io], (const T *)p->hist + (size_t)hk * 3 * p->n_free, Nt);
      };
      for (ddfd_problem *p : b->m) enqueue_ebe<T>(p, p->Mu[ic], true, sm, nk, p->XMu[ic], b->errflag);
      launch_groups<T>(b, true, all, b->maps.M_halo[ic], b->maps.M_ctr[io], fill, sm, nk, &b->items_all);
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

}  // namespace

namespace ddfd {
namespace host {

void drop_batch_graphs(ddfd_batch *b) {
  if (b->gfwd) cudaGraphExecDestroy(b->gfwd);
  if (b->gadj) cudaGraphExecDestroy(b->gadj);
  b->gfwd = b->gadj = nullptr;
}

}  // namespace host
}  // namespace ddfd

namespace {

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

void destroy_batch(ddfd_batch *b);

}  // namespace

namespace ddfd {
namespace host {

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
    b->launches += enqueue_det_sources(p, b->stream);
  }
  for (ddfd_problem *p : b->m) p->state = ST_FORWARD;
  int st = run_batch_sequence(b, true);
  if (st) return st;
  if ((st = batch_check_err(b))) return st;
  BCK(cudaStreamSynchronize(b->stream));
  for (ddfd_problem *p : b->m) p->state = ST_ADJOINT;
  return DDFD_OK;
}

}  // namespace host
}  // namespace ddfd

namespace {

void destroy_batch(ddfd_batch *b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (ddfd_problem *p : b->m) destroy_problem(p);
  for (void *v : b->allocs) cudaFree(v);
  for (int q = 0; q < 4; ++q)
    if (b->ev[q]) cudaEventDestroy(b->ev[q]);
  drop_batch_graphs(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  drop_fork(&b->fork);
  delete b;
}

}  // namespace

extern "C" {

int ddfd_create_batch(const ddfd_config *cfgs, int32_t count, ddfd_batch **out) {
  ddfd::set_thread_error("");
  if (!cfgs || !out || count < 1 || count > 256) {
    ddfd::set_thread_error("need 1..256 configurations and an output pointer");
    return DDFD_E_ARG;
  }
  int seg = 0;
  for (int i = 0; i < count; ++i) {
    const ddfd_config &c = cfgs[i];
    std::string m;
    int st = validate(&c, &m);
    if (st) {
      ddfd::set_thread_error("member " + std::to_string(i) + ": " + m);
      return st;
    }
    if (c.grad_variant != DDFD_GRAD_EXACT) {
      ddfd::set_thread_error("member " + std::to_string(i) + ": batches compute the exact gradient only");
      return DDFD_E_ARG;
    }
    if (c.n != cfgs[0].n || c.n_steps != cfgs[0].n_steps || c.cfl != cfgs[0].cfl ||
        c.precision != cfgs[0].precision) {
      ddfd::set_thread_error("member " + std::to_string(i) + ": n, n_steps, cfl and precision must match member 0");
      return DDFD_E_ARG;
    }
    if (c.n_src != 1) {
      ddfd::set_thread_error("member " + std::to_string(i) + ": batch members take one source");
      return DDFD_E_ARG;
    }
    if (c.n_snapshots > 0) {
      const int sg = (c.n_steps + c.n_snapshots - 1) / c.n_snapshots;
      if (seg && sg != seg) {
        ddfd::set_thread_error("member " + std::to_string(i) + ": checkpointing members must share the segment length");
        return DDFD_E_ARG;
      }
      seg = sg;
    }
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    ddfd::set_thread_error(std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
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
  b->kz_lean = cfgs[0].tile_kz_lean ? cfgs[0].tile_kz_lean : (b->n >= 128 ? 16 : 8);
  auto bail = [&](int code, const std::string &m) {
    ddfd::set_thread_error(m);
    destroy_batch(b);
    return code;
  };
  for (int q = 0; q < 4; ++q)
    if (cudaEventCreate(&b->ev[q]) != cudaSuccess) return bail(DDFD_E_CUDA, "cudaEventCreate failed");
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess || make_fork(&b->fork))
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
    c.tile_kz_lean = b->kz_lean;
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
    if (st) return bail(st, "member " + std::to_string(i) + ": " + thread_error());
    b->m.push_back(p);
  }
  if (build_batch_items(b)) return bail(DDFD_E_OOM, b->err);
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

int ddfd_batch_get_info(const ddfd_batch *b, ddfd_batch_info *info) {
  if (!b || !info) return DDFD_E_ARG;
  info->count = (int32_t)b->m.size();
  info->tile_kz = b->kz;
  info->tile_kz_lean = b->kz_lean;
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
