// The tile autotuner (ddfd_autotune, ddfd_batch_autotune): times a few
// forward and adjoint step launches per candidate z depth of the thread-block
// tiles with CUDA events and keeps the fastest: first the full kernel's depth
// (the lean one's fixed), then, in FP32, the lean kernel's depth.  A GPU
// tuning aid; the paper has no counterpart.
#include "ddfd_host.h"

using namespace ddfd;
using namespace ddfd::host;

namespace {

const int kTileKz[] = {4, 6, 8, 12, 16, 24, 32};

// Runs trial(kz, kz_lean, &ms) for every candidate z depth of one kernel
// (after one untimed warm-up trial), the other's held, and returns the
// fastest in *kz (lean = false) or *kz_lean (lean = true).
template <typename Trial>
int autotune_one(int n, bool lean, Trial trial, int *kz, int *kz_lean) {
  int st;
  float ms = 0.0f;
  auto run = [&](int c) { return lean ? trial(*kz, c, &ms) : trial(c, *kz_lean, &ms); };
  if ((st = run(kTileKz[0] <= n ? kTileKz[0] : n))) return st;
  float best_ms = 3.4e38f;
  int best = lean ? *kz_lean : *kz;
  for (int c : kTileKz) {
    if (c > n) break;
    if ((st = run(c))) return st;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  (lean ? *kz_lean : *kz) = best;
  return DDFD_OK;
}

template <typename Trial>
int autotune_kz(int n, bool fp32, Trial trial, int *kz, int *kz_lean) {
  int st = autotune_one(n, false, trial, kz, kz_lean);
  if (!st && fp32) st = autotune_one(n, true, trial, kz, kz_lean);
  return st;
}

// E^n on the free nodes for trial step st (any valid slot of the history).
long long trial_hist_index(const ddfd_problem *p, int st) {
  return p->nsnap ? (long long)(st % p->seg) + 1 : (long long)st + 1;
}

template <typename T>
int single_trial(ddfd_problem *p, int steps, int kz, int kz_lean, float *ms) {
  const size_t fbytes = 3 * (size_t)p->cs * sizeof(T);
  const size_t trn = (size_t)p->n_src * (p->Nt + 1) * p->n_det * 3;
  cudaStream_t sm = p->stream;
  p->kz = kz;
  p->kz_lean = kz_lean;
  if (int bs = build_items(p)) return bs;  // the trial runs the dispatch order (and split) of these depths
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
    nk += launch_forward_step(single_launch(P, p->mE_halo[ic], p->mE_ctr[io], p), sm, &p->fork);
    std::swap(ic, io);
  }
  ic = 1, io = 0;
  for (int k = p->fonly ? 0 : steps; k >= 1; --k) {  // forward_only handles time the forward alone
    set_adjoint_step(P, p, 0, k, p->Mu[ic], p->Mu[io], (const T *)p->hist + trial_hist_index(p, k - 1) * 3 * p->n_free,
                     steps);
    enqueue_ebe<T>(p, p->Mu[ic], true, sm, &nk, p->XMu[ic]);
    nk += launch_adjoint_step(single_launch(P, p->mM_halo[ic], p->mM_ctr[io], p), sm, &p->fork);
    std::swap(ic, io);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(p->ev[1], sm));
  CK(cudaEventSynchronize(p->ev[1]));
  CK(cudaEventElapsedTime(ms, p->ev[0], p->ev[1]));
  p->launches += nk;
  return DDFD_OK;
}

template <typename T>
int batch_trial(ddfd_batch *b, int steps, int kz, int kz_lean, float *ms) {
  const size_t fbytes = 3 * (size_t)b->cs * sizeof(T);
  const size_t slab = fbytes * b->m.size();
  cudaStream_t sm = b->stream;
  b->kz = kz;
  b->kz_lean = kz_lean;
  if (int bs = build_batch_items(b)) return bs;  // the trial runs the dispatch orders of these depths
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
        sm, &nk, &b->items_all);
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
        sm, &nk, &b->items_all);
    std::swap(ic, io);
  }
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(b->ev[1], sm));
  BCK(cudaEventSynchronize(b->ev[1]));
  BCK(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
  b->launches += nk;
  return DDFD_OK;
}

}  // namespace

extern "C" {

int ddfd_autotune(ddfd_problem *p, int32_t steps, int32_t *tile_kz_out) {
  if (!p) return DDFD_E_ARG;
  p->err.clear();
  if (steps < 1 || steps > p->Nt) return fail(p, DDFD_E_ARG, "steps must be in [1, n_steps]");
  const int kz0 = p->kz, kzl0 = p->kz_lean;
  int kz = kz0, kzl = kzl0;
  int st = autotune_kz(
      p->n, p->fp32 != 0,
      [&](int a, int l, float *ms) {
        return p->fp32 ? single_trial<float>(p, steps, a, l, ms) : single_trial<double>(p, steps, a, l, ms);
      },
      &kz, &kzl);
  if (!st && (st = check_err(p))) kz = kz0, kzl = kzl0;
  p->kz = kz;
  p->kz_lean = kzl;
  p->state = ST_READY;
  drop_graphs(p);
  if (!st) st = build_items(p);
  const size_t fbytes = 3 * (size_t)p->cs * p->esz;
  for (int q = 0; q < 2; ++q) {
    CK(cudaMemsetAsync(p->E[q], 0, fbytes, p->stream));
    if (p->Mu[q]) CK(cudaMemsetAsync(p->Mu[q], 0, fbytes, p->stream));
  }
  if (st) return st;
  if (tile_kz_out) *tile_kz_out = p->kz;
  return sync_check(p);
}

int ddfd_batch_autotune(ddfd_batch *b, int32_t steps, int32_t *tile_kz_out) {
  if (!b) return DDFD_E_ARG;
  b->err.clear();
  if (steps < 1 || steps > b->Nt) return bfail(b, DDFD_E_ARG, "steps must be in [1, n_steps]");
  const int kz0 = b->kz, kzl0 = b->kz_lean;
  int kz = kz0, kzl = kzl0;
  int st = autotune_kz(
      b->n, b->fp32 != 0,
      [&](int a, int l, float *ms) {
        return b->fp32 ? batch_trial<float>(b, steps, a, l, ms) : batch_trial<double>(b, steps, a, l, ms);
      },
      &kz, &kzl);
  if (!st && (st = batch_check_err(b))) kz = kz0, kzl = kzl0;
  b->kz = kz;
  b->kz_lean = kzl;
  drop_batch_graphs(b);
  for (ddfd_problem *p : b->m) {
    p->kz = b->kz;
    p->kz_lean = b->kz_lean;
    p->state = ST_READY;
    drop_graphs(p);
    if (!st && (st = build_items(p))) b->err = p->err;
  }
  if (!st) st = build_batch_items(b);
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

}  // extern "C"
