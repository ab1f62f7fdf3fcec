// Host side of the conjugate gradient reconstruction (ddfd_cg_run): the CGA
// of Sec. 4 over a batch whose members are the incident waves of one model.
// Every vector operation runs in the kernels of ddfd_cg.cu; the host applies
// the scalar step rules in FP64.
#include "ddfd_host.h"

using namespace ddfd;
using namespace ddfd::host;

namespace {

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

}  // namespace

extern "C" {

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

}  // extern "C"
