// Small kernels of the ddfd library: coefficient preparation, detector
// gather, residual and functional reductions, gradient finalisation, the
// non-finite watchdog and the operator apply used by the stability check.
//
// Every reduction is a fixed two-pass tree (per-block partials, then one
// block), so results are bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <math.h>

#include "ddfd_internal.h"

namespace ddfd {

constexpr int RB = 256;  // reduction block size

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RB / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < RB / 32) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;  // valid in thread 0
}

template <typename T>
__global__ void k_gather_trace(const T *E, long long cs, int n_det, const int *det_node, double *tr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 3 * n_det) {
    const int d = t / 3, c = t - 3 * d;
    tr[t] = (double)E[c * cs + det_node[d]];
  }
}

void launch_gather_trace(const void *E, int fp32, long long cs, int n_det, const int *det_node,
                         double *trace_n, cudaStream_t s) {
  if (n_det <= 0) return;
  const int nb = (3 * n_det + 255) / 256;
  if (fp32)
    k_gather_trace<float><<<nb, 256, 0, s>>>((const float *)E, cs, n_det, det_node, trace_n);
  else
    k_gather_trace<double><<<nb, 256, 0, s>>>((const double *)E, cs, n_det, det_node, trace_n);
}

// Per free node of the padded full-grid coefficient field (FP64 arithmetic,
// one rounding to the field type):
//   channel 0: s  = eps - 1                  (Gauss-law weight, eq. forward_prob)
//   channel 1: q1 = (eps - c) / (eps + c)    c = sigma tau / 2
//   channel 2: q2 = 1 / (eps + c)
// so that the step update reads E^{n+1} = E^n + q1 (E^n - E^{n-1}) - q2 tau^2 R.
// Vacuum nodes hold s = 0, q1 = q2 = 1 (set once at creation).
template <typename T>
__global__ void k_expand(const double *coef, int nf, int f0, int n, int px, long long cs, double tau, T *out,
                         long long stride) {
  const long long n_free = (long long)nf * nf * nf;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n_free;
       f += (long long)gridDim.x * blockDim.x) {
    const int li = (int)(f % nf), lj = (int)((f / nf) % nf), lk = (int)(f / ((long long)nf * nf));
    const long long off = (f0 + li) + (long long)px * ((f0 + lj) + (long long)n * (f0 + lk));
    const double eps = coef[f], c = coef[stride + f] * tau * 0.5;
    out[off] = (T)(eps - 1.0);
    out[cs + off] = (T)((eps - c) / (eps + c));
    out[2 * cs + off] = (T)(1.0 / (eps + c));
  }
}

// Vacuum values s = 0, q1 = q2 = 1 over the whole padded field.
template <typename T>
__global__ void k_coef_vacuum(long long cs, T *out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cs;
       q += (long long)gridDim.x * blockDim.x) {
    out[q] = T(0);
    out[cs + q] = T(1);
    out[2 * cs + q] = T(1);
  }
}

void launch_coef_vacuum(int fp32, long long cs, void *coef, cudaStream_t s) {
  const long long nb = (cs + 255) / 256;
  const int blocks = (int)(nb < 8192 ? nb : 8192);
  if (fp32)
    k_coef_vacuum<float><<<blocks, 256, 0, s>>>(cs, (float *)coef);
  else
    k_coef_vacuum<double><<<blocks, 256, 0, s>>>(cs, (double *)coef);
}

void launch_expand_coeffs(int fp32, const double *coef_free, int nf, int f0, int n, int px,
                          long long cs, double tau, void *coef, cudaStream_t s, long long stride) {
  const long long nfree = (long long)nf * nf * nf;
  if (stride < 0) stride = nfree;
  const int blocks = (int)((nfree + 255) / 256 < 4096 ? (nfree + 255) / 256 : 4096);
  if (fp32)
    k_expand<float><<<blocks, 256, 0, s>>>(coef_free, nf, f0, n, px, cs, tau, (float *)coef, stride);
  else
    k_expand<double><<<blocks, 256, 0, s>>>(coef_free, nf, f0, n, px, cs, tau, (double *)coef, stride);
}

template <typename T>
__global__ void k_expand_new(const double *coef, long long stride, long long first, int n_new, double tau,
                             T *out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_new; e += gridDim.x * blockDim.x) {
    const double eps = coef[first + e], c = coef[stride + first + e] * tau * 0.5;
    out[e] = (T)(eps - 1.0);
    out[n_new + e] = (T)((eps - c) / (eps + c));
    out[2 * n_new + e] = (T)(1.0 / (eps + c));
  }
}

void launch_expand_new(int fp32, const double *coef_free, long long stride, long long first, int n_new,
                       double tau, void *xcoef, cudaStream_t s) {
  if (n_new <= 0) return;
  const int blocks = (n_new + 255) / 256 < 1024 ? (n_new + 255) / 256 : 1024;
  if (fp32)
    k_expand_new<float><<<blocks, 256, 0, s>>>(coef_free, stride, first, n_new, tau, (float *)xcoef);
  else
    k_expand_new<double><<<blocks, 256, 0, s>>>(coef_free, stride, first, n_new, tau, (double *)xcoef);
}

__global__ void k_fill(double *x, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

void launch_fill(double *x, long long n, double v, cudaStream_t s) {
  if (n <= 0) return;
  const long long want = (n + 255) / 256;
  k_fill<<<(int)(want < 1024 ? want : 1024), 256, 0, s>>>(x, n, v);
}

__global__ void k_check(const double *coef, int n_free, double eps_max, double sig_max, int *flag) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n_free; f += gridDim.x * blockDim.x) {
    const double e = coef[f], g = coef[n_free + f], e0 = coef[2 * n_free + f], g0 = coef[3 * n_free + f];
    const bool bad = !(e >= 1.0 && e <= eps_max) || !(g >= 0.0 && g <= sig_max) || !isfinite(e0) ||
                     !isfinite(g0);
    if (bad) atomicOr(flag, 1);
  }
}

void launch_check_coeffs(const double *coef_free, int n_free, double eps_max, double sig_max,
                         int *flag, cudaStream_t s) {
  const int blocks = (n_free + 255) / 256 < 1024 ? (n_free + 255) / 256 : 1024;
  k_check<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(coef_free, n_free, eps_max, sig_max, flag);
}

// trace/eobs/res: [n_src][n_steps+1][n_det][3]
__global__ void k_residual(const double *trace, const double *eobs, const double *z, int n_steps,
                           int n_det, long long total, double tau, double *res, double *part) {
  const long long per = (long long)(n_steps + 1) * n_det * 3;
  double acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long within = q % per;
    const int step = (int)(within / (3LL * n_det));
    double r = 0.0;
    if (step >= 1) {
      const double d = trace[q] - eobs[q];
      acc += z[step] * d * d;
      r = tau * z[step] * d;
    }
    res[q] = r;
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

void launch_residual(const double *trace, const double *eobs, const double *z, int n_steps,
                     int n_det, int n_src, double tau, double *res, double *part, int n_part,
                     cudaStream_t s) {
  const long long total = (long long)n_src * (n_steps + 1) * n_det * 3;
  k_residual<<<n_part, RB, 0, s>>>(trace, eobs, z, n_steps, n_det, total, tau, res, part);
}

__global__ void k_det_sources(const double *res, long long rows, int n_det, int n_unode, const int *uptr,
                              const int *ulist, const int *uij, int n, double tau2, double inv_h3, float *out) {
  const long long total = rows * n_unode;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long row = q / n_unode;  // (source, step)
    const int u = (int)(q - row * n_unode);
    const int i = uij[2 * u], j = uij[2 * u + 1];
    const double wx = (i == 0 || i == n - 1) ? 0.5 : 1.0;
    const double wy = (j == 0 || j == n - 1) ? 0.5 : 1.0;
    const double sc = tau2 * inv_h3 / (wx * wy * 0.5);
    const double *r = res + row * n_det * 3;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int qq = uptr[u]; qq < uptr[u + 1]; ++qq) {
      const int d = ulist[qq];
      acc[0] += r[3 * d + 0];
      acc[1] += r[3 * d + 1];
      acc[2] += r[3 * d + 2];
    }
    for (int c = 0; c < 3; ++c) out[3 * q + c] = (float)(sc * acc[c]);
  }
}

void launch_det_sources(const double *res, int n_steps, int n_det, int n_src, int n_unode, const int *uptr,
                        const int *ulist, const int *uij, int n, double tau2, double inv_h3, float *out,
                        cudaStream_t s) {
  const long long rows = (long long)n_src * (n_steps + 1);
  const long long total = rows * n_unode;
  if (total <= 0) return;
  const long long want = (total + 255) / 256;
  const int blocks = (int)(want < 4096 ? want : 4096);
  k_det_sources<<<blocks, 256, 0, s>>>(res, rows, n_det, n_unode, uptr, ulist, uij, n, tau2, inv_h3, out);
}

// sum_f (eps - eps0)^2 into part[0..n_part), sum_f (sig - sig0)^2 into part[n_part..2 n_part)
__global__ void k_regul(const double *coef, int n_free, double *part, int n_part, const double *mass) {
  double ae = 0.0, as = 0.0;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n_free; f += gridDim.x * blockDim.x) {
    const double de = coef[f] - coef[2 * n_free + f];
    const double ds = coef[n_free + f] - coef[3 * n_free + f];
    const double w = mass ? mass[f] : 1.0;
    ae += w * de * de;
    as += w * ds * ds;
  }
  const double be = block_sum(ae);
  const double bs = block_sum(as);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = be;
    part[n_part + blockIdx.x] = bs;
  }
}

void launch_regulariser(const double *coef_free, int n_free, double *part, int n_part, cudaStream_t s,
                        const double *mass) {
  k_regul<<<n_part, RB, 0, s>>>(coef_free, n_free, part, n_part, mass);
}

__global__ void k_sum(const double *part, int n_part, double *out) {
  double a = 0.0;
  for (int q = threadIdx.x; q < n_part; q += blockDim.x) a += part[q];
  const double b = block_sum(a);
  if (threadIdx.x == 0) *out = b;
}

void launch_sum(const double *part, int n_part, double *out, cudaStream_t s) {
  k_sum<<<1, RB, 0, s>>>(part, n_part, out);
}

// With mass (refined meshes), node f has lumped mass mass[f] and the scales
// are given per unit mass; without it, every free node has mass m.
__global__ void k_grad_final(const double *coef, int n_free, const double *ge, const double *gs,
                             double ge_scale, double gs_scale, double m, double gam_e, double gam_s,
                             double *g_eps, double *g_sig, const double *mass) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n_free; f += gridDim.x * blockDim.x) {
    if (mass) {
      const double mf = mass[f];
      g_eps[f] = gam_e * mf * (coef[f] - coef[2 * n_free + f]) + mf * ge_scale * ge[f];
      g_sig[f] = gam_s * mf * (coef[n_free + f] - coef[3 * n_free + f]) + mf * gs_scale * gs[f];
    } else {
      g_eps[f] = gam_e * m * (coef[f] - coef[2 * n_free + f]) + ge_scale * ge[f];
      g_sig[f] = gam_s * m * (coef[n_free + f] - coef[3 * n_free + f]) + gs_scale * gs[f];
    }
  }
}

void launch_grad_finalize(const double *coef_free, int n_free, const double *gacc_e,
                          const double *gacc_s, double ge_scale, double gs_scale, double m,
                          double gamma_e, double gamma_s, double *g_eps, double *g_sig,
                          cudaStream_t s, const double *mass) {
  const int blocks = (n_free + 255) / 256 < 2048 ? (n_free + 255) / 256 : 2048;
  k_grad_final<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(coef_free, n_free, gacc_e, gacc_s, ge_scale,
                                                       gs_scale, m, gamma_e, gamma_s, g_eps, g_sig, mass);
}

__global__ void k_nonfinite(const double *x, long long count, int *flag) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[q])) {
      atomicOr(flag, 2);
      return;
    }
}

void launch_nonfinite(const double *x, long long count, int *flag, cudaStream_t s) {
  if (count <= 0) return;
  const long long nb = (count + 255) / 256;
  k_nonfinite<<<(int)(nb < 2048 ? nb : 2048), 256, 0, s>>>(x, count, flag);
}

// partial sums of x^2 (two-pass, deterministic)
__global__ void k_norm2(const double *x, long long count, double *part) {
  double a = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x)
    a += x[q] * x[q];
  const double b = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

void launch_norm2(const double *x, long long count, double *part, int n_part, cudaStream_t s) {
  k_norm2<<<n_part, RB, 0, s>>>(x, count, part);
}

__global__ void k_scale(double *x, long long count, const double *norm2) {
  const double inv = 1.0 / sqrt(*norm2);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x)
    x[q] *= inv;
}

void launch_scale(double *x, long long count, const double *norm2, cudaStream_t s) {
  const long long nb = (count + 255) / 256;
  k_scale<<<(int)(nb < 4096 ? nb : 4096), 256, 0, s>>>(x, count, norm2);
}

}  // namespace ddfd
