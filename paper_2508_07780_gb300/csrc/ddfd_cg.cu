// Vector kernels of the conjugate gradient reconstruction (Sec. 4, CGA), all
// over the free nodes in FP64.  Each reduction kernel writes one partial sum
// per block and quantity; k_cg_sum adds them in a fixed order, so the
// scalars the host builds the step rules from are reproducible run to run.
#include <cuda_runtime.h>

#include "ddfd_internal.h"

namespace ddfd {

namespace {

constexpr int CG_THREADS = 256;

// Block sums of K per-thread values into part[q * gridDim.x + blockIdx.x].
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double *part) {
  __shared__ double sh[K][CG_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[q][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int j = 0; j < CG_THREADS / 32; ++j) s += sh[threadIdx.x][j];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_cg_accum(double *ge, double *gs, const double *te, const double *ts, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    ge[i] += te[i];
    gs[i] += ts[i];
  }
}

// g = G / m + gamma (x - x_ref) for eps and sigma; partial sums of g_e^2, g_s^2,
// (eps - ref)^2, (sig - ref)^2 and, when use_d, (g, d_prev) for eps and sigma.
// With mass (refined meshes) node i has lumped mass mass[i]: the
// representative divides by it and the sums carry it as their weight;
// without it every node has mass 1/inv_m and the host scales the sums.
__global__ void k_cg_grad(const double *Ge, const double *Gs, const double *eps, const double *sig,
                          const double *re, const double *rs, double inv_m, double gam_e, double gam_s,
                          double *gte, double *gts, const double *dpe, const double *dps, int use_d, long long n,
                          double *part, const double *mass) {
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = mass ? mass[i] : 1.0, im = mass ? 1.0 / mass[i] : inv_m;
    const double de = eps[i] - re[i], ds = sig[i] - rs[i];
    const double a = Ge[i] * im + gam_e * de;
    const double b = Gs[i] * im + gam_s * ds;
    gte[i] = a;
    gts[i] = b;
    v[0] += w * a * a;
    v[1] += w * b * b;
    v[2] += w * de * de;
    v[3] += w * ds * ds;
    if (use_d) {
      v[4] += w * a * dpe[i];
      v[5] += w * b * dps[i];
    }
  }
  block_partials<6>(v, part);
}

// d = -g + beta d (d = -g on the first iteration), x_new = clamp(x + alpha d);
// partial sums of (g, d), (d, d), (x_new - x)^2 for eps then sigma.
__global__ void k_cg_update(const double *gte, const double *gts, double *de, double *ds, double beta_e,
                            double beta_s, double alpha_e, double alpha_s, const double *eps, const double *sig,
                            double *eps_new, double *sig_new, double eps_max, double sig_max, int first,
                            long long n, double *part, const double *mass) {
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = mass ? mass[i] : 1.0;
    const double ge = gte[i], gs = gts[i];
    const double d1 = first ? -ge : -ge + beta_e * de[i];
    const double d2 = first ? -gs : -gs + beta_s * ds[i];
    de[i] = d1;
    ds[i] = d2;
    const double e1 = fmin(fmax(eps[i] + alpha_e * d1, 1.0), eps_max);
    const double s1 = fmin(fmax(sig[i] + alpha_s * d2, 0.0), sig_max);
    eps_new[i] = e1;
    sig_new[i] = s1;
    v[0] += w * ge * d1;
    v[1] += w * d1 * d1;
    v[2] += w * (e1 - eps[i]) * (e1 - eps[i]);
    v[3] += w * gs * d2;
    v[4] += w * d2 * d2;
    v[5] += w * (s1 - sig[i]) * (s1 - sig[i]);
  }
  block_partials<6>(v, part);
}

// out[q] = sum of part[q * nb .. q * nb + nb - 1], one warp per quantity, fixed order.
__global__ void k_cg_sum(const double *part, int nb, int k, double *out) {
  const int q = blockIdx.x;
  if (q >= k) return;
  double s = 0.0;
  for (int j = threadIdx.x; j < nb; j += 32) s += part[q * nb + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[q] = s;
}

}  // namespace

void launch_cg_accum(double *ge, double *gs, const double *te, const double *ts, long long n, cudaStream_t s) {
  k_cg_accum<<<CG_BLOCKS, CG_THREADS, 0, s>>>(ge, gs, te, ts, n);
}

void launch_cg_grad(const double *Ge, const double *Gs, const double *eps, const double *sig, const double *re,
                    const double *rs, double inv_m, double gam_e, double gam_s, double *gte, double *gts,
                    const double *dpe, const double *dps, int use_d, long long n, double *part, double *out,
                    cudaStream_t s, const double *mass) {
  k_cg_grad<<<CG_BLOCKS, CG_THREADS, 0, s>>>(Ge, Gs, eps, sig, re, rs, inv_m, gam_e, gam_s, gte, gts, dpe, dps,
                                             use_d, n, part, mass);
  k_cg_sum<<<6, 32, 0, s>>>(part, CG_BLOCKS, 6, out);
}

void launch_cg_update(const double *gte, const double *gts, double *de, double *ds, double beta_e, double beta_s,
                      double alpha_e, double alpha_s, const double *eps, const double *sig, double *eps_new,
                      double *sig_new, double eps_max, double sig_max, int first, long long n, double *part,
                      double *out, cudaStream_t s, const double *mass) {
  k_cg_update<<<CG_BLOCKS, CG_THREADS, 0, s>>>(gte, gts, de, ds, beta_e, beta_s, alpha_e, alpha_s, eps, sig,
                                               eps_new, sig_new, eps_max, sig_max, first, n, part, mass);
  k_cg_sum<<<6, 32, 0, s>>>(part, CG_BLOCKS, 6, out);
}

}  // namespace ddfd
