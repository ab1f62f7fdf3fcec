// Paper-literal gradient (grad_variant = DDFD_GRAD_LITERAL): eq. gradeps of
// Sec. 4 as printed, with the approximation div(eps_bar E) ~ eps_bar div E.
//
// The step kernels accumulate the exact derivative's Gauss-law term
// E^k_i . (D^T D mu^k)_i = sum_{K ni i} |K| (grad phi_i . E^k_i) (div mu^k)_K.
// The literal form spreads each element's divergence evenly over its four
// vertices instead: sum_{K ni i} |K|/4 (div E^k)_K (div mu^k)_K (lumped
// quadrature of int phi_i div E div mu; P1 divergences are constant per tet).
// k_grad_literal adds the difference of the two, per free node and adjoint
// step, to the FP64 eps accumulator; it needs E^k on the neighbours of the free
// nodes, which k_copy_fem_nodes keeps for every forward step.
//
// Kuhn split of the cube with corner o: for each permutation (p0, p1, p2) the
// tet o, o + e_p0, o + e_p0 + e_p1, o + (1,1,1), whose barycentric gradients
// are -e_p0, e_p0 - e_p1, e_p1 - e_p2, e_p2 (units 1/h), volume h^3 / 6.
#include <cuda_runtime.h>

#include "ddfd_internal.h"

namespace ddfd {

template <typename T>
__global__ void k_copy_fem_nodes(const T *__restrict__ E, T *__restrict__ dst, int n, int px, long long cs, int a,
                                 int fm) {
  const long long nfu = (long long)fm * fm * fm;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nfu; q += (long long)gridDim.x * blockDim.x) {
    const int x = a + 1 + (int)(q % fm), y = a + 1 + (int)((q / fm) % fm), z = a + 1 + (int)(q / ((long long)fm * fm));
    const long long o = x + (long long)px * (y + (long long)n * z);
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[c * nfu + q] = E[c * cs + o];
  }
}

template <typename T>
void launch_copy_fem_nodes(const T *E, T *dst, int n, int px, long long cs, int a, int b, cudaStream_t s) {
  const int fm = b - a - 1;
  const long long nfu = (long long)fm * fm * fm;
  const long long nb = (nfu + 255) / 256;
  k_copy_fem_nodes<T><<<(int)(nb < 4096 ? nb : 4096), 256, 0, s>>>(E, dst, n, px, cs, a, fm);
}

template <typename T>
__global__ void k_grad_literal(const T *__restrict__ Efem, const T *__restrict__ mu, double *__restrict__ gacc, int n,
                               int px, long long cs, int a, int fm, int nf, double r2) {
  const long long nfree = (long long)nf * nf * nf, nfu = (long long)fm * fm * fm;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nfree;
       f += (long long)gridDim.x * blockDim.x) {
    const int x = a + 2 + (int)(f % nf), y = a + 2 + (int)((f / nf) % nf), z = a + 2 + (int)(f / ((long long)nf * nf));
    T acc = T(0);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      // cube with corner o = node - r, r in {0,1}^3
      const int r0 = corner & 1, r1 = (corner >> 1) & 1, r2c = (corner >> 2) & 1;
      const int ox = x - r0, oy = y - r1, oz = z - r2c;
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        // permutation t of the axes: p0 = t / 2, then the other two in order (t even) or swapped
        const int p0 = t >> 1, q0 = (p0 == 0) ? 1 : 0, q1 = (p0 == 2) ? 1 : 2;
        const int p1 = (t & 1) ? q1 : q0, p2 = (t & 1) ? q0 : q1;
        // relative vertices of the path tet
        int w[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
        w[1][p0] = 1;
        w[2][p0] = 1;
        w[2][p1] = 1;
        int va = -1;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (w[j][0] == r0 && w[j][1] == r1 && w[j][2] == r2c) va = j;
        if (va < 0) continue;  // the node is not a vertex of this tet (decided at compile time)
        T Ev[4][3], Mv[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int X = ox + w[j][0], Y = oy + w[j][1], Z = oz + w[j][2];
          const long long qf = (X - a - 1) + (long long)fm * ((Y - a - 1) + (long long)fm * (Z - a - 1));
          const long long qm = X + (long long)px * (Y + (long long)n * Z);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Ev[j][c] = Efem[c * nfu + qf];
            Mv[j][c] = mu[c * cs + qm];
          }
        }
        const T dE = (Ev[1][p0] - Ev[0][p0]) + (Ev[2][p1] - Ev[1][p1]) + (Ev[3][p2] - Ev[2][p2]);
        const T dM = (Mv[1][p0] - Mv[0][p0]) + (Mv[2][p1] - Mv[1][p1]) + (Mv[3][p2] - Mv[2][p2]);
        T own;
        if (va == 0)
          own = -Ev[0][p0];
        else if (va == 1)
          own = Ev[1][p0] - Ev[1][p1];
        else if (va == 2)
          own = Ev[2][p1] - Ev[2][p2];
        else
          own = Ev[3][p2];
        acc += dM * (T(0.25) * dE - own);
      }
    }
    gacc[f] += (r2 / 6.0) * (double)acc;
  }
}

template <typename T>
void launch_grad_literal(const T *Efem, const T *mu, double *gacc, int n, int px, long long cs, int a, int b,
                         double r2, cudaStream_t s) {
  const int fm = b - a - 1, nf = b - a - 3;
  const long long nfree = (long long)nf * nf * nf;
  if (nfree <= 0) return;
  const long long nb = (nfree + 255) / 256;
  k_grad_literal<T><<<(int)(nb < 4096 ? nb : 4096), 256, 0, s>>>(Efem, mu, gacc, n, px, cs, a, fm, nf, r2);
}

template void launch_copy_fem_nodes<float>(const float *, float *, int, int, long long, int, int, cudaStream_t);
template void launch_copy_fem_nodes<double>(const double *, double *, int, int, long long, int, int, cudaStream_t);
template void launch_grad_literal<float>(const float *, const float *, double *, int, int, long long, int, int,
                                         double, cudaStream_t);
template void launch_grad_literal<double>(const double *, const double *, double *, int, int, long long, int, int,
                                          double, cudaStream_t);

}  // namespace ddfd
