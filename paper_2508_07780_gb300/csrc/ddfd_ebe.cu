// Element-by-element FEM apply on an explicit tetrahedral mesh of the FEM
// cube (fem_kind = DDFD_FEM_EBE).
//
// For every node updated by FEM rows, the P1 stiffness of the stabilized
// operator is gathered element by element over the node's incident
// tetrahedra (a node-centric gather: each node owns its row, so no atomics
// and bitwise-reproducible sums):
//   forward:  (K E)_a   = sum_K |K| [ sum_b (g_a . g_b) E_b + g_a sum_b g_b . (s_b E_b) ]
//   adjoint:  (K^T mu)_a = sum_K |K| [ sum_b (g_a . g_b) mu_b ] + s_a (D^T D mu)_a,
//             (D^T D mu)_a = sum_K |K| g_a sum_b g_b . mu_b
// with g the P1 gradients (the Laplacian and the Gauss-law term of eq.
// forward_prob, weak form eq. lagrangian_weak).  Each tet stores its four
// nodes' offsets in the padded field layout and sqrt|K| g_b (so products of
// two carry |K|).  The output is scaled to the step kernel's units,
// R = h^2 M^-1 (K E), and, in the adjoint, also q = h^2 M^-1 (D^T D mu) for the
// gradient.
#include <cuda_runtime.h>

#include "ddfd_internal.h"

namespace ddfd {

// Component c of the field at node offset nb (grid node, or new node nb - cs).
template <typename T>
__device__ __forceinline__ T node_field(const EbeParams<T> &P, int nb, int c) {
  return nb < P.cs ? P.field[c * P.cs + nb] : P.xfield[c * (long long)P.n_new + (nb - P.cs)];
}
template <typename T>
__device__ __forceinline__ T node_s(const EbeParams<T> &P, int nb) {
  return nb < P.cs ? P.s[nb] : P.xs[nb - P.cs];
}

template <typename T, bool ADJ>
__global__ void k_ebe(const EbeParams<T> P) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.n_rows; r += gridDim.x * blockDim.x) {
    const int i = P.row_node[r];  // padded offset of the row's node
    double y[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0};
    const int e0 = P.row_ptr[r], e1 = P.row_ptr[r + 1];
    for (int e = e0; e < e1; ++e) {
      const int t = P.inc_tet[e];
      const int a = P.inc_local[e];
      const int *nodes = P.tet_node + 4 * t;
      const T *g = P.tet_grad + 12 * t;  // sqrt|K| g_b, b = 0..3
      const T ga0 = g[3 * a + 0], ga1 = g[3 * a + 1], ga2 = g[3 * a + 2];
      T lap[3] = {T(0), T(0), T(0)}, div = T(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int nb = nodes[b];
        const T gb0 = g[3 * b + 0], gb1 = g[3 * b + 1], gb2 = g[3 * b + 2];
        const T w = ga0 * gb0 + ga1 * gb1 + ga2 * gb2;
        const T e0v = node_field(P, nb, 0), e1v = node_field(P, nb, 1), e2v = node_field(P, nb, 2);
        lap[0] += w * e0v;
        lap[1] += w * e1v;
        lap[2] += w * e2v;
        const T sb = ADJ ? T(1) : node_s(P, nb);
        div += sb * (gb0 * e0v + gb1 * e1v + gb2 * e2v);
      }
      y[0] += (double)lap[0];
      y[1] += (double)lap[1];
      y[2] += (double)lap[2];
      q[0] += (double)(ga0 * div);
      q[1] += (double)(ga1 * div);
      q[2] += (double)(ga2 * div);
    }
    const double sc = P.scale[r];  // h^2 / m_a
    const double sa = ADJ ? (double)node_s(P, i) : 1.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P.out_r[c * P.n_rows + r] = (T)(sc * (y[c] + sa * q[c]));
      if (ADJ) P.out_q[c * P.n_rows + r] = (T)(sc * q[c]);
    }
  }
}

template <typename T>
void launch_ebe(const EbeParams<T> &P, bool adj, cudaStream_t s) {
  const int blocks = (P.n_rows + 255) / 256 < 4096 ? (P.n_rows + 255) / 256 : 4096;
  if (adj)
    k_ebe<T, true><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(P);
  else
    k_ebe<T, false><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(P);
}

template void launch_ebe<float>(const EbeParams<float> &, bool, cudaStream_t);
template void launch_ebe<double>(const EbeParams<double> &, bool, cudaStream_t);

// New nodes of a refined mesh: the update of the step kernels for interior
// FEM rows, E^{n+1} = E^n + q1 (E^n - E^{n-1}) - q2 tau^2 R (R from k_ebe), the
// adjoint likewise with its transposed rows, and the free-node bookkeeping.
template <typename T, bool ADJ>
__global__ void k_new_step(const NewStepParams<T> P) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.n_new; e += gridDim.x * blockDim.x) {
    const long long row = P.row0 + e;
    const T q1 = P.xcoef[P.n_new + e], q2 = P.xcoef[2 * P.n_new + e];
    T nw[3], cen[3], od[3], sx[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cen[c] = P.cur[c * (long long)P.n_new + e];
      od[c] = P.old[c * (long long)P.n_new + e];
      const T R = P.r2 * P.ebe_r[c * (long long)P.ebe_rows + row];
      sx[c] = ADJ ? P.ebe_q[c * (long long)P.ebe_rows + row] : T(0);
      nw[c] = cen[c] + (q1 * (cen[c] - od[c]) - q2 * R);
      P.old[c * (long long)P.n_new + e] = nw[c];
    }
    const long long f = P.f0 + e;
    if (!ADJ) {
      if (P.hist_w)
#pragma unroll
        for (int c = 0; c < 3; ++c) P.hist_w[c * P.n_free + f] = nw[c];
    } else {
      T ge = T(0), gs = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T hv = P.hist_r[c * P.n_free + f];
        ge += hv * ((nw[c] - T(2) * cen[c] + od[c]) + P.r2 * sx[c]);
        gs += hv * (nw[c] - od[c]);
      }
      if (sizeof(T) == 4) {
        // FP32 block sums folded into the FP64 accumulators (as in the step kernel)
        float2 *gp = reinterpret_cast<float2 *>(P.gpart) + f;
        float a = (float)ge, b = (float)gs;
        if (!(P.gmode & GM_FIRST)) {
          const float2 prev = *gp;
          a = prev.x + a;
          b = prev.y + b;
        }
        if (P.gmode & GM_FOLD) {
          P.gacc_e[f] += (double)a;
          P.gacc_s[f] += (double)b;
        } else {
          *gp = make_float2(a, b);
        }
      } else {
        P.gacc_e[f] += (double)ge;
        P.gacc_s[f] += (double)gs;
      }
    }
  }
}

template <typename T>
void launch_new_step(const NewStepParams<T> &P, bool adj, cudaStream_t s) {
  if (P.n_new <= 0) return;
  const int blocks = (P.n_new + 255) / 256 < 4096 ? (P.n_new + 255) / 256 : 4096;
  if (adj)
    k_new_step<T, true><<<blocks, 256, 0, s>>>(P);
  else
    k_new_step<T, false><<<blocks, 256, 0, s>>>(P);
}

template void launch_new_step<float>(const NewStepParams<float> &, bool, cudaStream_t);
template void launch_new_step<double>(const NewStepParams<double> &, bool, cudaStream_t);

}  // namespace ddfd
