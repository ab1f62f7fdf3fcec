// Element-by-element FEM apply on an explicit tetrahedral mesh of the FEM
// cube (fem_kind = DDFD_FEM_EBE and DDFD_FEM_MESH).
//
// For every node updated by FEM rows, the P1 stiffness of the stabilized
// operator is gathered element by element over the node's incident
// tetrahedra (a node-centric gather: each node owns its row, so no atomics
// and bitwise-reproducible sums):
//   forward:  (K E)_a   = sum_K |K| [ sum_b (g_a . g_b) E_b + g_a sum_b g_b . (s_b E_b) ]
//   adjoint:  (K^T mu)_a = sum_K |K| [ sum_b (g_a . g_b) mu_b ] + s_a (D^T D mu)_a,
//             (D^T D mu)_a = sum_K |K| g_a sum_b g_b . mu_b
// with g the P1 gradients (the Laplacian and the Gauss-law term of eq.
// forward_prob, weak form eq. lagrangian_weak).  Each tet carries
// sqrt|K| g_b (so products of two carry |K|).  The output is scaled to the
// step kernel's units, R = h^2 M^-1 (K E), and, in the adjoint, also
// q = h^2 M^-1 (D^T D mu) for the gradient.
//
// Staging: blocks of nearby rows (EbeBlock), double-buffered in shared
// memory by a persistent CTA per SM.  A block's tets arrive as one bulk copy
// and its nodes' values are gathered once into shared memory.  FP32 forward:
// one thread per tet forms the tet's terms of its four local rows, sum_b
// (g_a . g_b) E_b + g_a sum_b g_b . (s_b E_b), and writes them over the
// tet's gradients; each row then adds its incidences' three values (a row
// reads 3 values an incidence instead of 28).  FP64 and the adjoint: the tet
// divergences are formed once per tet, and each row sums its incident tets'
// terms from the gradients and node values.  Rows are summed by EBE_TPR
// threads, each taking every EBE_TPR-th incidence, combined in a fixed order.
// (A four-pass FP32 adjoint of the same kind -- divergences, q, Laplacian
// terms over the gradients, their sums -- measured slower, 352 against
// 339 us on 201^3, and is not used.)
#include <cuda_runtime.h>

#include "ddfd_internal.h"
#include "ddfd_tma.h"

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

// Vector loads from shared memory: 12 gradient values, 4 node values.
__device__ __forceinline__ void ld_grad(const float *g, float v[12]) {
  const float4 a = reinterpret_cast<const float4 *>(g)[0], b = reinterpret_cast<const float4 *>(g)[1],
               c = reinterpret_cast<const float4 *>(g)[2];
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y;
  v[6] = b.z, v[7] = b.w, v[8] = c.x, v[9] = c.y, v[10] = c.z, v[11] = c.w;
}
__device__ __forceinline__ void ld_grad(const double *g, double v[12]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double2 d = reinterpret_cast<const double2 *>(g)[i];
    v[2 * i] = d.x, v[2 * i + 1] = d.y;
  }
}
__device__ __forceinline__ void st_grad(float *g, const float v[12]) {
  float4 *p = reinterpret_cast<float4 *>(g);
  p[0] = make_float4(v[0], v[1], v[2], v[3]);
  p[1] = make_float4(v[4], v[5], v[6], v[7]);
  p[2] = make_float4(v[8], v[9], v[10], v[11]);
}
__device__ __forceinline__ void st_grad(double *g, const double v[12]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) reinterpret_cast<double2 *>(g)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}
__device__ __forceinline__ void ld_node(const float *n, float v[4]) {
  const float4 a = *reinterpret_cast<const float4 *>(n);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void ld_node(const double *n, double v[4]) {
  const double2 a = reinterpret_cast<const double2 *>(n)[0], b = reinterpret_cast<const double2 *>(n)[1];
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// Starts the copies of block `bi` into stage buffer D: the blob by one bulk
// copy (thread 0, counted on bar), the node values by per-thread copies.
template <typename T, bool ADJ>
__device__ __forceinline__ EbeBlock ebe_issue(const EbeParams<T> &P, int bi, unsigned char *D, uint64_t *bar) {
  const EbeBlock N = P.blocks[bi];
  // (test hook: block 0's copy is never started, so its wait runs out)
  if (threadIdx.x == 0 && !(P.test_skip_copy && bi == 0)) {
    fence_proxy_async_smem();  // earlier reads of this buffer (ordered by the last barrier) come first
    mbar_expect_tx(bar, (uint32_t)N.bytes);
    bulk_load(D, P.blob + N.blob, (uint32_t)N.bytes, bar);
  }
  T *sN = reinterpret_cast<T *>(D + N.bytes);
  for (int i = threadIdx.x; i < N.nn; i += EBE_THREADS) {
    const int o = P.blk_nodes[N.node0 + i];
    const T *f0, *f1, *f2, *sv;
    if (o < P.cs) {
      f0 = P.field + o;
      f1 = P.field + P.cs + o;
      f2 = P.field + 2 * P.cs + o;
      sv = P.s + o;
    } else {
      const long long e = o - P.cs;
      f0 = P.xfield + e;
      f1 = P.xfield + P.n_new + e;
      f2 = P.xfield + 2LL * P.n_new + e;
      sv = P.xs + e;
    }
    if (sizeof(T) == 4) {
      cp_async4(sN + 4 * i + 0, f0);
      cp_async4(sN + 4 * i + 1, f1);
      cp_async4(sN + 4 * i + 2, f2);
      if (!ADJ) cp_async4(sN + 4 * i + 3, sv);
    } else {
      cp_async8(sN + 4 * i + 0, f0);
      cp_async8(sN + 4 * i + 1, f1);
      cp_async8(sN + 4 * i + 2, f2);
      if (!ADJ) cp_async8(sN + 4 * i + 3, sv);
    }
    if (ADJ) sN[4 * i + 3] = T(1);
  }
  cp_async_commit();
  return N;
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(EBE_THREADS, 1) k_ebe(const EbeParams<T> P) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ int s_ok;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);  // one mbarrier per stage
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t parity = 0u;  // bit s: the phase stage s waits for
  int st = 0;
  auto stage = [&](int q) { return sm + 128 + (size_t)q * P.stage_bytes; };
  int bi = blockIdx.x;
  EbeBlock B;
  if (bi < P.n_blocks) B = ebe_issue<T, ADJ>(P, bi, stage(0), &bar[0]);
  for (; bi < P.n_blocks; bi += gridDim.x) {
    cp_async_wait_all();
    if (tid == 0) s_ok = mbar_wait_bounded(bar + st, (parity >> st) & 1u, P.spin_limit) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
      // the copy still in flight is this stage's: wait for it (bounded) and stop
      if (tid == 0) {
        atomicOr(P.err, 8);
        mbar_wait_bounded(bar + st, (parity >> st) & 1u, P.spin_limit);
      }
      break;
    }
    parity ^= 1u << st;
    EbeBlock next = B;
    if (bi + (int)gridDim.x < P.n_blocks) next = ebe_issue<T, ADJ>(P, bi + gridDim.x, stage(st ^ 1), bar + (st ^ 1));

    unsigned char *S = stage(st);
    const T *sG = reinterpret_cast<const T *>(S);
    const uint2 *sT = reinterpret_cast<const uint2 *>(S + (size_t)B.nt * 12 * sizeof(T));  // 4 x uint16 per tet
    const uint16_t *sI = reinterpret_cast<const uint16_t *>(sT + B.nt);
    const T *sN = reinterpret_cast<const T *>(S + B.bytes);
    T *sD = reinterpret_cast<T *>(S + B.bytes + ((4 * B.nn * (int)sizeof(T) + 15) & ~15));
    if constexpr (!ADJ && sizeof(T) == 4) {
      // FP32 forward: each tet's terms of its four local rows, written over its
      // gradients: o_a = sum_b (g_a . g_b) E_b + g_a sum_b s_b (g_b . E_b)
      for (int t = tid; t < B.nt; t += EBE_THREADS) {
        T g[12];
        ld_grad(sG + 12 * t, g);
        const uint2 nd = sT[t];
        const int ids[4] = {(int)(nd.x & 0xFFFF), (int)(nd.x >> 16), (int)(nd.y & 0xFFFF), (int)(nd.y >> 16)};
        T v[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) ld_node(sN + 4 * ids[b], v[b]);
        T div = T(0);
#pragma unroll
        for (int b = 0; b < 4; ++b)
          div += v[b][3] * (g[3 * b + 0] * v[b][0] + g[3 * b + 1] * v[b][1] + g[3 * b + 2] * v[b][2]);
        T o[12];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T l0 = T(0), l1 = T(0), l2 = T(0);
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const T w = g[3 * a + 0] * g[3 * b + 0] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2];
            l0 += w * v[b][0];
            l1 += w * v[b][1];
            l2 += w * v[b][2];
          }
          o[3 * a + 0] = l0 + g[3 * a + 0] * div;
          o[3 * a + 1] = l1 + g[3 * a + 1] * div;
          o[3 * a + 2] = l2 + g[3 * a + 2] * div;
        }
        st_grad(const_cast<T *>(sG) + 12 * t, o);
      }
      __syncthreads();
      const int lr = tid / EBE_TPR, j = tid % EBE_TPR;
      T y[3] = {T(0), T(0), T(0)};
      if (lr < B.nrows) {
        for (int e = j; e < B.maxinc; e += EBE_TPR) {
          const uint16_t code = sI[e * EBE_RB + lr];
          if (code == EBE_PAD) break;
          const T *o = sG + 12 * (code >> 2) + 3 * (code & 3);
          y[0] += o[0];
          y[1] += o[1];
          y[2] += o[2];
        }
      }
#pragma unroll
      for (int m = 1; m < EBE_TPR; m <<= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) y[c] += __shfl_xor_sync(0xffffffffu, y[c], m);
      }
      if (j == 0 && lr < B.nrows) {
        const int r = P.blk_rows[B.row0 + lr];
        const T sc = (T)P.scale[r];  // h^2 / m_a
#pragma unroll
        for (int c = 0; c < 3; ++c) P.out_r[c * (long long)P.n_rows + r] = sc * y[c];
      }
      // the next block's copy writes into the other stage; this stage's
      // gradients were overwritten, and its next copy comes after the
      // barrier at the top of the loop
      st ^= 1;
      B = next;
      continue;
    } else {
    // FP64, and the adjoint: per tet sum_b s_b (g_b . E_b) (forward) or
    // sum_b g_b . mu_b (adjoint); each row then sums its incidences' terms
    for (int t = tid; t < B.nt; t += EBE_THREADS) {
      T g[12];
      ld_grad(sG + 12 * t, g);
      const uint2 nd = sT[t];
      const int ids[4] = {(int)(nd.x & 0xFFFF), (int)(nd.x >> 16), (int)(nd.y & 0xFFFF), (int)(nd.y >> 16)};
      T div = T(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        T v[4];
        ld_node(sN + 4 * ids[b], v);
        div += v[3] * (g[3 * b + 0] * v[0] + g[3 * b + 1] * v[1] + g[3 * b + 2] * v[2]);
      }
      sD[t] = div;
    }
    __syncthreads();
    // rows: thread j of a row sums its incidences j, j + EBE_TPR, ... (in T:
    // at most a few terms each, as the stencil rows do)
    const int lr = tid / EBE_TPR, j = tid % EBE_TPR;
    T y[3] = {T(0), T(0), T(0)}, q[3] = {T(0), T(0), T(0)};
    if (lr < B.nrows) {
      for (int e = j; e < B.maxinc; e += EBE_TPR) {
        const uint16_t code = sI[e * EBE_RB + lr];
        if (code == EBE_PAD) break;
        const int t = code >> 2, a = code & 3;
        T g[12];
        ld_grad(sG + 12 * t, g);
        const uint2 nd = sT[t];
        const int ids[4] = {(int)(nd.x & 0xFFFF), (int)(nd.x >> 16), (int)(nd.y & 0xFFFF), (int)(nd.y >> 16)};
        // g_a by selection (a dynamic index would put g in local memory)
        T ga0 = g[0], ga1 = g[1], ga2 = g[2];
#pragma unroll
        for (int b = 1; b < 4; ++b)
          if (a == b) ga0 = g[3 * b + 0], ga1 = g[3 * b + 1], ga2 = g[3 * b + 2];
        T lap0 = T(0), lap1 = T(0), lap2 = T(0);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          T v[4];
          ld_node(sN + 4 * ids[b], v);
          const T w = ga0 * g[3 * b + 0] + ga1 * g[3 * b + 1] + ga2 * g[3 * b + 2];
          lap0 += w * v[0];
          lap1 += w * v[1];
          lap2 += w * v[2];
        }
        const T div = sD[t];
        y[0] += lap0;
        y[1] += lap1;
        y[2] += lap2;
        q[0] += ga0 * div;
        q[1] += ga1 * div;
        q[2] += ga2 * div;
      }
    }
    // the row's partial sums, merged by a butterfly (a + b == b + a, so all
    // lanes of the row hold the same bits; the order is fixed: reproducible)
#pragma unroll
    for (int m = 1; m < EBE_TPR; m <<= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        y[c] += __shfl_xor_sync(0xffffffffu, y[c], m);
        q[c] += __shfl_xor_sync(0xffffffffu, q[c], m);
      }
    }
    if (j == 0 && lr < B.nrows) {
      const int r = P.blk_rows[B.row0 + lr];
      const T sc = (T)P.scale[r];  // h^2 / m_a
      const T sa = ADJ ? node_s(P, P.row_node[r]) : T(1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        P.out_r[c * (long long)P.n_rows + r] = sc * (y[c] + sa * q[c]);
        if (ADJ) P.out_q[c * (long long)P.n_rows + r] = sc * q[c];
      }
    }
    st ^= 1;
    B = next;
    }
  }
}

// Kuhn stencil rows of an explicit mesh: the same R (and q) as the gather,
// from the 15-point block stencil of the uniform Kuhn split, R = (6 v_i -
// sum of the 6 axis neighbours) + sum_o B_o w_{i+o} with w = s E (forward);
// adjoint R = (6 mu_i - ...) + s_i sum_o B_o mu_{i+o}, q = sum_o B_o mu_{i+o}.
template <typename T, bool ADJ>
__global__ void k_kuhn_rows(const KuhnRowParams<T> P) {
  const long long sx = 1, sy = P.px, sz = (long long)P.px * P.n;
  const long long off[7] = {sx, sy, sz, sx + sy, sx + sz, sy + sz, sx + sy + sz};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < P.n_list; q += gridDim.x * blockDim.x) {
    const int r = P.list[q];
    const long long o = P.row_node[r];
    T lap[3], g[3] = {T(0), T(0), T(0)};
    const T s0 = P.s[o];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T *f = P.field + c * P.cs;
      lap[c] = T(6) * f[o] - (((((f[o + sx] + f[o - sx]) + f[o + sy]) + f[o - sy]) + f[o + sz]) + f[o - sz]);
    }
    {
      T w[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) w[d] = (ADJ ? T(1) : s0) * P.field[d * P.cs + o];
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] += P.B[0][3 * c] * w[0] + P.B[0][3 * c + 1] * w[1] + P.B[0][3 * c + 2] * w[2];
    }
#pragma unroll
    for (int b = 0; b < 7; ++b) {
      const long long up = o + off[b], dn = o - off[b];
      const T su = ADJ ? T(1) : P.s[up], sd = ADJ ? T(1) : P.s[dn];
      T w[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) w[d] = su * P.field[d * P.cs + up] + sd * P.field[d * P.cs + dn];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        g[c] += P.B[b + 1][3 * c] * w[0] + P.B[b + 1][3 * c + 1] * w[1] + P.B[b + 1][3 * c + 2] * w[2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P.out_r[c * (long long)P.n_rows + r] = lap[c] + (ADJ ? s0 : T(1)) * g[c];
      if (ADJ) P.out_q[c * (long long)P.n_rows + r] = g[c];
    }
  }
}

template <typename T>
void launch_kuhn_rows(const KuhnRowParams<T> &P, bool adj, cudaStream_t s) {
  if (P.n_list <= 0) return;
  const int blocks = (P.n_list + 255) / 256 < 4096 ? (P.n_list + 255) / 256 : 4096;
  if (adj)
    k_kuhn_rows<T, true><<<blocks, 256, 0, s>>>(P);
  else
    k_kuhn_rows<T, false><<<blocks, 256, 0, s>>>(P);
}

template void launch_kuhn_rows<float>(const KuhnRowParams<float> &, bool, cudaStream_t);
template void launch_kuhn_rows<double>(const KuhnRowParams<double> &, bool, cudaStream_t);

static int g_ebe_ctas = 0;  // one CTA per SM

template <typename T>
void launch_ebe(const EbeParams<T> &P, bool adj, cudaStream_t s) {
  if (P.n_blocks <= 0) return;
  const int ctas = g_ebe_ctas > 0 ? g_ebe_ctas : 1;
  const int grid = P.n_blocks < ctas ? P.n_blocks : ctas;
  const size_t smem = 128 + 2 * (size_t)P.stage_bytes;
  if (adj)
    k_ebe<T, true><<<grid, EBE_THREADS, smem, s>>>(P);
  else
    k_ebe<T, false><<<grid, EBE_THREADS, smem, s>>>(P);
}

template void launch_ebe<float>(const EbeParams<float> &, bool, cudaStream_t);
template void launch_ebe<double>(const EbeParams<double> &, bool, cudaStream_t);

cudaError_t prepare_ebe_kernels() {
  const int lim = 128 + 2 * EBE_SMEM_BUDGET;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaFuncSetAttribute(k_ebe<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_ebe<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_ebe<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_ebe<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)))
    return e;
  g_ebe_ctas = sms > 0 ? sms : 1;
  return cudaSuccess;
}

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
