// Explicit step kernels of the hybrid FE/FD scheme (forward and adjoint).
//
// One thread owns a grid column (i, j) over kz consecutive planes and keeps
// the planes k-1, k, k+1 of its own column in registers; in-plane neighbours
// come through the read-only cache.  Per node and step:
//   FD part (every node): 7-point Laplacian with ghost-node (mirror) Neumann
//     closure, i.e. h^2 M^-1 L of the hexahedral FD scheme;
//   FEM part (nodes strictly inside the FEM cube): the P1 Gauss-law term of
//     eq. forward_prob / eq. model1 on the Kuhn mesh, as a 15-point block
//     stencil: forward h^2 M^-1 (D^T D S E)_i = sum_o B_o (s E)_{i+o},
//     adjoint h^2 M^-1 (S D^T D mu)_i = s_i sum_o B_o mu_{i+o};
//   boundary: damping tau/h per absorbing face (first-order absorbing
//     condition of eq. model1 with lumped surface mass), Neumann flux on the
//     top face during the source phase;
//   update in the divided, difference form (V = E^n - E^{n-1}, c = tau C/(2M)):
//     E^{n+1} = E^n + ((eps - c) V - tau^2 (M^-1 K E^n - f^n)) / (eps + c),
//   algebraically the central scheme M E'' + C E' + K E = F, written so that
//   FP32 storage does not cancel 2 E^n - E^{n-1};
//   adjoint: the transposed recursion of the same scheme with the damping of
//     steps k-1 and k+1, detector residuals j^k / m as sources, and the
//     gradient time sums (eq. gradeps, summation-by-parts form) accumulated in
//     FP64 at the free nodes.
#include <cuda_runtime.h>

#include "ddfd_internal.h"

namespace ddfd {

__constant__ double c_Bd[72];
__constant__ float c_Bf[72];

template <typename T>
__device__ __forceinline__ T Bk(int i);
template <>
__device__ __forceinline__ double Bk<double>(int i) { return c_Bd[i]; }
template <>
__device__ __forceinline__ float Bk<float>(int i) { return c_Bf[i]; }

cudaError_t upload_kuhn_blocks(const KuhnBlocks &kb, cudaStream_t s) {
  double d[72];
  float f[72];
  for (int o = 0; o < 8; ++o)
    for (int e = 0; e < 9; ++e) {
      d[o * 9 + e] = kb.B[o][e];
      f[o * 9 + e] = (float)kb.B[o][e];
    }
  cudaError_t err = cudaMemcpyToSymbolAsync(c_Bd, d, sizeof(d), 0, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return err;
  err = cudaMemcpyToSymbolAsync(c_Bf, f, sizeof(f), 0, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return err;
  return cudaStreamSynchronize(s);
}

constexpr int BX = 32;
constexpr int BY = 4;

__device__ __forceinline__ double pulse_value(int kind, double f, double t0, double w, double t) {
  if (kind == DDFD_SRC_GAUSS) {
    const double s = t - t0;
    const double q = s / w;
    return sin(2.0 * 3.141592653589793 * f * s) * exp(-q * q);
  }
  return (t > 0.0 && t < 1.0 / f) ? sin(2.0 * 3.141592653589793 * f * t) : 0.0;
}

// sum_o B_o v_{i+o} for one node, with B_{-o} = B_o; v given as the centre
// value and the 7 (+o, -o) neighbour pairs already summed.
template <typename T>
__device__ __forceinline__ void block_apply(const T v0[3], const T vp[7][3], T out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T acc = Bk<T>(c * 3 + 0) * v0[0] + Bk<T>(c * 3 + 1) * v0[1] + Bk<T>(c * 3 + 2) * v0[2];
#pragma unroll
    for (int p = 0; p < 7; ++p)
      acc += Bk<T>((p + 1) * 9 + c * 3 + 0) * vp[p][0] + Bk<T>((p + 1) * 9 + c * 3 + 1) * vp[p][1] +
             Bk<T>((p + 1) * 9 + c * 3 + 2) * vp[p][2];
    out[c] = acc;
  }
}

__device__ __forceinline__ int face_count_xy(int i, int j, int n, uint32_t abs) {
  int f = 0;
  if (i == 0 && (abs & DDFD_ABS_X0)) ++f;
  if (i == n - 1 && (abs & DDFD_ABS_X1)) ++f;
  if (j == 0 && (abs & DDFD_ABS_Y0)) ++f;
  if (j == n - 1 && (abs & DDFD_ABS_Y1)) ++f;
  return f;
}

__device__ __forceinline__ int face_count_z(int k, int n, uint32_t abs) {
  int f = 0;
  if (k == 0 && (abs & DDFD_ABS_BOTTOM)) ++f;
  if (k == n - 1 && (abs & DDFD_ABS_TOP)) ++f;
  return f;
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(BX *BY) k_step(const StepParams<T> P) {
  const int n = P.n;
  const long long cs = P.cs;
  if (!ADJ && P.n_det > 0) {  // detector sampling of E^n (read-only in this kernel)
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z * (BX * BY);
    long long t = ((long long)blockIdx.x + gridDim.x * ((long long)blockIdx.y + gridDim.y * blockIdx.z)) *
                      (BX * BY) +
                  threadIdx.x + BX * threadIdx.y;
    for (; t < 3LL * P.n_det; t += nb) {
      const int d = (int)(t / 3), c = (int)(t - 3LL * d);
      P.trace_n[t] = (double)P.cur[c * cs + P.det_node[d]];
    }
  }
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int k0 = blockIdx.z * P.kz;
  if (k0 >= n) return;
  const int k1 = min(k0 + P.kz, n);
  const int nn2 = n * n;
  const int ip = (i + 1 < n) ? i + 1 : n - 2, im = (i > 0) ? i - 1 : 1;
  const int jp = (j + 1 < n) ? j + 1 : n - 2, jm = (j > 0) ? j - 1 : 1;
  const int row = n * j;
  const bool colfem = (i > P.a && i < P.b && j > P.a && j < P.b);
  const bool colfree = (i >= P.f0 && i < P.f0 + P.nf && j >= P.f0 && j < P.f0 + P.nf);
  const int fxy_now = face_count_xy(i, j, n, P.abs_now);
  const int fxy_next = ADJ ? face_count_xy(i, j, n, P.abs_next) : 0;
  const int fb = P.fem_n;
  const T *__restrict__ cur = P.cur;
  T *__restrict__ old = P.old;

  T below[3], cen[3];
  {
    const int kb = (k0 > 0) ? k0 - 1 : 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      below[c] = __ldg(cur + c * cs + (long long)kb * nn2 + row + i);
      cen[c] = __ldg(cur + c * cs + (long long)k0 * nn2 + row + i);
    }
  }
  for (int k = k0; k < k1; ++k) {
    const int kp = (k + 1 < n) ? k + 1 : n - 2;
    const long long pb = (long long)k * nn2;
    const long long me = pb + row + i;
    T above[3], xp[3], xm[3], yp[3], ym[3], lap[3], st[3] = {T(0), T(0), T(0)}, sx[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T *pc = cur + c * cs + pb;
      above[c] = __ldg(cur + c * cs + (long long)kp * nn2 + row + i);
      xp[c] = __ldg(pc + row + ip);
      xm[c] = __ldg(pc + row + im);
      yp[c] = __ldg(pc + n * jp + i);
      ym[c] = __ldg(pc + n * jm + i);
      lap[c] = T(6) * cen[c] - (xp[c] + xm[c] + yp[c] + ym[c] + above[c] + below[c]);
    }
    T eps = T(1), cc, ccn = T(0);
    const bool fem = colfem && k > P.a && k < P.b;
    const bool fre = colfree && k >= P.f0 && k < P.f0 + P.nf;
    if (fem) {
      const long long bi = (i - P.a) + (long long)fb * ((j - P.a) + (long long)fb * (k - P.a));
      const T s0 = __ldg(P.s_box + bi);
      eps = T(1) + s0;
      cc = __ldg(P.c_box + bi);
      ccn = cc;
      // offsets of the 7 pairs in the grid and in the box
      const long long og[7] = {1, n, nn2, 1 + n, 1 + nn2, n + nn2, 1 + n + nn2};
      const long long ob[7] = {1, fb, (long long)fb * fb, 1 + fb, 1 + (long long)fb * fb,
                               fb + (long long)fb * fb, 1 + fb + (long long)fb * fb};
      T v0[3], vp[7][3];
      if (!ADJ) {
        // w = s E at the centre and the 14 neighbours
        T sp[7], sm[7];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
          sp[p] = __ldg(P.s_box + bi + ob[p]);
          sm[p] = __ldg(P.s_box + bi - ob[p]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T *pc = cur + c * cs;
          v0[c] = s0 * cen[c];
          vp[0][c] = sp[0] * xp[c] + sm[0] * xm[c];
          vp[1][c] = sp[1] * yp[c] + sm[1] * ym[c];
          vp[2][c] = sp[2] * above[c] + sm[2] * below[c];
#pragma unroll
          for (int p = 3; p < 7; ++p) vp[p][c] = sp[p] * __ldg(pc + me + og[p]) + sm[p] * __ldg(pc + me - og[p]);
        }
        block_apply<T>(v0, vp, st);
      } else if (fre) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T *pc = cur + c * cs;
          v0[c] = cen[c];
          vp[0][c] = xp[c] + xm[c];
          vp[1][c] = yp[c] + ym[c];
          vp[2][c] = above[c] + below[c];
#pragma unroll
          for (int p = 3; p < 7; ++p) vp[p][c] = __ldg(pc + me + og[p]) + __ldg(pc + me - og[p]);
        }
        block_apply<T>(v0, vp, sx);
#pragma unroll
        for (int c = 0; c < 3; ++c) st[c] = s0 * sx[c];
      }
    } else {
      cc = P.cb * T(fxy_now + face_count_z(k, n, P.abs_now));
      if (ADJ) ccn = P.cb * T(fxy_next + face_count_z(k, n, P.abs_next));
    }
    T R[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) R[c] = P.r2 * (lap[c] + st[c]);
    if (!ADJ && k == n - 1 && P.src_on) {
      if (!P.oblique) {
        R[1] -= P.src_y;
      } else {
        const double v = P.src_scale * pulse_value(P.pulse_kind, P.freq, P.t0, P.width,
                                                   P.t_n - P.delay[row + i]);
#pragma unroll
        for (int c = 0; c < 3; ++c) R[c] -= (T)(P.pol[c] * v);
      }
    }
    if (ADJ && k == n - 1 && P.n_det > 0) {
      const int q0 = P.det_ptr[row + i], q1 = P.det_ptr[row + i + 1];
      if (q1 > q0) {
        const double wx = (i == 0 || i == n - 1) ? 0.5 : 1.0;
        const double wy = (j == 0 || j == n - 1) ? 0.5 : 1.0;
        const double sc = P.tau2 * P.inv_h3 / (wx * wy * 0.5);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int q = q0; q < q1; ++q) {
          const int d = P.det_list[q];
          acc[0] += P.res_k[3 * d + 0];
          acc[1] += P.res_k[3 * d + 1];
          acc[2] += P.res_k[3 * d + 2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) R[c] += (T)(sc * acc[c]);
      }
    }
    T nw[3], od[3];
    if (!ADJ) {
      const T inv = T(1) / (eps + cc);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        od[c] = old[c * cs + me];
        nw[c] = cen[c] + ((eps - cc) * (cen[c] - od[c]) - R[c]) * inv;
        old[c * cs + me] = nw[c];
      }
      if (fre) {
        const long long fi = (i - P.f0) + (long long)P.nf * ((j - P.f0) + (long long)P.nf * (k - P.f0));
#pragma unroll
        for (int c = 0; c < 3; ++c) P.hist_w[c * P.n_free + fi] = nw[c];
      }
    } else {
      // cc: damping at step k-1, ccn: at step k+1
      const T inv = T(1) / (eps + cc);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        od[c] = old[c * cs + me];
        nw[c] = cen[c] + ((eps - ccn) * (cen[c] - od[c]) + (ccn - cc) * cen[c] - R[c]) * inv;
        old[c * cs + me] = nw[c];
      }
      if (fre) {
        const long long fi = (i - P.f0) + (long long)P.nf * ((j - P.f0) + (long long)P.nf * (k - P.f0));
        T ge = T(0), gs = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T e = __ldg(P.hist_r + c * P.n_free + fi);
          ge += e * ((nw[c] - T(2) * cen[c] + od[c]) + P.r2 * sx[c]);
          gs += e * (nw[c] - od[c]);
        }
        P.gacc_e[fi] += (double)ge;
        P.gacc_s[fi] += (double)gs;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      below[c] = cen[c];
      cen[c] = above[c];
    }
  }
}

template <typename T>
static dim3 step_grid(const StepParams<T> &P) {
  return dim3((P.n + BX - 1) / BX, (P.n + BY - 1) / BY, (P.n + P.kz - 1) / P.kz);
}

template <typename T>
void launch_forward_step(const StepParams<T> &P, cudaStream_t s) {
  k_step<T, false><<<step_grid(P), dim3(BX, BY), 0, s>>>(P);
}
template <typename T>
void launch_adjoint_step(const StepParams<T> &P, cudaStream_t s) {
  k_step<T, true><<<step_grid(P), dim3(BX, BY), 0, s>>>(P);
}

template void launch_forward_step<float>(const StepParams<float> &, cudaStream_t);
template void launch_forward_step<double>(const StepParams<double> &, cudaStream_t);
template void launch_adjoint_step<float>(const StepParams<float> &, cudaStream_t);
template void launch_adjoint_step<double>(const StepParams<double> &, cudaStream_t);

}  // namespace ddfd

namespace ddfd {

// y = h^2 M_eps^-1 K x in FP64 on every node (no damping, no source): the
// operator whose largest eigenvalue bounds the stable time step.  One thread
// per node; used only by the stability check.
template <typename T>
__global__ void k_apply_op(const double *x, double *y, int n, int a, int b, const T *s_box, int fb) {
  const long long nn = (long long)n * n * n;
  const long long nn2 = (long long)n * n;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nn;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % n), j = (int)((q / n) % n), k = (int)(q / nn2);
    const int ip = (i + 1 < n) ? i + 1 : n - 2, im = (i > 0) ? i - 1 : 1;
    const int jp = (j + 1 < n) ? j + 1 : n - 2, jm = (j > 0) ? j - 1 : 1;
    const int kp = (k + 1 < n) ? k + 1 : n - 2, km = (k > 0) ? k - 1 : 1;
    const long long pk = nn2 * k, rj = (long long)n * j;
    double out[3];
    for (int c = 0; c < 3; ++c) {
      const double *xc = x + c * nn;
      out[c] = 6.0 * xc[q] - xc[pk + rj + ip] - xc[pk + rj + im] - xc[pk + (long long)n * jp + i] -
               xc[pk + (long long)n * jm + i] - xc[nn2 * kp + rj + i] - xc[nn2 * km + rj + i];
    }
    double eps = 1.0;
    if (i > a && i < b && j > a && j < b && k > a && k < b) {
      const long long bi = (i - a) + (long long)fb * ((j - a) + (long long)fb * (k - a));
      const double s0 = (double)s_box[bi];
      eps = 1.0 + s0;
      const long long og[7] = {1, n, nn2, 1 + n, 1 + nn2, n + nn2, 1 + n + nn2};
      const long long ob[7] = {1, fb, (long long)fb * fb, 1 + fb, 1 + (long long)fb * fb,
                               fb + (long long)fb * fb, 1 + fb + (long long)fb * fb};
      double v0[3], vp[7][3], st[3];
      for (int c = 0; c < 3; ++c) v0[c] = s0 * x[c * nn + q];
      for (int p = 0; p < 7; ++p)
        for (int c = 0; c < 3; ++c)
          vp[p][c] = (double)s_box[bi + ob[p]] * x[c * nn + q + og[p]] +
                     (double)s_box[bi - ob[p]] * x[c * nn + q - og[p]];
      block_apply<double>(v0, vp, st);
      for (int c = 0; c < 3; ++c) out[c] += st[c];
    }
    for (int c = 0; c < 3; ++c) y[c * nn + q] = out[c] / eps;
  }
}

void launch_apply_op(const double *x, double *y, int n, int a, int b, const void *s_box, int fp32,
                     int fem_n, cudaStream_t s) {
  const long long nn = (long long)n * n * n;
  const long long nb = (nn + 255) / 256;
  const int blocks = (int)(nb < 8192 ? nb : 8192);
  if (fp32)
    k_apply_op<float><<<blocks, 256, 0, s>>>(x, y, n, a, b, (const float *)s_box, fem_n);
  else
    k_apply_op<double><<<blocks, 256, 0, s>>>(x, y, n, a, b, (const double *)s_box, fem_n);
}

}  // namespace ddfd
