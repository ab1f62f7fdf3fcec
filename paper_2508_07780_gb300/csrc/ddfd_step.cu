// Explicit step kernels of the hybrid FE/FD scheme (forward and adjoint).
//
// Work decomposition: one CTA owns an (x, y) tile and a range of consecutive
// z planes (a dispatch item, or a z chunk of the 3-D grid), which it marches
// through plane by plane.
//   - FP32 (k_step_pair): 32 x 16 tiles, 8 compute warps; each thread owns
//     two x-adjacent nodes, whose arithmetic runs in packed FP32 (one
//     instruction for both nodes); on a grid of n = 32 m + 1 nodes the last
//     tile also updates the column x = n - 1.  One step is two launches side
//     by side: the full kernel for the items that hold FEM-cube or free nodes
//     (2 CTAs per SM) and the lean kernel, without the block stencil, the
//     gradient or the coefficient stages, for the finite-difference items
//     (3 CTAs per SM).
//   - FP64 (k_step): 32 x 8 tiles, one node per thread, 8 compute warps and
//     a producer warp, every tile on one kernel.
// The planes of the current field (with a one-node halo in y and a
// 16-byte-aligned halo in x), the centre tile of the previous level, and (on
// tiles that touch the FEM cube) the coefficient planes are staged into
// shared memory by TMA tile loads through a ring of stages guarded by
// mbarriers, so that several planes are in flight per CTA while the previous
// ones are computed.  A launch may carry a dispatch order (StepLaunch::items):
// whole z slabs of tiles, heaviest first.
//
// Per node and step:
//   FD part (every node): 7-point Laplacian with ghost-node (mirror) Neumann
//     closure, i.e. h^2 M^-1 L of the hexahedral FD scheme;
//   FEM part (nodes strictly inside the FEM cube): the P1 Gauss-law term of
//     eq. forward_prob / eq. model1 on the Kuhn mesh as a 15-point block
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
//
// Field layout: component-major, x pitch px (a multiple of 8 elements, so
// TMA row strides are 16-byte multiples), offset i + px (j + n k).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>

#include "ddfd_internal.h"
#include "ddfd_tma.h"

namespace ddfd {

// The Kuhn P1 div-div blocks of an interior node in integer form: (D^T D)_{i,i+o}
// = (h/6) kb(o, .), B_{-o} = B_o = B_o^T, offsets 0, (1,0,0), (0,1,0), (0,0,1),
// (1,1,0), (1,0,1), (0,1,1), (1,1,1).  Compiled in so that zero and unit
// weights cost nothing; ddfd_create checks them against the blocks it
// assembles from the 24 Kuhn tetrahedra (csrc/ddfd_kuhn.cpp) and refuses to
// run if they differ.
__host__ __device__ constexpr int kb(int o, int e) {
  constexpr int t[8][9] = {
      {12, -4, -4, -4, 12, -4, -4, -4, 12},  // 0
      {-6, 2, 2, 2, 0, -1, 2, -1, 0},        // (1,0,0)
      {0, 2, -1, 2, -6, 2, -1, 2, 0},        // (0,1,0)
      {0, -1, 2, -1, 0, 2, 2, 2, -6},        // (0,0,1)
      {0, -2, 1, -2, 0, 1, 1, 1, 0},         // (1,1,0)
      {0, 1, -2, 1, 0, 1, -2, 1, 0},         // (1,0,1)
      {0, 1, 1, 1, 0, -2, 1, -2, 0},         // (0,1,1)
      {0, -1, -1, -1, 0, -1, -1, -1, 0}};    // (1,1,1)
  return t[o][e];
}

static int kb_int(int o, int e) { return kb(o, e); }

cudaError_t check_kuhn_blocks(const KuhnBlocks &kb, cudaStream_t) {
  for (int o = 0; o < 8; ++o)
    for (int e = 0; e < 9; ++e)
      if (std::fabs(kb.B[o][e] * 6.0 - kb_int(o, e)) > 1e-12)
        return cudaErrorInvalidValue;
  return cudaSuccess;
}

__device__ __forceinline__ double pulse_value(int kind, double f, double t0, double w, double t) {
  if (kind == DDFD_SRC_GAUSS) {
    const double s = t - t0;
    const double q = s / w;
    return sin(2.0 * 3.141592653589793 * f * s) * exp(-q * q);
  }
  return (t > 0.0 && t < 1.0 / f) ? sin(2.0 * 3.141592653589793 * f * t) : 0.0;
}

// sum_o B_o v_{i+o} for one node (B = kb / 6), with B_{-o} = B_o; v given as
// the centre value and the 7 (+o, -o) neighbour pairs already summed.
template <typename T>
__device__ __forceinline__ void block_apply(const T v0[3], const T vp[7][3], T out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T acc = T(kb(0, c * 3 + 0)) * v0[0] + T(kb(0, c * 3 + 1)) * v0[1] + T(kb(0, c * 3 + 2)) * v0[2];
#pragma unroll
    for (int p = 0; p < 7; ++p) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int w = kb(p + 1, c * 3 + d);
        if (w == 1)
          acc += vp[p][d];
        else if (w == -1)
          acc -= vp[p][d];
        else if (w != 0)
          acc += T(w) * vp[p][d];
      }
    }
    out[c] = acc * T(1.0 / 6.0);
  }
}

__device__ __forceinline__ int face_count(int i, int j, int k, int n, uint32_t abs) {
  int f = 0;
  if (i == 0 && (abs & DDFD_ABS_X0)) ++f;
  if (i == n - 1 && (abs & DDFD_ABS_X1)) ++f;
  if (j == 0 && (abs & DDFD_ABS_Y0)) ++f;
  if (j == n - 1 && (abs & DDFD_ABS_Y1)) ++f;
  if (k == 0 && (abs & DDFD_ABS_BOTTOM)) ++f;
  if (k == n - 1 && (abs & DDFD_ABS_TOP)) ++f;
  return f;
}

template <typename T>
struct Stage {
  static constexpr int TX = STEP_TX;
  static constexpr int TY = StepTile<T>::TY;       // tile rows
  static constexpr int RPT = TY / 8;               // rows per thread (256 threads = 32 x 8)
  static constexpr int HX = 16 / (int)sizeof(T);   // x halo: one 16-byte unit
  static constexpr int BXW = STEP_TX + 2 * HX;     // staged row length
  static constexpr int ROWS = TY + 2;
  static constexpr int TXY = STEP_TX * TY;
  static constexpr int up128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int E_BYTES = 3 * ROWS * BXW * (int)sizeof(T);  // current level, halo
  static constexpr int O_BYTES = 3 * TXY * (int)sizeof(T);         // previous level, centre
  static constexpr int S_BYTES = ROWS * BXW * (int)sizeof(T);      // s = eps - 1, halo
  static constexpr int Q_BYTES = 2 * TXY * (int)sizeof(T);         // (q1, q2), centre
  static constexpr int E_OFF = 0;
  static constexpr int O_OFF = up128(E_BYTES);
  static constexpr int S_OFF = O_OFF + up128(O_BYTES);
  static constexpr int Q_OFF = S_OFF + up128(S_BYTES);
  static constexpr int BYTES = Q_OFF + up128(Q_BYTES);
  // FP32: 6 stages (3 CTAs per SM); FP64: 4 stages (2 CTAs per SM)
  static constexpr int RING = sizeof(T) == 4 ? 6 : 4;
  static constexpr int SMEM = RING * BYTES + 2 * RING * 8 + 128;
};

// FP32 stage: 32 x 16 tile, each computing thread owns two x-adjacent nodes
// (so every staged row is read as float2 pairs); 5 stages.  Full kernel
// (tiles with FEM-cube or free nodes): the current and previous levels, s and
// (q1, q2), 2 CTAs per SM.  Lean kernel (finite-difference tiles only): the
// two levels alone, 74 KB, 3 CTAs per SM.
constexpr int round128(int b) { return (b + 127) / 128 * 128; }
template <bool LEAN>
struct PairStageT {
  static constexpr int TX = STEP_TX;
  static constexpr int TY = StepTile<float>::TY;
  static constexpr int HX = 4;                     // x halo: one 16-byte unit
  static constexpr int BXW = TX + 2 * HX;          // staged row length (40)
  static constexpr int ROWS = TY + 2;
  static constexpr int RE = ROWS * BXW;            // component stride of a staged plane
  static constexpr int TXY = TX * TY;
  static constexpr int E_BYTES = 3 * RE * 4;
  static constexpr int O_BYTES = 3 * TXY * 4;
  static constexpr int S_BYTES = LEAN ? 0 : RE * 4;
  static constexpr int Q_BYTES = LEAN ? 0 : 2 * TXY * 4;
  static constexpr int E_OFF = 0;
  static constexpr int O_OFF = round128(E_BYTES);
  static constexpr int S_OFF = O_OFF + round128(O_BYTES);
  static constexpr int Q_OFF = S_OFF + round128(S_BYTES);
  static constexpr int BYTES = Q_OFF + round128(Q_BYTES);
  static constexpr int RING = 5;
  // stages, full and empty barriers, release counters, two ints, alignment
  static constexpr int SMEM = RING * BYTES + 2 * RING * 8 + RING * 4 + 8 + 128;
};
using PairStage = PairStageT<false>;

// Warp roles: warps 0..7 compute, warp 8 stages planes.
constexpr int STEP_CONSUMERS = 256;
constexpr int STEP_THREADS = STEP_CONSUMERS + 32;

// Stages plane p = kk - (k0 - 1) of the chunk into slot p % RING and arms the
// slot's "full" barrier with the byte count: the current level (halo box;
// mirrored ghost planes at kk = -1 and kk = n), the previous level (centre
// box, computed planes only) and, on tiles touching the FEM cube, s (halo
// box, planes a..b) and (q1, q2) (centre box, computed planes a..b).
template <class S>
__device__ __forceinline__ void stage_plane(int p, const CUtensorMap *mcur, const CUtensorMap *mold,
                                            const CUtensorMap *ms, const CUtensorMap *mq, unsigned char *smem,
                                            uint64_t *bar, int x0, int y0, int k0, int k1, int n, bool tile_fem,
                                            int a, int b, int ch) {
  const int slot = p % S::RING;
  const int kk = k0 - 1 + p;
  const int ksrc = kk < 0 ? 1 : (kk >= n ? n - 2 : kk);  // mirror ghost planes
  unsigned char *st = smem + slot * S::BYTES;
  const bool interior = kk >= k0 && kk < k1;
  const bool coef = tile_fem && kk >= a && kk <= b;
  const bool qc = coef && interior;
  const uint32_t bytes = S::E_BYTES + (interior ? S::O_BYTES : 0) + (coef ? S::S_BYTES : 0) +
                         (qc ? S::Q_BYTES : 0);
  uint64_t *bb = &bar[slot];
  mbar_expect_tx(bb, bytes);
  tma_load_4d(st + S::E_OFF, mcur, x0 - S::HX, y0 - 1, ksrc, ch, bb);
  if (interior) tma_load_4d(st + S::O_OFF, mold, x0, y0, kk, ch, bb);
  if (coef) tma_load_4d(st + S::S_OFF, ms, x0 - S::HX, y0 - 1, kk, ch, bb);
  if (qc) tma_load_4d(st + S::Q_OFF, mq, x0, y0, kk, ch + 1, bb);
}

// Producer (one thread): stages plane p = kk - (k0 - 1) of the chunk into
// slot p % RING once the consumers have released the slot's previous plane
// (p - RING): the current level (halo box; mirrored ghost planes at kk = -1
// and kk = n), the previous level (centre box, computed planes only) and, on
// tiles touching the FEM cube, s (halo box, planes a..b) and (q1, q2)
// (centre box, computed planes a..b).  Every wait is bounded; on give-up it
// sets error bit 4 and still waits (bounded) for its issued copies.
template <class S>
__device__ __forceinline__ void produce_planes(const CUtensorMap *mcur, const CUtensorMap *mold,
                                               const CUtensorMap *ms, const CUtensorMap *mq,
                                               unsigned char *smem, uint64_t *bar, uint64_t *emp, int x0,
                                               int y0, int k0, int k1, int n, bool tile_fem, int a, int b,
                                               int ch, uint32_t spin, int *err) {
  const int nplanes = k1 - k0 + 2;
  int p = 0;
  bool ok = true;
  for (; p < nplanes; ++p) {
    const int slot = p % S::RING;
    // plane p reuses the slot of plane p - RING, whose release is completion
    // number p/RING - 1 of that slot's empty barrier
    if (p >= S::RING && !mbar_wait_bounded(&emp[slot], (uint32_t)((p / S::RING - 1) & 1), spin)) {
      ok = false;
      break;
    }
    stage_plane<S>(p, mcur, mold, ms, mq, smem, bar, x0, y0, k0, k1, n, tile_fem, a, b, ch);
  }
  if (!ok) atomicOr(err, 4);
  // every issued plane must land before the CTA can retire (bounded)
  const int first = p > S::RING ? p - S::RING : 0;
  for (int q = first; q < p; ++q)
    mbar_wait_bounded(&bar[q % S::RING], (uint32_t)((q / S::RING) & 1), spin);
}

// Tiles per axis of the launch grid (device side of step_tiles_x / _y).  x
// tiles of the FP32 step kernel: with n = 32 m + 1 the last column is updated
// by the last of m tiles (k_step_pair's x tail) instead of by a tile of its own.
__host__ __device__ constexpr int tiles_pair_x(int n) { return n % STEP_TX == 1 ? n / STEP_TX : (n + STEP_TX - 1) / STEP_TX; }
template <typename T>
__device__ __forceinline__ int step_tiles_dev_x(int n) {
  return sizeof(T) == 4 ? tiles_pair_x(n) : (n + STEP_TX - 1) / STEP_TX;
}
template <typename T>
__device__ __forceinline__ int step_tiles_dev_y(int n) {
  return (n + StepTile<T>::TY - 1) / StepTile<T>::TY;
}

// Tile of this CTA: (problem of the launch, tile x, tile y) and its planes
// [k0, k1), from the launch's dispatch order if it has one, else from the 3-D
// grid (z chunks of kz planes).
struct CtaTile {
  int prob, tx, ty, k0, k1;
};
template <typename LT>
__device__ __forceinline__ CtaTile cta_tile(const LT &L) {
  CtaTile t;
  if (L.items) {
    const uint32_t it = L.items[blockIdx.x];
    t.tx = (int)(it & 31u);
    t.ty = (int)((it >> 5) & 127u);
    t.k0 = (int)((it >> 12) & 1023u);
    t.k1 = t.k0 + (int)((it >> 22) & 63u) + 1;
    t.prob = (int)(it >> 28);
  } else {
    t.tx = (int)blockIdx.x;
    t.ty = (int)blockIdx.y;
    t.prob = (int)blockIdx.z / L.zchunks;
    const int zc = (int)blockIdx.z - t.prob * L.zchunks;
    const int kz = L.p[sizeof(L.p) == sizeof(L.p[0]) ? 0 : t.prob].kz;
    t.k0 = zc * kz;
    t.k1 = t.k0 + kz;
  }
  return t;
}

// Forward detector sampling of E^n (read-only in the step kernels): the CTAs
// that own the bottom planes (k0 = 0) of a tile column, one per column
// whatever the z chunking, share the 3 n_det values by the first 256 threads'
// index within the column grid.
template <typename T>
__device__ __forceinline__ void sample_detectors(const StepParams<T> &P, const CtaTile &ct, int tid) {
  if (P.n_det <= 0 || ct.k0 != 0 || tid >= STEP_CONSUMERS) return;
  const int n = P.n;
  const int gx = step_tiles_dev_x<T>(n), gy = step_tiles_dev_y<T>(n);
  const long long nb = (long long)gx * gy * STEP_CONSUMERS;
  for (long long t = ((long long)ct.tx + (long long)gx * ct.ty) * STEP_CONSUMERS + tid; t < 3LL * P.n_det; t += nb) {
    const int d = (int)(t / 3), c = (int)(t - 3LL * d);
    P.trace_n[t] = (double)P.cur[c * P.cs + P.det_node[d]];
  }
}

template <typename T, bool ADJ, int NB>
__global__ void __launch_bounds__(STEP_THREADS, sizeof(T) == 4 ? 3 : 2)
    k_step(const __grid_constant__ StepLaunch<T, NB> L) {
  using S = Stage<T>;
  // problem of this CTA (uniform), its tile and z chunk
  const CtaTile ct = cta_tile(L);
  const StepParams<T> &P = L.p[NB == 1 ? 0 : ct.prob];
  constexpr int RE = S::ROWS * S::BXW;  // component stride of a staged plane
  constexpr int BW = S::BXW;
  // 128-byte aligned stage base, computed in the shared window so that the
  // compiler keeps every stage access a shared-memory access
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t *bar = (uint64_t *)(smem + S::RING * S::BYTES);  // "full": plane landed
  uint64_t *emp = bar + S::RING;                             // "empty": consumers released it
  const int n = P.n;
  const int tid = threadIdx.x;

  if (!ADJ) sample_detectors(P, ct, tid);

  const int tx = tid & 31, ty = tid >> 5;
  // one CTA per (tile, z range): planes k0-1 .. k1 are staged, plane index
  // p = kk - (k0 - 1) in slot p % RING
  const int x0 = ct.tx * STEP_TX, y0 = ct.ty * S::TY;
  const int k0 = ct.k0;
  if (k0 >= n) return;  // uniform per CTA
  const int k1 = min(ct.k1, n);
  const bool tile_fem = x0 <= P.b - 1 && x0 + STEP_TX - 1 >= P.a + 1 && y0 <= P.b - 1 &&
                        y0 + S::TY - 1 >= P.a + 1;

  if (tid == 0) {
    for (int s = 0; s < S::RING; ++s) {
      mbar_init(&bar[s], 1);
      mbar_init(&emp[s], STEP_CONSUMERS / 32);
    }
    mbar_fence_init();
    tma_prefetch_desc(&L.cur);
    tma_prefetch_desc(&L.old);
    tma_prefetch_desc(&L.s);
    tma_prefetch_desc(&L.q);
  }
  __syncthreads();

  if (tid >= STEP_CONSUMERS) {
    if (tid == STEP_CONSUMERS)
      produce_planes<S>(&L.cur, &L.old, &L.s, &L.q, smem, bar, emp, x0, y0, k0, k1, n, tile_fem, P.a, P.b,
                        P.chan, P.spin_limit, P.err);
    return;
  }

  const long long plane = (long long)P.px * n;
  const uint32_t cs = (uint32_t)P.cs;
  const uint32_t sides = (P.abs_now | P.abs_next) & (DDFD_ABS_X0 | DDFD_ABS_X1 | DDFD_ABS_Y0 | DDFD_ABS_Y1);
  int wq = 0, wslot = 0;   // planes waited so far, slot of the next wait
  uint32_t wphase = 0;     // parity of the next wait
  int sm1 = 0, s0 = 1, sp1 = 2;  // slots of planes p-1, p, p+1 (p = k - k0 + 1)
  {
    // per-row constants
    const int x = x0 + tx;
    int y[S::RPT], ci[S::RPT], oi[S::RPT], dym[S::RPT], dyp[S::RPT];
    bool live[S::RPT], colfem[S::RPT], colfree[S::RPT], colbnd[S::RPT];
    T *out[S::RPT];
#pragma unroll
    for (int r = 0; r < S::RPT; ++r) {
      const int yy = ty + 8 * r;
      y[r] = y0 + yy;
      ci[r] = (yy + 1) * BW + (tx + S::HX);
      oi[r] = yy * STEP_TX + tx;
      dym[r] = (y[r] == 0) ? BW : -BW;
      dyp[r] = (y[r] == n - 1) ? -BW : BW;
      live[r] = x < n && y[r] < n;
      colfem[r] = x > P.a && x < P.b && y[r] > P.a && y[r] < P.b;
      colfree[r] = x >= P.f0 && x < P.f0 + P.nf && y[r] >= P.f0 && y[r] < P.f0 + P.nf;
      // side columns need the boundary path only where a side face absorbs
      colbnd[r] = (x == 0 && (sides & DDFD_ABS_X0)) || (x == n - 1 && (sides & DDFD_ABS_X1)) ||
                  (y[r] == 0 && (sides & DDFD_ABS_Y0)) || (y[r] == n - 1 && (sides & DDFD_ABS_Y1));
      out[r] = P.old + (long long)k0 * plane + (long long)P.px * y[r] + x;
    }
    const int dxm = (x == 0) ? 1 : -1, dxp = (x == n - 1) ? -1 : 1;
    T below[S::RPT][3], cen[S::RPT][3];

    for (int k = k0; k < k1; ++k) {
      const int p = k - k0 + 1;
      bool ok = true;
      while (wq <= p + 1) {
        if (!mbar_wait_bounded(&bar[wslot], wphase, P.spin_limit)) {
          ok = false;
          break;
        }
        ++wq;
        if (++wslot == S::RING) {
          wslot = 0;
          wphase ^= 1u;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform, so __syncwarp below stays safe
        if ((tid & 31) == 0) atomicOr(P.err, 4);
        break;  // the producer times out on the slots we no longer release
      }
      const unsigned char *bm1 = smem + sm1 * S::BYTES;
      const unsigned char *b0 = smem + s0 * S::BYTES;
      const unsigned char *bp1 = smem + sp1 * S::BYTES;
      const T *Em = (const T *)(bm1 + S::E_OFF);
      const T *E0 = (const T *)(b0 + S::E_OFF);
      const T *Ep = (const T *)(bp1 + S::E_OFF);
      const T *O0 = (const T *)(b0 + S::O_OFF);
      const bool kfem = k > P.a && k < P.b;
      const bool kfree = k >= P.f0 && k < P.f0 + P.nf;
      // bottom plane: absorbing or plain Neumann; top plane: source, absorbing
      // face or detector residuals
      const bool kbnd = (k == 0 && ((P.abs_now | P.abs_next) & DDFD_ABS_BOTTOM)) || k == n - 1;
#pragma unroll
      for (int r = 0; r < S::RPT; ++r) {
        T above[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (k == k0) {
            below[r][c] = Em[c * RE + ci[r]];
            cen[r][c] = E0[c * RE + ci[r]];
          }
          above[c] = Ep[c * RE + ci[r]];
        }
        if (live[r]) {
          const bool fre = colfree[r] && kfree;
          long long fi = 0;
          if (fre) fi = (x - P.f0) + (long long)P.nf * ((y[r] - P.f0) + (long long)P.nf * (k - P.f0));
          T od[3], R[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T *e = E0 + c * RE + ci[r];
            od[c] = O0[c * S::TXY + oi[r]];
            R[c] = T(6) * cen[r][c] - (e[dxp] + e[dxm] + e[dyp[r]] + e[dym[r]] + above[c] + below[r][c]);
          }
          // update coefficients: nw = cen + A (cen - od) + Bc cen - Cq tau^2 R
          T A = T(1), Bc = T(0), Cq = T(1);
          T sx[3] = {T(0), T(0), T(0)};
          if (colfem[r] && kfem && P.ebe_r) {
            // element-by-element rows computed by k_ebe for this step
            const T *Q0 = (const T *)(b0 + S::Q_OFF);
            A = Q0[oi[r]];
            Cq = Q0[S::TXY + oi[r]];
            const int fm = P.b - P.a - 1;
            const long long row = (x - P.a - 1) + (long long)fm * ((y[r] - P.a - 1) + (long long)fm * (k - P.a - 1));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              R[c] = P.ebe_r[c * P.ebe_rows + row];
              if (ADJ) sx[c] = P.ebe_q[c * P.ebe_rows + row];
            }
          } else if (colfem[r] && kfem) {
            const T *S0 = (const T *)(b0 + S::S_OFF);
            const T *Q0 = (const T *)(b0 + S::Q_OFF);
            const int q = ci[r];
            const T s0v = S0[q];
            A = Q0[oi[r]];
            Cq = Q0[S::TXY + oi[r]];
            T v0[3], vp[7][3], st[3];
            if (!ADJ) {
              const T *Sm = (const T *)(bm1 + S::S_OFF);
              const T *Sp = (const T *)(bp1 + S::S_OFF);
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const T *e0 = E0 + c * RE, *ep = Ep + c * RE, *em = Em + c * RE;
                v0[c] = s0v * cen[r][c];
                vp[0][c] = S0[q + 1] * e0[q + 1] + S0[q - 1] * e0[q - 1];
                vp[1][c] = S0[q + BW] * e0[q + BW] + S0[q - BW] * e0[q - BW];
                vp[2][c] = Sp[q] * above[c] + Sm[q] * below[r][c];
                vp[3][c] = S0[q + 1 + BW] * e0[q + 1 + BW] + S0[q - 1 - BW] * e0[q - 1 - BW];
                vp[4][c] = Sp[q + 1] * ep[q + 1] + Sm[q - 1] * em[q - 1];
                vp[5][c] = Sp[q + BW] * ep[q + BW] + Sm[q - BW] * em[q - BW];
                vp[6][c] = Sp[q + 1 + BW] * ep[q + 1 + BW] + Sm[q - 1 - BW] * em[q - 1 - BW];
              }
              block_apply<T>(v0, vp, st);
#pragma unroll
              for (int c = 0; c < 3; ++c) R[c] += st[c];
            } else if (s0v != T(0) || fre) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const T *e0 = E0 + c * RE, *ep = Ep + c * RE, *em = Em + c * RE;
                v0[c] = cen[r][c];
                vp[0][c] = e0[q + 1] + e0[q - 1];
                vp[1][c] = e0[q + BW] + e0[q - BW];
                vp[2][c] = above[c] + below[r][c];
                vp[3][c] = e0[q + 1 + BW] + e0[q - 1 - BW];
                vp[4][c] = ep[q + 1] + em[q - 1];
                vp[5][c] = ep[q + BW] + em[q - BW];
                vp[6][c] = ep[q + 1 + BW] + em[q - 1 - BW];
              }
              block_apply<T>(v0, vp, sx);
#pragma unroll
              for (int c = 0; c < 3; ++c) R[c] += s0v * sx[c];
            }
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) R[c] *= P.r2;
          if (colbnd[r] || kbnd) {
            // boundary node: damping of the absorbing faces, top-face source or
            // detector residuals
            const int fn = face_count(x, y[r], k, n, P.abs_now);
            const T cc = P.cb * T(fn);
            const T ccn = ADJ ? P.cb * T(face_count(x, y[r], k, n, P.abs_next)) : cc;
            const T inv = P.inv_tab[fn];  // 1 / (1 + cc)
            A = (T(1) - ccn) * inv;
            Bc = (ccn - cc) * inv;
            Cq = inv;
            if (!ADJ && k == n - 1 && P.src_on) {
              if (!P.oblique) {
                R[1] -= P.src_y;
              } else {
                const double v = P.src_scale * pulse_value(P.pulse_kind, P.freq, P.t0, P.width,
                                                           P.t_n - P.delay[x + n * y[r]]);
#pragma unroll
                for (int c = 0; c < 3; ++c) R[c] -= (T)(P.pol[c] * v);
              }
            }
            if (ADJ && k == n - 1 && P.n_det > 0) {
              const int q0 = P.det_ptr[x + n * y[r]], q1 = P.det_ptr[x + n * y[r] + 1];
              if (q1 > q0) {
                const double wx = (x == 0 || x == n - 1) ? 0.5 : 1.0;
                const double wy = (y[r] == 0 || y[r] == n - 1) ? 0.5 : 1.0;
                const double sc = P.tau2 * P.inv_h3 / (wx * wy * 0.5);
                double acc[3] = {0.0, 0.0, 0.0};
                for (int qq = q0; qq < q1; ++qq) {
                  const int d = P.det_list[qq];
                  acc[0] += P.res_k[3 * d + 0];
                  acc[1] += P.res_k[3 * d + 1];
                  acc[2] += P.res_k[3 * d + 2];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) R[c] += (T)(sc * acc[c]);
              }
            }
          }
          T nw[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            nw[c] = cen[r][c] + (A * (cen[r][c] - od[c]) + (Bc * cen[r][c] - Cq * R[c]));
            out[r][c * cs] = nw[c];
          }
          if (fre) {
            if (!ADJ) {
            if (P.hist_w)
#pragma unroll
              for (int c = 0; c < 3; ++c) P.hist_w[c * P.n_free + fi] = nw[c];
            } else {
              T ge = T(0), gs = T(0);
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const T hv = __ldg(P.hist_r + c * P.n_free + fi);
                ge += hv * ((nw[c] - T(2) * cen[r][c] + od[c]) + P.r2 * sx[c]);
                gs += hv * (nw[c] - od[c]);
              }
              P.gacc_e[fi] += (double)ge;
              P.gacc_s[fi] += (double)gs;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          below[r][c] = cen[r][c];
          cen[r][c] = above[c];
        }
        out[r] += plane;
      }
      // release plane p-1 (its slot) to the producer: one arrival per warp
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&emp[sm1]);
      sm1 = s0;
      s0 = sp1;
      sp1 = (sp1 + 1 == S::RING) ? 0 : sp1 + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 step kernel, two x-adjacent nodes per thread
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// Moves the line holding p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// Packed FP32 (sm_100+): one instruction for the two nodes of a pair.  These
// round exactly like the scalar operations; a - b is written fma(b, -1, a),
// which is exact in its negation.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#define kOne f2(1.f)
#define kZero f2(0.f)
#define kM1 f2(-1.f)
#define kM6 f2(-6.f)
#define kSixth f2(1.f / 6.f)
#define kMSixth f2(-1.f / 6.f)

// acc + w v for a compile-time weight (0 and +-1 cost no multiply).
__device__ __forceinline__ float2 wacc2(float2 acc, int w, float2 v) {
  if (w == 0) return acc;
  if (w == 1) return add2(acc, v);
  if (w == -1) return fma2(v, kM1, acc);
  return fma2(f2((float)w), v, acc);
}

// Input component d of the pair's two 15-point block stencils (a at x, b at
// x+1): the centre values and the 7 (+o, -o) pair sums, added as
// out_c += B_o[c][d] * (...), B = kb / 6 applied by the caller; both nodes
// share the weights.
__device__ __forceinline__ void block_acc2(int d, float2 v0, const float2 ps[7], float2 out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 u = wacc2(out[c], kb(0, c * 3 + d), v0);
#pragma unroll
    for (int p = 0; p < 7; ++p) u = wacc2(u, kb(p + 1, c * 3 + d), ps[p]);
    out[c] = u;
  }
}

// The 22 positions the pair's two stencils touch, as 11 pairs: plane k (row y:
// x-1..x+2; row y+1: x..x+2; row y-1: x-1..x+1), plane k+1 (rows y, y+1:
// x..x+2) and plane k-1 (rows y, y-1: x-1..x+1).
struct PairVals2 {
  float2 c;         // plane k, row y: x, x+1
  float2 yp, ym;    // plane k, rows y+1 and y-1: x, x+1
  float2 pc, mc;    // planes k+1 and k-1, row y: x, x+1
  float2 py, my;    // plane k+1 row y+1, plane k-1 row y-1: x, x+1
  float2 mp;        // plane k, row y: x-1, x+2
  float2 e9;        // plane k: row y+1 x+2, row y-1 x-1
  float2 e10;       // plane k+1: row y x+2, row y+1 x+2
  float2 e11;       // plane k-1: row y x-1, row y-1 x-1
  __device__ __forceinline__ void mul(const PairVals2 &s) {
    c = mul2(c, s.c);
    yp = mul2(yp, s.yp);
    ym = mul2(ym, s.ym);
    pc = mul2(pc, s.pc);
    mc = mul2(mc, s.mc);
    py = mul2(py, s.py);
    my = mul2(my, s.my);
    mp = mul2(mp, s.mp);
    e9 = mul2(e9, s.e9);
    e10 = mul2(e10, s.e10);
    e11 = mul2(e11, s.e11);
  }
};

// Pair sums of the offsets (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,0,1) (0,1,1)
// (1,1,1): x is node a's v_{i+o} + v_{i-o}, y node b's.
__device__ __forceinline__ void pair_sums2(const PairVals2 &v, float2 ps[7]) {
  ps[0] = add2(make_float2(v.c.y, v.mp.y), make_float2(v.mp.x, v.c.x));
  ps[1] = add2(v.yp, v.ym);
  ps[2] = add2(v.pc, v.mc);
  ps[3] = add2(make_float2(v.yp.y, v.e9.x), make_float2(v.e9.y, v.ym.x));
  ps[4] = add2(make_float2(v.pc.y, v.e10.x), make_float2(v.e11.x, v.mc.x));
  ps[5] = add2(v.py, v.my);
  ps[6] = add2(make_float2(v.py.y, v.e10.y), make_float2(v.e11.y, v.my.x));
}

// Values of one component at the 22 positions; the ones the Laplacian already
// loaded are passed in (centre, planes k +- 1, rows y -+ 1, x-1 and x+2).
__device__ __forceinline__ PairVals2 pair_vals(const float *e0, const float *ep, const float *em, int ci,
                                               float2 cen, float2 ab, float2 bl, float2 ym, float2 yp, float xm,
                                               float xp2) {
  constexpr int BW = PairStage::BXW;
  PairVals2 v;
  v.c = cen;
  v.yp = yp;
  v.ym = ym;
  v.pc = ab;
  v.mc = bl;
  v.py = ld2(ep + ci + BW);
  v.my = ld2(em + ci - BW);
  v.mp = make_float2(xm, xp2);
  v.e9 = make_float2(e0[ci + BW + 2], e0[ci - BW - 1]);
  v.e10 = make_float2(ep[ci + 2], ep[ci + BW + 2]);
  v.e11 = make_float2(em[ci - 1], em[ci - BW - 1]);
  return v;
}

// The s = eps - 1 plane of a stage.
__device__ __forceinline__ const float *S0f(const unsigned char *stage) {
  return (const float *)(stage + PairStage::S_OFF);
}

// Staging: the forward CTA has no producer warp: thread 0 stages the first
// RING planes, and afterwards the last of the 8 warps to release a slot
// stages the plane that reuses it (per-slot release counters in shared
// memory); 8 warps per CTA and 2 CTAs per SM leave up to 128 registers per
// thread.  The adjoint CTA has a producer warp (warp 8) fed by per-slot
// "empty" mbarriers; it measured faster there (full kernel: 80 vs 84 us per
// 201^3 step; lean kernel: 54.6 vs 56.9 us).  The lean kernels (no FEM or
// free nodes) run 3 CTAs per SM (forward: 80 registers a thread, adjoint: 72).
template <bool ADJ, bool LEAN>
struct PairMode {
  static constexpr bool PRODUCER_WARP = ADJ;
  static constexpr int THREADS = PRODUCER_WARP ? STEP_THREADS : STEP_CONSUMERS;
  static constexpr int MIN_CTAS = LEAN ? 3 : 2;
};

template <bool ADJ, int NB, bool LEAN>
__global__ void __launch_bounds__(PairMode<ADJ, LEAN>::THREADS, PairMode<ADJ, LEAN>::MIN_CTAS)
    k_step_pair(const __grid_constant__ StepLaunch<float, NB> L) {
  constexpr bool PW = PairMode<ADJ, LEAN>::PRODUCER_WARP;
  using S = PairStageT<LEAN>;
  constexpr int RE = S::RE, BW = S::BXW, TXY = S::TXY;
  const CtaTile ct = cta_tile(L);
  const StepParams<float> &P = L.p[NB == 1 ? 0 : ct.prob];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t *bar = (uint64_t *)(smem + S::RING * S::BYTES);  // "full": plane landed
  uint64_t *emp = bar + S::RING;                              // producer warp: "empty" barriers
  unsigned *rel = (unsigned *)(emp + S::RING);                // otherwise: per-slot warp releases
  int *issued = (int *)(rel + S::RING);                       // planes staged so far (a prefix)
  int *exited = issued + 1;                                   // warps that left the loop
  const int n = P.n;
  const int tid = threadIdx.x;

  if (!ADJ) sample_detectors(P, ct, tid);

  const int x0 = ct.tx * S::TX, y0 = ct.ty * S::TY;
  const int k0 = ct.k0;
  if (k0 >= n) return;  // uniform per CTA
  const int k1 = min(ct.k1, n);
  const bool tile_fem =
      !LEAN && x0 <= P.b - 1 && x0 + S::TX - 1 >= P.a + 1 && y0 <= P.b - 1 && y0 + S::TY - 1 >= P.a + 1;
  const int nplanes = k1 - k0 + 2;

  if (tid == 0) {
    for (int s = 0; s < S::RING; ++s) {
      mbar_init(&bar[s], 1);
      if (PW) mbar_init(&emp[s], STEP_CONSUMERS / 32);
      rel[s] = 0;
    }
    *exited = 0;
    mbar_fence_init();
    tma_prefetch_desc(&L.cur);
    tma_prefetch_desc(&L.old);
    tma_prefetch_desc(&L.s);
    tma_prefetch_desc(&L.q);
    if (!PW) {
      const int first = nplanes < S::RING ? nplanes : S::RING;
      *issued = first;
      for (int q = 0; q < first; ++q)
        stage_plane<S>(q, &L.cur, &L.old, &L.s, &L.q, smem, bar, x0, y0, k0, k1, n, tile_fem, P.a, P.b, P.chan);
    }
  }
  __syncthreads();

  if (PW && tid >= STEP_CONSUMERS) {
    if (tid == STEP_CONSUMERS)
      produce_planes<S>(&L.cur, &L.old, &L.s, &L.q, smem, bar, emp, x0, y0, k0, k1, n, tile_fem, P.a, P.b,
                        P.chan, P.spin_limit, P.err);
    return;
  }

  // nodes a = (x, y) and b = (x + 1, y) of every plane; lanes 0-15 of warp w
  // take row 2w, lanes 16-31 row 2w + 1
  const int lane = tid & 31;
  const int yy = 2 * (tid >> 5) + (lane >> 4);
  const int xl = 2 * (lane & 15);
  const int x = x0 + xl, y = y0 + yy;
  const int ci = (yy + 1) * BW + S::HX + xl;  // centre of node a in a staged plane (even)
  const int oi = yy * S::TX + xl;             // node a in a centre box (even)
  const bool live_a = x < n && y < n, live_b = x + 1 < n && y < n;
  const int dym = (y == 0) ? BW : -BW, dyp = (y == n - 1) ? -BW : BW;  // mirror rows
  const bool ex0 = x == 0, exa = x == n - 1, exb = x + 1 == n - 1;   // mirror columns
  const bool rowfem = y > P.a && y < P.b;
  const bool colfem = rowfem && x + 1 > P.a && x < P.b;  // either node strictly inside the cube
  const bool fem_a = rowfem && x > P.a && x < P.b, fem_b = rowfem && x + 1 > P.a && x + 1 < P.b;
  const bool rowfree = y >= P.f0 && y < P.f0 + P.nf;
  const bool free_a = rowfree && x >= P.f0 && x < P.f0 + P.nf;
  const bool free_b = rowfree && x + 1 >= P.f0 && x + 1 < P.f0 + P.nf;
  const uint32_t sides = (P.abs_now | P.abs_next) & (DDFD_ABS_X0 | DDFD_ABS_X1 | DDFD_ABS_Y0 | DDFD_ABS_Y1);
  const bool ybnd = (y == 0 && (sides & DDFD_ABS_Y0)) || (y == n - 1 && (sides & DDFD_ABS_Y1));
  const bool bnd_a = ybnd || (x == 0 && (sides & DDFD_ABS_X0)) || (x == n - 1 && (sides & DDFD_ABS_X1));
  const bool bnd_b = ybnd || (x + 1 == n - 1 && (sides & DDFD_ABS_X1));
  const long long plane = (long long)P.px * n;
  const uint32_t cs = (uint32_t)P.cs;
  float *out = P.old + (long long)k0 * plane + (long long)P.px * y + x;

  // one absorbing-face / source / residual update of node (xn, y): the
  // boundary form of the update coefficients and the extra terms of R
  auto boundary = [&](int xn, int k, float R[3], float &A, float &Bc, float &Cq) {
    const int fn = face_count(xn, y, k, n, P.abs_now);
    const float cc = P.cb * (float)fn;
    const float ccn = ADJ ? P.cb * (float)face_count(xn, y, k, n, P.abs_next) : cc;
    const float inv = P.inv_tab[fn];  // 1 / (1 + cc)
    A = (1.f - ccn) * inv;
    Bc = (ccn - cc) * inv;
    Cq = inv;
    if (!ADJ && k == n - 1 && P.src_on) {
      if (!P.oblique) {
        R[1] -= P.src_y;
      } else {
        const double v = P.src_scale * pulse_value(P.pulse_kind, P.freq, P.t0, P.width, P.t_n - P.delay[xn + n * y]);
#pragma unroll
        for (int c = 0; c < 3; ++c) R[c] -= (float)(P.pol[c] * v);
      }
    }
    if (ADJ && k == n - 1 && P.n_det > 0) {
      // detector residual sources of this node at step k, summed and scaled
      // by k_det_sources
      const int u = P.det_slot[xn + n * y];
      if (u >= 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) R[c] += P.src_k[3 * u + c];
      }
    }
  };

  const float2 R2 = make_float2(P.r2, P.r2);
  int wq = 0, wslot = 0;   // planes waited so far, slot of the next wait
  uint32_t wphase = 0;     // parity of the next wait
  int sm1 = 0, s0 = 1, sp1 = 2;  // slots of planes p-1, p, p+1 (p = k - k0 + 1)
  float2 below[3], cen[3];
  for (int k = k0; k < k1; ++k) {
    const int p = k - k0 + 1;
    bool ok = true;
    while (wq <= p + 1) {
      if (!mbar_wait_bounded(&bar[wslot], wphase, P.spin_limit)) {
        ok = false;
        break;
      }
      ++wq;
      if (++wslot == S::RING) {
        wslot = 0;
        wphase ^= 1u;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform, so __syncwarp below stays safe
      if (lane == 0) atomicOr(P.err, 4);
      break;  // the producer times out on the slots we no longer release
    }
    const unsigned char *bm1 = smem + sm1 * S::BYTES;
    const unsigned char *b0 = smem + s0 * S::BYTES;
    const unsigned char *bp1 = smem + sp1 * S::BYTES;
    const float *Em = (const float *)(bm1 + S::E_OFF);
    const float *E0 = (const float *)(b0 + S::E_OFF);
    const float *Ep = (const float *)(bp1 + S::E_OFF);
    const bool kfem = k > P.a && k < P.b;
    const bool kfree = k >= P.f0 && k < P.f0 + P.nf;
    const bool kbnd = (k == 0 && ((P.abs_now | P.abs_next) & DDFD_ABS_BOTTOM)) || k == n - 1;
    float2 ab[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (k == k0) {
        below[c] = ld2(Em + c * RE + ci);
        cen[c] = ld2(E0 + c * RE + ci);
      }
      ab[c] = ld2(Ep + c * RE + ci);
    }
    if (live_a) {
      if (ADJ && !LEAN && (free_a || free_b) && kfree) {
        // the gradient operands of this plane's free nodes (E^k history, block
        // sums, at a fold the FP64 sums), read after the update below: fetched
        // into L2 now, so that the stencil work hides their DRAM latency
        const long long fp = (x - P.f0) + (long long)P.nf * ((y - P.f0) + (long long)P.nf * (k - P.f0));
#pragma unroll
        for (int c = 0; c < 3; ++c) prefetch_l2(P.hist_r + c * P.n_free + fp);
        prefetch_l2(reinterpret_cast<const float2 *>(P.gpart) + fp);
        if (P.gmode & GM_FOLD) {
          prefetch_l2(P.gacc_e + fp);
          prefetch_l2(P.gacc_s + fp);
        }
      }
      // The pair's arithmetic runs in packed FP32 (x: node a, y: node b).  Q
      // holds -R, so that every subtraction is a multiply-add with a constant
      // (exact negations); a boundary node converts to R for the scalar
      // boundary terms.
      float2 Q[3], ym[3], yp[3];
      float xm[3], xp2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float *e = E0 + c * RE + ci;
        ym[c] = ld2(e + dym);
        yp[c] = ld2(e + dyp);
        xm[c] = e[-1];
        xp2[c] = e[2];
        const float xma = ex0 ? cen[c].y : xm[c];   // ghost x-1 = x+1 at x = 0
        const float xpa = exa ? xm[c] : cen[c].y;   // ghost x+1 = x-1 at x = n-1
        const float xpb = exb ? cen[c].x : xp2[c];
        float2 sn = add2(make_float2(xpa, xpb), make_float2(xma, cen[c].x));
        sn = add2(add2(add2(add2(sn, yp[c]), ym[c]), ab[c]), below[c]);
        Q[c] = fma2(kM6, cen[c], sn);  // (neighbour sum) - 6 E
      }
      float2 A2 = kOne, B2 = kZero, C2 = kOne;
      float2 SX[3] = {kZero, kZero, kZero};
      // (a lean launch carries no tile with FEM-cube or free nodes)
      const bool fre_a = !LEAN && free_a && kfree, fre_b = !LEAN && free_b && kfree;
      const bool fem_pair = !LEAN && colfem && kfem;
      if (fem_pair) {
        const float *Q0 = (const float *)(b0 + S::Q_OFF);
        A2 = ld2(Q0 + oi);
        C2 = ld2(Q0 + TXY + oi);
        if (P.ebe_r) {
          // element-by-element rows computed by k_ebe for this step
          const int fm = P.b - P.a - 1;
          const long long row = (x - P.a - 1) + (long long)fm * ((y - P.a - 1) + (long long)fm * (k - P.a - 1));
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (fem_a) {
              Q[c].x = -P.ebe_r[c * P.ebe_rows + row];
              if (ADJ) SX[c].x = P.ebe_q[c * P.ebe_rows + row];
            }
            if (fem_b) {
              Q[c].y = -P.ebe_r[c * P.ebe_rows + row + 1];
              if (ADJ) SX[c].y = P.ebe_q[c * P.ebe_rows + row + 1];
            }
          }
        } else if (!ADJ) {
          // forward: sum_o B_o (s E)_{i+o} for both nodes
          const PairVals2 sv = pair_vals(S0f(b0), S0f(bp1), S0f(bm1), ci, ld2(S0f(b0) + ci), ld2(S0f(bp1) + ci),
                                         ld2(S0f(bm1) + ci), ld2(S0f(b0) + ci - BW), ld2(S0f(b0) + ci + BW),
                                         S0f(b0)[ci - 1], S0f(b0)[ci + 2]);
          float2 O[3] = {kZero, kZero, kZero};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            PairVals2 v = pair_vals(E0 + d * RE, Ep + d * RE, Em + d * RE, ci, cen[d], ab[d], below[d], ym[d],
                                    yp[d], xm[d], xp2[d]);
            v.mul(sv);
            float2 Ps[7];
            pair_sums2(v, Ps);
            block_acc2(d, v.c, Ps, O);
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) Q[c] = fma2(O[c], kMSixth, Q[c]);
        } else {
          // adjoint: s_i sum_o B_o mu_{i+o}; the sums are kept for the gradient
          const float2 s0v = ld2(S0f(b0) + ci);
          if (s0v.x != 0.f || s0v.y != 0.f || fre_a || fre_b) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const PairVals2 v = pair_vals(E0 + d * RE, Ep + d * RE, Em + d * RE, ci, cen[d], ab[d], below[d],
                                            ym[d], yp[d], xm[d], xp2[d]);
              float2 Ps[7];
              pair_sums2(v, Ps);
              block_acc2(d, v.c, Ps, SX);
            }
            const float2 ns0 = mul2(s0v, kM1);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              SX[c] = mul2(SX[c], kSixth);
              Q[c] = fma2(ns0, SX[c], Q[c]);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Q[c] = mul2(Q[c], R2);
      const bool bnd_pa = bnd_a || kbnd, bnd_pb = live_b && (bnd_b || kbnd);
      if (bnd_pa || bnd_pb) {
        float Rn[3];
        if (bnd_pa) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Rn[c] = -Q[c].x;
          boundary(x, k, Rn, A2.x, B2.x, C2.x);
#pragma unroll
          for (int c = 0; c < 3; ++c) Q[c].x = -Rn[c];
        }
        if (bnd_pb) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Rn[c] = -Q[c].y;
          boundary(x + 1, k, Rn, A2.y, B2.y, C2.y);
#pragma unroll
          for (int c = 0; c < 3; ++c) Q[c].y = -Rn[c];
        }
      }
      const float *O0 = (const float *)(b0 + S::O_OFF);
      const bool plain = !fem_pair && !bnd_pa && !bnd_pb;  // A = 1, B = 0, C = 1
      float2 od[3], nw[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        od[c] = ld2(O0 + c * TXY + oi);
        const float2 dv = fma2(od[c], kM1, cen[c]);  // E^n - E^{n-1}
        // E^{n+1} = E^n + A (E^n - E^{n-1}) + B E^n - C R, with R = -Q
        nw[c] = plain ? add2(cen[c], add2(dv, Q[c]))
                      : add2(cen[c], add2(mul2(A2, dv), fma2(C2, Q[c], mul2(B2, cen[c]))));
        if (live_b)
          *reinterpret_cast<float2 *>(out + c * cs) = nw[c];
        else
          out[c * cs] = nw[c].x;
      }
      if (fre_a || fre_b) {
        const long long fi = (x - P.f0) + (long long)P.nf * ((y - P.f0) + (long long)P.nf * (k - P.f0));
        if (!ADJ) {
          if (P.hist_w) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              if (fre_a) P.hist_w[c * P.n_free + fi] = nw[c].x;
              if (fre_b) P.hist_w[c * P.n_free + fi + 1] = nw[c].y;
            }
          }
        } else {
          // both nodes' gradient terms in packed FP32 (a node that is not free
          // adds nothing: its E^k operand is zero and nothing is stored)
          const float *hr = P.hist_r + fi;
          float2 ge = kZero, gs = kZero;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 hv = make_float2(fre_a ? __ldg(hr + c * P.n_free) : 0.f, fre_b ? __ldg(hr + c * P.n_free + 1) : 0.f);
            const float2 te = fma2(R2, SX[c], add2(fma2(cen[c], f2(-2.f), nw[c]), od[c]));
            ge = fma2(hv, te, ge);
            gs = fma2(hv, fma2(od[c], kM1, nw[c]), gs);
          }
          // block sums in FP32, folded into the FP64 accumulators
          float2 *gp = reinterpret_cast<float2 *>(P.gpart) + fi;
          if (!(P.gmode & GM_FIRST)) {
            const float2 pa = fre_a ? gp[0] : kZero, pb = fre_b ? gp[1] : kZero;
            ge = add2(make_float2(pa.x, pb.x), ge);
            gs = add2(make_float2(pa.y, pb.y), gs);
          }
          if (P.gmode & GM_FOLD) {
            if (fre_a) {
              P.gacc_e[fi] += (double)ge.x;
              P.gacc_s[fi] += (double)gs.x;
            }
            if (fre_b) {
              P.gacc_e[fi + 1] += (double)ge.y;
              P.gacc_s[fi + 1] += (double)gs.y;
            }
          } else {
            if (fre_a) gp[0] = make_float2(ge.x, gs.x);
            if (fre_b) gp[1] = make_float2(ge.y, gs.y);
          }
        }
      }
      if (x0 + S::TX == n - 1 && xl == S::TX - 2) {
        // x tail: with n = 32 m + 1 the launch has m tiles in x, the last
        // ending at x = n - 2, and its lanes owning columns 30, 31 also update
        // the boundary node e = (n - 1, y), in the staged x halo (an FD node,
        // never FEM or free): 7-point row with the mirror ghost x + 1 = x - 1,
        // summed in the order of the pair's rows; operands re-read from the
        // staged planes (the pair's registers are free again here)
        float Re[3], Ae = 1.f, Be = 0.f, Ce = 1.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float *e = E0 + c * RE + ci + 2;
          const float xme = e[-1];
          Re[c] = 6.f * e[0] - (((((xme + xme) + e[dyp]) + e[dym]) + Ep[c * RE + ci + 2]) + Em[c * RE + ci + 2]);
          Re[c] *= P.r2;
        }
        if (ybnd || (sides & DDFD_ABS_X1) || kbnd) boundary(n - 1, k, Re, Ae, Be, Ce);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float ce = E0[c * RE + ci + 2];
          const float ov = out[c * cs + 2];  // the previous level, read before it is overwritten
          out[c * cs + 2] = ce + (Ae * (ce - ov) + (Be * ce - Ce * Re[c]));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      below[c] = cen[c];
      cen[c] = ab[c];
    }
    out += plane;
    // release plane p-1: the warp that completes the slot's release count
    // stages plane p-1+RING into it
    __syncwarp();
    if (PW) {
      if (lane == 0) mbar_arrive(&emp[sm1]);
    } else if (lane == 0) {
      __threadfence_block();
      const unsigned prev = atomicAdd(&rel[sm1], 1u);
      if ((prev + 1) % (STEP_CONSUMERS / 32) == 0) {
        const int q = p - 1 + S::RING;
        if (q < nplanes) {
          __threadfence_block();
          fence_proxy_async_smem();
          stage_plane<S>(q, &L.cur, &L.old, &L.s, &L.q, smem, bar, x0, y0, k0, k1, n, tile_fem, P.a, P.b,
                         P.chan);
          atomicMax(issued, q + 1);
        }
      }
    }
    sm1 = s0;
    s0 = sp1;
    sp1 = (sp1 + 1 == S::RING) ? 0 : sp1 + 1;
  }
  // the last warp out waits (bounded) for the copies still in flight, if a
  // timeout cut the loop short (otherwise they have all landed already); with
  // a producer warp, that warp does it
  __syncwarp();
  if (!PW && lane == 0) {
    __threadfence_block();
    if (atomicAdd(exited, 1) == STEP_CONSUMERS / 32 - 1) {
      const int iss = atomicAdd(issued, 0);
      for (int q = iss > S::RING ? iss - S::RING : 0; q < iss; ++q)
        mbar_wait_bounded(&bar[q % S::RING], (uint32_t)((q / S::RING) & 1), P.spin_limit);
    }
  }
}

template <bool ADJ, int NB>
static cudaError_t set_smem_f64() {
  return cudaFuncSetAttribute(k_step<double, ADJ, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Stage<double>::SMEM);
}
template <bool ADJ, int NB>
static cudaError_t set_smem_f32() {
  cudaError_t e = cudaFuncSetAttribute(k_step_pair<ADJ, NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PairStageT<false>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_step_pair<ADJ, NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              PairStageT<true>::SMEM);
}

cudaError_t prepare_step_kernels() {
  cudaError_t e;
  if ((e = set_smem_f32<false, 1>()) != cudaSuccess || (e = set_smem_f32<true, 1>()) != cudaSuccess ||
      (e = set_smem_f64<false, 1>()) != cudaSuccess || (e = set_smem_f64<true, 1>()) != cudaSuccess ||
      (e = set_smem_f32<false, BATCH_MAX>()) != cudaSuccess || (e = set_smem_f32<true, BATCH_MAX>()) != cudaSuccess ||
      (e = set_smem_f64<false, BATCH_MAX>()) != cudaSuccess || (e = set_smem_f64<true, BATCH_MAX>()) != cudaSuccess)
    return e;
  return cudaSuccess;
}

int step_tiles_x(int n, bool fp32) { return fp32 ? tiles_pair_x(n) : (n + STEP_TX - 1) / STEP_TX; }
int step_tiles_y(int n, bool fp32) {
  const int ty = fp32 ? StepTile<float>::TY : StepTile<double>::TY;
  return (n + ty - 1) / ty;
}

// Launch grid: 1-D over the dispatch items, or the 3-D tile grid.
template <typename T, int NB>
static dim3 step_grid(const StepLaunch<T, NB> &L) {
  const int gx = step_tiles_x(L.p[0].n, sizeof(T) == 4), gy = step_tiles_y(L.p[0].n, sizeof(T) == 4);
  if (L.items) return dim3((unsigned)L.n_items);
  return dim3(gx, gy, L.zchunks * L.nprob);
}

template <bool ADJ, int NB>
static int launch_step(const StepLaunch<double, NB> &L, cudaStream_t s, const StepFork *) {
  k_step<double, ADJ, NB><<<step_grid(L), STEP_THREADS, Stage<double>::SMEM, s>>>(L);
  return 1;
}
// FP32: the dispatch order's FEM/free tiles on the full kernel, the others on
// the lean one, side by side when fk provides a side stream.
template <bool ADJ, int NB>
static int launch_step(const StepLaunch<float, NB> &L, cudaStream_t s, const StepFork *fk) {
  using Full = PairMode<ADJ, false>;
  using Lean = PairMode<ADJ, true>;
  const dim3 g = step_grid(L);
  if (!L.items || L.n_full >= (int)g.x) {
    k_step_pair<ADJ, NB, false><<<g, Full::THREADS, PairStageT<false>::SMEM, s>>>(L);
    return 1;
  }
  StepLaunch<float, NB> F = L;
  F.items = L.items + L.n_full;
  const unsigned n_lean = g.x - (unsigned)L.n_full;
  if (L.n_full == 0) {
    k_step_pair<ADJ, NB, true><<<n_lean, Lean::THREADS, PairStageT<true>::SMEM, s>>>(F);
    return 1;
  }
  cudaStream_t s2 = s;
  if (fk && fk->side && cudaEventRecord(fk->ev_fork, s) == cudaSuccess &&
      cudaStreamWaitEvent(fk->side, fk->ev_fork, 0) == cudaSuccess)
    s2 = fk->side;
  k_step_pair<ADJ, NB, false><<<(unsigned)L.n_full, Full::THREADS, PairStageT<false>::SMEM, s>>>(L);
  k_step_pair<ADJ, NB, true><<<n_lean, Lean::THREADS, PairStageT<true>::SMEM, s2>>>(F);
  if (s2 != s) {
    // a failure here is left in the runtime's last error for the caller's check
    if (cudaEventRecord(fk->ev_join, s2) == cudaSuccess) cudaStreamWaitEvent(s, fk->ev_join, 0);
  }
  return 2;
}

template <typename T, int NB>
int launch_forward_step(const StepLaunch<T, NB> &L, cudaStream_t s, const StepFork *fk) {
  return launch_step<false, NB>(L, s, fk);
}
template <typename T, int NB>
int launch_adjoint_step(const StepLaunch<T, NB> &L, cudaStream_t s, const StepFork *fk) {
  return launch_step<true, NB>(L, s, fk);
}

#define DDFD_STEP_INST(T, NB)                                                                           \
  template int launch_forward_step<T, NB>(const StepLaunch<T, NB> &, cudaStream_t, const StepFork *); \
  template int launch_adjoint_step<T, NB>(const StepLaunch<T, NB> &, cudaStream_t, const StepFork *);
DDFD_STEP_INST(float, 1)
DDFD_STEP_INST(double, 1)
DDFD_STEP_INST(float, BATCH_MAX)
DDFD_STEP_INST(double, BATCH_MAX)
#undef DDFD_STEP_INST

// y = h^2 M_eps^-1 K x in FP64 on every node (no damping, no source): the
// operator whose largest eigenvalue bounds the stable time step.  One thread
// per node; x, y unpadded (3 n^3); s read from the padded coefficient field.
template <typename T>
__global__ void k_apply_op(const double *x, double *y, int n, int px, int a, int b, const T *coef_s) {
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
      auto sv = [&](int di, int dj, int dk) {
        return (double)coef_s[(i + di) + (long long)px * ((j + dj) + (long long)n * (k + dk))];
      };
      const double s0 = sv(0, 0, 0);
      eps = 1.0 + s0;
      const int dx[7] = {1, 0, 0, 1, 1, 0, 1}, dy[7] = {0, 1, 0, 1, 0, 1, 1}, dz[7] = {0, 0, 1, 0, 1, 1, 1};
      double v0[3], vp[7][3], st[3];
      for (int c = 0; c < 3; ++c) v0[c] = s0 * x[c * nn + q];
      for (int p = 0; p < 7; ++p) {
        const long long og = dx[p] + n * (dy[p] + (long long)n * dz[p]);
        for (int c = 0; c < 3; ++c)
          vp[p][c] = sv(dx[p], dy[p], dz[p]) * x[c * nn + q + og] +
                     sv(-dx[p], -dy[p], -dz[p]) * x[c * nn + q - og];
      }
      block_apply<double>(v0, vp, st);
      for (int c = 0; c < 3; ++c) out[c] += st[c];
    }
    for (int c = 0; c < 3; ++c) y[c * nn + q] = out[c] / eps;
  }
}

void launch_apply_op(const double *x, double *y, int n, int px, int a, int b, const void *coef_s, int fp32,
                     cudaStream_t s) {
  const long long nn = (long long)n * n * n;
  const long long nb = (nn + 255) / 256;
  const int blocks = (int)(nb < 8192 ? nb : 8192);
  if (fp32)
    k_apply_op<float><<<blocks, 256, 0, s>>>(x, y, n, px, a, b, (const float *)coef_s);
  else
    k_apply_op<double><<<blocks, 256, 0, s>>>(x, y, n, px, a, b, (const double *)coef_s);
}

}  // namespace ddfd
