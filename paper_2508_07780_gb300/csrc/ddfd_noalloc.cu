// Allocation-free misfit reduction: ddfd_misfit_noalloc.
//
// Who needs it: callers that must not allocate device memory -- for example
// code running under a strict memory budget or inside a host framework that
// owns every device allocation (a custom allocator, a pre-planned arena, a
// real-time loop where cudaMalloc's implicit synchronisation and latency are
// not acceptable).  Such a caller cannot create a ddfd handle, because
// ddfd_create allocates the field buffers; this entry point needs no handle.
//
// Its only scratch is the file-scope array below: one FP64 partial sum per
// (source, time step) row of the trace.  It is part of the library image,
// so every GPU that loads the library holds it (512 KB) until the process
// exits; no call allocates or frees anything.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ddfd_internal.h"

namespace ddfd {
void set_thread_error(const std::string &msg);
}

namespace {

constexpr int kNoallocMaxRows = 65536;  // n_src * (n_steps + 1) at most
constexpr int kRB = 256;

static __device__ __align__(256) double g_misfit_rows[kNoallocMaxRows];

__device__ __forceinline__ double block_sum256(double v) {
  __shared__ double sh[kRB / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kRB / 32) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Pass 1: rows[s (n_steps+1) + n] = z(t_n) sum_d |trace - eobs|^2 (0 for n = 0).
// Every row in [0, n_rows) is written, so the scratch needs no clearing.
__global__ void k_misfit_rows(const double *trace, const double *eobs, int n_steps, int n_det, int n_rows,
                              double tau, double z_delta_frac, double *rows) {
  const double T = n_steps * tau, dl = z_delta_frac * T;
  for (int row = blockIdx.x; row < n_rows; row += gridDim.x) {
    const int step = row % (n_steps + 1);
    const double t = step * tau;
    const double z = (dl <= 0.0 || t <= T - dl) ? 1.0 : 0.5 * (1.0 + cos(3.141592653589793 * (t - T + dl) / dl));
    double acc = 0.0;
    if (step >= 1) {
      const long long base = (long long)row * n_det * 3;
      for (int q = threadIdx.x; q < 3 * n_det; q += blockDim.x) {
        const double d = trace[base + q] - eobs[base + q];
        acc += d * d;
      }
    }
    const double b = block_sum256(acc);
    if (threadIdx.x == 0) rows[row] = z * b;
  }
}

// Pass 2: J = tau/2 sum of the rows, fixed-order tree (bitwise reproducible).
__global__ void k_misfit_total(const double *rows, int n_rows, double tau, double *J) {
  double a = 0.0;
  for (int q = threadIdx.x; q < n_rows; q += blockDim.x) a += rows[q];
  const double b = block_sum256(a);
  if (threadIdx.x == 0) *J = 0.5 * tau * b;
}

// Device address of the scratch array.  The array's host-side name is not a
// device address, so it is resolved with cudaGetSymbolAddress, with the
// device current, once per device context: the cache entry of a device is
// keyed on the context's process-unique id (cuCtxGetId), so a context that
// was reset and re-created (cudaDeviceReset) resolves the address again
// instead of reusing a stale one.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

std::mutex g_mu;
struct RowsAddr {
  unsigned long long ctx_id = 0;  // 0: not resolved
  double *addr = nullptr;
};
RowsAddr g_rows_addr[64];
PfnCtxGetCurrent g_ctx_current = nullptr;
PfnCtxGetId g_ctx_id = nullptr;

int driver_fn(const char *name, void **fn) {
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !*fn) {
    ddfd::set_thread_error(std::string(name) + " is not available from the driver");
    return DDFD_E_CUDA;
  }
  return DDFD_OK;
}

// Id of the current context (0 if none is current yet).
int current_ctx_id(unsigned long long *id) {
  *id = 0;
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) {
    ddfd::set_thread_error("cuCtxGetCurrent failed");
    return DDFD_E_CUDA;
  }
  if (ctx && g_ctx_id(ctx, id) != CUDA_SUCCESS) {
    ddfd::set_thread_error("cuCtxGetId failed");
    return DDFD_E_CUDA;
  }
  return DDFD_OK;
}

int rows_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ddfd::set_thread_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return DDFD_E_CUDA;
  }
  if (dev < 0 || dev >= 64) {
    ddfd::set_thread_error("device ordinal out of range");
    return DDFD_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  int st;
  if (!g_ctx_current && ((st = driver_fn("cuCtxGetCurrent", (void **)&g_ctx_current)) != DDFD_OK ||
                         (st = driver_fn("cuCtxGetId", (void **)&g_ctx_id)) != DDFD_OK)) {
    g_ctx_current = nullptr;
    return st;
  }
  unsigned long long id = 0;
  if ((st = current_ctx_id(&id)) != DDFD_OK) return st;
  RowsAddr &c = g_rows_addr[dev];
  if (id == 0 || c.ctx_id != id) {
    // first use on this device or context: resolving the symbol also makes
    // the device's primary context current if nothing was current yet
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_misfit_rows);
    if (e != cudaSuccess || !p) {
      ddfd::set_thread_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return DDFD_E_CUDA;
    }
    if (id == 0 && (st = current_ctx_id(&id)) != DDFD_OK) return st;
    c.ctx_id = id;
    c.addr = (double *)p;
  }
  *out = c.addr;
  return DDFD_OK;
}

}  // namespace

extern "C" int ddfd_misfit_noalloc(const double *trace, const double *eobs, int32_t n_src, int32_t n_steps,
                                   int32_t n_det, double tau, double z_delta_frac, double *J, void *stream) {
  if (!J || n_src < 1 || n_steps < 1 || n_det < 0 || !(tau > 0.0) || !(z_delta_frac >= 0.0 && z_delta_frac < 1.0) ||
      (n_det > 0 && (!trace || !eobs))) {
    ddfd::set_thread_error("ddfd_misfit_noalloc: bad argument");
    return DDFD_E_ARG;
  }
  const long long n_rows = (long long)n_src * ((long long)n_steps + 1);
  if (n_rows < 1 || n_rows > kNoallocMaxRows) {
    ddfd::set_thread_error("ddfd_misfit_noalloc: n_src * (n_steps + 1) = " + std::to_string(n_rows) +
                           " exceeds the fixed scratch of " + std::to_string(kNoallocMaxRows) + " rows");
    return DDFD_E_ARG;
  }
  double *rows = nullptr;
  const int st = rows_address(&rows);
  if (st != DDFD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = (int)(n_rows < 4096 ? n_rows : 4096);
  k_misfit_rows<<<grid, kRB, 0, s>>>(trace, eobs, n_steps, n_det, (int)n_rows, tau, z_delta_frac, rows);
  k_misfit_total<<<1, kRB, 0, s>>>(rows, (int)n_rows, tau, J);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ddfd::set_thread_error(std::string("ddfd_misfit_noalloc launch: ") + cudaGetErrorString(e));
    return DDFD_E_CUDA;
  }
  return DDFD_OK;
}
