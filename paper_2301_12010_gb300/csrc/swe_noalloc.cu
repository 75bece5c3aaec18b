// swe_noalloc.cu -- an allocation-free variant of the mass reduction.
//
// swe_mass() sums the water volume with a two-pass FP64 reduction whose
// per-block partials live in memory the handle allocated with cudaMalloc.
// Some callers cannot allocate at all when they need this number:
//   - hosts that reserve their whole device-memory budget up front (a
//     serving process admitting work under a fixed HBM budget) and forbid any
//     later allocation;
//   - latency-sensitive loops that must not take the device-wide
//     synchronisation a cudaMalloc / cudaFree implies;
//   - plain C hosts that link only this ABI and hold no allocator or handle.
// swe_mass_noalloc() serves them: the caller passes the depth field and the
// output slot, both in its own device memory, and the scratch (one FP64
// partial per grid row) is a fixed array in this library's device image.
//
// Contract:
//   - At most SWE_NOALLOC_MAX_ROWS rows; larger grids are rejected with
//     SWE_EINVAL before any device work.
//   - The first call on a device looks up the scratch array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it with the
//     device's current context; make that first call before any stream
//     capture on the device.  A later call in another context of the device
//     (after cudaDeviceReset, which loads the library's device image anew)
//     looks the address up again instead of using the old one.
//   - Every call on a device shares the one scratch array: calls whose work
//     overlaps on the GPU (different streams, or several host threads) race
//     and may return wrong sums.  Calls ordered on one stream are safe; each
//     call rewrites every partial it reads, so nothing needs clearing between
//     calls.
//   - No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda.h>  // CUcontext (the type only; the entry point is resolved through the runtime)
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/swe.h"

namespace {

constexpr int kMaxDevices = 64;

// Per-row FP64 partial sums; modest and fixed: SWE_NOALLOC_MAX_ROWS doubles
// (128 KiB) held by every device that loads the library, until exit.
static __device__ __align__(256) double g_row_partials[SWE_NOALLOC_MAX_ROWS];

// Pass 1: one warp per row sums h over the row in FP64, fixed lane order.
template <typename T>
__global__ void k_row_sums(const T *__restrict__ h, int nx, int ny, double *__restrict__ part) {
  const int warps = blockDim.x >> 5;
  const int j = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= ny) return;
  const T *row = h + (size_t)j * nx;
  double s = 0.0;
  for (int i = lane; i < nx; i += 32) s += (double)row[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[j] = s;
}

// Pass 2: one block sums the ny partials in a fixed tree order.
__global__ void k_rows_total(const double *__restrict__ part, int ny, double area, double *__restrict__ out) {
  __shared__ double sm[1024];
  double s = 0.0;
  for (int q = threadIdx.x; q < ny; q += blockDim.x) s += part[q];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0] * area;
}

std::mutex g_lock;
double *g_scratch[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // context in which g_scratch[dev] was looked up

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

// cuCtxGetCurrent from the driver, resolved once through the runtime (no
// link-time dependence on the driver library); nullptr if unavailable.
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// Device address of the scratch array for the current device: looked up once
// per device and context (a new context, e.g. after cudaDeviceReset, holds a
// new copy of the array at another address).
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // the context current on this thread; none before the runtime's first
  // call on the device, in which case the lookup below makes it current
  const CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_row_partials);
    if (e != cudaSuccess) return e;
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    g_scratch[dev] = static_cast<double *>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int swe_mass_noalloc(const void *h, int32_t precision, int32_t nx, int32_t ny, double dx, double dy,
                                double *mass, void *stream) {
  if (!h || !mass || nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0)) return SWE_EINVAL;
  if (precision != SWE_F32 && precision != SWE_F64) return SWE_EINVAL;
  if (ny > SWE_NOALLOC_MAX_ROWS) return SWE_EINVAL;
  double *part = nullptr;
  cudaError_t e = scratch_for_current_device(&part);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SWE_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 256, rows_per_block = threads / 32;
  const int blocks = (ny + rows_per_block - 1) / rows_per_block;
  if (precision == SWE_F64) k_row_sums<double><<<blocks, threads, 0, st>>>(static_cast<const double *>(h), nx, ny, part);
  else k_row_sums<float><<<blocks, threads, 0, st>>>(static_cast<const float *>(h), nx, ny, part);
  k_rows_total<<<1, 1024, 0, st>>>(part, ny, dx * dy, mass);
  e = cudaGetLastError();
  return e == cudaSuccess ? SWE_OK : SWE_ECUDA;
}
