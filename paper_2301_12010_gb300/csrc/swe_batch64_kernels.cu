// swe_batch64_kernels.cu -- the persistent multi-scenario kernel in FP64 (the
// batch path's parity mode): k RK3 steps of every live scenario of a batch in
// one cooperative launch, on one tile shape (32 x 32, 128 threads); with the
// paper's WENO faces (three inlined stage bodies) or the shoreline variant's
// (SHORE: one copy of the stage code with the stage a run-time value).
#include "swe_batch.cuh"
#include "swe_launch.h"

namespace swe {

namespace {
constexpr int kShape64 = 1;
using P64 = ShapeP<kShape64>;
constexpr size_t kSmem64 = TileGeom<double, P64::TX, P64::TY>::BYTES;
}  // namespace

template <bool STRIDED, bool SHORE>
__global__ void __launch_bounds__(ShapeP<kShape64>::NT, ShapeP<kShape64>::MINB64)
    batch_kernel_f64(const BatchSlot<double> *slots, BatchCtl *ctl, int k_steps) {
  using P = ShapeP<kShape64>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ Phys sp;
  double *smem = reinterpret_cast<double *>(smem_raw);
  const int nslots = *(volatile int *)&ctl->nslots;
  const int total = *(volatile int *)&ctl->total_items;
  for (int k = 0; k < k_steps; ++k) {
    if constexpr (SHORE) {
#pragma unroll 1
      for (int st = 1; st <= 3; ++st) {
        batch_stage<double, P::TX, P::TY, P::NT, P::S, 0, STRIDED, true>(slots, nslots, total, smem, red, sp, ctl, st);
        if (!grid_barrier(ctl, gridDim.x)) return;
      }
      continue;
    }
    batch_stage<double, P::TX, P::TY, P::NT, P::S, 1, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<double, P::TX, P::TY, P::NT, P::S, 2, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<double, P::TX, P::TY, P::NT, P::S, 3, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
  }
}

int batch64_shape() { return kShape64; }

cudaError_t batch64_resident(bool shore, int *per_sm) {
  int n[2] = {0, 0};
  auto k0 = shore ? batch_kernel_f64<false, true> : batch_kernel_f64<false, false>;
  auto k1 = shore ? batch_kernel_f64<true, true> : batch_kernel_f64<true, false>;
  cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], k0, P64::NT, kSmem64);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], k1, P64::NT, kSmem64);
  *per_sm = n[0] < n[1] ? n[0] : n[1];
  return e;
}

cudaError_t batch64_launch(const BatchSlot<double> *slots, BatchCtl *ctl, int k, int grid, bool strided, bool shore,
                           cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(P64::NT);
  cfg.dynamicSmemBytes = kSmem64;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (shore)
    return strided ? cudaLaunchKernelEx(&cfg, batch_kernel_f64<true, true>, slots, ctl, k)
                   : cudaLaunchKernelEx(&cfg, batch_kernel_f64<false, true>, slots, ctl, k);
  return strided ? cudaLaunchKernelEx(&cfg, batch_kernel_f64<true, false>, slots, ctl, k)
                 : cudaLaunchKernelEx(&cfg, batch_kernel_f64<false, false>, slots, ctl, k);
}

}  // namespace swe
