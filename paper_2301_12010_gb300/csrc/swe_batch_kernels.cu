// swe_batch_kernels.cu -- the persistent multi-scenario kernel for one tile
// shape (SWE_SHAPE): k RK3 steps of every live scenario of a batch in one
// cooperative launch, the three stages separated by a bounded grid barrier.
// FP32.
#ifndef SWE_SHAPE
#define SWE_SHAPE 1
#endif
#include "swe_batch.cuh"
#include "swe_launch.h"

namespace swe {

using P = ShapeP<SWE_SHAPE>;

// Templated on the shape index so that every unit's kernel has a distinct
// name, and on the work order (contiguous chunks or strided items).
template <int K, bool STRIDED>
__global__ void __launch_bounds__(ShapeP<K>::NT, ShapeP<K>::MINB32)
    batch_kernel(const BatchSlot<float> *slots, BatchCtl *ctl, int k_steps) {
  using P = ShapeP<K>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ Phys sp;
  float *smem = reinterpret_cast<float *>(smem_raw);
  const int nslots = *(volatile int *)&ctl->nslots;
  const int total = *(volatile int *)&ctl->total_items;
  for (int k = 0; k < k_steps; ++k) {
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 1, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 2, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 3, STRIDED>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
  }
}

namespace {
constexpr size_t kSmem = TileGeom<float, P::TX, P::TY>::BYTES;
}

#define SWE_CAT2(a, b) a##b
#define SWE_CAT(a, b) SWE_CAT2(a, b)

// resident CTAs per SM of both work orders (the smaller, so that one grid
// size suits either launch)
cudaError_t SWE_CAT(batch_resident_, SWE_SHAPE)(int *per_sm) {
  int n[2] = {0, 0};
  cudaError_t e =
      cudaFuncSetAttribute(batch_kernel<SWE_SHAPE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel<SWE_SHAPE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], batch_kernel<SWE_SHAPE, false>, P::NT, kSmem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], batch_kernel<SWE_SHAPE, true>, P::NT, kSmem);
  *per_sm = n[0] < n[1] ? n[0] : n[1];
  return e;
}

cudaError_t SWE_CAT(batch_launch_, SWE_SHAPE)(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid,
                                              bool strided, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(P::NT);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return strided ? cudaLaunchKernelEx(&cfg, batch_kernel<SWE_SHAPE, true>, slots, ctl, k)
                 : cudaLaunchKernelEx(&cfg, batch_kernel<SWE_SHAPE, false>, slots, ctl, k);
}

}  // namespace swe
