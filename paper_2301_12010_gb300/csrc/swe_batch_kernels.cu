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

// Templated on the shape index so that every unit's kernel has a distinct name.
template <int K>
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
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 1>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 2>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, P::TX, P::TY, P::NT, P::S, 3>(slots, nslots, total, smem, red, sp, ctl);
    if (!grid_barrier(ctl, gridDim.x)) return;
  }
}

namespace {
constexpr size_t kSmem = TileGeom<float, P::TX, P::TY>::BYTES;
}

#define SWE_CAT2(a, b) a##b
#define SWE_CAT(a, b) SWE_CAT2(a, b)

cudaError_t SWE_CAT(batch_resident_, SWE_SHAPE)(int *per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(batch_kernel<SWE_SHAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<SWE_SHAPE>, P::NT, kSmem);
}

cudaError_t SWE_CAT(batch_launch_, SWE_SHAPE)(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid,
                                              cudaStream_t st) {
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
  return cudaLaunchKernelEx(&cfg, batch_kernel<SWE_SHAPE>, slots, ctl, k);
}

}  // namespace swe
