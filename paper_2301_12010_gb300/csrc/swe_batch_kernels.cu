// swe_batch_kernels.cu -- the persistent multi-scenario kernel for one tile
// shape (SWE_SHAPE): k RK3 steps of every live scenario of a batch in one
// cooperative launch, the three stages separated by a bounded grid barrier.
// FP32; two forms, chosen per launch by the host (see batch_kernel_rt).
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

// The same with one copy of the stage code, the stage a run-time value: for
// launches with few tiles per CTA and stage (serving, a single mid-size
// scenario), where three inlined stage bodies keep missing the instruction
// cache; with many tiles per CTA the inlined form above is faster.
template <int K, bool STRIDED>
__global__ void __launch_bounds__(ShapeP<K>::NT, ShapeP<K>::MINB32)
    batch_kernel_rt(const BatchSlot<float> *slots, BatchCtl *ctl, int k_steps) {
  using P = ShapeP<K>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ Phys sp;
  float *smem = reinterpret_cast<float *>(smem_raw);
  const int nslots = *(volatile int *)&ctl->nslots;
  const int total = *(volatile int *)&ctl->total_items;
  for (int k = 0; k < k_steps; ++k) {
#pragma unroll 1
    for (int st = 1; st <= 3; ++st) {
      batch_stage<float, P::TX, P::TY, P::NT, P::S, 0, STRIDED>(slots, nslots, total, smem, red, sp, ctl, st);
      if (!grid_barrier(ctl, gridDim.x)) return;
    }
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
  int n[4] = {0, 0, 0, 0};
  const void *k[4] = {(const void *)batch_kernel<SWE_SHAPE, false>, (const void *)batch_kernel<SWE_SHAPE, true>,
                      (const void *)batch_kernel_rt<SWE_SHAPE, false>, (const void *)batch_kernel_rt<SWE_SHAPE, true>};
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 4 && e == cudaSuccess; ++q)
    e = cudaFuncSetAttribute(k[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[q], k[q], P::NT, kSmem);
  int m = n[0];
  for (int q = 1; q < 4; ++q) m = n[q] < m ? n[q] : m;
  *per_sm = m;
  return e;
}

cudaError_t SWE_CAT(batch_launch_, SWE_SHAPE)(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid,
                                              bool strided, bool small, cudaStream_t st) {
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
  if (small)
    return strided ? cudaLaunchKernelEx(&cfg, batch_kernel_rt<SWE_SHAPE, true>, slots, ctl, k)
                   : cudaLaunchKernelEx(&cfg, batch_kernel_rt<SWE_SHAPE, false>, slots, ctl, k);
  return strided ? cudaLaunchKernelEx(&cfg, batch_kernel<SWE_SHAPE, true>, slots, ctl, k)
                 : cudaLaunchKernelEx(&cfg, batch_kernel<SWE_SHAPE, false>, slots, ctl, k);
}

}  // namespace swe
