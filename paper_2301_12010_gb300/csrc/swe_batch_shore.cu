// swe_batch_shore.cu -- the batch kernel of the shoreline variant
// (hydrostatic-reconstruction faces wherever a WENO stencil meets a dry cell;
// see sweep_strip, SHORE): k RK3 steps of every live scenario in one
// cooperative launch, FP32, one tile shape (96 x 32, 384 threads), one copy
// of the stage code with the stage a run-time value.
#include "swe_batch.cuh"
#include "swe_launch.h"

namespace swe {

namespace {
constexpr int kShoreShape = 7;
using PS = ShapeP<kShoreShape>;
constexpr size_t kSmemS = TileGeom<float, PS::TX, PS::TY>::BYTES;
}  // namespace

template <bool STRIDED>
__global__ void __launch_bounds__(ShapeP<kShoreShape>::NT, 1)
    batch_kernel_shore(const BatchSlot<float> *slots, BatchCtl *ctl, int k_steps) {
  using P = ShapeP<kShoreShape>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ Phys sp;
  float *smem = reinterpret_cast<float *>(smem_raw);
  const int nslots = *(volatile int *)&ctl->nslots;
  const int total = *(volatile int *)&ctl->total_items;
  for (int k = 0; k < k_steps; ++k) {
#pragma unroll 1
    for (int st = 1; st <= 3; ++st) {
      batch_stage<float, P::TX, P::TY, P::NT, P::S, 0, STRIDED, true>(slots, nslots, total, smem, red, sp, ctl, st);
      if (!grid_barrier(ctl, gridDim.x)) return;
    }
  }
}

int batch_shore_shape() { return kShoreShape; }

cudaError_t batch_shore_resident(int *per_sm) {
  int n[2] = {0, 0};
  cudaError_t e = cudaFuncSetAttribute(batch_kernel_shore<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemS);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel_shore<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemS);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], batch_kernel_shore<false>, PS::NT, kSmemS);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], batch_kernel_shore<true>, PS::NT, kSmemS);
  *per_sm = n[0] < n[1] ? n[0] : n[1];
  return e;
}

cudaError_t batch_shore_launch(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, bool strided,
                               cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(PS::NT);
  cfg.dynamicSmemBytes = kSmemS;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return strided ? cudaLaunchKernelEx(&cfg, batch_kernel_shore<true>, slots, ctl, k)
                 : cudaLaunchKernelEx(&cfg, batch_kernel_shore<false>, slots, ctl, k);
}

}  // namespace swe
