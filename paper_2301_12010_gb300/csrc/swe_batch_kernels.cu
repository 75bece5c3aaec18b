// swe_batch_kernels.cu -- the persistent multi-scenario kernel: k RK3 steps
// of every live scenario of a batch in one cooperative launch, the three
// stages separated by a bounded grid barrier.  FP32, one instantiation per
// tile shape.
#include "swe_batch.h"

namespace swe {

template <int TX, int TY, int NT, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    batch_kernel(const BatchSlot<float> *slots, BatchCtl *ctl, int k_steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ Phys sp;
  float *smem = reinterpret_cast<float *>(smem_raw);
  const int nslots = *(volatile int *)&ctl->nslots;
  const int total = *(volatile int *)&ctl->total_items;
  for (int k = 0; k < k_steps; ++k) {
    batch_stage<float, TX, TY, NT, S, 1>(slots, nslots, total, smem, red, sp);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, TX, TY, NT, S, 2>(slots, nslots, total, smem, red, sp);
    if (!grid_barrier(ctl, gridDim.x)) return;
    batch_stage<float, TX, TY, NT, S, 3>(slots, nslots, total, smem, red, sp);
    if (!grid_barrier(ctl, gridDim.x)) return;
  }
}

template <int TX, int TY, int NT, int S, int MINB>
struct BatchShape {
  static constexpr size_t smem = TileGeom<float, TX, TY>::BYTES;
  static cudaError_t resident(int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<TX, TY, NT, S, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<TX, TY, NT, S, MINB>, NT, smem);
  }
  static cudaError_t launch(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<TX, TY, NT, S, MINB>, slots, ctl, k);
  }
};

using B1 = BatchShape<32, 32, 128, 8, 3>;
using B2 = BatchShape<64, 32, 256, 8, 1>;
using B3 = BatchShape<32, 64, 256, 8, 1>;

cudaError_t batch_resident(int shape, int *per_sm) {
  switch (shape) {
    case 1: return B1::resident(per_sm);
    case 2: return B2::resident(per_sm);
    case 3: return B3::resident(per_sm);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch(int shape, const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, cudaStream_t st) {
  switch (shape) {
    case 1: return B1::launch(slots, ctl, k, grid, st);
    case 2: return B2::launch(slots, ctl, k, grid, st);
    case 3: return B3::launch(slots, ctl, k, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace swe
