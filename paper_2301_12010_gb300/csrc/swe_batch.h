// swe_batch.h -- host-side interface of the persistent batch kernel.
#pragma once
#include "swe_launch.h"

namespace swe {

// CTAs per SM of the batch kernel for a tile shape (1-based, as swe_tile_shape).
cudaError_t batch_resident(int shape, int *per_sm);
// One cooperative launch of k RK3 steps over the slot table.
cudaError_t batch_launch(int shape, const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, cudaStream_t st);

}  // namespace swe
