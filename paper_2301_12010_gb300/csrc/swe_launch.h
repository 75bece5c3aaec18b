// swe_launch.h -- host-side interface between the ABI layer and the kernel
// translation units.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "swe_core.cuh"

namespace swe {

struct TileShape {
  int tx, ty, threads;
};

int num_shapes();
const TileShape *shape(int k);  // k = 1 .. num_shapes()
size_t shape_smem(int k, int elem_bytes);

template <typename T>
cudaError_t prepare_shape(int k);
template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st);

}  // namespace swe
