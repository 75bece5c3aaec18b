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

constexpr int kMassBlocks = 1024;  // partials of the fixed-order mass reduction

// helper kernels (swe_aux.cu)
template <typename T>
cudaError_t import_plane(const void *src, bool src_f64, T *dst, const T *bed_for_depth, double zref, int nx, int ny,
                         int pitch, cudaStream_t st);
template <typename T>
cudaError_t export_plane(const T *src, void *dst, bool dst_f64, const T *bed_for_depth, double zref, int nx, int ny,
                         int pitch, cudaStream_t st);
cudaError_t reset_scalars(DevScalars *sc, double t, double cfl, double t_end, cudaStream_t st);
cudaError_t set_cfl(DevScalars *sc, double cfl, cudaStream_t st);
template <typename T>
cudaError_t state_stats(const Field<T> &fd, const Phys &p, DevScalars *sc, cudaStream_t st);
template <typename T>
cudaError_t mass(const T *ha, const T *bed, double zref, int nx, int ny, int pitch, double area, double *partials,
                 double *out, cudaStream_t st);
float thr32(double thr);

template <typename T>
cudaError_t prepare_shape(int k);
template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st);

}  // namespace swe
