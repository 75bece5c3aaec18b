// swe_launch.h -- host-side interface between the ABI layer and the kernel
// translation units.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "swe_batch.cuh"
#include "swe_core.cuh"

namespace swe {

struct TileShape {
  int tx, ty, threads;
};

// Compiled tile shapes: (index, TX, TY, threads, strip length S, CTAs per SM
// asked of the register allocator in FP32, in FP64).  One translation unit
// per (precision, shape) builds the stage kernels, one per shape the batch
// kernel.
#define SWE_SHAPES(X)              \
  X(1, 32, 32, 128, 8, 3, 2)       \
  X(2, 64, 32, 256, 8, 1, 1)       \
  X(3, 32, 64, 256, 8, 1, 1)       \
  X(4, 32, 32, 128, 8, 2, 1)       \
  X(5, 64, 64, 256, 16, 1, 1)      \
  X(6, 64, 48, 384, 8, 1, 1)       \
  X(7, 96, 32, 384, 8, 1, 1)       \
  X(8, 64, 64, 512, 8, 1, 1)       \
  X(9, 128, 32, 512, 8, 1, 1)      \
  X(10, 64, 24, 192, 8, 2, 1)      \
  X(11, 96, 16, 192, 8, 2, 1)

template <int K>
struct ShapeP;
#define SWE_PICK(K, TX_, TY_, NT_, S_, M32_, M64_)                                                   \
  template <>                                                                                    \
  struct ShapeP<K> {                                                                             \
    static constexpr int TX = TX_, TY = TY_, NT = NT_, S = S_, MINB32 = M32_, MINB64 = M64_;    \
  };
SWE_SHAPES(SWE_PICK)
#undef SWE_PICK

#define SWE_DECL(K, TX_, TY_, NT_, S_, M32_, M64_)                                                   \
  template <typename T>                                                                          \
  cudaError_t prepare_shape_##K();                                                               \
  template <typename T>                                                                          \
  cudaError_t launch_shape_##K(const Field<T> &fd, const Phys &p, DevScalars *sc, int stage,      \
                               cudaStream_t st, const BoxMaps *maps);                            \
  template <typename T>                                                                          \
  cudaError_t make_maps_##K(const Field<T> &fd, BoxMaps out[3]);                                 \
  cudaError_t batch_resident_##K(int *per_sm);                                                   \
  cudaError_t batch_launch_##K(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, bool strided, \
                               bool small, cudaStream_t st);
SWE_SHAPES(SWE_DECL)
#undef SWE_DECL

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
// Device-accessible address of a host array of `bytes` bytes when its first
// and last bytes lie in page-locked memory mapped for the device (cudaHostAlloc,
// cudaHostRegister, a pinned torch tensor) at the same offset, i.e. one pinned
// allocation or registration: the conversion kernels then read or write it
// directly across the host link, with no staging copy.  nullptr otherwise
// (pageable memory takes the staging copy).
const void *pinned_device_ptr(const void *p, size_t bytes);
// Reset a scenario's device scalars (time t, or the current time if t is
// NaN; CFL number; horizon t_end) and clear its per-CTA partials `part`,
// which the scalars then point to.
cudaError_t reset_scalars(DevScalars *sc, DevPartials *part, double t, double cfl, double t_end, cudaStream_t st);
cudaError_t set_cfl(DevScalars *sc, double cfl, cudaStream_t st);
// A scenario's clamp and edge volumes: its per-CTA FP64 running sums added
// in CTA order (deterministic).  Synchronises the stream.
cudaError_t read_volumes(const DevPartials *part, double *clamp, double *edge, cudaStream_t st);
template <typename T>
cudaError_t state_stats(const Field<T> &fd, const Phys &p, DevScalars *sc, cudaStream_t st);
template <typename T>
cudaError_t mass(const T *ha, const T *bed, double zref, int nx, int ny, int pitch, double area, double *partials,
                 double *out, cudaStream_t st);
float thr32(double thr);

// The fused-step variant (swe_fused.cu): one kernel per RK3 step reading the
// planes of set `from` (0 or 1) and writing set 1 - from, between a step
// preparation and a step finishing kernel (one thread each).  With ev != NULL,
// events ev[0..3] are recorded before the preparation, before and after the
// step kernel, and after the finishing kernel.
template <typename T>
cudaError_t prepare_fused();
template <typename T>
cudaError_t launch_fused(const Field<T> &fd, int from, const Phys &p, DevScalars *sc, double margin,
                         cudaStream_t st, cudaEvent_t *ev = nullptr);
size_t fused_smem(int elem_bytes);

// The shoreline variant's stage kernels (swe_shore.cu): one compiled tile
// shape per precision (shore_shape), the handle's tensor maps built for it.
int shore_shape(int elem_bytes);
template <typename T>
cudaError_t prepare_shore();
template <typename T>
cudaError_t launch_shore(const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st,
                         const BoxMaps *maps);

template <typename T>
cudaError_t prepare_shape(int k);
// Tensor maps of the halo-box copies for shape k: out[s] covers the input
// planes of RK stage s + 1 (ha, hu, hv of U^n, U1, U2 and the bed).
template <typename T>
cudaError_t make_maps(int k, const Field<T> &fd, BoxMaps out[3]);
template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st,
                         const BoxMaps *maps);
// cuTensorMapEncodeTiled from the driver (resolved once through the runtime;
// nullptr if unavailable)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();
// The shoreline variant's batch kernel (swe_batch_shore.cu): FP32, one
// compiled tile shape.
int batch_shore_shape();
cudaError_t batch_shore_resident(int *per_sm);
cudaError_t batch_shore_launch(const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, bool strided,
                               cudaStream_t st);
// The FP64 batch kernel (swe_batch64_kernels.cu): one compiled tile shape,
// with the paper's faces or (shore) the shoreline variant's.
int batch64_shape();
cudaError_t batch64_resident(bool shore, int *per_sm);
cudaError_t batch64_launch(const BatchSlot<double> *slots, BatchCtl *ctl, int k, int grid, bool strided, bool shore,
                           cudaStream_t st);
// CTAs per SM of the batch kernel for a shape, and one cooperative launch
// (small: the form with one run-time-stage copy of the stage code, for
// launches with few tiles per CTA and stage).
constexpr int kSmallItemsPerCta = 24;  // below this many tiles per CTA and stage a launch is small
cudaError_t batch_resident(int shape, int *per_sm);
cudaError_t batch_launch(int shape, const BatchSlot<float> *slots, BatchCtl *ctl, int k, int grid, bool strided,
                         bool small, cudaStream_t st);

}  // namespace swe
