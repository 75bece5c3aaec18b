// swe_kernels.cu -- persistent stage kernels of the single-scenario path for
// one precision (SWE_PREC = 32 or 64) and one tile shape (SWE_SHAPE, see
// SWE_SHAPES in swe_launch.h); the build compiles one unit per pair.
#ifndef SWE_PREC
#define SWE_PREC 32
#endif
#ifndef SWE_SHAPE
#define SWE_SHAPE 1
#endif
#include "swe_core.cuh"
#include "swe_launch.h"

namespace swe {

#if SWE_PREC == 32
using Real = float;
#else
using Real = double;
#endif
using P = ShapeP<SWE_SHAPE>;
constexpr int MINB = SWE_PREC == 32 ? P::MINB32 : P::MINB64;

// Persistent: CTA b handles tiles b, b + gridDim.x, ... of the scenario.
// Templated on the shape index and precision so that every unit's kernels have
// distinct names.
template <int K, typename R, int STAGE>
__global__ void __launch_bounds__(ShapeP<K>::NT, MINB)
    stage_kernel(StageIO<R> io, const __grid_constant__ BoxMaps maps, Phys p, DevScalars *sc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  using Q = ShapeP<K>;
  stage_persistent<R, Q::TX, Q::TY, Q::NT, Q::S, STAGE>(io, maps, p, sc, reinterpret_cast<R *>(smem_raw), red,
                                                        blockIdx.x, gridDim.x, blockIdx.x == 0 && !p.follower);
}

namespace {
constexpr size_t kSmem = TileGeom<Real, P::TX, P::TY>::BYTES;
int g_resident = 1, g_sms = 1;
}  // namespace

#define SWE_CAT2(a, b) a##b
#define SWE_CAT(a, b) SWE_CAT2(a, b)

template <>
cudaError_t SWE_CAT(prepare_shape_, SWE_SHAPE)<Real>() {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<SWE_SHAPE, Real, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<SWE_SHAPE, Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<SWE_SHAPE, Real, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, nb = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<SWE_SHAPE, Real, 2>, P::NT, kSmem);
  g_resident = nb > 0 ? nb : 1;
  return e;
}

template <>
cudaError_t SWE_CAT(launch_shape_, SWE_SHAPE)<Real>(const Field<Real> &fd, const Phys &p, DevScalars *sc, int stage,
                                                     cudaStream_t st, const BoxMaps *maps) {
  const int ntiles = ((fd.nx + P::TX - 1) / P::TX) * ((fd.ny + P::TY - 1) / P::TY);
  int grid = g_resident * (g_sms > 0 ? g_sms : 1);
  if (grid > ntiles) grid = ntiles;
  if (grid > kPartSlots) return cudaErrorInvalidConfiguration;  // one partial slot per CTA
  const StageIO<Real> io = io_of(fd, stage);
  const BoxMaps &m = maps[stage - 1];
  switch (stage) {
    case 1: stage_kernel<SWE_SHAPE, Real, 1><<<grid, P::NT, kSmem, st>>>(io, m, p, sc); break;
    case 2: stage_kernel<SWE_SHAPE, Real, 2><<<grid, P::NT, kSmem, st>>>(io, m, p, sc); break;
    default: stage_kernel<SWE_SHAPE, Real, 3><<<grid, P::NT, kSmem, st>>>(io, m, p, sc); break;
  }
  return cudaGetLastError();
}

// 2D tensor maps over the planes (nx x ny elements, row pitch in bytes), one
// box P x BH per copy; elements outside the plane read as zero.
template <>
cudaError_t SWE_CAT(make_maps_, SWE_SHAPE)<Real>(const Field<Real> &fd, BoxMaps out[3]) {
  using G = TileGeom<Real, P::TX, P::TY>;
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const CUtensorMapDataType dtype = sizeof(Real) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  // a strip's maps also cover its halo rows (the kernels offset y by halo_rows)
  const cuuint64_t dims[2] = {(cuuint64_t)fd.nx, (cuuint64_t)(fd.ny + 2 * fd.halo)};
  const size_t hoff = (size_t)fd.halo * fd.pitch;
  const cuuint64_t strides[1] = {(cuuint64_t)fd.pitch * sizeof(Real)};
  const cuuint32_t box[2] = {(cuuint32_t)G::P, (cuuint32_t)G::BH};
  const cuuint32_t estr[2] = {1u, 1u};
  for (int s = 0; s < 3; ++s) {
    const void *planes[4] = {fd.h[s] - hoff, fd.hu[s] - hoff, fd.hv[s] - hoff, fd.b - hoff};
    for (int f = 0; f < 4; ++f) {
      const CUresult r = enc(&out[s].m[f], dtype, 2, const_cast<void *>(planes[f]), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

}  // namespace swe
