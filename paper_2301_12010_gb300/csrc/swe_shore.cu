// swe_shore.cu -- stage kernels of the shoreline variant: the stage kernels of
// swe_kernels.cu with hydrostatic-reconstruction faces wherever a WENO stencil
// meets a dry cell (see sweep_strip, SHORE).  One tile shape per precision:
// 96 x 32 (384 threads) in FP32, 64 x 32 (256 threads) in FP64.
#include "swe_core.cuh"
#include "swe_launch.h"

namespace swe {

template <typename R> struct ShoreShape;
template <> struct ShoreShape<float> { static constexpr int K = 7; };
template <> struct ShoreShape<double> { static constexpr int K = 2; };

template <typename R, int STAGE>
__global__ void __launch_bounds__(ShapeP<ShoreShape<R>::K>::NT, 1)
    stage_kernel_shore(StageIO<R> io, const __grid_constant__ BoxMaps maps, Phys p, DevScalars *sc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  using Q = ShapeP<ShoreShape<R>::K>;
  stage_persistent<R, Q::TX, Q::TY, Q::NT, Q::S, STAGE, true>(io, maps, p, sc, reinterpret_cast<R *>(smem_raw), red,
                                                               blockIdx.x, gridDim.x,
                                                               blockIdx.x == 0 && !p.follower);
}

namespace {
int g_resident[2] = {0, 0}, g_sms[2] = {0, 0};  // [0] FP32, [1] FP64
template <typename R> constexpr int pidx() { return sizeof(R) == 8 ? 1 : 0; }
template <typename R> size_t smem_of() {
  using Q = ShapeP<ShoreShape<R>::K>;
  return TileGeom<R, Q::TX, Q::TY>::BYTES;
}
}  // namespace

int shore_shape(int elem_bytes) { return elem_bytes == 8 ? ShoreShape<double>::K : ShoreShape<float>::K; }

template <typename R>
cudaError_t prepare_shore() {
  const int bytes = (int)smem_of<R>();
  cudaError_t e = cudaFuncSetAttribute(stage_kernel_shore<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel_shore<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel_shore<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int dev = 0, nb = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel_shore<R, 2>, ShapeP<ShoreShape<R>::K>::NT,
                                                      smem_of<R>());
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  g_resident[pidx<R>()] = nb;
  g_sms[pidx<R>()] = sms;
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_shore(const Field<R> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st,
                         const BoxMaps *maps) {
  using Q = ShapeP<ShoreShape<R>::K>;
  if (g_resident[pidx<R>()] < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = ((fd.nx + Q::TX - 1) / Q::TX) * ((fd.ny + Q::TY - 1) / Q::TY);
  int grid = g_resident[pidx<R>()] * g_sms[pidx<R>()];
  if (grid > ntiles) grid = ntiles;
  if (grid > kPartSlots) return cudaErrorInvalidConfiguration;  // one partial slot per CTA
  const StageIO<R> io = io_of(fd, stage);
  const BoxMaps &m = maps[stage - 1];
  const size_t bytes = smem_of<R>();
  switch (stage) {
    case 1: stage_kernel_shore<R, 1><<<grid, Q::NT, bytes, st>>>(io, m, p, sc); break;
    case 2: stage_kernel_shore<R, 2><<<grid, Q::NT, bytes, st>>>(io, m, p, sc); break;
    default: stage_kernel_shore<R, 3><<<grid, Q::NT, bytes, st>>>(io, m, p, sc); break;
  }
  return cudaGetLastError();
}

template cudaError_t prepare_shore<float>();
template cudaError_t prepare_shore<double>();
template cudaError_t launch_shore<float>(const Field<float> &, const Phys &, DevScalars *, int, cudaStream_t,
                                         const BoxMaps *);
template cudaError_t launch_shore<double>(const Field<double> &, const Phys &, DevScalars *, int, cudaStream_t,
                                          const BoxMaps *);

}  // namespace swe
