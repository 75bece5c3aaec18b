// swe_kernels.cu -- stage kernels of the single-scenario path, one per
// (precision, tile shape, RK stage), plus their launch table.  Compiled once
// per precision (SWE_PREC = 32 or 64) so that the two halves build in
// parallel; the FP32 unit also carries the shape table.
#ifndef SWE_PREC
#define SWE_PREC 32
#endif
#include "swe_core.cuh"
#include "swe_launch.h"

namespace swe {

// Persistent: CTA b handles tiles b, b + gridDim.x, ... of the scenario.
template <typename T, int TX, int TY, int NT, int S, int STAGE, int MINB>
__global__ void __launch_bounds__(NT, MINB) stage_kernel(StageIO<T> io, Phys p, DevScalars *sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RedSmem red;
  stage_persistent<T, TX, TY, NT, S, STAGE>(io, p, sc, reinterpret_cast<T *>(smem_raw), red, blockIdx.x,
                                            gridDim.x, blockIdx.x == 0);
}

template <typename T>
static StageIO<T> stage_io(const Field<T> &fd, int stage) {
  StageIO<T> io;
  const int in = stage - 1, out = stage % 3;
  io.b = fd.b;
  io.ha = fd.h[in];
  io.hu = fd.hu[in];
  io.hv = fd.hv[in];
  io.ha0 = fd.h[0];
  io.hu0 = fd.hu[0];
  io.hv0 = fd.hv[0];
  io.oha = fd.h[out];
  io.ohu = fd.hu[out];
  io.ohv = fd.hv[out];
  io.nx = fd.nx;
  io.ny = fd.ny;
  io.pitch = fd.pitch;
  return io;
}

template <typename T, int TX, int TY, int NT, int S, int MINB>
struct Shape {
  static constexpr size_t smem = TileGeom<T, TX, TY>::BYTES;
  static int resident;  // CTAs per SM, from the occupancy calculator
  static int sms;

  static cudaError_t prepare() {
    cudaError_t e;
    e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 1, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 2, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 3, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nb = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<T, TX, TY, NT, S, 2, MINB>, NT, smem);
    resident = nb > 0 ? nb : 1;
    return e;
  }

  static cudaError_t launch(const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st) {
    const int ntiles = ((fd.nx + TX - 1) / TX) * ((fd.ny + TY - 1) / TY);
    int grid = resident * (sms > 0 ? sms : 1);
    if (grid > ntiles) grid = ntiles;
    const StageIO<T> io = stage_io(fd, stage);
    switch (stage) {
      case 1: stage_kernel<T, TX, TY, NT, S, 1, MINB><<<grid, NT, smem, st>>>(io, p, sc); break;
      case 2: stage_kernel<T, TX, TY, NT, S, 2, MINB><<<grid, NT, smem, st>>>(io, p, sc); break;
      default: stage_kernel<T, TX, TY, NT, S, 3, MINB><<<grid, NT, smem, st>>>(io, p, sc); break;
    }
    return cudaGetLastError();
  }
};
template <typename T, int TX, int TY, int NT, int S, int MINB> int Shape<T, TX, TY, NT, S, MINB>::resident = 1;
template <typename T, int TX, int TY, int NT, int S, int MINB> int Shape<T, TX, TY, NT, S, MINB>::sms = 1;

template <typename T> using Shape1 = Shape<T, 32, 32, 128, 8, sizeof(T) == 8 ? 1 : 3>;
template <typename T> using Shape2 = Shape<T, 64, 32, 256, 8, 1>;
template <typename T> using Shape3 = Shape<T, 32, 64, 256, 8, 1>;

#if SWE_PREC == 32
// Compiled tile shapes: {TX, TY, threads}.  Strips of 8 cells per thread.
static const TileShape kShapes[] = {{32, 32, 128}, {64, 32, 256}, {32, 64, 256}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int num_shapes() { return kNumShapes; }
const TileShape *shape(int k) { return (k >= 1 && k <= kNumShapes) ? &kShapes[k - 1] : nullptr; }

size_t shape_smem(int k, int elem) {
  switch (k) {
    case 1: return elem == 8 ? TileGeom<double, 32, 32>::BYTES : TileGeom<float, 32, 32>::BYTES;
    case 2: return elem == 8 ? TileGeom<double, 64, 32>::BYTES : TileGeom<float, 64, 32>::BYTES;
    case 3: return elem == 8 ? TileGeom<double, 32, 64>::BYTES : TileGeom<float, 32, 64>::BYTES;
  }
  return 0;
}
#endif

template <typename T>
cudaError_t prepare_shape(int k) {
  switch (k) {
    case 1: return Shape1<T>::prepare();
    case 2: return Shape2<T>::prepare();
    case 3: return Shape3<T>::prepare();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st) {
  switch (k) {
    case 1: return Shape1<T>::launch(fd, p, sc, stage, st);
    case 2: return Shape2<T>::launch(fd, p, sc, stage, st);
    case 3: return Shape3<T>::launch(fd, p, sc, stage, st);
  }
  return cudaErrorInvalidValue;
}

#if SWE_PREC == 32
template cudaError_t prepare_shape<float>(int);
template cudaError_t launch_stage<float>(int, const Field<float> &, const Phys &, DevScalars *, int, cudaStream_t);
#else
template cudaError_t prepare_shape<double>(int);
template cudaError_t launch_stage<double>(int, const Field<double> &, const Phys &, DevScalars *, int, cudaStream_t);
#endif

}  // namespace swe
