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

template <typename T, int TX, int TY, int NT, int S, int STAGE, int MINB>
__global__ void __launch_bounds__(NT, MINB) stage_kernel(Field<T> fd, Phys p, DevScalars *sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RedSmem red;
  stage_tile<T, TX, TY, NT, S, STAGE>(fd, p, sc, blockIdx.x * TX, blockIdx.y * TY, reinterpret_cast<T *>(smem_raw),
                                      red, blockIdx.x == 0 && blockIdx.y == 0);
}

template <typename T, int TX, int TY, int NT, int S, int MINB>
static cudaError_t launch_stages(const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st) {
  constexpr size_t smem = sizeof(T) * TileGeom<TX, TY>::ELEMS;
  const dim3 grid((fd.nx + TX - 1) / TX, (fd.ny + TY - 1) / TY);
  switch (stage) {
    case 1: stage_kernel<T, TX, TY, NT, S, 1, MINB><<<grid, NT, smem, st>>>(fd, p, sc); break;
    case 2: stage_kernel<T, TX, TY, NT, S, 2, MINB><<<grid, NT, smem, st>>>(fd, p, sc); break;
    default: stage_kernel<T, TX, TY, NT, S, 3, MINB><<<grid, NT, smem, st>>>(fd, p, sc); break;
  }
  return cudaGetLastError();
}

template <typename T, int TX, int TY, int NT, int S, int MINB>
static cudaError_t prepare(int) {
  constexpr size_t smem = sizeof(T) * TileGeom<TX, TY>::ELEMS;
  cudaError_t e;
  e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 1, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 2, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, S, 3, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#if SWE_PREC == 32
// Compiled tile shapes: {TX, TY, threads}.  Strips of 8 cells per thread.
static const TileShape kShapes[] = {{32, 32, 128}, {64, 32, 256}, {32, 64, 256}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int num_shapes() { return kNumShapes; }
const TileShape *shape(int k) { return (k >= 1 && k <= kNumShapes) ? &kShapes[k - 1] : nullptr; }

size_t shape_smem(int k, int elem) {
  switch (k) {
    case 1: return (size_t)elem * TileGeom<32, 32>::ELEMS;
    case 2: return (size_t)elem * TileGeom<64, 32>::ELEMS;
    case 3: return (size_t)elem * TileGeom<32, 64>::ELEMS;
  }
  return 0;
}
#endif

template <typename T>
cudaError_t prepare_shape(int k) {
  constexpr bool D = sizeof(T) == 8;
  switch (k) {
    case 1: return prepare<T, 32, 32, 128, 8, D ? 2 : 4>(0);
    case 2: return prepare<T, 64, 32, 256, 8, D ? 1 : 2>(0);
    case 3: return prepare<T, 32, 64, 256, 8, D ? 1 : 2>(0);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st) {
  constexpr bool D = sizeof(T) == 8;
  switch (k) {
    case 1: return launch_stages<T, 32, 32, 128, 8, D ? 2 : 4>(fd, p, sc, stage, st);
    case 2: return launch_stages<T, 64, 32, 256, 8, D ? 1 : 2>(fd, p, sc, stage, st);
    case 3: return launch_stages<T, 32, 64, 256, 8, D ? 1 : 2>(fd, p, sc, stage, st);
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
