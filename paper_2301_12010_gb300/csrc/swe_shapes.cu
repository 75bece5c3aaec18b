// swe_shapes.cu -- the table of compiled tile shapes and the dispatch from a
// shape index to its per-shape kernels.
#include "swe_launch.h"

namespace swe {

static const TileShape kShapes[] = {
#define SWE_ROW(K, TX, TY, NT, S, M32, M64) {TX, TY, NT},
    SWE_SHAPES(SWE_ROW)
#undef SWE_ROW
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int num_shapes() { return kNumShapes; }
const TileShape *shape(int k) { return (k >= 1 && k <= kNumShapes) ? &kShapes[k - 1] : nullptr; }

size_t shape_smem(int k, int elem) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return elem == 8 ? TileGeom<double, TX, TY>::BYTES : TileGeom<float, TX, TY>::BYTES;
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return 0;
}

template <typename T>
cudaError_t prepare_shape(int k) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return prepare_shape_##K<T>();
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t make_maps(int k, const Field<T> &fd, BoxMaps out[3]) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return make_maps_##K<T>(fd, out);
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return cudaErrorInvalidValue;
}

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

template <typename T>
cudaError_t launch_stage(int k, const Field<T> &fd, const Phys &p, DevScalars *sc, int stage, cudaStream_t st,
                         const BoxMaps *maps) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return launch_shape_##K<T>(fd, p, sc, stage, st, maps);
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_resident(int k, int *per_sm) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return batch_resident_##K(per_sm);
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch(int k, const BatchSlot<float> *slots, BatchCtl *ctl, int steps, int grid, bool strided,
                         bool small, cudaStream_t st) {
  switch (k) {
#define SWE_CASE(K, TX, TY, NT, S, M32, M64) \
  case K: return batch_launch_##K(slots, ctl, steps, grid, strided, small, st);
    SWE_SHAPES(SWE_CASE)
#undef SWE_CASE
  }
  return cudaErrorInvalidValue;
}

template cudaError_t prepare_shape<float>(int);
template cudaError_t prepare_shape<double>(int);
template cudaError_t make_maps<float>(int, const Field<float> &, BoxMaps[3]);
template cudaError_t make_maps<double>(int, const Field<double> &, BoxMaps[3]);
template cudaError_t launch_stage<float>(int, const Field<float> &, const Phys &, DevScalars *, int, cudaStream_t,
                                         const BoxMaps *);
template cudaError_t launch_stage<double>(int, const Field<double> &, const Phys &, DevScalars *, int, cudaStream_t,
                                          const BoxMaps *);

}  // namespace swe
