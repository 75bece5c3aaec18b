// swe_aux.cu -- small helper kernels shared by the single-scenario and the
// batch paths: host-format conversion, per-state statistics (wave speeds,
// runup), scalar resets and the fixed-order FP64 mass reduction.
#include <cmath>
#include <new>

#include "swe_launch.h"

namespace swe {
namespace {

// Host-format [ny][nx] -> pitched planes.  With bed != nullptr the field is
// a depth h stored as the anomaly ha = h - max(z_ref - b, 0) (in FP64).  CTA
// b takes rows b, b + gridDim.x, ...; the source may be device memory or
// page-locked host memory read across the host link (four loads in flight
// per thread).
template <typename T, typename S>
__global__ void k_import(const S *__restrict__ src, T *__restrict__ dst, const T *__restrict__ bed, double zref,
                         int nx, int ny, int pitch) {
  for (int j = blockIdx.x; j < ny; j += gridDim.x) {
    const S *srow = src + (size_t)j * nx;
    T *drow = dst + (size_t)j * pitch;
    const T *brow = bed ? bed + (size_t)j * pitch : nullptr;
    for (int i0 = threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        v[u] = i < nx ? (double)srow[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < nx) drow[i] = (T)(brow ? v[u] - fmax(zref - (double)brow[i], 0.0) : v[u]);
      }
    }
  }
}

// Pitched planes -> contiguous [ny][nx] (device memory or page-locked host
// memory written across the host link); with bed != nullptr, h = ha + d.
template <typename T, typename S>
__global__ void k_export(const T *__restrict__ src, S *__restrict__ dst, const T *__restrict__ bed, double zref,
                         int nx, int ny, int pitch) {
  for (int j = blockIdx.x; j < ny; j += gridDim.x) {
    const T *srow = src + (size_t)j * pitch;
    const T *brow = bed ? bed + (size_t)j * pitch : nullptr;
    S *drow = dst + (size_t)j * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      double v = (double)srow[i];
      if (brow) v += fmax(zref - (double)brow[i], 0.0);
      drow[i] = (S)v;
    }
  }
}

__global__ void k_set_cfl(DevScalars *sc, double cfl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc->cfl = cfl;
}

__global__ void k_reset(DevScalars *sc, DevPartials *part, double t, double cfl, double t_end) {
  for (int b = threadIdx.x; b < kPartSlots; b += blockDim.x) {
    part->clamp[b] = 0.0;
    part->edge[b] = 0.0;
  }
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double tk = t == t ? t : sc->t;  // NaN: keep the current time
    sc->part = part;
    sc->check = 0ull;
    for (int s = 0; s < 3; ++s) sc->alpha[s][0] = sc->alpha[s][1] = 0ull;
    sc->dt = 0.0;
    sc->t = tk;
    sc->t_step = tk;
    sc->steps = 0;
    sc->runup_now[0] = sc->runup_now[1] = 0ull;
    sc->runup_max = 0ull;
    sc->t_end = t_end;
    sc->cfl = cfl;
    sc->status = 0u;
    sc->running = 0u;
    sc->parity = 1u;  // runup_now of "step -1" lives at parity 1 (steps = 0 -> next writes parity 0)
    sc->active = 1u;
  }
}

// Wave speeds (slot 0) and runup of the current state U^n, with the same
// in-precision arithmetic as the stage epilogue (so that a state written out
// and set again gives the same time step as an uninterrupted run).
template <typename T>
__global__ void k_state_stats(Field<T> fd, Phys p, DevScalars *sc) {
  __shared__ double sm[32][3];
  __shared__ unsigned sbad;
  if (threadIdx.x == 0) sbad = 0u;
  __syncthreads();
  T mx = T(0), my = T(0), ru = T(0);
  bool bad = false;
  const Consts<T> &K = consts<T>(p);
  const size_t n = (size_t)fd.nx * fd.ny;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const size_t j = q / fd.nx, i = q - j * fd.nx;
    const size_t o = j * fd.pitch + i;
    const T b = fd.b[o];
    const T h = fd.h[0][o] + still_depth(b, T(p.z_ref)), hu = fd.hu[0][o], hv = fd.hv[0][o];
    if (!(fabs(h) <= T(3.0e38)) || !(fabs(hu) <= T(3.0e38)) || !(fabs(hv) <= T(3.0e38))) { bad = true; continue; }
    T u = T(0), v = T(0), rr, cel;
    Num<T>::speed(h > T(0) ? h : T(0), K.g, K.sqg, rr, cel);
    if (!Num<T>::below(h, p.h_dry32, p.h_dry)) { u = hu * rr; v = hv * rr; }
    const T sx = fabs(u) + cel, sy = fabs(v) + cel;
    mx = sx > mx ? sx : mx;
    my = sy > my ? sy : my;
    if (!Num<T>::below(h, p.h_wet32, p.h_wet) && b > T(0)) { const T e = h + b; ru = e > ru ? e : ru; }
  }
  mx = warp_max(mx);
  my = warp_max(my);
  ru = warp_max(ru);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) sbad = 1u;
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5][0] = (double)mx;
    sm[threadIdx.x >> 5][1] = (double)my;
    sm[threadIdx.x >> 5][2] = (double)ru;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = sm[0][0], b = sm[0][1], r = sm[0][2];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = fmax(a, sm[w][0]);
      b = fmax(b, sm[w][1]);
      r = fmax(r, sm[w][2]);
    }
    atomicMax(&sc->alpha[0][0], (unsigned long long)__double_as_longlong(a));
    atomicMax(&sc->alpha[0][1], (unsigned long long)__double_as_longlong(b));
    if (r > 0.0) {
      atomicMax(&sc->runup_now[1], (unsigned long long)__double_as_longlong(r));
      atomicMax(&sc->runup_max, (unsigned long long)__double_as_longlong(r));
    }
    if (sbad) atomicOr(&sc->status, ST_NONFINITE);
  }
}

// Mass, pass 1: per-block FP64 partial sums of h over rows, fixed order.
template <typename T>
__global__ void k_mass_partial(const T *__restrict__ ha, const T *__restrict__ bed, double zref, int nx, int ny,
                               int pitch, double *__restrict__ part) {
  __shared__ double sm[32];
  double s = 0.0;
  const size_t n = (size_t)nx * ny;
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  for (size_t q = lo + threadIdx.x; q < hi; q += blockDim.x) {
    const size_t j = q / nx, i = q - j * nx;
    const size_t o = j * pitch + i;
    s += (double)ha[o] + fmax(zref - (double)bed[o], 0.0);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}

// Mass, pass 2: one block sums the partials in a fixed tree order.
__global__ void k_mass_final(const double *__restrict__ part, int n, double area, double *__restrict__ out) {
  __shared__ double sm[1024];
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0] * area;
}

}  // namespace

static int blocks_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

// Conversion grids: four 256-thread CTAs per SM keep enough loads in flight to
// fill the host link, and leave room for a second conversion (an upload and a
// read-back on two streams) to run beside it.
static int conversion_blocks(int ny) {
  static int sms = 0;
  if (sms <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
      (void)cudaGetLastError();
      sms = 152;
    }
  }
  const int cap = 4 * sms;
  return ny < cap ? ny : cap;
}

template <typename T>
cudaError_t import_plane(const void *src, bool src_f64, T *dst, const T *bed_for_depth, double zref, int nx, int ny,
                         int pitch, cudaStream_t st) {
  const int nb = conversion_blocks(ny);
  if (src_f64) k_import<T, double><<<nb, 256, 0, st>>>((const double *)src, dst, bed_for_depth, zref, nx, ny, pitch);
  else k_import<T, T><<<nb, 256, 0, st>>>((const T *)src, dst, bed_for_depth, zref, nx, ny, pitch);
  return cudaGetLastError();
}

template <typename T>
cudaError_t export_plane(const T *src, void *dst, bool dst_f64, const T *bed_for_depth, double zref, int nx, int ny,
                         int pitch, cudaStream_t st) {
  const int nb = conversion_blocks(ny);
  if (dst_f64) k_export<T, double><<<nb, 256, 0, st>>>(src, (double *)dst, bed_for_depth, zref, nx, ny, pitch);
  else k_export<T, T><<<nb, 256, 0, st>>>(src, (T *)dst, bed_for_depth, zref, nx, ny, pitch);
  return cudaGetLastError();
}

const void *pinned_device_ptr(const void *p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || !a0.devicePointer) return nullptr;
  const char *last = (const char *)p + (bytes - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a1.type != cudaMemoryTypeHost || !a1.devicePointer) return nullptr;
  if ((const char *)a1.devicePointer - (const char *)a0.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
  return a0.devicePointer;
}

cudaError_t reset_scalars(DevScalars *sc, DevPartials *part, double t, double cfl, double t_end, cudaStream_t st) {
  k_reset<<<1, 256, 0, st>>>(sc, part, t, cfl, t_end);
  return cudaGetLastError();
}

cudaError_t read_volumes(const DevPartials *part, double *clamp, double *edge, cudaStream_t st) {
  double tot[2] = {0.0, 0.0};
  DevPartials *h = new (std::nothrow) DevPartials;
  if (!h) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpyAsync(h, part, sizeof(DevPartials), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    for (int b = 0; b < kPartSlots; ++b) {  // CTA order
      tot[0] += h->clamp[b];
      tot[1] += h->edge[b];
    }
    if (clamp) *clamp = tot[0];
    if (edge) *edge = tot[1];
  }
  delete h;
  return e;
}

cudaError_t set_cfl(DevScalars *sc, double cfl, cudaStream_t st) {
  k_set_cfl<<<1, 32, 0, st>>>(sc, cfl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t state_stats(const Field<T> &fd, const Phys &p, DevScalars *sc, cudaStream_t st) {
  k_state_stats<T><<<blocks_for((size_t)fd.nx * fd.ny, 256), 256, 0, st>>>(fd, p, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t mass(const T *ha, const T *bed, double zref, int nx, int ny, int pitch, double area, double *partials,
                 double *out, cudaStream_t st) {
  k_mass_partial<T><<<kMassBlocks, 256, 0, st>>>(ha, bed, zref, nx, ny, pitch, partials);
  k_mass_final<<<1, 1024, 0, st>>>(partials, kMassBlocks, area, out);
  return cudaGetLastError();
}

template cudaError_t import_plane<float>(const void *, bool, float *, const float *, double, int, int, int, cudaStream_t);
template cudaError_t import_plane<double>(const void *, bool, double *, const double *, double, int, int, int, cudaStream_t);
template cudaError_t export_plane<float>(const float *, void *, bool, const float *, double, int, int, int, cudaStream_t);
template cudaError_t export_plane<double>(const double *, void *, bool, const double *, double, int, int, int, cudaStream_t);
template cudaError_t state_stats<float>(const Field<float> &, const Phys &, DevScalars *, cudaStream_t);
template cudaError_t state_stats<double>(const Field<double> &, const Phys &, DevScalars *, cudaStream_t);
template cudaError_t mass<float>(const float *, const float *, double, int, int, int, double, double *, double *, cudaStream_t);
template cudaError_t mass<double>(const double *, const double *, double, int, int, int, double, double *, double *, cudaStream_t);

}  // namespace swe
