// swe_api.cu -- C ABI of the single-scenario solver (include/swe.h): handle
// life cycle, host/device transfers, the CUDA-graph step loop, diagnostics
// and the small helper kernels (format conversion, state statistics, mass).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "../../include/swe.h"
#include "swe_launch.h"
#include "swe_trace.h"
#include "swe_alloc.h"

using namespace swe;


namespace swe {
namespace {
std::atomic<int> g_alloc_countdown{0};  // > 0: allocations left before the one that fails
}
bool alloc_should_fail() {
  int n = g_alloc_countdown.load();
  while (n > 0 && !g_alloc_countdown.compare_exchange_weak(n, n - 1)) {
  }
  return n == 1;
}

float thr32(double thr) {
  // smallest float f with (double)f >= thr: comparing h < f in FP32 is the
  // same predicate as (double)h < thr
  float f = (float)thr;
  if ((double)f < thr) f = std::nextafter(f, INFINITY);
  while ((double)std::nextafter(f, -INFINITY) >= thr) f = std::nextafter(f, -INFINITY);
  return f;
}
}  // namespace swe

struct swe_handle {
  int nx = 0, ny = 0, pitch = 0;
  double dx = 0, dy = 0;
  swe_params prm{};
  Phys phys{};
  int prec = SWE_F32;
  int tile = 1;
  size_t elem = 4;
  cudaStream_t stream = nullptr;  // caller's stream (may be the legacy default)
  cudaStream_t cap = nullptr;     // private stream used for graph capture
  void *mem = nullptr;            // one device allocation for all planes
  void *b = nullptr;
  void *h[3] = {}, *hu[3] = {}, *hv[3] = {};
  double *staging = nullptr;      // ny*nx doubles: host-format transfers
  DevScalars *sc = nullptr;
  DevPartials *cta = nullptr;     // per-CTA partials of the clamp and edge volumes
  double *partials = nullptr;     // kMassBlocks + 1 (last: mass result)
  BoxMaps maps[3] = {};           // tensor maps of the halo-box copies, per RK stage
  cudaGraphExec_t graph = nullptr;   // one step (fused_step: two steps, plane sets 0 -> 1 -> 0)
  cudaGraphExec_t graph1 = nullptr;  // fused_step: one step 0 -> 1 and the copy of set 1 back to set 0
  double cfl_dev = -1.0;          // CFL value last written to the device scalars
  double t_end = 0.0;             // horizon (swe_set_horizon), kept when the state changes
  int sticky = SWE_OK;            // first host-visible error
  // asynchronous read-back (swe_get_state_async), two slots used in turn:
  // U^n is converted into slot k's FP64 planes on the caller's stream and a
  // copy engine carries them to the host on the read-back stream, so that the
  // next step and conversion need not wait for this copy
  double *xstage[2] = {nullptr, nullptr};  // three FP64 [ny][nx] planes each: the host format
  cudaStream_t xfer = nullptr;             // read-back stream (non-blocking)
  cudaEvent_t ev_conv[2] = {nullptr, nullptr};  // slot converted
  cudaEvent_t ev_done[2] = {nullptr, nullptr};  // slot's copy to the host finished (slot free again)
  bool pending[2] = {false, false};
  int xk = 0;  // slot of the next read-back
  // asynchronous upload (swe_set_state_async), two slots used in turn: copy
  // engines carry the host FP64 state into slot k on the upload stream; the
  // conversion into U^n runs on the caller's stream after it
  double *instage[2] = {nullptr, nullptr};  // three FP64 [ny][nx] planes each
  cudaStream_t upl = nullptr;               // upload stream (non-blocking)
  cudaEvent_t ev_up[2] = {nullptr, nullptr};    // upload landed
  cudaEvent_t ev_used[2] = {nullptr, nullptr};  // slot converted (free for the upload after next)
  bool up_used[2] = {false, false};
  int uk = 0;  // slot of the next upload
};

namespace {

int fail(swe_handle *s, int code) {
  if (s && s->sticky == SWE_OK) s->sticky = code;
  return code;
}

int cuda_check(swe_handle *s, cudaError_t e) {
  if (e == cudaSuccess) return SWE_OK;
  (void)cudaGetLastError();
  return fail(s, e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA);
}

template <typename T>
Field<T> field_of(const swe_handle *s) {
  Field<T> f;
  f.b = (const T *)s->b;
  for (int k = 0; k < 3; ++k) {
    f.h[k] = (T *)s->h[k];
    f.hu[k] = (T *)s->hu[k];
    f.hv[k] = (T *)s->hv[k];
  }
  f.nx = s->nx;
  f.ny = s->ny;
  f.pitch = s->pitch;
  f.halo = 0;
  return f;
}

// The plane set 1 (U1 of the stage kernels) copied back into set 0 (U^n).
cudaError_t copy_back(swe_handle *s, cudaStream_t st) {
  const size_t bytes = (size_t)s->pitch * s->ny * s->elem;
  cudaError_t e = cudaMemcpyAsync(s->h[0], s->h[1], bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->hu[0], s->hu[1], bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->hv[0], s->hv[1], bytes, cudaMemcpyDeviceToDevice, st);
  return e;
}

// One fused step from plane set `from` to 1 - from.
cudaError_t enqueue_fused(swe_handle *s, int from, cudaStream_t st, cudaEvent_t *ev = nullptr) {
  return s->prec == SWE_F64
             ? launch_fused<double>(field_of<double>(s), from, s->phys, s->sc, s->prm.alpha_margin, st, ev)
             : launch_fused<float>(field_of<float>(s), from, s->phys, s->sc, s->prm.alpha_margin, st, ev);
}

// One stage kernel: the paper's WENO faces, or the shoreline variant's.
cudaError_t launch_one_stage(swe_handle *s, int stage, cudaStream_t st) {
  if (s->prm.shore)
    return s->prec == SWE_F64 ? launch_shore<double>(field_of<double>(s), s->phys, s->sc, stage, st, s->maps)
                              : launch_shore<float>(field_of<float>(s), s->phys, s->sc, stage, st, s->maps);
  return s->prec == SWE_F64 ? launch_stage<double>(s->tile, field_of<double>(s), s->phys, s->sc, stage, st, s->maps)
                            : launch_stage<float>(s->tile, field_of<float>(s), s->phys, s->sc, stage, st, s->maps);
}

// What one replay of s->graph does: one step of three stage kernels, or (fused
// step) two fused steps that end in plane set 0 again.
cudaError_t enqueue_step(swe_handle *s, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (s->prm.fused_step) {
    e = enqueue_fused(s, 0, st);
    if (e == cudaSuccess) e = enqueue_fused(s, 1, st);
    return e;
  }
  for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage) e = launch_one_stage(s, stage, st);
  return e;
}

int device_status(swe_handle *s) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, &s->sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  if (st & ST_TIMEOUT) return SWE_ETIMEOUT;
  if (st & ST_NONFINITE) return SWE_ENONFINITE;
  if (st & ST_DRY) return SWE_EINVAL;
  return SWE_OK;
}

// Host FP64 [ny][nx] -> device plane; depth fields (is_depth) are stored as
// the anomaly ha (the bed must already be on the device).
// A page-locked host array is read by the conversion kernel directly (one
// pass across the host link); pageable memory goes through the staging plane,
// and so does any array while an asynchronous read-back is in flight: the
// copy engines carry both directions of the link at once, a kernel reading
// host memory beside them does not.
bool readback_in_flight(swe_handle *s) {
  for (int k = 0; k < 2; ++k) {
    if (!s->pending[k]) continue;
    const cudaError_t e = cudaEventQuery(s->ev_done[k]);
    if (e == cudaErrorNotReady) {
      (void)cudaGetLastError();
      return true;
    }
  }
  return false;
}

int upload_field(swe_handle *s, const double *src, void *dst, bool is_depth) {
  const size_t bytes = sizeof(double) * (size_t)s->nx * s->ny;
  const void *in = readback_in_flight(s) ? nullptr : pinned_device_ptr(src, bytes);
  cudaError_t e = cudaSuccess;
  if (!in) {
    e = cudaMemcpyAsync(s->staging, src, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_check(s, e);
    in = s->staging;
  }
  if (s->prec == SWE_F64)
    e = import_plane<double>(in, true, (double *)dst, is_depth ? (const double *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  else
    e = import_plane<float>(in, true, (float *)dst, is_depth ? (const float *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  return cuda_check(s, e);
}

// The converse: the conversion kernel writes a page-locked host array
// directly; a pageable one is filled from the staging plane.
int download_field(swe_handle *s, const void *src, double *dst, bool is_depth) {
  const size_t bytes = sizeof(double) * (size_t)s->nx * s->ny;
  void *out = const_cast<void *>(pinned_device_ptr(dst, bytes));
  void *target = out ? out : s->staging;
  cudaError_t e;
  if (s->prec == SWE_F64)
    e = export_plane<double>((const double *)src, target, true, is_depth ? (const double *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  else
    e = export_plane<float>((const float *)src, target, true, is_depth ? (const float *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  if (e == cudaSuccess && !out) e = cudaMemcpyAsync(dst, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream);
  return cuda_check(s, e);
}

// Caller device arrays (handle precision, contiguous) <-> planes.
int import_device(swe_handle *s, const void *src, void *dst, bool is_depth) {
  cudaError_t e;
  if (s->prec == SWE_F64)
    e = import_plane<double>(src, false, (double *)dst, is_depth ? (const double *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  else
    e = import_plane<float>(src, false, (float *)dst, is_depth ? (const float *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  return cuda_check(s, e);
}

int export_device(swe_handle *s, const void *src, void *dst, bool is_depth) {
  cudaError_t e;
  if (s->prec == SWE_F64)
    e = export_plane<double>((const double *)src, dst, false, is_depth ? (const double *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  else
    e = export_plane<float>((const float *)src, dst, false, is_depth ? (const float *)s->b : nullptr, s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  return cuda_check(s, e);
}

int after_state_change(swe_handle *s) {
  // scalars: keep t, clear everything else; then wave speeds + runup of U^n
  double t = 0.0;
  cudaError_t e = cudaMemcpyAsync(&t, &s->sc->t, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  e = reset_scalars(s->sc, s->cta, t, s->cfl_dev > 0 ? s->cfl_dev : 0.4, s->t_end, s->stream);
  if (e == cudaSuccess)
    e = s->prec == SWE_F64 ? state_stats<double>(field_of<double>(s), s->phys, s->sc, s->stream)
                           : state_stats<float>(field_of<float>(s), s->phys, s->sc, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (s->cfl_dev <= 0) s->cfl_dev = 0.4;
  return cuda_check(s, e);
}

}  // namespace

namespace swe {
// Parameters a solver (or a batch, under its own extra rules) accepts.
bool valid_params(const swe_params *p) {
  if (!p) return false;
  if (p->precision != SWE_F32 && p->precision != SWE_F64) return false;
  for (int k = 0; k < 4; ++k)
    if (p->bc[k] < SWE_BC_WALL || p->bc[k] > SWE_BC_PERIODIC) return false;
  if ((p->bc[0] == SWE_BC_PERIODIC) != (p->bc[1] == SWE_BC_PERIODIC)) return false;
  if ((p->bc[2] == SWE_BC_PERIODIC) != (p->bc[3] == SWE_BC_PERIODIC)) return false;
  if (p->bc[1] == SWE_BC_INFLOW || p->bc[2] == SWE_BC_INFLOW || p->bc[3] == SWE_BC_INFLOW) return false;
  if (p->bc[0] == SWE_BC_INFLOW && !(p->inflow_depth > 0.0 && p->inflow_period > 0.0)) return false;
  if (!(p->g > 0.0) || !(p->manning_n >= 0.0) || !(p->h_dry >= 0.0) || !(p->h_wet >= 0.0) || !(p->h_film >= 0.0) ||
      !(p->weno_eps > 0.0))
    return false;
  if (!std::isfinite(p->z_ref) || !std::isfinite(p->fixed_dt)) return false;
  if (p->tile < 0 || p->tile > num_shapes()) return false;
  if (p->fused_step != 0 && p->fused_step != 1) return false;
  if (p->shore != 0 && p->shore != 1) return false;
  if (p->shore && p->fused_step) return false;  // the fused step has WENO faces only
  if (p->shore && p->tile != 0 && p->tile != shore_shape(p->precision == SWE_F64 ? 8 : 4)) return false;
  if (p->fused_step) {
    for (int k = 0; k < 4; ++k)
      if (p->bc[k] == SWE_BC_PERIODIC) return false;  // the fused step has wall and inflow ghosts only
    if (!(p->alpha_margin >= 1.0) || !std::isfinite(p->alpha_margin)) return false;
  }
  return true;
}
}  // namespace swe

extern "C" {

void swe_params_default(swe_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->g = 9.81;
  p->manning_n = 0.0;
  p->h_dry = 1e-5;
  p->h_wet = 1e-3;
  p->h_film = 1e-3;
  p->weno_eps = 1e-6;
  p->fixed_dt = 0.0;
  p->z_ref = 0.0;
  for (int k = 0; k < 4; ++k) p->bc[k] = SWE_BC_WALL;
  p->precision = SWE_F32;
  p->tile = 0;
  p->fused_step = 0;
  p->alpha_margin = 1.1;
  p->stream = nullptr;
}

const char *swe_strerror(int code) {
  switch (code) {
    case SWE_OK: return "ok";
    case SWE_EINVAL: return "invalid argument (or CFL time step undefined: dry, still domain)";
    case SWE_ENOMEM: return "out of memory";
    case SWE_ECUDA: return "CUDA error";
    case SWE_ENONFINITE: return "non-finite value in the state";
    case SWE_ETIMEOUT: return "bounded device wait expired";
    case SWE_EBUDGET: return "HBM budget exceeded";
    case SWE_EFULL: return "no free slot";
  }
  return "unknown status";
}

int swe_debug_fail_alloc(int32_t n) {
  if (n < 0) return SWE_EINVAL;
  g_alloc_countdown.store(n);
  return SWE_OK;
}

int swe_tile_count(void) { return num_shapes(); }

int swe_checked_build(void) {
#ifdef SWE_CHECKED
  return 1;
#else
  return 0;
#endif
}

int swe_check_status(swe_handle *s, uint64_t *word) {
  if (!s || !word) return SWE_EINVAL;
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, &s->sc->check, sizeof(w), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  *word = (uint64_t)w;
  return SWE_OK;
}

int swe_tile_shape(int k, int32_t *tx, int32_t *ty, int32_t *threads) {
  const TileShape *t = shape(k);
  if (!t) return SWE_EINVAL;
  if (tx) *tx = t->tx;
  if (ty) *ty = t->ty;
  if (threads) *threads = t->threads;
  return SWE_OK;
}

int swe_create(const swe_grid *grid, double dx, double dy, const double *bathymetry, const swe_params *params,
               swe_handle **out) {
  const TraceRange trace("swe_create");
  if (out) *out = nullptr;
  if (!grid || !out || !bathymetry || !valid_params(params)) return SWE_EINVAL;
  if (grid->nx < 3 || grid->ny < 3 || !(dx > 0.0) || !(dy > 0.0)) return SWE_EINVAL;
  if ((long long)grid->nx * grid->ny > (1ll << 31)) return SWE_EINVAL;
  swe_handle *s = new (std::nothrow) swe_handle();
  if (!s) return SWE_ENOMEM;
  s->nx = grid->nx;
  s->ny = grid->ny;
  s->dx = dx;
  s->dy = dy;
  s->prm = *params;
  s->prec = params->precision;
  s->elem = s->prec == SWE_F64 ? 8 : 4;
  if (params->shore) s->tile = shore_shape((int)s->elem);  // the shoreline kernels' one shape
  else if (params->tile > 0) s->tile = params->tile;
  else {
    const int cached = swe_autotune_lookup(params->precision, 0, (double)grid->nx * grid->ny);
    s->tile = cached > 0 ? cached : 1;
  }
  s->stream = (cudaStream_t)params->stream;
  const int align = 32;  // elements: 128 B rows in FP32, 256 B in FP64
  s->pitch = ((s->nx + align - 1) / align) * align;

  Phys &ph = s->phys;
  ph.g = params->g;
  ph.n2 = params->manning_n * params->manning_n;
  ph.h_dry = params->h_dry;
  ph.h_wet = params->h_wet;
  ph.h_film = params->h_film;
  ph.hf4 = params->h_film * params->h_film * params->h_film * params->h_film;
  ph.h_film32 = thr32(params->h_film);
  ph.weno_eps = params->weno_eps;
  ph.fixed_dt = params->fixed_dt;
  ph.z_ref = params->z_ref;
  ph.b_jump_x = params->b_jump_x;
  ph.b_jump_y = params->b_jump_y;
  ph.inflow_amp = params->inflow_amp;
  ph.inflow_period = params->inflow_period;
  ph.inflow_depth = params->inflow_depth;
  ph.dx = dx;
  ph.dy = dy;
  ph.h_dry32 = thr32(params->h_dry);
  ph.h_wet32 = thr32(params->h_wet);
  for (int k = 0; k < 4; ++k) ph.bc[k] = params->bc[k];
  ph.wait_cycles = kDefaultWaitCycles;
  ph.copy_extra = 0u;
  finish_phys(ph);

  const size_t plane = (size_t)s->pitch * s->ny * s->elem;
  const size_t plane_al = (plane + 255) & ~(size_t)255;
  const size_t stag = ((sizeof(double) * (size_t)s->nx * s->ny) + 255) & ~(size_t)255;
  const size_t scal = (sizeof(DevScalars) + 255) & ~(size_t)255;
  const size_t ctap = (sizeof(DevPartials) + 255) & ~(size_t)255;
  const size_t part = sizeof(double) * (kMassBlocks + 1);
  const size_t total = plane_al * 10 + stag + scal + ctap + part;
  cudaError_t e = dev_malloc(&s->mem, total);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    delete s;
    return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
  }
  char *q = (char *)s->mem;
  s->b = q; q += plane_al;
  for (int k = 0; k < 3; ++k) {
    s->h[k] = q; q += plane_al;
    s->hu[k] = q; q += plane_al;
    s->hv[k] = q; q += plane_al;
  }
  s->staging = (double *)q; q += stag;
  s->sc = (DevScalars *)q; q += scal;
  s->cta = (DevPartials *)q; q += ctap;
  s->partials = (double *)q;
#ifdef SWE_CHECKED
  ph.check = &s->sc->check;  // the checked build records out-of-range indexes here
#endif

  int rc = SWE_OK;
  {
    // the tile shape must fit in the opt-in shared memory of this device
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = SWE_ECUDA;
    } else if (shape_smem(s->tile, (int)s->elem) + sizeof(RedSmem) > (size_t)optin) {
      rc = SWE_EINVAL;
    } else if (params->fused_step && fused_smem((int)s->elem) + sizeof(RedSmem) + 256 > (size_t)optin) {
      rc = SWE_EINVAL;
    }
  }
  if (rc == SWE_OK && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) rc = SWE_ECUDA;
  if (rc == SWE_OK) {
    e = s->prec == SWE_F64 ? prepare_shape<double>(s->tile) : prepare_shape<float>(s->tile);
    rc = cuda_check(s, e);
  }
  if (rc == SWE_OK && params->shore) {
    e = s->prec == SWE_F64 ? prepare_shore<double>() : prepare_shore<float>();
    rc = cuda_check(s, e);
  }
  if (rc == SWE_OK && params->fused_step) {
    e = s->prec == SWE_F64 ? prepare_fused<double>() : prepare_fused<float>();
    rc = cuda_check(s, e);
  }
  if (rc == SWE_OK) {
    e = s->prec == SWE_F64 ? make_maps<double>(s->tile, field_of<double>(s), s->maps)
                           : make_maps<float>(s->tile, field_of<float>(s), s->maps);
    rc = cuda_check(s, e);
  }
  if (rc == SWE_OK) rc = cuda_check(s, cudaMemsetAsync(s->mem, 0, plane_al * 10, s->stream));
  if (rc == SWE_OK) rc = cuda_check(s, reset_scalars(s->sc, s->cta, 0.0, 0.4, 0.0, s->stream));
  if (rc == SWE_OK) rc = upload_field(s, bathymetry, s->b, false);
  if (rc == SWE_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream));
  if (rc != SWE_OK) {
    swe_destroy(s);
    return rc;
  }
  s->cfl_dev = 0.4;
  *out = s;
  return SWE_OK;
}

int swe_set_state(swe_handle *s, const double *h, const double *hu, const double *hv) {
  const TraceRange trace("swe_set_state");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  int rc = upload_field(s, h, s->h[0], true);
  if (rc == SWE_OK) rc = upload_field(s, hu, s->hu[0], false);
  if (rc == SWE_OK) rc = upload_field(s, hv, s->hv[0], false);
  if (rc == SWE_OK) rc = after_state_change(s);
  return rc;
}
int swe_set_state_device(swe_handle *s, const void *h, const void *hu, const void *hv) {
  const TraceRange trace("swe_set_state_device");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  int rc = import_device(s, h, s->h[0], true);
  if (rc == SWE_OK) rc = import_device(s, hu, s->hu[0], false);
  if (rc == SWE_OK) rc = import_device(s, hv, s->hv[0], false);
  if (rc != SWE_OK) return rc;
  return after_state_change(s);
}

int swe_set_state_async(swe_handle *s, const double *h, const double *hu, const double *hv) {
  const TraceRange trace("swe_set_state_async");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  if (s->sticky != SWE_OK) return s->sticky;
  const size_t n = (size_t)s->nx * s->ny, nb = sizeof(double) * n;
  if (!pinned_device_ptr(h, nb) || !pinned_device_ptr(hu, nb) || !pinned_device_ptr(hv, nb))
    return swe_set_state(s, h, hu, hv);  // pageable: synchronous
  cudaError_t e = cudaSuccess;
  if (!s->instage[0]) {  // first asynchronous upload: its buffers, stream and events
    double *st[2] = {nullptr, nullptr};
    cudaStream_t us = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dev_malloc((void **)&st[k], 3 * nb);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {  // nothing half-made stays behind
      for (int k = 0; k < 4; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
      if (us) cudaStreamDestroy(us);
      for (int k = 0; k < 2; ++k)
        if (st[k]) cudaFree(st[k]);
      if (e == cudaErrorMemoryAllocation) {  // no room now: the handle is unchanged and usable
        (void)cudaGetLastError();
        return SWE_ENOMEM;
      }
      return cuda_check(s, e);
    }
    s->upl = us;
    for (int k = 0; k < 2; ++k) {
      s->instage[k] = st[k];
      s->ev_up[k] = ev[2 * k];
      s->ev_used[k] = ev[2 * k + 1];
    }
  }
  // the copy engines fill slot k once the conversion of the upload before
  // last is done with it; the conversion into U^n follows on the caller's
  // stream, after the work enqueued so far (steps, read-back conversions)
  const int k = s->uk;
  double *in = s->instage[k];
  if (s->up_used[k]) e = cudaStreamWaitEvent(s->upl, s->ev_used[k], 0);
  const double *src[3] = {h, hu, hv};
  for (int f = 0; f < 3 && e == cudaSuccess; ++f)
    e = cudaMemcpyAsync(in + f * n, src[f], nb, cudaMemcpyHostToDevice, s->upl);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_up[k], s->upl);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_up[k], 0);
  void *dst[3] = {s->h[0], s->hu[0], s->hv[0]};
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    if (s->prec == SWE_F64)
      e = import_plane<double>(in + f * n, true, (double *)dst[f], f == 0 ? (const double *)s->b : nullptr,
                               s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
    else
      e = import_plane<float>(in + f * n, true, (float *)dst[f], f == 0 ? (const float *)s->b : nullptr,
                              s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_used[k], s->stream);
  if (e == cudaSuccess) {
    s->up_used[k] = true;
    s->uk = 1 - k;
  }
  // the scalars of the new state, on the stream: time kept, the rest cleared,
  // wave speeds and runup of U^n
  if (s->cfl_dev <= 0) s->cfl_dev = 0.4;
  if (e == cudaSuccess) e = reset_scalars(s->sc, s->cta, NAN, s->cfl_dev, s->t_end, s->stream);
  if (e == cudaSuccess)
    e = s->prec == SWE_F64 ? state_stats<double>(field_of<double>(s), s->phys, s->sc, s->stream)
                           : state_stats<float>(field_of<float>(s), s->phys, s->sc, s->stream);
  return cuda_check(s, e);
}

int swe_step(swe_handle *s, int32_t n, double cfl) {
  const TraceRange trace("swe_step");
  if (!s || n < 0) return SWE_EINVAL;
  if (s->prm.fixed_dt <= 0.0 && !(cfl > 0.0 && std::isfinite(cfl))) return SWE_EINVAL;
  if (n == 0) return SWE_OK;
  cudaError_t e = cudaSuccess;
  if (s->prm.fixed_dt <= 0.0 && cfl != s->cfl_dev) {
    // ordered on the stream before the steps; the captured graph reads it
    e = set_cfl(s->sc, cfl, s->stream);
    if (e != cudaSuccess) return cuda_check(s, e);
    s->cfl_dev = cfl;
  }
  auto capture = [s](cudaGraphExec_t *out, bool single) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = single ? enqueue_fused(s, 0, s->cap) : enqueue_step(s, s->cap);
      if (single && le == cudaSuccess) le = copy_back(s, s->cap);
      e = cudaStreamEndCapture(s->cap, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) *out = nullptr;
    return e;
  };
  if (!s->graph && (e = capture(&s->graph, false)) != cudaSuccess) return cuda_check(s, e);
  if (s->prm.fused_step) {
    // the graph advances two steps; an odd count ends with one more and the copy back
    for (int32_t k = 0; k < n / 2 && e == cudaSuccess; ++k) e = cudaGraphLaunch(s->graph, s->stream);
    if (e == cudaSuccess && (n & 1)) {
      if (!s->graph1) e = capture(&s->graph1, true);
      if (e == cudaSuccess) e = cudaGraphLaunch(s->graph1, s->stream);
    }
    return cuda_check(s, e);
  }
  for (int32_t k = 0; k < n && e == cudaSuccess; ++k) e = cudaGraphLaunch(s->graph, s->stream);
  return cuda_check(s, e);
}

int swe_sync(swe_handle *s) {
  const TraceRange trace("swe_sync");
  if (!s) return SWE_EINVAL;
  if (s->sticky != SWE_OK) return s->sticky;
  return device_status(s);
}

int swe_status(swe_handle *s) {
  if (!s) return SWE_EINVAL;
  if (s->sticky != SWE_OK) return s->sticky;
  cudaError_t q = cudaStreamQuery(s->stream);
  if (q == cudaErrorNotReady) return SWE_OK;
  if (q != cudaSuccess) return cuda_check(s, q);
  return device_status(s);
}

int swe_get_state(swe_handle *s, double *h, double *hu, double *hv) {
  const TraceRange trace("swe_get_state");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  int rc = download_field(s, s->h[0], h, true);
  if (rc == SWE_OK) rc = download_field(s, s->hu[0], hu, false);
  if (rc == SWE_OK) rc = download_field(s, s->hv[0], hv, false);
  if (rc == SWE_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream));
  if (rc == SWE_OK) rc = swe_sync(s);
  return rc;
}

int swe_get_state_async(swe_handle *s, double *h, double *hu, double *hv) {
  const TraceRange trace("swe_get_state_async");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  if (s->sticky != SWE_OK) return s->sticky;
  const size_t bytes = sizeof(double) * (size_t)s->nx * s->ny;
  void *out[3] = {const_cast<void *>(pinned_device_ptr(h, bytes)), const_cast<void *>(pinned_device_ptr(hu, bytes)),
                  const_cast<void *>(pinned_device_ptr(hv, bytes))};
  if (!out[0] || !out[1] || !out[2]) return swe_get_state(s, h, hu, hv);  // pageable: synchronous
  cudaError_t e = cudaSuccess;
  const size_t nb = sizeof(double) * (size_t)s->nx * s->ny;
  if (!s->xstage[0]) {  // first asynchronous read-back: its buffers, stream and events
    double *xs[2] = {nullptr, nullptr};
    cudaStream_t xf = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dev_malloc((void **)&xs[k], 3 * nb);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xf, cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {  // nothing half-made stays behind
      for (int k = 0; k < 4; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
      if (xf) cudaStreamDestroy(xf);
      for (int k = 0; k < 2; ++k)
        if (xs[k]) cudaFree(xs[k]);
      if (e == cudaErrorMemoryAllocation) {  // no room now: the handle is unchanged and usable
        (void)cudaGetLastError();
        return SWE_ENOMEM;
      }
      return cuda_check(s, e);
    }
    s->xfer = xf;
    for (int k = 0; k < 2; ++k) {
      s->xstage[k] = xs[k];
      s->ev_conv[k] = ev[2 * k];
      s->ev_done[k] = ev[2 * k + 1];
    }
  }
  // slot k is free once the read-back before last has reached the host; the
  // conversion reads U^n in stream order (after the steps enqueued so far),
  // then a copy engine carries the slot to the host (it overlaps an upload in
  // the other direction better than a kernel writing host memory)
  const int k = s->xk;
  double *xs = s->xstage[k];
  if (s->pending[k]) e = cudaStreamWaitEvent(s->stream, s->ev_done[k], 0);
  const size_t n = (size_t)s->nx * s->ny;
  const void *src[3] = {s->h[0], s->hu[0], s->hv[0]};
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    if (s->prec == SWE_F64)
      e = export_plane<double>((const double *)src[f], xs + f * n, true, f == 0 ? (const double *)s->b : nullptr,
                               s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
    else
      e = export_plane<float>((const float *)src[f], xs + f * n, true, f == 0 ? (const float *)s->b : nullptr,
                              s->phys.z_ref, s->nx, s->ny, s->pitch, s->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_conv[k], s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->xfer, s->ev_conv[k], 0);
  double *hosts[3] = {h, hu, hv};
  for (int f = 0; f < 3 && e == cudaSuccess; ++f)
    e = cudaMemcpyAsync(hosts[f], xs + f * n, nb, cudaMemcpyDeviceToHost, s->xfer);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_done[k], s->xfer);
  if (e != cudaSuccess) return cuda_check(s, e);
  s->pending[k] = true;
  s->xk = 1 - k;
  return SWE_OK;
}

int swe_wait_state(swe_handle *s) {
  const TraceRange trace("swe_wait_state");
  if (!s) return SWE_EINVAL;
  for (int k = 0; k < 2; ++k) {
    if (!s->pending[k]) continue;
    const cudaError_t e = cudaEventSynchronize(s->ev_done[k]);
    s->pending[k] = false;
    if (e != cudaSuccess) return cuda_check(s, e);
  }
  return s->sticky;
}

int swe_get_state_device(swe_handle *s, void *h, void *hu, void *hv) {
  const TraceRange trace("swe_get_state_device");
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  int rc = export_device(s, s->h[0], h, true);
  if (rc == SWE_OK) rc = export_device(s, s->hu[0], hu, false);
  if (rc == SWE_OK) rc = export_device(s, s->hv[0], hv, false);
  if (rc == SWE_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream));
  if (rc != SWE_OK) return rc;
  return swe_sync(s);
}

int swe_mass(swe_handle *s, double *mass, double *clamp_mass) {
  const TraceRange trace("swe_mass");
  if (!s) return SWE_EINVAL;
  cudaError_t e =
      s->prec == SWE_F64
          ? swe::mass<double>((const double *)s->h[0], (const double *)s->b, s->phys.z_ref, s->nx, s->ny, s->pitch, s->dx * s->dy, s->partials, s->partials + kMassBlocks, s->stream)
          : swe::mass<float>((const float *)s->h[0], (const float *)s->b, s->phys.z_ref, s->nx, s->ny, s->pitch, s->dx * s->dy, s->partials, s->partials + kMassBlocks, s->stream);
  double r[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r[0], s->partials + kMassBlocks, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = read_volumes(s->cta, &r[1], nullptr, s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  if (mass) *mass = r[0];
  if (clamp_mass) *clamp_mass = r[1];
  return swe_sync(s);
}

int swe_diagnostics(swe_handle *s, swe_diag *d) {
  const TraceRange trace("swe_diagnostics");
  if (!s || !d) return SWE_EINVAL;
  DevScalars h;
  cudaError_t e = cudaMemcpyAsync(&h, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = read_volumes(s->cta, &d->clamp_mass, &d->boundary_mass, s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  auto dbl = [](unsigned long long u) { double x; std::memcpy(&x, &u, 8); return x; };
  d->t = h.t;
  d->steps = h.steps;
  d->last_dt = h.dt;
  d->alpha_x = dbl(h.alpha[0][0]);
  d->alpha_y = dbl(h.alpha[0][1]);
  const unsigned long long rn = h.runup_now[(h.steps + 1) & 1];
  d->runup_now = rn ? dbl(rn) : -INFINITY;
  d->runup_max = h.runup_max ? dbl(h.runup_max) : -INFINITY;
  d->tile = s->tile;
  d->status = SWE_OK;
  if (h.status & ST_TIMEOUT) d->status = SWE_ETIMEOUT;
  else if (h.status & ST_NONFINITE) d->status = SWE_ENONFINITE;
  else if (h.status & ST_DRY) d->status = SWE_EINVAL;
  if (s->sticky != SWE_OK) d->status = s->sticky;
  return d->status;
}

int swe_runup(swe_handle *s, double *runup_max, double *runup_now) {
  swe_diag d;
  int rc = swe_diagnostics(s, &d);
  if (!s) return SWE_EINVAL;
  if (runup_max) *runup_max = d.runup_max;
  if (runup_now) *runup_now = d.runup_now;
  return rc;
}

int swe_get_time(swe_handle *s, double *t, int64_t *steps) {
  swe_diag d;
  int rc = swe_diagnostics(s, &d);
  if (!s) return SWE_EINVAL;
  if (t) *t = d.t;
  if (steps) *steps = d.steps;
  return rc;
}

int swe_set_time(swe_handle *s, double t) {
  if (!s || !std::isfinite(t)) return SWE_EINVAL;
  const long long zero = 0;
  cudaError_t e = cudaMemcpyAsync(&s->sc->t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&s->sc->t_step, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&s->sc->steps, &zero, sizeof(long long), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_check(s, e);
}

int swe_set_horizon(swe_handle *s, double t_end) {
  const TraceRange trace("swe_set_horizon");
  if (!s || !std::isfinite(t_end) || t_end < 0.0) return SWE_EINVAL;
  cudaError_t e = cudaMemcpyAsync(&s->sc->t_end, &t_end, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) s->t_end = t_end;
  return cuda_check(s, e);
}

int swe_set_wait(swe_handle *s, double timeout_s, int32_t extra_copy_bytes) {
  if (!s || !(timeout_s > 0.0 && timeout_s <= 60.0) || extra_copy_bytes < 0 || extra_copy_bytes > 65536)
    return SWE_EINVAL;
  const cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_check(s, e);
  s->phys.wait_cycles = (long long)(timeout_s * 2.2e9);  // SM clock at most ~2.1 GHz
  s->phys.copy_extra = (unsigned)extra_copy_bytes;
  if (s->graph) {  // the step graph holds the old values: capture again at the next step
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (s->graph1) {
    cudaGraphExecDestroy(s->graph1);
    s->graph1 = nullptr;
  }
  if (s->sticky == SWE_ETIMEOUT) s->sticky = SWE_OK;
  return SWE_OK;
}

int swe_destroy(swe_handle *s) {
  if (!s) return SWE_OK;
  if (s->stream || s->mem) cudaStreamSynchronize(s->stream);
  if (s->xfer) {
    cudaStreamSynchronize(s->xfer);
    cudaStreamDestroy(s->xfer);
  }
  if (s->upl) {
    cudaStreamSynchronize(s->upl);
    cudaStreamDestroy(s->upl);
  }
  for (int k = 0; k < 2; ++k) {
    if (s->ev_up[k]) cudaEventDestroy(s->ev_up[k]);
    if (s->ev_used[k]) cudaEventDestroy(s->ev_used[k]);
    if (s->instage[k]) cudaFree(s->instage[k]);
    if (s->ev_conv[k]) cudaEventDestroy(s->ev_conv[k]);
    if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
    if (s->xstage[k]) cudaFree(s->xstage[k]);
  }
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->graph1) cudaGraphExecDestroy(s->graph1);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->mem) cudaFree(s->mem);
  delete s;
  return SWE_OK;
}

int swe_time_stages(swe_handle *s, int32_t n, double cfl, double *ms_total, double *ms_stage) {
  const TraceRange trace("swe_time_stages");
  if (!s || n <= 0) return SWE_EINVAL;
  int rc = swe_step(s, 1, cfl);  // make sure cfl is on the device and the graph exists
  if (rc != SWE_OK) return rc;
  cudaEvent_t ev[4];
  for (int k = 0; k < 4; ++k)
    if (cudaEventCreate(&ev[k]) != cudaSuccess) return fail(s, SWE_ECUDA);
  double acc[3] = {0, 0, 0}, tot = 0.0;
  cudaError_t e = cudaSuccess;
  if (s->prm.fused_step) {
    // steps alternate between the plane sets; an odd count ends with the copy back
    for (int32_t it = 0; it < n && e == cudaSuccess; ++it) {
      e = enqueue_fused(s, it & 1, s->stream, ev);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
      float m[3];
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&m[k], ev[k], ev[k + 1]);
      if (e != cudaSuccess) break;
      acc[0] += m[1];
      acc[1] += m[0] + m[2];
      tot += m[0] + m[1] + m[2];
    }
    if (e == cudaSuccess && (n & 1)) e = copy_back(s, s->stream);
  }
  for (int32_t it = 0; it < n && e == cudaSuccess && !s->prm.fused_step; ++it) {
    e = cudaEventRecord(ev[0], s->stream);
    for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage) {
      e = launch_one_stage(s, stage, s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[stage], s->stream);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    float m;
    for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage) {
      e = cudaEventElapsedTime(&m, ev[stage - 1], ev[stage]);
      acc[stage - 1] += m;
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m, ev[0], ev[3]);
    tot += m;
  }
  for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return cuda_check(s, e);
  if (ms_total) *ms_total = tot;
  if (ms_stage)
    for (int k = 0; k < 3; ++k) ms_stage[k] = acc[k];
  return swe_sync(s);
}

}  // extern "C"
