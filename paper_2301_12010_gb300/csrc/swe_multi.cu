// swe_multi.cu -- C ABI of a row-partitioned domain (include/swe.h,
// swe_multi_*): the paper's parallel scheme ("TPU implementation", Table 1)
// on the GB300 kernels.  The grid is cut along y into strips of whole rows;
// each strip's planes carry three halo rows above and below.  Every RK stage
// runs the stage kernel over each strip, then copies the three boundary rows
// of every strip's stage output into its neighbours' halo rows (the halo
// exchange the paper performs between TPU cores); the global wave speeds of
// each stage are one maximum over all strips (the strips publish into one
// set of device scalars, the cross-core reduction of the paper).  A strip's
// sides towards its neighbours are BC_HALO: their ghost values are the halo
// rows.  The result is the same as the undivided grid's, bit for bit.
//
// All strips live on the calling device and run on one stream, one after
// another; across devices the row copies would be peer copies and the
// maximum a collective.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/swe.h"
#include "swe_alloc.h"
#include "swe_launch.h"
#include "swe_trace.h"

using namespace swe;

namespace {

constexpr int kHalo = 3;     // WENO5 ghost width
constexpr int kRowAlign = 32;  // strip boundaries on multiples of this many rows (strips of 64 rows or more)

struct Part {
  int row0 = 0, rows = 0;
  void *mem = nullptr;        // 10 planes of (rows + 6) x pitch
  void *b = nullptr;
  void *h[3] = {}, *hu[3] = {}, *hv[3] = {};  // row 0 of each plane
  Phys phys{};
  BoxMaps maps[3] = {};
};

int strip_bounds(int ny, int nparts, int k, int *row0, int *rows) {
  if (ny < 3 || nparts < 1 || k < 0 || k >= nparts) return SWE_EINVAL;
  const long long align = (long long)ny >= 2ll * kRowAlign * nparts ? kRowAlign : 1;
  auto edge = [&](int q) -> int {
    if (q <= 0) return 0;
    if (q >= nparts) return ny;
    const long long r = ((long long)q * ny + (long long)nparts * align / 2) / ((long long)nparts * align);
    return (int)(r * align);
  };
  const int a = edge(k), b = edge(k + 1);
  for (int q = 0; q < nparts; ++q)  // every strip holds at least the halo width
    if (edge(q + 1) - edge(q) < kHalo) return SWE_EINVAL;
  *row0 = a;
  *rows = b - a;
  return SWE_OK;
}

}  // namespace

struct swe_multi {
  int nx = 0, ny = 0, pitch = 0, nparts = 0;
  double dx = 0, dy = 0;
  swe_params prm{};
  int prec = SWE_F32, tile = 1;
  size_t elem = 4;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::vector<Part> parts;
  void *smem_block = nullptr;  // scalars, per-CTA partials, mass partials, staging
  DevScalars *sc = nullptr;
  DevPartials *cta = nullptr;
  double *partials = nullptr;  // kMassBlocks + one result per strip
  double *staging = nullptr;   // the largest strip's rows x nx doubles
  cudaGraphExec_t graph = nullptr;
  double cfl_dev = 0.4;
  int sticky = SWE_OK;
};

namespace {

int mfail(swe_multi *m, cudaError_t e) {
  if (e == cudaSuccess) return SWE_OK;
  (void)cudaGetLastError();
  const int code = e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
  if (m && m->sticky == SWE_OK) m->sticky = code;
  return code;
}

template <typename T>
Field<T> field_of(const swe_multi *m, const Part &pt) {
  Field<T> f;
  f.b = (const T *)pt.b;
  for (int k = 0; k < 3; ++k) {
    f.h[k] = (T *)pt.h[k];
    f.hu[k] = (T *)pt.hu[k];
    f.hv[k] = (T *)pt.hv[k];
  }
  f.nx = m->nx;
  f.ny = pt.rows;
  f.pitch = m->pitch;
  f.halo = kHalo;
  return f;
}

// The halo exchange of one plane set (index q of U^n, U1, U2; q < 0: the bed):
// each interface copies the lower strip's top three rows into the upper
// strip's low halo rows and the upper strip's bottom three rows into the
// lower strip's high halo rows.
cudaError_t exchange(swe_multi *m, int q, cudaStream_t st) {
  const size_t rowb = (size_t)m->pitch * m->elem, band = kHalo * rowb;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k + 1 < m->nparts && e == cudaSuccess; ++k) {
    Part &lo = m->parts[k], &hi = m->parts[k + 1];
    void *plo[3], *phi[3];
    int nf = 3;
    if (q < 0) {
      plo[0] = lo.b;
      phi[0] = hi.b;
      nf = 1;
    } else {
      plo[0] = lo.h[q], plo[1] = lo.hu[q], plo[2] = lo.hv[q];
      phi[0] = hi.h[q], phi[1] = hi.hu[q], phi[2] = hi.hv[q];
    }
    for (int f = 0; f < nf && e == cudaSuccess; ++f) {
      char *a = (char *)plo[f], *b = (char *)phi[f];
      e = cudaMemcpyAsync(b - band, a + (size_t)(lo.rows - kHalo) * rowb, band, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(a + (size_t)lo.rows * rowb, b, band, cudaMemcpyDeviceToDevice, st);
    }
  }
  return e;
}

cudaError_t enqueue_step(swe_multi *m, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage) {
    for (int k = 0; k < m->nparts && e == cudaSuccess; ++k) {
      Part &pt = m->parts[k];
      e = m->prec == SWE_F64 ? launch_stage<double>(m->tile, field_of<double>(m, pt), pt.phys, m->sc, stage, st, pt.maps)
                             : launch_stage<float>(m->tile, field_of<float>(m, pt), pt.phys, m->sc, stage, st, pt.maps);
    }
    if (e == cudaSuccess) e = exchange(m, stage % 3, st);  // the stage's output planes
  }
  return e;
}

// Host FP64 rows [row0, row0 + rows) of a full-grid array -> a strip plane
// (depth fields stored as the anomaly; the strip's bed must be on the device).
int upload_rows(swe_multi *m, const Part &pt, const double *src, void *dst, bool is_depth) {
  const double *rows = src + (size_t)pt.row0 * m->nx;
  const size_t bytes = sizeof(double) * (size_t)m->nx * pt.rows;
  const void *in = pinned_device_ptr(rows, bytes);
  cudaError_t e = cudaSuccess;
  if (!in) {
    e = cudaMemcpyAsync(m->staging, rows, bytes, cudaMemcpyHostToDevice, m->stream);
    in = m->staging;
  }
  if (e == cudaSuccess)
    e = m->prec == SWE_F64
            ? import_plane<double>(in, true, (double *)dst, is_depth ? (const double *)pt.b : nullptr, m->prm.z_ref,
                                   m->nx, pt.rows, m->pitch, m->stream)
            : import_plane<float>(in, true, (float *)dst, is_depth ? (const float *)pt.b : nullptr, m->prm.z_ref,
                                  m->nx, pt.rows, m->pitch, m->stream);
  // the staging plane is reused by the next strip: finish this one first
  if (e == cudaSuccess && in == m->staging) e = cudaStreamSynchronize(m->stream);
  return mfail(m, e);
}

int download_rows(swe_multi *m, const Part &pt, const void *src, double *dst, bool is_depth) {
  double *rows = dst + (size_t)pt.row0 * m->nx;
  const size_t bytes = sizeof(double) * (size_t)m->nx * pt.rows;
  void *out = const_cast<void *>(pinned_device_ptr(rows, bytes));
  void *target = out ? out : m->staging;
  cudaError_t e =
      m->prec == SWE_F64
          ? export_plane<double>((const double *)src, target, true, is_depth ? (const double *)pt.b : nullptr,
                                 m->prm.z_ref, m->nx, pt.rows, m->pitch, m->stream)
          : export_plane<float>((const float *)src, target, true, is_depth ? (const float *)pt.b : nullptr,
                                m->prm.z_ref, m->nx, pt.rows, m->pitch, m->stream);
  if (e == cudaSuccess && !out) e = cudaMemcpyAsync(rows, m->staging, bytes, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && !out) e = cudaStreamSynchronize(m->stream);
  return mfail(m, e);
}

bool valid_multi_params(const swe_params *p) {
  if (!p) return false;
  if (p->precision != SWE_F32 && p->precision != SWE_F64) return false;
  for (int k = 0; k < 4; ++k)
    if (p->bc[k] < SWE_BC_WALL || p->bc[k] > SWE_BC_PERIODIC) return false;
  if ((p->bc[0] == SWE_BC_PERIODIC) != (p->bc[1] == SWE_BC_PERIODIC)) return false;
  // the strips' y sides are their neighbours or walls: no wrap-around or inflow in y
  if (p->bc[2] != SWE_BC_WALL || p->bc[3] != SWE_BC_WALL || p->bc[1] == SWE_BC_INFLOW) return false;
  if (p->bc[0] == SWE_BC_INFLOW && !(p->inflow_depth > 0.0 && p->inflow_period > 0.0)) return false;
  if (!(p->g > 0.0) || !(p->manning_n >= 0.0) || !(p->h_dry >= 0.0) || !(p->h_wet >= 0.0) || !(p->h_film >= 0.0) ||
      !(p->weno_eps > 0.0))
    return false;
  if (!std::isfinite(p->z_ref) || !std::isfinite(p->fixed_dt)) return false;
  if (p->tile < 0 || p->tile > num_shapes()) return false;
  return true;
}

Phys phys_for(const swe_params *q, double dx, double dy) {
  Phys ph{};
  ph.g = q->g;
  ph.n2 = q->manning_n * q->manning_n;
  ph.h_dry = q->h_dry;
  ph.h_wet = q->h_wet;
  ph.h_film = q->h_film;
  ph.hf4 = q->h_film * q->h_film * q->h_film * q->h_film;
  ph.h_film32 = thr32(q->h_film);
  ph.weno_eps = q->weno_eps;
  ph.fixed_dt = q->fixed_dt;
  ph.z_ref = q->z_ref;
  ph.b_jump_x = q->b_jump_x;
  ph.b_jump_y = q->b_jump_y;
  ph.inflow_amp = q->inflow_amp;
  ph.inflow_period = q->inflow_period;
  ph.inflow_depth = q->inflow_depth;
  ph.dx = dx;
  ph.dy = dy;
  ph.h_dry32 = thr32(q->h_dry);
  ph.h_wet32 = thr32(q->h_wet);
  for (int k = 0; k < 4; ++k) ph.bc[k] = q->bc[k];
  ph.wait_cycles = kDefaultWaitCycles;
  ph.copy_extra = 0u;
  finish_phys(ph);
  return ph;
}

int after_state(swe_multi *m) {
  // wave speeds and runup of U^n over all strips, into the shared scalars
  double t = 0.0;
  cudaError_t e = cudaMemcpyAsync(&t, &m->sc->t, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = exchange(m, 0, m->stream);
  if (e == cudaSuccess) e = reset_scalars(m->sc, m->cta, t, m->cfl_dev, 0.0, m->stream);
  for (int k = 0; k < m->nparts && e == cudaSuccess; ++k) {
    Part &pt = m->parts[k];
    e = m->prec == SWE_F64 ? state_stats<double>(field_of<double>(m, pt), pt.phys, m->sc, m->stream)
                           : state_stats<float>(field_of<float>(m, pt), pt.phys, m->sc, m->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return mfail(m, e);
}

int device_status(swe_multi *m) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, &m->sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, e);
  if (st & ST_TIMEOUT) return SWE_ETIMEOUT;
  if (st & ST_NONFINITE) return SWE_ENONFINITE;
  if (st & ST_DRY) return SWE_EINVAL;
  return SWE_OK;
}

}  // namespace

extern "C" {

int swe_strip_bounds(int32_t ny, int32_t nparts, int32_t k, int32_t *row0, int32_t *rows) {
  if (!row0 || !rows) return SWE_EINVAL;
  int a = 0, n = 0;
  const int rc = strip_bounds(ny, nparts, k, &a, &n);
  if (rc == SWE_OK) {
    *row0 = a;
    *rows = n;
  }
  return rc;
}

int swe_multi_create(const swe_grid *grid, double dx, double dy, const double *bathymetry, const swe_params *params,
                     int32_t nparts, swe_multi **out) {
  const TraceRange trace("swe_multi_create");
  if (out) *out = nullptr;
  if (!grid || !out || !bathymetry || !valid_multi_params(params)) return SWE_EINVAL;
  if (params->fused_step) return SWE_EINVAL;  // strips exchange halos between the stages
  if (params->shore) return SWE_EINVAL;       // strips run the paper's WENO faces
  if (grid->nx < 3 || grid->ny < 3 || !(dx > 0.0) || !(dy > 0.0) || nparts < 1 || nparts > 64) return SWE_EINVAL;
  if ((long long)grid->nx * grid->ny > (1ll << 31)) return SWE_EINVAL;
  int r0 = 0, rn = 0;
  if (strip_bounds(grid->ny, nparts, 0, &r0, &rn) != SWE_OK) return SWE_EINVAL;
  swe_multi *m = new (std::nothrow) swe_multi();
  if (!m) return SWE_ENOMEM;
  m->nx = grid->nx;
  m->ny = grid->ny;
  m->dx = dx;
  m->dy = dy;
  m->nparts = nparts;
  m->prm = *params;
  m->prec = params->precision;
  m->elem = m->prec == SWE_F64 ? 8 : 4;
  m->pitch = (m->nx + 31) / 32 * 32;
  m->stream = (cudaStream_t)params->stream;
  if (params->tile > 0) m->tile = params->tile;
  else {
    const int cached = swe_autotune_lookup(m->prec, 0, (double)m->nx * m->ny / nparts);
    m->tile = cached > 0 ? cached : 1;
  }
  m->parts.resize(nparts);
  const Phys base = phys_for(params, dx, dy);
  size_t maxrows = 0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < nparts && e == cudaSuccess; ++k) {
    Part &pt = m->parts[k];
    strip_bounds(m->ny, nparts, k, &pt.row0, &pt.rows);
    if ((size_t)pt.rows > maxrows) maxrows = pt.rows;
    const size_t plane = (size_t)m->pitch * (pt.rows + 2 * kHalo) * m->elem;
    const size_t plane_al = (plane + 255) & ~(size_t)255;
    e = dev_malloc(&pt.mem, plane_al * 10);
    if (e != cudaSuccess) break;
    char *q = (char *)pt.mem + (size_t)kHalo * m->pitch * m->elem;  // row 0 of the first plane
    pt.b = q; q += plane_al;
    for (int s = 0; s < 3; ++s) {
      pt.h[s] = q; q += plane_al;
      pt.hu[s] = q; q += plane_al;
      pt.hv[s] = q; q += plane_al;
    }
    pt.phys = base;
    pt.phys.halo_rows = kHalo;
    pt.phys.follower = k > 0 ? 1 : 0;     // strip 0 keeps the step's time and count
    if (k > 0) pt.phys.bc[2] = BC_HALO;
    if (k + 1 < nparts) pt.phys.bc[3] = BC_HALO;
    pt.phys.c32.ewy = 0.0f;                // y sides carry no edge inflow (walls or neighbours)
    pt.phys.c64.ewy = 0.0;
    e = cudaMemsetAsync(pt.mem, 0, plane_al * 10, m->stream);
  }
  const size_t scal = (sizeof(DevScalars) + 255) & ~(size_t)255;
  const size_t ctap = (sizeof(DevPartials) + 255) & ~(size_t)255;
  const size_t part = (sizeof(double) * (kMassBlocks + nparts) + 255) & ~(size_t)255;
  const size_t stag = sizeof(double) * maxrows * (size_t)m->nx;
  if (e == cudaSuccess) e = dev_malloc(&m->smem_block, scal + ctap + part + stag);
  if (e == cudaSuccess) {
    char *q = (char *)m->smem_block;
    m->sc = (DevScalars *)q; q += scal;
    m->cta = (DevPartials *)q; q += ctap;
    m->partials = (double *)q; q += part;
    m->staging = (double *)q;
#ifdef SWE_CHECKED
    for (auto &pt : m->parts) pt.phys.check = &m->sc->check;
#endif
  }
  int rc = mfail(m, e);
  if (rc == SWE_OK) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = SWE_ECUDA;
    } else if (shape_smem(m->tile, (int)m->elem) + sizeof(RedSmem) > (size_t)optin) {
      rc = SWE_EINVAL;
    }
  }
  if (rc == SWE_OK && cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) rc = SWE_ECUDA;
  if (rc == SWE_OK) rc = mfail(m, m->prec == SWE_F64 ? prepare_shape<double>(m->tile) : prepare_shape<float>(m->tile));
  for (int k = 0; k < nparts && rc == SWE_OK; ++k) {
    Part &pt = m->parts[k];
    rc = mfail(m, m->prec == SWE_F64 ? make_maps<double>(m->tile, field_of<double>(m, pt), pt.maps)
                                     : make_maps<float>(m->tile, field_of<float>(m, pt), pt.maps));
  }
  if (rc == SWE_OK) rc = mfail(m, reset_scalars(m->sc, m->cta, 0.0, 0.4, 0.0, m->stream));
  for (int k = 0; k < nparts && rc == SWE_OK; ++k) rc = upload_rows(m, m->parts[k], bathymetry, m->parts[k].b, false);
  if (rc == SWE_OK) rc = mfail(m, exchange(m, -1, m->stream));  // bed halos, once
  if (rc == SWE_OK) rc = mfail(m, cudaStreamSynchronize(m->stream));
  if (rc != SWE_OK) {
    swe_multi_destroy(m);
    return rc;
  }
  *out = m;
  return SWE_OK;
}

int swe_multi_set_state(swe_multi *m, const double *h, const double *hu, const double *hv) {
  const TraceRange trace("swe_multi_set_state");
  if (!m || !h || !hu || !hv) return SWE_EINVAL;
  int rc = SWE_OK;
  for (int k = 0; k < m->nparts && rc == SWE_OK; ++k) {
    Part &pt = m->parts[k];
    rc = upload_rows(m, pt, h, pt.h[0], true);
    if (rc == SWE_OK) rc = upload_rows(m, pt, hu, pt.hu[0], false);
    if (rc == SWE_OK) rc = upload_rows(m, pt, hv, pt.hv[0], false);
  }
  if (rc == SWE_OK) rc = after_state(m);
  return rc;
}

int swe_multi_set_time(swe_multi *m, double t) {
  if (!m || !std::isfinite(t)) return SWE_EINVAL;
  const long long zero = 0;
  cudaError_t e = cudaMemcpyAsync(&m->sc->t, &t, sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&m->sc->t_step, &t, sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&m->sc->steps, &zero, sizeof(long long), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return mfail(m, e);
}

int swe_multi_step(swe_multi *m, int32_t n, double cfl) {
  const TraceRange trace("swe_multi_step");
  if (!m || n < 0) return SWE_EINVAL;
  if (m->prm.fixed_dt <= 0.0 && !(cfl > 0.0 && std::isfinite(cfl))) return SWE_EINVAL;
  if (m->sticky != SWE_OK) return m->sticky;
  if (n == 0) return SWE_OK;
  cudaError_t e = cudaSuccess;
  if (m->prm.fixed_dt <= 0.0 && cfl != m->cfl_dev) {
    e = set_cfl(m->sc, cfl, m->stream);
    if (e != cudaSuccess) return mfail(m, e);
    m->cfl_dev = cfl;
  }
  if (!m->graph) {  // one step: three stages over every strip, each followed by its halo exchange
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = enqueue_step(m, m->cap);
      e = cudaStreamEndCapture(m->cap, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      m->graph = nullptr;
      return mfail(m, e);
    }
  }
  for (int32_t k = 0; k < n && e == cudaSuccess; ++k) e = cudaGraphLaunch(m->graph, m->stream);
  return mfail(m, e);
}

int swe_multi_get_state(swe_multi *m, double *h, double *hu, double *hv) {
  const TraceRange trace("swe_multi_get_state");
  if (!m || !h || !hu || !hv) return SWE_EINVAL;
  int rc = SWE_OK;
  for (int k = 0; k < m->nparts && rc == SWE_OK; ++k) {
    Part &pt = m->parts[k];
    rc = download_rows(m, pt, pt.h[0], h, true);
    if (rc == SWE_OK) rc = download_rows(m, pt, pt.hu[0], hu, false);
    if (rc == SWE_OK) rc = download_rows(m, pt, pt.hv[0], hv, false);
  }
  if (rc == SWE_OK) rc = mfail(m, cudaStreamSynchronize(m->stream));
  if (rc != SWE_OK) return rc;
  return m->sticky != SWE_OK ? m->sticky : device_status(m);
}

int swe_multi_mass(swe_multi *m, double *mass) {
  if (!m || !mass) return SWE_EINVAL;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < m->nparts && e == cudaSuccess; ++k) {
    Part &pt = m->parts[k];
    e = m->prec == SWE_F64
            ? swe::mass<double>((const double *)pt.h[0], (const double *)pt.b, m->prm.z_ref, m->nx, pt.rows, m->pitch,
                                m->dx * m->dy, m->partials, m->partials + kMassBlocks + k, m->stream)
            : swe::mass<float>((const float *)pt.h[0], (const float *)pt.b, m->prm.z_ref, m->nx, pt.rows, m->pitch,
                               m->dx * m->dy, m->partials, m->partials + kMassBlocks + k, m->stream);
  }
  std::vector<double> r(m->nparts, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r.data(), m->partials + kMassBlocks, sizeof(double) * m->nparts, cudaMemcpyDeviceToHost,
                        m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, e);
  double s = 0.0;
  for (double x : r) s += x;  // strip order
  *mass = s;
  return SWE_OK;
}

int swe_multi_diagnostics(swe_multi *m, swe_diag *d) {
  if (!m || !d) return SWE_EINVAL;
  DevScalars h;
  cudaError_t e = cudaMemcpyAsync(&h, m->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = read_volumes(m->cta, &d->clamp_mass, &d->boundary_mass, m->stream);
  if (e != cudaSuccess) return mfail(m, e);
  auto dbl = [](unsigned long long u) { double x; std::memcpy(&x, &u, 8); return x; };
  d->t = h.t;
  d->steps = h.steps;
  d->last_dt = h.dt;
  d->alpha_x = dbl(h.alpha[0][0]);
  d->alpha_y = dbl(h.alpha[0][1]);
  const unsigned long long rn = h.runup_now[(h.steps + 1) & 1];
  d->runup_now = rn ? dbl(rn) : -INFINITY;
  d->runup_max = h.runup_max ? dbl(h.runup_max) : -INFINITY;
  d->tile = m->tile;
  d->status = SWE_OK;
  if (h.status & ST_TIMEOUT) d->status = SWE_ETIMEOUT;
  else if (h.status & ST_NONFINITE) d->status = SWE_ENONFINITE;
  else if (h.status & ST_DRY) d->status = SWE_EINVAL;
  if (m->sticky != SWE_OK) d->status = m->sticky;
  return d->status;
}

int swe_multi_destroy(swe_multi *m) {
  if (!m) return SWE_OK;
  if (m->stream || m->parts.size()) cudaStreamSynchronize(m->stream);
  if (m->graph) cudaGraphExecDestroy(m->graph);
  for (auto &pt : m->parts)
    if (pt.mem) cudaFree(pt.mem);
  if (m->smem_block) cudaFree(m->smem_block);
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
  return SWE_OK;
}

}  // extern "C"
