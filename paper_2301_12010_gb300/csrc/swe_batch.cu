// swe_batch.cu -- C ABI of the batched ensemble / serving path
// (include/swe.h, swe_batch_*): slots admitted under an HBM budget, a slot
// table in device memory, and k-step cooperative persistent launches replayed
// from CUDA graphs.  Scenarios are independent (scenario-level data
// parallelism); each keeps its own wave speeds, time step, time and step
// count in device memory, so a scenario's result does not depend on what
// else is in the batch.
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/swe.h"
#include "swe_launch.h"
#include "swe_trace.h"
#include "swe_alloc.h"

namespace swe {
bool valid_params(const swe_params *p);  // swe_api.cu
}

using namespace swe;

namespace {

struct Slot {
  bool live = false;
  bool selected = true;  // advanced by the runs (swe_batch_select)
  int nx = 0, ny = 0, pitch = 0;
  double dx = 0, dy = 0, t_end = 0;
  size_t bytes = 0;
  void *mem = nullptr;
  double *staging = nullptr;
  Field<float> fd{};     // the planes of an FP32 batch
  Field<double> fd64{};  // the planes of an FP64 batch
  Phys p{};
  BoxMaps maps[3] = {};  // tensor maps of the halo-box copies (the batch's tile shape)
};

size_t plane_bytes(int nx, int ny, int *pitch_out, size_t elem = sizeof(float)) {
  const int pitch = ((nx + 31) / 32) * 32;
  if (pitch_out) *pitch_out = pitch;
  return (((size_t)pitch * ny * elem) + 255) & ~(size_t)255;
}

size_t slot_bytes(int nx, int ny, size_t elem = sizeof(float)) {
  const size_t plane = plane_bytes(nx, ny, nullptr, elem);
  const size_t stag = ((sizeof(double) * (size_t)nx * ny) + 255) & ~(size_t)255;
  return plane * 10 + stag;
}

template <typename T> Field<T> &field_of(Slot &sl);
template <> Field<float> &field_of<float>(Slot &sl) { return sl.fd; }
template <> Field<double> &field_of<double>(Slot &sl) { return sl.fd64; }
static_assert(sizeof(BatchSlot<float>) == sizeof(BatchSlot<double>), "one table size for both precisions");

}  // namespace

struct swe_batch {
  int nslots = 0;
  size_t budget = 0, used = 0;
  swe_params prm{};
  int prec = SWE_F32;
  size_t elem = sizeof(float);
  int tile = 1;
  int grid = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::vector<Slot> slots;
  DevScalars *d_sc = nullptr;          // one per slot
  DevPartials *d_cta = nullptr;        // one per slot: per-CTA partials of the clamp volume
  void *d_table = nullptr;             // BatchSlot<float or double>: live slots, work-list order
  BatchCtl *d_ctl = nullptr;
  double *d_part = nullptr;            // mass partials + result
  std::map<int, cudaGraphExec_t> graphs;
  double timeout_s = 1.0;
  unsigned extra = 0;
  double cfl = 0.4;  // CFL number in the slots' device scalars
  bool strided = false;  // work order of the current table (the launch must match it)
  bool small = false;    // few tiles per CTA and stage: the run-time-stage form of the kernel
  int sticky = SWE_OK;
};

namespace {

int bfail(swe_batch *b, cudaError_t e) {
  if (e == cudaSuccess) return SWE_OK;
  (void)cudaGetLastError();
  const int code = e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
  if (b && b->sticky == SWE_OK) b->sticky = code;
  return code;
}

Phys phys_of(const swe_params &q, double dx, double dy) {
  Phys ph{};
  ph.g = q.g;
  ph.n2 = q.manning_n * q.manning_n;
  ph.h_dry = q.h_dry;
  ph.h_wet = q.h_wet;
  ph.h_film = q.h_film;
  ph.hf4 = q.h_film * q.h_film * q.h_film * q.h_film;
  ph.h_film32 = thr32(q.h_film);
  ph.weno_eps = q.weno_eps;
  ph.fixed_dt = q.fixed_dt;
  ph.z_ref = q.z_ref;
  ph.b_jump_x = q.b_jump_x;
  ph.b_jump_y = q.b_jump_y;
  ph.inflow_amp = q.inflow_amp;
  ph.inflow_period = q.inflow_period;
  ph.inflow_depth = q.inflow_depth;
  ph.dx = dx;
  ph.dy = dy;
  ph.h_dry32 = thr32(q.h_dry);
  ph.h_wet32 = thr32(q.h_wet);
  for (int k = 0; k < 4; ++k) ph.bc[k] = q.bc[k];
  ph.wait_cycles = kDefaultWaitCycles;
  ph.copy_extra = 0u;
  finish_phys(ph);
  return ph;
}

// Rebuild the work list (live, selected slots in index order) and the
// control block.
template <typename T>
int upload_table_t(swe_batch *b) {
  std::vector<BatchSlot<T>> tab;
  int total = 0;
  const TileShape *ts = shape(b->tile);
  for (int s = 0; s < b->nslots; ++s) {
    Slot &sl = b->slots[s];
    if (!sl.live || !sl.selected) continue;
    BatchSlot<T> e{};
    for (int k = 0; k < 3; ++k) e.maps[k] = sl.maps[k];
    e.fd = field_of<T>(sl);
    e.p = sl.p;
    e.sc = b->d_sc + s;
    e.tiles_x = (sl.nx + ts->tx - 1) / ts->tx;
    e.ntiles = e.tiles_x * ((sl.ny + ts->ty - 1) / ts->ty);
    e.first_item = total;
    total += e.ntiles;
    tab.push_back(e);
  }
  BatchCtl c{};
  c.nslots = (int)tab.size();
  c.total_items = total;
  c.bar_count = 0;
  c.bar_gen = 0;
  c.status = 0;
  c.bar_extra = b->extra;
  c.bar_cycles = (long long)(b->timeout_s * 2.2e9);  // SM clock at most ~2.1 GHz
  // strided work order when every scenario spans at least two tiles per CTA:
  // neighbouring tiles in flight together, few scenario switches per CTA
  bool big = !tab.empty();
  for (const auto &e : tab) big = big && e.ntiles >= 2 * b->grid;
  c.strided = big ? 1 : 0;
  b->strided = big;
  b->small = total < kSmallItemsPerCta * b->grid;
  cudaError_t e = cudaSuccess;
  if (!tab.empty())
    e = cudaMemcpyAsync(b->d_table, tab.data(), sizeof(BatchSlot<T>) * tab.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bfail(b, e);
}

int upload_table(swe_batch *b) { return b->prec == SWE_F64 ? upload_table_t<double>(b) : upload_table_t<float>(b); }

bool valid_slot(const swe_batch *b, int32_t s) { return b && s >= 0 && s < b->nslots && b->slots[s].live; }

// A new slot's planes in its device memory (bed, U^n, U1, U2, staging), its
// tensor maps, physics, the host FP64 inputs converted in (page-locked host
// arrays read by the conversion kernel directly, pageable ones through the
// staging plane), its scalars and the wave speeds and runup of its state.
template <typename T>
cudaError_t fill_slot(swe_batch *b, Slot &sl, int s, size_t plane, const double *const srcs[4]) {
  Field<T> &fd = field_of<T>(sl);
  char *q = (char *)sl.mem;
  T *bplane = (T *)q;
  fd.b = bplane;
  q += plane;
  for (int k = 0; k < 3; ++k) {
    fd.h[k] = (T *)q; q += plane;
    fd.hu[k] = (T *)q; q += plane;
    fd.hv[k] = (T *)q; q += plane;
  }
  sl.staging = (double *)q;
  fd.nx = sl.nx;
  fd.ny = sl.ny;
  fd.pitch = sl.pitch;
  fd.halo = 0;
  cudaError_t e = make_maps<T>(b->tile, fd, sl.maps);
  if (e != cudaSuccess) return e;
  sl.p = phys_of(b->prm, sl.dx, sl.dy);
#ifdef SWE_CHECKED
  sl.p.check = &(b->d_sc + s)->check;  // the checked build records out-of-range indexes here
#endif
  const size_t nb = sizeof(double) * (size_t)sl.nx * sl.ny;
  e = cudaMemsetAsync(sl.mem, 0, plane * 10, b->stream);
  T *dsts[4] = {bplane, fd.h[0], fd.hu[0], fd.hv[0]};
  for (int f = 0; f < 4 && e == cudaSuccess; ++f) {
    const void *in = pinned_device_ptr(srcs[f], nb);
    if (!in) {
      e = cudaMemcpyAsync(sl.staging, srcs[f], nb, cudaMemcpyHostToDevice, b->stream);
      in = sl.staging;
    }
    if (e == cudaSuccess)
      e = import_plane<T>(in, true, dsts[f], f == 1 ? bplane : nullptr, sl.p.z_ref, sl.nx, sl.ny, sl.pitch, b->stream);
  }
  if (e == cudaSuccess) e = reset_scalars(b->d_sc + s, b->d_cta + s, 0.0, b->cfl, sl.t_end, b->stream);
  if (e == cudaSuccess) e = state_stats<T>(fd, sl.p, b->d_sc + s, b->stream);
  return e;
}

// A live slot's state to host FP64 arrays and its mass (synchronous).
template <typename T>
cudaError_t slot_state(swe_batch *b, Slot &sl, double *const dst[3]) {
  const Field<T> &fd = field_of<T>(sl);
  const size_t nb = sizeof(double) * (size_t)sl.nx * sl.ny;
  const T *src[3] = {fd.h[0], fd.hu[0], fd.hv[0]};
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    void *out = const_cast<void *>(pinned_device_ptr(dst[f], nb));
    e = export_plane<T>(src[f], out ? out : sl.staging, true, f == 0 ? fd.b : nullptr, sl.p.z_ref, sl.nx, sl.ny,
                        sl.pitch, b->stream);
    if (e == cudaSuccess && !out) e = cudaMemcpyAsync(dst[f], sl.staging, nb, cudaMemcpyDeviceToHost, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}
template <typename T>
cudaError_t slot_mass(swe_batch *b, Slot &sl, double *mass) {
  const Field<T> &fd = field_of<T>(sl);
  cudaError_t e = swe::mass<T>(fd.h[0], fd.b, sl.p.z_ref, sl.nx, sl.ny, sl.pitch, sl.dx * sl.dy, b->d_part,
                               b->d_part + kMassBlocks, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mass, b->d_part + kMassBlocks, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

}  // namespace

extern "C" {

size_t swe_batch_slot_bytes(const swe_grid *grid) {
  if (!grid || grid->nx < 3 || grid->ny < 3) return 0;
  return slot_bytes(grid->nx, grid->ny);
}

int swe_batch_create(int32_t nslots, size_t hbm_budget_bytes, const swe_params *params, swe_batch **out) {
  const TraceRange trace("swe_batch_create");
  if (out) *out = nullptr;
  if (!out || !params || nslots < 1 || nslots > 4096 || hbm_budget_bytes == 0) return SWE_EINVAL;
  if (params->fused_step) return SWE_EINVAL;             // the batch runs the paper's per-stage alpha
  if (!valid_params(params)) return SWE_EINVAL;          // sides and physics as for one scenario
  const bool f64 = params->precision == SWE_F64;         // FP64: one compiled tile shape
  if (f64 && params->tile != 0 && params->tile != batch64_shape()) return SWE_EINVAL;
  const bool shore = params->shore != 0;                 // the shoreline variant: one compiled shape per precision
  if (shore && !f64 && params->tile != 0 && params->tile != batch_shore_shape()) return SWE_EINVAL;
  swe_batch *b = new (std::nothrow) swe_batch();
  if (!b) return SWE_ENOMEM;
  b->nslots = nslots;
  b->budget = hbm_budget_bytes;
  b->prm = *params;
  b->prec = f64 ? SWE_F64 : SWE_F32;
  b->elem = f64 ? sizeof(double) : sizeof(float);
  if (f64) b->tile = batch64_shape();
  else if (shore) b->tile = batch_shore_shape();
  else if (params->tile > 0) b->tile = params->tile;
  else {
    const int cached = swe_autotune_lookup(SWE_F32, 1, 0.0);
    b->tile = cached > 0 ? cached : 1;
  }
  b->stream = (cudaStream_t)params->stream;
  b->slots.resize(nslots);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dev_malloc((void **)&b->d_sc, sizeof(DevScalars) * nslots);
  if (e == cudaSuccess) e = dev_malloc((void **)&b->d_cta, sizeof(DevPartials) * nslots);
  if (e == cudaSuccess) e = dev_malloc(&b->d_table, sizeof(BatchSlot<double>) * nslots);
  if (e == cudaSuccess) e = dev_malloc((void **)&b->d_ctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = dev_malloc((void **)&b->d_part, sizeof(double) * (kMassBlocks + 1));
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = f64 ? batch64_resident(shore, &per_sm) : (shore ? batch_shore_resident(&per_sm) : batch_resident(b->tile, &per_sm));
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && (per_sm < 1 || per_sm * sms > kPartSlots)) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) {
    int rc = bfail(b, e);
    swe_batch_destroy(b);
    return rc;
  }
  b->grid = per_sm * sms;
  int rc = upload_table(b);
  if (rc != SWE_OK) {
    swe_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SWE_OK;
}

int swe_batch_admit(swe_batch *b, const swe_grid *grid, double dx, double dy, const double *bathymetry,
                    const double *h, const double *hu, const double *hv, double t_end, int32_t *slot) {
  const TraceRange trace("swe_batch_admit");
  if (slot) *slot = -1;
  if (!b || !grid || !bathymetry || !h || !hu || !hv || !slot) return SWE_EINVAL;
  if (grid->nx < 3 || grid->ny < 3 || !(dx > 0.0) || !(dy > 0.0) || !(t_end > 0.0)) return SWE_EINVAL;
  if ((long long)grid->nx * grid->ny > (1ll << 31)) return SWE_EINVAL;
  const size_t need = slot_bytes(grid->nx, grid->ny, b->elem);
  if (b->used + need > b->budget) return SWE_EBUDGET;
  int s = -1;
  for (int k = 0; k < b->nslots; ++k)
    if (!b->slots[k].live) { s = k; break; }
  if (s < 0) return SWE_EFULL;
  Slot &sl = b->slots[s];
  sl = Slot();
  sl.nx = grid->nx;
  sl.ny = grid->ny;
  sl.dx = dx;
  sl.dy = dy;
  sl.t_end = t_end;
  const size_t plane = plane_bytes(sl.nx, sl.ny, &sl.pitch, b->elem);
  cudaError_t e = dev_malloc_async(&sl.mem, need, b->stream);
  if (e == cudaErrorMemoryAllocation) {  // no room now: the batch is unchanged and usable
    (void)cudaGetLastError();
    sl = Slot();
    return SWE_ENOMEM;
  }
  if (e != cudaSuccess) return bfail(b, e);
  const double *srcs[4] = {bathymetry, h, hu, hv};
  e = b->prec == SWE_F64 ? fill_slot<double>(b, sl, s, plane, srcs) : fill_slot<float>(b, sl, s, plane, srcs);
  if (e != cudaSuccess) {
    cudaFreeAsync(sl.mem, b->stream);
    sl = Slot();
    return bfail(b, e);
  }
  sl.live = true;
  sl.bytes = need;
  b->used += need;
  const int rc = upload_table(b);
  if (rc != SWE_OK) return rc;
  *slot = s;
  return SWE_OK;
}

int swe_batch_run(swe_batch *b, int32_t k_steps, double cfl) {
  const TraceRange trace("swe_batch_run");
  if (!b || k_steps < 0 || !(cfl > 0.0)) return SWE_EINVAL;
  if (b->sticky != SWE_OK) return b->sticky;
  if (k_steps == 0) return SWE_OK;
  cudaError_t e = cudaSuccess;
  if (cfl != b->cfl) {
    for (int s = 0; s < b->nslots && e == cudaSuccess; ++s)
      if (b->slots[s].live) e = set_cfl(b->d_sc + s, cfl, b->stream);
    if (e != cudaSuccess) return bfail(b, e);
    b->cfl = cfl;
  }
  // one graph per step count, work order and kernel form
  const int key = 4 * k_steps + (b->small ? 2 : 0) + (b->strided ? 1 : 0);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaMemsetAsync(&b->d_ctl->bar_count, 0, sizeof(unsigned), b->cap);
      if (le == cudaSuccess) {
        if (b->prec == SWE_F64)
          le = batch64_launch((const BatchSlot<double> *)b->d_table, b->d_ctl, k_steps, b->grid, b->strided,
                              b->prm.shore != 0, b->cap);
        else if (b->prm.shore)
          le = batch_shore_launch((const BatchSlot<float> *)b->d_table, b->d_ctl, k_steps, b->grid, b->strided, b->cap);
        else
          le = batch_launch(b->tile, (const BatchSlot<float> *)b->d_table, b->d_ctl, k_steps, b->grid, b->strided,
                            b->small, b->cap);
      }
      e = cudaStreamEndCapture(b->cap, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, e);
    it = b->graphs.emplace(key, ex).first;
  }
  e = cudaGraphLaunch(it->second, b->stream);
  return bfail(b, e);
}

int swe_batch_status(swe_batch *b) {
  if (!b) return SWE_EINVAL;
  if (b->sticky != SWE_OK) return b->sticky;
  BatchCtl c;
  cudaError_t e = cudaMemcpyAsync(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  return (c.status & ST_TIMEOUT) ? SWE_ETIMEOUT : SWE_OK;
}

int swe_batch_poll(swe_batch *b, int32_t *done_slots, int32_t *ndone) {
  const TraceRange trace("swe_batch_poll");
  if (!b || !ndone) return SWE_EINVAL;
  *ndone = 0;
  std::vector<DevScalars> h(b->nslots);
  cudaError_t e = cudaMemcpyAsync(h.data(), b->d_sc, sizeof(DevScalars) * b->nslots, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  int n = 0;
  for (int s = 0; s < b->nslots; ++s) {
    if (!b->slots[s].live) continue;
    if (h[s].t >= b->slots[s].t_end || h[s].status != 0u) {
      if (done_slots) done_slots[n] = s;
      ++n;
    }
  }
  *ndone = n;
  return swe_batch_status(b);
}

int swe_batch_select(swe_batch *b, const int32_t *slots, int32_t n) {
  if (!b) return SWE_EINVAL;
  if (slots && n > 0) {
    for (int32_t k = 0; k < n; ++k)
      if (!valid_slot(b, slots[k])) return SWE_EINVAL;
    for (auto &sl : b->slots) sl.selected = false;
    for (int32_t k = 0; k < n; ++k) b->slots[slots[k]].selected = true;
  } else {
    for (auto &sl : b->slots) sl.selected = true;
  }
  return upload_table(b);
}

int swe_batch_set_time(swe_batch *b, int32_t slot, double t) {
  if (!valid_slot(b, slot) || !std::isfinite(t) || !(t < b->slots[slot].t_end)) return SWE_EINVAL;
  DevScalars *sc = b->d_sc + slot;
  cudaError_t e = cudaMemcpyAsync(&sc->t, &t, sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sc->t_step, &t, sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? SWE_OK : bfail(b, e);
}

int swe_batch_times(swe_batch *b, double *t) {
  if (!b || !t) return SWE_EINVAL;
  std::vector<DevScalars> h(b->nslots);
  cudaError_t e = cudaMemcpyAsync(h.data(), b->d_sc, sizeof(DevScalars) * b->nslots, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  for (int s = 0; s < b->nslots; ++s) t[s] = b->slots[s].live ? h[s].t : NAN;
  return SWE_OK;
}

int swe_batch_diagnostics(swe_batch *b, int32_t slot, swe_diag *d) {
  if (!valid_slot(b, slot) || !d) return SWE_EINVAL;
  DevScalars h;
  cudaError_t e = cudaMemcpyAsync(&h, b->d_sc + slot, sizeof(h), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = read_volumes(b->d_cta + slot, &d->clamp_mass, &d->boundary_mass, b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  auto dbl = [](unsigned long long u) { double x; std::memcpy(&x, &u, 8); return x; };
  d->t = h.t;
  d->steps = h.steps;
  d->last_dt = h.dt;
  d->alpha_x = dbl(h.alpha[0][0]);
  d->alpha_y = dbl(h.alpha[0][1]);
  const unsigned long long rn = h.runup_now[(h.steps + 1) & 1];
  d->runup_now = rn ? dbl(rn) : -INFINITY;
  d->runup_max = h.runup_max ? dbl(h.runup_max) : -INFINITY;
  d->tile = b->tile;
  d->status = (h.status & ST_NONFINITE) ? SWE_ENONFINITE : ((h.status & ST_DRY) ? SWE_EINVAL : SWE_OK);
  const int bs = swe_batch_status(b);
  if (bs != SWE_OK) d->status = bs;
  return d->status;
}

int swe_batch_get_state(swe_batch *b, int32_t slot, double *h, double *hu, double *hv) {
  const TraceRange trace("swe_batch_get_state");
  if (!valid_slot(b, slot) || !h || !hu || !hv) return SWE_EINVAL;
  Slot &sl = b->slots[slot];
  double *dst[3] = {h, hu, hv};
  const cudaError_t e = b->prec == SWE_F64 ? slot_state<double>(b, sl, dst) : slot_state<float>(b, sl, dst);
  return bfail(b, e);
}

int swe_batch_retire(swe_batch *b, int32_t slot, double *h, double *hu, double *hv, double *mass, double *runup_max) {
  const TraceRange trace("swe_batch_retire");
  if (!valid_slot(b, slot)) return SWE_EINVAL;
  Slot &sl = b->slots[slot];
  int rc = SWE_OK;
  if (h && hu && hv) rc = swe_batch_get_state(b, slot, h, hu, hv);
  if (rc == SWE_OK && mass)
    rc = bfail(b, b->prec == SWE_F64 ? slot_mass<double>(b, sl, mass) : slot_mass<float>(b, sl, mass));
  if (rc == SWE_OK && runup_max) {
    swe_diag d;
    swe_batch_diagnostics(b, slot, &d);
    *runup_max = d.runup_max;
  }
  if (rc != SWE_OK) return rc;
  cudaError_t e = cudaFreeAsync(sl.mem, b->stream);
  b->used -= sl.bytes;
  sl = Slot();
  if (e != cudaSuccess) return bfail(b, e);
  return upload_table(b);
}

int swe_batch_check_status(swe_batch *b, int32_t slot, uint64_t *word) {
  if (!valid_slot(b, slot) || !word) return SWE_EINVAL;
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, &(b->d_sc + slot)->check, sizeof(w), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  *word = (uint64_t)w;
  return SWE_OK;
}

int swe_batch_memory(swe_batch *b, size_t *used, size_t *budget) {
  if (!b) return SWE_EINVAL;
  if (used) *used = b->used;
  if (budget) *budget = b->budget;
  return SWE_OK;
}

int swe_batch_set_barrier(swe_batch *b, double timeout_s, int32_t extra_arrivals) {
  if (!b || !(timeout_s > 0.0) || extra_arrivals < 0) return SWE_EINVAL;
  b->timeout_s = timeout_s;
  b->extra = (unsigned)extra_arrivals;
  b->sticky = SWE_OK;
  return upload_table(b);  // also clears the barrier words and the status
}

int swe_batch_destroy(swe_batch *b) {
  if (!b) return SWE_OK;
  cudaStreamSynchronize(b->stream);
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &sl : b->slots)
    if (sl.mem) cudaFreeAsync(sl.mem, b->stream);
  cudaStreamSynchronize(b->stream);
  if (b->d_sc) cudaFree(b->d_sc);
  if (b->d_cta) cudaFree(b->d_cta);
  if (b->d_table) cudaFree(b->d_table);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_part) cudaFree(b->d_part);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return SWE_OK;
}

}  // extern "C"
