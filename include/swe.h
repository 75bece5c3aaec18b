/*
 * swe.h -- C ABI of the GB300 (sm_103a) shallow-water solver.
 *
 * The solver advances the 2-D nonlinear shallow-water equations of the paper
 * (Madden, Marras & Suckale, arXiv:2301.12010, "Numerical approximation",
 * Eqs. (1)-(3)) with fifth-order WENO reconstruction and global
 * Lax-Friedrichs flux splitting in x and y (Eqs. (5)-(6)), the well-balanced
 * bed source term and explicit Manning friction, advanced by the TVD
 * (SSP) Runge-Kutta scheme of Eq. (8).  The caller supplies bathymetry and an
 * initial state, the library advances it, and the caller gathers results:
 * the division of labour of the paper's "TPU implementation" (host
 * initialises, device steps, host gathers).
 *
 * Conventions (all calls):
 *  - Arrays are row-major [ny][nx] with x fastest, SI units (m, m^2/s).
 *  - Host arrays passed to the library are FP64 and are copied; the caller
 *    keeps ownership.  Device arrays (the *_device calls) are contiguous
 *    [ny][nx] of the handle's precision (float for SWE_F32, double for
 *    SWE_F64) and stay owned by the caller.
 *  - Every call returns an SWE_* status.  No call aborts and no device code
 *    traps.  Errors raised by asynchronous work (swe_step) surface at the next
 *    synchronising call (swe_get_state, swe_mass, swe_runup, swe_get_time,
 *    swe_diagnostics, swe_sync) or at swe_status.
 *  - A handle is not thread-safe: one host thread at a time.
 *  - Grids need nx >= 3 and ny >= 3 (the WENO5 ghost width).
 */
#ifndef SWE_H
#define SWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
  SWE_OK = 0,
  SWE_EINVAL = 1,     /* invalid argument, or CFL time step undefined (fully dry, still domain) */
  SWE_ENOMEM = 2,     /* device or host allocation failed */
  SWE_ECUDA = 3,      /* a CUDA call failed (kernel launch, copy, graph) */
  SWE_ENONFINITE = 4, /* NaN/Inf met in a reduction; later stages were skipped */
  SWE_ETIMEOUT = 5,   /* a bounded device-side wait expired (persistent batch barrier) */
  SWE_EBUDGET = 6,    /* admission would exceed the batch's HBM budget */
  SWE_EFULL = 7       /* no free batch slot */
};

typedef enum { SWE_F32 = 0, SWE_F64 = 1 } swe_precision;

/* Boundary types, per side.  WALL: free-slip, no-penetration wall (the
 * tsunami runs of "Validation for tsunami simulations": ghost cells mirror
 * depth, bed and tangential momentum and negate normal momentum).  INFLOW
 * (x- side only): ghost cells carry the Carrier N-wave of Eq. (20) in time
 * with amplitude inflow_amp (peak elevation), period inflow_period and
 * offshore depth inflow_depth, as an incoming long wave.  PERIODIC (tests):
 * wrap-around, with the bed offset b_jump_x/y added across the seam. */
typedef enum { SWE_BC_WALL = 0, SWE_BC_INFLOW = 1, SWE_BC_PERIODIC = 2 } swe_bc;

typedef struct {
  int32_t nx, ny; /* interior cells along x and y */
} swe_grid;

typedef struct {
  double g;             /* gravity, 9.81 m s^-2 (Eqs. (1)-(3)) */
  double manning_n;     /* Manning n of Eqs. (2)-(3); 0 disables friction */
  double h_dry;         /* depth below which a cell is dry (compared in FP64); 1e-5 m */
  double h_wet;         /* depth from which a land cell (b > 0) counts for runup; 1e-3 m */
  double h_film;        /* films with h_dry <= h < h_film get the Kurganov-Petrova velocity
                           desingularisation hu := sqrt(2) h^2 hu / sqrt(h^4 + h_film^4); 1e-3 m */
  double weno_eps;      /* WENO5 epsilon; 1e-6 */
  double fixed_dt;      /* > 0: fixed time step (the paper's runs use 5e-3 s); else CFL */
  double z_ref;         /* still-water level of the bed splitting; 0 m */
  double b_jump_x;      /* PERIODIC x: b(i + nx) = b(i) + b_jump_x */
  double b_jump_y;      /* PERIODIC y: b(j + ny) = b(j) + b_jump_y */
  double inflow_amp;    /* INFLOW: peak surface elevation (m) */
  double inflow_period; /* INFLOW: N-wave period T (s) */
  double inflow_depth;  /* INFLOW: offshore depth d0 (m) */
  double alpha_margin;  /* fused_step: splitting speed = alpha_margin x alpha(U^n), >= 1; 1.1 */
  int32_t bc[4];        /* sides x-, x+, y-, y+ (swe_bc) */
  int32_t precision;    /* swe_precision of state and arithmetic */
  int32_t tile;         /* 0: autotuned/default tile shape; k > 0: compiled shape k */
  int32_t fused_step;   /* 0: one kernel per RK stage with the paper's per-stage alpha (Eq. (8) with
                           Eq. (6) at every stage); 1: the fused-step variant, one kernel per step
                           splitting all three stages with alpha_margin x alpha(U^n) (walls and the
                           inflow edge only; not a batch or strip option) */
  int32_t shore;        /* 0: WENO at every face (the paper); 1: the shoreline variant, first-order
                           hydrostatic-reconstruction faces (Audusse et al. 2004) wherever a WENO
                           stencil meets a dry cell, so that lakes at rest at or below z_ref stay at
                           rest beside dry land (tile 0 or its one compiled shape: 96x32 in FP32,
                           64x32 in FP64; also a batch option, on 96x32 in FP32 and 32x32 in FP64; not
                           a strip or fused_step option) */
  void *stream;         /* cudaStream_t to run on (e.g. torch.cuda.Stream().cuda_stream); NULL = legacy default */
} swe_params;

typedef struct {
  double t;             /* simulated time of the current state */
  int64_t steps;        /* RK3 steps taken since the last swe_set_time/swe_create */
  double last_dt;       /* time step of the last step */
  double alpha_x;       /* global max |u| + sqrt(g h) of the current state */
  double alpha_y;       /* global max |v| + sqrt(g h) of the current state */
  double clamp_mass;    /* mass added by the h < 0 clamp, RK-weighted (m^3) */
  double boundary_mass; /* mass that entered through the edges, RK-weighted (m^3) */
  double runup_now;     /* max h+b over land cells (b > 0) with h >= h_wet; -inf if none */
  double runup_max;     /* running maximum of runup_now */
  int32_t status;       /* SWE_* status of the device work so far */
  int32_t tile;         /* tile shape in use */
} swe_diag;

typedef struct swe_handle swe_handle; /* opaque; owns its device memory */

/* Fill *p with the defaults listed above (walls on all sides, FP32). */
void swe_params_default(swe_params *p);

/* Create a solver for grid *grid with spacings dx, dy (m) over the host FP64
 * bathymetry b[ny][nx] (m, positive up).  Allocates all device memory the
 * stepping needs; no later call allocates.  Until swe_set_state the state is
 * still water at z_ref.  *out receives the handle, or NULL on error. */
int swe_create(const swe_grid *grid, double dx, double dy, const double *bathymetry,
               const swe_params *params, swe_handle **out);

/* Copy a host FP64 state h, hu, hv [ny][nx] to the device (converted to the
 * handle's precision), and evaluate the wave speeds and runup of that
 * state.  Synchronous. */
int swe_set_state(swe_handle *s, const double *h, const double *hu, const double *hv);

/* Same from device arrays of the handle's precision (contiguous [ny][nx],
 * owned by the caller, read on the handle's stream). */
int swe_set_state_device(swe_handle *s, const void *h, const void *hu, const void *hv);

/* Asynchronous form of swe_set_state for page-locked host FP64 arrays
 * [ny][nx] (cudaHostAlloc, cudaHostRegister, a pinned torch tensor): returns
 * at once; copy engines carry the arrays to the device on a second stream
 * (overlapping steps and read-backs already enqueued), and the conversion
 * into the state, the wave speeds and the runup follow on the handle's
 * stream, so that the next swe_step uses the new state.  The time is kept.
 * The arrays must stay unchanged until the next synchronising call
 * (swe_sync, swe_get_state, swe_wait_state, swe_diagnostics).  Pageable
 * arrays: swe_set_state (synchronous).  Two staging slots of 3 FP64 planes
 * each are used in turn, so that an upload need not wait for the conversion
 * of the one before it (only for that of the one before last); they are
 * allocated at the first call, and SWE_ENOMEM leaves the handle usable. */
int swe_set_state_async(swe_handle *s, const double *h, const double *hu, const double *hv);

/* Enqueue n RK3 steps (Eq. (8)) on the handle's stream.  Each step runs three
 * stage kernels; the time step is dt = cfl / (alpha_x/dx + alpha_y/dy) from
 * the step's first stage (ignored if fixed_dt > 0).  Asynchronous: no host
 * synchronisation; steps are replayed from a captured CUDA graph.  With
 * fused_step each step is one kernel (between two one-thread bookkeeping
 * kernels) that reads U^n and writes U^{n+1} into a second set of planes;
 * steps are replayed in pairs, and an odd n ends with a device copy of the
 * state back into the first set. */
int swe_step(swe_handle *s, int32_t n, double cfl);

/* Wait for the handle's stream and report the device status. */
int swe_sync(swe_handle *s);

/* Copy the current state to host FP64 arrays [ny][nx].  Synchronises. */
int swe_get_state(swe_handle *s, double *h, double *hu, double *hv);

/* Start copying the current state to host FP64 arrays [ny][nx] and return at
 * once: the state is converted on the device into one of two staging slots
 * of 3 FP64 planes (on the handle's stream, in stream order after the steps
 * enqueued so far) and a copy engine carries the slot to the arrays on a
 * second stream, so that later calls (swe_set_state, swe_step) overlap the
 * copy.  The arrays must each be one page-locked allocation (cudaHostAlloc,
 * cudaHostRegister, a pinned torch tensor); they hold the state once
 * swe_wait_state returns and must not be read or freed before.  With
 * pageable arrays this is swe_get_state (synchronous).  The slots are used in
 * turn: a call waits on the device for the copy of the read-back before last
 * to finish before it converts into that slot.  The slots are allocated at
 * the first call; SWE_ENOMEM leaves the handle usable.  No counterpart in the
 * paper: an interface for pipelining input upload and result read-back. */
int swe_get_state_async(swe_handle *s, double *h, double *hu, double *hv);

/* Bounded-wait settings of the halo-box copies of the stage kernels: a wait
 * gives up after timeout_s seconds (default 1, at most 60), the kernel flags
 * a timeout, and later calls report SWE_ETIMEOUT until the state is set again
 * (swe_set_state); the step in which it happened did not complete.
 * extra_copy_bytes > 0 (at most 65536) is a test hook that makes every wait
 * expect bytes that never arrive, so that the timeout path can be exercised
 * without a fault; 0 for normal use.  Synchronises.  No counterpart in the
 * paper. */
int swe_set_wait(swe_handle *s, double timeout_s, int32_t extra_copy_bytes);

/* Test hook for the error paths: the n-th device allocation the library
 * makes from now on (handle and batch creation, a batch admission, the first
 * asynchronous read-back's buffers) fails as if the device were out of
 * memory, and the call that made it returns SWE_ENOMEM with nothing leaked
 * and its handle or batch still usable; later allocations succeed again.
 * n = 0 disarms; n < 0 gives SWE_EINVAL.  Process-wide, thread-safe.  No
 * counterpart in the paper. */
int swe_debug_fail_alloc(int32_t n);

/* Wait for the read-backs started by swe_get_state_async (no-op if none);
 * returns the handle's first error, if any. */
int swe_wait_state(swe_handle *s);

/* Copy the current state into caller device arrays of the handle's
 * precision (contiguous [ny][nx]).  Synchronises. */
int swe_get_state_device(swe_handle *s, void *h, void *hu, void *hv);

/* Total water volume sum(h) dx dy (FP64, fixed summation order) and the
 * clamp-added volume.  Synchronises. */
int swe_mass(swe_handle *s, double *mass, double *clamp_mass);

/* Runup: running maximum and current value (m; -inf if no wet land cell).
 * Synchronises. */
int swe_runup(swe_handle *s, double *runup_max, double *runup_now);

/* Simulated time and step count.  Synchronises. */
int swe_get_time(swe_handle *s, double *t, int64_t *steps);

/* Set the simulated time (resume from a checkpoint); resets the step count. */
int swe_set_time(swe_handle *s, double t);

/* Simulated-time horizon: with t_end > 0 the step that would pass t_end is
 * shortened to end on it and later steps do nothing (no error; the step count
 * stops), as a run to a set output time does; 0 removes the horizon.  Kept
 * across swe_set_state*.  Synchronises.  SWE_EINVAL for a negative or
 * non-finite t_end. */
int swe_set_horizon(swe_handle *s, double t_end);

/* All diagnostics at once.  Synchronises. */
int swe_diagnostics(swe_handle *s, swe_diag *d);

/* Status of the device work so far, without waiting for it. */
int swe_status(swe_handle *s);

/* Static text for a status code. */
const char *swe_strerror(int code);

/* Free the handle and its device memory.  NULL-safe; returns SWE_OK. */
int swe_destroy(swe_handle *s);

/* 1 if this library is the checked build (libswe_checked.so, compiled with
 * SWE_CHECKED), else 0.  The checked build compares every index into a
 * tile's shared-memory halo box and flux buffer and into a global plane with
 * its extent before the access; an index out of range is recorded (the first
 * one) and the access skipped, with no trap.  It stands in for a memory
 * checker on devices where none can run.  No counterpart in the paper. */
int swe_checked_build(void);

/* The handle's check word (checked build): 0 if no index was out of range so
 * far, else bit 63 set, the access site in bits 40..47 (1 ghost write, 2 wall
 * mirror read, 3 periodic read, 4 x-pass box chunk, 5 box cell, 6/7 x-pass
 * epilogue box/flux buffer, 8/9 y-pass epilogue box/flux buffer, 10 output
 * plane, 11 U^n read) and the index in bits 0..39.  Always 0 in the normal
 * build.  Reset by swe_set_state.  Synchronises. */
int swe_check_status(swe_handle *s, uint64_t *word);

/* Number of compiled tile shapes and the shape of entry k (1-based). */
int swe_tile_count(void);
int swe_tile_shape(int k, int32_t *tx, int32_t *ty, int32_t *threads);

/* Timing helper for benchmarks: enqueue n steps as individual stage launches
 * (not the graph) with a CUDA event recorded on the handle's stream around
 * each stage kernel, wait, and return the summed milliseconds of whole steps
 * (*ms_total) and of each stage kernel (ms_stage[3], may be NULL).  With
 * fused_step: ms_stage[0] is the fused kernel's time, ms_stage[1] that of the
 * two bookkeeping kernels, ms_stage[2] zero. */
int swe_time_stages(swe_handle *s, int32_t n, double cfl, double *ms_total, double *ms_stage);

/* Tile-shape autotuner (native timing loop).  Times every compiled tile
 * shape for `steps` RK3 steps on a synthetic moving-water scenario: of grid
 * grids[0] on the single-scenario path (mode 0), or of all ngrids grids in
 * one batch (mode 1, FP32).  Returns the fastest shape in *best_tile and the
 * milliseconds per step of each shape in ms_per_step[swe_tile_count()] (may be
 * NULL; -1 for a shape that does not fit), and records the winner in a JSON
 * cache ($SWE_AUTOTUNE_CACHE, default ~/.cache/swe_gb300_autotune.json) keyed
 * by GPU name, precision, mode and size bucket (log2 of the cell count; one
 * entry for batches).  swe_create and swe_batch_create use the cached shape
 * when params->tile == 0 (shape 1 if there is none).  Allocates and frees
 * its own scratch handles; synchronises. */
int swe_autotune(const swe_grid *grids, int32_t ngrids, int32_t precision, int32_t mode, int32_t steps,
                 int32_t *best_tile, double *ms_per_step);

/* Cached shape for (precision, mode, cell count), or 0 if none. */
int swe_autotune_lookup(int32_t precision, int32_t mode, double cells);

/* ----------------------------------------------------------------------
 * Batched ensemble and continuous-batching serving (FP32; FP64 for parity).
 * A batch holds up to nslots independent scenarios ("slots") of any grid
 * size, admitted while device memory stays within hbm_budget_bytes.
 * swe_batch_run advances every live slot by up to k RK3 steps (each slot
 * with its own CFL time step, stopping at its t_end) in ONE cooperative
 * persistent kernel launch over a work list of (scenario, tile) pairs,
 * with a bounded grid barrier between the three RK stages, replayed from a
 * CUDA graph.  Each scenario keeps its own wave speeds, dt, time and step
 * count on the device, so its result is the same alone and in any mix.
 * ---------------------------------------------------------------------- */
typedef struct swe_batch swe_batch;

/* Device bytes one admission of this grid takes in an FP32 batch (counted
 * against the budget; an FP64 batch counts its ten planes at 8 bytes). */
size_t swe_batch_slot_bytes(const swe_grid *grid);

/* Create an empty batch.  params: fused_step 0; the sides (walls, the inflow
 * edge, periodic pairs) and the physical parameters are those of every slot,
 * under the rules of swe_create; precision SWE_F32 (tile 0 picks the default
 * shape) or SWE_F64 (the parity mode: its one compiled shape, 32x32, taken
 * for tile 0); shore 1 runs the shoreline variant on the precision's one
 * compiled shape for it (96x32 in FP32, 32x32 in FP64); stream as for
 * swe_create.  SWE_EINVAL otherwise. */
int swe_batch_create(int32_t nslots, size_t hbm_budget_bytes, const swe_params *params, swe_batch **out);

/* Admit a scenario: host FP64 bathymetry and state [ny][nx] (copied), run until
 * simulated time t_end (> 0).  Allocates the slot's device memory stream-ordered
 * (cudaMallocAsync).  Returns the slot index in *slot; SWE_EBUDGET if the
 * budget would be exceeded, SWE_EFULL if no slot is free, SWE_ENOMEM if the
 * device has no room now (the batch is unchanged and usable in all three
 * cases).  Call between runs. */
int swe_batch_admit(swe_batch *b, const swe_grid *grid, double dx, double dy, const double *bathymetry,
                    const double *h, const double *hu, const double *hv, double t_end, int32_t *slot);

/* Set a live slot's simulated time (its inflow N-wave is read at that time;
 * t_end stays absolute).  Call between runs, before the slot's first run. */
int swe_batch_set_time(swe_batch *b, int32_t slot, double t);

/* Enqueue one persistent launch of k RK3 steps over all live slots with the
 * given CFL number (asynchronous; slots past t_end are skipped). */
int swe_batch_run(swe_batch *b, int32_t k_steps, double cfl);

/* List live slots that reached t_end or failed (synchronises).  done_slots
 * must hold nslots entries (may be NULL to count only). */
int swe_batch_poll(swe_batch *b, int32_t *done_slots, int32_t *ndone);

/* Copy a live slot's state to host FP64 arrays [ny][nx] (synchronises). */
int swe_batch_get_state(swe_batch *b, int32_t slot, double *h, double *hu, double *hv);

/* Diagnostics of a live slot (synchronises). */
int swe_batch_diagnostics(swe_batch *b, int32_t slot, swe_diag *d);

/* Copy out (any pointer may be NULL) and free a slot (stream-ordered free). */
int swe_batch_retire(swe_batch *b, int32_t slot, double *h, double *hu, double *hv, double *mass,
                     double *runup_max);

/* Restrict the following runs to the n live slots listed (the others keep
 * their state and resume when selected again); slots == NULL or n <= 0
 * selects every live slot, as after swe_batch_create.  Admitted slots are
 * selected.  EINVAL if a listed slot is not live.  Call between runs.  No
 * counterpart in the paper: a scheduling hook for the serving loop. */
int swe_batch_select(swe_batch *b, const int32_t *slots, int32_t n);

/* Simulated time of every slot (t[0 .. nslots-1]; NaN for free slots) in one
 * read-back.  Synchronises. */
int swe_batch_times(swe_batch *b, double *t);

/* The check word of a live slot (see swe_check_status); 0 in the normal
 * build.  Synchronises. */
int swe_batch_check_status(swe_batch *b, int32_t slot, uint64_t *word);

/* Device bytes in use by live slots and the budget. */
int swe_batch_memory(swe_batch *b, size_t *used, size_t *budget);

/* SWE_ETIMEOUT if a grid-barrier wait ran out in a run (the launch then
 * ended early; slots keep their last completed stage), else SWE_OK. */
int swe_batch_status(swe_batch *b);

/* Bounded-wait settings of the grid barrier: give up after timeout_s seconds
 * (default 1).  extra_arrivals > 0 is a test hook that makes every barrier
 * wait for arrivals that never come, so the timeout path can be exercised;
 * 0 for normal use.  Also clears a timeout status.  Call between runs. */
int swe_batch_set_barrier(swe_batch *b, double timeout_s, int32_t extra_arrivals);

/* Free the batch and all slots.  NULL-safe. */
int swe_batch_destroy(swe_batch *b);

/* ----------------------------------------------------------------------
 * Row-partitioned domain: the paper's parallel scheme ("TPU
 * implementation", Table 1: the domain split among TPU cores, halos
 * exchanged every RK stage, the wave speed reduced across cores).  The grid
 * is cut along y into nparts strips of whole rows (boundaries on multiples
 * of 32 rows when strips hold 64 rows or more; swe_strip_bounds); each strip
 * keeps three halo rows above and
 * below.  Every RK stage runs the stage kernel over each strip and then
 * copies every strip's three boundary rows of the stage output into its
 * neighbours' halo rows; the wave speeds of a stage are one maximum over all
 * strips.  The result equals the undivided grid's (swe_create) bit for bit.
 * The strips run on the calling device, one after another on one stream.
 * The y sides must be walls (SWE_EINVAL otherwise); x sides as swe_create.
 * Arrays are full-grid [ny][nx] host FP64, as for swe_create.
 * ---------------------------------------------------------------------- */
typedef struct swe_multi swe_multi;

/* Strip k (0-based) of a partition of ny rows into nparts strips: first row
 * and row count.  SWE_EINVAL if a strip would hold fewer than 3 rows.  Host
 * only (no device work). */
int swe_strip_bounds(int32_t ny, int32_t nparts, int32_t k, int32_t *row0, int32_t *rows);

/* Create a row-partitioned solver (as swe_create, nparts strips). */
int swe_multi_create(const swe_grid *grid, double dx, double dy, const double *bathymetry,
                     const swe_params *params, int32_t nparts, swe_multi **out);

/* Set the state (host FP64 [ny][nx], copied) and exchange the halos.  Synchronous. */
int swe_multi_set_state(swe_multi *m, const double *h, const double *hu, const double *hv);

/* Set the simulated time; resets the step count. */
int swe_multi_set_time(swe_multi *m, double t);

/* Enqueue n RK3 steps (asynchronous, replayed from a captured CUDA graph). */
int swe_multi_step(swe_multi *m, int32_t n, double cfl);

/* Gather the state into host FP64 arrays [ny][nx].  Synchronises. */
int swe_multi_get_state(swe_multi *m, double *h, double *hu, double *hv);

/* Water volume sum(h) dx dy (FP64; per strip in fixed order, then strip order). */
int swe_multi_mass(swe_multi *m, double *mass);

/* Diagnostics of the whole domain (as swe_diagnostics).  Synchronises. */
int swe_multi_diagnostics(swe_multi *m, swe_diag *d);

/* Free the solver.  NULL-safe. */
int swe_multi_destroy(swe_multi *m);

/* Allocation-free water volume of a caller-owned device depth field.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the diagnostic (a process
 * that reserves its whole HBM budget up front, a loop that must not take
 * the device-wide synchronisation of cudaMalloc/cudaFree, or a C host with no
 * allocator or handle).  It computes sum(h) dx dy in FP64 with a fixed
 * summation order, like swe_mass, using a scratch array of one FP64 partial
 * per row that lives in the library's device image (SWE_NOALLOC_MAX_ROWS
 * doubles, held by every device that loads the library until exit).
 *   h         device array [ny][nx] (contiguous) of float (SWE_F32) or double
 *             (SWE_F64), owned by the caller
 *   mass      device pointer to one double, owned by the caller; written when
 *             the enqueued work completes
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream)
 * Returns SWE_EINVAL for null pointers, non-positive sizes or spacings, an
 * unknown precision, or ny > SWE_NOALLOC_MAX_ROWS (checked before any device
 * work); SWE_ECUDA if the launch fails.  Asynchronous; allocates nothing.
 * The first call on a device looks up the scratch array's address and caches
 * it with the device's current context: make that first call before any
 * stream capture on the device.  After cudaDeviceReset the next call looks
 * the address up again in the new context.  All
 * calls on a device share the scratch array, so calls whose work overlaps on
 * the GPU (several streams or host threads) race; calls ordered on one
 * stream are safe and need no clearing in between. */
#define SWE_NOALLOC_MAX_ROWS 16384
int swe_mass_noalloc(const void *h, int32_t precision, int32_t nx, int32_t ny, double dx, double dy,
                     double *mass, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SWE_H */
