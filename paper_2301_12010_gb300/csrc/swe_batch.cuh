// swe_batch.cuh -- device code of the batch path: the slot table, the
// bounded grid barrier and one RK stage over the (scenario, tile) work list
// of a batch, built on the tile arithmetic of swe_core.cuh.  Kept apart from
// the single-scenario driver so that the two evolve separately.
#pragma once
#include "swe_core.cuh"

namespace swe {

// ------------------------------------------------------------ batch driver
// One scenario of a batch as the kernels see it (device memory).
template <typename T>
struct BatchSlot {
  BoxMaps maps[3];  // tensor maps of the halo-box copies, per RK stage
  Field<T> fd;
  Phys p;
  DevScalars *sc;
  int tiles_x, ntiles, first_item, pad;
};

// Batch control block (device memory).
struct BatchCtl {
  int nslots;               // entries of the slot table
  int total_items;          // tiles over all entries (the work list)
  unsigned bar_count;       // grid barrier: arrivals in the current round
  unsigned bar_gen;         // grid barrier: completed rounds
  unsigned status;          // ST_TIMEOUT when a barrier wait ran out
  unsigned bar_extra;       // test hook: arrivals expected beyond the grid (0)
  long long bar_cycles;     // bounded wait: SM clock cycles before giving up
  int strided;              // work order of the table (set by the host; the launch matches it)
  int pad_;
};

// Grid-wide barrier of a cooperative launch with a bounded wait.  Returns
// false if the other CTAs did not arrive in time (ST_TIMEOUT is set) or if
// another CTA already flagged a batch-wide status (that status is kept as
// it is); the caller then leaves the kernel.
__device__ __forceinline__ bool grid_barrier(BatchCtl *ctl, unsigned nblocks) {
  __shared__ unsigned ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1u;
    volatile unsigned *gen = &ctl->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned expect = nblocks + ctl->bar_extra;
    if (atomicAdd(&ctl->bar_count, 1u) == expect - 1u) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*(volatile unsigned *)&ctl->status) {  // another CTA gave up: leave with its status
          ok = 0u;
          break;
        }
        if (clock64() - t0 > ctl->bar_cycles) {
          atomicOr(&ctl->status, ST_TIMEOUT);
          ok = 0u;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();  // acquire: later loads see what other CTAs wrote before the barrier
  }
  __syncthreads();
  return ok != 0u;
}

// The batch kernel reads the tensor maps of its halo-box copies from the slot
// table in global memory, which the host rewrites between launches (a new
// mix, a paused scenario's place taken by another): before a CTA's first copy
// with a scenario's map it acquires that map for the tensor-map proxy, so
// that the copy unit does not act on an older descriptor at that address.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(reinterpret_cast<unsigned long long>(m))
               : "memory");
}

template <typename T>
__device__ __forceinline__ int slot_of_item(const BatchSlot<T> *slots, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (slots[mid].first_item <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__host__ __device__ __forceinline__ StageIO<T> io_of(const Field<T> &fd, int stage) {
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

// One RK stage over the work list of a batch (scenario after scenario, tiles
// in row order).  Contiguous order: CTA b handles the chunk of items
// [b W, (b+1) W), W = ceil(total / G), so that it meets one or two scenarios
// rather than a new one at every item.  Strided order (STRIDED; the host's
// choice when every scenario has at least 2 G tiles): CTA b takes items
// b, b + G, ..., so that the G CTAs work on neighbouring tiles at any time
// (halo rows shared through L2) while each still stays in one scenario for
// runs of items.  Per-scenario scalars are taken when the CTA enters a
// scenario and its accumulators are published when it leaves it; the lead
// CTA of a scenario is the one that owns its tile 0.  Thread 0 walks the
// CTA's items with a cursor that advances without searching the slot table,
// and hands each item's slot and tile origin to the CTA through shared
// memory when it issues the item's halo-box copies: no thread reads the slot
// table on the way to a tile.
template <typename T, int TX, int TY, int NT, int S, int STAGE, bool STRIDED, bool SHORE = false>
__device__ void batch_stage(const BatchSlot<T> *slots, int nslots, int total, T *smem, RedSmem &red, Phys &sp,
                            BatchCtl *ctl, int stage_rt = 0) {
  const int st = STAGE ? STAGE : stage_rt;  // STAGE 0: the stage is given at run time
  using G = TileGeom<T, TX, TY>;
  constexpr unsigned kBoxBytes = 4u * G::BH * G::P * (unsigned)sizeof(T);
  __shared__ unsigned long long bar[2];
  __shared__ unsigned s_fail;
  __shared__ int4 s_item[2];  // (slot, i0, j0) of the item in each box buffer, written when its copies are issued
  __shared__ unsigned s_skip, s_lead;  // the current scenario's skip and lead flags (CTA-uniform)
  __shared__ StageIO<T> s_io;  // planes of the current scenario (kept out of registers)
  T *box0 = smem, *box1 = smem + G::BOX, *sL = smem + 2 * G::BOX;
  const int tid = threadIdx.x;
  const int W = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int item_end = STRIDED ? total : min((int)(blockIdx.x + 1) * W, total);
  const int step = STRIDED ? (int)gridDim.x : 1;
  // the current scenario's per-stage values stay in shared memory (red, s_skip,
  // s_lead) rather than in registers across the item loop
  int cur = -1;
  Acc<T> acc;
  int item = STRIDED ? (int)blockIdx.x : (int)blockIdx.x * W;
  // thread 0's cursor, kept in shared memory (not in every thread's
  // registers): slot of the next item to issue and that slot's tile columns
  // tx; contiguous order: the item's tile column i and row j and the tiles
  // n left in the slot; strided order: the item's tile index i in the slot
  // and the slot's tiles n
  struct Cursor {
    int slot, i, j, tx, n;
  };
  __shared__ Cursor q;
  __shared__ int s_acq;  // slot whose maps this CTA acquired last (thread 0)
  // halo box of the cursor's item by tensor copies into buffer bb, with the
  // tensor maps of its scenario; then the cursor moves to the next item
  auto issue = [&](int bb, unsigned long long *b) {
    Cursor c = q;
    const int i0 = (STRIDED ? c.i % c.tx : c.i) * TX, j0 = (STRIDED ? c.i / c.tx : c.j) * TY;
    s_item[bb] = make_int4(c.slot, i0, j0, 0);
    mbar_expect_tx(b, kBoxBytes);
    const CUtensorMap *m = slots[c.slot].maps[st - 1].m;
    if (c.slot != s_acq) {
#pragma unroll
      for (int f = 0; f < 4; ++f) tensormap_acquire(&m[f]);
      s_acq = c.slot;
    }
    T *dst = bb ? box1 : box0;
#pragma unroll
    for (int f = 0; f < 4; ++f) tma_load_2d(dst + f * G::FIELD, &m[f], i0 - G::OX, j0 - G::OY, b);
    if constexpr (STRIDED) {
      c.i += step;
      while (c.i >= c.n && ++c.slot < nslots) {  // into the next scenario(s)
        c.i -= c.n;
        c.n = slots[c.slot].ntiles;
        c.tx = slots[c.slot].tiles_x;
      }
    } else if (--c.n == 0) {  // next scenario
      if (++c.slot < nslots) {
        c.tx = slots[c.slot].tiles_x;
        c.n = slots[c.slot].ntiles;
      }
      c.i = c.j = 0;
    } else if (++c.i == c.tx) {
      c.i = 0;
      ++c.j;
    }
    q = c;
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1u);
    mbar_init(&bar[1], 1u);
    mbar_fence_init();
    s_fail = 0u;
    s_acq = -1;
    if (item < item_end) {
      const int s0 = slot_of_item(slots, nslots, item);
      const int t = item - slots[s0].first_item, tx = slots[s0].tiles_x;
      q = STRIDED ? Cursor{s0, t, 0, tx, slots[s0].ntiles} : Cursor{s0, t % tx, t / tx, tx, slots[s0].ntiles - t};
      // the buffer may hold the previous stage's ghost patching (generic
      // writes): order them before the tensor copy overwrites it
      fence_proxy_async();
      issue(0, &bar[0]);
    }
  }
  __syncthreads();
  unsigned phase = 0u;  // bit b: parity of the next wait on bar[b]
  for (int it = 0; item < item_end; ++it, item += step) {
    const int bsel = it & 1;
    if (!mbar_wait(&bar[bsel], (phase >> bsel) & 1u, ctl->bar_cycles)) s_fail = 1u;
    phase ^= 1u << bsel;
    // this item's box has landed, and every thread is done with the previous
    // item (whose buffer and s_item entry are reused below); a copy that never
    // completed ends the CTA (no other copy is in flight) and the batch
    // reports ST_TIMEOUT
    __syncthreads();
    if (s_fail) {
      if (tid == 0) atomicOr(&ctl->status, ST_TIMEOUT);
      return;
    }
    const int4 inf = s_item[bsel];
    const int s = inf.x;
    if (s != cur) {
      if (cur >= 0 && !s_skip) publish<T, NT, STAGE>(sp, slots[cur].sc, s_lead != 0u, red, red.dt, acc, st);
      acc = Acc<T>();
      __syncthreads();
      if (tid == 0) {
        const BatchSlot<T> &sl = slots[s];
        sp = sl.p;
        s_io = io_of(sl.fd, st);
        const bool ld = (STRIDED ? sl.first_item % (int)gridDim.x : sl.first_item / W) == (int)blockIdx.x;
        stage_scalars<T, STAGE>(sp, sl.sc, ld, red, st);
        s_skip = red.skip;
        s_lead = ld ? 1u : 0u;
      }
      __syncthreads();
      cur = s;
    }
    T *box = bsel ? box1 : box0;
    if (tid == 0 && item + step < item_end) {
      fence_proxy_async();  // order the ghost patching's generic writes into that buffer before the copies
      issue(bsel ^ 1, &bar[bsel ^ 1]);
    }
    if (!s_skip) {
      const int i0 = inf.y, j0 = inf.z;
      if (i0 == 0 || j0 == 0 || i0 + TX + 3 > s_io.nx || j0 + TY + 3 > s_io.ny) {
        patch_box<T, TX, TY, NT>(s_io, sp, i0, j0, box, consts<T>(sp).zref, red_v<T>(red, SV_ETA),
                                 red_v<T>(red, SV_UIN));
        __syncthreads();
      }
      tile_compute<T, TX, TY, NT, S, STAGE, SHORE>(s_io, sp, i0, j0, box, sL, red_v<T>(red, SV_DT), red_v<T>(red, SV_RCAP),
                                            red_v<T>(red, SV_AX), red_v<T>(red, SV_AY), acc, st);
    }
  }
  if (cur >= 0 && !s_skip) publish<T, NT, STAGE>(sp, slots[cur].sc, s_lead != 0u, red, red.dt, acc, st);
}

}  // namespace swe
