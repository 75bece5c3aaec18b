// swe_fused.cu -- the fused-step variant: one persistent kernel per RK3 step
// (Eq. (8)) instead of one per stage.
//
// The paper takes the global Lax-Friedrichs speed alpha (Eq. (6)) of every
// stage's input ("TPU implementation"), a grid-wide reduction between the
// stages.  This variant splits all three stages of a step with one speed,
// alpha_margin x the alpha of U^n, so that a step depends on U^n and the bed
// alone: each CTA reads U^n on its output tile with a 9-cell halo (three
// stages x the three cells of a WENO5 stencil) and computes
//   stage 1 on the tile grown by 6 cells,
//   stage 2 on the tile grown by 3 cells,
//   stage 3 on the tile,
// keeping U1 and U2 in shared memory; only U^n is read from and U^{n+1}
// written to HBM (28 B per cell-update in FP32 instead of the 108 B of the
// stage kernels).  The cells of the grown regions are recomputed by every
// tile whose halo covers them, with the same inputs and the same arithmetic,
// so they agree bit for bit with their owner's.  U^{n+1} goes to a second set
// of planes (other CTAs still read U^n); steps alternate between the two.
//
// Each stage reuses the sweeps of the stage kernels (sweep_strip: split
// fluxes, WENO5 windows, the bed source weights); the cells' epilogue and the
// ghost values are this file's.  Ghost values follow the rules of the stage
// kernels for walls and the inflow edge (Carrier N-wave at the stage's input
// time); periodic sides and the strips of a row-partitioned domain are not
// supported here (their ghost cells belong to other tiles' stages).
#include <cstdio>

#include "swe_core.cuh"
#include "swe_launch.h"

namespace swe {

enum : unsigned {  // access sites of the checked build (beyond swe_core.cuh's)
  CK_F_LOAD = 32, CK_F_GHOST, CK_F_MIRROR, CK_F_XEPI, CK_F_YEPI, CK_F_OUT, CK_F_COPY
};

// Shared-memory frame of one output tile of TX x TY cells: the tile plus a
// 9-cell margin on every side, row pitch P, one plane per field:
//   U^n (ha, hu, hv), plane set A (ha, hu, hv), plane set B (ha, hu, hv), bed.
// Stage 1 reads U^n and writes U1 into A (its x pass parks L_x there first);
// stage 2 reads A and writes U2 into B (L_x parked in B); stage 3 reads B and
// writes HBM (L_x parked in A, dead by then).  Strips run over whole multiples
// of S cells; a strip's cells past its region's end are computed and thrown
// away, and its reads past the frame's last row land in the next plane or in
// the tail, never outside the allocation.
template <typename T, int TX, int TY>
struct FusedGeom {
  static constexpr int S = 8;    // strip length of the sweeps
  static constexpr int M = 9;    // margin of U^n: three stages of three cells
  static constexpr int FW = TX + 2 * M, FH = TY + 2 * M;
  static constexpr int P = FW | 1;  // odd pitch: x-pass lanes on consecutive rows hit distinct banks
  static constexpr int PLANE = FH * P;
  static constexpr int TAIL = (S + 1) * P;  // reads of the last plane's padded strips
  static constexpr int ELEMS = 10 * PLANE + TAIL;
  static constexpr size_t BYTES = sizeof(T) * (size_t)ELEMS;
  static constexpr int UN = 0, A = 3 * PLANE, B = 6 * PLANE, BED = 9 * PLANE;
};

// Compiled shapes of the fused kernel: (TX, TY, threads, CTAs per SM asked
// of the register allocator) per precision.
template <typename T> struct FusedShape;
template <> struct FusedShape<float> { static constexpr int TX = 64, TY = 32, NT = 384, MINB = 1; };
template <> struct FusedShape<double> { static constexpr int TX = 32, TY = 16, NT = 192, MINB = 1; };

template <typename T>
struct FusedIO {
  const T *b;
  const T *ha, *hu, *hv;  // U^n
  T *oha, *ohu, *ohv;     // U^{n+1}
  int nx, ny, pitch;
};

// Per-step values every CTA needs (computed from the device scalars that the
// step's preparation kernel wrote).
template <typename T>
struct FusedStep {
  double dt, t;
  T tdt, rcap, sx, sy;   // dt, 1/dt, splitting speeds
  T eta[3], uin[3];      // inflow ghosts at the stage input times t, t + dt, t + dt/2
  bool run;
};

// Ghost values of one plane set of the frame (cells outside the domain along
// exactly one axis, within three cells of its edge), from the frame's own
// cells: walls mirror (normal momentum odd), the inflow edge carries the
// N-wave.  Other cells outside the domain are never read by a cell of a
// stage's region and are left as they are.
template <typename T, int TX, int TY, int NT>
__device__ void fused_ghosts(const Phys &p, int nx, int ny, int i0, int j0, T *pl, const T *bb, T zref, T eta_in,
                             T u_in) {
  using G = FusedGeom<T, TX, TY>;
  T *ha = pl, *hu = pl + G::PLANE, *hv = pl + 2 * G::PLANE;
  for (int q = threadIdx.x; q < G::FH * G::FW; q += NT) {
    const int r = q / G::FW, c = q - r * G::FW;
    const int i = i0 - G::M + c, j = j0 - G::M + r;
    const bool in_i = i >= 0 && i < nx, in_j = j >= 0 && j < ny;
    const bool xg = !in_i && in_j && i >= -3 && i < nx + 3;
    const bool yg = in_i && !in_j && j >= -3 && j < ny + 3;
    if (!xg && !yg) continue;
    const int o = r * G::P + c;
    int mc = c, mr = r;
    if (xg) mc = (i < 0 ? -1 - i : 2 * nx - 1 - i) - (i0 - G::M);
    else mr = (j < 0 ? -1 - j : 2 * ny - 1 - j) - (j0 - G::M);
    const int m = mr * G::P + mc;
    if (!SWE_CHK(p, o, G::PLANE, CK_F_GHOST) || !SWE_CHK(p, m, G::PLANE, CK_F_MIRROR)) continue;
    const int side = xg ? (i < 0 ? 0 : 1) : (j < 0 ? 2 : 3);
    if (p.bc[side] == BC_INFLOW) {
      const T cb = bb[o];
      const T dg = still_depth(cb, zref);
      T a;
      if (cb < zref) { a = eta_in - zref; a = a > -dg ? a : -dg; }
      else { a = eta_in - cb; a = a > T(0) ? a : T(0); }
      ha[o] = a;
      hu[o] = (a + dg) * u_in;
      hv[o] = T(0);
    } else {
      ha[o] = ha[m];
      hu[o] = xg ? -hu[m] : hu[m];
      hv[o] = xg ? hv[m] : -hv[m];
    }
  }
}

// U^n and the bed of one tile's frame: interior cells by asynchronous 4- or
// 8-byte copies, then the bed's and U^n's ghost values.
template <typename T, int TX, int TY, int NT>
__device__ void fused_load(const FusedIO<T> &io, const Phys &p, int i0, int j0, T *sm, T zref, T eta_in, T u_in) {
  using G = FusedGeom<T, TX, TY>;
  const int nx = io.nx, ny = io.ny;
  const T *src[4] = {io.ha, io.hu, io.hv, io.b};
  const int dst[4] = {G::UN, G::UN + G::PLANE, G::UN + 2 * G::PLANE, G::BED};
  for (int q = threadIdx.x; q < G::FH * G::FW; q += NT) {
    const int r = q / G::FW, c = q - r * G::FW;
    const int i = i0 - G::M + c, j = j0 - G::M + r;
    if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
    const size_t go = (size_t)j * io.pitch + i;
    const int o = r * G::P + c;
    if (!SWE_CHK(p, go, (long long)ny * io.pitch, CK_F_LOAD) || !SWE_CHK(p, o, G::PLANE, CK_F_LOAD)) continue;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const unsigned d = smem_u32(sm + dst[f] + o);
      if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src[f] + go) : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src[f] + go) : "memory");
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // bed ghosts (walls and inflow both mirror the bed)
  T *bb = sm + G::BED;
  for (int q = threadIdx.x; q < G::FH * G::FW; q += NT) {
    const int r = q / G::FW, c = q - r * G::FW;
    const int i = i0 - G::M + c, j = j0 - G::M + r;
    const bool in_i = i >= 0 && i < nx, in_j = j >= 0 && j < ny;
    const bool xg = !in_i && in_j && i >= -3 && i < nx + 3;
    const bool yg = in_i && !in_j && j >= -3 && j < ny + 3;
    if (!xg && !yg) continue;
    int mc = c, mr = r;
    if (xg) mc = (i < 0 ? -1 - i : 2 * nx - 1 - i) - (i0 - G::M);
    else mr = (j < 0 ? -1 - j : 2 * ny - 1 - j) - (j0 - G::M);
    const int o = r * G::P + c, m = mr * G::P + mc;
    if (SWE_CHK(p, o, G::PLANE, CK_F_GHOST) && SWE_CHK(p, m, G::PLANE, CK_F_MIRROR)) bb[o] = bb[m];
  }
  __syncthreads();
  fused_ghosts<T, TX, TY, NT>(p, nx, ny, i0, j0, sm + G::UN, bb, zref, eta_in, u_in);
  __syncthreads();
}

// One RK stage of the fused step (STAGE 1, 2 or 3, a runtime value: one copy
// of the sweeps' code serves all three stages, which keeps the kernel in the
// instruction cache) on the tile (i0, j0) grown by MG cells and
// clipped to the domain: x pass (L_x parked in the output planes, or in A for
// stage 3), then y pass (sources, friction, the RK combination with U^n from
// the frame, the post-stage rule; stage 3 writes HBM).  Diagnostics count the
// cells (and edge faces) of the tile itself only, with the stage's RK weight:
// clamp 1/6, 2/3, 1; edge flux dt/6, dt/6, 2 dt/3 (dt applied at publication).
template <typename T, int TX, int TY, int NT>
__device__ __forceinline__ void fused_stage(const FusedIO<T> &io, const Phys &p, const FusedStep<T> &fs, int i0,
                                            int j0, T *sm, Acc<T> &acc, const int STAGE) {
  using G = FusedGeom<T, TX, TY>;
  constexpr int S = G::S;
  const int MG = (3 - STAGE) * 3;
  const int IN = STAGE == 1 ? G::UN : (STAGE == 2 ? G::A : G::B);
  const int OUT = STAGE == 1 ? G::A : (STAGE == 2 ? G::B : G::A);  // stage 3: L_x only
  constexpr int FIELD = G::PLANE + G::TAIL;
  const Consts<T> &K = consts<T>(p);
  const int nx = io.nx, ny = io.ny, tid = threadIdx.x;
  const int ri0 = max(i0 - MG, 0), ri1 = min(i0 + TX + MG, nx);
  const int rj0 = max(j0 - MG, 0), rj1 = min(j0 + TY + MG, ny);
  const int RW = ri1 - ri0, RH = rj1 - rj0;
  const int fc0 = ri0 - (i0 - G::M), fr0 = rj0 - (j0 - G::M);
  const T *iha = sm + IN, *ihu = sm + IN + G::PLANE, *ihv = sm + IN + 2 * G::PLANE, *bb = sm + G::BED;
  T *lha = sm + OUT, *lhu = sm + OUT + G::PLANE, *lhv = sm + OUT + 2 * G::PLANE;
  const T wc = STAGE == 1 ? T(1.0 / 6.0) : (STAGE == 2 ? T(2.0 / 3.0) : T(1));   // clamp weight
  const T wf = STAGE == 3 ? T(2.0 / 3.0) : T(1.0 / 6.0);                          // edge-flux weight
  const T ewx = K.ewx * wf, ewy = K.ewy * wf;
  // Edge faces count once, in the tile that owns the cell beside them: a tile
  // that does not own the last column (row) passes an edge index no face can
  // reach, since a padded strip may run past the domain's edge with cells the
  // region does not hold.
  const int ex = i0 + TX >= nx ? nx : 1 << 30, ey = j0 + TY >= ny ? ny : 1 << 30;
  const bool own_ex = i0 == 0 || i0 + TX >= nx, own_ey = j0 == 0 || j0 + TY >= ny;

  // x pass: lane -> row (consecutive rows: distinct banks), strips across
  const int nsx = (RW + S - 1) / S;
  for (int q = tid; q < RH * nsx; q += NT) {
    const int r = q % RH, c0 = (q / RH) * S;
    const int j = rj0 + r;
    const int row = (fr0 + r) * G::P + fc0;
    auto emit = [&](int k, T dF0, T dF1, T dF2, T dbk) {
      const int c = c0 + k;
      if (c >= RW) return;
      const int o = row + c;
      if (!SWE_CHK(p, o, G::PLANE, CK_F_XEPI)) return;
      const T ha = iha[o];
      lha[o] = -dF0 * K.rfx;
      lhu[o] = -dF1 * K.rfx - K.g12dx * ha * dbk;
      lhv[o] = -dF2 * K.rfx;
    };
    sweep_strip<T, S, false, FIELD>(iha, ihu, ihv, bb, row + c0 - 3, 1, fs.sx, K, p, ri0 + c0, ex,
                                    own_ex && j >= j0 && j < j0 + TY, ewx, emit, acc.edge);
  }
  __syncthreads();

  // y pass: lane -> column, strips down
  const int nsy = (RH + S - 1) / S;
  const T wrk = STAGE == 2 ? T(0.25) : T(2.0 / 3.0);
  const bool friction = K.gn2 > T(0);
  const T *uha = sm + G::UN, *uhu = sm + G::UN + G::PLANE, *uhv = sm + G::UN + 2 * G::PLANE;
  for (int q = tid; q < RW * nsy; q += NT) {
    const int c = q % RW, r0 = (q / RW) * S;
    const int i = ri0 + c;
    const bool own_col = i >= i0 && i < i0 + TX;
    auto emit = [&](int k, T dF0, T dF1, T dF2, T dbk) {
      const int r = r0 + k;
      if (r >= RH) return;
      const int j = rj0 + r;
      const int o = (fr0 + r) * G::P + fc0 + c;
      if (!SWE_CHK(p, o, G::PLANE, CK_F_YEPI)) return;
      const bool own = own_col && j >= j0 && j < j0 + TY;
      const T ha = iha[o], hu = ihu[o], hv = ihv[o], bc = bb[o];
      const T d = still_depth(bc, K.zref);
      const T h = ha + d;
      T Lh = lha[o] - dF0 * K.rfy;
      T Lhu = lhu[o] - dF2 * K.rfy;
      T Lhv = lhv[o] - dF1 * K.rfy - K.g12dy * ha * dbk;
      if (friction && !Num<T>::below(h, p.h_dry32, p.h_dry)) {
        T kap = K.gn2 * Num<T>::fric(hu * hu + hv * hv, h);
        kap = kap > fs.rcap ? fs.rcap : kap;
        Lhu -= kap * hu;
        Lhv -= kap * hv;
      }
      T nha = ha + fs.tdt * Lh, nhu = hu + fs.tdt * Lhu, nhv = hv + fs.tdt * Lhv;
      if (STAGE != 1) {
        const T a0 = uha[o], u0 = uhu[o], v0 = uhv[o];
        nha = a0 + wrk * (nha - a0);
        nhu = u0 + wrk * (nhu - u0);
        nhv = v0 + wrk * (nhv - v0);
      }
      if (nha < -d) {
        if (own) acc.deficit += wc * (-(nha + d));
        nha = -d;
      }
      const T nh = nha + d;
      T u = T(0), v = T(0), rr, cel;
      Num<T>::speed(nh, K.g, K.sqg, rr, cel);
      if (Num<T>::below(nh, p.h_dry32, p.h_dry)) { nhu = T(0); nhv = T(0); }
      else {
        if (Num<T>::below(nh, p.h_film32, p.h_film)) {  // film: bounded velocity
          const T h2 = nh * nh;
          const T f = T(1.4142135623730951) * h2 * Num<T>::rsqrt_(h2 * h2 + K.hf4);
          nhu *= f;
          nhv *= f;
        }
        u = nhu * rr;
        v = nhv * rr;
      }
      if (STAGE == 3) {
        const size_t go = (size_t)j * io.pitch + i;
        if (own && SWE_CHK(p, go, (long long)ny * io.pitch, CK_F_OUT)) {
          io.oha[go] = nha;
          io.ohu[go] = nhu;
          io.ohv[go] = nhv;
        }
      } else {
        lha[o] = nha;
        lhu[o] = nhu;
        lhv[o] = nhv;
      }
      if (own) {
        const T sx = fabs(u) + cel, sy = fabs(v) + cel;
        acc.chk += sx + sy;  // non-finite values propagate to the per-CTA check
        if (STAGE == 3) {
          acc.ax = sx > acc.ax ? sx : acc.ax;
          acc.ay = sy > acc.ay ? sy : acc.ay;
          if (!Num<T>::below(nh, p.h_wet32, p.h_wet) && bc > T(0)) {
            const T e = nh + bc;
            acc.ru = e > acc.ru ? e : acc.ru;
          }
        }
      }
    };
    sweep_strip<T, S, false, FIELD>(iha, ihv, ihu, bb, (fr0 + r0 - 3) * G::P + fc0 + c, G::P, fs.sy, K, p,
                                    rj0 + r0, ey, own_ey && own_col, ewy, emit, acc.edge);
  }
  __syncthreads();
}

// Block reduction of the per-thread accumulators; the speeds of U^{n+1} go
// to alpha slot 1 (the step's finishing kernel moves them to slot 0).
template <typename T, int NT>
__device__ __noinline__ void fused_publish(const Phys &p, DevScalars *sc, RedSmem &red, double dt, const Acc<T> &acc) {
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const T ax = warp_max(acc.ax), ay = warp_max(acc.ay), ru = warp_max(acc.ru);
  const T de = warp_sum(acc.deficit), ef = warp_sum(acc.edge);
  const bool bad = !(acc.chk <= T(3.0e38));
  const unsigned anybad = __any_sync(0xffffffffu, bad);
  T *wv = red_w<T>(red);
  if (l == 0) {
    wv[5 * w + 0] = ax;
    wv[5 * w + 1] = ay;
    wv[5 * w + 2] = de;
    wv[5 * w + 3] = ef;
    wv[5 * w + 4] = ru;
    if (anybad) red.bad = 1u;
  }
  __syncthreads();
  if (tid == 0) {
    T mx = T(0), my = T(0), dsum = T(0), fsum = T(0), rmax = T(0);
    for (int q = 0; q < NT / 32; ++q) {
      mx = fmax(mx, wv[5 * q + 0]);
      my = fmax(my, wv[5 * q + 1]);
      dsum += wv[5 * q + 2];
      fsum += wv[5 * q + 3];
      rmax = fmax(rmax, wv[5 * q + 4]);
    }
    atomicMax(&sc->alpha[1][0], dbits((double)mx));
    atomicMax(&sc->alpha[1][1], dbits((double)my));
    if (dsum != T(0)) sc->part->clamp[blockIdx.x] += p.area * (double)dsum;
    if (fsum != T(0)) sc->part->edge[blockIdx.x] += dt * (double)fsum;
    if (rmax > T(0)) {
      const unsigned long long rb = dbits((double)rmax);
      atomicMax(&sc->runup_now[__ldcg(&sc->parity)], rb);
      atomicMax(&sc->runup_max, rb);
    }
    if (red.bad) atomicOr(&sc->status, ST_NONFINITE);
  }
}

template <typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, FusedShape<T>::MINB)
    fused_step_kernel(FusedIO<T> io, Phys p, DevScalars *sc, double margin) {
  using G = FusedGeom<T, TX, TY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ RedSmem red;
  __shared__ FusedStep<T> fs;
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    // written by the preparation kernel before this launch; stable during it
    const bool run = __ldcg(&sc->running) != 0u;
    const double dt = run ? __ldcg(&sc->dt) : 0.0, t = __ldcg(&sc->t_step);
    fs.run = run;
    fs.dt = dt;
    fs.t = t;
    fs.tdt = T(dt);
    fs.rcap = dt > 0.0 ? T(1) / T(dt) : T(0);
    fs.sx = T(margin * bitsd(__ldcg(&sc->alpha[0][0])));
    fs.sy = T(margin * bitsd(__ldcg(&sc->alpha[0][1])));
    const bool inflow = p.bc[0] == BC_INFLOW;
    const double ts[3] = {t, t + dt, t + 0.5 * dt};
    for (int s = 0; s < 3; ++s) {
      fs.eta[s] = inflow ? inflow_eta<T>(p, ts[s]) : T(0);
      fs.uin[s] = inflow ? fs.eta[s] * T(p.in_uf) : T(0);
    }
    red.bad = 0u;
  }
  __syncthreads();
  const int tiles_x = (io.nx + TX - 1) / TX, tiles_y = (io.ny + TY - 1) / TY;
  const int ntiles = tiles_x * tiles_y;
  if (!fs.run) {
    // skipped step (horizon reached or an earlier error): U^{n+1} = U^n, so
    // that the alternating planes stay consistent
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int i0 = (t % tiles_x) * TX, j0 = (t / tiles_x) * TY;
      for (int q = tid; q < TX * TY; q += NT) {
        const int i = i0 + q % TX, j = j0 + q / TX;
        if (i >= io.nx || j >= io.ny) continue;
        const size_t go = (size_t)j * io.pitch + i;
        if (!SWE_CHK(p, go, (long long)io.ny * io.pitch, CK_F_COPY)) continue;
        io.oha[go] = io.ha[go];
        io.ohu[go] = io.hu[go];
        io.ohv[go] = io.hv[go];
      }
    }
    return;
  }
  const T zref = consts<T>(p).zref;
  Acc<T> acc;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (t % tiles_x) * TX, j0 = (t / tiles_x) * TY;
    __syncthreads();  // every thread is done with the previous tile's frame
    fused_load<T, TX, TY, NT>(io, p, i0, j0, sm, zref, fs.eta[0], fs.uin[0]);
#pragma unroll 1
    for (int st = 1; st <= 3; ++st) {
      fused_stage<T, TX, TY, NT>(io, p, fs, i0, j0, sm, acc, st);
      if (st < 3) {
        fused_ghosts<T, TX, TY, NT>(p, io.nx, io.ny, i0, j0, sm + (st == 1 ? G::A : G::B), sm + G::BED, zref,
                                    fs.eta[st], fs.uin[st]);
        __syncthreads();
      }
    }
  }
  fused_publish<T, NT>(p, sc, red, fs.dt, acc);
}

// Before each fused step (one thread): the step's dt from the CFL condition on
// U^n's speeds (alpha slot 0) or the fixed dt, truncated at t_end, the skip
// decision, and the clearing of what the step accumulates into.
__global__ void fused_prep_kernel(Phys p, DevScalars *sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double ax = bitsd(sc->alpha[0][0]), ay = bitsd(sc->alpha[0][1]);
  const double t = sc->t, t_end = sc->t_end;
  unsigned skip = sc->status != 0u;
  if (t_end > 0.0 && t >= t_end) skip = 1u;
  double dt = 0.0;
  if (p.fixed_dt > 0.0) dt = p.fixed_dt;
  else {
    const double den = ax * p.rdx + ay * p.rdy;
    if (den > 0.0) dt = sc->cfl / den;
    else if (!skip) {
      skip = 1u;
      sc->status |= ST_DRY;
    }
  }
  if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
  sc->running = skip ? 0u : 1u;
  if (!skip) {
    sc->dt = dt;
    sc->t_step = t;
    sc->parity = (unsigned)(sc->steps & 1);
    sc->runup_now[sc->steps & 1] = 0ull;
    sc->alpha[1][0] = 0ull;
    sc->alpha[1][1] = 0ull;
  }
}

// After each fused step (one thread): U^{n+1}'s speeds to slot 0, time and
// step count.
__global__ void fused_finish_kernel(DevScalars *sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!sc->running) return;
  sc->alpha[0][0] = sc->alpha[1][0];
  sc->alpha[0][1] = sc->alpha[1][1];
  const double tn = sc->t_step + sc->dt, te = sc->t_end;
  sc->t = (te > 0.0 && tn >= te) ? te : tn;
  sc->steps = sc->steps + 1;
  sc->running = 0u;
}

namespace {
template <typename T>
struct FusedLaunch {
  using Sh = FusedShape<T>;
  using G = FusedGeom<T, Sh::TX, Sh::TY>;
};
int g_resident[2] = {0, 0}, g_sms[2] = {0, 0};  // per precision: [0] FP32, [1] FP64
template <typename T> constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }
}  // namespace

template <typename T>
cudaError_t prepare_fused() {
  using L = FusedLaunch<T>;
  using Sh = FusedShape<T>;
  auto *k = fused_step_kernel<T, Sh::TX, Sh::TY, Sh::NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::G::BYTES);
  int dev = 0, nb = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, Sh::NT, L::G::BYTES);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  g_resident[prec_index<T>()] = nb;
  g_sms[prec_index<T>()] = sms;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_fused(const Field<T> &fd, int from, const Phys &p, DevScalars *sc, double margin,
                         cudaStream_t st, cudaEvent_t *ev) {
  using L = FusedLaunch<T>;
  using Sh = FusedShape<T>;
  const int resident = g_resident[prec_index<T>()];
  if (resident < 1 || (from != 0 && from != 1)) return cudaErrorInvalidConfiguration;
  const int ntiles = ((fd.nx + Sh::TX - 1) / Sh::TX) * ((fd.ny + Sh::TY - 1) / Sh::TY);
  int grid = resident * g_sms[prec_index<T>()];
  if (grid > ntiles) grid = ntiles;
  if (grid > kPartSlots) return cudaErrorInvalidConfiguration;  // one partial slot per CTA
  FusedIO<T> io;
  io.b = fd.b;
  io.ha = fd.h[from];
  io.hu = fd.hu[from];
  io.hv = fd.hv[from];
  io.oha = fd.h[1 - from];
  io.ohu = fd.hu[1 - from];
  io.ohv = fd.hv[1 - from];
  io.nx = fd.nx;
  io.ny = fd.ny;
  io.pitch = fd.pitch;
  cudaError_t e = ev ? cudaEventRecord(ev[0], st) : cudaSuccess;
  if (e != cudaSuccess) return e;
  fused_prep_kernel<<<1, 32, 0, st>>>(p, sc);
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  fused_step_kernel<T, Sh::TX, Sh::TY, Sh::NT><<<grid, Sh::NT, L::G::BYTES, st>>>(io, p, sc, margin);
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  fused_finish_kernel<<<1, 32, 0, st>>>(sc);
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t fused_smem(int elem_bytes) {
  return elem_bytes == 8 ? FusedLaunch<double>::G::BYTES : FusedLaunch<float>::G::BYTES;
}

template cudaError_t prepare_fused<float>();
template cudaError_t prepare_fused<double>();
template cudaError_t launch_fused<float>(const Field<float> &, int, const Phys &, DevScalars *, double, cudaStream_t,
                                         cudaEvent_t *);
template cudaError_t launch_fused<double>(const Field<double> &, int, const Phys &, DevScalars *, double,
                                          cudaStream_t, cudaEvent_t *);

}  // namespace swe
