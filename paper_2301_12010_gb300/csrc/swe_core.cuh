// swe_core.cuh -- device code of one SSP-RK3 stage over one tile of cells.
//
// Method (Madden, Marras & Suckale, arXiv:2301.12010, "Numerical
// approximation"): the 2-D SWE of Eqs. (1)-(3) in the vector form Eq. (4),
// fifth-order WENO face values (Eq. (5)) combined by global Lax-Friedrichs
// flux splitting (Eq. (6)), the explicit update Eq. (7) with the source
// evaluated at the cell centre, advanced by the RK3 stages of Eq. (8).  The
// global maximum wave speed is reduced across the whole domain as in "TPU
// implementation"; here it is a warp-shuffle / block reduction followed by a
// device-scope atomic max on the order-preserving bits of a double.
//
// One stage kernel fuses, per tile of TX x TY cells:
//   ghost values (walls / inflow / periodic) computed while loading the halo,
//   the dry rule, split fluxes f+- = (F +- alpha Q)/2, six WENO5
//   reconstructions per face and direction, the bed source with the
//   normal-momentum weights, explicit Manning friction, the RK combination,
//   the post-stage positivity rule and the reductions for the next stage
//   (alpha_x, alpha_y), the clamp mass, the edge mass flux and (stage 3) the
//   runup.  Bed terms use the splitting of Eqs. (2)-(3) relative to the
//   still-water depth d = max(z_ref - b, 0): pressure g (h^2 - d^2)/2, source
//   -g (h - d) db/dx, mass viscosity on h - d.
//
// Storage: the depth is held as the still-water anomaly ha = h - d (= h + b -
// z_ref at sea, = h on land), a change of variables that is exact in real
// arithmetic and keeps full FP32 precision both for small waves over deep
// water and for thin films on land; d is recomputed from b.  The RK
// combinations are written in increment form U0 + w (U' - U0), whose weights
// sum to one exactly in any precision.
//
// Shared-memory plan (per CTA): the bed over the halo box, one split-flux
// buffer reused by the x pass and then the y pass, the x-pass result L_x, and
// the anomaly ha of the tile's own cells.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swe {

enum : int { BC_WALL = 0, BC_INFLOW = 1, BC_PERIODIC = 2 };
enum : unsigned { ST_NONFINITE = 1u, ST_DRY = 2u, ST_TIMEOUT = 4u };

// Per-scenario device scalars (one struct per handle or batch slot).
struct DevScalars {
  unsigned long long alpha[3][2];   // wave speeds (x, y) per stage slot, bits of a double
  double dt;                        // time step of the running step
  double t;                         // time of U^n
  double t_step;                    // time at the start of the running step
  long long steps;                  // steps taken
  unsigned long long runup_now[2];  // bits of a double, per step parity; 0 = no wet land cell
  unsigned long long runup_max;     // bits of a double; 0 = none
  double clamp_mass;                // RK-weighted clamp additions, m^3
  double boundary_mass;             // RK-weighted edge inflow, m^3
  double t_end;                     // > 0: last step truncated at t_end; no step once t >= t_end
  double cfl;                       // CFL number when fixed_dt <= 0
  unsigned status;                  // ST_* flags
  unsigned running;                 // 1 while the current step runs (set by stage 1)
  unsigned parity;                  // steps & 1 of the running step
  unsigned active;                  // batch: slot is live
};

// Physical and numerical parameters, constant over a run.
struct Phys {
  double g, n2, h_dry, h_wet, weno_eps, fixed_dt, z_ref;
  double b_jump_x, b_jump_y;
  double inflow_amp, inflow_period, inflow_depth;
  double dx, dy;
  float h_dry32, h_wet32;  // smallest floats whose double value is >= h_dry / h_wet
  int bc[4];
};

template <typename T>
struct Field {
  const T *b;
  T *h[3], *hu[3], *hv[3];  // planes of U^n, U1, U2; h[] holds ha = h - d
  int nx, ny, pitch;
};

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long u) { return __longlong_as_double((long long)u); }

template <typename T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  // h^(7/3) for h > 0 through exp2/log2 hardware approximations
  static __device__ __forceinline__ float pow73(float h) { return exp2f(2.33333333f * __log2f(h)); }
  static __device__ __forceinline__ bool below(float h, float thr32, double) { return h < thr32; }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double pow73(double h) { return h * h * cbrt(h); }
  static __device__ __forceinline__ bool below(double h, float, double thr) { return h < thr; }
};

// WENO5-JS value at the right face of v2 (Jiang & Shu 1996), scaled by 6:
// returns 6*W and the unnormalised weights a_k and 1/sum(d_k a_k') needed to
// apply the same weights to the bed.  t_k = 12 eps + 12 beta_k, so that
// a_k = d_k / t_k^2 has the ratios of d_k / (eps + beta_k)^2.
template <typename T>
__device__ __forceinline__ T weno5x6(T v0, T v1, T v2, T v3, T v4, T eps12, T &a0, T &a1, T &a2, T &rdn) {
  const T d20 = v0 - T(2) * v1 + v2;
  const T d21 = v1 - T(2) * v2 + v3;
  const T d22 = v2 - T(2) * v3 + v4;
  const T e0 = v0 - T(4) * v1 + T(3) * v2;
  const T e1 = v1 - v3;
  const T e2 = T(3) * v2 - T(4) * v3 + v4;
  const T t0 = T(13) * d20 * d20 + T(3) * e0 * e0 + eps12;
  const T t1 = T(13) * d21 * d21 + T(3) * e1 * e1 + eps12;
  const T t2 = T(13) * d22 * d22 + T(3) * e2 * e2 + eps12;
  const T r0 = Num<T>::rcp(t0), r1 = Num<T>::rcp(t1), r2 = Num<T>::rcp(t2);
  a0 = T(0.1) * r0 * r0;
  a1 = T(0.6) * r1 * r1;
  a2 = T(0.3) * r2 * r2;
  const T p0 = T(2) * v0 - T(7) * v1 + T(11) * v2;
  const T p1 = -v1 + T(5) * v2 + T(2) * v3;
  const T p2 = T(2) * v2 + T(5) * v3 - v4;
  rdn = Num<T>::rcp(a0 + a1 + a2);
  return (a0 * p0 + a1 * p1 + a2 * p2) * rdn;
}

// 6 * (weighted candidate values) of a stencil with given weights.
template <typename T>
__device__ __forceinline__ T weighted6(T v0, T v1, T v2, T v3, T v4, T a0, T a1, T a2, T rdn) {
  const T p0 = T(2) * v0 - T(7) * v1 + T(11) * v2;
  const T p1 = -v1 + T(5) * v2 + T(2) * v3;
  const T p2 = T(2) * v2 + T(5) * v3 - v4;
  return (a0 * p0 + a1 * p1 + a2 * p2) * rdn;
}

// Carrier N-wave of Eq. (20) entering through the x- edge (peak elevation
// amp, a1 = amp/2, a2 = a1/3, lambda = T sqrt(g d0)), read at
// s = 1.3 lambda - c0 t.
__device__ __forceinline__ double inflow_eta(const Phys &p, double t) {
  const double c0 = sqrt(p.g * p.inflow_depth);
  const double lam = p.inflow_period * c0;
  const double a1 = 0.5 * p.inflow_amp, a2 = a1 / 3.0;
  const double k1 = 28.416 / (lam * lam), k2 = 256.0 / (lam * lam);
  const double s = 1.3 * lam - c0 * t;
  const double q1 = s - 0.5151125 * lam, q2 = s - 0.2048 * lam;
  return 2.0 * (a1 * exp(-k1 * q1 * q1) - a2 * exp(-k2 * q2 * q2));
}

template <typename T>
__device__ __forceinline__ T still_depth(T b, T zref) {
  T d = zref - b;
  return d > T(0) ? d : T(0);
}

// State (ha, hu, hv) and bed of cell (i, j), where (i, j) may lie up to 3
// cells outside the interior in at most one direction (ghosts per boundary
// type: mirrored walls, the inflow wave, or periodic wrap with bed offset).
template <typename T>
__device__ __forceinline__ void load_cell(const T *__restrict__ b, const T *__restrict__ ha,
                                          const T *__restrict__ hu, const T *__restrict__ hv, int nx, int ny,
                                          int pitch, const Phys &p, T zref, T eta_in, T u_in, int i, int j, T &ch,
                                          T &chu, T &chv, T &cb) {
  int si = i, sj = j;
  bool fu = false, fv = false, inflow = false, seam = false;
  T bshift = T(0);
  if (i < 0) {
    if (p.bc[0] == BC_PERIODIC) { si = i + nx; bshift = T(-p.b_jump_x); seam = true; }
    else { si = -1 - i; fu = true; inflow = (p.bc[0] == BC_INFLOW); }
  } else if (i >= nx) {
    if (p.bc[1] == BC_PERIODIC) { si = i - nx; bshift = T(p.b_jump_x); seam = true; }
    else { si = 2 * nx - 1 - i; fu = true; }
  }
  if (j < 0) {
    if (p.bc[2] == BC_PERIODIC) { sj = j + ny; bshift = T(-p.b_jump_y); seam = true; }
    else { sj = -1 - j; fv = true; }
  } else if (j >= ny) {
    if (p.bc[3] == BC_PERIODIC) { sj = j - ny; bshift = T(p.b_jump_y); seam = true; }
    else { sj = 2 * ny - 1 - j; fv = true; }
  }
  const size_t o = (size_t)sj * pitch + si;
  const T bs = b[o];
  cb = bs + bshift;
  if (inflow) {
    // h = max(eta_in - b, 0), u = eta_in sqrt(g/d0), v = 0; in anomaly form
    const T dg = still_depth(cb, zref);
    if (cb < zref) {
      const T a = eta_in - zref;
      ch = a > -dg ? a : -dg;
    } else {
      const T hg = eta_in - cb;
      ch = hg > T(0) ? hg : T(0);
    }
    chu = (ch + dg) * u_in;
    chv = T(0);
  } else {
    ch = ha[o];
    chu = hu[o];
    chv = hv[o];
    if (seam) ch = (ch + still_depth(bs, zref)) - still_depth(cb, zref);  // same h, new d
    if (fu) chu = -chu;
    if (fv) chv = -chv;
  }
}

// Split fluxes of one cell along direction DIR (0: x with F, 1: y with G)
// from the anomaly form: h = ha + d, pressure g ha (h + d)/2 = g (h^2-d^2)/2,
// Q = (ha, hu, hv).
template <typename T, int DIR>
__device__ __forceinline__ void split_cell(T ha, T hu, T hv, T b, T alpha, T g, T zref, const Phys &p, T fp[3],
                                           T fm[3]) {
  const T d = still_depth(b, zref);
  const T h = ha + d;
  T u = T(0), v = T(0);
  if (!Num<T>::below(h, p.h_dry32, p.h_dry)) {
    const T r = Num<T>::rcp(h);
    u = hu * r;
    v = hv * r;
  }
  const T pres = T(0.5) * g * ha * (h + d);
  T F0, F1, F2;
  if (DIR == 0) { F0 = hu; F1 = hu * u + pres; F2 = hv * u; }
  else { F0 = hv; F1 = hu * v; F2 = hv * v + pres; }
  const T q0 = alpha * ha, q1 = alpha * hu, q2 = alpha * hv;
  fp[0] = T(0.5) * (F0 + q0); fm[0] = T(0.5) * (F0 - q0);
  fp[1] = T(0.5) * (F1 + q1); fm[1] = T(0.5) * (F1 - q1);
  fp[2] = T(0.5) * (F2 + q2); fm[2] = T(0.5) * (F2 - q2);
}

// Strip of S cells along a line: faces k = 0..S lie at the left of cell
// c0+k (face c0+k-1/2).  sp points at the f+ value of component 0 for the
// cell c0-3; cells along the line are `st` apart, components `cs` apart and
// f- sits `pm` after f+.  bl points at b of cell c0-3 (stride bst).
// For each cell k of the strip: dF[m][k] = 6*(Fhat_{k+1/2} - Fhat_{k-1/2}),
// db[k] = 6*(bhat_{k+1/2} - bhat_{k-1/2}) * 2 (bhat of b/2, scaled), and the
// first/last face values of component 0 (edge mass flux).
template <typename T, int S, int MOM>
__device__ __forceinline__ void sweep_strip(const T *__restrict__ sp, int st, int cs, int pm,
                                            const T *__restrict__ bl, int bst, T eps12, T dF[3][S], T db[S],
                                            T Fface0[S + 1]) {
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const T *fpp = sp + m * cs;
    const T *fmm = fpp + pm;
    T wp[6], wm[6], wb[6];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      wp[q] = fpp[q * st];
      wm[q] = fmm[q * st];
      if (m == MOM) wb[q] = bl[q * bst];
    }
    T prevF = T(0), prevB = T(0);
#pragma unroll
    for (int k = 0; k <= S; ++k) {
      // window: cells c0-3+k .. c0+2+k at wp[0..5]
      wp[5] = fpp[(k + 5) * st];
      wm[5] = fmm[(k + 5) * st];
      if (m == MOM) wb[5] = bl[(k + 5) * bst];
      T a0, a1, a2, rp, c0, c1, c2, rm;
      const T Fp = weno5x6<T>(wp[0], wp[1], wp[2], wp[3], wp[4], eps12, a0, a1, a2, rp);
      const T Fm = weno5x6<T>(wm[5], wm[4], wm[3], wm[2], wm[1], eps12, c0, c1, c2, rm);
      const T F = Fp + Fm;
      T B = T(0);
      if (m == MOM)
        B = weighted6<T>(wb[0], wb[1], wb[2], wb[3], wb[4], a0, a1, a2, rp) +
            weighted6<T>(wb[5], wb[4], wb[3], wb[2], wb[1], c0, c1, c2, rm);
      if (m == 0) Fface0[k] = F;
      if (k > 0) {
        dF[m][k - 1] = F - prevF;
        if (m == MOM) db[k - 1] = B - prevB;
      }
      prevF = F;
      prevB = B;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        wp[q] = wp[q + 1];
        wm[q] = wm[q + 1];
        if (m == MOM) wb[q] = wb[q + 1];
      }
    }
  }
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory footprint of one tile (elements of T).
template <int TX, int TY>
struct TileGeom {
  static constexpr int BW = TX + 6;                    // halo box width
  static constexpr int BH = TY + 6;                    // halo box height
  static constexpr int XP = ((TX + 6 + 7) / 8) * 8 + 1;  // x-pass row pitch: = 1 mod 8 (bank spread)
  static constexpr int XS = TY * XP;                   // one x-split component
  static constexpr int YS = BH * TX;                   // one y-split component
  static constexpr int SPL = (XS > YS ? XS : YS);      // split buffer per component
  static constexpr int NB = BH * BW;                   // bed box
  static constexpr int NC = TX * TY;                   // own cells
  static constexpr int ELEMS = NB + 6 * SPL + NC + 3 * NC;
};

// Reduction scratch in shared memory (per CTA).
struct RedSmem {
  double a[32][2];
  double s[32][2];
  double r[32];
  double dt;
  double eta_in;
  unsigned bad;
  unsigned skip;
};

// One RK3 stage (Eq. (8), Shu-Osher form) over the tile whose first cell is
// (i0, j0):
//   stage 1: U1 = U^n + dt L(U^n)
//   stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
//   stage 3: U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2))   (written over U^n)
// followed by the post-stage rule, with L of Eq. (7).  NT threads; strips of
// S cells.  `lead` marks the one tile per scenario that does the per-step
// bookkeeping (dt, time, step count, slot resets).
//
// Stage s reads the wave speeds of its input from slot s-1, publishes those
// of its output to slot s mod 3 and clears slot (s+1) mod 3, which nothing
// reads or writes during stage s.
template <typename T, int TX, int TY, int NT, int S, int STAGE>
__device__ void stage_tile(const Field<T> &fd, const Phys &p, DevScalars *sc, int i0, int j0, T *smem,
                           RedSmem &red, bool lead) {
  using G = TileGeom<TX, TY>;
  static_assert(TX % S == 0 && TY % S == 0, "strip length must divide the tile");
  static_assert((TX / S) * TY == NT && (TY / S) * TX == NT, "one strip per thread in both passes");
  static_assert(TY % 8 == 0 && (TX / S) % 4 == 0, "x-pass warp covers 8 rows x 4 strips");
  const int tid = threadIdx.x;
  const int nx = fd.nx, ny = fd.ny, pitch = fd.pitch;
  constexpr int IN = STAGE - 1;         // U^n, U1, U2 as stage input
  constexpr int OUTB = STAGE % 3;       // U1, U2, U^n as stage output
  const T *__restrict__ bb = fd.b;
  const T *__restrict__ hin = fd.h[IN];
  const T *__restrict__ huin = fd.hu[IN];
  const T *__restrict__ hvin = fd.hv[IN];

  T *sb = smem;               // bed over the halo box
  T *spl = sb + G::NB;        // 6 split components
  T *sha = spl + 6 * G::SPL;  // ha of own cells
  T *sL = sha + G::NC;        // L_x, 3 components

  // ---- stage scalars and the skip decision (uniform over the CTA)
  const double ax = bitsd(sc->alpha[STAGE - 1][0]);
  const double ay = bitsd(sc->alpha[STAGE - 1][1]);
  if (tid == 0) {
    double dt = 0.0;
    unsigned skip = sc->status != 0u;
    if (STAGE == 1) {
      const double t = sc->t;
      if (sc->t_end > 0.0 && t >= sc->t_end) skip = 1;
      if (p.fixed_dt > 0.0) dt = p.fixed_dt;
      else {
        const double den = ax / p.dx + ay / p.dy;
        if (den > 0.0) dt = sc->cfl / den;
        else if (!skip) { skip = 1; atomicOr(&sc->status, ST_DRY); }
      }
      if (sc->t_end > 0.0 && t + dt > sc->t_end) dt = sc->t_end - t;
      if (lead) {
        sc->running = skip ? 0u : 1u;
        if (!skip) {
          sc->dt = dt;
          sc->t_step = t;
          sc->parity = (unsigned)(sc->steps & 1);
          sc->runup_now[sc->steps & 1] = 0ull;
          sc->alpha[2][0] = 0ull;
          sc->alpha[2][1] = 0ull;
        }
      }
    } else {
      if (!sc->running) skip = 1;
      dt = sc->dt;
      if (lead && !skip) {
        sc->alpha[STAGE == 2 ? 0 : 1][0] = 0ull;
        sc->alpha[STAGE == 2 ? 0 : 1][1] = 0ull;
      }
    }
    red.skip = skip;
    red.bad = 0u;
    red.dt = dt;
    const double tst = (STAGE == 1) ? sc->t : sc->t_step;
    const double ts = (STAGE == 1) ? tst : (STAGE == 2 ? tst + dt : tst + 0.5 * dt);
    red.eta_in = (p.bc[0] == BC_INFLOW && i0 == 0) ? inflow_eta(p, ts) : 0.0;
  }
  __syncthreads();
  if (red.skip) return;
  const double dt = red.dt;
  const T eta_in = T(red.eta_in);
  const T u_in = (p.bc[0] == BC_INFLOW) ? T(red.eta_in * sqrt(p.g / p.inflow_depth)) : T(0);
  const T g = T(p.g), zref = T(p.z_ref), eps12 = T(12.0 * p.weno_eps);
  const T alx = T(ax), aly = T(ay);

  // ---- phase A: bed box, x-split fluxes (own rows, halo columns), ha of own cells
  for (int idx = tid; idx < G::NB; idx += NT) {
    const int r = idx / G::BW, c = idx - r * G::BW;
    const int i = i0 - 3 + c, j = j0 - 3 + r;
    const bool xin = (i >= -3 && i < nx + 3), yin = (j >= -3 && j < ny + 3);
    const bool ix = (i >= 0 && i < nx), jy = (j >= 0 && j < ny);
    const bool own_row = (r >= 3 && r < TY + 3);
    T cb = T(0);
    if ((ix && yin) || (jy && xin)) {
      T ch, chu, chv;
      load_cell<T>(bb, hin, huin, hvin, nx, ny, pitch, p, zref, eta_in, u_in, i, j, ch, chu, chv, cb);
      if (own_row) {
        T fp[3], fm[3];
        if (jy) split_cell<T, 0>(ch, chu, chv, cb, alx, g, zref, p, fp, fm);
        else { fp[0] = fp[1] = fp[2] = fm[0] = fm[1] = fm[2] = T(0); }
        const int o = (r - 3) * G::XP + c;
#pragma unroll
        for (int m = 0; m < 3; ++m) { spl[m * G::SPL + o] = fp[m]; spl[(3 + m) * G::SPL + o] = fm[m]; }
        if (c >= 3 && c < TX + 3) sha[(r - 3) * TX + (c - 3)] = ch;
      }
    } else if (own_row) {
      const int o = (r - 3) * G::XP + c;
#pragma unroll
      for (int m = 0; m < 6; ++m) spl[m * G::SPL + o] = T(0);
      if (c >= 3 && c < TX + 3) sha[(r - 3) * TX + (c - 3)] = T(0);
    }
    sb[idx] = cb;
  }
  __syncthreads();

  T fsum_edge = T(0);  // 6 x (mass flux into the domain through its edges), per unit length in y
  // ---- phase B: x pass.  Lane l of warp w covers row 8*(w % (TY/8)) + l/4 and
  // strip 4*(w / (TY/8)) + l%4 (8 rows x 4 strips: conflict-free with XP = 1 mod 8).
  {
    const int w = tid >> 5, l = tid & 31;
    const int r = 8 * (w % (TY / 8)) + (l >> 2);
    const int c0 = (4 * (w / (TY / 8)) + (l & 3)) * S;
    T dF[3][S], db[S], Ff[S + 1];
    sweep_strip<T, S, 1>(spl + r * G::XP + c0, 1, G::SPL, 3 * G::SPL, sb + (r + 3) * G::BW + c0, 1, eps12, dF,
                         db, Ff);
    const T inv6dx = T(1.0 / (6.0 * p.dx));
    const T g12dx = T(p.g / (12.0 * p.dx));
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int o = r * TX + c0 + k;
      sL[o] = -dF[0][k] * inv6dx;
      sL[G::NC + o] = -dF[1][k] * inv6dx - g12dx * sha[o] * db[k];
      sL[2 * G::NC + o] = -dF[2][k] * inv6dx;
    }
    if (j0 + r < ny) {
      const int ia = i0 + c0;  // global index of the strip's first cell
      if (ia == 0) fsum_edge += Ff[0];
      const int kk = nx - ia;  // face nx-1/2 is face kk of the strip
#pragma unroll
      for (int k = 1; k <= S; ++k)
        if (k == kk) fsum_edge -= Ff[k];
    }
  }
  __syncthreads();

  // ---- phase B': y-split fluxes (halo rows, own columns) into the same buffer
  for (int idx = tid; idx < G::BH * TX; idx += NT) {
    const int r = idx / TX, c = idx - r * TX;
    const int i = i0 + c, j = j0 - 3 + r;
    T fp[3], fm[3];
    if (i < nx && j >= -3 && j < ny + 3) {
      T ch, chu, chv, cb;
      load_cell<T>(bb, hin, huin, hvin, nx, ny, pitch, p, zref, eta_in, u_in, i, j, ch, chu, chv, cb);
      split_cell<T, 1>(ch, chu, chv, cb, aly, g, zref, p, fp, fm);
    } else {
      fp[0] = fp[1] = fp[2] = fm[0] = fm[1] = fm[2] = T(0);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) { spl[m * G::SPL + idx] = fp[m]; spl[(3 + m) * G::SPL + idx] = fm[m]; }
  }
  __syncthreads();

  // ---- phase C: y pass, sources, RK combination, post rule, reductions
  T amax_x = T(0), amax_y = T(0), runup = T(0);
  double deficit = 0.0;
  bool bad = false;
  {
    const int c = tid % TX, r0 = (tid / TX) * S;
    T dG[3][S], db[S], Gf[S + 1];
    sweep_strip<T, S, 2>(spl + r0 * TX + c, TX, G::SPL, 3 * G::SPL, sb + r0 * G::BW + (c + 3), G::BW, eps12, dG,
                         db, Gf);
    const int i = i0 + c;
    if (i < nx) {
      const T rxy = T(p.dx / p.dy);
      const int jb = j0 + r0;
      if (jb == 0) fsum_edge += Gf[0] * rxy;
      const int kk = ny - jb;
#pragma unroll
      for (int k = 1; k <= S; ++k)
        if (k == kk) fsum_edge -= Gf[k] * rxy;
    }
    const T inv6dy = T(1.0 / (6.0 * p.dy));
    const T g12dy = T(p.g / (12.0 * p.dy));
    const T tdt = T(dt);
    const T rcap = dt > 0.0 ? T(1.0 / dt) : T(0);
    const T gn2 = T(p.g * p.n2);
    const bool friction = p.n2 > 0.0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int j = j0 + r0 + k;
      if (i < nx && j < ny) {
        const int o = (r0 + k) * TX + c;
        const size_t go = (size_t)j * pitch + i;
        const T ha = hin[go], hu = huin[go], hv = hvin[go];
        const T bc = bb[go];
        const T d = still_depth(bc, zref);
        const T h = ha + d;
        T Lh = sL[o] - dG[0][k] * inv6dy;
        T Lhu = sL[G::NC + o] - dG[1][k] * inv6dy;
        T Lhv = sL[2 * G::NC + o] - dG[2][k] * inv6dy - g12dy * sha[o] * db[k];
        if (friction && !Num<T>::below(h, p.h_dry32, p.h_dry)) {
          const T q = Num<T>::sqrt_(hu * hu + hv * hv);
          T kap = gn2 * q * Num<T>::rcp(Num<T>::pow73(h));
          if (dt > 0.0 && kap > rcap) kap = rcap;
          Lhu -= kap * hu;
          Lhv -= kap * hv;
        }
        // RK combination in increment form: U0 + w (U + dt L - U0)
        T nha = ha + tdt * Lh, nhu = hu + tdt * Lhu, nhv = hv + tdt * Lhv;
        if (STAGE != 1) {
          const T w = (STAGE == 2) ? T(0.25) : T(2.0 / 3.0);
          const T ha0 = fd.h[0][go], hu0 = fd.hu[0][go], hv0 = fd.hv[0][go];
          nha = ha0 + w * (nha - ha0);
          nhu = hu0 + w * (nhu - hu0);
          nhv = hv0 + w * (nhv - hv0);
        }
        // post-stage rule: clamp negative depth (counted), dry cells at rest
        if (nha < -d) { deficit -= (double)(nha + d); nha = -d; }
        const T nh = nha + d;
        T u = T(0), v = T(0);
        if (Num<T>::below(nh, p.h_dry32, p.h_dry)) { nhu = T(0); nhv = T(0); }
        else { const T rr = Num<T>::rcp(nh); u = nhu * rr; v = nhv * rr; }
        fd.h[OUTB][go] = nha;
        fd.hu[OUTB][go] = nhu;
        fd.hv[OUTB][go] = nhv;
        const T cel = Num<T>::sqrt_(g * nh);
        const T sx = fabs(u) + cel, sy = fabs(v) + cel;
        if (!(sx <= T(3.0e38)) || !(sy <= T(3.0e38)) || !(fabs(nhu) <= T(3.0e38)) || !(fabs(nhv) <= T(3.0e38)))
          bad = true;
        amax_x = sx > amax_x ? sx : amax_x;
        amax_y = sy > amax_y ? sy : amax_y;
        if (STAGE == 3 && !Num<T>::below(nh, p.h_wet32, p.h_wet) && bc > T(0)) {
          const T e = nh + bc;
          runup = e > runup ? e : runup;
        }
      }
    }
  }

  // ---- block reductions and device-scope publication
  const int w = tid >> 5, l = tid & 31;
  amax_x = warp_max(amax_x);
  amax_y = warp_max(amax_y);
  runup = warp_max(runup);
  deficit = warp_sum(deficit);
  const double ef = warp_sum((double)fsum_edge);
  const unsigned anybad = __any_sync(0xffffffffu, bad);
  if (l == 0) {
    red.a[w][0] = (double)amax_x;
    red.a[w][1] = (double)amax_y;
    red.s[w][0] = deficit;
    red.s[w][1] = ef;
    red.r[w] = (double)runup;
    if (anybad) red.bad = 1u;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0, my = 0.0, de = 0.0, fe = 0.0, ru = 0.0;
    for (int q = 0; q < NT / 32; ++q) {
      mx = fmax(mx, red.a[q][0]);
      my = fmax(my, red.a[q][1]);
      de += red.s[q][0];
      fe += red.s[q][1];
      ru = fmax(ru, red.r[q]);
    }
    atomicMax(&sc->alpha[STAGE % 3][0], dbits(mx));
    atomicMax(&sc->alpha[STAGE % 3][1], dbits(my));
    constexpr double wgt = (STAGE == 3) ? 1.0 : (STAGE == 2 ? 2.0 / 3.0 : 1.0 / 6.0);
    constexpr double wfl = (STAGE == 3) ? 2.0 / 3.0 : 1.0 / 6.0;
    if (de != 0.0) atomicAdd(&sc->clamp_mass, wgt * de * p.dx * p.dy);
    if (fe != 0.0) atomicAdd(&sc->boundary_mass, wfl * dt * fe * p.dy / 6.0);
    if (STAGE == 3 && ru > 0.0) {
      const unsigned long long rb = dbits(ru);
      atomicMax(&sc->runup_now[sc->parity], rb);
      atomicMax(&sc->runup_max, rb);
    }
    if (red.bad || !(mx <= 1e300) || !(my <= 1e300)) atomicOr(&sc->status, ST_NONFINITE);
    if (STAGE == 3 && lead) {
      const double tn = sc->t_step + dt;
      sc->t = (sc->t_end > 0.0 && tn >= sc->t_end) ? sc->t_end : tn;
      sc->steps += 1;
    }
  }
}

}  // namespace swe
