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

// Derived constants of the stage arithmetic, precomputed on the host in the
// state's precision (keeps FP64 work out of the FP32 kernels).
template <typename T>
struct Consts {
  T g, zref, eps12, inv6dx, g12dx, inv6dy, g12dy, gn2, hf4;
};

// Physical and numerical parameters, constant over a run.
struct Phys {
  double g, n2, h_dry, h_wet, h_film, hf4, weno_eps, fixed_dt, z_ref;
  double b_jump_x, b_jump_y;
  double inflow_amp, inflow_period, inflow_depth;
  double dx, dy;
  float h_dry32, h_wet32, h_film32;  // smallest floats whose double value is >= h_dry / h_wet / h_film
  int bc[4];
  Consts<float> c32;
  Consts<double> c64;
};

template <typename T>
__host__ __device__ __forceinline__ const Consts<T> &consts(const Phys &p);
template <>
__host__ __device__ __forceinline__ const Consts<float> &consts<float>(const Phys &p) { return p.c32; }
template <>
__host__ __device__ __forceinline__ const Consts<double> &consts<double>(const Phys &p) { return p.c64; }

// Fill the derived constants of a Phys (host side, once).
inline void finish_phys(Phys &p) {
  Consts<double> c;
  c.g = p.g;
  c.zref = p.z_ref;
  c.eps12 = 12.0 * p.weno_eps;
  c.inv6dx = 1.0 / (6.0 * p.dx);
  c.g12dx = p.g / (12.0 * p.dx);
  c.inv6dy = 1.0 / (6.0 * p.dy);
  c.g12dy = p.g / (12.0 * p.dy);
  c.gn2 = p.g * p.n2;
  c.hf4 = p.hf4;
  p.c64 = c;
  p.c32 = {(float)c.g, (float)c.zref, (float)c.eps12, (float)c.inv6dx, (float)c.g12dx, (float)c.inv6dy,
           (float)c.g12dy, (float)c.gn2, (float)c.hf4};
}

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
  static __device__ __forceinline__ float rsqrt_(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double pow73(double h) { return h * h * cbrt(h); }
  static __device__ __forceinline__ bool below(double h, float, double thr) { return h < thr; }
  static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
};

// WENO5-JS (Jiang & Shu 1996) at the right face of v2, scaled by 6.
// With t_k = 12 eps + 12 beta_k = q_k + 3 e_k^2, where q_k = 13 D2_k^2 + 12 eps
// is the second-difference part of the stencil's smoothness (cached by the
// caller: it depends on the 3-cell window only) and e_k its first-difference
// part, the weights d_k / t_k^2 have the ratios of d_k / (eps + beta_k)^2.
// Returns 6 W; a_k = 1/t_k^2 and rdn = 1 / sum d_k a_k are returned for
// applying the same weights to the bed.  Linear weights d_k are folded into
// the candidate coefficients (wc*).
template <typename T>
__device__ __forceinline__ T weno5q(T v0, T v1, T v2, T v3, T v4, T q0, T q1, T q2, T &a0, T &a1, T &a2,
                                    T &rdn) {
  const T e0 = v0 - T(4) * v1 + T(3) * v2;
  const T e1 = v1 - v3;
  const T e2 = T(3) * v2 - T(4) * v3 + v4;
  const T r0 = Num<T>::rcp(T(3) * e0 * e0 + q0);
  const T r1 = Num<T>::rcp(T(3) * e1 * e1 + q1);
  const T r2 = Num<T>::rcp(T(3) * e2 * e2 + q2);
  a0 = r0 * r0;
  a1 = r1 * r1;
  a2 = r2 * r2;
  rdn = Num<T>::rcp(T(0.1) * a0 + T(0.6) * a1 + T(0.3) * a2);
  // d_k * (6 p_k): 0.1 (2, -7, 11), 0.6 (-1, 5, 2), 0.3 (2, 5, -1)
  const T p0 = T(0.2) * v0 - T(0.7) * v1 + T(1.1) * v2;
  const T p1 = T(-0.6) * v1 + T(3.0) * v2 + T(1.2) * v3;
  const T p2 = T(0.6) * v2 + T(1.5) * v3 - T(0.3) * v4;
  return (a0 * p0 + a1 * p1 + a2 * p2) * rdn;
}

// 6 * (weighted candidate values) of a stencil with given weights.
template <typename T>
__device__ __forceinline__ T weighted6(T v0, T v1, T v2, T v3, T v4, T a0, T a1, T a2, T rdn) {
  const T p0 = T(0.2) * v0 - T(0.7) * v1 + T(1.1) * v2;
  const T p1 = T(-0.6) * v1 + T(3.0) * v2 + T(1.2) * v3;
  const T p2 = T(0.6) * v2 + T(1.5) * v3 - T(0.3) * v4;
  return (a0 * p0 + a1 * p1 + a2 * p2) * rdn;
}

// Second-difference smoothness part of the 3-cell window (a, b, c).
template <typename T>
__device__ __forceinline__ T qwin(T a, T b, T c, T eps12) {
  const T d2 = a - T(2) * b + c;
  return T(13) * d2 * d2 + eps12;
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

// Split fluxes of one cell in the frame of a sweep: qn is the discharge
// normal to the faces (hu for x, hv for y) and qt the tangential one.  With
// h = ha + d and pressure g ha (h + d)/2 = g (h^2 - d^2)/2:
//   F = (qn, qn un + pressure, qt un),  Q = (ha, qn, qt),  f+- = (F +- alpha Q)/2,
// i.e. F of Eq. (2) in x and G of Eq. (3) (with its momentum components
// swapped) in y.
template <typename T>
__device__ __forceinline__ void split_cell(T ha, T qn, T qt, T b, T alpha, T g, T zref, const Phys &p, T fp[3],
                                           T fm[3]) {
  const T d = still_depth(b, zref);
  const T h = ha + d;
  T un = T(0);
  if (!Num<T>::below(h, p.h_dry32, p.h_dry)) un = qn * Num<T>::rcp(h);
  const T pres = T(0.5) * g * ha * (h + d);
  const T F0 = qn, F1 = qn * un + pres, F2 = qt * un;
  const T q0 = alpha * ha, q1 = alpha * qn, q2 = alpha * qt;
  fp[0] = T(0.5) * (F0 + q0); fm[0] = T(0.5) * (F0 - q0);
  fp[1] = T(0.5) * (F1 + q1); fm[1] = T(0.5) * (F1 - q1);
  fp[2] = T(0.5) * (F2 + q2); fm[2] = T(0.5) * (F2 - q2);
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

// ------------------------------------------------------- asynchronous copies
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Shared-memory geometry of one tile.
template <typename T, int TX, int TY>
struct TileGeom {
  static constexpr int BW = TX + 6;  // halo box width (cells i0-3 .. i0+TX+2)
  static constexpr int BH = TY + 6;  // halo box height
  // row pitch: = 1 mod 8 floats (x-pass lanes on 8 rows x 4 strips hit distinct banks)
  static constexpr int P = ((BW + 7) / 8) * 8 + 1;
  static constexpr int FIELD = BH * P;  // one field of the box
  static constexpr int BOX = 4 * FIELD; // ha, hu, hv, b
  static constexpr int LP = TX + 1;        // L_x row pitch (x-pass lanes on 8 rows hit distinct banks)
  static constexpr int NC = TY * LP;       // one L_x component
  static constexpr int ELEMS = 2 * BOX + 3 * NC;  // two boxes (double buffer) + L_x
  static constexpr size_t BYTES = sizeof(T) * (size_t)ELEMS;
};

// Reduction scratch in shared memory (per CTA).
struct RedSmem {
  double a[32][2];
  double s[32][2];
  double r[32];
  double dt;
  double eta_in[3];
  unsigned bad;
  unsigned skip;
};

// The state planes a stage reads and writes.
template <typename T>
struct StageIO {
  const T *b;
  const T *ha, *hu, *hv;     // stage input (halo reads)
  const T *ha0, *hu0, *hv0;  // U^n (own cells, stages 2 and 3)
  T *oha, *ohu, *ohv;        // stage output
  int nx, ny, pitch;
};

// Issue the asynchronous copies of the halo box of tile (i0, j0) into box:
// interior cells only; ghost positions are patched after arrival.
template <typename T, int TX, int TY, int NT>
__device__ __forceinline__ void issue_box(const StageIO<T> &io, int i0, int j0, T *box) {
  using G = TileGeom<T, TX, TY>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T *src[4] = {io.ha, io.hu, io.hv, io.b};
  for (int r = warp; r < G::BH; r += NT / 32) {
    const int j = j0 - 3 + r;
    if (j < 0 || j >= io.ny) continue;
#pragma unroll
    for (int c = lane; c < ((G::BW + 31) / 32) * 32; c += 32) {
      const int i = i0 - 3 + c;
      if (c < G::BW && i >= 0 && i < io.nx) {
        const size_t go = (size_t)j * io.pitch + i;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (sizeof(T) == 4) cp_async4(box + f * G::FIELD + r * G::P + c, src[f] + go);
          else cp_async8(box + f * G::FIELD + r * G::P + c, src[f] + go);
        }
      }
    }
  }
}

// Fill every box position outside the domain (tiles whose box crosses the
// domain edge): cells within 3 of the edge along one axis get ghost values,
// all others (beyond the ghosts, or outside along both axes) are zeroed and
// never read by a valid cell.  Walls mirror cells of the same box; inflow
// ghosts carry the N-wave; periodic ghosts are read across the seam.
template <typename T, int TX, int TY, int NT>
__device__ __noinline__ void patch_box(const StageIO<T> &io, const Phys &p, int i0, int j0, T *box, T zref,
                                       T eta_in, T u_in) {
  using G = TileGeom<T, TX, TY>;
  const int nx = io.nx, ny = io.ny;
  T *bha = box, *bhu = box + G::FIELD, *bhv = box + 2 * G::FIELD, *bb = box + 3 * G::FIELD;
  for (int q = threadIdx.x; q < G::BH * G::BW; q += NT) {
    const int r = q / G::BW, c = q - r * G::BW;
    const int i = i0 - 3 + c, j = j0 - 3 + r;
    const bool in_i = i >= 0 && i < nx, in_j = j >= 0 && j < ny;
    if (in_i && in_j) continue;  // a real cell, already loaded
    const int o = r * G::P + c;
    const bool xg = !in_i && in_j && i >= -3 && i < nx + 3;  // x ghost
    const bool yg = in_i && !in_j && j >= -3 && j < ny + 3;  // y ghost
    if (!xg && !yg) {
      bha[o] = bhu[o] = bhv[o] = bb[o] = T(0);
      continue;
    }
    const int side = xg ? (i < 0 ? 0 : 1) : (j < 0 ? 2 : 3);
    const int bc = p.bc[side];
    if (bc == BC_PERIODIC) {
      int si = i, sj = j;
      T shift;
      if (xg) { si = i < 0 ? i + nx : i - nx; shift = T(i < 0 ? -p.b_jump_x : p.b_jump_x); }
      else { sj = j < 0 ? j + ny : j - ny; shift = T(j < 0 ? -p.b_jump_y : p.b_jump_y); }
      const size_t go = (size_t)sj * io.pitch + si;
      const T bs = io.b[go], cb = bs + shift;
      bb[o] = cb;
      bha[o] = (io.ha[go] + still_depth(bs, zref)) - still_depth(cb, zref);
      bhu[o] = io.hu[go];
      bhv[o] = io.hv[go];
      continue;
    }
    // mirror source: a real cell of the same box
    int mc = c, mr = r;
    if (xg) mc = (i < 0 ? (-1 - i) : (2 * nx - 1 - i)) - (i0 - 3);
    else mr = (j < 0 ? (-1 - j) : (2 * ny - 1 - j)) - (j0 - 3);
    const int m = mr * G::P + mc;
    const T cb = bb[m];
    bb[o] = cb;
    if (bc == BC_INFLOW) {
      const T dg = still_depth(cb, zref);
      T a;
      if (cb < zref) { a = eta_in - zref; a = a > -dg ? a : -dg; }
      else { a = eta_in - cb; a = a > T(0) ? a : T(0); }
      bha[o] = a;
      bhu[o] = (a + dg) * u_in;
      bhv[o] = T(0);
    } else {
      bha[o] = bha[m];
      bhu[o] = xg ? -bhu[m] : bhu[m];
      bhv[o] = xg ? bhv[m] : -bhv[m];
    }
  }
}

// Sliding WENO5 window along one line of the box (one strip of S cells), in
// the frame of the sweep.  Slots 0..5 hold cells c0-3+k .. c0+2+k for face k
// (between slots 2 and 3); qp[s] / qm[s] cache the second-difference
// smoothness of the 3-cell window centred at slot s for f+ / f-.
template <typename T>
struct Window {
  T fp[3][6], fm[3][6], bw[6];
  T qp[3][5], qm[3][5];
  __device__ __forceinline__ void put(int q, const T *bha, const T *bqn, const T *bqt, const T *bb, int o, T alpha,
                                      T g, T zref, const Phys &p) {
    T a[3], m[3];
    const T b = bb[o];
    split_cell<T>(bha[o], bqn[o], bqt[o], b, alpha, g, zref, p, a, m);
#pragma unroll
    for (int c = 0; c < 3; ++c) { fp[c][q] = a[c]; fm[c][q] = m[c]; }
    bw[q] = b;
  }
  __device__ __forceinline__ void window_terms(int s, T eps12) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      qp[c][s] = qwin(fp[c][s - 1], fp[c][s], fp[c][s + 1], eps12);
      qm[c][s] = qwin(fm[c][s - 1], fm[c][s], fm[c][s + 1], eps12);
    }
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { fp[c][q] = fp[c][q + 1]; fm[c][q] = fm[c][q + 1]; }
      bw[q] = bw[q + 1];
    }
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) { qp[c][q] = qp[c][q + 1]; qm[c][q] = qm[c][q + 1]; }
  }
  // face between slots 2 and 3: F6[c] = 6 Fhat_c, B12 = 12 bhat (weights of c = 1)
  __device__ __forceinline__ void face(T F6[3], T &B12) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T a0, a1, a2, rp, c0, c1, c2, rm;
      const T Fp = weno5q<T>(fp[c][0], fp[c][1], fp[c][2], fp[c][3], fp[c][4], qp[c][1], qp[c][2], qp[c][3], a0,
                             a1, a2, rp);
      const T Fm = weno5q<T>(fm[c][5], fm[c][4], fm[c][3], fm[c][2], fm[c][1], qm[c][4], qm[c][3], qm[c][2], c0,
                             c1, c2, rm);
      F6[c] = Fp + Fm;
      if (c == 1)
        B12 = weighted6<T>(bw[0], bw[1], bw[2], bw[3], bw[4], a0, a1, a2, rp) +
              weighted6<T>(bw[5], bw[4], bw[3], bw[2], bw[1], c0, c1, c2, rm);
    }
  }
};

// ------------------------------------------------- packed FP32 (f32x2) path
// Components 0 (mass) and 1 (normal momentum) of a sweep share every stencil
// position, so their reconstructions run as float2 pairs with the packed
// FP32 instructions of sm_100+ (one issue slot for two lanes); component 2
// stays scalar.  Each lane follows the same operation sequence as the scalar
// reconstruction below, so both lanes round exactly like scalar code.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(Num<float>::rcp(a.x), Num<float>::rcp(a.y)); }

// Scalar FP32 reconstruction with the explicit operation sequence of weno5p.
__device__ __forceinline__ float weno5s(float v0, float v1, float v2, float v3, float v4, float q0, float q1, float q2,
                                        float &a0, float &a1, float &a2, float &rdn) {
  const float e0 = fmaf(3.f, v2, fmaf(-4.f, v1, v0));
  const float e1 = fmaf(-1.f, v3, v1);
  const float e2 = fmaf(-4.f, v3, fmaf(3.f, v2, v4));
  const float r0 = Num<float>::rcp(fmaf(3.f * e0, e0, q0));
  const float r1 = Num<float>::rcp(fmaf(3.f * e1, e1, q1));
  const float r2 = Num<float>::rcp(fmaf(3.f * e2, e2, q2));
  a0 = r0 * r0;
  a1 = r1 * r1;
  a2 = r2 * r2;
  rdn = Num<float>::rcp(fmaf(0.3f, a2, fmaf(0.6f, a1, 0.1f * a0)));
  const float p0 = fmaf(1.1f, v2, fmaf(-0.7f, v1, 0.2f * v0));
  const float p1 = fmaf(1.2f, v3, fmaf(3.0f, v2, -0.6f * v1));
  const float p2 = fmaf(-0.3f, v4, fmaf(1.5f, v3, 0.6f * v2));
  return fmaf(a2, p2, fmaf(a1, p1, a0 * p0)) * rdn;
}

__device__ __forceinline__ float2 weno5p(float2 v0, float2 v1, float2 v2, float2 v3, float2 v4, float2 q0, float2 q1,
                                         float2 q2, float2 &a0, float2 &a1, float2 &a2, float2 &rdn) {
  const float2 e0 = fma2(f2(3.f), v2, fma2(f2(-4.f), v1, v0));
  const float2 e1 = fma2(f2(-1.f), v3, v1);
  const float2 e2 = fma2(f2(-4.f), v3, fma2(f2(3.f), v2, v4));
  const float2 r0 = rcp2(fma2(mul2(f2(3.f), e0), e0, q0));
  const float2 r1 = rcp2(fma2(mul2(f2(3.f), e1), e1, q1));
  const float2 r2 = rcp2(fma2(mul2(f2(3.f), e2), e2, q2));
  a0 = mul2(r0, r0);
  a1 = mul2(r1, r1);
  a2 = mul2(r2, r2);
  rdn = rcp2(fma2(f2(0.3f), a2, fma2(f2(0.6f), a1, mul2(f2(0.1f), a0))));
  const float2 p0 = fma2(f2(1.1f), v2, fma2(f2(-0.7f), v1, mul2(f2(0.2f), v0)));
  const float2 p1 = fma2(f2(1.2f), v3, fma2(f2(3.0f), v2, mul2(f2(-0.6f), v1)));
  const float2 p2 = fma2(f2(-0.3f), v4, fma2(f2(1.5f), v3, mul2(f2(0.6f), v2)));
  return mul2(fma2(a2, p2, fma2(a1, p1, mul2(a0, p0))), rdn);
}

__device__ __forceinline__ float weighted6s(float v0, float v1, float v2, float v3, float v4, float a0, float a1,
                                            float a2, float rdn) {
  const float p0 = fmaf(1.1f, v2, fmaf(-0.7f, v1, 0.2f * v0));
  const float p1 = fmaf(1.2f, v3, fmaf(3.0f, v2, -0.6f * v1));
  const float p2 = fmaf(-0.3f, v4, fmaf(1.5f, v3, 0.6f * v2));
  return fmaf(a2, p2, fmaf(a1, p1, a0 * p0)) * rdn;
}

__device__ __forceinline__ float qwins(float a, float b, float c, float eps12) {
  const float d2 = fmaf(-2.f, b, a) + c;
  return fmaf(13.f * d2, d2, eps12);
}
__device__ __forceinline__ float2 qwinp(float2 a, float2 b, float2 c, float2 eps12) {
  const float2 d2 = add2(fma2(f2(-2.f), b, a), c);
  return fma2(mul2(f2(13.f), d2), d2, eps12);
}

// Packed FP32 window: (component 0, component 1) as float2, component 2 scalar.
struct WindowP {
  float2 fp01[6], fm01[6];
  float fp2[6], fm2[6], bw[6];
  float2 qp01[5], qm01[5];
  float qp2[5], qm2[5];
  __device__ __forceinline__ void put(int q, const float *bha, const float *bqn, const float *bqt, const float *bb,
                                      int o, float alpha, float g, float zref, const Phys &p) {
    const float ha = bha[o], qn = bqn[o], qt = bqt[o], b = bb[o];
    const float d = still_depth(b, zref);
    const float h = ha + d;
    float un = 0.f;
    if (!Num<float>::below(h, p.h_dry32, p.h_dry)) un = qn * Num<float>::rcp(h);
    const float pres = 0.5f * g * ha * (h + d);
    // F = (qn, qn un + pres, qt un), Q = (ha, qn, qt); f+- = F/2 +- (alpha/2) Q
    const float2 hF = mul2(f2(0.5f), make_float2(qn, fmaf(qn, un, pres)));
    const float2 hQ = mul2(f2(0.5f * alpha), make_float2(ha, qn));
    fp01[q] = add2(hF, hQ);
    fm01[q] = fma2(f2(-1.f), hQ, hF);
    const float hF2 = 0.5f * (qt * un), hQ2 = (0.5f * alpha) * qt;
    fp2[q] = hF2 + hQ2;
    fm2[q] = hF2 - hQ2;
    bw[q] = b;
  }
  __device__ __forceinline__ void window_terms(int s, float eps12) {
    qp01[s] = qwinp(fp01[s - 1], fp01[s], fp01[s + 1], f2(eps12));
    qm01[s] = qwinp(fm01[s - 1], fm01[s], fm01[s + 1], f2(eps12));
    qp2[s] = qwins(fp2[s - 1], fp2[s], fp2[s + 1], eps12);
    qm2[s] = qwins(fm2[s - 1], fm2[s], fm2[s + 1], eps12);
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      fp01[q] = fp01[q + 1];
      fm01[q] = fm01[q + 1];
      fp2[q] = fp2[q + 1];
      fm2[q] = fm2[q + 1];
      bw[q] = bw[q + 1];
    }
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      qp01[q] = qp01[q + 1];
      qm01[q] = qm01[q + 1];
      qp2[q] = qp2[q + 1];
      qm2[q] = qm2[q + 1];
    }
  }
  __device__ __forceinline__ void face(float F6[3], float &B12) const {
    float2 a0, a1, a2, rp, c0, c1, c2, rm;
    const float2 Fp = weno5p(fp01[0], fp01[1], fp01[2], fp01[3], fp01[4], qp01[1], qp01[2], qp01[3], a0, a1, a2, rp);
    const float2 Fm = weno5p(fm01[5], fm01[4], fm01[3], fm01[2], fm01[1], qm01[4], qm01[3], qm01[2], c0, c1, c2, rm);
    const float2 F01 = add2(Fp, Fm);
    F6[0] = F01.x;
    F6[1] = F01.y;
    // bed with the weights of component 1 (the .y lanes)
    B12 = weighted6s(bw[0], bw[1], bw[2], bw[3], bw[4], a0.y, a1.y, a2.y, rp.y) +
          weighted6s(bw[5], bw[4], bw[3], bw[2], bw[1], c0.y, c1.y, c2.y, rm.y);
    float s0, s1, s2, sr, t0, t1, t2, tr;
    const float Gp = weno5s(fp2[0], fp2[1], fp2[2], fp2[3], fp2[4], qp2[1], qp2[2], qp2[3], s0, s1, s2, sr);
    const float Gm = weno5s(fm2[5], fm2[4], fm2[3], fm2[2], fm2[1], qm2[4], qm2[3], qm2[2], t0, t1, t2, tr);
    F6[2] = Gp + Gm;
  }
};

template <typename T> struct WindowOf { using type = Window<T>; };
template <> struct WindowOf<float> { using type = WindowP; };

// One strip: faces k = 0..S (face k at the left of strip cell k).  Returns
// dF[c][k] = 6 (Fhat_c(k+1) - Fhat_c(k)) and db[k] = 12 (bhat(k+1) - bhat(k))
// for the S cells, and adds the mass flux through the domain edges that the
// strip owns (face -1/2 at k = 0 of the first strip, face n-1/2 at k >= 1).
template <typename T, int S>
__device__ __forceinline__ void sweep_strip(const T *bha, const T *bqn, const T *bqt, const T *bb, int o0, int st,
                                            T alpha, T g, T zref, T eps12, const Phys &p, int ia, int n,
                                            bool edge_ok, T dF[3][S], T db[S], T &edge) {
  typename WindowOf<T>::type win;
#pragma unroll
  for (int q = 0; q < 5; ++q) win.put(q, bha, bqn, bqt, bb, o0 + q * st, alpha, g, zref, p);
#pragma unroll
  for (int q = 1; q < 4; ++q) win.window_terms(q, eps12);
  T prevF[3], prevB = T(0);
#pragma unroll
  for (int k = 0; k <= S; ++k) {
    win.put(5, bha, bqn, bqt, bb, o0 + (k + 5) * st, alpha, g, zref, p);
    win.window_terms(4, eps12);
    T F6[3], B12 = T(0);
    win.face(F6, B12);
    if (edge_ok && ((k == 0 && ia == 0) || (k > 0 && ia + k == n))) edge += (k == 0) ? F6[0] : -F6[0];
    if (k > 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) dF[c][k - 1] = F6[c] - prevF[c];
      db[k - 1] = B12 - prevB;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) prevF[c] = F6[c];
    prevB = B12;
    win.shift();
  }
}

// Per-CTA accumulators carried across the tiles of one launch.
template <typename T>
struct Acc {
  T ax = T(0), ay = T(0), ru = T(0), chk = T(0);
  T deficit = T(0), edge = T(0);  // diagnostics, summed in the state's precision per thread
};

// One RK3 stage (Eq. (8), Shu-Osher form, increment form) on one tile whose
// halo box is resident in shared memory:
//   stage 1: U1 = U^n + dt L(U^n)
//   stage 2: U2 = U^n + 1/4 (U1 + dt L(U1) - U^n)
//   stage 3: U^{n+1} = U^n + 2/3 (U2 + dt L(U2) - U^n)   (written over U^n)
// followed by the post-stage rule, with L of Eq. (7).  Pass 0 sweeps x and
// stores L_x; pass 1 sweeps y, adds L_y and the sources and updates.  Both
// passes run the same sweep code (loop not unrolled: one copy of the WENO
// body in the instruction stream).
template <typename T, int TX, int TY, int NT, int S, int STAGE>
__device__ __forceinline__ void tile_compute(const StageIO<T> &io, const Phys &p, int i0, int j0, const T *box,
                                             T *sL, T tdt, T rcap, T alx, T aly, Acc<T> &acc) {
  using G = TileGeom<T, TX, TY>;
  static_assert(TX % S == 0 && TY % S == 0, "strip length must divide the tile");
  static_assert((TX / S) * TY == NT && (TY / S) * TX == NT, "one strip per thread in both passes");
  // x pass: a warp covers RW rows x SW strips; with the box row pitch = 1 mod 8
  // the lanes' window loads hit distinct banks (8 rows x 4 strips of 8 cells,
  // or 16 rows x 2 strips of 16 cells)
  constexpr int SW = (S >= 16) ? 2 : 4, RW = 32 / SW;
  static_assert(TY % RW == 0 && (TX / S) % SW == 0 && (TY / RW) * ((TX / S) / SW) == NT / 32,
                "x-pass warps tile the rows and strips");
  const int tid = threadIdx.x;
  const int nx = io.nx, ny = io.ny;
  const T *bha = box, *bhu = box + G::FIELD, *bhv = box + 2 * G::FIELD, *bb = box + 3 * G::FIELD;
  const Consts<T> &K = consts<T>(p);
  const T g = K.g, zref = K.zref, eps12 = K.eps12;
  // x pass: lane l of warp w takes row RW*(w % (TY/RW)) + l/SW and strip SW*(w / (TY/RW)) + l%SW
  const int w = tid >> 5, l = tid & 31;
  const int xr = RW * (w % (TY / RW)) + l / SW;
  const int xc0 = (SW * (w / (TY / RW)) + l % SW) * S;
  // y pass: thread takes column tid % TX and strip tid / TX
  const int yc = tid % TX, yr0 = (tid / TX) * S;
  const int i = i0 + yc;

#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const bool X = pass == 0;
    // U^n of the y-pass cells (stages 2, 3), fetched before the sweep so that
    // the global-memory latency hides behind it
    T u0[3][S];
    if (STAGE != 1 && !X) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const int j = j0 + yr0 + k;
        const bool ok = i < nx && j < ny;
        const size_t go = ok ? (size_t)j * io.pitch + i : 0;
        u0[0][k] = ok ? io.ha0[go] : T(0);
        u0[1][k] = ok ? io.hu0[go] : T(0);
        u0[2][k] = ok ? io.hv0[go] : T(0);
      }
    }
    T dF[3][S], db[S];
    sweep_strip<T, S>(bha, X ? bhu : bhv, X ? bhv : bhu, bb, X ? (xr + 3) * G::P + xc0 : yr0 * G::P + yc + 3,
                      X ? 1 : G::P, X ? alx : aly, g, zref, eps12, p, X ? i0 + xc0 : j0 + yr0, X ? nx : ny,
                      X ? (j0 + xr < ny) : (i < nx), dF, db, acc.edge);
    if (X) {
      const T inv6dx = K.inv6dx;
      const T g12dx = K.g12dx;
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const int o = xr * G::LP + xc0 + k;
        const T ha = bha[(xr + 3) * G::P + xc0 + k + 3];
        sL[o] = -dF[0][k] * inv6dx;
        sL[G::NC + o] = -dF[1][k] * inv6dx - g12dx * ha * db[k];
        sL[2 * G::NC + o] = -dF[2][k] * inv6dx;
      }
      __syncthreads();
      continue;
    }
    // y pass epilogue: sources, RK combination, post rule (dF[1] is hv, dF[2] hu)
    const T inv6dy = K.inv6dy;
    const T g12dy = K.g12dy;
    const T gn2 = K.gn2;
    const bool friction = p.n2 > 0.0;
    const T wrk = (STAGE == 2) ? T(0.25) : T(2.0 / 3.0);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int j = j0 + yr0 + k;
      if (i < nx && j < ny) {
        const int o = (yr0 + k) * G::LP + yc;
        const int bo = (yr0 + k + 3) * G::P + yc + 3;
        const T ha = bha[bo], hu = bhu[bo], hv = bhv[bo], bc = bb[bo];
        const T d = still_depth(bc, zref);
        const T h = ha + d;
        T Lh = sL[o] - dF[0][k] * inv6dy;
        T Lhu = sL[G::NC + o] - dF[2][k] * inv6dy;
        T Lhv = sL[2 * G::NC + o] - dF[1][k] * inv6dy - g12dy * ha * db[k];
        if (friction && !Num<T>::below(h, p.h_dry32, p.h_dry)) {
          const T q = Num<T>::sqrt_(hu * hu + hv * hv);
          T kap = gn2 * q * Num<T>::rcp(Num<T>::pow73(h));
          kap = kap > rcap ? rcap : kap;  // rcap = 1/dt
          Lhu -= kap * hu;
          Lhv -= kap * hv;
        }
        T nha = ha + tdt * Lh, nhu = hu + tdt * Lhu, nhv = hv + tdt * Lhv;
        const size_t go = (size_t)j * io.pitch + i;
        if (STAGE != 1) {
          nha = u0[0][k] + wrk * (nha - u0[0][k]);
          nhu = u0[1][k] + wrk * (nhu - u0[1][k]);
          nhv = u0[2][k] + wrk * (nhv - u0[2][k]);
        }
        if (nha < -d) { acc.deficit -= nha + d; nha = -d; }
        const T nh = nha + d;
        T u = T(0), v = T(0);
        if (Num<T>::below(nh, p.h_dry32, p.h_dry)) { nhu = T(0); nhv = T(0); }
        else {
          if (Num<T>::below(nh, p.h_film32, p.h_film)) {  // film: bounded velocity
            const T h2 = nh * nh;
            const T f = T(1.4142135623730951) * h2 * Num<T>::rsqrt_(h2 * h2 + K.hf4);
            nhu *= f;
            nhv *= f;
          }
          const T rr = Num<T>::rcp(nh);
          u = nhu * rr;
          v = nhv * rr;
        }
        io.oha[go] = nha;
        io.ohu[go] = nhu;
        io.ohv[go] = nhv;
        const T cel = Num<T>::sqrt_(g * nh);
        const T sx = fabs(u) + cel, sy = fabs(v) + cel;
        acc.chk += sx + sy;  // non-finite values propagate to the per-CTA check
        acc.ax = sx > acc.ax ? sx : acc.ax;
        acc.ay = sy > acc.ay ? sy : acc.ay;
        if (STAGE == 3 && !Num<T>::below(nh, p.h_wet32, p.h_wet) && bc > T(0)) {
          const T e = nh + bc;
          acc.ru = e > acc.ru ? e : acc.ru;
        }
      }
    }
  }
}

// Per-stage scalars and the skip decision, taken by thread 0 of every CTA;
// the lead CTA of a scenario also does the per-step bookkeeping.  Stage s
// reads the wave speeds of its input from slot s-1, publishes those of its
// output to slot s mod 3 and clears slot (s+1) mod 3, which nothing reads or
// writes during stage s.
template <int STAGE>
__device__ __forceinline__ void stage_scalars(const Phys &p, DevScalars *sc, bool lead, RedSmem &red, double &ax,
                                              double &ay) {
  // read through L2 (other CTAs wrote these before the last grid barrier or launch)
  ax = bitsd(__ldcg(&sc->alpha[STAGE - 1][0]));
  ay = bitsd(__ldcg(&sc->alpha[STAGE - 1][1]));
  const double t_now = __ldcg(&sc->t), t_end = __ldcg(&sc->t_end);
  double dt = 0.0;
  unsigned skip = __ldcg(&sc->status) != 0u;
  if (STAGE == 1) {
    if (t_end > 0.0 && t_now >= t_end) skip = 1;
    if (p.fixed_dt > 0.0) dt = p.fixed_dt;
    else {
      const double den = ax / p.dx + ay / p.dy;
      if (den > 0.0) dt = __ldcg(&sc->cfl) / den;
      else if (!skip) { skip = 1; atomicOr(&sc->status, ST_DRY); }
    }
    if (t_end > 0.0 && t_now + dt > t_end) dt = t_end - t_now;
    if (lead) {
      sc->running = skip ? 0u : 1u;
      if (!skip) {
        const long long steps = __ldcg(&sc->steps);
        sc->dt = dt;
        sc->t_step = t_now;
        sc->parity = (unsigned)(steps & 1);
        sc->runup_now[steps & 1] = 0ull;
        sc->alpha[2][0] = 0ull;
        sc->alpha[2][1] = 0ull;
      }
    }
  } else {
    if (!__ldcg(&sc->running)) skip = 1;
    dt = __ldcg(&sc->dt);
    if (lead && !skip) {
      sc->alpha[STAGE == 2 ? 0 : 1][0] = 0ull;
      sc->alpha[STAGE == 2 ? 0 : 1][1] = 0ull;
    }
  }
  red.skip = skip;
  red.bad = 0u;
  red.dt = dt;
  const double tst = (STAGE == 1) ? t_now : __ldcg(&sc->t_step);
  const double ts = (STAGE == 1) ? tst : (STAGE == 2 ? tst + dt : tst + 0.5 * dt);
  red.eta_in[0] = (p.bc[0] == BC_INFLOW) ? inflow_eta(p, ts) : 0.0;
}

// Block reduction of the per-thread accumulators and device-scope
// publication for one scenario.
template <typename T, int NT, int STAGE>
__device__ __forceinline__ void publish(const Phys &p, DevScalars *sc, bool lead, RedSmem &red, double dt,
                                        const Acc<T> &acc) {
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const T ax = warp_max(acc.ax), ay = warp_max(acc.ay), ru = warp_max(acc.ru);
  const double de = warp_sum((double)acc.deficit), ef = warp_sum((double)acc.edge);
  const bool bad = !(acc.chk <= T(3.0e38));
  const unsigned anybad = __any_sync(0xffffffffu, bad);
  if (l == 0) {
    red.a[w][0] = (double)ax;
    red.a[w][1] = (double)ay;
    red.s[w][0] = de;
    red.s[w][1] = ef;
    red.r[w] = (double)ru;
    if (anybad) red.bad = 1u;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0, my = 0.0, dsum = 0.0, fsum = 0.0, rmax = 0.0;
    for (int q = 0; q < NT / 32; ++q) {
      mx = fmax(mx, red.a[q][0]);
      my = fmax(my, red.a[q][1]);
      dsum += red.s[q][0];
      fsum += red.s[q][1];
      rmax = fmax(rmax, red.r[q]);
    }
    atomicMax(&sc->alpha[STAGE % 3][0], dbits(mx));
    atomicMax(&sc->alpha[STAGE % 3][1], dbits(my));
    constexpr double wgt = (STAGE == 3) ? 1.0 : (STAGE == 2 ? 2.0 / 3.0 : 1.0 / 6.0);
    constexpr double wfl = (STAGE == 3) ? 2.0 / 3.0 : 1.0 / 6.0;
    if (dsum != 0.0) atomicAdd(&sc->clamp_mass, wgt * dsum * p.dx * p.dy);
    if (fsum != 0.0) atomicAdd(&sc->boundary_mass, wfl * dt * fsum * p.dy / 6.0);
    if (STAGE == 3 && rmax > 0.0) {
      const unsigned long long rb = dbits(rmax);
      atomicMax(&sc->runup_now[__ldcg(&sc->parity)], rb);
      atomicMax(&sc->runup_max, rb);
    }
    if (red.bad) atomicOr(&sc->status, ST_NONFINITE);
    if (STAGE == 3 && lead) {
      const double tn = __ldcg(&sc->t_step) + dt, te = __ldcg(&sc->t_end);
      sc->t = (te > 0.0 && tn >= te) ? te : tn;
      sc->steps = __ldcg(&sc->steps) + 1;
    }
  }
}

// Persistent stage over all tiles of one scenario: CTA b handles tiles
// b, b + gridDim.x, ...; the halo box of the next tile is copied
// asynchronously while the current one is computed.
template <typename T, int TX, int TY, int NT, int S, int STAGE>
__device__ void stage_persistent(const StageIO<T> &io, const Phys &p, DevScalars *sc, T *smem, RedSmem &red,
                                 int first, int stride, bool lead) {
  using G = TileGeom<T, TX, TY>;
  const int tid = threadIdx.x;
  const int tiles_x = (io.nx + TX - 1) / TX, tiles_y = (io.ny + TY - 1) / TY;
  const int ntiles = tiles_x * tiles_y;
  if (tid == 0) {
    double ax, ay;
    stage_scalars<STAGE>(p, sc, lead, red, ax, ay);
    red.a[0][0] = ax;
    red.a[0][1] = ay;
  }
  __syncthreads();
  if (red.skip) return;
  const double dt = red.dt;
  const T tdt = T(dt), rcap = dt > 0.0 ? T(1.0 / dt) : T(0);
  const T alx = T(red.a[0][0]), aly = T(red.a[0][1]);
  const T zref = consts<T>(p).zref;
  const T eta_in = T(red.eta_in[0]);
  const T u_in = (p.bc[0] == BC_INFLOW) ? T(red.eta_in[0] * sqrt(p.g / p.inflow_depth)) : T(0);
  T *box0 = smem, *box1 = smem + G::BOX, *sL = smem + 2 * G::BOX;
  Acc<T> acc;
  int t = first;
  if (t < ntiles) issue_box<T, TX, TY, NT>(io, (t % tiles_x) * TX, (t / tiles_x) * TY, box0);
  cp_commit();
  for (int it = 0; t < ntiles; ++it, t += stride) {
    T *box = (it & 1) ? box1 : box0;
    const int tn = t + stride;
    if (tn < ntiles) issue_box<T, TX, TY, NT>(io, (tn % tiles_x) * TX, (tn / tiles_x) * TY, (it & 1) ? box0 : box1);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int i0 = (t % tiles_x) * TX, j0 = (t / tiles_x) * TY;
    if (i0 == 0 || j0 == 0 || i0 + TX + 3 > io.nx || j0 + TY + 3 > io.ny) {
      patch_box<T, TX, TY, NT>(io, p, i0, j0, box, zref, eta_in, u_in);
      __syncthreads();
    }
    tile_compute<T, TX, TY, NT, S, STAGE>(io, p, i0, j0, box, sL, tdt, rcap, alx, aly, acc);
    __syncthreads();
  }
  cp_wait<0>();
  publish<T, NT, STAGE>(p, sc, lead, red, dt, acc);
}

// ------------------------------------------------------------ batch driver
// One scenario of a batch as the kernels see it (device memory).
template <typename T>
struct BatchSlot {
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
};

// Grid-wide barrier of a cooperative launch with a bounded wait.  Returns
// false (and sets ST_TIMEOUT) if the other CTAs did not arrive in time; the
// caller then leaves the kernel.
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
        if (clock64() - t0 > ctl->bar_cycles || *(volatile unsigned *)&ctl->status) {
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

// One RK stage over the work list of a batch: CTA b handles items b,
// b + gridDim.x, ...  Per-scenario scalars are taken when the CTA enters a
// scenario and its accumulators are published when it leaves it; the lead
// CTA of a scenario is the one that owns its tile 0.
template <typename T, int TX, int TY, int NT, int S, int STAGE>
__device__ void batch_stage(const BatchSlot<T> *slots, int nslots, int total, T *smem, RedSmem &red, Phys &sp) {
  using G = TileGeom<T, TX, TY>;
  __shared__ int s_slot;
  __shared__ unsigned s_skip;
  __shared__ StageIO<T> s_io;  // planes of the current scenario (kept out of registers)
  T *box0 = smem, *box1 = smem + G::BOX, *sL = smem + 2 * G::BOX;
  const int tid = threadIdx.x;
  const int G0 = gridDim.x;
  int cur = -1;
  bool lead = false, skip = true;
  double dt = 0.0;
  T tdt = T(0), rcap = T(0), alx = T(0), aly = T(0), eta_in = T(0), u_in = T(0);
  Acc<T> acc;
  int item = blockIdx.x;
  if (item < total) {
    const int s0 = slot_of_item(slots, nslots, item);
    const int t0 = item - slots[s0].first_item;
    issue_box<T, TX, TY, NT>(io_of(slots[s0].fd, STAGE), (t0 % slots[s0].tiles_x) * TX, (t0 / slots[s0].tiles_x) * TY, box0);
  }
  cp_commit();
  for (int it = 0; item < total; ++it, item += G0) {
    if (tid == 0) s_slot = slot_of_item(slots, nslots, item);
    __syncthreads();
    const int s = s_slot;
    const BatchSlot<T> &sl = slots[s];
    if (s != cur) {
      if (cur >= 0 && !skip) publish<T, NT, STAGE>(sp, slots[cur].sc, lead, red, dt, acc);
      acc = Acc<T>();
      __syncthreads();
      if (tid == 0) {
        sp = sl.p;
        s_io = io_of(sl.fd, STAGE);
        double ax, ay;
        const bool ld = (sl.first_item % G0) == (int)blockIdx.x;
        stage_scalars<STAGE>(sp, sl.sc, ld, red, ax, ay);
        red.a[0][0] = ax;
        red.a[0][1] = ay;
        s_skip = red.skip;
      }
      __syncthreads();
      cur = s;
      lead = (sl.first_item % G0) == (int)blockIdx.x;
      skip = s_skip != 0u;
      dt = red.dt;
      tdt = T(dt);
      rcap = dt > 0.0 ? T(1.0 / dt) : T(0);
      alx = T(red.a[0][0]);
      aly = T(red.a[0][1]);
      eta_in = T(red.eta_in[0]);
      u_in = (sp.bc[0] == BC_INFLOW) ? T(red.eta_in[0] * sqrt(sp.g / sp.inflow_depth)) : T(0);
    }
    T *box = (it & 1) ? box1 : box0;
    const int nitem = item + G0;
    if (nitem < total) {
      const int ns = slot_of_item(slots, nslots, nitem);
      const int nt = nitem - slots[ns].first_item;
      issue_box<T, TX, TY, NT>(io_of(slots[ns].fd, STAGE), (nt % slots[ns].tiles_x) * TX,
                               (nt / slots[ns].tiles_x) * TY, (it & 1) ? box0 : box1);
    }
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    if (!skip) {
      const int t = item - sl.first_item;
      const int tiles_x = sl.tiles_x;
      const int i0 = (t % tiles_x) * TX, j0 = (t / tiles_x) * TY;
      if (i0 == 0 || j0 == 0 || i0 + TX + 3 > s_io.nx || j0 + TY + 3 > s_io.ny) {
        patch_box<T, TX, TY, NT>(s_io, sp, i0, j0, box, consts<T>(sp).zref, eta_in, u_in);
        __syncthreads();
      }
      tile_compute<T, TX, TY, NT, S, STAGE>(s_io, sp, i0, j0, box, sL, tdt, rcap, alx, aly, acc);
    }
    __syncthreads();
  }
  cp_wait<0>();
  if (cur >= 0 && !skip) publish<T, NT, STAGE>(sp, slots[cur].sc, lead, red, dt, acc);
}

}  // namespace swe
