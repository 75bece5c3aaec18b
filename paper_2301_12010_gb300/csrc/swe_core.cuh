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
//   ghost values (walls / inflow / periodic) patched into the halo box,
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
// Shared-memory plan (per CTA, persistent over its tiles): two halo boxes of
// (ha, hu, hv, b), double-buffered and filled by tensor copies while the
// other tile is computed, and the x-pass result L_x; split fluxes and their
// differences live in registers, in sliding windows along each strip.
#pragma once
#include <cuda.h>  // CUtensorMap (the descriptor type only; no driver calls here)
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace swe {

// BC_HALO (y sides of a strip of a row-partitioned domain): the ghost rows are
// the neighbouring strip's rows, copied into the plane's halo rows before the
// stage (the halo exchange of the paper's per-core partitions).
enum : int { BC_WALL = 0, BC_INFLOW = 1, BC_PERIODIC = 2, BC_HALO = 3 };
enum : unsigned { ST_NONFINITE = 1u, ST_DRY = 2u, ST_TIMEOUT = 4u };

// Slots for per-CTA sums of the clamp and edge volumes: at least the CTAs of
// any persistent launch (resident CTAs x SMs).
constexpr int kPartSlots = 1024;

// Per-CTA running sums of one scenario (device memory, FP64): CTA b adds its
// share of every RK stage to slot b, in time order, and only CTA b touches
// slot b; the host adds the slots in CTA order when it reads the totals.  The
// totals thus do not depend on the order in which CTAs finish (as atomic adds
// would), and no kernel waits for another CTA.
struct DevPartials {
  double clamp[kPartSlots];  // RK-weighted clamp volume (m^3)
  double edge[kPartSlots];   // RK-weighted edge inflow volume (m^3)
};

// Per-scenario device scalars (one struct per handle or batch slot).
struct DevScalars {
  unsigned long long alpha[3][2];   // wave speeds (x, y) per stage slot, bits of a double
  double dt;                        // time step of the running step
  double t;                         // time of U^n
  double t_step;                    // time at the start of the running step
  long long steps;                  // steps taken
  unsigned long long runup_now[2];  // bits of a double, per step parity; 0 = no wet land cell
  unsigned long long runup_max;     // bits of a double; 0 = none
  double clamp_mass;                // unused: the clamp and edge volumes live in the per-CTA slots
  double boundary_mass;             // (DevPartials), which the host adds in CTA order
  double t_end;                     // > 0: last step truncated at t_end; no step once t >= t_end
  double cfl;                       // CFL number when fixed_dt <= 0
  unsigned status;                  // ST_* flags
  unsigned running;                 // 1 while the current step runs (set by stage 1)
  unsigned parity;                  // steps & 1 of the running step
  unsigned active;                  // batch: slot is live
  DevPartials *part;                // this scenario's per-CTA clamp and edge volumes (set by the host)
  unsigned long long check;         // checked build: first index found out of range (see SWE_CHK), 0 = none
};

// Derived constants of the stage arithmetic, precomputed on the host in the
// state's precision (keeps FP64 work out of the FP32 kernels).
template <typename T>
struct Consts {
  T g, zref, eps12;
  T pg;          // sqrt(3)/4 g: pressure factor of the carried split fluxes
  T rfx, rfy;    // 1 / (6 sqrt(3) dx), 1 / (6 sqrt(3) dy): carried flux sums to dF/dx
  T g12dx, g12dy;  // g / (12 dx), g / (12 dy): bed source from 12 bhat differences
  T ewx, ewy;    // dy / (6 sqrt(3)), dx / (6 sqrt(3)): edge flux sums to m^3/s
  T gn2, hf4;
  T sqg;         // sqrt(g)
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
  // derived on the host (FP64 work is slow on the device): 1/dx, 1/dy, the
  // cell area, and the inflow wave's constants (see inflow_eta)
  double rdx, rdy, area;
  double in_c0, in_s0, in_o1, in_o2, in_a1, in_a2, in_k1, in_k2, in_uf;
  // bounded waits for the halo-box copies: give up after wait_cycles SM
  // cycles; copy_extra > 0 (test hook) makes each wait expect bytes that never
  // arrive, so that the timeout path runs
  long long wait_cycles;
  unsigned copy_extra, pad_;
  // checked build: where an out-of-range index is recorded (the scenario's
  // DevScalars::check); nullptr in the normal build
  unsigned long long *check;
  // strips of a row-partitioned domain: the planes carry halo_rows rows above
  // and below (the tensor maps start there), and a follower strip leaves the
  // per-step bookkeeping of the shared device scalars to the lead strip
  // (a strip's edge fluxes through its y sides are not counted: its host sets
  // the y edge weights ewy to zero; the true y edges of a partitioned domain
  // are walls, whose mass flux is zero)
  int halo_rows, follower;
};

constexpr long long kDefaultWaitCycles = 1ll << 31;  // ~1 s at the maximum SM clock

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
  const double s3 = 1.7320508075688772;  // sqrt(3)
  c.eps12 = 12.0 * p.weno_eps;
  c.pg = 0.25 * s3 * p.g;
  c.rfx = 1.0 / (6.0 * s3 * p.dx);
  c.rfy = 1.0 / (6.0 * s3 * p.dy);
  c.g12dx = p.g / (12.0 * p.dx);
  c.g12dy = p.g / (12.0 * p.dy);
  c.ewx = p.dy / (6.0 * s3);
  c.ewy = p.dx / (6.0 * s3);
  c.gn2 = p.g * p.n2;
  c.hf4 = p.hf4;
  c.sqg = std::sqrt(p.g);
  p.c64 = c;
  p.c32 = {(float)c.g,   (float)c.zref,  (float)c.eps12, (float)c.pg,  (float)c.rfx, (float)c.rfy,
           (float)c.g12dx, (float)c.g12dy, (float)c.ewx,  (float)c.ewy, (float)c.gn2, (float)c.hf4,
           (float)c.sqg};
  p.rdx = 1.0 / p.dx;
  p.rdy = 1.0 / p.dy;
  p.area = p.dx * p.dy;
  // carrier N-wave of Eq. (20): c0 = sqrt(g d0), lambda = T c0, a1 = amp/2,
  // a2 = a1/3, k1 = 28.416/lambda^2, k2 = 256/lambda^2, read at
  // s = 1.3 lambda - c0 t, with centres 0.5151125 lambda and 0.2048 lambda;
  // the inflow velocity is eta sqrt(g/d0)
  const double c0 = p.inflow_depth > 0.0 ? std::sqrt(p.g * p.inflow_depth) : 0.0;
  const double lam = p.inflow_period * c0;
  p.in_c0 = c0;
  p.in_s0 = 1.3 * lam;
  p.in_o1 = 0.5151125 * lam;
  p.in_o2 = 0.2048 * lam;
  p.in_a1 = 0.5 * p.inflow_amp;
  p.in_a2 = p.in_a1 / 3.0;
  p.in_k1 = lam > 0.0 ? 28.416 / (lam * lam) : 0.0;
  p.in_k2 = lam > 0.0 ? 256.0 / (lam * lam) : 0.0;
  p.in_uf = p.inflow_depth > 0.0 ? std::sqrt(p.g / p.inflow_depth) : 0.0;
}

// Checked build (compiled with SWE_CHECKED): every index into the shared
// halo box and L_x and into a global plane is compared with its extent before
// the access.  An index out of range is recorded in *p.check -- the first one
// only: bit 63 set, the access site in bits 40..47, the index in bits 0..39 --
// and the access is skipped (a load reads zero).  No trap, no fault: the host
// reads the word (swe_check_status).  In the normal build SWE_CHK is `true`
// and the checks compile out.
#ifdef SWE_CHECKED
__device__ __forceinline__ bool swe_chk(unsigned long long *word, long long i, long long n, unsigned site) {
  if (i >= 0 && i < n) return true;
  if (word)
    atomicCAS(word, 0ull, (1ull << 63) | ((unsigned long long)(site & 0xffu) << 40) |
                              ((unsigned long long)i & 0xffffffffffull));
  return false;
}
#define SWE_CHK(p, i, n, site) swe_chk((p).check, (long long)(i), (long long)(n), (site))
#else
#define SWE_CHK(p, i, n, site) true
#endif
enum : unsigned {  // access sites of the checked build
  CK_PATCH_W = 1, CK_PATCH_MIRROR, CK_PATCH_GLOBAL, CK_CHUNK, CK_CELL, CK_XEPI_BOX, CK_XEPI_L, CK_YEPI_BOX,
  CK_YEPI_L, CK_OUT, CK_U0
};

template <typename T>
struct Field {
  const T *b;
  T *h[3], *hu[3], *hv[3];  // planes of U^n, U1, U2; h[] holds ha = h - d
  int nx, ny, pitch;
  int halo;                 // rows allocated above row 0 and below row ny-1 (a strip's halo rows), else 0
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
  static __device__ __forceinline__ float lg2(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  // |q| / h^(7/3) from |q|^2 and h > 0, as 2^(lg2(q^2)/2 - 7/3 lg2(h))
  // (three hardware approximations; q = 0 gives 2^-inf = 0)
  static __device__ __forceinline__ float fric(float q2, float h) {
    return ex2(fmaf(0.5f, lg2(q2), -2.3333333f * lg2(h)));
  }
  // 1/h and sqrt(g h) from one reciprocal square root (h >= 0; h below
  // 1e-30 is raised to it, which leaves sqrt(g h) at ~0 and 1/h unused)
  static __device__ __forceinline__ void speed(float h, float, float sqg, float &rh, float &cel) {
    const float rs = rsqrt_(h > 1e-30f ? h : 1e-30f);
    rh = rs * rs;
    cel = sqg * (h * rs);
  }
  static __device__ __forceinline__ bool below(float h, float thr32, double) { return h < thr32; }
  static __device__ __forceinline__ float rsqrt_(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
};
// 1/x for positive normal x in FP64 by Newton-Raphson: the hardware seed
// (relative error below 2^-20) and two steps r <- r + r (1 - x r), each of
// which squares the relative error, end within an ulp or two of 1/x, at a
// fraction of the cost of an IEEE division on this part's FP64 pipe.
__device__ __forceinline__ double rcp_newton(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

template <> struct Num<double> {
  static __device__ __forceinline__ double rcp(double x) { return rcp_newton(x); }  // x >= h_dry > 0 at every use
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double fric(double q2, double h) { return sqrt(q2) / (h * h * cbrt(h)); }
  static __device__ __forceinline__ void speed(double h, double g, double, double &rh, double &cel) {
    rh = 1.0 / h;
    cel = sqrt(g * h);
  }
  static __device__ __forceinline__ bool below(double h, float, double thr) { return h < thr; }
  static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
};

// ------------------------------------------ reconstruction value operations
// Overloads for FP32 scalars, packed FP32 pairs (float2: the f32x2 FMA, ADD
// and MUL instructions of sm_100+ issue both lanes in one slot), FP64
// scalars and FP64 pairs (double2, lane by lane).  sp<V>(c) splats a constant.
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vrcp(float a) { return Num<float>::rcp(a); }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vrcp(double a) { return rcp_newton(a); }  // WENO terms: positive normal
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(vrcp(a.x), vrcp(a.y)); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vrcp(double2 a) { return make_double2(rcp_newton(a.x), rcp_newton(a.y)); }
template <typename V> __device__ __forceinline__ V sp(double c);
template <> __device__ __forceinline__ float sp<float>(double c) { return (float)c; }
template <> __device__ __forceinline__ double sp<double>(double c) { return c; }
template <> __device__ __forceinline__ float2 sp<float2>(double c) { return make_float2((float)c, (float)c); }
template <> __device__ __forceinline__ double2 sp<double2>(double c) { return make_double2(c, c); }
template <typename V> __device__ __forceinline__ V vsub(V a, V b) { return vfma(sp<V>(-1.0), b, a); }

template <bool B> struct BoolC { static constexpr bool value = B; };

// Pair type of a precision: components 0 and 1 of a sweep travel together.
template <typename T> struct Pair;
template <> struct Pair<float> {
  using type = float2;
  static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <> struct Pair<double> {
  using type = double2;
  static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};

// ------------------------------------------------------- WENO5 reconstruction
// Fifth-order WENO of Jiang and Shu (Sec. 2) written in first differences.
// For the five upwind values v0..v4 of a face (upwind cell v2) let
// d_j = v_j - v_{j-1}, j = 1..4.  Then
//   12 beta_k = 13 D_k^2 + 3 E_k^2,  D_k = d_{k+2} - d_{k+1},
//   E_0 = d_1 - 3 d_2,  E_1 = d_2 + d_3,  E_2 = d_4 - 3 d_3   (signs irrelevant),
// and the candidate values are 6 p_k = 6 v2 + C_k with
//   C_0 = 5 d_2 - 2 d_1,  C_1 = d_2 + 2 d_3,  C_2 = 4 d_3 - d_4.
// The sweep carries the split fluxes times sqrt(3), so that 3 E_k^2 is the
// square e_k^2 of the same combination of the carried differences and
// 12 (eps + beta_k) = q_k + e_k^2, where q_k = 13/3 D_k^2 + 12 eps is cached
// per stencil centre.  With a_k = 1 / (12 (eps + beta_k))^2 and the linear
// weights gamma = (0.1, 0.6, 0.3), 6 W = 6 v2 + S rdn with
//   S = sum_k gamma_k a_k C_k,  rdn = 1 / sum_k gamma_k a_k.
// A_k = (-0.1 a_0, 0.6 a_1, -0.3 a_2) carry the signs of the forms -C_0 =
// 2 e_0 + d_2, C_1 = e_1 + d_3, -C_2 = e_2 - d_3 and are returned for the bed.
// MIR: the mirrored side (f- reconstructed from the right), whose differences
// arrive in the sweep's order, i.e. negated; S comes out negated and rdn is
// returned negated, so that S rdn is unchanged.  A constant state has all
// d_j = 0 and reconstructs to exactly v2.
//
// FP64 scales the a_k by (t_0 t_1 t_2)^2, t_k = 12 (eps + beta_k), which S rdn
// does not see: a_0 -> t_1^2 t_2^2 etc., one reciprocal (rdn) per side instead
// of four, each an approximation plus two Newton steps on the FP64 pipe
// (+17 % FP64 throughput).  FP32 keeps the four reciprocals: there the
// products cost registers and issue slots that the MUFU pipe does not (-3 %
// measured), and t^4 would also narrow FP32's exponent range.
template <typename V> struct IsF64 { static constexpr bool value = false; };
template <> struct IsF64<double> { static constexpr bool value = true; };
template <> struct IsF64<double2> { static constexpr bool value = true; };

template <bool MIR, typename V>
__device__ __forceinline__ V weno_side(V d1, V d2, V d3, V d4, V q0, V q1, V q2, V &A0, V &A1, V &A2, V &rdn) {
  const V e0 = vfma(sp<V>(-3.0), d2, d1);
  const V e1 = vadd(d2, d3);
  const V e2 = vfma(sp<V>(-3.0), d3, d4);
  if constexpr (IsF64<V>::value) {
    const V t0 = vfma(e0, e0, q0), t1 = vfma(e1, e1, q1), t2 = vfma(e2, e2, q2);
    const V s0 = vmul(t0, t0), s1 = vmul(t1, t1), s2 = vmul(t2, t2);
    A0 = vmul(vmul(s1, sp<V>(-0.1)), s2);
    A1 = vmul(vmul(s0, sp<V>(0.6)), s2);
    A2 = vmul(vmul(s0, sp<V>(-0.3)), s1);
  } else {
    const V r0 = vrcp(vfma(e0, e0, q0));
    const V r1 = vrcp(vfma(e1, e1, q1));
    const V r2 = vrcp(vfma(e2, e2, q2));
    A0 = vmul(vmul(r0, r0), sp<V>(-0.1));
    A1 = vmul(vmul(r1, r1), sp<V>(0.6));
    A2 = vmul(vmul(r2, r2), sp<V>(-0.3));
  }
  rdn = vrcp(MIR ? vadd(vsub(A0, A1), A2) : vsub(vsub(A1, A0), A2));
  const V c0 = vfma(sp<V>(2.0), e0, d2);
  const V c1 = vadd(e1, d3);
  const V c2 = vsub(e2, d3);
  return vfma(A2, c2, vfma(A1, c1, vmul(A0, c0)));
}

// The same weighted sum for other values (the bed) under given weights A_k.
template <typename V>
__device__ __forceinline__ V weighted_side(V d1, V d2, V d3, V d4, V A0, V A1, V A2) {
  const V c0 = vfma(sp<V>(-5.0), d2, vmul(sp<V>(2.0), d1));  // -C_0
  const V c1 = vfma(sp<V>(2.0), d3, d2);                      //  C_1
  const V c2 = vfma(sp<V>(-4.0), d3, d4);                     // -C_2
  return vfma(A2, c2, vfma(A1, c1, vmul(A0, c0)));
}

// q = 13/3 D^2 + 12 eps of the stencil centred between differences a and b.
template <typename V>
__device__ __forceinline__ V qterm(V a, V b, V eps12) {
  const V D = vsub(b, a);
  return vfma(vmul(sp<V>(13.0 / 3.0), D), D, eps12);
}

// Carrier N-wave of Eq. (20) entering through the x- edge, with the constants
// of finish_phys: eta = 2 (a1 exp(-k1 q1^2) - a2 exp(-k2 q2^2)), q = s - centre,
// s = 1.3 lambda - c0 t.  The phase is taken in FP64 (t is large); the
// exponentials in the state's precision.
template <typename T> __device__ __forceinline__ T inflow_eta(const Phys &p, double t);
template <>
__device__ __forceinline__ double inflow_eta<double>(const Phys &p, double t) {
  const double s = p.in_s0 - p.in_c0 * t;
  const double q1 = s - p.in_o1, q2 = s - p.in_o2;
  return 2.0 * (p.in_a1 * exp(-p.in_k1 * q1 * q1) - p.in_a2 * exp(-p.in_k2 * q2 * q2));
}
template <>
__device__ __forceinline__ float inflow_eta<float>(const Phys &p, double t) {
  const double s = p.in_s0 - p.in_c0 * t;
  const double q1 = s - p.in_o1, q2 = s - p.in_o2;
  return 2.f * ((float)p.in_a1 * expf((float)(-p.in_k1 * q1 * q1)) -
                (float)p.in_a2 * expf((float)(-p.in_k2 * q2 * q2)));
}

template <typename T>
__device__ __forceinline__ T still_depth(T b, T zref) {
  T d = zref - b;
  return d > T(0) ? d : T(0);
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------- tensor copies (TMA) + mbarrier
// The single-scenario stage kernels load each tile's halo box with one 2D
// tensor copy per field (box P x BH at (i0 - 4, j0 - 3); elements outside the
// plane read as zero), completing on an mbarrier of the destination buffer.
struct BoxMaps {
  CUtensorMap m[4];  // ha, hu, hv, b of the stage input
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes));
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Bounded wait for phase `parity` of bar: false if it did not complete within
// `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory geometry of one tile.  The halo box covers columns
// i0-4 .. i0+TX+3 (OX = 4: a 16-byte aligned start for the chunked copies;
// the stencils read i0-3 .. i0+TX+2) and rows j0-3 .. j0+TY+2 (OY = 3).
template <typename T, int TX, int TY>
struct TileGeom {
  static constexpr int OX = 4, OY = 3;
  static constexpr int BW = TX + 8;  // halo box width
  static constexpr int BH = TY + 6;  // halo box height
  static constexpr int CH = 16 / (int)sizeof(T);  // elements per 16-byte chunk
  // row pitch: 16-byte rows; FP32: P/4 odd, so that the x-pass 16-byte window
  // loads of a quarter-warp (2 rows x 4 strips of 8, or 4 rows x 2 strips of
  // 16) fall in distinct bank groups; FP64: P = 2 mod 8 (2-way at most for the
  // scalar x-pass loads)
  static constexpr int P = sizeof(T) == 4 ? ((((BW + 3) / 4) % 2) ? (BW + 3) / 4 * 4 : (BW + 3) / 4 * 4 + 4)
                                          : ((BW + 1) / 2 * 2 + ((10 - (BW + 1) / 2 * 2 % 8) % 8));
  static constexpr int FA = 128 / (int)sizeof(T);  // 128-byte alignment of each field (tensor copies)
  static constexpr int FIELD = (BH * P + FA - 1) / FA * FA;  // one field of the box
  static constexpr int BOX = 4 * FIELD; // ha, hu, hv, b
  static constexpr int LP = TX + 1;        // L_x row pitch (x-pass lanes on 8 rows hit distinct banks)
  static constexpr int NC = TY * LP;       // one L_x component
  static constexpr int ELEMS = 2 * BOX + 3 * NC;  // two boxes (double buffer) + L_x
  static constexpr size_t BYTES = sizeof(T) * (size_t)ELEMS;
  static_assert(TX % 4 == 0 && P % CH == 0 && P >= BW, "16-byte aligned box rows");
};

// Per-stage values broadcast from thread 0 to the CTA, in both precisions.
enum { SV_DT = 0, SV_RCAP, SV_AX, SV_AY, SV_ETA, SV_UIN, SV_N };

// Reduction scratch and broadcast values in shared memory (per CTA).
struct RedSmem {
  float wf[32][5];    // per-warp partials, FP32 kernels: alpha_x, alpha_y, deficit, edge flux, runup
  double wd[32][5];   // the same, FP64 kernels
  double dt;          // time step of the running RK step
  float v32[SV_N];    // dt, 1/dt, alpha_x, alpha_y, inflow eta, inflow u
  double v64[SV_N];
  unsigned bad;
  unsigned skip;
};
template <typename T> __device__ __forceinline__ T *red_w(RedSmem &r);
template <> __device__ __forceinline__ float *red_w<float>(RedSmem &r) { return &r.wf[0][0]; }
template <> __device__ __forceinline__ double *red_w<double>(RedSmem &r) { return &r.wd[0][0]; }
template <typename T> __device__ __forceinline__ T red_v(const RedSmem &r, int k);
template <> __device__ __forceinline__ float red_v<float>(const RedSmem &r, int k) { return r.v32[k]; }
template <> __device__ __forceinline__ double red_v<double>(const RedSmem &r, int k) { return r.v64[k]; }

// The state planes a stage reads and writes.
template <typename T>
struct StageIO {
  const T *b;
  const T *ha, *hu, *hv;     // stage input (halo reads)
  const T *ha0, *hu0, *hv0;  // U^n (own cells, stages 2 and 3)
  T *oha, *ohu, *ohv;        // stage output
  int nx, ny, pitch;
};

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
    const int i = i0 - G::OX + c, j = j0 - G::OY + r;
    const bool in_i = i >= 0 && i < nx, in_j = j >= 0 && j < ny;
    if (in_i && in_j) continue;  // a real cell, already loaded
    const int o = r * G::P + c;
    if (!SWE_CHK(p, o, G::FIELD, CK_PATCH_W)) continue;
    const bool xg = !in_i && in_j && i >= -3 && i < nx + 3;  // x ghost
    const bool yg = in_i && !in_j && j >= -3 && j < ny + 3;  // y ghost
    if (yg && p.bc[j < 0 ? 2 : 3] == BC_HALO) continue;      // the neighbour's rows, loaded with the box
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
      if (!SWE_CHK(p, go, (long long)io.ny * io.pitch, CK_PATCH_GLOBAL)) continue;
      // through L2: in the batch kernel other CTAs wrote these planes earlier
      // in the same launch, and an SM's L1 is not refreshed within a launch
      const T bs = __ldcg(io.b + go), cb = bs + shift;
      bb[o] = cb;
      bha[o] = (__ldcg(io.ha + go) + still_depth(bs, zref)) - still_depth(cb, zref);
      bhu[o] = __ldcg(io.hu + go);
      bhv[o] = __ldcg(io.hv + go);
      continue;
    }
    // mirror source: a real cell of the same box
    int mc = c, mr = r;
    if (xg) mc = (i < 0 ? (-1 - i) : (2 * nx - 1 - i)) - (i0 - G::OX);
    else mr = (j < 0 ? (-1 - j) : (2 * ny - 1 - j)) - (j0 - G::OY);
    const int m = mr * G::P + mc;
    if (!SWE_CHK(p, m, G::FIELD, CK_PATCH_MIRROR)) continue;
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

// Sliding window of one strip, in the frame of the sweep.  For face k, which
// lies between window slots 2 and 3 (cells c0-1+k and c0+k), it holds for each
// carried value (split fluxes f+ and f- times sqrt 3, and the bed) the
// differences d[s] = v(slot s) - v(slot s-1), s = 1..5, the second-difference
// terms q[s] centred at slots 1..4, and the value last put (slot 5).
// Components 0 and 1 (mass and normal momentum) travel as pairs, component 2
// (tangential momentum) and the bed as scalars.
//
// With the face sums Fs(k) = 6 sqrt(3) Fhat(k) = 6 (f+(2) + f-(3)) + X(k)
// (X: the WENO corrections of both sides), the difference over the cell at
// slot 2 is Fs(k) - Fs(k-1) = 6 (d+[2] + d-[3]) + X(k) - X(k-1); for the bed,
// 12 bhat(k) - 12 bhat(k-1) = 6 (db[2] + db[3]) + Xb(k) - Xb(k-1).
template <typename T>
struct Window {
  using V2 = typename Pair<T>::type;
  V2 lp01, lm01;
  T lp2, lm2, lb;
  V2 dp01[6], dm01[6];
  T dp2[6], dm2[6], db[6];
  V2 qp01[5], qm01[5];
  T qp2[5], qm2[5];
  V2 xp01;  // X of the previous face
  T xp2, xb;

  // Put the cell at box offset o into slot s.  sa = sqrt(3)/2 alpha,
  // pg = sqrt(3)/4 g: with h = ha + d and pressure g ha (h + d)/2,
  //   F = (qn, qn un + pressure, qt un),  Q = (ha, qn, qt),
  //   f+- = (F +- alpha Q)/2   (carried times sqrt 3),
  // i.e. F of Eq. (2) in x and G of Eq. (3), momentum components swapped, in y.
  template <int s>
  __device__ __forceinline__ void put(T ha, T qn, T qt, T b, T sa, T pg, T zref, V2 eps2, T eps1, const Phys &p) {
    const T d = still_depth(b, zref);
    const T h = ha + d;
    T un = T(0);
    if (!Num<T>::below(h, p.h_dry32, p.h_dry)) un = qn * Num<T>::rcp(h);
    const T f0 = T(0.8660254037844386) * qn;  // sqrt(3)/2 qn
    const T f1 = fma(f0, un, pg * ha * (h + d));
    const T f2 = (T(0.8660254037844386) * qt) * un;
    const V2 F = Pair<T>::mk(f0, f1), Q = Pair<T>::mk(ha, qn);
    const V2 up = vfma(Pair<T>::mk(sa, sa), Q, F), um = vfma(Pair<T>::mk(-sa, -sa), Q, F);
    const T up2 = fma(sa, qt, f2), um2 = fma(-sa, qt, f2);
    if constexpr (s >= 1) {
      dp01[s] = vsub(up, lp01);
      dm01[s] = vsub(um, lm01);
      dp2[s] = up2 - lp2;
      dm2[s] = um2 - lm2;
      db[s] = b - lb;
      if constexpr (s >= 2) {
        qp01[s - 1] = qterm(dp01[s - 1], dp01[s], eps2);
        qm01[s - 1] = qterm(dm01[s - 1], dm01[s], eps2);
        qp2[s - 1] = qterm(dp2[s - 1], dp2[s], eps1);
        qm2[s - 1] = qterm(dm2[s - 1], dm2[s], eps1);
      }
    }
    lp01 = up;
    lm01 = um;
    lp2 = up2;
    lm2 = um2;
    lb = b;
  }

  // WENO corrections X of face k for components 0-1, 2 and the bed (the bed
  // with the weights of component 1, the second lane).
  __device__ __forceinline__ void face(V2 &x01, T &x2, T &x3) const {
    V2 A0, A1, A2, rp, B0, B1, B2, rm;
    const V2 Sp = weno_side<false>(dp01[1], dp01[2], dp01[3], dp01[4], qp01[1], qp01[2], qp01[3], A0, A1, A2, rp);
    const V2 Sm = weno_side<true>(dm01[5], dm01[4], dm01[3], dm01[2], qm01[4], qm01[3], qm01[2], B0, B1, B2, rm);
    x01 = vfma(Sm, rm, vmul(Sp, rp));
    const T Bp = weighted_side<T>(db[1], db[2], db[3], db[4], A0.y, A1.y, A2.y);
    const T Bm = weighted_side<T>(db[5], db[4], db[3], db[2], B0.y, B1.y, B2.y);
    x3 = fma(Bm, rm.y, Bp * rp.y);
    T a0, a1, a2, r2p, b0, b1, b2, r2m;
    const T Gp = weno_side<false>(dp2[1], dp2[2], dp2[3], dp2[4], qp2[1], qp2[2], qp2[3], a0, a1, a2, r2p);
    const T Gm = weno_side<true>(dm2[5], dm2[4], dm2[3], dm2[2], qm2[4], qm2[3], qm2[2], b0, b1, b2, r2m);
    x2 = fma(Gm, r2m, Gp * r2p);
  }

  // Fs(k) of component 0 (mass flux times 6 sqrt 3), for the domain edges.
  __device__ __forceinline__ T edge_flux(V2 x01) const {
    const T fp = lp01.x - dp01[5].x - dp01[4].x - dp01[3].x;  // f+ at slot 2
    const T fm = lm01.x - dm01[5].x - dm01[4].x;              // f- at slot 3
    return fma(T(6), fp + fm, x01.x);
  }

  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int q = 1; q < 5; ++q) {
      dp01[q] = dp01[q + 1];
      dm01[q] = dm01[q + 1];
      dp2[q] = dp2[q + 1];
      dm2[q] = dm2[q + 1];
      db[q] = db[q + 1];
    }
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      qp01[q] = qp01[q + 1];
      qm01[q] = qm01[q + 1];
      qp2[q] = qp2[q + 1];
      qm2[q] = qm2[q + 1];
    }
  }
};

// One strip: faces k = 0..S (face k at the left of strip cell k).  As soon as
// both faces of strip cell k are known, emit(k, dF0, dF1, dF2, db) receives
// dF_c = Fs_c(k+1) - Fs_c(k) (flux differences times 6 sqrt 3) and
// db = 12 (bhat(k+1) - bhat(k)).  Adds ew times the mass flux sum Fs_0
// through the domain edges that the strip owns (face -1/2 at k = 0 of the
// first strip, face n-1/2 at k >= 1).
//
// SHORE (the shoreline variant): a face whose six window cells hold a dry
// cell takes the first-order hydrostatic reconstruction (Audusse et al.,
// 2004) instead of the WENO values: face bed b_f = max(b_L, b_R), face depths
// h*_s = max(0, h_s + b_s - b_f), the global-LF flux of the standard SWE flux
// of those states with this line's alpha; each side s sees the normal
// momentum flux raised by g (h_s^2 - h*_s^2 - d_s^2)/2 and the bed value b_s
// (the cell update then adds g (h_s - d_s) b_s), which puts a lake at rest
// beside dry land in balance at any level at or below z_ref.  The face values
// enter the differences as corrections to the WENO values of the face.
template <typename T>
struct ShoreFace {
  T f0, f2;    // 6 sqrt(3) F_0, 6 sqrt(3) F_2 of the face (both sides)
  T f1l, f1r;  // 6 sqrt(3) of the normal-momentum flux as the left and the right cell see it
  T bl, br;    // 12 b_L, 12 b_R
};
struct ChkWord {
  unsigned long long *check;
};

// The hydrostatic-reconstruction values of the face between box cells oL and
// oL + st (SHORE, see sweep_strip), out of line: only faces next to dry cells
// take it, and one copy keeps the sweeps' unrolled face bodies small enough
// for the instruction cache.
template <typename T>
__device__ __noinline__ ShoreFace<T> shore_face(const T *bha, const T *bqn, const T *bqt, const T *bb, int oL, int st,
                                                int field, T alpha, T g, T zref, float thr32, double thr,
                                                unsigned long long *check) {
  const ChkWord ck{check};
  (void)ck;
  (void)field;
  T ha_[2], qn_[2], qt_[2], b_[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int o = oL + s * st;
    const bool ok = SWE_CHK(ck, o, field, CK_CELL);
    ha_[s] = ok ? bha[o] : T(0);
    qn_[s] = ok ? bqn[o] : T(0);
    qt_[s] = ok ? bqt[o] : T(0);
    b_[s] = ok ? bb[o] : T(0);
  }
  const T bL = b_[0], bR = b_[1];
  const T dL = still_depth(bL, zref), dR = still_depth(bR, zref);
  const T hL = ha_[0] + dL, hR = ha_[1] + dR;
  T uL = T(0), vL = T(0), uR = T(0), vR = T(0);
  if (!Num<T>::below(hL, thr32, thr)) { uL = qn_[0] / hL; vL = qt_[0] / hL; }
  if (!Num<T>::below(hR, thr32, thr)) { uR = qn_[1] / hR; vR = qt_[1] / hR; }
  const T bf = bL > bR ? bL : bR;
  T sL = hL + (bL - bf), sR = hR + (bR - bf);  // bed difference first: films keep their digits
  sL = sL > T(0) ? sL : T(0);
  sR = sR > T(0) ? sR : T(0);
  const T g2 = T(0.5) * g, ah = T(0.5) * alpha;
  const T qL = sL * uL, qR = sR * uR;
  const T F0 = T(0.5) * (qL + qR) - ah * (sR - sL);
  const T F1 = T(0.5) * (qL * uL + g2 * sL * sL + qR * uR + g2 * sR * sR) - ah * (qR - qL);
  const T F2 = T(0.5) * (qL * vL + qR * vR) - ah * (sR * vR - sL * vL);
  const T c6 = T(10.392304845413264);  // 6 sqrt 3
  ShoreFace<T> r;
  r.f0 = c6 * F0;
  r.f2 = c6 * F2;
  r.f1l = c6 * (F1 + g2 * (hL * hL - sL * sL - dL * dL));
  r.f1r = c6 * (F1 + g2 * (hR * hR - sR * sR - dR * dR));
  r.bl = T(12) * bL;
  r.br = T(12) * bR;
  return r;
}

template <typename T, int S, bool XP, int FIELD, typename E, bool SHORE = false>
__device__ __forceinline__ void sweep_strip(const T *bha, const T *bqn, const T *bqt, const T *bb, int o0, int st,
                                            T alpha, const Consts<T> &K, const Phys &p, int ia, int n, bool edge_ok,
                                            T ew, const E &emit, T &edge) {
  using V2 = typename Pair<T>::type;
  Window<T> win;
  const T sa = T(0.8660254037844386) * alpha, pg = K.pg, zref = K.zref, eps1 = K.eps12;
  const V2 eps2 = Pair<T>::mk(eps1, eps1);
  // Window slot q is box offset o0 + q st.  FP32 x pass: the slots lie along
  // one box row and o0 - 1 is 16-byte aligned, so slot q is element (q+1) % 4
  // of the 16-byte chunk (q+1) / 4 of each field, loaded once before its first
  // use (four fields per chunk).
  constexpr bool VEC = XP && sizeof(T) == 4;
  constexpr int NCH = (S + 9) / 4;
  float4 ch[4][NCH];
  auto cell = [&](int q, T &ha, T &qn, T &qt, T &b) {
    if constexpr (VEC) {
      const int m = (q + 1) >> 2, e = (q + 1) & 3;
      if (q == 0 || e == 0) {
        const int c0 = o0 - 1 + 4 * m;
        if (SWE_CHK(p, c0, FIELD - 3, CK_CHUNK)) {
          ch[0][m] = *reinterpret_cast<const float4 *>(bha + c0);
          ch[1][m] = *reinterpret_cast<const float4 *>(bqn + c0);
          ch[2][m] = *reinterpret_cast<const float4 *>(bqt + c0);
          ch[3][m] = *reinterpret_cast<const float4 *>(bb + c0);
        } else {
          ch[0][m] = ch[1][m] = ch[2][m] = ch[3][m] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      const auto pick = [e](const float4 &v) { return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w)); };
      ha = pick(ch[0][m]);
      qn = pick(ch[1][m]);
      qt = pick(ch[2][m]);
      b = pick(ch[3][m]);
    } else {
      const int o = o0 + q * st;
      const bool ok = SWE_CHK(p, o, FIELD, CK_CELL);
      ha = ok ? bha[o] : T(0);
      qn = ok ? bqn[o] : T(0);
      qt = ok ? bqt[o] : T(0);
      b = ok ? bb[o] : T(0);
    }
  };
  // SHORE: bit s of `dry` flags window slot s as dry; (c0, c1, c2, cb) the
  // corrections of the previous face as its right-hand cell sees them
  unsigned dry = 0u;
  T r0 = T(0), r1 = T(0), r2 = T(0), rb = T(0);
  auto note = [&](T ha_, T b_) {
    if constexpr (SHORE)
      dry = (dry >> 1) | (Num<T>::below(ha_ + still_depth(b_, zref), p.h_dry32, p.h_dry) ? 32u : 0u);
  };
  T ha, qn, qt, b;
  cell(0, ha, qn, qt, b);
  note(ha, b);
  win.template put<0>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
  cell(1, ha, qn, qt, b);
  note(ha, b);
  win.template put<1>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
  cell(2, ha, qn, qt, b);
  note(ha, b);
  win.template put<2>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
  cell(3, ha, qn, qt, b);
  note(ha, b);
  win.template put<3>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
  cell(4, ha, qn, qt, b);
  note(ha, b);
  win.template put<4>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
#pragma unroll
  for (int k = 0; k <= S; ++k) {
    cell(k + 5, ha, qn, qt, b);
    note(ha, b);
    win.template put<5>(ha, qn, qt, b, sa, pg, zref, eps2, eps1, p);
    V2 x01;
    T x2, x3;
    // corrections of this face as its left (l*) and right (r*) cells see them
    T l0 = T(0), l1 = T(0), l2 = T(0), lb = T(0), n0 = T(0), n1 = T(0), n2 = T(0), nb = T(0);
    bool hr = false;
    if constexpr (SHORE) hr = (dry & 63u) != 0u;
    if (!hr) {
      win.face(x01, x2, x3);
    } else {
      // the WENO corrections X of a face that the hydrostatic values replace
      // cancel from the cells' differences whatever they are: zero
      x01 = sp<V2>(0.0);
      x2 = x3 = T(0);
    }
    if constexpr (SHORE) {
      if (hr) {
        const ShoreFace<T> f = shore_face<T>(bha, bqn, bqt, bb, o0 + (k + 2) * st, st, FIELD, alpha, K.g, zref,
                                             p.h_dry32, p.h_dry, p.check);
        // the WENO values of this face, carried: Fs_c = 6 (f+_c(2) + f-_c(3)) + X_c
        const V2 fp2 = vsub(vsub(vsub(win.lp01, win.dp01[5]), win.dp01[4]), win.dp01[3]);
        const V2 fm3 = vsub(vsub(win.lm01, win.dm01[5]), win.dm01[4]);
        const V2 w01 = vfma(sp<V2>(6.0), vadd(fp2, fm3), x01);
        const T w2 = fma(T(6), (win.lp2 - win.dp2[5] - win.dp2[4] - win.dp2[3]) + (win.lm2 - win.dm2[5] - win.dm2[4]),
                         x2);
        const T wb = fma(T(6), (win.lb - win.db[5] - win.db[4] - win.db[3]) + (win.lb - win.db[5] - win.db[4]), x3);
        l0 = n0 = f.f0 - w01.x;
        l2 = n2 = f.f2 - w2;
        l1 = f.f1l - w01.y;
        n1 = f.f1r - w01.y;
        lb = f.bl - wb;
        nb = f.br - wb;
      }
    }
    if (edge_ok && ((k == 0 && ia == 0) || (k > 0 && ia + k == n))) {
      T fs = win.edge_flux(x01);
      if constexpr (SHORE) fs += l0;  // the face's mass flux, either form
      const T fe = fs * ew;
      edge += (k == 0) ? fe : -fe;
    }
    if (k > 0) {
      V2 d01 = vfma(sp<V2>(6.0), vadd(win.dp01[2], win.dm01[3]), vsub(x01, win.xp01));
      T d2 = fma(T(6), win.dp2[2] + win.dm2[3], x2 - win.xp2);
      T dbk = fma(T(6), win.db[2] + win.db[3], x3 - win.xb);
      if constexpr (SHORE) {
        d01.x += l0 - r0;
        d01.y += l1 - r1;
        d2 += l2 - r2;
        dbk += lb - rb;
      }
      emit(k - 1, d01.x, d01.y, d2, dbk);
    }
    if constexpr (SHORE) {
      r0 = n0;
      r1 = n1;
      r2 = n2;
      rb = nb;
    }
    (void)hr;
    win.xp01 = x01;
    win.xp2 = x2;
    win.xb = x3;
    win.shift();
  }
}

// Per-CTA accumulators carried across the tiles of one launch.
template <typename T>
struct Acc {
  T ax = T(0), ay = T(0), ru = T(0), chk = T(0);
  T deficit = T(0), edge = T(0);  // diagnostics, summed in the state's precision per thread
};

// Per-cell work of a pass, done as soon as both faces of the cell are known.
// x pass: store L_x = -dF/dx (+ the bed source of the x momentum).  y pass
// (dF1 is hv, dF2 hu in the y frame): add L_y and the sources, combine the RK
// stage, apply the post-stage rule, write the cell and accumulate the wave
// speeds and diagnostics.
template <typename T, int TX, int TY, int S, int STAGE>
struct CellEpilogue {
  using G = TileGeom<T, TX, TY>;
  const StageIO<T> &io;
  const Phys &p;
  const Consts<T> &K;
  const T *box;
  T *sL;
  bool X;
  int xr, xc0, yc, yr0, i, j0;
  T tdt, rcap, wrk;
  bool friction;  // Manning n > 0
  const T (&u0)[3][S];
  Acc<T> &acc;
  int stage_rt;  // the stage when STAGE is 0 (given at run time)

  __device__ __forceinline__ void operator()(int k, T dF0, T dF1, T dF2, T dbk) const {
    const int st = STAGE ? STAGE : stage_rt;
    const T *bha = box, *bhu = box + G::FIELD, *bhv = box + 2 * G::FIELD, *bb = box + 3 * G::FIELD;
    if (X) {
      const int o = xr * G::LP + xc0 + k;
      const int hb = (xr + G::OY) * G::P + xc0 + k + G::OX;
      const T ha = SWE_CHK(p, hb, G::FIELD, CK_XEPI_BOX) ? bha[hb] : T(0);
      if (!SWE_CHK(p, o, G::NC, CK_XEPI_L)) return;
      sL[o] = -dF0 * K.rfx;
      sL[G::NC + o] = -dF1 * K.rfx - K.g12dx * ha * dbk;
      sL[2 * G::NC + o] = -dF2 * K.rfx;
      return;
    }
    const int j = j0 + yr0 + k;
    if (i >= io.nx || j >= io.ny) return;
    const int o = (yr0 + k) * G::LP + yc;
    const int bo = (yr0 + k + G::OY) * G::P + yc + G::OX;
    if (!SWE_CHK(p, bo, G::FIELD, CK_YEPI_BOX) || !SWE_CHK(p, o, G::NC, CK_YEPI_L)) return;
    const T ha = bha[bo], hu = bhu[bo], hv = bhv[bo], bc = bb[bo];
    const T d = still_depth(bc, K.zref);
    const T h = ha + d;
    T Lh = sL[o] - dF0 * K.rfy;
    T Lhu = sL[G::NC + o] - dF2 * K.rfy;
    T Lhv = sL[2 * G::NC + o] - dF1 * K.rfy - K.g12dy * ha * dbk;
    if (friction && !Num<T>::below(h, p.h_dry32, p.h_dry)) {
      T kap = K.gn2 * Num<T>::fric(hu * hu + hv * hv, h);
      kap = kap > rcap ? rcap : kap;  // rcap = 1/dt
      Lhu -= kap * hu;
      Lhv -= kap * hv;
    }
    T nha = ha + tdt * Lh, nhu = hu + tdt * Lhu, nhv = hv + tdt * Lhv;
    const size_t go = (size_t)j * io.pitch + i;
    if (!SWE_CHK(p, go, (long long)io.ny * io.pitch, CK_OUT)) return;
    if (st != 1) {
      nha = u0[0][k] + wrk * (nha - u0[0][k]);
      nhu = u0[1][k] + wrk * (nhu - u0[1][k]);
      nhv = u0[2][k] + wrk * (nhv - u0[2][k]);
    }
    if (nha < -d) { acc.deficit -= nha + d; nha = -d; }
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
    io.oha[go] = nha;
    io.ohu[go] = nhu;
    io.ohv[go] = nhv;
    const T sx = fabs(u) + cel, sy = fabs(v) + cel;
    acc.chk += sx + sy;  // non-finite values propagate to the per-CTA check
    acc.ax = sx > acc.ax ? sx : acc.ax;
    acc.ay = sy > acc.ay ? sy : acc.ay;
    if (st == 3 && !Num<T>::below(nh, p.h_wet32, p.h_wet) && bc > T(0)) {
      const T e = nh + bc;
      acc.ru = e > acc.ru ? e : acc.ru;
    }
  }
};

// One RK3 stage (Eq. (8), Shu-Osher form, increment form) on one tile whose
// halo box is resident in shared memory:
//   stage 1: U1 = U^n + dt L(U^n)
//   stage 2: U2 = U^n + 1/4 (U1 + dt L(U1) - U^n)
//   stage 3: U^{n+1} = U^n + 2/3 (U2 + dt L(U2) - U^n)   (written over U^n)
// followed by the post-stage rule, with L of Eq. (7).  Pass 0 sweeps x and
// stores L_x; pass 1 sweeps y, adds L_y and the sources and updates.  The
// pass loop is unrolled, so each pass runs code specialised for its frame.
template <typename T, int TX, int TY, int NT, int S, int STAGE, bool SHORE = false>
__device__ __forceinline__ void tile_compute(const StageIO<T> &io, const Phys &p, int i0, int j0, const T *box,
                                             T *sL, T tdt, T rcap, T alx, T aly, Acc<T> &acc, int stage_rt = 0) {
  const int st = STAGE ? STAGE : stage_rt;  // STAGE 0: the stage is given at run time
  using G = TileGeom<T, TX, TY>;
  static_assert(TX % S == 0 && TY % S == 0, "strip length must divide the tile");
  static_assert((TX / S) * TY == NT && (TY / S) * TX == NT, "one strip per thread in both passes");
  // x pass: a warp covers RW rows x SW strips (8 rows x 4 strips of 8 cells, or
  // 16 rows x 2 strips of 16 cells); with the box row pitch P/4 odd, the
  // 16-byte window loads of each quarter-warp fall in distinct bank groups
  constexpr int SW = (S >= 16) ? 2 : 4, RW = 32 / SW;
  static_assert(TY % RW == 0 && (TX / S) % SW == 0 && (TY / RW) * ((TX / S) / SW) == NT / 32,
                "x-pass warps tile the rows and strips");
  const int tid = threadIdx.x;
  const int nx = io.nx, ny = io.ny;
  const T *bha = box, *bhu = box + G::FIELD, *bhv = box + 2 * G::FIELD, *bb = box + 3 * G::FIELD;
  const Consts<T> &K = consts<T>(p);
  // x pass: lane l of warp w takes row RW*(w % (TY/RW)) + l/SW and strip SW*(w / (TY/RW)) + l%SW
  const int w = tid >> 5, l = tid & 31;
  const int xr = RW * (w % (TY / RW)) + l / SW;
  const int xc0 = (SW * (w / (TY / RW)) + l % SW) * S;
  // y pass: thread takes column tid % TX and strip tid / TX
  const int yc = tid % TX, yr0 = (tid / TX) * S;
  const int i = i0 + yc;

  const T wrk = (st == 2) ? T(0.25) : T(2.0 / 3.0);
  const bool friction = K.gn2 > T(0);  // FP32 compare (g n^2 > 0 iff n > 0)
  // one body per pass, specialised at compile time (X: the x pass)
  auto pass = [&](auto xflag) {
    constexpr bool X = decltype(xflag)::value;
    // U^n of the y-pass cells (stages 2, 3), fetched before the sweep so that
    // the global-memory latency hides behind it
    T u0[3][S];
    if (st != 1 && !X) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const int j = j0 + yr0 + k;
        const bool ok = i < nx && j < ny && SWE_CHK(p, (size_t)j * io.pitch + i, (long long)ny * io.pitch, CK_U0);
        const size_t go = ok ? (size_t)j * io.pitch + i : 0;
        // through L2 (the batch kernel's U^n was written by other CTAs in
        // an earlier step of the same launch; L1 is not refreshed within it)
        u0[0][k] = ok ? __ldcg(io.ha0 + go) : T(0);
        u0[1][k] = ok ? __ldcg(io.hu0 + go) : T(0);
        u0[2][k] = ok ? __ldcg(io.hv0 + go) : T(0);
      }
    }
    const CellEpilogue<T, TX, TY, S, STAGE> emit{io, p, K, box, sL, X, xr, xc0, yc, yr0, i, j0, tdt, rcap, wrk, friction, u0, acc, st};
    sweep_strip<T, S, X, G::FIELD, CellEpilogue<T, TX, TY, S, STAGE>, SHORE>(bha, X ? bhu : bhv, X ? bhv : bhu, bb,
                         X ? (xr + G::OY) * G::P + xc0 + G::OX - 3 : yr0 * G::P + yc + G::OX,
                         X ? 1 : G::P, X ? alx : aly, K, p, X ? i0 + xc0 : j0 + yr0, X ? nx : ny,
                         X ? (j0 + xr < ny) : (i < nx), X ? K.ewx : K.ewy, emit, acc.edge);
  };
  pass(BoolC<true>{});
  __syncthreads();
  pass(BoolC<false>{});
}

// Per-stage scalars and the skip decision, taken by thread 0 of every CTA;
// the lead CTA of a scenario also does the per-step bookkeeping.  Stage s
// reads the wave speeds of its input from slot s-1, publishes those of its
// output to slot s mod 3 and clears slot (s+1) mod 3, which nothing reads or
// writes during stage s.
template <typename T, int STAGE>
__device__ __forceinline__ void stage_scalars(const Phys &p, DevScalars *sc, bool lead, RedSmem &red,
                                              int stage_rt = 0) {
  const int st = STAGE ? STAGE : stage_rt;  // STAGE 0: the stage is given at run time
  double ax, ay;
  // read through L2 (other CTAs wrote these before the last grid barrier or launch)
  ax = bitsd(__ldcg(&sc->alpha[st - 1][0]));
  ay = bitsd(__ldcg(&sc->alpha[st - 1][1]));
  const double t_now = __ldcg(&sc->t), t_end = __ldcg(&sc->t_end);
  double dt = 0.0;
  unsigned skip = __ldcg(&sc->status) != 0u;
  if (st == 1) {
    if (t_end > 0.0 && t_now >= t_end) skip = 1;
    if (p.fixed_dt > 0.0) dt = p.fixed_dt;
    else {
      const double den = ax * p.rdx + ay * p.rdy;
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
      sc->alpha[st == 2 ? 0 : 1][0] = 0ull;
      sc->alpha[st == 2 ? 0 : 1][1] = 0ull;
    }
  }
  red.skip = skip;
  red.bad = 0u;
  red.dt = dt;
  const double tst = (st == 1) ? t_now : __ldcg(&sc->t_step);
  const double ts = (st == 1) ? tst : (st == 2 ? tst + dt : tst + 0.5 * dt);
  const bool inflow = p.bc[0] == BC_INFLOW;
  const T eta = inflow ? inflow_eta<T>(p, ts) : T(0);
  const T v[SV_N] = {T(dt), dt > 0.0 ? T(1) / T(dt) : T(0), T(ax), T(ay), eta, inflow ? eta * T(p.in_uf) : T(0)};
#pragma unroll
  for (int k = 0; k < SV_N; ++k) {
    red.v32[k] = (float)v[k];
    red.v64[k] = (double)v[k];
  }
  red.v64[SV_DT] = dt;
  red.v64[SV_AX] = ax;
  red.v64[SV_AY] = ay;
}

// Block reduction of the per-thread accumulators and device-scope
// publication for one scenario.
template <typename T, int NT, int STAGE>
__device__ __noinline__ void publish(const Phys &p, DevScalars *sc, bool lead, RedSmem &red, double dt,
                                     const Acc<T> &acc, int stage_rt = 0) {
  const int st = STAGE ? STAGE : stage_rt;  // STAGE 0: the stage is given at run time
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  // in the state's precision (FP64 arithmetic is slow on this part); one
  // conversion per published value
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
    atomicMax(&sc->alpha[st % 3][0], dbits((double)mx));
    atomicMax(&sc->alpha[st % 3][1], dbits((double)my));
    const double wgt = (st == 3) ? 1.0 : (st == 2 ? 2.0 / 3.0 : 1.0 / 6.0);
    const double wfl = (st == 3) ? 2.0 / 3.0 : 1.0 / 6.0;
    // this CTA's own FP64 slot (no other CTA writes it: deterministic totals)
    if (dsum != T(0)) sc->part->clamp[blockIdx.x] += (wgt * p.area) * (double)dsum;
    if (fsum != T(0)) sc->part->edge[blockIdx.x] += wfl * dt * (double)fsum;
    if (st == 3 && rmax > T(0)) {
      const unsigned long long rb = dbits((double)rmax);
      atomicMax(&sc->runup_now[__ldcg(&sc->parity)], rb);
      atomicMax(&sc->runup_max, rb);
    }
    if (red.bad) atomicOr(&sc->status, ST_NONFINITE);
    if (st == 3 && lead) {
      const double tn = __ldcg(&sc->t_step) + dt, te = __ldcg(&sc->t_end);
      sc->t = (te > 0.0 && tn >= te) ? te : tn;
      sc->steps = __ldcg(&sc->steps) + 1;
    }
  }
}

// Persistent stage over all tiles of one scenario: CTA b handles tiles
// b, b + gridDim.x, ...; the halo box of the next tile arrives by tensor
// copies (thread 0 issues one per field) into the second buffer while the
// current tile is computed.  Each buffer has an mbarrier; every thread waits
// on it with a bounded spin (on expiry the CTA flags ST_TIMEOUT and returns,
// no other copy being in flight at that point).
template <typename T, int TX, int TY, int NT, int S, int STAGE, bool SHORE = false>
__device__ void stage_persistent(const StageIO<T> &io, const BoxMaps &maps, const Phys &p, DevScalars *sc, T *smem,
                                 RedSmem &red, int first, int stride, bool lead) {
  using G = TileGeom<T, TX, TY>;
  constexpr unsigned kBoxBytes = 4u * G::BH * G::P * (unsigned)sizeof(T);
  __shared__ unsigned long long bar[2];
  __shared__ unsigned s_fail;
  const int tid = threadIdx.x;
  const int tiles_x = (io.nx + TX - 1) / TX, tiles_y = (io.ny + TY - 1) / TY;
  const int ntiles = tiles_x * tiles_y;
  T *box0 = smem, *box1 = smem + G::BOX, *sL = smem + 2 * G::BOX;
  auto issue = [&](int tile, T *dst, unsigned long long *b) {
    const int x = (tile % tiles_x) * TX - G::OX, y = (tile / tiles_x) * TY - G::OY + p.halo_rows;
    mbar_expect_tx(b, kBoxBytes + p.copy_extra);
#pragma unroll
    for (int f = 0; f < 4; ++f) tma_load_2d(dst + f * G::FIELD, &maps.m[f], x, y, b);
  };
  // the first box is in flight while thread 0 takes the stage's scalars
  int t = first;
  if (tid == 0) {
    mbar_init(&bar[0], 1u);
    mbar_init(&bar[1], 1u);
    mbar_fence_init();
    s_fail = 0u;
    if (t < ntiles) issue(t, box0, &bar[0]);
    stage_scalars<T, STAGE>(p, sc, lead, red);
  }
  __syncthreads();
  if (red.skip) {
    if (tid == 0 && t < ntiles && !mbar_wait(&bar[0], 0u, p.wait_cycles)) atomicOr(&sc->status, ST_TIMEOUT);
    __syncthreads();
    return;
  }
  const double dt = red.dt;
  const T tdt = red_v<T>(red, SV_DT), rcap = red_v<T>(red, SV_RCAP);
  const T alx = red_v<T>(red, SV_AX), aly = red_v<T>(red, SV_AY);
  const T zref = consts<T>(p).zref;
  const T eta_in = red_v<T>(red, SV_ETA), u_in = red_v<T>(red, SV_UIN);
  Acc<T> acc;
  unsigned phase = 0u;  // bit b: parity of the next wait on bar[b]
  for (int it = 0; t < ntiles; ++it, t += stride) {
    const int b = it & 1;
    T *box = b ? box1 : box0;
    if (!mbar_wait(&bar[b], (phase >> b) & 1u, p.wait_cycles)) s_fail = 1u;
    phase ^= 1u << b;
    // one barrier: this tile's box has landed, and every thread is done with
    // the previous tile (whose buffer is refilled next)
    __syncthreads();
    if (s_fail) {
      if (tid == 0) atomicOr(&sc->status, ST_TIMEOUT);
      return;
    }
    const int tn = t + stride;
    if (tid == 0 && tn < ntiles) {
      fence_proxy_async();  // order the generic writes into that buffer (ghost patching) before the copies
      issue(tn, b ? box0 : box1, &bar[b ^ 1]);
    }
    const int i0 = (t % tiles_x) * TX, j0 = (t / tiles_x) * TY;
    if (i0 == 0 || j0 == 0 || i0 + TX + 3 > io.nx || j0 + TY + 3 > io.ny) {
      patch_box<T, TX, TY, NT>(io, p, i0, j0, box, zref, eta_in, u_in);
      __syncthreads();
    }
    tile_compute<T, TX, TY, NT, S, STAGE, SHORE>(io, p, i0, j0, box, sL, tdt, rcap, alx, aly, acc);
  }
  publish<T, NT, STAGE>(p, sc, lead, red, dt, acc);
}

}  // namespace swe
