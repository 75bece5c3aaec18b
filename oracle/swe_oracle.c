/*
 * Plain, slow FP64 CPU oracle for the explicit SSP-RK3 time step of the 2-D
 * nonlinear shallow-water equations with fifth-order WENO reconstruction,
 * global Lax-Friedrichs flux splitting, the well-balanced bed source, explicit
 * Manning friction and a wet/dry rule.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The CUDA library neither
 * links nor calls it, and the two share no source, header, table or helper.
 *
 * Paper: I. Madden, S. Marras, J. Suckale, "Leveraging Google's Tensor
 * Processing Units for tsunami-risk mitigation planning in the Pacific
 * Northwest and beyond", arXiv:2301.12010.  Equation numbers are the paper's
 * own: (1)-(3) the SWE with the 1/2 g (h^2 - b^2) momentum flux and the
 * -g (h+b) db/dx source, (4) the vector form, (5) the WENO face states,
 * (6) the Lax-Friedrichs flux, (7) the explicit update, (8) the RK3 stages,
 * (20) the Carrier N-wave.
 *
 * The code follows the method's steps in order: ghost fill, primitive
 * variables with the dry rule, global wave speeds, split fluxes, WENO5 face
 * fluxes in x then y, the bed and friction sources, the RK3 combination and
 * the post-stage positivity rule.  Where the paper is silent or garbled this
 * file takes the following readings:
 *  - LF (6) is applied as global Lax-Friedrichs flux SPLITTING on point values
 *    (finite-difference WENO of Shu and Osher): f+- = (F +- alpha Q)/2.
 *  - The bed terms follow the splitting of (2)-(3) (after Xing 2005, the
 *    paper's source-term reference) taken relative to the still-water depth
 *    d = max(z_ref - b, 0): pressure flux g (h^2 - d^2)/2 and source
 *    -g (h - d) db/dx.  Where b < z_ref (all of the sea) and z_ref = 0 this is
 *    exactly the printed g (h^2 - b^2)/2 and -g (h+b) db/dx; on land above
 *    z_ref it is the plain g h^2/2 and -g h db/dx, so that dry land carries no
 *    fictitious +-g b^2/2 terms.  Q = (h - d, hu, hv): the mass viscosity acts
 *    on the surface anomaly h - d (= h + b - z_ref in the sea, = h on land).
 *  - db/dx in the source is (bhat_{i+1/2} - bhat_{i-1/2})/dx, where bhat is
 *    the WENO reconstruction of b/2 with the nonlinear weights of the
 *    normal-momentum flux (both split halves), so that flux and source cancel
 *    for a lake at rest at any level in the sea (Xing & Shu's device); at
 *    rest at z_ref both vanish, shorelines included.  The y-momentum source
 *    uses db/dy (the print repeats db/dx).
 *  - alpha_x = max(|u| + sqrt(g h)), alpha_y = max(|v| + sqrt(g h)) over the
 *    interior cells, recomputed at every RK stage from that stage's input.
 *  - dt = cfl / (alpha_x/dx + alpha_y/dy) from the step's first stage, or a
 *    fixed dt; optionally truncated so that t never passes t_end.
 *  - Fused-step variant (alpha_margin > 0; not the paper's scheme, which takes
 *    alpha at every stage): all three stages split with one speed per step,
 *    alpha_margin x the alpha of U^n, so that a step depends on U^n and the
 *    bed alone and can be computed in one pass over tiles with a 9-cell halo.
 *    dt is still the CFL step of U^n's alpha.  alpha_margin >= 1 keeps
 *    the splitting speed above the speeds of U^n; whether it stays above
 *    those of the intermediate stages is the margin's job.
 *  - (8) is the Shu-Osher SSP-RK3 form (the printed nesting is the same map).
 *  - Wet/dry (not described in the paper): velocities are zero where
 *    h < h_dry; after every stage h < 0 is set to 0 and hu = hv = 0 where
 *    h < h_dry; the mass added by that clamp is counted with the stage's
 *    weight in the final RK combination (1/6, 2/3, 1).  Films with
 *    h_dry <= h < h_film get the velocity desingularisation of Kurganov &
 *    Petrova (2007): u = sqrt(2) h hu / sqrt(h^4 + h_film^4), hu := h u (and
 *    the same for v), which keeps thin-film velocities bounded.
 *  - Shoreline variant (shore = 1; not in the paper, which is silent on wet/dry
 *    fronts): a face whose six-cell WENO stencil holds a dry cell (h < h_dry)
 *    takes the first-order hydrostatic reconstruction
 *    of Audusse et al. (2004) instead: face bed b_f = max(b_L, b_R), face
 *    depths h*_s = max(0, h_s + b_s - b_f), the global-LF flux of the standard
 *    SWE flux (pressure g h*^2/2) of those face states with the line's alpha,
 *    and for each side s the normal-momentum flux it sees raised by
 *    g (h_s^2 - h*_s^2)/2.  Each side's value is then shifted by the
 *    cell-local -g d_s^2/2 + g (h_s - d_s) b_s, which carries it into this
 *    file's still-depth form: at rest a WENO face and such a face give the same
 *    value g (h - d)(eta + z_ref)/2 to a cell between them, so a lake at rest
 *    at any level at or below z_ref is exact beside any dry land, and shore
 *    cells update with the positivity-preserving first-order scheme.
 *  - Friction is explicit, applied only where h >= h_dry, with the rate
 *    kappa = g n^2 |q| / h^(7/3) capped at 1/dt.
 *  - Walls: ghost k mirrors interior k-1 (h, b, tangential momentum even,
 *    normal momentum odd).  Inflow (x- side only): ghosts carry the Carrier
 *    N-wave (20) evaluated in time, h = max(eta_in - b, 0), u = eta_in
 *    sqrt(g/d0), v = 0.  Periodic: wrap, with an optional bed offset.
 *  - Runup: max of h+b over cells with h >= h_wet and b > 0 (-inf if none).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 3 /* ghost width: WENO5 needs three cells beyond each face */

enum { OR_WALL = 0, OR_INFLOW = 1, OR_PERIODIC = 2 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENONFINITE = 4 };

typedef struct {
  double g;          /* gravity, (1)-(3) */
  double manning_n;  /* Manning coefficient n of (2)-(3); 0 = no friction */
  double h_dry;      /* depth below which a cell is dry */
  double h_wet;      /* depth above which a land cell counts for runup */
  double weno_eps;   /* WENO epsilon */
  double fixed_dt;   /* > 0: fixed time step; else CFL */
  double cfl;        /* CFL number when fixed_dt <= 0 */
  double t_end;      /* > 0: truncate the last step at t_end */
  double b_jump_x;   /* periodic-x bed offset: b(i+nx) = b(i) + b_jump_x */
  double b_jump_y;   /* periodic-y bed offset */
  double inflow_amp;    /* peak surface elevation of the inflow N-wave */
  double inflow_period; /* N-wave period T; lambda = T sqrt(g d0) */
  double inflow_depth;  /* offshore depth d0 */
  double z_ref;         /* still-water level: d = max(z_ref - b, 0) */
  double h_film;        /* film depth of the velocity desingularisation */
  double alpha_margin;  /* > 0: fused-step variant, splitting speed alpha_margin x alpha(U^n)
                           in all three stages; 0: alpha of each stage's input (the paper) */
  int32_t bc[4];        /* x-, x+, y-, y+ */
  int32_t shore;        /* 1: shoreline variant, hydrostatic-reconstruction faces where a WENO
                           stencil meets a dry cell; 0: WENO at every face (the paper) */
  int32_t pad_;
} or_params;

typedef struct {
  double t, last_dt;
  double alpha_x, alpha_y; /* wave speeds of the current state */
  double mass;             /* sum h dx dy */
  double clamp_mass;       /* RK-weighted mass added by the h<0 clamp */
  double boundary_mass;    /* RK-weighted mass that entered through the edges */
  double runup_now, runup_max;
  int64_t steps;
  int32_t status, pad;
} or_state;

typedef struct {
  int nx, ny, nxg, nyg;
  double dx, dy;
  const or_params *p;
} grid_t;

static inline size_t ix(const grid_t *g, int i, int j) {
  return (size_t)(j + NG) * (size_t)g->nxg + (size_t)(i + NG);
}
static inline double sq(double x) { return x * x; }

/* ---------------------------------------------------------------- WENO5 */
/* Candidate values of the three 3-point stencils at the right face of v[2]
 * (Jiang & Shu 1996, the paper's WENO reference in "Numerical approximation"). */
static void weno5_candidates(const double v[5], double p[3]) {
  p[0] = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
  p[1] = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
  p[2] = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
}

/* Left-biased WENO5-JS value at the right face of v[2]; w receives the
 * normalised nonlinear weights. */
static double weno5(const double v[5], double eps, double w[3]) {
  double p[3];
  weno5_candidates(v, p);
  double beta[3];
  beta[0] = 13.0 / 12.0 * sq(v[0] - 2.0 * v[1] + v[2]) + 0.25 * sq(v[0] - 4.0 * v[1] + 3.0 * v[2]);
  beta[1] = 13.0 / 12.0 * sq(v[1] - 2.0 * v[2] + v[3]) + 0.25 * sq(v[1] - v[3]);
  beta[2] = 13.0 / 12.0 * sq(v[2] - 2.0 * v[3] + v[4]) + 0.25 * sq(3.0 * v[2] - 4.0 * v[3] + v[4]);
  const double d[3] = {0.1, 0.6, 0.3};
  double a[3], s = 0.0;
  for (int k = 0; k < 3; ++k) {
    a[k] = d[k] / sq(eps + beta[k]);
    s += a[k];
  }
  double r = 0.0;
  for (int k = 0; k < 3; ++k) {
    w[k] = a[k] / s;
    r += w[k] * p[k];
  }
  return r;
}

/* ------------------------------------------------------- boundary values */
/* Carrier N-wave (20) with a1 = amp/2, a2 = a1/3, lambda = T sqrt(g d0),
 * entering through the x- edge: the profile is read at s = 1.3 lambda - c0 t,
 * so that the leading crest arrives after t ~ 0.8 T. */
double or_inflow_eta(const or_params *p, double t) {
  double c0 = sqrt(p->g * p->inflow_depth);
  double lam = p->inflow_period * c0;
  double a1 = 0.5 * p->inflow_amp, a2 = a1 / 3.0;
  double k1 = 28.416 / (lam * lam), k2 = 256.0 / (lam * lam);
  double x1 = 0.5151125 * lam, x2 = 0.2048 * lam;
  double s = 1.3 * lam - c0 * t;
  return 2.0 * (a1 * exp(-k1 * sq(s - x1)) - a2 * exp(-k2 * sq(s - x2)));
}

static void fill_bed_ghosts(const grid_t *g, double *b) {
  const or_params *p = g->p;
  for (int j = 0; j < g->ny; ++j)
    for (int k = 0; k < NG; ++k) {
      b[ix(g, -1 - k, j)] = (p->bc[0] == OR_PERIODIC) ? b[ix(g, g->nx - 1 - k, j)] - p->b_jump_x
                                                      : b[ix(g, k, j)];
      b[ix(g, g->nx + k, j)] = (p->bc[1] == OR_PERIODIC) ? b[ix(g, k, j)] + p->b_jump_x
                                                         : b[ix(g, g->nx - 1 - k, j)];
    }
  for (int i = 0; i < g->nx; ++i)
    for (int k = 0; k < NG; ++k) {
      b[ix(g, i, -1 - k)] = (p->bc[2] == OR_PERIODIC) ? b[ix(g, i, g->ny - 1 - k)] - p->b_jump_y
                                                      : b[ix(g, i, k)];
      b[ix(g, i, g->ny + k)] = (p->bc[3] == OR_PERIODIC) ? b[ix(g, i, k)] + p->b_jump_y
                                                         : b[ix(g, i, g->ny - 1 - k)];
    }
}

/* Ghost ring of the state at time t.  Corner ghosts are never read. */
static void fill_state_ghosts(const grid_t *g, const double *b, double *h, double *hu, double *hv,
                              double t) {
  const or_params *p = g->p;
  const int nx = g->nx, ny = g->ny;
  double eta_in = 0.0, u_in = 0.0;
  if (p->bc[0] == OR_INFLOW) {
    eta_in = or_inflow_eta(p, t);
    u_in = eta_in * sqrt(p->g / p->inflow_depth);
  }
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k < NG; ++k) {
      size_t gl = ix(g, -1 - k, j), gr = ix(g, nx + k, j);
      if (p->bc[0] == OR_WALL) {
        size_t s = ix(g, k, j);
        h[gl] = h[s]; hu[gl] = -hu[s]; hv[gl] = hv[s];
      } else if (p->bc[0] == OR_PERIODIC) {
        size_t s = ix(g, nx - 1 - k, j);
        h[gl] = h[s]; hu[gl] = hu[s]; hv[gl] = hv[s];
      } else { /* inflow */
        double hg = eta_in - b[gl];
        if (hg < 0.0) hg = 0.0;
        h[gl] = hg; hu[gl] = hg * u_in; hv[gl] = 0.0;
      }
      if (p->bc[1] == OR_WALL) {
        size_t s = ix(g, nx - 1 - k, j);
        h[gr] = h[s]; hu[gr] = -hu[s]; hv[gr] = hv[s];
      } else { /* periodic */
        size_t s = ix(g, k, j);
        h[gr] = h[s]; hu[gr] = hu[s]; hv[gr] = hv[s];
      }
    }
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < NG; ++k) {
      size_t gb = ix(g, i, -1 - k), gt = ix(g, i, ny + k);
      if (p->bc[2] == OR_WALL) {
        size_t s = ix(g, i, k);
        h[gb] = h[s]; hu[gb] = hu[s]; hv[gb] = -hv[s];
      } else {
        size_t s = ix(g, i, ny - 1 - k);
        h[gb] = h[s]; hu[gb] = hu[s]; hv[gb] = hv[s];
      }
      if (p->bc[3] == OR_WALL) {
        size_t s = ix(g, i, ny - 1 - k);
        h[gt] = h[s]; hu[gt] = hu[s]; hv[gt] = -hv[s];
      } else {
        size_t s = ix(g, i, k);
        h[gt] = h[s]; hu[gt] = hu[s]; hv[gt] = hv[s];
      }
    }
}

/* ------------------------------------------------- primitives and speeds */
static inline void velocity(const or_params *p, double h, double hu, double hv, double *u,
                            double *v) {
  if (h < p->h_dry) {
    *u = 0.0;
    *v = 0.0;
  } else {
    *u = hu / h;
    *v = hv / h;
  }
}

/* Global maximum characteristic speeds over the interior ("TPU
 * implementation": one maximum for the whole domain).  Returns nonzero if a
 * non-finite value is met. */
static int max_speeds(const grid_t *g, const double *h, const double *hu, const double *hv,
                      double *ax, double *ay) {
  const or_params *p = g->p;
  double mx = 0.0, my = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : mx, my) reduction(| : bad)
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      size_t c = ix(g, i, j);
      if (!isfinite(h[c]) || !isfinite(hu[c]) || !isfinite(hv[c])) {
        bad = 1;
        continue;
      }
      double u, v;
      velocity(p, h[c], hu[c], hv[c], &u, &v);
      double cel = sqrt(p->g * (h[c] > 0.0 ? h[c] : 0.0));
      double sx = fabs(u) + cel, sy = fabs(v) + cel;
      if (sx > mx) mx = sx;
      if (sy > my) my = sy;
    }
  *ax = mx;
  *ay = my;
  return bad;
}

/* Still-water depth d = max(z_ref - b, 0). */
static inline double still_depth(const or_params *p, double b) {
  double d = p->z_ref - b;
  return d > 0.0 ? d : 0.0;
}

/* Split fluxes f+- = (F +- alpha Q)/2 of one cell for direction dir
 * (0: F of (2), 1: G of (3)) with pressure g (h^2 - d^2)/2 and
 * Q = (h - d, hu, hv). */
static void split_flux(const or_params *p, int dir, double h, double hu, double hv, double b,
                       double alpha, double fp[3], double fm[3]) {
  double u, v;
  velocity(p, h, hu, hv, &u, &v);
  double d = still_depth(p, b);
  double pres = 0.5 * p->g * (h - d) * (h + d);
  double F[3], Q[3] = {h - d, hu, hv};
  if (dir == 0) {
    F[0] = hu;
    F[1] = hu * u + pres;
    F[2] = hv * u;
  } else {
    F[0] = hv;
    F[1] = hu * v;
    F[2] = hv * v + pres;
  }
  for (int m = 0; m < 3; ++m) {
    fp[m] = 0.5 * (F[m] + alpha * Q[m]);
    fm[m] = 0.5 * (F[m] - alpha * Q[m]);
  }
}

/* Face fluxes along one grid line of n interior cells.  Line arrays hold
 * cells -3 .. n+2 at offsets 0 .. n+5.  For the face i+1/2, i = -1 .. n-1,
 * stored at index i+1:
 *   Fhat_m = W(f+_m[i-2..i+2]) + W(f-_m[i+3, i+2, i+1, i, i-1])
 *   bhat   = sum_k w+_k p_k(b/2 [i-2..i+2]) + sum_k w-_k p_k(b/2 [i+3..i-1])
 * where w+- are the weights of component `mom` (the normal momentum). */
static void sweep_line(int n, double eps, int mom, double *const fp[3], double *const fm[3],
                       const double *bl, double *const Fhat[3], double *bhat) {
  for (int i = -1; i < n; ++i) {
    int c = i + NG;
    double wp[3] = {0, 0, 0}, wm[3] = {0, 0, 0};
    for (int m = 0; m < 3; ++m) {
      double vp[5] = {fp[m][c - 2], fp[m][c - 1], fp[m][c], fp[m][c + 1], fp[m][c + 2]};
      double vm[5] = {fm[m][c + 3], fm[m][c + 2], fm[m][c + 1], fm[m][c], fm[m][c - 1]};
      double w1[3], w2[3];
      double fl = weno5(vp, eps, w1);
      double fr = weno5(vm, eps, w2);
      Fhat[m][i + 1] = fl + fr;
      if (m == mom)
        for (int k = 0; k < 3; ++k) {
          wp[k] = w1[k];
          wm[k] = w2[k];
        }
    }
    double bp[5], bm[5], pp[3], pm[3];
    for (int k = 0; k < 5; ++k) {
      bp[k] = 0.5 * bl[c - 2 + k];
      bm[k] = 0.5 * bl[c + 3 - k];
    }
    weno5_candidates(bp, pp);
    weno5_candidates(bm, pm);
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += wp[k] * pp[k] + wm[k] * pm[k];
    bhat[i + 1] = s;
  }
}

/* Shoreline variant along one grid line (see the header): for every face
 * i+1/2, i = -1 .. n-1 (index i+1), whose stencil cells i-2 .. i+3 hold a
 * dry cell, the values the left and the right cell see replace
 * the WENO face values: FL[m], bL for cell i, FR[m], bR for cell i+1 (the
 * bed values enter through g (h - d) b of the cell update).  Elsewhere
 * FL = FR = Fhat and bL = bR = bhat.  hl, ql, tl, bl: depth, normal and
 * tangential momentum and bed along the line (cells -3 .. n+2).  mom: the
 * component of the normal momentum (1 in x, 2 in y). */
static void shore_faces(const or_params *p, int n, double alpha, int mom, const double *hl, const double *ql,
                        const double *tl, const double *bl, double *const Fhat[3], const double *bhat,
                        double *const FL[3], double *const FR[3], double *bL, double *bR) {
  const int tan = 3 - mom;
  for (int i = -1; i < n; ++i) {
    const int c = i + NG, f = i + 1;
    int shore = 0;
    for (int k = c - 2; k <= c + 3; ++k)
      if (hl[k] < p->h_dry) shore = 1;
    if (!shore) {
      for (int m = 0; m < 3; ++m) FL[m][f] = FR[m][f] = Fhat[m][f];
      bL[f] = bR[f] = bhat[f];
      continue;
    }
    const int side[2] = {c, c + 1};
    const double bf = bl[c] > bl[c + 1] ? bl[c] : bl[c + 1];
    double hs[2], F[2][3], U[2][3];
    for (int s = 0; s < 2; ++s) {
      const int k = side[s];
      double u, v;
      velocity(p, hl[k], ql[k], tl[k], &u, &v); /* u: normal, v: tangential velocity */
      hs[s] = hl[k] + (bl[k] - bf);
      if (hs[s] < 0.0) hs[s] = 0.0;
      U[s][0] = hs[s];
      U[s][mom] = hs[s] * u;
      U[s][tan] = hs[s] * v;
      F[s][0] = hs[s] * u;
      F[s][mom] = hs[s] * u * u + 0.5 * p->g * hs[s] * hs[s];
      F[s][tan] = hs[s] * u * v;
    }
    double Fhr[3];
    for (int m = 0; m < 3; ++m) Fhr[m] = 0.5 * (F[0][m] + F[1][m]) - 0.5 * alpha * (U[1][m] - U[0][m]);
    for (int s = 0; s < 2; ++s) {
      const int k = side[s];
      const double d = still_depth(p, bl[k]);
      double *const *out = s == 0 ? FL : FR;
      out[0][f] = Fhr[0];
      out[tan][f] = Fhr[tan];
      out[mom][f] = Fhr[mom] + 0.5 * p->g * (hl[k] * hl[k] - hs[s] * hs[s]) - 0.5 * p->g * d * d;
      (s == 0 ? bL : bR)[f] = bl[k];
    }
  }
}

/* Per-line scratch of the face values each side of a face sees. */
typedef struct {
  double *mem;
  double *h, *q, *t;              /* depth, normal and tangential momentum, cells -3 .. n+2 */
  double *FL[3], *FR[3], *bL, *bR; /* faces -1/2 .. n-1/2 */
} line_t;

static int line_alloc(line_t *ln, size_t len, int n) {
  const size_t nf = (size_t)n + 1;
  ln->mem = (double *)malloc(sizeof(double) * (3 * len + 8 * nf));
  if (!ln->mem) return 1;
  ln->h = ln->mem;
  ln->q = ln->h + len;
  ln->t = ln->q + len;
  double *f = ln->t + len;
  for (int m = 0; m < 3; ++m) {
    ln->FL[m] = f + m * nf;
    ln->FR[m] = f + (3 + m) * nf;
  }
  ln->bL = f + 6 * nf;
  ln->bR = f + 7 * nf;
  return 0;
}

/* The face values of one line: the WENO values, or with the shoreline
 * variant the hydrostatic-reconstruction values where a stencil meets a dry
 * cell. */
static void line_faces(const or_params *p, line_t *ln, int n, double alpha, int mom, const double *bl,
                       double *const Fhat[3], const double *bhat) {
  if (p->shore) {
    shore_faces(p, n, alpha, mom, ln->h, ln->q, ln->t, bl, Fhat, bhat, ln->FL, ln->FR, ln->bL, ln->bR);
    return;
  }
  for (int f = 0; f <= n; ++f) {
    for (int m = 0; m < 3; ++m) ln->FL[m][f] = ln->FR[m][f] = Fhat[m][f];
    ln->bL[f] = ln->bR[f] = bhat[f];
  }
}

/* L(U) of (7): L = -(Fhat_{i+1/2} - Fhat_{i-1/2})/dx - (Ghat_{j+1/2} - Ghat_{j-1/2})/dy + S.
 * Ghosts of h, hu, hv and b must be filled.  Writes interior-sized L arrays
 * and the net mass flux into the domain through its edges (per unit time). */
static int operator_L(const grid_t *g, const double *b, const double *h, const double *hu,
                      const double *hv, double ax, double ay, double dt, double *Lh, double *Lhu,
                      double *Lhv, double *edge_flux) {
  const or_params *p = g->p;
  const int nx = g->nx, ny = g->ny;
  int fail = 0;
  double flux_x = 0.0, flux_y = 0.0;
  double *rowflux = (double *)calloc((size_t)ny, sizeof(double));
  double *colflux = (double *)calloc((size_t)nx, sizeof(double));
  if (!rowflux || !colflux) {
    free(rowflux);
    free(colflux);
    return OR_ENOMEM;
  }

  /* x sweep, one row at a time */
#pragma omp parallel
  {
    int n = nx;
    size_t len = (size_t)(n + 2 * NG);
    double *buf = (double *)malloc(sizeof(double) * (len * 7 + (size_t)(n + 1) * 4));
    if (!buf) {
#pragma omp atomic write
      fail = 1;
    } else {
      double *fp[3] = {buf, buf + len, buf + 2 * len};
      double *fm[3] = {buf + 3 * len, buf + 4 * len, buf + 5 * len};
      double *bl = buf + 6 * len;
      double *Fh[3] = {buf + 7 * len, buf + 7 * len + (n + 1), buf + 7 * len + 2 * (n + 1)};
      double *bh = buf + 7 * len + 3 * (n + 1);
      line_t ln;
      if (line_alloc(&ln, len, n)) {
#pragma omp atomic write
        fail = 1;
      }
#pragma omp for
      for (int j = 0; j < ny; ++j) {
        if (!ln.mem) continue;
        for (int i = -NG; i < n + NG; ++i) {
          size_t c = ix(g, i, j);
          double a[3], m_[3];
          split_flux(p, 0, h[c], hu[c], hv[c], b[c], ax, a, m_);
          for (int m = 0; m < 3; ++m) {
            fp[m][i + NG] = a[m];
            fm[m][i + NG] = m_[m];
          }
          bl[i + NG] = b[c];
          ln.h[i + NG] = h[c];
          ln.q[i + NG] = hu[c];
          ln.t[i + NG] = hv[c];
        }
        sweep_line(n, p->weno_eps, 1, fp, fm, bl, Fh, bh);
        line_faces(p, &ln, n, ax, 1, bl, Fh, bh);
        for (int i = 0; i < n; ++i) {
          size_t c = ix(g, i, j);
          size_t o = (size_t)j * nx + i;
          double ha = h[c] - still_depth(p, b[c]);
          Lh[o] = -(ln.FL[0][i + 1] - ln.FR[0][i]) / g->dx;
          Lhu[o] = -(ln.FL[1][i + 1] - ln.FR[1][i]) / g->dx - p->g * ha * (ln.bL[i + 1] - ln.bR[i]) / g->dx;
          Lhv[o] = -(ln.FL[2][i + 1] - ln.FR[2][i]) / g->dx;
        }
        rowflux[j] = (ln.FR[0][0] - ln.FL[0][n]) * g->dy;
      }
      free(ln.mem);
      free(buf);
    }
  }
  if (fail) {
    free(rowflux);
    free(colflux);
    return OR_ENOMEM;
  }

  /* y sweep, one column at a time */
#pragma omp parallel
  {
    int n = ny;
    size_t len = (size_t)(n + 2 * NG);
    double *buf = (double *)malloc(sizeof(double) * (len * 7 + (size_t)(n + 1) * 4));
    if (!buf) {
#pragma omp atomic write
      fail = 1;
    } else {
      double *fp[3] = {buf, buf + len, buf + 2 * len};
      double *fm[3] = {buf + 3 * len, buf + 4 * len, buf + 5 * len};
      double *bl = buf + 6 * len;
      double *Gh[3] = {buf + 7 * len, buf + 7 * len + (n + 1), buf + 7 * len + 2 * (n + 1)};
      double *bh = buf + 7 * len + 3 * (n + 1);
      line_t ln;
      if (line_alloc(&ln, len, n)) {
#pragma omp atomic write
        fail = 1;
      }
#pragma omp for
      for (int i = 0; i < nx; ++i) {
        if (!ln.mem) continue;
        for (int j = -NG; j < n + NG; ++j) {
          size_t c = ix(g, i, j);
          double a[3], m_[3];
          split_flux(p, 1, h[c], hu[c], hv[c], b[c], ay, a, m_);
          for (int m = 0; m < 3; ++m) {
            fp[m][j + NG] = a[m];
            fm[m][j + NG] = m_[m];
          }
          bl[j + NG] = b[c];
          ln.h[j + NG] = h[c];
          ln.q[j + NG] = hv[c];
          ln.t[j + NG] = hu[c];
        }
        sweep_line(n, p->weno_eps, 2, fp, fm, bl, Gh, bh);
        line_faces(p, &ln, n, ay, 2, bl, Gh, bh);
        for (int j = 0; j < n; ++j) {
          size_t c = ix(g, i, j);
          size_t o = (size_t)j * nx + i;
          double ha = h[c] - still_depth(p, b[c]);
          Lh[o] += -(ln.FL[0][j + 1] - ln.FR[0][j]) / g->dy;
          Lhu[o] += -(ln.FL[1][j + 1] - ln.FR[1][j]) / g->dy;
          Lhv[o] += -(ln.FL[2][j + 1] - ln.FR[2][j]) / g->dy - p->g * ha * (ln.bL[j + 1] - ln.bR[j]) / g->dy;
        }
        colflux[i] = (ln.FR[0][0] - ln.FL[0][n]) * g->dx;
      }
      free(ln.mem);
      free(buf);
    }
  }
  if (fail) {
    free(rowflux);
    free(colflux);
    return OR_ENOMEM;
  }
  for (int j = 0; j < ny; ++j) flux_x += rowflux[j];
  for (int i = 0; i < nx; ++i) flux_y += colflux[i];
  free(rowflux);
  free(colflux);
  *edge_flux = flux_x + flux_y;

  /* explicit Manning friction, (2)-(3), capped at 1/dt */
  if (p->manning_n > 0.0) {
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = ix(g, i, j);
        size_t o = (size_t)j * nx + i;
        if (h[c] >= p->h_dry) {
          double q = sqrt(hu[c] * hu[c] + hv[c] * hv[c]);
          double kappa = p->g * p->manning_n * p->manning_n * q / pow(h[c], 7.0 / 3.0);
          if (dt > 0.0 && kappa > 1.0 / dt) kappa = 1.0 / dt;
          Lhu[o] -= kappa * hu[c];
          Lhv[o] -= kappa * hv[c];
        }
      }
  }
  return OR_OK;
}

/* Post-stage rule: h < 0 -> 0 (returns the added depth summed in row order),
 * then hu = hv = 0 where h < h_dry, and the film desingularisation where
 * h_dry <= h < h_film. */
static double post_rule(const grid_t *g, double *h, double *hu, double *hv) {
  const or_params *p = g->p;
  double *rows = (double *)calloc((size_t)g->ny, sizeof(double));
#pragma omp parallel for
  for (int j = 0; j < g->ny; ++j) {
    double s = 0.0;
    for (int i = 0; i < g->nx; ++i) {
      size_t c = ix(g, i, j);
      if (h[c] < 0.0) {
        s += -h[c];
        h[c] = 0.0;
      }
      if (h[c] < p->h_dry) {
        hu[c] = 0.0;
        hv[c] = 0.0;
      } else if (h[c] < p->h_film) {
        double h2 = h[c] * h[c];
        double f = sqrt(2.0) * h2 / sqrt(h2 * h2 + pow(p->h_film, 4.0));
        hu[c] *= f;
        hv[c] *= f;
      }
    }
    if (rows) rows[j] = s;
  }
  double t = 0.0;
  if (rows)
    for (int j = 0; j < g->ny; ++j) t += rows[j];
  free(rows);
  return t;
}

static double total_mass(const grid_t *g, const double *h) {
  double t = 0.0;
  for (int j = 0; j < g->ny; ++j) {
    double s = 0.0;
    for (int i = 0; i < g->nx; ++i) s += h[ix(g, i, j)];
    t += s;
  }
  return t * g->dx * g->dy;
}

static double runup_now(const grid_t *g, const double *b, const double *h) {
  double r = -INFINITY;
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      size_t c = ix(g, i, j);
      if (h[c] >= g->p->h_wet && b[c] > 0.0 && h[c] + b[c] > r) r = h[c] + b[c];
    }
  return r;
}

/* ------------------------------------------------------------ RK3 step */
typedef struct {
  double *h, *hu, *hv;
} fields_t;

static int rk3_step(const grid_t *g, const double *b, fields_t U0, fields_t U1, fields_t U2,
                    fields_t UN, double *Lh, double *Lhu, double *Lhv, or_state *st) {
  const or_params *p = g->p;
  const int nx = g->nx, ny = g->ny;
  const double t = st->t;
  double ax, ay, flux;

  /* stage 1: U1 = U0 + dt L(U0) */
  fill_state_ghosts(g, b, U0.h, U0.hu, U0.hv, t);
  if (max_speeds(g, U0.h, U0.hu, U0.hv, &ax, &ay)) return OR_ENONFINITE;
  double dt;
  if (p->fixed_dt > 0.0) {
    dt = p->fixed_dt;
  } else {
    double den = ax / g->dx + ay / g->dy;
    if (!(den > 0.0)) return OR_EINVAL; /* fully dry and still: CFL step undefined */
    dt = p->cfl / den;
  }
  if (p->t_end > 0.0 && t + dt > p->t_end) dt = p->t_end - t;
  if (!(dt > 0.0)) return OR_EINVAL;

  /* the fused-step variant keeps this splitting speed for the whole step */
  const int fused = p->alpha_margin > 0.0;
  const double sx = fused ? p->alpha_margin * ax : ax, sy = fused ? p->alpha_margin * ay : ay;

  double clamp = 0.0, bmass = 0.0;
  int rc = operator_L(g, b, U0.h, U0.hu, U0.hv, sx, sy, dt, Lh, Lhu, Lhv, &flux);
  if (rc) return rc;
  bmass += dt * flux / 6.0;
#pragma omp parallel for
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(g, i, j), o = (size_t)j * nx + i;
      U1.h[c] = U0.h[c] + dt * Lh[o];
      U1.hu[c] = U0.hu[c] + dt * Lhu[o];
      U1.hv[c] = U0.hv[c] + dt * Lhv[o];
    }
  clamp += post_rule(g, U1.h, U1.hu, U1.hv) / 6.0;

  /* stage 2: U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)) */
  fill_state_ghosts(g, b, U1.h, U1.hu, U1.hv, t + dt);
  if (max_speeds(g, U1.h, U1.hu, U1.hv, &ax, &ay)) return OR_ENONFINITE;
  if (fused) { ax = sx; ay = sy; }
  rc = operator_L(g, b, U1.h, U1.hu, U1.hv, ax, ay, dt, Lh, Lhu, Lhv, &flux);
  if (rc) return rc;
  bmass += dt * flux / 6.0;
#pragma omp parallel for
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(g, i, j), o = (size_t)j * nx + i;
      U2.h[c] = 0.75 * U0.h[c] + 0.25 * (U1.h[c] + dt * Lh[o]);
      U2.hu[c] = 0.75 * U0.hu[c] + 0.25 * (U1.hu[c] + dt * Lhu[o]);
      U2.hv[c] = 0.75 * U0.hv[c] + 0.25 * (U1.hv[c] + dt * Lhv[o]);
    }
  clamp += post_rule(g, U2.h, U2.hu, U2.hv) * (2.0 / 3.0);

  /* stage 3: U^{n+1} = 1/3 U0 + 2/3 (U2 + dt L(U2)) */
  fill_state_ghosts(g, b, U2.h, U2.hu, U2.hv, t + 0.5 * dt);
  if (max_speeds(g, U2.h, U2.hu, U2.hv, &ax, &ay)) return OR_ENONFINITE;
  if (fused) { ax = sx; ay = sy; }
  rc = operator_L(g, b, U2.h, U2.hu, U2.hv, ax, ay, dt, Lh, Lhu, Lhv, &flux);
  if (rc) return rc;
  bmass += dt * flux * (2.0 / 3.0);
#pragma omp parallel for
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(g, i, j), o = (size_t)j * nx + i;
      UN.h[c] = U0.h[c] / 3.0 + (2.0 / 3.0) * (U2.h[c] + dt * Lh[o]);
      UN.hu[c] = U0.hu[c] / 3.0 + (2.0 / 3.0) * (U2.hu[c] + dt * Lhu[o]);
      UN.hv[c] = U0.hv[c] / 3.0 + (2.0 / 3.0) * (U2.hv[c] + dt * Lhv[o]);
    }
  clamp += post_rule(g, UN.h, UN.hu, UN.hv);

  if (max_speeds(g, UN.h, UN.hu, UN.hv, &ax, &ay)) return OR_ENONFINITE;
  /* accept the step */
  for (int j = 0; j < ny; ++j) {
    size_t c = ix(g, 0, j);
    memcpy(U0.h + c, UN.h + c, sizeof(double) * nx);
    memcpy(U0.hu + c, UN.hu + c, sizeof(double) * nx);
    memcpy(U0.hv + c, UN.hv + c, sizeof(double) * nx);
  }
  st->t = (p->t_end > 0.0 && t + dt >= p->t_end) ? p->t_end : t + dt;
  st->last_dt = dt;
  st->steps += 1;
  st->alpha_x = ax;
  st->alpha_y = ay;
  st->clamp_mass += clamp * g->dx * g->dy;
  st->boundary_mass += bmass;
  double r = runup_now(g, b, U0.h);
  st->runup_now = r;
  if (r > st->runup_max) st->runup_max = r;
  return OR_OK;
}

/* ----------------------------------------------------------- public API */
static int validate(int nx, int ny, double dx, double dy, const or_params *p) {
  if (nx < NG || ny < NG || !(dx > 0.0) || !(dy > 0.0) || !p) return OR_EINVAL;
  for (int s = 0; s < 4; ++s)
    if (p->bc[s] < OR_WALL || p->bc[s] > OR_PERIODIC) return OR_EINVAL;
  if ((p->bc[0] == OR_PERIODIC) != (p->bc[1] == OR_PERIODIC)) return OR_EINVAL;
  if ((p->bc[2] == OR_PERIODIC) != (p->bc[3] == OR_PERIODIC)) return OR_EINVAL;
  if (p->bc[1] == OR_INFLOW || p->bc[2] == OR_INFLOW || p->bc[3] == OR_INFLOW) return OR_EINVAL;
  if (p->bc[0] == OR_INFLOW && !(p->inflow_depth > 0.0 && p->inflow_period > 0.0)) return OR_EINVAL;
  if (!(p->g > 0.0) || p->manning_n < 0.0 || !(p->h_dry >= 0.0) || !(p->weno_eps > 0.0))
    return OR_EINVAL;
  if (!(p->fixed_dt > 0.0) && !(p->cfl > 0.0)) return OR_EINVAL;
  if (!(p->alpha_margin == 0.0 || p->alpha_margin >= 1.0)) return OR_EINVAL;
  if (p->shore != 0 && p->shore != 1) return OR_EINVAL;
  return OR_OK;
}

typedef struct {
  grid_t g;
  double *mem;
  double *b;
  fields_t U0, U1, U2, UN;
  double *Lh, *Lhu, *Lhv;
} work_t;

static int work_alloc(work_t *w, int nx, int ny, double dx, double dy, const or_params *p,
                      const double *b_in, const double *h, const double *hu, const double *hv) {
  w->g.nx = nx;
  w->g.ny = ny;
  w->g.nxg = nx + 2 * NG;
  w->g.nyg = ny + 2 * NG;
  w->g.dx = dx;
  w->g.dy = dy;
  w->g.p = p;
  size_t ng = (size_t)w->g.nxg * w->g.nyg, ni = (size_t)nx * ny;
  w->mem = (double *)calloc(ng * 13 + ni * 3, sizeof(double));
  if (!w->mem) return OR_ENOMEM;
  double *q = w->mem;
  w->b = q; q += ng;
  fields_t *F[4] = {&w->U0, &w->U1, &w->U2, &w->UN};
  for (int k = 0; k < 4; ++k) {
    F[k]->h = q; q += ng;
    F[k]->hu = q; q += ng;
    F[k]->hv = q; q += ng;
  }
  w->Lh = q; q += ni;
  w->Lhu = q; q += ni;
  w->Lhv = q;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(&w->g, i, j), o = (size_t)j * nx + i;
      w->b[c] = b_in[o];
      if (h) {
        w->U0.h[c] = h[o];
        w->U0.hu[c] = hu[o];
        w->U0.hv[c] = hv[o];
      }
    }
  fill_bed_ghosts(&w->g, w->b);
  return OR_OK;
}

/* Advance the state (h, hu, hv; row-major [ny][nx], in/out) by up to nsteps
 * RK3 steps (fewer if t reaches t_end or an error occurs).  st carries time,
 * step count and diagnostics across calls.  Returns an OR_* code; on error the
 * arrays hold the last accepted state. */
int or_steps(int nx, int ny, double dx, double dy, const or_params *p, const double *b,
             double *h, double *hu, double *hv, int64_t nsteps, or_state *st) {
  int rc = validate(nx, ny, dx, dy, p);
  if (rc) return rc;
  work_t w;
  rc = work_alloc(&w, nx, ny, dx, dy, p, b, h, hu, hv);
  if (rc) return rc;
  for (int64_t s = 0; s < nsteps; ++s) {
    if (p->t_end > 0.0 && st->t >= p->t_end) break;
    rc = rk3_step(&w.g, w.b, w.U0, w.U1, w.U2, w.UN, w.Lh, w.Lhu, w.Lhv, st);
    if (rc) break;
  }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(&w.g, i, j), o = (size_t)j * nx + i;
      h[o] = w.U0.h[c];
      hu[o] = w.U0.hu[c];
      hv[o] = w.U0.hv[c];
    }
  st->mass = total_mass(&w.g, w.U0.h);
  st->status = rc;
  free(w.mem);
  return rc;
}

/* Diagnostics of a state without stepping: mass, wave speeds, runup now
 * (runup_max is raised to it). */
int or_diagnose(int nx, int ny, double dx, double dy, const or_params *p, const double *b,
                const double *h, const double *hu, const double *hv, or_state *st) {
  int rc = validate(nx, ny, dx, dy, p);
  if (rc) return rc;
  work_t w;
  rc = work_alloc(&w, nx, ny, dx, dy, p, b, h, hu, hv);
  if (rc) return rc;
  if (max_speeds(&w.g, w.U0.h, w.U0.hu, w.U0.hv, &st->alpha_x, &st->alpha_y)) rc = OR_ENONFINITE;
  st->mass = total_mass(&w.g, w.U0.h);
  st->runup_now = runup_now(&w.g, w.b, w.U0.h);
  if (st->runup_now > st->runup_max) st->runup_max = st->runup_now;
  free(w.mem);
  return rc;
}

/* One evaluation of the spatial operator L of (7) at time t (dt only enters
 * the friction cap), split with the speeds (*ax, *ay) if use_given, else with
 * the wave speeds of the given state, which are returned in *ax, *ay.  Writes
 * the interior L arrays and returns the edge mass flux through *edge_flux. */
static int operator_once(int nx, int ny, double dx, double dy, const or_params *p, const double *b,
                         const double *h, const double *hu, const double *hv, double t, double dt,
                         double *Lh, double *Lhu, double *Lhv, int use_given, double *ax, double *ay,
                         double *edge_flux) {
  int rc = validate(nx, ny, dx, dy, p);
  if (rc) return rc;
  work_t w;
  rc = work_alloc(&w, nx, ny, dx, dy, p, b, h, hu, hv);
  if (rc) return rc;
  fill_state_ghosts(&w.g, w.b, w.U0.h, w.U0.hu, w.U0.hv, t);
  double sx, sy;
  if (max_speeds(&w.g, w.U0.h, w.U0.hu, w.U0.hv, &sx, &sy)) {
    free(w.mem);
    return OR_ENONFINITE;
  }
  if (use_given) {
    sx = *ax;
    sy = *ay;
  }
  rc = operator_L(&w.g, w.b, w.U0.h, w.U0.hu, w.U0.hv, sx, sy, dt, Lh, Lhu, Lhv, edge_flux);
  *ax = sx;
  *ay = sy;
  free(w.mem);
  return rc;
}

/* L of (7) with the state's own wave speeds (returned in alpha2[0..1]). */
int or_operator(int nx, int ny, double dx, double dy, const or_params *p, const double *b,
                const double *h, const double *hu, const double *hv, double t, double dt,
                double *Lh, double *Lhu, double *Lhv, double *alpha2, double *edge_flux) {
  double ax = 0.0, ay = 0.0;
  int rc = operator_once(nx, ny, dx, dy, p, b, h, hu, hv, t, dt, Lh, Lhu, Lhv, 0, &ax, &ay, edge_flux);
  if (alpha2) {
    alpha2[0] = ax;
    alpha2[1] = ay;
  }
  return rc;
}

/* L of (7) split with given speeds ax, ay (the fused-step variant's stages). */
int or_operator_split(int nx, int ny, double dx, double dy, const or_params *p, const double *b,
                      const double *h, const double *hu, const double *hv, double t, double dt,
                      double ax, double ay, double *Lh, double *Lhu, double *Lhv, double *edge_flux) {
  if (!(ax >= 0.0) || !(ay >= 0.0)) return OR_EINVAL;
  return operator_once(nx, ny, dx, dy, p, b, h, hu, hv, t, dt, Lh, Lhu, Lhv, 1, &ax, &ay, edge_flux);
}

/* The post-stage rule alone (for pins): applies to the state h, hu, hv
 * [ny][nx] (in/out) exactly what every RK stage applies after its update --
 * h < 0 -> 0, no momentum below h_dry, the film velocity desingularisation
 * below h_film -- and returns the depth it added in *added (m, summed over
 * cells; not multiplied by the cell area). */
int or_post_stage(int nx, int ny, const or_params *p, double *h, double *hu, double *hv,
                  double *added) {
  int rc = validate(nx, ny, 1.0, 1.0, p);
  if (rc) return rc;
  double *zero = (double *)calloc((size_t)nx * ny, sizeof(double));
  if (!zero) return OR_ENOMEM;
  work_t w;
  rc = work_alloc(&w, nx, ny, 1.0, 1.0, p, zero, h, hu, hv);
  free(zero);
  if (rc) return rc;
  double a = post_rule(&w.g, w.U0.h, w.U0.hu, w.U0.hv);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = ix(&w.g, i, j), o = (size_t)j * nx + i;
      h[o] = w.U0.h[c];
      hu[o] = w.U0.hu[c];
      hv[o] = w.U0.hv[c];
    }
  if (added) *added = a;
  free(w.mem);
  return OR_OK;
}

/* WENO5-JS value at the right face of v[2] and its weights (for pins). */
double or_weno5(const double *v, double eps, double *w) {
  double ww[3];
  double r = weno5(v, eps, ww);
  if (w) {
    w[0] = ww[0];
    w[1] = ww[1];
    w[2] = ww[2];
  }
  return r;
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
