"""Closed-form solutions and definitions the tests compare the oracle to.

Each is written from its own source (the paper's printed formula or a
textbook definition), independently of the oracle's code.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import polynomial as P

G = 9.81


def stoker_cm(h_l: float, h_r: float, g: float = G) -> float:
    """Root c_m of Eq. (15) of Section 2.1 on (sqrt(g h_r), sqrt(g h_l)), by bisection."""
    def f(c):
        return -8.0 * g * h_r * c * c * (math.sqrt(g * h_l) - c) ** 2 + (c * c - g * h_r) ** 2 * (c * c + g * h_r)
    lo, hi = math.sqrt(g * h_r), math.sqrt(g * h_l)
    flo = f(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def stoker(x: np.ndarray, t: float, x0: float, h_l: float, h_r: float, g: float = G):
    """Wet dam break, Eqs. (11)-(15) of Section 2.1.  Returns (h, x3)."""
    cm = stoker_cm(h_l, h_r, g)
    x1 = x0 - t * math.sqrt(g * h_l)
    x2 = x0 + t * (2.0 * math.sqrt(g * h_l) - 3.0 * cm)
    x3 = x0 + t * (2.0 * cm * cm * (math.sqrt(g * h_l) - cm)) / (cm * cm - g * h_r)
    h = np.where(x <= x1, h_l,
                 np.where(x <= x2, 4.0 / (9.0 * g) * (math.sqrt(g * h_l) - (x - x0) / (2.0 * t)) ** 2,
                          np.where(x <= x3, cm * cm / g, h_r)))
    return h, x3


def thacker(x: np.ndarray, t: float, L: float, a: float, h0: float, g: float = G):
    """Planar parabolic bowl, Eq. (18) of Section 2.2, wet where the formula is
    positive (the printed x1(t) carries a sign slip; the interval used is the
    one on which Eq. (18) is positive, which matches Eq. (17) at t = 0).
    Returns (h, u) with u = (omega/2) sin(omega t) in the wet region."""
    om = math.sqrt(2.0 * g * h0) / a
    s = (2.0 * x - L) / (2.0 * a) + math.cos(om * t) / (2.0 * a)
    h = np.maximum(-h0 * (s * s - 1.0), 0.0)
    u = np.where(h > 0, 0.5 * om * math.sin(om * t), 0.0)
    return h, u


def manning_normal_discharge(h: float, slope: float, n: float) -> float:
    """Eq. (19) of Section 2.3: hu = sqrt(S) h^(5/3) / n."""
    return math.sqrt(slope) * h ** (5.0 / 3.0) / n


def synolakis_runup(H_over_d: float, cot_beta: float, d: float) -> float:
    """Runup law of a non-breaking solitary wave on a plane beach
    (Synolakis 1987): R/d = 2.831 sqrt(cot beta) (H/d)^(5/4)."""
    return d * 2.831 * math.sqrt(cot_beta) * H_over_d ** 1.25


def standing_wave_on_slope(r: np.ndarray, t: float, amp: float, L: float, slope: float, g: float = G):
    """Linear SWE on still-water depth slope * r (r = distance from the
    shoreline, x = L - r) with a wall at r = L: eta = amp J0(xi) cos(w t),
    xi = 2 w sqrt(r/(g slope)), solves eta_tt = g slope (r eta_r)_r (Bessel's
    equation of order 0 in xi), and the wall condition eta_r(L) = 0 asks
    J1(xi_L) = 0, so 2 w sqrt(L/(g slope)) = j11.  The x-velocity follows
    from u_t = -g eta_x = g eta_r: u = (g amp / w) dJ0(xi)/dr sin(w t), with
    dJ0/dr = -J1(xi) w / sqrt(g slope r).  Returns (eta, hu = slope r u, w)."""
    from scipy.special import j0, j1, jn_zeros
    j11 = float(jn_zeros(1, 1)[0])
    w = 0.5 * j11 * math.sqrt(g * slope / L)
    rr = np.maximum(r, 0.0)
    xi = 2.0 * w * np.sqrt(rr / (g * slope))
    eta = amp * j0(xi) * math.cos(w * t)
    # slope r dJ0/dr = -J1(xi) w slope r / sqrt(g slope r) = -J1(xi) w sqrt(slope r / g)
    hu = (g * amp / w) * (-j1(xi) * w * np.sqrt(slope * rr / g)) * math.sin(w * t)
    return eta, hu, w


def golden(name: str) -> dict:
    """Values of a cited text fixture under tests/golden/ ("key value" lines;
    '#' starts a comment)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error of Eq. (9)."""
    return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))


def rel_linf(a: np.ndarray, ref: np.ndarray) -> float:
    """Relative L-infinity error of Eq. (9)."""
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


# ---------------------------------------------------------- WENO5 definitions
def _cell_average_poly(values, cells):
    """Quadratic q with (1/dx) int_{cell} q = value for each cell (dx = 1),
    cells given by their centre offsets."""
    A = np.zeros((3, 3))
    for r, c in enumerate(cells):
        lo, hi = c - 0.5, c + 0.5
        for k in range(3):
            A[r, k] = (hi ** (k + 1) - lo ** (k + 1)) / (k + 1)
    return np.linalg.solve(A, np.asarray(values, dtype=np.float64))


def jiang_shu_beta(v):
    """Smoothness indicators from their definition: for each 3-cell stencil,
    the sum over l = 1, 2 of dx^(2l-1) times the integral over the centre cell
    of the squared l-th derivative of the stencil's reconstruction polynomial
    (cell centres at -2..2, reconstruction cell = centre 0, dx = 1)."""
    out = []
    for k in range(3):
        cells = [-2 + k, -1 + k, k]
        vals = v[k:k + 3]
        q = _cell_average_poly(vals, cells)
        total = 0.0
        for l in (1, 2):
            d = P.polyder(q, l)
            sq = P.polymul(d, d)
            I = P.polyint(sq)
            total += P.polyval(0.5, I) - P.polyval(-0.5, I)
        out.append(total)
    return np.array(out)


def stencil_face_value(v):
    """Value at x = +1/2 of each stencil's reconstruction polynomial."""
    out = []
    for k in range(3):
        q = _cell_average_poly(v[k:k + 3], [-2 + k, -1 + k, k])
        out.append(P.polyval(0.5, q))
    return np.array(out)
