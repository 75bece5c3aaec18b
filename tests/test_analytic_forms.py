"""The closed forms the pins use, checked against properties that do not come
from the same formula: conservation laws, jump conditions and PDE residuals.
A mistyped closed form fails here before it can make a pin pass or fail."""
import math

import numpy as np
import pytest

from tests import analytic as A

G = A.G
trapezoid = getattr(np, "trapezoid", None) or np.trapz  # numpy 1 and 2


def test_stoker_state_satisfies_the_jump_conditions_and_conserves_volume():
    h_l, h_r, x0, t = 2.0, 1.0, 50.0, 2.5
    cm = A.stoker_cm(h_l, h_r)
    assert math.sqrt(G * h_r) < cm < math.sqrt(G * h_l)
    h_m = cm * cm / G
    u_m = 2.0 * (math.sqrt(G * h_l) - cm)  # left Riemann invariant through the rarefaction
    x = np.linspace(0.0, 100.0, 200001)
    h, x3 = A.stoker(x, t, x0, h_l, h_r)
    s = (x3 - x0) / t
    # Rankine-Hugoniot at the shock between (h_m, u_m) and (h_r, 0)
    assert s * (h_m - h_r) == pytest.approx(h_m * u_m, rel=1e-10)
    assert s * h_m * u_m == pytest.approx(h_m * u_m * u_m + 0.5 * G * (h_m * h_m - h_r * h_r), rel=1e-10)
    # plateau and rarefaction meet continuously; the volume is that of t = 0
    x2 = x0 + t * (2.0 * math.sqrt(G * h_l) - 3.0 * cm)
    assert A.stoker(np.array([x2 - 1e-9]), t, x0, h_l, h_r)[0][0] == pytest.approx(h_m, rel=1e-6)
    v0 = h_l * x0 + h_r * (100.0 - x0)  # the volume at t = 0 on [0, 100]
    assert trapezoid(h, x) == pytest.approx(v0, rel=2e-5)


def test_thacker_bowl_solves_the_shallow_water_equations():
    # bed of the planar bowl b = h0 ((2x - L)/(2a))^2 - h0; in the wet region
    # h_t + (h u)_x = 0 and u_t + u u_x + g (h + b)_x = 0
    L, a, h0 = 400.0, 100.0, 1.0
    x = np.linspace(0.0, L, 4001)
    b = h0 * ((2.0 * x - L) / (2.0 * a)) ** 2 - h0
    om = math.sqrt(2.0 * G * h0) / a
    for t in (1.3, 3.5, 12.5):
        e = 1e-4
        h, u = A.thacker(x, t, L, a, h0)
        hp, up = A.thacker(x, t + e, L, a, h0)
        hm, um = A.thacker(x, t - e, L, a, h0)
        wet = (hm > 0.05) & (h > 0.05) & (hp > 0.05)
        wet[:2] = wet[-2:] = False
        dxs = x[1] - x[0]
        ht = (hp - hm) / (2 * e)
        qx = np.gradient(h * u, dxs)
        ut = (up - um) / (2 * e)
        etax = np.gradient(h + b, dxs)
        assert np.abs((ht + qx)[wet]).max() <= 1e-6
        assert np.abs((ut + u * np.gradient(u, dxs) + G * etax)[wet]).max() <= 1e-6
        assert np.all(h >= 0)
    # the volume is the same at every time: 4/3 h0 a (a parabola over 2a)
    for t in np.linspace(0.0, 2 * math.pi / om, 7):
        assert trapezoid(A.thacker(x, t, L, a, h0)[0], x) == pytest.approx(4.0 / 3.0 * h0 * a, rel=1e-5)


def test_manning_normal_discharge_balances_gravity_and_friction():
    for h, slope, n in ((0.5, 0.05, 0.033), (2.0, 0.001, 0.025)):
        q = A.manning_normal_discharge(h, slope, n)
        # steady uniform flow: g h S = g n^2 q |q| / h^(7/3)
        assert G * h * slope == pytest.approx(G * n * n * q * abs(q) / h ** (7.0 / 3.0), rel=1e-12)


def test_synolakis_law_at_the_planar_beach_case():
    # R/d = 2.831 sqrt(cot beta) (H/d)^(5/4): 0.952 m for d = 10 m, H/d = 0.02, cot beta = 20
    assert A.synolakis_runup(0.02, 20.0, 10.0) == pytest.approx(0.952, abs=5e-4)


def test_standing_wave_solves_the_linear_equations_with_a_wall():
    pytest.importorskip("scipy")
    L, slope, amp = 1000.0, 0.05, 0.002
    r = np.linspace(1.0, L, 20001)  # r = L - x, depth slope r
    dr = r[1] - r[0]
    eta, hu, w = A.standing_wave_on_slope(r, 0.7, amp, L, slope)
    e = 1e-3
    eta_p, hu_p, _ = A.standing_wave_on_slope(r, 0.7 + e, amp, L, slope)
    eta_m, hu_m, _ = A.standing_wave_on_slope(r, 0.7 - e, amp, L, slope)
    inner = slice(2, -2)
    # continuity eta_t + (hu)_x = 0 and momentum (hu)_t + g (slope r) eta_x = 0, with d/dx = -d/dr
    cont = (eta_p - eta_m) / (2 * e) - np.gradient(hu, dr)
    mom = (hu_p - hu_m) / (2 * e) - G * slope * r * np.gradient(eta, dr)
    scale_c = np.abs((eta_p - eta_m) / (2 * e)).max()
    scale_m = np.abs((hu_p - hu_m) / (2 * e)).max()
    assert np.abs(cont[inner]).max() <= 1e-4 * scale_c
    assert np.abs(mom[inner]).max() <= 1e-4 * scale_m
    # no flux through the wall at r = L
    assert abs(hu[-1]) <= 1e-6 * np.abs(hu).max()
