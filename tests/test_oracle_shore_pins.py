"""Pins of the oracle's shoreline variant (shore = 1): the faces whose WENO
stencil holds a dry cell take the first-order hydrostatic reconstruction of
Audusse et al. (2004), carried into the still-depth form of the bed terms.

The paper is silent on wet/dry fronts.  What the variant must do is fixed
by the mathematics: a lake at rest stays at rest beside dry land at any level
at or below z_ref; away from dry cells the step is the paper's step bit for
bit; the shoreline of a small standing wave on a beach follows the linear
Carrier-Greenspan solution; Thacker's bowl and the Synolakis runup law hold;
depth stays non-negative without the clamp adding mass.
"""
import dataclasses
import math

import numpy as np

import oracle
import workloads as W
from tests import analytic as A
from tests.test_oracle_pins import _standing_wave_case


def _run(sc, steps):
    sim = oracle.Simulation(sc)
    sim.step(steps)
    return sim


def _two_lakes(z_ref=0.5):
    # two lakes at 0.5 m and -0.5 m over a rough bed, parted by a dry ridge,
    # with islands in both: z_ref at the higher level
    n = 48
    rng = np.random.default_rng(5)
    b = -6.0 + 0.8 * rng.standard_normal((n, n))
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    b[:, 22:26] = 2.0  # the ridge
    b[np.hypot(X - 10, Y - 12) < 4] = 1.5  # islands
    b[np.hypot(X - 36, Y - 30) < 5] = 0.2
    level = np.where(X < 24, 0.5, -0.5)
    h = np.maximum(level - b, 0.0)
    z = np.zeros_like(b)
    return W.Scenario("two_lakes", 1.0, 1.0, b, h, z, z.copy(), z_ref=z_ref), level


def test_lakes_at_rest_at_and_below_z_ref_beside_dry_land_are_exact():
    sc, level = _two_lakes()
    wet = sc.h > 0
    assert (~wet).sum() > 100 and wet.sum() > 1000
    sim = _run(dataclasses.replace(sc, shore=1), 200)
    assert np.abs((sim.h + sc.b - level)[wet]).max() <= 1e-12
    assert sim.h[~wet].max() == 0.0
    assert np.abs(sim.hu).max() <= 1e-11 and np.abs(sim.hv).max() <= 1e-11
    assert sim.diag()["clamp_mass"] == 0.0
    # the paper's scheme is not balanced for the lower lake's shores
    paper = _run(sc, 200)
    assert np.abs((paper.h + sc.b - level)[wet]).max() > 1e-3


def test_away_from_dry_cells_the_step_is_the_papers():
    for sc in (W.gaussian_hump(n=64), W.dam_break(nx=200, ny=4)):
        a = _run(sc, 40)
        b = _run(dataclasses.replace(sc, shore=1), 40)
        for x, y in ((a.h, b.h), (a.hu, b.hu), (a.hv, b.hv)):
            assert np.array_equal(x, y)


def test_faces_change_only_within_a_stencil_of_dry_cells():
    # one dry cell on a moving wet state: the operator differs from the
    # paper's only at cells whose faces' stencils reach it (3 cells along its
    # row and column), and there it does differ
    rng = np.random.default_rng(2)
    n = 24
    b = -2.0 + 0.1 * rng.standard_normal((n, n))
    b[12, 9] = 1.0
    h = np.maximum(0.2 * rng.standard_normal((n, n)) * 0.1 - b, 0.0)
    assert (h == 0).sum() == 1
    hu = np.where(h > 0, 0.3 * rng.standard_normal((n, n)), 0.0)
    hv = np.where(h > 0, 0.3 * rng.standard_normal((n, n)), 0.0)
    sc = W.Scenario("one_dry", 1.0, 1.0, b, h, hu, hv)
    La = oracle.operator(sc)[:3]
    Lb = oracle.operator(dataclasses.replace(sc, shore=1))[:3]
    diff = np.zeros((n, n), bool)
    for x, y in zip(La, Lb):
        diff |= x != y
    J, I = np.nonzero(diff)
    assert diff.any()
    for j, i in zip(J, I):
        assert (j == 12 and abs(i - 9) <= 3) or (i == 9 and abs(j - 12) <= 3), (j, i)
    assert diff[12, 9 - 3:9 + 4].sum() >= 5 and diff[12 - 3:12 + 4, 9].sum() >= 5


def test_standing_wave_shoreline_follows_linear_theory():
    # the case whose shoreline the paper's scheme misses by 9.7 % of A at T/2
    # (R5'): with the shoreline faces the wet side follows the linear
    # Carrier-Greenspan solution to 1 % of A over a whole period (observed
    # 0.57 % at T/2, 0.72 % at T), the offshore half to 1e-4 A until T/4, and
    # the clamp adds nothing
    sc, amp, L, slope, r, T = _standing_wave_case()
    sim = oracle.Simulation(dataclasses.replace(sc, shore=1))
    wet, off = r > 0.0, r >= 0.5 * L
    for frac in (0.125, 0.25, 0.5, 1.0):
        sim.run_until(frac * T)
        eta = sim.h[1] + sc.b[1]
        ex, _, _ = A.standing_wave_on_slope(r, frac * T, amp, L, slope)
        assert np.sqrt(np.mean((eta[wet] - ex[wet]) ** 2)) <= 0.01 * amp, frac
        if frac <= 0.25:
            assert np.sqrt(np.mean((eta[off] - ex[off]) ** 2)) <= 1e-4 * amp
    assert sim.diag()["clamp_mass"] == 0.0


def test_thacker_bowl_with_shoreline_faces():
    sc = dataclasses.replace(W.parabolic_bowl(), shore=1)
    sim = oracle.Simulation(sc)
    x = (np.arange(sc.nx) + 0.5) * sc.dx
    om = math.sqrt(2 * 9.81 * 1.0) / 100.0
    vt = A.golden("verification_times.txt")
    for t in (vt["bowl_t1"], vt["bowl_t2"], 2 * math.pi / om):
        sim.run_until(t)
        ha, _ = A.thacker(x, t, 400.0, 100.0, 1.0)
        assert A.rel_l2(sim.h[0], ha) <= 1e-3  # observed 1.7e-4 after a period (3.2e-3 without)
        wet_num, wet_ana = x[sim.h[0] > 1e-3], x[ha > 1e-3]
        assert abs(wet_num.min() - wet_ana.min()) <= sc.dx
        assert abs(wet_num.max() - wet_ana.max()) <= sc.dx
    assert sim.diag()["clamp_mass"] == 0.0


def test_solitary_wave_runup_with_shoreline_faces():
    sc = dataclasses.replace(W.planar_beach(ny=4, manning_n=0.0), shore=1)
    sim = oracle.Simulation(sc)
    sim.run_until(70.0)
    law = A.synolakis_runup(0.02, 20.0, 10.0)
    assert abs(sim.diag()["runup_max"] - law) / law <= 0.10  # observed -2.9 %


def test_mass_with_wet_dry_and_friction():
    # a violently stirred lake with islands and a coastal DEM with inflow:
    # mass - clamp mass = initial (+ edge inflow) to round-off, no negative depth
    sc = W.lake_at_rest(32, 32, eta0=0.5, depth=10.0, rms=2.0, islands=True)
    rng = np.random.default_rng(3)
    sc.hu = np.where(sc.h > 0, 2.0 * rng.standard_normal(sc.h.shape), 0.0)
    sc.hv = np.where(sc.h > 0, 2.0 * rng.standard_normal(sc.h.shape), 0.0)
    m0 = sc.h.sum()
    sim = oracle.Simulation(dataclasses.replace(sc, shore=1, manning_n=0.03))
    for _ in range(20):
        sim.step(5)
        assert sim.h.min() >= 0.0
    d = sim.diag()
    assert abs(d["mass"] - d["clamp_mass"] - m0) <= 1e-13 * m0
    dem = dataclasses.replace(W.coastal_dem(n=64, dx=100.0, t0=500.0), shore=1)
    sim = oracle.Simulation(dem)
    m0 = dem.h.sum() * dem.dx * dem.dy
    sim.step(40)
    d = sim.diag()
    assert abs(d["mass"] - d["clamp_mass"] - d["boundary_mass"] - m0) <= 1e-12 * m0
