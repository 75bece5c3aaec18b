"""Pins of the oracle's fused-step variant (one splitting speed per step).

The paper evaluates the global Lax-Friedrichs speed alpha of Eq. (6) before
every RK stage of Eq. (8).  The fused-step variant splits all three stages of
a step with alpha_margin x the alpha of U^n, so that a step depends on U^n and
the bed alone.  These tests tie the variant to the paper's (pinned) step and
to what does not depend on the splitting speed: the CFL step, the
well-balanced lake at rest and conservation.  Where alpha drifts during a
run the variant lags it by up to a step, a time error of first order (in a
term scaled by the splitting's dissipation) beside the third order of
SSP-RK3, which the paper's step keeps (Eq. (8)); both are pinned here.
"""
import dataclasses
import math

import numpy as np

import oracle
import workloads as W


def _cfl_dt(sc, h, hu, hv):
    wet = h >= sc.h_dry
    hs = np.where(wet, h, 1.0)
    c = np.where(wet, np.sqrt(sc.g * np.maximum(h, 0.0)), 0.0)
    ax = np.max(np.where(wet, np.abs(hu / hs), 0.0) + c)
    ay = np.max(np.where(wet, np.abs(hv / hs), 0.0) + c)
    return sc.cfl / (ax / sc.dx + ay / sc.dy)


def _hole_and_hump(n=48):
    """Still water over a flat 10 m bed with a 20 m deep hole in one corner
    and a moving mound of compact support (radius 8 cells) in the opposite
    one, more than 9 cells apart.  One RK3 step reaches 3 x 3 cells, so the
    hole, where the fastest speed sqrt(g 20) lies, stays at rest through the
    step and every stage's alpha equals that of U^n."""
    b = np.full((n, n), -10.0)
    b[2:6, 2:6] = -20.0
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    r = np.hypot(X - (n - 12), Y - (n - 12))
    eta = np.where(r < 8.0, 0.05 * np.cos(np.pi * r / 16.0) ** 2, 0.0)
    h = eta - b
    hu = 0.4 * eta * h
    hv = -0.3 * eta * h
    return W.Scenario("hole_and_hump", 1.0, 1.0, b, h, hu, hv)


def _run(sc, steps):
    sim = oracle.Simulation(sc)
    sim.step(steps)
    return sim


def test_variant_is_the_papers_step_while_the_speeds_hold():
    sc = _hole_and_hump()
    paper = _run(sc, 1)
    fused = _run(dataclasses.replace(sc, alpha_margin=1.0), 1)
    assert fused.diag()["last_dt"] == paper.diag()["last_dt"]
    assert np.abs(paper.h - sc.h).max() > 1e-4  # the mound moved
    for a, b in ((paper.h, fused.h), (paper.hu, fused.hu), (paper.hv, fused.hv)):
        assert np.abs(a - b).max() <= 1e-13
    assert fused.diag()["alpha_x"] == paper.diag()["alpha_x"]


def test_variant_step_is_eq8_with_the_start_speed_in_every_stage():
    # the variant's step composed by hand from Eq. (8): the spatial operator of
    # Eq. (7) (pinned against the PDE) split with margin x alpha(U^n) in all
    # three stages, at the stage times t, t + dt, t + dt/2 (inflow ghosts), and
    # the post-stage rule (pinned against Kurganov-Petrova) after each stage;
    # a coastal DEM with inflow, friction and a dry shore, after 30 paper steps
    base = W.coastal_dem(n=64, dx=40.0, steps=0)
    warm = _run(base, 30)
    margin = 1.3
    sc = dataclasses.replace(base, h=warm.h, hu=warm.hu, hv=warm.hv, t0=warm.t, alpha_margin=margin)
    t0 = sc.t0
    U0 = (sc.h, sc.hu, sc.hv)
    ax, ay = oracle.operator(sc, t0, 0.0)[3]
    dt = sc.cfl / (ax / sc.dx + ay / sc.dy)
    speeds = (margin * ax, margin * ay)

    def stage(U, t, w0, w1):
        L = oracle.operator(sc, t, dt, *U, speeds=speeds)[:3]
        V = [w0 * u0 + w1 * (u + dt * l) for u0, u, l in zip(U0, U, L)]
        return oracle.post_stage(sc, *V)[:3]

    U1 = stage(U0, t0, 0.0, 1.0)
    U2 = stage(U1, t0 + dt, 0.75, 0.25)
    U3 = stage(U2, t0 + 0.5 * dt, 1.0 / 3.0, 2.0 / 3.0)
    sim = _run(sc, 1)
    assert sim.diag()["last_dt"] == dt
    assert (sim.h == 0).any() and (sim.h > 0).any()
    for got, want in zip((sim.h, sim.hu, sim.hv), U3):
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    # and the paper's per-stage speeds would have given another step
    paper = _run(dataclasses.replace(sc, alpha_margin=0.0), 1)
    assert np.abs(paper.hu - sim.hu).max() > 1e-6


def test_variant_keeps_the_speed_of_the_steps_start_where_the_paper_updates_it():
    # dam break: the flow speeds up within the step, so the paper's stages
    # split with larger speeds than the variant's; the two agree to within the
    # size of that change, and both conserve mass between walls
    sc = W.dam_break(nx=200, ny=4)
    paper = _run(sc, 1)
    fused = _run(dataclasses.replace(sc, alpha_margin=1.0), 1)
    assert fused.diag()["last_dt"] == paper.diag()["last_dt"] == _cfl_dt(sc, sc.h, sc.hu, sc.hv)
    d = max(np.abs(paper.hu - fused.hu).max(), np.abs(paper.h - fused.h).max())
    assert 1e-9 < d < 1e-2
    m0 = sc.h.sum() * sc.dx * sc.dy
    for s in (paper, fused):
        assert abs(s.diag()["mass"] - m0) <= 1e-13 * m0


def test_margin_scales_the_splitting_speed_but_not_the_time_step():
    rng = np.random.default_rng(31)
    ny, nx, dx, dy = 20, 36, 2.0, 3.0
    b = -1.0 + 0.2 * rng.standard_normal((ny, nx))
    b[5:9, 10:14] = 0.5  # a dry island
    h = np.maximum(0.1 - b + 0.02 * rng.standard_normal((ny, nx)), 0.0)
    hu = np.where(h > 0, 0.3 * rng.standard_normal((ny, nx)) * h, 0.0)
    hv = np.where(h > 0, 0.2 * rng.standard_normal((ny, nx)) * h, 0.0)
    sc = W.Scenario("margin", dx, dy, b, h, hu, hv)
    one = _run(dataclasses.replace(sc, alpha_margin=1.0), 1)
    wide = _run(dataclasses.replace(sc, alpha_margin=1.5), 1)
    want = _cfl_dt(sc, h, hu, hv)
    assert abs(wide.diag()["last_dt"] - want) <= 1e-13 * want
    assert wide.diag()["last_dt"] == one.diag()["last_dt"]
    assert np.abs(wide.hu - one.hu).max() > 1e-6  # the wider splitting acts
    m0 = h.sum() * dx * dy
    for s in (one, wide):
        d = s.diag()
        assert abs(d["mass"] - d["clamp_mass"] - m0) <= 1e-13 * m0


def test_variant_keeps_a_lake_with_islands_at_rest_at_any_margin():
    sc = W.lake_at_rest(32, 32, eta0=0.5, depth=10.0, rms=2.0, islands=True)
    wet = sc.h > 0
    for m in (1.0, 1.5, 3.0):
        sim = _run(dataclasses.replace(sc, alpha_margin=m), 100)
        assert np.abs((sim.h + sc.b - 0.5)[wet]).max() <= 1e-12
        assert sim.h[~wet].max() <= 1e-12
        assert np.abs(sim.hu).max() <= 1e-11 and np.abs(sim.hv).max() <= 1e-11


def _smooth_periodic(margin):
    n = 48
    d = 1.0 / n
    c = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(c, c)
    h = 1.0 + 0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    hu = 0.2 * np.cos(2 * np.pi * (X + Y))
    hv = 0.1 * np.sin(2 * np.pi * (X - 2 * Y))
    return W.Scenario("smooth", d, d, np.zeros_like(h), h, hu, hv, bc=(W.PERIODIC,) * 4, alpha_margin=margin)


def _fixed_step_runs(sc, T=0.04, first=40, count=4):
    sols = []
    for k in range(count):
        steps = first * 2 ** k
        sim = _run(dataclasses.replace(sc, fixed_dt=T / steps), steps)
        assert math.isclose(sim.t, T, rel_tol=1e-12)
        sols.append(np.concatenate([sim.h.ravel(), sim.hu.ravel(), sim.hv.ravel()]))
    return sols


def test_rk3_step_is_third_order_in_time():
    # Eq. (8) with the per-stage alpha: fixed steps dt, dt/2, dt/4, dt/8 to the
    # same time on a smooth periodic wave; the differences of successive
    # solutions fall by 2^3
    sols = _fixed_step_runs(_smooth_periodic(0.0))
    e = [np.abs(sols[k] - sols[k + 1]).max() for k in range(3)]
    for k in range(2):
        assert 7.0 < e[k] / e[k + 1] < 9.0, e


def test_variant_lags_alpha_by_up_to_a_step_a_first_order_time_error():
    # the variant's operator within a step is that of alpha(U^n): it lags the
    # state's alpha, which the paper follows stage by stage.  On the smooth
    # wave (alpha drifts slowly) the two differ by O(dt): halving dt halves
    # the difference, which stays far below the wave's amplitude
    paper = _fixed_step_runs(_smooth_periodic(0.0), count=3)
    fused = _fixed_step_runs(_smooth_periodic(1.0), count=3)
    d = [np.abs(p - f).max() for p, f in zip(paper, fused)]
    assert d[0] < 1e-6, d
    for k in range(2):
        assert 1.8 < d[k] / d[k + 1] < 2.2, d


def test_margin_below_one_is_rejected():
    sc = W.gaussian_hump(n=16)
    for m in (0.5, -1.0, float("nan")):
        try:
            oracle.Simulation(dataclasses.replace(sc, alpha_margin=m)).step(1)
        except oracle.OracleError as e:
            assert e.code == oracle.EINVAL
        else:
            raise AssertionError("alpha_margin %r accepted" % m)
