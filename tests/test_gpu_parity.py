"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances: FP64 GPU max |d eta| <= 1e-10 m; FP32 relative L2 of the surface
anomaly eta~ (h+b on wet cells, 0 on dry) <= 1e-4 and runup error <= 1 cm.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402


# compiled tile shapes (1..11); in FP64 the 32x64, 64x64, 64x48, 96x32 and
# 128x32 tiles need more shared memory than a CTA may use
ALL_TILES = list(range(1, 12))
FP64_TILES = [1, 2, 4, 10, 11]
FP64_TOO_BIG = [3, 5, 6, 7, 8, 9]


def stream():
    return torch.cuda.current_stream().cuda_stream


def eta_tilde(h, b, h_dry=1e-5):
    return np.where(h >= h_dry, h + b, 0.0)


def rel_l2(a, ref):
    return float(np.sqrt(((a - ref) ** 2).sum() / max((ref ** 2).sum(), 1e-300)))


def run_gpu(sc, steps, precision, tile=0):
    with swe.Solver(sc, precision=precision, stream=stream(), tile=tile) as s:
        s.step(steps)
        h, hu, hv = s.get_state()
        d = s.diagnostics()
        m = s.mass()
    return h, hu, hv, d, m


def run_oracle(sc, steps):
    sim = oracle.Simulation(sc)
    sim.step(steps)
    return sim


# ------------------------------------------------------------------ FP64
@pytest.mark.parametrize("tile", FP64_TOO_BIG)
def test_fp64_tile_that_does_not_fit_is_rejected(tile):
    # these shapes need more shared memory than a CTA may use in FP64
    with pytest.raises(swe.SweError) as ei:
        swe.Solver(W.gaussian_hump(n=32), precision=swe.F64, stream=stream(), tile=tile)
    assert ei.value.code == swe.EINVAL


@pytest.mark.parametrize("tile", FP64_TILES)
def test_fp64_hump_128(tile):
    sc = W.gaussian_hump()
    ref = run_oracle(sc, 200)
    h, hu, hv, d, (m, cm) = run_gpu(sc, 200, swe.F64, tile)
    assert np.abs(h - ref.h).max() <= 1e-10
    assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10
    assert d["steps"] == 200 and d["t"] == pytest.approx(ref.t, rel=1e-12)
    assert abs(m - ref.diag()["mass"]) <= 1e-11 * m


@pytest.mark.parametrize("shape", [(77, 45), (3, 3), (37, 4), (130, 97)])
@pytest.mark.parametrize("tile", FP64_TILES)
def test_fp64_ragged_random(shape, tile):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    sc = W.lake_at_rest(nx, ny, eta0=0.0, depth=4.0, rms=1.0, seed=nx + ny)
    sc.h = sc.h + 0.2 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.3 * rng.normal(size=sc.h.shape)
    sc.hv = 0.3 * rng.normal(size=sc.h.shape)
    sc.manning_n = 0.03
    ref = run_oracle(sc, 12)
    h, hu, hv, d, _ = run_gpu(sc, 12, swe.F64, tile)
    assert np.abs(h - ref.h).max() <= 1e-10
    assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10


def test_fp64_wet_dry_bowl_and_clamp_mass():
    sc = W.parabolic_bowl(nx=400, ny=8)
    ref = run_oracle(sc, 300)
    h, hu, hv, d, (m, cm) = run_gpu(sc, 300, swe.F64)
    assert np.abs(h - ref.h).max() <= 1e-10
    assert cm == pytest.approx(ref.diag()["clamp_mass"], rel=1e-9, abs=1e-12)


def test_fp64_periodic_manning():
    from tests.analytic import manning_normal_discharge
    qn = manning_normal_discharge(0.5, 1 / 20, 0.033)
    sc = W.manning_slope(nx=64, ny=8, q=0.8 * qn)
    ref = run_oracle(sc, 300)
    h, hu, hv, d, _ = run_gpu(sc, 300, swe.F64)
    assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(h - ref.h).max() <= 1e-10


def test_fp64_inflow_and_boundary_mass():
    sc = W.coastal_dem(n=96, dx=150.0, t0=500.0)
    ref = run_oracle(sc, 40)
    h, hu, hv, d, (m, cm) = run_gpu(sc, 40, swe.F64)
    assert np.abs(h - ref.h).max() <= 1e-10
    rd = ref.diag()
    assert d["boundary_mass"] == pytest.approx(rd["boundary_mass"], rel=1e-9)
    assert d["t"] == pytest.approx(rd["t"], rel=1e-13)


def test_fp64_planar_beach_full_5000_steps():
    # 2048 x 64 on the GPU; the y-uniform problem is row-for-row the same as
    # the oracle's 2048 x 4 run (walls in y keep it exactly one-dimensional)
    sc = W.planar_beach()
    sc4 = W.planar_beach(ny=4)
    ref = run_oracle(sc4, 5000)
    h, hu, hv, d, _ = run_gpu(sc, 5000, swe.F64)
    eta_ref = ref.h[0] + sc4.b[0]
    assert np.abs(h + sc.b - eta_ref[None, :]).max() <= 1e-10
    assert d["runup_max"] == pytest.approx(ref.diag()["runup_max"], abs=1e-10)


def test_fp64_standing_wave_on_slope():
    # 2 mm standing wave over a 1:20 beach with dry land beyond the shore
    sc = W.standing_wave_slope(nx_sea=100, nx_land=20, dx=10.0, amp=0.002)
    ref = run_oracle(sc, 400)
    h, hu, hv, d, _ = run_gpu(sc, 400, swe.F64)
    assert np.abs((h + sc.b) - (ref.h + sc.b)).max() <= 1e-10
    assert np.abs(hu - ref.hu).max() <= 1e-10


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_fixed_time_step_hump_and_planar_beach(precision):
    # the paper's timed runs use a fixed dt of 5e-3 s (Tables 1-3): every step
    # takes exactly that dt and t accumulates it as the oracle's does; the hump
    # of config 1 for 200 steps and the planar beach of config 2 (wet/dry,
    # Manning friction; ny = 4, y-uniform) for 1000 steps
    cases = ((W.gaussian_hump(), 200), (W.planar_beach(ny=4), 1000))
    for base, steps in cases:
        sc = base.copy(fixed_dt=5e-3)
        ref = run_oracle(sc, steps)
        rd = ref.diag()
        h, hu, hv, d, _ = run_gpu(sc, steps, precision)
        assert d["steps"] == steps and d["last_dt"] == 5e-3 and d["t"] == rd["t"], sc.name
        if precision == swe.F64:
            assert np.abs(h - ref.h).max() <= 1e-10, sc.name
            assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10, sc.name
        else:
            assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4, sc.name
            assert rel_l2(hu, ref.hu) <= 1e-4, sc.name
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= (1e-10 if precision == swe.F64 else 0.01)


def _film_beach(nx=96, ny=24, seed=43):
    # a rough 1:40 beach with still water at 0 and, on land, a patchwork of
    # films of depth h_dry .. 3 h_film with random velocities: the post-stage
    # film rule (Kurganov-Petrova desingularisation below h_film) acts on
    # hundreds of cells in every stage
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5)[None, :] * np.ones((ny, 1))
    b = (x - nx / 2) / 40.0 + 0.02 * rng.standard_normal((ny, nx))
    h = np.maximum(-b, 0.0)
    land = h == 0.0
    film = land & (rng.random((ny, nx)) < 0.6)
    h[film] = np.exp(rng.uniform(np.log(1e-5), np.log(3e-3), size=film.sum()))
    u = rng.normal(size=(ny, nx)) * 0.3
    v = rng.normal(size=(ny, nx)) * 0.3
    sc = W.Scenario("film_beach", 1.0, 1.0, b, h, h * u, h * v, manning_n=0.02)
    return sc


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_thin_films_on_land(precision):
    sc = _film_beach()
    assert ((sc.h >= sc.h_dry) & (sc.h < sc.h_film)).sum() >= 400
    ref = run_oracle(sc, 30)
    h, hu, hv, d, (m, cm) = run_gpu(sc, 30, precision)
    if precision == swe.F64:
        assert np.abs(h - ref.h).max() <= 1e-10
        assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10
        assert cm == pytest.approx(ref.diag()["clamp_mass"], rel=1e-9, abs=1e-12)
    else:
        assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4
        assert rel_l2(hu, ref.hu) <= 1e-4 and rel_l2(hv, ref.hv) <= 1e-4


# ------------------------------------------------------------------ FP32
def test_fp32_standing_wave_on_slope():
    sc = W.standing_wave_slope(nx_sea=100, nx_land=20, dx=10.0, amp=0.002)
    ref = run_oracle(sc, 400)
    h, hu, hv, d, _ = run_gpu(sc, 400, swe.F32)
    assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4
    assert rel_l2(hu, ref.hu) <= 1e-4


@pytest.mark.parametrize("tile", ALL_TILES)
def test_fp32_hump_128(tile):
    sc = W.gaussian_hump()
    ref = run_oracle(sc, 200)
    h, hu, hv, d, _ = run_gpu(sc, 200, swe.F32, tile)
    e = rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b))
    assert e <= 1e-4


@pytest.mark.parametrize("shape", [(77, 45), (3, 3), (37, 4), (130, 97)])
@pytest.mark.parametrize("tile", ALL_TILES)
def test_fp32_ragged_random(shape, tile):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    sc = W.lake_at_rest(nx, ny, eta0=0.0, depth=4.0, rms=1.0, seed=nx + ny)
    sc.h = sc.h + 0.2 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.3 * rng.normal(size=sc.h.shape)
    sc.hv = 0.3 * rng.normal(size=sc.h.shape)
    sc.manning_n = 0.03
    ref = run_oracle(sc, 12)
    h, hu, hv, d, _ = run_gpu(sc, 12, swe.F32, tile)
    assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4
    assert rel_l2(hu, ref.hu) <= 1e-4 and rel_l2(hv, ref.hv) <= 1e-4


def test_fp32_planar_beach_against_fp64_oracle():
    sc = W.planar_beach()
    sc4 = W.planar_beach(ny=4)
    ref = oracle.Simulation(sc4)
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        for target in (5000, 8000):  # 8000 steps covers the maximum runup
            ref.step(target - ref.diag()["steps"])
            s.step(target - s.diagnostics()["steps"])
            h, hu, hv = s.get_state()
            d = s.diagnostics()
            et = eta_tilde(h, sc.b)
            er = eta_tilde(ref.h, sc4.b)[0][None, :].repeat(sc.ny, axis=0)
            assert rel_l2(et, er) <= 1e-4, target
            assert abs(d["runup_max"] - ref.diag()["runup_max"]) <= 0.01, target


def test_fp32_lake_at_rest_with_islands():
    sc = W.lake_at_rest(96, 64, eta0=0.5, depth=10.0, rms=2.0, islands=True)
    h, hu, hv, d, _ = run_gpu(sc, 500, swe.F32)
    wet = sc.h > 0
    assert np.abs((h + sc.b - 0.5)[wet]).max() <= 1e-5
    assert np.abs(hu).max() <= 1e-4 and np.abs(hv).max() <= 1e-4


def test_coastal_dem_full_size_against_the_oracle():
    # the bench's workload at its full size (4096^2: N-wave inflow, rough
    # shelf, land and shoreline, Manning friction), 10 steps, in the tile
    # shape the bench times (96x32) for FP32 and the autotuner's FP64 shape
    sc = W.coastal_dem()
    steps = 10
    ref = run_oracle(sc, steps)
    h64, hu64, _, d64, _ = run_gpu(sc, steps, swe.F64, tile=2)
    assert np.abs(h64 - ref.h).max() <= 1e-10  # eta = h + b, b shared
    assert d64["t"] == pytest.approx(ref.t, rel=1e-12)
    h, hu, hv, d, _ = run_gpu(sc, steps, swe.F32, tile=7)
    e = rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b))
    assert e <= 1e-4, e
    assert rel_l2(hu, ref.hu) <= 1e-4


# ------------------------------------------------------------- edge cases
def test_fp32_large_grid_rows_agree_and_match_the_oracle():
    # 16384 x 4096 cells (67 M): a y-uniform solitary wave on the 1:20 beach.
    # Far tile indices and tensor-copy coordinates: every row must stay equal
    # to row 0 bit for bit, and row 0 must match the FP64 oracle on 16384 x 4.
    big = W.planar_beach(nx=16384, ny=4096, manning_n=0.0)
    small = W.planar_beach(nx=16384, ny=4, manning_n=0.0)
    steps = 20
    ref = run_oracle(small, steps)
    h, hu, hv, d, _ = run_gpu(big, steps, swe.F32)
    assert np.all(h == h[0]) and np.all(hu == hu[0]) and not hv.any()
    assert rel_l2(eta_tilde(h[0], big.b[0]), eta_tilde(ref.h[0], small.b[0])) <= 1e-4
    assert rel_l2(hu[0], ref.hu[0]) <= 1e-4


def test_dry_still_domain_reports_einval():
    sc = W.lake_at_rest(16, 16, eta0=-100.0, depth=10.0, rms=1.0)
    assert sc.h.max() == 0.0
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.step(1)
        with pytest.raises(swe.SweError) as ei:
            s.sync()
        assert ei.value.code == swe.EINVAL


def test_nonfinite_state_is_reported():
    sc = W.gaussian_hump(n=32)
    sc.h[5, 7] = np.nan
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        with pytest.raises(swe.SweError) as ei:
            s.step(2)
            s.sync()
        assert ei.value.code == swe.ENONFINITE


def test_checkpoint_resume_is_bitwise():
    sc = W.planar_beach(nx=256, ny=8, steps=0)
    sc.manning_n = 0.025
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as a:
        a.step(60)
        ha, hua, hva = a.get_state()
        ta, _ = a.time()
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as b:
        b.step(25)
        st = b.get_state()
        t1, _ = b.time()
    sc2 = sc.copy(h=st[0], hu=st[1], hv=st[2], t0=t1)
    with swe.Solver(sc2, precision=swe.F32, stream=stream()) as c:
        c.step(35)
        hc, huc, hvc = c.get_state()
        tc, _ = c.time()
    assert np.array_equal(ha, hc) and np.array_equal(hua, huc) and np.array_equal(hva, hvc)
    assert ta == tc


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_diagnostic_volumes_are_the_same_run_to_run(precision):
    # the clamp volume (wet/dry bowl) and the edge inflow volume (inflow DEM)
    # are sums over all CTAs: per-CTA partials added in CTA order make them
    # bit-identical from run to run, whatever order the CTAs finish in
    cases = [(W.parabolic_bowl(nx=400, ny=40), 150, "clamp_mass"),
             (W.coastal_dem(n=192, dx=100.0, t0=500.0), 40, "boundary_mass")]
    for sc, steps, key in cases:
        seen = []
        for _ in range(3):
            with swe.Solver(sc, precision=precision, stream=stream()) as s:
                s.step(steps)
                seen.append(s.diagnostics()[key])
        assert seen[0] != 0.0 and seen[0] == seen[1] == seen[2], (key, seen)


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
@pytest.mark.parametrize("fused", [False, True])
def test_horizon_ends_the_run_on_t_end(precision, fused):
    # swe_set_horizon: the step that would pass t_end is shortened to end on
    # it and later steps do nothing, as the oracle runs to a set time; the
    # horizon survives a new state and 0 removes it
    sc = W.gaussian_hump(n=96)
    if fused:
        sc = sc.copy(alpha_margin=1.1)
    t_end = 0.4137
    ref = oracle.Simulation(sc)
    n = ref.run_until(t_end)
    rd = ref.diag()
    assert rd["t"] == t_end and n > 5
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        s.set_horizon(t_end)
        s.step(n + 7)
        d = s.diagnostics()
        assert d["t"] == t_end and d["steps"] == n
        h, hu, hv = s.get_state()
        if precision == swe.F64:
            for a, r in ((h, ref.h), (hu, ref.hu), (hv, ref.hv)):
                assert np.abs(a - r).max() <= 1e-10
        else:
            assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4
        s.step(3)  # past the horizon: nothing changes, no error
        s.sync()
        assert s.diagnostics()["steps"] == n
        for a, b in zip(s.get_state(), (h, hu, hv)):
            assert np.array_equal(a, b)
        s.set_state(h, hu, hv)  # the horizon is kept across a new state (which restarts the step count)
        s.step(2)
        d = s.diagnostics()
        assert d["t"] == t_end and d["steps"] == 0
        s.set_horizon(0.0)
        s.step(2)
        d = s.diagnostics()
        assert d["t"] > t_end and d["steps"] == 2
        with pytest.raises(swe.SweError):
            s.set_horizon(-1.0)
