"""The row-partitioned domain (swe_multi: strips with three halo rows,
exchanged after every RK stage, one wave-speed maximum over all strips)
against the undivided grid (swe_create) and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def _film_beach(nx=96, ny=80, seed=43):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5)[None, :] * np.ones((ny, 1))
    b = (x - nx / 2) / 40.0 + 0.02 * rng.standard_normal((ny, nx))
    h = np.maximum(-b, 0.0)
    land = h == 0.0
    film = land & (rng.random((ny, nx)) < 0.6)
    h[film] = np.exp(rng.uniform(np.log(1e-5), np.log(3e-3), size=film.sum()))
    u = rng.normal(size=(ny, nx)) * 0.3
    v = rng.normal(size=(ny, nx)) * 0.3
    return W.Scenario("film_beach", 1.0, 1.0, b, h, h * u, h * v, manning_n=0.02)


CASES = {
    "hump": lambda: W.gaussian_hump(),
    "inflow_dem": lambda: W.coastal_dem(n=256, dx=80.0, t0=500.0),
    "film_beach": _film_beach,
}


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
@pytest.mark.parametrize("case,nparts,tile", [("hump", 2, 1), ("hump", 3, 7), ("inflow_dem", 2, 7), ("inflow_dem", 4, 2),
                                              ("film_beach", 2, 1)])
def test_strips_equal_the_undivided_grid_bit_for_bit(precision, case, nparts, tile):
    sc = CASES[case]()
    if precision == swe.F64 and tile == 7:
        tile = 2  # 96x32 needs more shared memory than a CTA has in FP64
    steps = 25
    with swe.Solver(sc, precision=precision, stream=stream(), tile=tile) as s:
        s.step(steps)
        ref = s.get_state()
        dr = s.diagnostics()
        mr, _ = s.mass()
    with swe.Multi(sc, nparts, precision=precision, stream=stream(), tile=tile) as m:
        m.step(steps)
        got = m.get_state()
        dm = m.diagnostics()
        mm = m.mass()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    for k in ("t", "steps", "last_dt", "alpha_x", "alpha_y", "runup_max", "runup_now"):
        assert dm[k] == dr[k], k
    # the same terms in other groups: each thread sums its own cells in the
    # state's precision before the FP64 reduction, and a strip's threads hold
    # other cells than the undivided grid's; the undivided grid also adds its
    # y walls' fluxes, zero but for FP32 rounding of the reconstructed fluxes
    tol, atol = (1e-12, 1e-12) if precision == swe.F64 else (1e-6, 1e-9 * mr)
    for k in ("clamp_mass", "boundary_mass"):
        assert dm[k] == pytest.approx(dr[k], rel=tol, abs=atol), k
    assert mm == pytest.approx(mr, rel=1e-12)


def test_strips_match_the_fp64_oracle():
    sc = W.coastal_dem(n=192, dx=100.0, t0=500.0)
    ref = oracle.Simulation(sc)
    ref.step(30)
    with swe.Multi(sc, 3, precision=swe.F64, stream=stream()) as m:
        m.step(30)
        h, hu, hv = m.get_state()
        d = m.diagnostics()
    assert np.abs(h - ref.h).max() <= 1e-10
    assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10
    assert d["boundary_mass"] == pytest.approx(ref.diag()["boundary_mass"], rel=1e-9)


def test_strips_reject_periodic_or_inflow_y_sides():
    sc = W.gaussian_hump(n=64)
    for bc in ((0, 0, 2, 2),):
        with pytest.raises(swe.SweError) as ei:
            swe.Multi(sc.copy(bc=bc), 2, stream=stream())
        assert ei.value.code == swe.EINVAL
