"""GPU parity of the shoreline variant (hydrostatic-reconstruction faces
wherever a WENO stencil meets a dry cell) against the oracle's variant on
the same seeded inputs, and its balance on the GPU itself.

Tolerances as for the paper's scheme: FP64 max |d| <= 1e-10; FP32 relative
L2 of the surface anomaly and of the momenta <= 1e-4, runup within 1 cm.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402

from tests import analytic as A  # noqa: E402
from tests.test_gpu_parity import eta_tilde, rel_l2, run_gpu, run_oracle, stream, _film_beach  # noqa: E402
from tests.test_oracle_pins import _standing_wave_case  # noqa: E402
from tests.test_oracle_shore_pins import _two_lakes  # noqa: E402


def _check(sc, steps, precision, name, still=False):
    ref = run_oracle(sc, steps)
    rd = ref.diag()
    h, hu, hv, d, (m, cm) = run_gpu(sc, steps, precision)
    assert d["steps"] == rd["steps"], name
    if precision == swe.F64:
        for a, r in ((h, ref.h), (hu, ref.hu), (hv, ref.hv)):
            assert np.abs(a - r).max() <= 1e-10, name
        assert abs(m - rd["mass"]) <= 1e-11 * m, name
        assert cm == pytest.approx(rd["clamp_mass"], rel=1e-8, abs=1e-12 * m), name
        assert d["boundary_mass"] == pytest.approx(rd["boundary_mass"], rel=1e-8, abs=1e-12 * m), name
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= 1e-10, name
    else:
        assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4, name
        if not still:  # (water at rest: the momenta are round-off on both sides)
            # the momentum vector (hu, hv): a cross-shore flow's small hv alone is noisier
            assert rel_l2(np.stack([hu, hv]), np.stack([ref.hu, ref.hv])) <= 1e-4, name
        assert abs(m - rd["mass"]) <= 1e-6 * m, name
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= 0.01, name
    return h, hu, hv, d


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_two_lakes_at_rest_beside_dry_land(precision):
    sc, level = _two_lakes()
    sc = dataclasses.replace(sc, shore=1)
    wet = sc.h > 0
    h, hu, hv, d = _check(sc, 100, precision, "two lakes", still=True)
    tol = 1e-12 if precision == swe.F64 else 2e-6
    assert np.abs((h + sc.b - level)[wet]).max() <= tol
    assert np.abs(hu).max() <= tol * 10 and np.abs(hv).max() <= tol * 10


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_standing_wave_shoreline(precision):
    sc, amp, L, slope, r, T = _standing_wave_case()
    sc = dataclasses.replace(sc, shore=1)
    probe = oracle.Simulation(sc)
    probe.run_until(0.5 * T)  # the step count that reaches T/2 (its last step shortened)
    n = probe.diag()["steps"]
    ref = oracle.Simulation(sc)
    ref.step(n)  # n full CFL steps, as the GPU takes them
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        s.step(n)
        h, hu, hv = s.get_state()
    if precision == swe.F64:
        assert np.abs(h - ref.h).max() <= 1e-10 and np.abs(hu - ref.hu).max() <= 1e-10
    else:
        assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4
    ex, _, _ = A.standing_wave_on_slope(r, ref.t, amp, L, slope)
    wet = r > 0.0
    assert np.sqrt(np.mean(((h[1] + sc.b[1]) - ex)[wet] ** 2)) <= 0.01 * amp


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_wet_dry_cases(precision):
    for sc, steps in ((W.parabolic_bowl(nx=400, ny=8), 200), (_film_beach(), 30),
                      (W.coastal_dem(n=160, dx=100.0, t0=500.0), 20), (W.planar_beach(ny=8), 300)):
        _check(dataclasses.replace(sc, shore=1), steps, precision, sc.name)


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
@pytest.mark.parametrize("shape", [(3, 3), (37, 19), (77, 45), (130, 97), (200, 33)])
def test_ragged_with_dry_cells(shape, precision):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    b = -1.0 + 1.2 * rng.uniform(size=(ny, nx))
    h = np.maximum(0.5 - b + 0.1 * rng.uniform(size=(ny, nx)), 0.0)
    h[rng.uniform(size=(ny, nx)) < 0.1] = 0.0
    hu = np.where(h > 0, 0.3 * rng.normal(size=(ny, nx)) * h, 0.0)
    hv = np.where(h > 0, 0.3 * rng.normal(size=(ny, nx)) * h, 0.0)
    sc = W.Scenario("ragged_dry", 1.0, 1.0, b, h, hu, hv, manning_n=0.02, shore=1)
    _check(sc, 10, precision, "ragged %dx%d" % shape)


def test_away_from_dry_cells_the_same_as_the_paper():
    sc = W.gaussian_hump()
    a = run_gpu(sc, 50, swe.F64)
    b = run_gpu(dataclasses.replace(sc, shore=1), 50, swe.F64)
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-14


def test_other_tile_shapes_are_rejected():
    sc = dataclasses.replace(W.gaussian_hump(n=32), shore=1)
    with pytest.raises(swe.SweError) as ei:
        swe.Solver(sc, precision=swe.F32, stream=stream(), tile=1)
    assert ei.value.code == swe.EINVAL


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_batch_with_shoreline_faces_matches_oracle_and_alone(precision):
    # the ensemble path with the shoreline variant: coasts with hills and a
    # dry shore in one batch against the oracle's variant (FP64: 1e-10), and
    # one of them run alone bit for bit
    ens = [sc.copy(t_end=1e6, shore=1) for sc in
           W.mitigation_ensemble(count=4, seed=23, nx_range=(96, 224), ny_range=(32, 160), land_width=90.0)]
    with swe.Batch(4, 1 << 30, ens[0], stream=stream(), precision=precision) as b:
        slots = [b.admit(sc) for sc in ens]
        b.run(25)
        mix = [b.get_state(s) for s in slots]
    for sc, (h, hu, hv) in zip(ens, mix):
        ref = oracle.Simulation(sc)
        ref.step(25)
        if precision == swe.F64:
            for a, r in ((h, ref.h), (hu, ref.hu), (hv, ref.hv)):
                assert np.abs(a - r).max() <= 1e-10, sc.name
        else:
            assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4, sc.name
            assert rel_l2(np.stack([hu, hv]), np.stack([ref.hu, ref.hv])) <= 1e-4, sc.name
    with swe.Batch(1, 1 << 30, ens[1], stream=stream(), precision=precision) as b:
        s = b.admit(ens[1])
        b.run(25)
        alone = b.get_state(s)
    for x, y in zip(alone, mix[1]):
        assert np.array_equal(x, y)
