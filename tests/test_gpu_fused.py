"""GPU parity of the fused-step variant (one kernel per RK3 step, one
splitting speed per step: alpha_margin x alpha of U^n) against the oracle's
variant on the same seeded inputs.

Tolerances as for the stage kernels: FP64 max |d| <= 1e-10; FP32 relative L2
of the surface anomaly and of the momenta <= 1e-4, runup within 1 cm.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402

from tests.test_gpu_parity import eta_tilde, rel_l2, run_gpu, run_oracle, stream, _film_beach  # noqa: E402
from tests.test_oracle_fused_pins import _hole_and_hump  # noqa: E402

MARGIN = 1.1


def _ragged(nx, ny, seed=0):
    rng = np.random.default_rng(nx * 1000 + ny + seed)
    sc = W.lake_at_rest(nx, ny, eta0=0.0, depth=4.0, rms=1.0, seed=nx + ny)
    sc.h = sc.h + 0.2 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.3 * rng.normal(size=sc.h.shape)
    sc.hv = 0.3 * rng.normal(size=sc.h.shape)
    sc.manning_n = 0.03
    return sc


def _check(sc, steps, precision, name):
    ref = run_oracle(sc, steps)
    rd = ref.diag()
    h, hu, hv, d, (m, cm) = run_gpu(sc, steps, precision)
    assert d["steps"] == rd["steps"], name
    if precision == swe.F64:
        for a, r in ((h, ref.h), (hu, ref.hu), (hv, ref.hv)):
            assert np.abs(a - r).max() <= 1e-10, name
        assert d["t"] == pytest.approx(rd["t"], rel=1e-12), name
        assert d["alpha_x"] == pytest.approx(rd["alpha_x"], rel=1e-10), name
        assert d["alpha_y"] == pytest.approx(rd["alpha_y"], rel=1e-10), name
        assert abs(m - rd["mass"]) <= 1e-11 * m, name
        assert cm == pytest.approx(rd["clamp_mass"], rel=1e-8, abs=1e-12 * m), name
        assert d["boundary_mass"] == pytest.approx(rd["boundary_mass"], rel=1e-8, abs=1e-12 * m), name
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= 1e-10, name
    else:
        assert rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b)) <= 1e-4, name
        assert rel_l2(hu, ref.hu) <= 1e-4 and rel_l2(hv, ref.hv) <= 1e-4, name
        assert d["t"] == pytest.approx(rd["t"], rel=1e-5), name
        assert abs(m - rd["mass"]) <= 1e-6 * m, name
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= 0.01, name
    return h, hu, hv, d


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
@pytest.mark.parametrize("shape", [(3, 3), (8, 8), (37, 19), (77, 45), (130, 97), (200, 33), (64, 32), (65, 33)])
def test_fused_ragged_random(shape, precision):
    # grids smaller than a tile, exactly one tile, and several tiles with
    # ragged tails in both directions; walls, friction, a rough bed
    sc = _ragged(*shape).copy(alpha_margin=MARGIN)
    _check(sc, 12, precision, "ragged %dx%d" % shape)


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_fused_hump_and_wet_dry(precision):
    for sc, steps in ((W.gaussian_hump(), 100), (W.parabolic_bowl(nx=400, ny=8), 100), (_film_beach(), 30)):
        _check(sc.copy(alpha_margin=MARGIN), steps, precision, sc.name)


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_fused_inflow_dem_with_friction(precision):
    # the N-wave inflow edge (ghosts at the three stage times), Manning
    # friction, a dry shore; the edge volume counted once per face
    sc = W.coastal_dem(n=160, dx=100.0, t0=500.0).copy(alpha_margin=MARGIN)
    _, _, _, d = _check(sc, 20, precision, "inflow DEM 160")
    assert d["boundary_mass"] > 0.0


def test_fused_fixed_dt_and_wider_margin():
    sc = W.planar_beach(ny=4).copy(fixed_dt=5e-3, alpha_margin=1.5)
    _, _, _, d = _check(sc, 300, swe.F64, "planar beach, fixed dt")
    assert d["last_dt"] == 5e-3


def test_fused_equals_stage_kernels_while_the_speeds_hold():
    # the fastest cell stays at rest through the step: every stage's alpha is
    # alpha(U^n), so with margin 1 the fused kernel and the three stage
    # kernels compute the same step
    sc = _hole_and_hump()
    a = run_gpu(sc, 1, swe.F64)
    b = run_gpu(sc.copy(alpha_margin=1.0), 1, swe.F64)
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-12


@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_fused_odd_and_even_step_counts_agree(precision):
    # steps run in pairs (plane set 0 -> 1 -> 0); an odd count ends with one
    # step and a copy back: 1 + 2 + 4 steps equal 7 steps bit for bit
    sc = _ragged(77, 45).copy(alpha_margin=MARGIN)
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        for n in (1, 2, 4):
            s.step(n)
        a = s.get_state()
        da = s.diagnostics()
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        s.step(7)
        b = s.get_state()
        db = s.diagnostics()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert da["steps"] == db["steps"] == 7 and da["t"] == db["t"]


def test_fused_nonfinite_is_reported_and_skipped_steps_keep_the_state():
    # a NaN in the state: the status reports it and the steps are skipped;
    # a skipped step copies U^n into the other plane set, so that the state
    # read back is the one set, whatever the step count's parity
    sc = W.gaussian_hump(n=96).copy(alpha_margin=MARGIN)
    sc.h[5, 7] = np.nan

    def read(s):  # the read-back fills the arrays, then reports the status
        out = tuple(np.empty((s.ny, s.nx)) for _ in range(3))
        with pytest.raises(swe.SweError) as ei:
            s.get_state(out)
        assert ei.value.code == swe.ENONFINITE
        return out

    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        before = read(s)
        assert np.isnan(before[0][5, 7])
        for n in (2, 1, 3):
            s.step(n)
            with pytest.raises(swe.SweError) as ei:
                s.sync()
            assert ei.value.code == swe.ENONFINITE
            for x, y in zip(before, read(s)):
                assert np.array_equal(x, y, equal_nan=True)


def test_fused_dry_still_domain_reports_einval():
    # no water, no CFL step: the step's preparation flags it, nothing moves
    sc = W.lake_at_rest(16, 16, eta0=-100.0, depth=10.0, rms=1.0).copy(alpha_margin=MARGIN)
    assert sc.h.max() == 0.0
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.step(3)
        with pytest.raises(swe.SweError) as ei:
            s.sync()
        assert ei.value.code == swe.EINVAL


def test_fused_is_deterministic():
    sc = W.coastal_dem(n=128, dx=120.0, t0=500.0).copy(alpha_margin=MARGIN)
    outs = []
    for _ in range(3):
        with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
            s.step(10)
            outs.append((s.get_state(), s.diagnostics()))
    for (st, d) in outs[1:]:
        for x, y in zip(st, outs[0][0]):
            assert np.array_equal(x, y)
        for k in ("clamp_mass", "boundary_mass", "alpha_x", "alpha_y", "runup_max"):
            assert d[k] == outs[0][1][k]


def test_fused_time_stages_reports_the_step_kernel():
    sc = W.gaussian_hump(n=256).copy(alpha_margin=MARGIN)
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        tot, st = s.time_stages(3, 0.4)
        d = s.diagnostics()
    assert d["steps"] == 1 + 3
    assert tot > 0 and st[0] > 0 and st[1] >= 0 and st[2] == 0.0
    assert st[0] <= tot


def test_fused_periodic_is_rejected():
    sc = W.manning_slope(nx=64, ny=8).copy(alpha_margin=MARGIN)
    with pytest.raises(swe.SweError) as ei:
        swe.Solver(sc, precision=swe.F32, stream=stream())
    assert ei.value.code == swe.EINVAL
