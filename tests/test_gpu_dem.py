"""A real-format elevation grid driven through the GPU path: an ESRI ASCII
grid or a GeoTIFF (rough shelf, coast, land with a NODATA patch, a sea level
away from 0) is written to disk, read by workloads.dem_scenario and advanced
on the GPU in FP64 and FP32 against the FP64 oracle on the same scenario, with
the inflow N-wave of Eq. (20) entering through the ocean edge and Manning
friction."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402


def _write_grid(path, fmt="asc", nx=150, ny=96, cell=20.0, seed=61):
    # elevations in the file's own order: first row = north, x fastest
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) * cell
    L = nx * cell
    shelf = np.where(x < 0.7 * L, -60.0 + 60.0 * x / (0.7 * L), 12.0 * (x - 0.7 * L) / (0.3 * L))
    z = shelf[None, :] + 1.5 * rng.standard_normal((ny, nx))
    z[10:20, nx - 25:nx - 12] = -9999.0  # a NODATA patch on land
    if fmt == "tif":  # float32 samples in 32 x 32 tiles, Deflate with the floating-point predictor
        from tests.test_geotiff import write_tiff
        write_tiff(path, z, dtype="f4", tile=(32, 32), deflate=True, predictor=3, scale=(cell, cell),
                   tiepoint=(0.0, 0.0, 5000.0, 8000.0 + ny * cell), nodata="-9999")
        return
    with open(path, "w") as f:
        f.write("ncols %d\nnrows %d\nxllcorner 5000\nyllcorner 8000\ncellsize %g\nNODATA_value -9999\n"
                % (nx, ny, cell))
        for row in z:
            f.write(" ".join("%.10g" % v for v in row) + "\n")


def _scenario(tmp_path, fmt="asc"):
    p = tmp_path / ("coast." + fmt)
    _write_grid(str(p), fmt)
    sc = W.dem_scenario(str(p), sea_level=0.5, manning_n=0.025, bc=(W.INFLOW, W.WALL, W.WALL, W.WALL),
                        inflow_amp=2.0, inflow_period=300.0, inflow_depth=60.0, t0=200.0)
    return sc


def _eta_tilde(h, b, h_dry=1e-5):
    return np.where(h >= h_dry, h + b, 0.0)


def _rel_l2(a, ref):
    return float(np.sqrt(((a - ref) ** 2).sum() / max((ref ** 2).sum(), 1e-300)))


@pytest.mark.parametrize("fmt", ["asc", "tif"])
@pytest.mark.parametrize("precision", [swe.F64, swe.F32])
def test_ingested_dem_against_the_oracle(tmp_path, precision, fmt):
    sc = _scenario(tmp_path, fmt)
    assert sc.z_ref == 0.5 and (sc.h == 0).any() and (sc.h > 0).any()
    steps = 60
    ref = oracle.Simulation(sc)
    ref.step(steps)
    rd = ref.diag()
    st = torch.cuda.current_stream().cuda_stream
    with swe.Solver(sc, precision=precision, stream=st) as s:
        s.step(steps)
        h, hu, hv = s.get_state()
        d = s.diagnostics()
    # FP32 wave speeds set an FP32-rounded CFL step
    assert d["steps"] == steps and d["t"] == pytest.approx(rd["t"], rel=1e-12 if precision == swe.F64 else 1e-5)
    assert rd["boundary_mass"] > 0  # the wave entered
    if precision == swe.F64:
        assert np.abs(h - ref.h).max() <= 1e-10
        assert np.abs(hu - ref.hu).max() <= 1e-10 and np.abs(hv - ref.hv).max() <= 1e-10
        assert d["boundary_mass"] == pytest.approx(rd["boundary_mass"], rel=1e-9)
    else:
        # the anomaly against the sea level (the still-water surface)
        e, er = _eta_tilde(h, sc.b) - 0.5 * (h >= sc.h_dry), _eta_tilde(ref.h, sc.b) - 0.5 * (ref.h >= sc.h_dry)
        assert _rel_l2(e, er) <= 1e-4
        assert _rel_l2(hu, ref.hu) <= 1e-4
    if rd["runup_max"] > -np.inf:
        assert abs(d["runup_max"] - rd["runup_max"]) <= (1e-10 if precision == swe.F64 else 0.01)
