"""Reading real elevation grids (ESRI ASCII) into scenarios."""
import numpy as np
import pytest

import oracle
import workloads as W


def _write(path, z_north_first, header):
    with open(path, "w") as f:
        for k, v in header:
            f.write("%s %s\n" % (k, v))
        for row in z_north_first:
            f.write(" ".join("%.17g" % x for x in row) + "\n")


def test_orientation_spacing_and_nodata(tmp_path):
    z = np.array([[5.0, 6.0, 7.0], [-1.0, -9999.0, 1.0]])  # first row = north
    p = tmp_path / "g.asc"
    _write(p, z, [("NCOLS", 3), ("NROWS", 2), ("XLLCENTER", 12.5), ("YLLCORNER", 100.0),
                  ("CELLSIZE", 5.0), ("NODATA_value", -9999)])
    g, dx, dy, x0, y0, nodata = W.read_esri_ascii(str(p))
    assert g.shape == (2, 3) and dx == dy == 5.0 and x0 == 10.0 and y0 == 100.0
    assert np.array_equal(g[0], [-1.0, -9999.0, 1.0]) and np.array_equal(g[1], [5.0, 6.0, 7.0])
    assert nodata.tolist() == [[False, True, False], [False, False, False]]
    sc = W.dem_scenario(str(p), sea_level=0.0)
    assert sc.b[0, 1] == 7.0                      # NODATA -> highest valid elevation (land)
    assert np.array_equal(sc.h, np.maximum(0.0 - sc.b, 0.0))
    assert sc.z_ref == 0.0 and not sc.hu.any() and not sc.hv.any()


def test_dx_dy_header_crop_and_stride(tmp_path):
    rng = np.random.default_rng(3)
    z = rng.uniform(-20.0, 5.0, size=(8, 10))
    p = tmp_path / "g2.asc"
    _write(p, z, [("ncols", 10), ("nrows", 8), ("xllcorner", 0), ("yllcorner", 0), ("dx", 2.0), ("dy", 3.0)])
    sc = W.dem_scenario(str(p), sea_level=1.0, crop=(2, 8, 0, 10), stride=2, manning_n=0.025, bc=(1, 0, 0, 0),
                        inflow_amp=1.0, inflow_period=300.0, inflow_depth=20.0)
    up = z[::-1]
    assert np.array_equal(sc.b, up[2:8, 0:10][::2, ::2])
    assert (sc.dx, sc.dy) == (4.0, 6.0) and sc.z_ref == 1.0 and sc.manning_n == 0.025 and sc.bc == (1, 0, 0, 0)


def test_lake_over_a_read_grid_stays_at_rest(tmp_path):
    rng = np.random.default_rng(5)
    z = -10.0 + 2.0 * rng.standard_normal((24, 20))
    p = tmp_path / "g3.asc"
    _write(p, z, [("ncols", 20), ("nrows", 24), ("xllcorner", 0), ("yllcorner", 0), ("cellsize", 1.0)])
    sc = W.dem_scenario(str(p), sea_level=0.0)
    sim = oracle.Simulation(sc)
    sim.step(20)
    assert np.abs(sim.h + sc.b).max() <= 1e-12 and np.abs(sim.hu).max() <= 1e-12


def test_short_grid_is_rejected(tmp_path):
    p = tmp_path / "bad.asc"
    p.write_text("ncols 3\nnrows 2\nxllcorner 0\nyllcorner 0\ncellsize 1\n1 2 3\n4 5\n")
    with pytest.raises(ValueError):
        W.read_esri_ascii(str(p))
