"""Parity cases run on the index-checked build (libswe_checked.so): every
index into the shared halo box, the flux buffer and the global planes is
compared with its extent before the access.  Run as a script in a process
whose SWE_LIB_VARIANT=checked (tests/test_gpu_checked.py does this); prints
one line per case and "CHECKED OK" at the end if every check word stayed 0
and every result matched the FP64 oracle at the usual tolerances."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402

assert os.environ.get("SWE_LIB_VARIANT") == "checked"
import paper_2301_12010_gb300 as swe  # noqa: E402

assert swe.lib.swe_checked_build() == 1, "not the checked build"
ST = torch.cuda.current_stream().cuda_stream


def eta_tilde(h, b):
    return np.where(h >= 1e-5, h + b, 0.0)


def rel_l2(a, r):
    return float(np.sqrt(((a - r) ** 2).sum() / max((r ** 2).sum(), 1e-300)))


def run(sc, steps, precision, tile=0):
    with swe.Solver(sc, precision=precision, stream=ST, tile=tile) as s:
        s.step(steps)
        h, hu, hv = s.get_state()
        word = s.check_word()
    return h, hu, hv, word


def compare(name, sc, steps, precision, tile=0):
    ref = oracle.Simulation(sc)
    ref.step(steps)
    h, hu, hv, word = run(sc, steps, precision, tile)
    assert word == 0, "%s: index out of range, check word %#x" % (name, word)
    if precision == swe.F64:
        err = float(np.abs(h - ref.h).max())
        assert err <= 1e-10, (name, err)
    else:
        err = rel_l2(eta_tilde(h, sc.b), eta_tilde(ref.h, sc.b))
        assert err <= 1e-4, (name, err)
    print("%-40s tile %2d %s err %.2e" % (name, tile, "f64" if precision == swe.F64 else "f32", err), flush=True)


def ragged(nx, ny):
    rng = np.random.default_rng(nx * 1000 + ny)
    sc = W.lake_at_rest(nx, ny, eta0=0.0, depth=4.0, rms=1.0, seed=nx + ny)
    sc.h = sc.h + 0.2 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.3 * rng.normal(size=sc.h.shape)
    sc.hv = 0.3 * rng.normal(size=sc.h.shape)
    sc.manning_n = 0.03
    return sc


def main():
    tiles = list(range(1, swe.lib.swe_tile_count() + 1))
    fp64_tiles = [1, 2, 4, 10, 11]
    for shape in [(77, 45), (3, 3), (8, 8), (37, 19), (37, 4), (130, 97), (200, 33)]:
        sc = ragged(*shape)
        for t in tiles:
            compare("ragged %dx%d" % shape, sc, 6, swe.F32, t)
        for t in fp64_tiles:
            compare("ragged %dx%d" % shape, sc, 6, swe.F64, t)
    compare("hump 128", W.gaussian_hump(), 40, swe.F32)
    compare("wet/dry bowl 400x8", W.parabolic_bowl(nx=400, ny=8), 100, swe.F64)
    from tests.analytic import manning_normal_discharge
    qn = manning_normal_discharge(0.5, 1 / 20, 0.033)
    compare("periodic Manning 64x8", W.manning_slope(nx=64, ny=8, q=0.8 * qn), 50, swe.F64)
    compare("inflow DEM 96", W.coastal_dem(n=96, dx=150.0, t0=500.0), 20, swe.F64)
    compare("inflow DEM 96", W.coastal_dem(n=96, dx=150.0, t0=500.0), 20, swe.F32)
    # the fused-step variant (one kernel per step, 9-cell halo frames)
    for shape in [(3, 3), (8, 8), (37, 19), (77, 45), (130, 97), (65, 33), (200, 33)]:
        sc = ragged(*shape).copy(alpha_margin=1.1)
        compare("fused ragged %dx%d" % shape, sc, 6, swe.F32)
        compare("fused ragged %dx%d" % shape, sc, 6, swe.F64)
    fdem = W.coastal_dem(n=96, dx=150.0, t0=500.0).copy(alpha_margin=1.1)
    compare("fused inflow DEM 96", fdem, 20, swe.F32)
    compare("fused inflow DEM 96", fdem, 20, swe.F64)
    # the shoreline variant (hydrostatic-reconstruction faces at dry cells)
    for shape in [(3, 3), (37, 19), (77, 45), (200, 33)]:
        sc = ragged(*shape).copy(shore=1)
        sc.h[::5, ::3] = 0.0
        compare("shore ragged %dx%d" % shape, sc, 6, swe.F32)
        compare("shore ragged %dx%d" % shape, sc, 6, swe.F64)
    compare("shore inflow DEM 96", W.coastal_dem(n=96, dx=150.0, t0=500.0).copy(shore=1), 20, swe.F32)
    # the batch kernel over a mix of small coasts
    ens = W.mitigation_ensemble(count=5, seed=41, nx_range=(96, 192), ny_range=(32, 128), land_width=90.0)
    with swe.Batch(len(ens), 1 << 30, ens[0], stream=ST) as b:
        slots = [b.admit(sc.copy(t_end=1e6)) for sc in ens]
        b.run(8)
        for s in slots:
            word = b.check_word(s)
            assert word == 0, "batch slot %d: check word %#x" % (s, word)
        assert b.status() == swe.OK
    print("batch of %d coasts: check words 0" % len(ens))
    with swe.Batch(len(ens), 1 << 30, ens[0], stream=ST, precision=swe.F64) as b:
        slots = [b.admit(sc.copy(t_end=1e6)) for sc in ens]
        b.run(4)
        for s in slots:
            word = b.check_word(s)
            assert word == 0, "FP64 batch slot %d: check word %#x" % (s, word)
        assert b.status() == swe.OK
    print("FP64 batch of %d coasts: check words 0" % len(ens))
    print("CHECKED OK")


if __name__ == "__main__":
    main()
