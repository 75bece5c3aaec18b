"""The seeded synthetic inputs follow the recipe the design notes state
(sizes, ranges, spectra, determinism).  They stand in for the paper's
unavailable data; they hold none of the method's arithmetic."""
import math

import numpy as np

import workloads as W


def test_fractal_field_has_the_stated_rms_and_spectral_slope():
    f = W._fractal_field_2d(256, 256, seed=3, rms=3.0)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 3.0) < 1e-9
    p = np.abs(np.fft.rfft2(f)) ** 2
    ky = np.fft.fftfreq(256)[:, None]
    kx = np.fft.rfftfreq(256)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    sel = (k > 0.02) & (k < 0.4)
    slope = np.polyfit(np.log(k[sel]), np.log(p[sel]), 1)[0]
    assert abs(slope - (-2.0)) < 0.15  # power spectrum ~ k^-2
    assert np.array_equal(f, W._fractal_field_2d(256, 256, seed=3, rms=3.0))  # seeded


def test_coastal_dem_profile():
    sc = W.coastal_dem(n=512, dx=40.0)
    L = 512 * 40.0
    x = (np.arange(512) + 0.5) * 40.0
    mean_b = sc.b.mean(axis=0)
    base = np.where(x < 0.8 * L, -200.0 + 200.0 * x / (0.8 * L), 20.0 * (x - 0.8 * L) / (0.2 * L))
    # shelf ramp to 0 at 0.8 L and land to +20 m under the noise's large scales
    assert np.abs(mean_b - base).max() < 3.0
    assert abs((sc.b - base[None, :]).std() - 3.0) < 1e-6  # 3 m rms
    assert sc.bc[0] == W.INFLOW and sc.inflow_amp == 4.0 and sc.inflow_period == 600.0
    assert sc.manning_n == 0.025 and sc.t0 == 600.0
    assert (sc.h[:, x >= 0.9 * L] == 0).mean() > 0.95  # inland is dry


def test_ensemble_sizes_and_determinism():
    ens = W.mitigation_ensemble()
    assert len(ens) == 64
    for sc in ens:
        assert 512 <= sc.nx <= 1024 and 256 <= sc.ny <= 1024
        assert sc.nx % 32 == 0 and sc.ny % 32 == 0 and sc.dx == 2.0
        assert sc.bc == (W.WALL, W.WALL, W.WALL, W.WALL)
    assert len({(sc.nx, sc.ny) for sc in ens}) > 20  # uneven grids
    again = W.mitigation_ensemble(count=3)
    for a, b in zip(ens[:3], again):
        assert (a.nx, a.ny) == (b.nx, b.ny) and np.array_equal(a.b, b.b) and np.array_equal(a.h, b.h)


def test_serving_requests_are_poisson_with_log_uniform_sizes():
    reqs = W.serving_requests(rate=10.0, count=400, horizon=20.0, n_range=(64, 512))  # small grids: fast
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() - 0.1) < 0.02  # mean inter-arrival 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15  # exponential gaps
    n = np.array([r.scenario.nx for r in reqs])
    assert np.all(n % 32 == 0) and n.min() >= 64 and n.max() <= 512
    assert all(r.scenario.nx == r.scenario.ny and r.scenario.t_end == 20.0 for r in reqs)
    ln = np.log(n)
    assert abs(np.median(ln) - 0.5 * (math.log(64) + math.log(512))) < 0.15  # log-uniform
