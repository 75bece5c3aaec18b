"""The native tile-shape autotuner and its cache."""
import json
import os

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SWE_AUTOTUNE_CACHE", str(path))
    return path


def test_single_scenario_autotune_is_cached_and_used(cache):
    best, ms = swe.autotune([(320, 256)], precision=swe.F32, steps=3)
    assert 1 <= best <= len(swe.tile_shapes())
    assert all(m > 0 for m in ms) and ms[best - 1] == min(ms)
    text = cache.read_text()
    assert "|f32|single|" in text and json.loads(text)
    sc = W.lake_at_rest(320, 256, eta0=0.0, depth=10.0, rms=1.0)
    with swe.Solver(sc, precision=swe.F32, stream=torch.cuda.current_stream().cuda_stream, tile=0) as s:
        assert s.diagnostics()["tile"] == best


def test_fp64_skips_shapes_that_do_not_fit(cache):
    best, ms = swe.autotune([(128, 128)], precision=swe.F64, steps=2)
    too_big = [3, 5, 6, 7, 8, 9]  # need more shared memory than a CTA may use in FP64
    assert all(ms[k - 1] == -1.0 for k in too_big)
    assert best not in too_big and ms[best - 1] > 0.0


def test_batch_autotune_is_cached_and_used(cache):
    best, ms = swe.autotune([(256, 128), (192, 96), (160, 160)], precision=swe.F32, batch=True, steps=3)
    assert 1 <= best <= len(swe.tile_shapes())
    ens = W.mitigation_ensemble(count=1, seed=3, nx_range=(128, 128), ny_range=(64, 64), land_width=90.0)
    with swe.Batch(2, 1 << 30, ens[0], stream=torch.cuda.current_stream().cuda_stream, tile=0) as b:
        s = b.admit(ens[0].copy(t_end=1e6))
        assert b.diagnostics(s)["tile"] == best
