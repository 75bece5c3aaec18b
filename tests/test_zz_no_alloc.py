"""The allocation-free volume entry point, swe_mass_noalloc, called through
the C ABI and checked against swe_mass of the same state.

It serves callers that cannot allocate device memory when they need the
diagnostic (a process holding a fixed HBM budget, a loop that must not take
the synchronisation of cudaMalloc/cudaFree, a C host without a handle).
This file is collected last so that a failure here stops a run only after
every other test has run; it passes alone in a fresh process as well."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402


def _max_rows() -> int:
    # the limit as the C header states it (one source for library and test)
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "swe.h")) as f:
        return int(re.search(r"#define\s+SWE_NOALLOC_MAX_ROWS\s+(\d+)", f.read()).group(1))


MAX_ROWS = _max_rows()


def _fn():
    f = swe.lib.swe_mass_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                  ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    return f


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_noalloc_mass_matches_swe_mass_on_two_calls(precision):
    f = _fn()
    stream = torch.cuda.current_stream()
    dtype = torch.float32 if precision == swe.F32 else torch.float64
    tol = 1e-6 if precision == swe.F32 else 1e-12
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    refs = []
    cases = [W.planar_beach(nx=300, ny=40, steps=0), W.gaussian_hump(n=96)]
    for k, sc in enumerate(cases):
        with swe.Solver(sc, precision=precision, stream=stream.cuda_stream) as s:
            s.step(30)
            h, hu, hv = (torch.empty((sc.ny, sc.nx), dtype=dtype, device="cuda") for _ in range(3))
            s.get_state_device(h, hu, hv)
            ref, _ = s.mass()
        refs.append(ref)
        # two calls in a row on the same field (the scratch is reused)
        for c in range(2):
            rc = f(h.data_ptr(), precision, sc.nx, sc.ny, sc.dx, sc.dy, out[2 * k + c:].data_ptr(),
                   stream.cuda_stream)
            assert rc == swe.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k, ref in enumerate(refs):
        assert got[2 * k] == pytest.approx(ref, rel=tol)
        assert got[2 * k + 1] == got[2 * k]


def test_noalloc_rejects_sizes_beyond_the_maximum():
    f = _fn()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    h = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    assert f(h.data_ptr(), swe.F32, 4, MAX_ROWS + 1, 1.0, 1.0, out.data_ptr(), None) == swe.EINVAL
    assert f(h.data_ptr(), 9, 4, 4, 1.0, 1.0, out.data_ptr(), None) == swe.EINVAL
    assert f(None, swe.F32, 4, 4, 1.0, 1.0, out.data_ptr(), None) == swe.EINVAL


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
@pytest.mark.parametrize("shape", [(8, MAX_ROWS), (5, 1025), (70, 1030)])
def test_noalloc_mass_at_row_counts_up_to_the_maximum(precision, shape):
    # the largest accepted grid (every block of the row pass full), a row
    # count just past one 1024-thread block of the final pass (its strided
    # loop) and partial last blocks; against the correctly rounded sum of the
    # same values on the host, twice in a row
    f = _fn()
    nx, ny = shape
    rng = np.random.default_rng(nx * 7 + ny)
    host = rng.uniform(0.0, 3.0, size=(ny, nx)).astype(np.float32 if precision == swe.F32 else np.float64)
    h = torch.from_numpy(host).to("cuda")
    dx, dy = 2.0, 0.5
    want = math.fsum(host.astype(np.float64).ravel()) * dx * dy
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for c in range(2):
        assert f(h.data_ptr(), precision, nx, ny, dx, dy, out[c:].data_ptr(), stream.cuda_stream) == swe.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(want, rel=1e-12)
    assert got[1] == got[0]
