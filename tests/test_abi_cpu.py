"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/swe.h declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swe_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def swe():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not b.up_to_date():
        b.build()
    import paper_2301_12010_gb300 as m
    return m


def test_every_declared_symbol_is_exported(swe):
    names = _declared("swe.h")
    assert len(names) >= 18
    for n in names:
        assert hasattr(swe.lib, n), n


def test_defaults_and_strerror(swe):
    p = swe.Params()
    swe.lib.swe_params_default(ctypes.byref(p))
    assert p.g == 9.81 and p.h_dry == 1e-5 and p.weno_eps == 1e-6 and list(p.bc) == [0, 0, 0, 0]
    assert p.fused_step == 0 and p.alpha_margin == 1.1
    for code in range(8):
        assert swe.lib.swe_strerror(code)
    assert swe.lib.swe_destroy(None) == swe.OK


def test_invalid_arguments_rejected_without_gpu(swe):
    p = swe.Params()
    swe.lib.swe_params_default(ctypes.byref(p))
    b = np.zeros((4, 4))
    h = ctypes.c_void_p()
    dp = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(2, 4)), 1.0, 1.0, dp, ctypes.byref(p), ctypes.byref(h)) == swe.EINVAL
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 0.0, 1.0, dp, ctypes.byref(p), ctypes.byref(h)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.bc[1] = swe.INFLOW
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.bc[0] = swe.PERIODIC
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.precision = 7
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    # the fused-step variant: a margin below 1, periodic sides, an unknown mode
    for field, value in (("alpha_margin", 0.9), ("alpha_margin", float("nan")), ("fused_step", 2)):
        q = swe.Params.from_buffer_copy(p)
        q.fused_step = 1
        setattr(q, field, value)
        assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    # the shoreline variant: its own tile shape only, not with the fused step
    for field, value in (("shore", 2), ("tile", 1), ("fused_step", 1)):
        q = swe.Params.from_buffer_copy(p)
        q.shore = 1
        setattr(q, field, value)
        assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.fused_step = 1
    q.bc[0] = q.bc[1] = swe.PERIODIC
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(4, 4)), 1.0, 1.0, dp, ctypes.byref(q), ctypes.byref(h)) == swe.EINVAL
    # more than 2^31 cells: rejected before anything is read or allocated
    assert swe.lib.swe_create(ctypes.byref(swe.Grid(65536, 32769)), 1.0, 1.0, dp, ctypes.byref(p), ctypes.byref(h)) == swe.EINVAL
    assert not h.value
    assert swe.lib.swe_step(None, 1, 0.4) == swe.EINVAL
    assert swe.lib.swe_set_horizon(None, 1.0) == swe.EINVAL


def test_tile_shapes(swe):
    shapes = swe.tile_shapes()
    assert len(shapes) >= 3
    for tx, ty, nt in shapes:
        # one strip of S = 8 or 16 cells per thread in both sweep directions
        assert any((tx // S) * ty == nt and (ty // S) * tx == nt for S in (8, 16))


def test_batch_arguments_rejected_without_gpu(swe):
    p = swe.Params()
    swe.lib.swe_params_default(ctypes.byref(p))
    b = ctypes.c_void_p()
    assert swe.lib.swe_batch_destroy(None) == swe.OK
    assert swe.lib.swe_batch_create(0, 1 << 30, ctypes.byref(p), ctypes.byref(b)) == swe.EINVAL
    assert swe.lib.swe_batch_create(4, 0, ctypes.byref(p), ctypes.byref(b)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.precision, q.tile = swe.F64, 7  # FP64 batches run on their one compiled shape
    assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.bc[0] = swe.INFLOW  # an inflow edge needs the N-wave's depth and period
    assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.bc[1] = swe.INFLOW  # the inflow edge is the x- side only
    assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.bc[2] = swe.PERIODIC  # periodic sides come in pairs
    assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    for prec, tile in ((swe.F64, 7), (swe.F32, 1)):  # the shoreline batch: its one shape per precision
        q = swe.Params.from_buffer_copy(p)
        q.shore, q.precision, q.tile = 1, prec, tile
        assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    q = swe.Params.from_buffer_copy(p)
    q.fused_step = 1  # the batch runs the per-stage alpha
    assert swe.lib.swe_batch_create(4, 1 << 30, ctypes.byref(q), ctypes.byref(b)) == swe.EINVAL
    assert not b.value
    assert swe.lib.swe_batch_run(None, 1, 0.4) == swe.EINVAL
    assert swe.lib.swe_batch_poll(None, None, None) == swe.EINVAL


def test_checked_build_exports_the_same_calls(swe):
    # the index-checked library (SWE_CHECKED) is the same ABI; it says which
    # build it is, and the normal one says it is not checked
    import ctypes as C
    b = __import__("__graft_entry__")._build_module()
    if not b.up_to_date(checked=True):
        b.build(checked=True)
    chk = C.CDLL(b.LIB_CHECKED)
    for n in _declared("swe.h"):
        assert hasattr(chk, n), n
    assert chk.swe_checked_build() == 1
    assert swe.lib.swe_checked_build() == 0
