"""Host transfers through the C ABI: page-locked host arrays are read and
written by the conversion kernels directly, pageable ones through a staging
plane; both must give the same device state bit for bit."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
pytestmark = pytest.mark.gpu

import paper_2301_12010_gb300 as swe  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def pinned_like(a):
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_pinned_and_pageable_host_arrays_agree(precision):
    sc = W.lake_at_rest(131, 77, eta0=0.0, depth=4.0, rms=1.0, seed=5)  # ragged sizes
    rng = np.random.default_rng(11)
    sc.h = sc.h + 0.1 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.2 * rng.normal(size=sc.h.shape)
    sc.hv = 0.2 * rng.normal(size=sc.h.shape)
    keep = [pinned_like(x) for x in (sc.h, sc.hu, sc.hv)]
    outs = [torch.empty(sc.h.shape, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    with swe.Solver(sc, precision=precision, stream=stream()) as a, \
            swe.Solver(sc, precision=precision, stream=stream()) as b:
        a.set_state(sc.h, sc.hu, sc.hv)                   # pageable in
        b.set_state(*(t.numpy() for t in keep))           # page-locked in
        assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))
        a.step(7)
        b.step(7)
        ref = a.get_state()                               # pageable out
        got = b.get_state(tuple(t.numpy() for t in outs))  # page-locked out
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)


def test_batch_admit_from_page_locked_arrays():
    ens = W.mitigation_ensemble(count=1, seed=3, nx_range=(160, 160), ny_range=(96, 96), land_width=90.0)
    sc = ens[0]
    pinned = sc.copy(b=pinned_like(sc.b).numpy(), h=pinned_like(sc.h).numpy(), hu=pinned_like(sc.hu).numpy(),
                     hv=pinned_like(sc.hv).numpy())
    with swe.Batch(2, 1 << 30, sc, stream=stream()) as bt:
        s0 = bt.admit(sc.copy(t_end=1e6))
        s1 = bt.admit(pinned.copy(t_end=1e6))
        bt.run(10)
        x, y = bt.get_state(s0), bt.get_state(s1)
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def _wavy(nx=131, ny=77, seed=11):
    sc = W.lake_at_rest(nx, ny, eta0=0.0, depth=4.0, rms=1.0, seed=5)
    rng = np.random.default_rng(seed)
    sc.h = sc.h + 0.1 * rng.uniform(size=sc.h.shape)
    sc.hu = 0.2 * rng.normal(size=sc.h.shape)
    sc.hv = 0.2 * rng.normal(size=sc.h.shape)
    return sc


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_async_read_back_overlaps_the_next_upload(precision):
    sc, other = _wavy(seed=11), _wavy(seed=12)
    outs = [torch.empty(sc.h.shape, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    out = tuple(t.numpy() for t in outs)
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        s.step(5)
        ref = s.get_state()
        s.get_state_async(out)
        # a new upload and more steps while the read-back is in flight
        s.set_state(other.h, other.hu, other.hv)
        s.step(3)
        s.wait_state()
        for x, y in zip(out, ref):
            assert np.array_equal(x, y)
        now = s.get_state()
        s.get_state_async(out)
        s.get_state_async(out)  # the second waits for the first on the device
        s.wait_state()
        for x, y in zip(out, now):
            assert np.array_equal(x, y)


def test_async_read_back_into_pageable_arrays_is_synchronous():
    sc = _wavy()
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.step(4)
        ref = s.get_state()
        out = tuple(np.empty(sc.h.shape) for _ in range(3))
        s.get_state_async(out)
        for x, y in zip(out, ref):  # already filled
            assert np.array_equal(x, y)
        s.wait_state()


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_async_upload_gives_the_synchronous_state(precision):
    # swe_set_state_async from page-locked arrays, pipelined with steps and
    # asynchronous read-backs as a streaming caller does: every step's result
    # equals the synchronous upload + step, bit for bit, and the time is kept;
    # five rounds, so that each of the two staging slots per direction is
    # reused while the other is in flight
    states = [_wavy(seed=20 + k) for k in range(5)]
    pin = [[pinned_like(x) for x in (sc.h, sc.hu, sc.hv)] for sc in states]
    outs = [[torch.empty(states[0].h.shape, dtype=torch.float64, pin_memory=True) for _ in range(3)]
            for _ in states]
    with swe.Solver(states[0], precision=precision, stream=stream()) as a:
        a.set_time(5.0)
        for k, p in enumerate(pin):
            a.set_state_async(*(t.numpy() for t in p))
            a.step(2)
            a.get_state_async(tuple(t.numpy() for t in outs[k]))
        a.wait_state()
        t_a, n_a = a.time()
    with swe.Solver(states[0], precision=precision, stream=stream()) as b:
        b.set_time(5.0)
        for k, sc in enumerate(states):
            b.set_state(sc.h, sc.hu, sc.hv)
            b.step(2)
            ref = b.get_state()
            for x, y in zip(outs[k], ref):
                assert np.array_equal(x.numpy(), y)
        t_b, n_b = b.time()
    assert t_a == t_b and n_a == n_b == 2


def test_async_upload_from_pageable_arrays_is_synchronous():
    sc, other = _wavy(seed=30), _wavy(seed=31)
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.set_state_async(other.h, other.hu, other.hv)  # pageable numpy arrays
        got = s.get_state()
    with swe.Solver(other, precision=swe.F32, stream=stream()) as r:
        ref = r.get_state()
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
