"""Fault injection on the host with a GPU present: failed device allocations
(the swe_debug_fail_alloc hook) leave handles and batches usable, and the
serving loop drops expired, cancelled and impossible requests cleanly.  No
test faults, traps or hangs the GPU."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402
from paper_2301_12010_gb300.serve import Server  # noqa: E402

GB = 1 << 30


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.fixture(autouse=True)
def disarm():
    yield
    swe.debug_fail_alloc(0)


def small_coasts(count, seed=41):
    ens = W.mitigation_ensemble(count=count, seed=seed, nx_range=(96, 192), ny_range=(32, 128), land_width=90.0)
    return [sc.copy(t_end=1e6) for sc in ens]


def pinned(shape):
    return [torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]


def test_failed_readback_buffers_leave_the_handle_usable():
    sc = W.gaussian_hump(n=64)
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.step(5)
        ref = s.get_state()
        out = pinned(sc.h.shape)
        for n in (1, 2):  # the first staging slot, then the second
            swe.debug_fail_alloc(n)
            with pytest.raises(swe.SweError) as ei:
                s.get_state_async(out)
            assert ei.value.code == swe.ENOMEM
            swe.debug_fail_alloc(0)
            assert s.status() == swe.OK
        s.get_state_async(out)
        s.wait_state()
        for a, b in zip(out, ref):
            assert np.array_equal(a, b)
        s.step(5)
        assert s.status() == swe.OK


def test_failed_upload_buffers_leave_the_handle_usable():
    sc, other = W.gaussian_hump(n=64), W.gaussian_hump(n=64, amp=0.3)
    with swe.Solver(other, precision=swe.F32, stream=stream()) as r:
        ref = r.get_state()
    src = pinned(sc.h.shape)
    for a, x in zip(src, (other.h, other.hu, other.hv)):
        a[...] = x
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        for n in (1, 2):  # the first staging slot, then the second
            swe.debug_fail_alloc(n)
            with pytest.raises(swe.SweError) as ei:
                s.set_state_async(*src)
            assert ei.value.code == swe.ENOMEM
            swe.debug_fail_alloc(0)
            assert s.status() == swe.OK
        s.set_state_async(*src)
        for a, b in zip(s.get_state(), ref):
            assert np.array_equal(a, b)
        s.step(5)
        s.sync()


def test_failed_batch_creation_and_admission_leave_no_trace():
    scs = small_coasts(3)
    for n in (1, 2, 3, 4, 5):  # each device allocation of swe_batch_create
        swe.debug_fail_alloc(n)
        with pytest.raises(swe.SweError) as ei:
            swe.Batch(4, GB, scs[0], stream=stream())
        assert ei.value.code == swe.ENOMEM
    swe.debug_fail_alloc(0)
    with swe.Batch(4, GB, scs[0], stream=stream()) as b:
        a = b.admit(scs[0])
        swe.debug_fail_alloc(1)
        with pytest.raises(swe.SweError) as ei:
            b.admit(scs[1])
        assert ei.value.code == swe.ENOMEM
        swe.debug_fail_alloc(1)
        assert b.try_admit(scs[1]) is None  # no room now: wait, do not fail
        assert b.memory()[0] == swe.slot_bytes(scs[0].nx, scs[0].ny)
        c = b.admit(scs[1])
        b.run(12)
        assert b.status() == swe.OK
        got = [b.get_state(a), b.get_state(c)]
    for sc, st in zip(scs[:2], got):
        with swe.Batch(2, GB, sc, stream=stream()) as b1:
            s1 = b1.admit(sc)
            b1.run(12)
            ref = b1.get_state(s1)
        for x, y in zip(st, ref):
            assert np.array_equal(x, y)


def test_serving_drops_expired_cancelled_and_impossible_requests():
    scs = small_coasts(4, seed=43)
    done = [sc.copy(t_end=1.0) for sc in scs[:2]]
    big = W.mitigation_ensemble(count=1, seed=44, nx_range=(1024, 1024), ny_range=(1024, 1024))[0]
    budget = 4 * max(swe.slot_bytes(sc.nx, sc.ny) for sc in scs)
    assert swe.slot_bytes(big.nx, big.ny) > budget
    reqs = [W.Request(0.0, done[0]),
            W.Request(0.0, scs[2].copy(t_end=1.0), deadline=0.0),         # expires before admission
            W.Request(0.0, scs[3].copy(t_end=1e6), cancel_at=0.3),        # withdrawn while running
            W.Request(0.0, big.copy(t_end=1.0)),                          # never fits the budget
            W.Request(0.01, done[1])]
    with Server(scs[0], nslots=4, budget_bytes=budget, k_steps=10, stream=stream(), keep_state=True) as srv:
        rep = srv.serve(reqs)
        assert srv.batch.memory()[0] == 0  # every slot retired, nothing left resident
    status = {r.index: r.status for r in rep.results}
    assert status == {0: "done", 1: "expired", 2: "cancelled", 3: "rejected", 4: "done"}
    cancelled = next(r for r in rep.results if r.index == 2)
    assert cancelled.steps > 0 and cancelled.state is None
    s = rep.summary()
    assert s["expired"] == 1 and s["cancelled"] == 1 and s["rejected"] == 1
    for r in rep.results:
        if r.status != "done":
            continue
        sc = reqs[r.index].scenario
        with swe.Batch(2, GB, sc, stream=stream()) as b1:
            s1 = b1.admit(sc)
            while not b1.poll():
                b1.run(10)
            ref = b1.get_state(s1)
        for x, y in zip(r.state, ref):
            assert np.array_equal(x, y)
