"""The serving loop's host logic (admission order, the SRPT choice, expiry,
cancellation, rejection, accounting) against a stand-in batch that advances
simulated time on the CPU.  The GPU path of the same loop is tested in
tests/test_gpu_serve.py and tests/test_gpu_failures.py."""
import time
import types

import numpy as np
import pytest

serve = pytest.importorskip("paper_2301_12010_gb300.serve")


class FakeBatch:
    """Batch interface over plain Python: slots hold (t, steps, t_end, dt,
    cells); run(k) advances the selected live slots k steps of dt each,
    stopping at t_end; the budget counts cells."""

    def __init__(self, nslots, budget_cells, step_wall=0.0):
        self.nslots, self.budget, self.step_wall = nslots, budget_cells, step_wall
        self.slots = {}
        self.sel = None
        self.runs = []  # (k, sorted slots advanced) per run

    def try_admit(self, sc, t_end=None):
        used = sum(v["cells"] for v in self.slots.values())
        if len(self.slots) >= self.nslots or used + sc.cells > self.budget:
            return None
        s = min(set(range(self.nslots)) - set(self.slots))
        self.slots[s] = {"t": 0.0, "steps": 0, "t_end": sc.t_end, "dt": sc.dt, "cells": sc.cells}
        self.sel = None
        return s

    def select(self, slots=None):
        self.sel = None if slots is None else list(slots)

    def times(self):
        t = np.zeros(self.nslots)
        for s, v in self.slots.items():
            t[s] = v["t"]
        return t

    def run(self, k, cfl=0.4):
        adv = sorted(self.slots if self.sel is None else self.sel)
        for s in adv:
            v = self.slots[s]
            for _ in range(k):
                if v["t"] >= v["t_end"]:
                    break
                v["t"] = min(v["t"] + v["dt"], v["t_end"])
                v["steps"] += 1
        self.runs.append((k, adv))
        if self.step_wall:
            time.sleep(self.step_wall)

    def poll(self):
        return sorted(s for s, v in self.slots.items() if v["t"] >= v["t_end"])

    def diagnostics(self, slot, check=True):
        v = self.slots[slot]
        return {"t": v["t"], "steps": v["steps"]}

    def retire(self, slot, want_state=True):
        v = self.slots.pop(slot)
        self.sel = None
        return (("state", slot) if want_state else None), float(v["cells"]), 0.0

    def memory(self):
        return sum(v["cells"] for v in self.slots.values()), self.budget

    def close(self):
        pass


def request(arrival, cells, t_end, dt=0.125, **kw):  # dt exact in binary
    sc = types.SimpleNamespace(cells=cells, nx=cells, ny=1, dx=1.0, dy=1.0, t_end=t_end, dt=dt)
    return types.SimpleNamespace(arrival=arrival, scenario=sc, **kw)


def server(fake, policy="all", fill=10 ** 9, k=5, keep=True):
    return serve.Server(None, policy=policy, fill_cells=fill, k_steps=k, keep_state=keep, batch=fake)


def test_every_request_completes_with_its_steps():
    fake = FakeBatch(4, 1000)
    reqs = [request(0.0, 100, 1.0), request(0.0, 200, 2.0), request(0.0, 50, 0.5)]
    rep = server(fake).serve(reqs)
    assert sorted(r.index for r in rep.results) == [0, 1, 2]
    for r in rep.results:
        assert r.status == "done"
        assert r.t == pytest.approx(reqs[r.index].scenario.t_end)
        assert r.steps == round(reqs[r.index].scenario.t_end / 0.125)
    assert rep.cell_updates == pytest.approx(100 * 8 + 200 * 16 + 50 * 4)
    assert fake.memory()[0] == 0
    assert rep.summary()["requests"] == 3 and "expired" not in rep.summary()


def test_srpt_advances_the_least_remaining_work_first():
    fake = FakeBatch(4, 10 ** 6)
    big, small = request(0.0, 1000, 5.0), request(0.0, 10, 1.0)
    rep = server(fake, policy="srpt", fill=10).serve([big, small])
    order = [r.index for r in sorted(rep.results, key=lambda r: r.finished)]
    assert order == [1, 0]
    # while both were live, only the small one (slot 1) advanced
    first = fake.runs[0]
    assert first[1] == [1]


def test_all_policy_advances_every_live_request():
    fake = FakeBatch(4, 10 ** 6)
    server(fake, policy="all").serve([request(0.0, 1000, 5.0), request(0.0, 10, 1.0)])
    assert fake.runs[0][1] == [0, 1]


def test_admission_waits_in_arrival_order_for_budget():
    fake = FakeBatch(4, 300)
    reqs = [request(0.0, 200, 1.0), request(0.0, 200, 0.5), request(0.0, 50, 0.5)]
    rep = server(fake).serve(reqs)
    adm = {r.index: r.admitted for r in rep.results}
    # the second waits for the first; the third, behind it in arrival order, waits too
    assert adm[1] >= adm[0] and adm[2] >= adm[1]
    assert all(r.status == "done" for r in rep.results)


def test_expired_cancelled_and_rejected_requests_leave_cleanly():
    fake = FakeBatch(4, 1000, step_wall=0.002)
    reqs = [request(0.0, 100, 1.0),
            request(0.0, 100, 1.0, deadline=0.0),        # expires before admission
            request(0.0, 100, 1e9, cancel_at=0.05),      # withdrawn while running
            request(0.0, 5000, 1.0),                     # larger than the budget
            request(0.0, 100, 1.0)]
    rep = server(fake).serve(reqs)
    st = {r.index: r.status for r in rep.results}
    assert st == {0: "done", 1: "expired", 2: "cancelled", 3: "rejected", 4: "done"}
    cancelled = next(r for r in rep.results if r.index == 2)
    assert cancelled.steps > 0 and cancelled.state is None and np.isnan(cancelled.mass)
    s = rep.summary()
    assert s["expired"] == s["cancelled"] == s["rejected"] == 1
    done = [r.latency for r in rep.results if r.status == "done"]
    assert rep.latency_ms(50) == pytest.approx(np.percentile(np.array(done) * 1e3, 50))
    assert fake.memory()[0] == 0


class FailingBatch(FakeBatch):
    """A stand-in whose listed requests (by cell count) fail after a few
    steps the way the device reports it: the slot stops, carries a nonzero
    status (SWE_ENONFINITE) and is listed by poll() as finished."""

    def __init__(self, *a, fail_cells=(), fail_after=3, **kw):
        super().__init__(*a, **kw)
        self.fail_cells, self.fail_after = set(fail_cells), fail_after

    def run(self, k, cfl=0.4):
        super().run(k, cfl)
        for v in self.slots.values():
            if v["cells"] in self.fail_cells and v["steps"] >= self.fail_after:
                v["status"] = 4
                v["steps"] = self.fail_after

    def poll(self):
        return sorted(s for s, v in self.slots.items() if v["t"] >= v["t_end"] or v.get("status", 0))

    def diagnostics(self, slot, check=True):
        d = super().diagnostics(slot, check)
        d["status"] = self.slots[slot].get("status", 0)
        return d


def test_failed_solves_are_reported_failed_and_left_out_of_the_figures():
    fake = FailingBatch(4, 10 ** 6, fail_cells=(77,), fail_after=2)
    reqs = [request(0.0, 100, 1.0), request(0.0, 77, 1.0), request(0.0, 50, 0.5)]
    rep = server(fake).serve(reqs)
    st = {r.index: r.status for r in rep.results}
    assert st == {0: "done", 1: "failed", 2: "done"}
    bad = next(r for r in rep.results if r.index == 1)
    assert bad.state is None and np.isnan(bad.mass) and bad.t < 1.0
    # cell updates and latency percentiles count the completed requests only
    assert rep.cell_updates == pytest.approx(100 * 8 + 50 * 4)
    done = [r.latency for r in rep.results if r.status == "done"]
    assert rep.latency_ms(99) == pytest.approx(np.percentile(np.array(done) * 1e3, 99))
    assert rep.summary()["failed"] == 1
    assert fake.memory()[0] == 0
