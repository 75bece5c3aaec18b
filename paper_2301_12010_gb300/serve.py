"""Continuous-batching serving loop over the batch ABI.

Requests (scenario solves of different sizes) arrive on a wall-clock
timeline.  Between K-step macro-launches the loop admits waiting requests in
arrival order as slots and HBM budget free up (swe_batch_admit; states stay
resident on the device), launches one persistent kernel that advances every
live scenario (swe_batch_run), and retires the scenarios that reached their
horizon (swe_batch_retire: result copied to the host).  Work of requests that
arrive while others run overlaps on the device.  Latency is arrival ->
result on the host.

A request may carry `deadline` (seconds after its arrival by which the
result is wanted) and `cancel_at` (seconds after its arrival at which the
client withdraws it).  Between launches the loop drops such requests, waiting
or live (a live one is retired without its state and its slot and memory are
freed), and reports them as "expired" or "cancelled".  A request that cannot
be admitted even into an empty batch (larger than the budget or the device
memory) is reported as "rejected".  A scenario that stops before its horizon
because its solve failed (a non-finite state, or a domain that ran dry: the
batch then reports the slot as finished with a nonzero status) is reported as
"failed", without its state; like the other unfinished requests it is left
out of the latency percentiles and of the cell-update count.

Scheduling policy between macro-launches:
  * "all": every live request advances K steps per launch (processor
    sharing by steps: a small request takes as many launches as its steps,
    each as long as the largest live request makes it);
  * "srpt": shortest remaining work first.  The live requests are ordered by
    remaining work (cells x remaining simulated time / cell size: the step is
    proportional to the cell size at similar wave speeds) and the launch
    advances the smallest ones, adding requests until their cells fill the
    GPU (fill_cells); the others wait in their slots (swe_batch_select).
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import OK, Batch, slot_bytes


@dataclasses.dataclass
class Result:
    index: int
    arrival: float      # s, on the loop's clock
    admitted: float
    finished: float
    cells: int
    steps: int
    t: float
    mass: float
    runup_max: float
    state: Optional[tuple] = None
    status: str = "done"  # "done", "expired", "cancelled", "rejected" or "failed"

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclasses.dataclass
class Report:
    results: List[Result]
    wall: float
    macro_launches: int
    max_live: int
    cell_updates: float

    def latency_ms(self, q: float) -> float:
        """Latency percentile (ms) of the completed requests."""
        lat = np.array([r.latency for r in self.results if r.status == "done"]) * 1e3
        return float(np.percentile(lat, q)) if len(lat) else float("nan")

    def count(self, status: str) -> int:
        return sum(1 for r in self.results if r.status == status)

    def summary(self) -> Dict[str, float]:
        out = {"requests": len(self.results), "p50_ms": self.latency_ms(50), "p99_ms": self.latency_ms(99),
               "throughput_cell_updates_per_s": self.cell_updates / self.wall if self.wall > 0 else 0.0,
               "wall_s": self.wall, "macro_launches": self.macro_launches, "max_live_slots": self.max_live}
        for st in ("expired", "cancelled", "rejected", "failed"):
            if self.count(st):
                out[st] = self.count(st)
        return out


class Server:
    """A serving loop with nslots slots and an HBM budget (bytes)."""

    def __init__(self, template, nslots: int = 64, budget_bytes: int = 150 << 30, k_steps: int = 50,
                 cfl: float = 0.4, stream: Optional[int] = None, tile: int = 0, keep_state: bool = False,
                 policy: str = "all", fill_cells: int = 152 * 4 * 3072, batch=None):
        """batch: an object with the Batch interface to serve through instead
        of a new Batch (the host logic can then run against a stand-in)."""
        if policy not in ("all", "srpt"):
            raise ValueError("policy must be 'all' or 'srpt'")
        self.batch = batch if batch is not None else Batch(nslots, budget_bytes, template, stream=stream, tile=tile)
        self.k = int(k_steps)
        self.cfl = float(cfl)
        self.keep_state = keep_state
        self.policy = policy
        self.fill_cells = int(fill_cells)

    def _choose(self, requests, live) -> List[int]:
        """Slots to advance in the next launch under the SRPT policy."""
        t = self.batch.times()
        work = []
        for slot, (k, _) in live.items():
            sc = requests[k].scenario
            rem = max(float(sc.t_end) - float(t[slot]), 0.0)
            work.append((sc.cells * rem / min(sc.dx, sc.dy), slot, sc.cells))
        work.sort()
        chosen, cells = [], 0
        for _, slot, c in work:
            chosen.append(slot)
            cells += c
            if cells >= self.fill_cells:
                break
        return sorted(chosen)

    @staticmethod
    def _overdue(req, now: float, time_scale: float) -> Optional[str]:
        """"cancelled" or "expired" once the request's cancel or deadline
        time (seconds after its arrival) has passed on the loop's clock."""
        arrival = req.arrival / time_scale
        cancel, deadline = getattr(req, "cancel_at", None), getattr(req, "deadline", None)
        if cancel is not None and now >= arrival + cancel / time_scale:
            return "cancelled"
        if deadline is not None and now >= arrival + deadline / time_scale:
            return "expired"
        return None

    def close(self):
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def serve(self, requests: Sequence, time_scale: float = 1.0, max_wall: Optional[float] = None) -> Report:
        """requests: objects with .arrival (s) and .scenario (with .t_end).
        time_scale compresses the arrival timeline (arrival / time_scale)."""
        order = sorted(range(len(requests)), key=lambda k: requests[k].arrival)
        incoming = deque(order)
        waiting: deque = deque()
        live: Dict[int, tuple] = {}  # slot -> (request index, admitted time)
        results: List[Result] = []
        launches = 0
        max_live = 0
        cell_updates = 0.0
        steps_seen: Dict[int, int] = {}
        selected: Optional[List[int]] = None
        t0 = time.perf_counter()
        while incoming or waiting or live:
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                break
            while incoming and requests[incoming[0]].arrival / time_scale <= now:
                waiting.append(incoming.popleft())
            # withdrawn and expired requests leave, waiting or live
            for k in [k for k in waiting if self._overdue(requests[k], now, time_scale)]:
                waiting.remove(k)
                sc = requests[k].scenario
                results.append(Result(k, requests[k].arrival / time_scale, float("nan"), now, sc.cells, 0, 0.0,
                                      float("nan"), float("nan"), None, self._overdue(requests[k], now, time_scale)))
            for slot, (k, adm) in list(live.items()):
                why = self._overdue(requests[k], now, time_scale)
                if why is None:
                    continue
                live.pop(slot)
                selected = None
                d = self.batch.diagnostics(slot, check=False)
                self.batch.retire(slot, want_state=False)
                sc = requests[k].scenario
                results.append(Result(k, requests[k].arrival / time_scale, adm, time.perf_counter() - t0, sc.cells,
                                      d["steps"], d["t"], float("nan"), float("nan"), None, why))
                cell_updates += float(sc.cells) * d["steps"]
            # admit in arrival order while slots and budget allow
            while waiting:
                k = waiting[0]
                sc = requests[k].scenario
                slot = self.batch.try_admit(sc)
                if slot is None:
                    break
                waiting.popleft()
                live[slot] = (k, time.perf_counter() - t0)
                steps_seen[slot] = 0
            max_live = max(max_live, len(live))
            if not live and waiting:
                # not even an empty batch takes the head request: it never will
                k = waiting.popleft()
                sc = requests[k].scenario
                results.append(Result(k, requests[k].arrival / time_scale, float("nan"), time.perf_counter() - t0,
                                      sc.cells, 0, 0.0, float("nan"), float("nan"), None, "rejected"))
                continue
            if not live:
                if incoming:
                    wait = requests[incoming[0]].arrival / time_scale - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            if self.policy == "srpt":
                chosen = self._choose(requests, live) if len(live) > 1 else sorted(live)
                if chosen != selected:
                    self.batch.select(chosen)
                    selected = chosen
            self.batch.run(self.k, self.cfl)
            launches += 1
            for slot in self.batch.poll():
                selected = None  # the work list changes with the retirement
                k, adm = live.pop(slot)
                d = self.batch.diagnostics(slot, check=False)
                sc = requests[k].scenario
                # a slot also finishes when its solve failed (nonzero device
                # status: non-finite state, dry domain) before its horizon
                failed = int(d.get("status", OK)) != OK or not d["t"] >= float(sc.t_end)
                st, m, r = self.batch.retire(slot, want_state=self.keep_state and not failed)
                fin = time.perf_counter() - t0
                if failed:
                    results.append(Result(k, requests[k].arrival / time_scale, adm, fin, sc.cells, d["steps"],
                                          d["t"], float("nan"), float("nan"), None, "failed"))
                    continue
                results.append(Result(k, requests[k].arrival / time_scale, adm, fin, sc.cells, d["steps"], d["t"],
                                      m, r, st))
                cell_updates += float(sc.cells) * d["steps"]
        wall = time.perf_counter() - t0
        return Report(results, wall, launches, max_live, cell_updates)


def budget_for(requests: Sequence) -> int:
    """Device bytes needed to hold every request at once."""
    return int(sum(slot_bytes(r.scenario.nx, r.scenario.ny) for r in requests))
