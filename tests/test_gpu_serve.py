"""Continuous-batching serving: requests that arrive while others run are
admitted as slots and budget free up, their work overlaps on the device, and
each result is the same alone and in the mix."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402
from paper_2301_12010_gb300.serve import Server, budget_for  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def small_requests(count, rate, horizon=2.0, seed=5):
    reqs = W.serving_requests(rate=rate, count=count, seed=seed, horizon=horizon, n_range=(96, 192))
    # narrow land strip for these small grids
    out = []
    rng = np.random.Generator(np.random.PCG64(seed))
    shore = W._shoreline_offsets(192, 2.0, seed + 7)
    for r in reqs:
        sc = W.mitigation_scenario(r.scenario.nx, r.scenario.ny, rng, shore, land_width=90.0)
        sc.t_end = horizon
        out.append(W.Request(r.arrival, sc))
    return out


def alone_in_batch(sc, k):
    with swe.Batch(2, 1 << 30, sc, stream=stream()) as b:
        s = b.admit(sc)
        while not b.poll():
            b.run(k)
        st = b.get_state(s)
        d = b.diagnostics(s)
    return st, d


@pytest.mark.parametrize("policy", ["all", "srpt"])
def test_served_results_equal_alone_and_overlap(policy):
    reqs = small_requests(7, rate=200.0)
    # srpt with a fill of one small grid: launches advance only part of the live requests
    with Server(reqs[0].scenario, nslots=3, budget_bytes=1 << 30, k_steps=7, stream=stream(),
                keep_state=True, policy=policy, fill_cells=100 * 100) as srv:
        rep = srv.serve(reqs)
    assert len(rep.results) == len(reqs)
    assert rep.max_live >= 2  # work of different requests overlapped on the device
    for res in rep.results:
        sc = reqs[res.index].scenario
        st, d = alone_in_batch(sc, 5)  # different macro-launch size alone
        assert res.t == d["t"] == sc.t_end and res.steps == d["steps"]
        for a, m in zip(st, res.state):
            assert np.array_equal(a, m)
    s = rep.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_admission_respects_the_hbm_budget():
    rng = np.random.Generator(np.random.PCG64(9))
    shore = W._shoreline_offsets(128, 2.0, 11)
    reqs = []
    for k in range(6):
        sc = W.mitigation_scenario(128, 96, rng, shore, land_width=90.0)
        sc.t_end = 1.0
        reqs.append(W.Request(0.001 * k, sc))
    budget = 2 * swe.slot_bytes(128, 96)  # room for two at a time
    with Server(reqs[0].scenario, nslots=8, budget_bytes=budget, k_steps=10, stream=stream()) as srv:
        rep = srv.serve(reqs)
        used, cap = srv.batch.memory()
    assert len(rep.results) == len(reqs)
    assert rep.max_live == 2 and used == 0 and cap == budget
    assert budget_for(reqs) > budget


def test_paused_slot_keeps_its_state_and_resumes_bit_for_bit():
    reqs = small_requests(2, rate=200.0)
    a, b = reqs[0].scenario.copy(t_end=1e6), reqs[1].scenario.copy(t_end=1e6)
    with swe.Batch(2, 1 << 30, a, stream=stream()) as bt:
        sa, sb = bt.admit(a), bt.admit(b)
        before = bt.get_state(sb)
        bt.select([sa])
        bt.run(6)
        t = bt.times()
        assert t[sa] > 0.0 and t[sb] == 0.0
        for x, y in zip(before, bt.get_state(sb)):
            assert np.array_equal(x, y)
        bt.select(None)
        bt.run(9)
        got = bt.get_state(sb)
        steps_b = bt.diagnostics(sb)["steps"]
    with swe.Batch(2, 1 << 30, b, stream=stream()) as ref:
        s = ref.admit(b)
        ref.run(9)
        want = ref.get_state(s)
        assert ref.diagnostics(s)["steps"] == steps_b == 9
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_served_results_match_the_fp64_oracle():
    # three requests of the serving mix (coast, hills, N-wave; small grids)
    # served together, each result against the FP64 oracle run to the same
    # horizon: relative L2 of the surface anomaly and of the momentum <= 1e-4
    # (FP32), runup within 1 cm
    import oracle
    reqs = small_requests(3, rate=1000.0, horizon=4.0, seed=11)
    with Server(reqs[0].scenario, nslots=3, budget_bytes=1 << 30, k_steps=20, stream=stream(),
                keep_state=True, policy="srpt", fill_cells=10 ** 9) as srv:
        rep = srv.serve(reqs)
    assert sorted(r.index for r in rep.results) == [0, 1, 2] and rep.max_live >= 2
    for res in rep.results:
        sc = reqs[res.index].scenario
        assert res.status == "done" and res.t == sc.t_end
        ref = oracle.Simulation(sc)
        ref.run_until(sc.t_end)
        assert ref.t == sc.t_end
        h, hu, hv = res.state
        et = np.where(h >= sc.h_dry, h + sc.b, 0.0)
        er = np.where(ref.h >= sc.h_dry, ref.h + sc.b, 0.0)
        rel = lambda a, r: float(np.sqrt(((a - r) ** 2).sum() / (r ** 2).sum()))
        assert rel(et, er) <= 1e-4, (res.index, rel(et, er))
        assert rel(hu, ref.hu) <= 1e-4 and rel(hv, ref.hv) <= 1e-4, res.index
        rd = ref.diag()["runup_max"]
        if rd > -np.inf:
            assert abs(res.runup_max - rd) <= 0.01
