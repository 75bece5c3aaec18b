"""The batched ensemble path (persistent multi-scenario kernel) against the
single-scenario path and the FP64 oracle, plus its admission, completion and
bounded-barrier behaviour."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_12010_gb300 as swe  # noqa: E402

GB = 1 << 30
ALL_TILES = list(range(1, 12))  # compiled tile shapes


def stream():
    return torch.cuda.current_stream().cuda_stream


def small_ensemble(count=5, seed=21):
    # small grids with a narrow land strip (sea on the x- side, hills on land)
    ens = W.mitigation_ensemble(count=count, seed=seed, nx_range=(96, 224), ny_range=(32, 160), land_width=90.0)
    return [sc.copy(t_end=1e6) for sc in ens]


def alone(sc, steps, cfl=0.4):
    with swe.Solver(sc, precision=swe.F32, stream=stream()) as s:
        s.step(steps, cfl)
        st = s.get_state()
        d = s.diagnostics()
    return st, d


def batch_run(scs, steps, tile=0, runs=(20, 15)):
    with swe.Batch(max(2, len(scs)), 4 * GB, scs[0], stream=stream(), tile=tile) as b:
        slots = [b.admit(sc) for sc in scs]
        done = 0
        for k in runs:
            b.run(k)
            done += k
        assert done == steps
        return [(b.get_state(s), b.diagnostics(s)) for s in slots]


@pytest.mark.parametrize("tile", ALL_TILES)
def test_batch_result_is_the_same_alone_and_in_the_mix(tile):
    # each scenario keeps its own wave speeds, dt and time: bit-for-bit the
    # same whether it runs alone or with the others
    ens = small_ensemble()
    mix = batch_run(ens, 35, tile)
    for sc, (st_mix, d_mix) in zip(ens, mix):
        (st_alone, d_alone), = batch_run([sc], 35, tile)
        for a, m in zip(st_alone, st_mix):
            assert np.array_equal(a, m)
        assert d_alone["t"] == d_mix["t"] and d_mix["steps"] == 35


def test_result_is_the_same_whichever_kernel_form_the_launch_takes():
    # a launch with few tiles per CTA runs the run-time-stage form of the
    # batch kernel, a large one the inlined form: a coast alone (small launch)
    # and inside a mix of 4000+ tiles (large launch) must agree bit for bit
    ens = W.mitigation_ensemble()
    sc = small_ensemble(1, seed=9)[0]
    assert sum(e.cells for e in ens) // 3072 > 24 * 152
    with swe.Batch(80, 16 * GB, sc, stream=stream(), tile=7) as b:
        s = b.admit(sc)
        b.run(12)
        alone = b.get_state(s)
    with swe.Batch(80, 16 * GB, sc, stream=stream(), tile=7) as b:
        for e in ens:
            b.admit(e.copy(t_end=1e6))
        s = b.admit(sc)
        b.run(12)
        mixed = b.get_state(s)
    for x, y in zip(alone, mixed):
        assert np.array_equal(x, y)


def test_paused_and_resumed_in_turn_is_the_same_as_alone():
    # scenarios advanced in turn, one or two per launch, the others paused
    # (swe_batch_select): every launch puts another scenario at the same
    # place of the slot table, whose tensor maps the kernel must then read
    # afresh; each result equals the scenario run alone, bit for bit
    ens = small_ensemble(5, seed=17)
    alone_res = []
    for sc in ens:
        with swe.Batch(2, GB, sc, stream=stream()) as b:
            s = b.admit(sc.copy(t_end=0.6))
            while not b.poll():
                b.run(6)
            alone_res.append(b.get_state(s))
    for width in (1, 2):
        with swe.Batch(8, GB, ens[0], stream=stream()) as b:
            slots = [b.admit(sc.copy(t_end=0.6)) for sc in ens]
            done, it = {}, 0
            while len(done) < len(slots) and it < 400:
                live = [s for s in slots if s not in done]
                b.select([live[(it + j) % len(live)] for j in range(min(width, len(live)))])
                b.run(6)
                for s in b.poll():
                    if s not in done:
                        done[s] = b.get_state(s)
                it += 1
            for k, s in enumerate(slots):
                for x, y in zip(done[s], alone_res[k]):
                    assert np.array_equal(x, y), (width, k)


def test_work_chunks_that_cross_many_scenarios():
    # sixty one-tile grids among four larger ones, more tiles than CTAs: each
    # CTA's chunk of the work list crosses several scenarios (the per-CTA
    # cursor moves from slot to slot inside a launch); every result is still
    # bit for bit that of the scenario run alone
    rng = np.random.default_rng(31)
    scs = []
    for k in range(64):
        n = 300 + 64 * (k // 16) if k % 16 == 0 else int(rng.integers(3, 30))
        scs.append(W.gaussian_hump(n=n, sigma_cells=max(1.0, n / 8.0)).copy(t_end=1e6))
    tiles = sum(-(-sc.nx // 96) * -(-sc.ny // 32) for sc in scs)
    assert tiles > 2 * torch.cuda.get_device_properties(0).multi_processor_count
    mix = batch_run(scs, 12, tile=7, runs=(12,))
    for sc, (st_mix, d_mix) in zip(scs, mix):
        (st_alone, d_alone), = batch_run([sc], 12, tile=7, runs=(12,))
        for a, m in zip(st_alone, st_mix):
            assert np.array_equal(a, m)
        assert d_alone["t"] == d_mix["t"] and d_mix["steps"] == 12


def test_work_order_does_not_change_results():
    # two grids of more than 2 x 152 tiles each run in strided order (CTA b
    # takes items b, b + G, ...); with a small grid in the table the order is
    # contiguous chunks.  Each scenario's result is bit for bit the same.
    big = [W.gaussian_hump(n=n, sigma_cells=n / 12.0).copy(t_end=1e6) for n in (1024, 1056)]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert all(-(-sc.nx // 96) * -(-sc.ny // 32) >= 2 * sms for sc in big)
    strided = batch_run(big, 6, tile=7, runs=(6,))
    mixed = batch_run(big + small_ensemble(2, seed=3), 6, tile=7, runs=(6,))
    for (st_s, d_s), (st_m, d_m) in zip(strided, mixed[:2]):
        for a, m in zip(st_s, st_m):
            assert np.array_equal(a, m)
        assert d_s["t"] == d_m["t"]
    (h, hu, hv), d = strided[0]
    (rh, rhu, rhv), dr = alone(big[0], 6)
    assert np.sqrt(((h - rh) ** 2).sum() / (rh ** 2).sum()) <= 1e-6


def test_batch_matches_single_scenario_solver():
    # same arithmetic in a separately compiled kernel: FP32 rounding level
    ens = small_ensemble()
    mix = batch_run(ens, 35)
    for sc, ((h, hu, hv), d) in zip(ens, mix):
        (rh, rhu, rhv), dr = alone(sc, 35)
        et, er = h + sc.b, rh + sc.b
        assert np.sqrt(((et - er) ** 2).sum() / (er ** 2).sum()) <= 1e-6
        assert np.abs(hu - rhu).max() <= 1e-4 * max(np.abs(rhu).max(), 1.0)
        assert d["t"] == pytest.approx(dr["t"], rel=1e-6)


def test_batch_matches_fp64_oracle():
    sc = small_ensemble(1, seed=5)[0]
    ref = oracle.Simulation(sc)
    ref.step(40)
    with swe.Batch(2, GB, sc, stream=stream()) as b:
        s = b.admit(sc)
        b.run(40)
        h, hu, hv = b.get_state(s)
    et = np.where(h >= 1e-5, h + sc.b, 0.0)
    er = np.where(ref.h >= 1e-5, ref.h + sc.b, 0.0)
    assert np.sqrt(((et - er) ** 2).sum() / (er ** 2).sum()) <= 1e-4


def test_ensemble_at_full_size_matches_fp64_oracle():
    # the ensemble of the batched-ensemble workload itself (64 coasts of
    # 512-1024 x 256-1024 cells, hills and a shoreline): the largest and the
    # smallest coast, each run in one batch together with two others, against
    # the oracle after 30 steps
    ens = W.mitigation_ensemble()
    sizes = [sc.cells for sc in ens]
    pick = [int(np.argmax(sizes)), int(np.argmin(sizes))]
    others = [k for k in range(len(ens)) if k not in pick][:2]
    with swe.Batch(4, 8 * GB, ens[0], stream=stream()) as b:
        slots = {k: b.admit(ens[k]) for k in pick + others}
        b.run(30)
        got = {k: (b.get_state(slots[k]), b.diagnostics(slots[k])) for k in pick}
    for k in pick:
        sc = ens[k]
        ref = oracle.Simulation(sc)
        ref.step(30)
        (h, hu, hv), d = got[k]
        et = np.where(h >= 1e-5, h + sc.b, 0.0)
        er = np.where(ref.h >= 1e-5, ref.h + sc.b, 0.0)
        assert np.sqrt(((et - er) ** 2).sum() / (er ** 2).sum()) <= 1e-4, sc.name
        assert np.sqrt(((hu - ref.hu) ** 2).sum() / (ref.hu ** 2).sum()) <= 1e-4, sc.name
        assert d["t"] == pytest.approx(ref.t, rel=1e-5), sc.name
        rd = ref.diag()
        if rd["runup_max"] > -np.inf:
            assert abs(d["runup_max"] - rd["runup_max"]) <= 0.01, sc.name


def test_batch_with_the_inflow_edge_matches_fp64_oracle():
    # coastal DEMs with the N-wave inflow edge, Manning friction and a dry
    # shore, each starting at its own time, advanced together in one batch
    cases = [W.coastal_dem(n=n, dx=dx, t0=t0) for n, dx, t0 in ((96, 150.0, 500.0), (128, 120.0, 450.0),
                                                                 (160, 100.0, 520.0))]
    with swe.Batch(4, 4 * GB, cases[0], stream=stream()) as b:
        slots = [b.admit(sc, t_end=1e6) for sc in cases]
        b.run(20)
        got = [(b.get_state(s), b.diagnostics(s)) for s in slots]
    for sc, ((h, hu, hv), d) in zip(cases, got):
        ref = oracle.Simulation(sc)
        ref.step(20)
        rd = ref.diag()
        et = np.where(h >= 1e-5, h + sc.b, 0.0)
        er = np.where(ref.h >= 1e-5, ref.h + sc.b, 0.0)
        assert np.sqrt(((et - er) ** 2).sum() / (er ** 2).sum()) <= 1e-4, sc.name
        assert np.sqrt(((hu - ref.hu) ** 2).sum() / (ref.hu ** 2).sum()) <= 1e-4, sc.name
        assert d["t"] == pytest.approx(rd["t"], rel=1e-6), sc.name
        assert d["boundary_mass"] == pytest.approx(rd["boundary_mass"], rel=1e-4), sc.name


def test_batch_with_periodic_sides_matches_fp64_oracle():
    # flow down a periodic 1:20 slope with Manning friction (bed offset of one
    # period): two discharges in one batch
    from tests.analytic import manning_normal_discharge
    qn = manning_normal_discharge(0.5, 1 / 20, 0.033)
    cases = [W.manning_slope(nx=64, ny=8, q=f * qn) for f in (0.8, 1.2)]
    with swe.Batch(2, GB, cases[0], stream=stream()) as b:
        slots = [b.admit(sc, t_end=1e6) for sc in cases]
        b.run(60)
        got = [b.get_state(s) for s in slots]
    for sc, (h, hu, hv) in zip(cases, got):
        ref = oracle.Simulation(sc)
        ref.step(60)
        assert np.sqrt(((h - ref.h) ** 2).sum() / (ref.h ** 2).sum()) <= 1e-5
        assert np.sqrt(((hu - ref.hu) ** 2).sum() / (ref.hu ** 2).sum()) <= 1e-4


def test_fp64_batch_matches_fp64_oracle_and_is_the_same_alone_and_in_the_mix():
    # the batch path's parity mode: every scenario of an FP64 batch against
    # the oracle to 1e-10, and one of them run alone bit for bit
    ens = small_ensemble(4, seed=13)
    with swe.Batch(4, GB, ens[0], stream=stream(), precision=swe.F64) as b:
        slots = [b.admit(sc) for sc in ens]
        b.run(25)
        mix = [(b.get_state(s), b.diagnostics(s)) for s in slots]
        _, m0, _ = b.retire(slots[0])
    ref0 = oracle.Simulation(ens[0])
    ref0.step(25)
    assert abs(m0 - ref0.diag()["mass"]) <= 1e-11 * m0
    for sc, ((h, hu, hv), d) in zip(ens, mix):
        ref = oracle.Simulation(sc)
        ref.step(25)
        for x, r in ((h, ref.h), (hu, ref.hu), (hv, ref.hv)):
            assert np.abs(x - r).max() <= 1e-10, sc.name
        assert d["t"] == pytest.approx(ref.t, rel=1e-12)
        assert d["clamp_mass"] == pytest.approx(ref.diag()["clamp_mass"], rel=1e-8, abs=1e-9)
    with swe.Batch(1, GB, ens[2], stream=stream(), precision=swe.F64) as b:
        s = b.admit(ens[2])
        b.run(25)
        alone = b.get_state(s)
    for x, y in zip(alone, mix[2][0]):
        assert np.array_equal(x, y)


def test_batch_stops_at_t_end_and_reports_done():
    ens = small_ensemble(3, seed=8)
    with swe.Batch(4, GB, ens[0], stream=stream()) as b:
        s0 = b.admit(ens[0], t_end=0.7)
        s1 = b.admit(ens[1], t_end=1e6)
        b.run(50)
        assert b.poll() == [s0]
        d0 = b.diagnostics(s0)
        assert d0["t"] == 0.7
        st, m, r = b.retire(s0)
        ref, dr = alone(ens[0].copy(t_end=0.7), 0)
        assert st[0].shape == ens[0].h.shape and m > 0
        assert b.diagnostics(s1)["steps"] == 50


def test_batch_budget_full_and_retire_accounting():
    ens = small_ensemble(3, seed=9)
    need = [swe.slot_bytes(sc.nx, sc.ny) for sc in ens]
    with swe.Batch(2, need[0] + need[1], ens[0], stream=stream()) as b:
        a = b.admit(ens[0])
        c = b.admit(ens[1])
        assert b.memory()[0] == need[0] + need[1]
        with pytest.raises(swe.SweError) as ei:
            b.admit(ens[2])
        assert ei.value.code in (swe.EFULL, swe.EBUDGET)
        b.retire(a, want_state=False)
        assert b.memory()[0] == need[1]
        assert b.try_admit(ens[2]) is not None or need[2] > need[0]


def test_batch_barrier_timeout_is_reported_and_recoverable():
    ens = small_ensemble(2, seed=13)
    ref = batch_run(ens, 12, runs=(12,))
    with swe.Batch(4, GB, ens[0], stream=stream()) as b:
        slots = [b.admit(sc) for sc in ens]
        b.set_barrier(0.02, extra_arrivals=1)  # waits for an arrival that never comes
        b.run(1)
        assert b.status() == swe.ETIMEOUT
        b.set_barrier(1.0, 0)
        assert b.status() == swe.OK
        b.run(12)
        for s, (st, d) in zip(slots, ref):
            got = b.get_state(s)
            for g, r in zip(got, st):
                assert np.array_equal(g, r)
