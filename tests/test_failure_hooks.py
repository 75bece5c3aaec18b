"""Host-side fault injection without a GPU fault: the allocation-failure hook
of the C ABI.  The first device allocation of swe_create fails through the
hook before any CUDA call, so this runs on a machine without a GPU too."""
import pytest

import workloads as W

swe = pytest.importorskip("paper_2301_12010_gb300")


def test_failed_allocation_gives_enomem_and_leaves_nothing_armed():
    sc = W.gaussian_hump(n=16)
    swe.debug_fail_alloc(1)
    try:
        with pytest.raises(swe.SweError) as ei:
            swe.Solver(sc, precision=swe.F32, tile=1)
        assert ei.value.code == swe.ENOMEM
    finally:
        swe.debug_fail_alloc(0)
    with pytest.raises(swe.SweError) as ei:
        swe.debug_fail_alloc(-1)
    assert ei.value.code == swe.EINVAL
