"""Bounded waits of the halo-box copies: a test hook makes every wait expect
bytes that never arrive; the step ends early with a timeout status that the
host reads, and the handle keeps working once the state is set again."""
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


@pytest.mark.parametrize("precision", [swe.F32, swe.F64])
def test_copy_wait_timeout_is_reported_and_recoverable(precision):
    sc = W.gaussian_hump(n=96)
    with swe.Solver(sc, precision=precision, stream=stream()) as ref:
        ref.step(4)
        want = ref.get_state()
        t_want = ref.time()
    with swe.Solver(sc, precision=precision, stream=stream()) as s:
        s.set_wait(0.01, 64)  # 10 ms; 64 bytes that never arrive
        s.step(1)
        with pytest.raises(swe.SweError) as ei:
            s.sync()
        assert ei.value.code == swe.ETIMEOUT
        s.set_wait(1.0, 0)
        s.set_state(sc.h, sc.hu, sc.hv)  # clears the device status; t unchanged
        s.step(4)
        got = s.get_state()
        assert s.time() == t_want
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
