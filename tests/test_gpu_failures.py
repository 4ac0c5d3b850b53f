"""Failure detection without a GPU fault: bounded waits give up and report,
and the context stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("timeout_us", [200, 5000])
def test_device_bounded_wait_gives_up(timeout_us):
    gave_up, waited = binding.composite_selftest_bounded_wait(timeout_us)
    assert gave_up
    assert timeout_us <= waited < timeout_us + 200_000


def test_host_wait_times_out_and_context_recovers():
    # about 10 ms of resident work (32 adds of 512 masks of 2048^2) against a
    # 1 ms wait limit: the wait gives up, nothing is stuck, nothing is lost
    w = h = 2048
    ens = synth.ensemble(3, w, h, 8)
    small = synth.masks(ens)
    dev = torch.from_numpy(small).cuda().repeat(64, 1, 1)
    with binding.Composite(w, h, wait_timeout_ms=1) as comp:
        for _ in range(32):
            comp.add(dev)
        with pytest.raises(binding.CompositeError) as e:
            comp.sync()
        assert e.value.code == binding.CPT_ETIMEOUT
        torch.cuda.synchronize()
        time.sleep(0.05)
        comp.sync()
        got = comp.render_host()
    np.testing.assert_array_equal(got["counts"].astype(np.int64), oracle.count(small) * 32 * 64)
