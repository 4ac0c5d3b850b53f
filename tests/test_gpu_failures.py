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


# Host-side fault injection (CPT_FAULT_INJECT): a listed site behaves as if
# its allocation, or its threads, had been refused; nothing on the device.

def test_injected_pinned_ring_refusal_then_recovery(monkeypatch):
    w, h, n = 96, 40, 50
    m = synth.scramble_nonzero(synth.random_masks(170, n, h, w), 170)
    with binding.Composite(w, h, chunk_members=8) as comp:
        monkeypatch.setenv("CPT_FAULT_INJECT", "pinned_ring")
        with pytest.raises(binding.CompositeError) as e:
            comp.add(m)                      # pageable: needs the pinned ring
        assert e.value.code == binding.CPT_ENOMEM
        assert comp.n == 0
        monkeypatch.delenv("CPT_FAULT_INJECT")
        comp.add(m)
        got = comp.render_host()
    np.testing.assert_array_equal(got["counts"].astype(np.int64), oracle.count(m))


def test_injected_staging_refusal_at_begin(monkeypatch):
    monkeypatch.setenv("CPT_FAULT_INJECT", "staging_alloc")
    with pytest.raises(binding.CompositeError) as e:
        binding.Composite(64, 8)
    assert e.value.code == binding.CPT_ENOMEM
    monkeypatch.delenv("CPT_FAULT_INJECT")
    with binding.Composite(64, 8) as comp:
        comp.add(np.ones((3, 8, 64), np.uint8))
        assert (comp.render_host()["counts"] == 3).all()


def test_injected_thread_refusal_copies_on_the_calling_thread(monkeypatch):
    w, h, n = 300, 200, 40
    m = synth.random_masks(171, n, h, w)
    monkeypatch.setenv("CPT_FAULT_INJECT", "ingest_threads,engine_plane_unused")
    with binding.Composite(w, h, ingest_threads=8, chunk_members=16) as comp:
        comp.add(m)
        got = comp.render_host()
    np.testing.assert_array_equal(got["counts"].astype(np.int64), oracle.count(m))


def test_injected_engine_and_server_refusals(monkeypatch):
    monkeypatch.setenv("CPT_FAULT_INJECT", "engine_plane,server_stage")
    with binding.Engine() as eng:
        with pytest.raises(binding.CompositeError) as e:
            eng.add_plane(32, 8)
        assert e.value.code == binding.CPT_ENOMEM
        res = torch.zeros((4, 8, 32), dtype=torch.uint8, device="cuda")
        ovf = torch.zeros((4, 8, 32), dtype=torch.uint8).pin_memory()
        with pytest.raises(binding.CompositeError) as e:
            binding.Server(res, ovf)
        assert e.value.code == binding.CPT_ENOMEM
        monkeypatch.delenv("CPT_FAULT_INJECT")
        p = eng.add_plane(32, 8)
        eng.submit([eng.op(p, res)])
        eng.sync()
        assert eng.member_count(p) == 4
