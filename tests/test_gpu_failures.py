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


# A failure part-way through an add or remove: the chunks queued before it
# still fold into the composite while N stays that of the call before, so the
# context must refuse further work until it is cleared (CPT_ESTATE), and a
# clear must bring back exact results.  chunk_fail=K refuses chunk K's upload
# on the host.

def _texture_device(m):
    return torch.from_numpy(m).cuda()


@pytest.mark.parametrize("kind,path", [("pinned", "linear"), ("pageable", "linear"), ("device", "texture"),
                                       ("pinned", "tma")])
@pytest.mark.parametrize("sign", [1, -1])
def test_chunk_failure_poisons_until_clear(monkeypatch, kind, path, sign):
    w, h, n = 96, 40, 22
    m = synth.scramble_nonzero(synth.random_masks(180, n, h, w), 180)
    src = m if kind == "pageable" else (torch.from_numpy(m).pin_memory() if kind == "pinned" else _texture_device(m))
    with binding.Composite(w, h, read_path=path, chunk_members=4, staging_buffers=2) as comp:
        if sign < 0:
            comp.add(src)
        monkeypatch.setenv("CPT_FAULT_INJECT", "chunk_fail=2")
        with pytest.raises(binding.CompositeError) as e:
            (comp.add if sign > 0 else comp.remove)(src)
        assert e.value.code == binding.CPT_ECUDA and "injected" in str(e.value)
        assert comp.n == (0 if sign > 0 else n)          # N is that of the call before
        monkeypatch.delenv("CPT_FAULT_INJECT")
        for call in (lambda: comp.add(src), comp.render_host):
            with pytest.raises(binding.CompositeError) as e:
                call()
            assert e.value.code == binding.CPT_ESTATE and "part-way" in str(e.value)
        comp.sync()                                       # the queued chunks finish; no fault
        comp.clear()
        comp.add(src)
        comp.remove(src[: n // 2])
        got = comp.render_host()
    keep = m[n // 2:]
    np.testing.assert_array_equal(got["counts"].astype(np.int64), oracle.count(keep))
    np.testing.assert_array_equal(got["bucket"], oracle.bucket(oracle.count(keep), len(keep)))


def test_failure_before_the_first_chunk_changes_nothing(monkeypatch):
    w, h, n = 64, 16, 12
    m = synth.random_masks(181, n, h, w)
    pinned = torch.from_numpy(m).pin_memory()
    with binding.Composite(w, h, chunk_members=4) as comp:
        comp.add(pinned[:4])
        monkeypatch.setenv("CPT_FAULT_INJECT", "chunk_fail=0")
        with pytest.raises(binding.CompositeError) as e:
            comp.add(pinned[4:])
        assert e.value.code == binding.CPT_ECUDA
        monkeypatch.delenv("CPT_FAULT_INJECT")
        assert comp.n == 4
        comp.add(pinned[4:])                             # not poisoned: goes on
        got = comp.render_host()
    np.testing.assert_array_equal(got["counts"].astype(np.int64), oracle.count(m))


def test_engine_submit_failure_leaves_planes_unchanged(monkeypatch):
    w, h = 64, 24
    m = synth.random_masks(182, 30, h, w)
    dev = torch.from_numpy(m).cuda()
    with binding.Engine() as eng:
        p = eng.add_plane(w, h)
        eng.submit([eng.op(p, dev[:10])])
        monkeypatch.setenv("CPT_FAULT_INJECT", "engine_submit")
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, dev[10:]), eng.op(p, dev[:5], sign=-1)])
        assert e.value.code == binding.CPT_ECUDA
        monkeypatch.delenv("CPT_FAULT_INJECT")
        assert eng.member_count(p) == 10
        eng.submit([eng.op(p, dev[10:])])
        out = torch.empty((h, w), dtype=torch.int32, device="cuda")
        eng.render([eng.render_op(p, out)])
        eng.sync()
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), oracle.count(m))


def test_server_cycle_failure_drops_its_sessions_only(monkeypatch):
    w, h, pitch, n_res, n_ovf = 96, 20, 96, 12, 16
    m = synth.scramble_nonzero(synth.random_masks(183, n_res + n_ovf, h, w), 183)
    res = torch.from_numpy(m[:n_res]).cuda()
    ovf = torch.from_numpy(m[n_res:]).pin_memory()
    outs = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(3)]
    with binding.Server(res, ovf, max_batch=1, staging_members=4) as srv:
        bad, good = srv.open_session(), srv.open_session()
        # the bad session's request toggles overflow members: its cycle fails at
        # the first overflow chunk, after the resident submit was queued
        srv.request(bad, np.array([0, 1, n_res + 2, n_res + 3], np.int32), outs[0])
        srv.request(bad, np.array([5], np.int32), outs[1])           # queued behind it: dropped
        monkeypatch.setenv("CPT_FAULT_INJECT", "server_chunk_fail=0")
        with pytest.raises(binding.CompositeError) as e:
            srv.pump()
        assert e.value.code == binding.CPT_ECUDA and "dropped" in str(e.value)
        monkeypatch.delenv("CPT_FAULT_INJECT")
        with pytest.raises(binding.CompositeError) as e:
            srv.request(bad, np.array([1], np.int32))
        assert e.value.code == binding.CPT_ESTATE
        ids = np.array([2, 3, n_res + 1, n_res + 7], np.int32)
        srv.request(good, ids, outs[2])
        srv.drain()
        srv.close_session(bad)                          # nothing pending: closes
        st = srv.stats()
    assert st["queued"] == 0 and st["in_flight"] == 0 and st["requests_done"] == 1
    np.testing.assert_array_equal(outs[2].cpu().numpy().astype(np.int64), oracle.count(m[ids]))
