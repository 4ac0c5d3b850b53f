"""The interactive server (include/composite_server.h): every request's
rendered composite equals the oracle over the session's member set at that
point; a request's result is the same served alone (max_batch 1) and in a
mix; overflow members stream through the staging halves; recompute and
incremental paths agree."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu

W, H = 200, 60
PITCH = 208
N_RES, N_OVF = 40, 30


def ensemble():
    ens = synth.ensemble(77, W, H, N_RES + N_OVF)
    m = synth.scramble_nonzero(synth.masks(ens), 77)
    buf = np.zeros((N_RES + N_OVF, H, PITCH), np.uint8)
    buf[:, :, :W] = m
    res = torch.from_numpy(buf[:N_RES]).cuda()[:, :, :W]
    ovf = torch.from_numpy(buf[N_RES:]).pin_memory()[:, :, :W]
    return m, res, ovf


def trace(seed, n_sessions, n_requests):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_requests):
        s = int(rng.integers(n_sessions))
        k = int(rng.integers(0, 50))
        out.append((s, rng.integers(0, N_RES + N_OVF, k).astype(np.int32)))   # duplicates allowed
    return out


def serve(res, ovf, reqs, n_sessions, **kw):
    outs = []
    with binding.Server(res, ovf, **kw) as srv:
        sessions = [srv.open_session() for _ in range(n_sessions)]
        for i, (s, tog) in enumerate(reqs):
            o = (torch.empty((H, W), dtype=torch.int32, device="cuda"),
                 torch.empty((H, W), dtype=torch.uint8, device="cuda"),
                 torch.empty((H, W, 4), dtype=torch.uint8, device="cuda"))
            srv.request(sessions[s], tog, *o)
            outs.append(o)
            if i % 3 == 0:
                srv.pump()
        srv.drain()
        stats = srv.stats()
    torch.cuda.synchronize()
    return [tuple(t.cpu().numpy() for t in o) for o in outs], stats


def expected_sets(reqs, n_sessions):
    sets = [np.zeros(N_RES + N_OVF, bool) for _ in range(n_sessions)]
    out = []
    for s, tog in reqs:
        for t in tog:
            sets[s][t] ^= True
        out.append(np.flatnonzero(sets[s]))
    return out


def test_every_result_matches_the_oracle_and_alone_equals_mixed():
    m, res, ovf = ensemble()
    reqs = trace(1, 5, 40)
    mixed, st = serve(res, ovf, reqs, 5, max_batch=8, staging_members=7)
    alone, st1 = serve(res, ovf, reqs, 5, max_batch=1, staging_members=7)
    assert st["requests_done"] == 40 and st["cycles"] < st1["cycles"] == 40
    assert st["overflow_uploads"] > 0
    for (counts, bucket, rgba), members in zip(mixed, expected_sets(reqs, 5)):
        c = oracle.count(m[members]) if len(members) else np.zeros((H, W), np.int64)
        b = oracle.bucket(c, len(members))
        np.testing.assert_array_equal(counts.astype(np.int64), c)
        np.testing.assert_array_equal(bucket, b)
        np.testing.assert_array_equal(rgba, oracle.rgba(b))
    for a, b in zip(mixed, alone):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_recompute_path_matches_incremental():
    m, res, ovf = ensemble()
    everything = np.arange(N_RES + N_OVF, dtype=np.int32)
    # fill the set, then toggle almost everything away: the server clears and re-adds
    reqs = [(0, everything), (0, everything[:-3]), (0, np.array([5, 60, 61], np.int32))]
    outs, st = serve(res, ovf, reqs, 1, max_batch=4, staging_members=16)
    assert st["recomputes"] >= 1
    for (counts, _, _), members in zip(outs, expected_sets(reqs, 1)):
        np.testing.assert_array_equal(counts.astype(np.int64), oracle.count(m[members]))


def test_session_rules_and_errors():
    _, res, ovf = ensemble()
    with binding.Server(res, ovf, max_sessions=2) as srv:
        a = srv.open_session()
        srv.open_session()
        with pytest.raises(binding.CompositeError) as e:
            srv.open_session()
        assert e.value.code == binding.CPT_ENOMEM
        with pytest.raises(binding.CompositeError) as e:
            srv.request(a, [N_RES + N_OVF])
        assert e.value.code == binding.CPT_EINVAL
        srv.request(a, [1, 2, 2, 3])
        assert srv.session_members(a) == 2
        with pytest.raises(binding.CompositeError) as e:
            srv.close_session(a)
        assert e.value.code == binding.CPT_ESTATE
        srv.drain()
        srv.close_session(a)
    plane = ((W + 15) // 16 * 16) * H * 4
    with pytest.raises(binding.CompositeError) as e:
        with binding.Server(res, ovf, staging_members=4, hbm_budget_bytes=2 * 4 * PITCH * H + plane // 2) as srv:
            srv.open_session()
    assert e.value.code == binding.CPT_ENOMEM


def test_bit_packed_ensemble_matches_byte_ensemble():
    m, res, ovf = ensemble()
    packed = synth.pack_masks(m)
    wb = packed.shape[-1]
    buf = np.zeros((N_RES + N_OVF, H, 32), np.uint8)
    buf[:, :, :wb] = packed
    pres = torch.from_numpy(buf[:N_RES]).cuda()[:, :, :wb]
    povf = torch.from_numpy(buf[N_RES:]).pin_memory()[:, :, :wb]
    reqs = trace(2, 4, 24)
    as_bytes, _ = serve(res, ovf, reqs, 4, max_batch=6, staging_members=5)
    as_bits, st = serve(pres, povf, reqs, 4, max_batch=6, staging_members=5, mask_format="bits", width=W)
    assert st["overflow_uploads"] > 0
    for a, b in zip(as_bytes, as_bits):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    for (counts, _, _), members in zip(as_bits, expected_sets(reqs, 4)):
        c = oracle.count(m[members]) if len(members) else np.zeros((H, W), np.int64)
        np.testing.assert_array_equal(counts.astype(np.int64), c)


def test_request_histograms_match_the_oracle():
    # composite_server_request_histogram: the class histogram of every
    # request's composite, with and without image outputs, in mixed cycles
    m, res, ovf = ensemble()
    reqs = trace(5, 4, 24)
    hists, buckets = [], []
    with binding.Server(res, ovf, max_batch=8, staging_members=7) as srv:
        sessions = [srv.open_session() for _ in range(4)]
        for i, (s, tog) in enumerate(reqs):
            hist = torch.full((256,), -1, dtype=torch.int64, device="cuda")
            bucket = torch.empty((H, W), dtype=torch.uint8, device="cuda") if i % 2 else None
            srv.request(sessions[s], tog, None, bucket, None, histogram_out=hist)
            hists.append(hist)
            buckets.append(bucket)
            if i % 3 == 0:
                srv.pump()
        srv.drain()
        bad = torch.zeros(258, dtype=torch.int64, device="cuda")
        with pytest.raises(binding.CompositeError) as ei:
            srv.request(sessions[0], [1], histogram_out=bad[1:257])   # 8 bytes off a 16-byte boundary
        assert ei.value.code == binding.CPT_EINVAL
        with pytest.raises(binding.CompositeError) as ei:
            srv.request(sessions[0], [1], histogram_out=np.zeros(256, np.int64))   # pageable host memory
        assert ei.value.code == binding.CPT_EINVAL
        with pytest.raises(ValueError, match="bucket_out"):   # refused by the binding: too short
            srv.request(sessions[0], [1], bucket_out=torch.empty((H - 1, W), dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    for hist, bucket, members in zip(hists, buckets, expected_sets(reqs, 4)):
        c = oracle.count(m[members]) if len(members) else np.zeros((H, W), np.int64)
        b = oracle.bucket(c, len(members))
        np.testing.assert_array_equal(hist.cpu().numpy(), oracle.histogram(b).astype(np.int64))
        if bucket is not None:
            np.testing.assert_array_equal(bucket.cpu().numpy(), b)
