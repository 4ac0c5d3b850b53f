"""The batched engine (include/composite_engine.h) against the CPU oracle:
many planes of different shapes in one persistent launch, member index lists,
add/remove, underflow per plane, CUDA-graph capture/replay and the autotuner."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu


def padded(m: np.ndarray):
    """Device copy of uint8[n, H, W] with rows padded to 16 bytes."""
    n, h, w = m.shape
    pitch = (w + 15) // 16 * 16
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(m).cuda()
    return buf[:, :, :w]


def outputs(w, h, count_bits=32):
    # counts of a 16-bit plane come back as uint16 (held in an int16 tensor)
    return (torch.empty((h, w), dtype=torch.int32 if count_bits == 32 else torch.int16, device="cuda"),
            torch.empty((h, w), dtype=torch.uint8, device="cuda"),
            torch.empty((h, w, 4), dtype=torch.uint8, device="cuda"))


def check(outs, masks_np, lut=None):
    counts, bucket, rgba = outs
    c = oracle.count(masks_np)
    b = oracle.bucket(c, masks_np.shape[0])
    got = counts.cpu().numpy()
    if got.dtype == np.int16:
        got = got.view(np.uint16)
    np.testing.assert_array_equal(got.astype(np.int64), c)
    np.testing.assert_array_equal(bucket.cpu().numpy(), b)
    np.testing.assert_array_equal(rgba.cpu().numpy(), oracle.rgba(b, lut))


SHAPES = [(1024, 1024, 16), (13, 7, 5), (100, 37, 40), (257, 131, 300), (4096, 3, 9), (1, 1, 2), (48, 600, 1)]


@pytest.mark.parametrize("count_bits", [32, 16])
@pytest.mark.parametrize("schedule", ["persistent", "grid"])
def test_many_planes_one_launch(schedule, count_bits):
    with binding.Engine(schedule=schedule) as eng:
        data, ops, rops, outs = [], [], [], []
        for i, (w, h, n) in enumerate(SHAPES):
            m = synth.scramble_nonzero(synth.random_masks(50 + i, n, h, w, density=0.3 + 0.05 * i), i)
            p = eng.add_plane(w, h, count_bits)
            dev = padded(m)
            o = outputs(w, h, count_bits)
            data.append((m, dev))
            outs.append(o)
            ops.append(eng.op(p, dev))
            rops.append(eng.render_op(p, *o))
        eng.submit(ops)
        eng.render(rops)
        eng.sync()
        for (m, _), o, (w, h, n), p in zip(data, outs, SHAPES, range(len(SHAPES))):
            assert eng.member_count(p) == n
            check(o, m)


@pytest.mark.parametrize("count_bits", [32, 16])
@pytest.mark.parametrize("schedule", ["persistent", "grid"])
def test_index_lists_add_and_remove(schedule, count_bits):
    w, h, total = 300, 70, 500
    ens = synth.scramble_nonzero(synth.random_masks(60, total, h, w, density=0.2), 60)
    dev = padded(ens)
    rng = np.random.default_rng(1)
    a = rng.choice(total, 300, replace=False).astype(np.int32)
    b = rng.choice(total, 120, replace=False).astype(np.int32)
    drop = a[:170]
    with binding.Engine(slab_members=64, schedule=schedule) as eng:
        p = eng.add_plane(w, h, count_bits)
        q = eng.add_plane(w, h, count_bits)
        ia, ib, idrop = (torch.from_numpy(x).cuda() for x in (a, b, drop))
        eng.submit([eng.op(p, dev, 1, ia), eng.op(q, dev, 1, ib), eng.op(p, dev, 1, ib)])
        eng.submit([eng.op(p, dev, -1, idrop)])
        op_, oq = outputs(w, h, count_bits), outputs(w, h, count_bits)
        eng.render([eng.render_op(p, *op_), eng.render_op(q, *oq)])
        eng.sync()
        keep = np.concatenate([a[170:], b])
        check(op_, ens[keep])
        check(oq, ens[b])
        assert eng.member_count(p) == len(keep)


@pytest.mark.parametrize("count_bits", [32, 16])
def test_underflow_is_reported_per_plane_and_cleared(count_bits):
    w, h = 64, 20
    m = synth.random_masks(61, 2, h, w, density=0.5)
    dev = padded(m)
    with binding.Engine() as eng:
        good = eng.add_plane(w, h, count_bits)
        bad = eng.add_plane(w, h, count_bits)
        eng.submit([eng.op(good, dev), eng.op(bad, dev[:1])])
        eng.submit([eng.op(bad, dev[1:], -1)])
        with pytest.raises(binding.CompositeError) as e:
            eng.sync()
        assert e.value.code == binding.CPT_EUNDERFLOW and e.value.plane == bad
        eng.clear(bad)
        eng.submit([eng.op(bad, dev)])
        o = outputs(w, h, count_bits)
        eng.render([eng.render_op(bad, *o)])
        eng.sync()
        check(o, m)


@pytest.mark.parametrize("count_bits", [32, 16])
def test_capture_replay_matches_direct_and_repeats(count_bits):
    shapes = [(512, 64, 37), (77, 45, 260), (16, 16, 3)]
    with binding.Engine() as eng:
        items = []
        for i, (w, h, n) in enumerate(shapes):
            m = synth.random_masks(70 + i, n, h, w, density=0.4)
            items.append((m, padded(m), eng.add_plane(w, h, count_bits), outputs(w, h, count_bits)))
        ops = [eng.op(p, dev) for _, dev, p, _ in items]
        rops = [eng.render_op(p, *o) for _, _, p, o in items]
        eng.capture(ops, rops)
        for _ in range(3):
            eng.replay()
            eng.sync()
            for m, _, p, o in items:
                check(o, m)
                assert eng.member_count(p) == m.shape[0]


def test_tuner_picks_a_candidate_and_keeps_results_exact():
    shapes = [(1024, 256, 300), (130, 90, 40)]
    with binding.Engine() as eng:
        items = []
        for i, (w, h, n) in enumerate(shapes):
            m = synth.random_masks(80 + i, n, h, w, density=0.25)
            items.append((m, padded(m), eng.add_plane(w, h), outputs(w, h)))
        slab, ctas = eng.tune([eng.op(p, dev) for _, dev, p, _ in items], repeats=1)
        assert slab in (32, 64, 128, 255) and ctas in (0, 3, 4, 5)
        assert eng.tuning() == (slab, ctas)
        eng.render([eng.render_op(p, *o) for _, _, p, o in items])
        eng.sync()
        for m, _, p, o in items:
            check(o, m)


def test_invalid_ops_rejected_before_anything_runs():
    with binding.Engine() as eng:
        p = eng.add_plane(32, 8)
        dev = padded(synth.random_masks(90, 2, 8, 32))
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p + 7, dev)])
        assert e.value.code == binding.CPT_EINVAL
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, dev, -1)])
        assert e.value.code == binding.CPT_EINVAL
        odd = torch.zeros((2, 8, 33), dtype=torch.uint8, device="cuda")[:, :, 1:]
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, odd)])
        assert e.value.code == binding.CPT_EINVAL
        assert eng.member_count(p) == 0


def test_sixteen_bit_plane_limit():
    w, h = 16, 2
    with binding.Engine() as eng:
        with pytest.raises(binding.CompositeError) as e:
            eng.add_plane(w, h, 8)
        assert e.value.code == binding.CPT_EINVAL
        p = eng.add_plane(w, h, 16)
        ones = torch.ones((65535, h, w), dtype=torch.uint8, device="cuda")
        eng.submit([eng.op(p, ones)])
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, ones[:1])])
        assert e.value.code == binding.CPT_EINVAL
        o = outputs(w, h, 16)
        eng.render([eng.render_op(p, *o)])
        eng.sync()
        assert eng.member_count(p) == 65535
        assert (o[0].cpu().numpy().view(np.uint16) == 65535).all() and (o[1].cpu().numpy() == 255).all()


def padded_bits(m: np.ndarray):
    """Device copy of bit-packed masks with rows padded to 16 bytes."""
    p = synth.pack_masks(m)
    n, h, wb = p.shape
    pitch = (wb + 15) // 16 * 16
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :wb] = torch.from_numpy(p).cuda()
    return buf[:, :, :wb]


@pytest.mark.parametrize("count_bits", [32, 16])
@pytest.mark.parametrize("schedule", ["persistent", "grid"])
def test_bit_packed_ops_mixed_with_byte_ops(schedule, count_bits):
    shapes = [(300, 70, 280), (33, 9, 5), (1024, 64, 40)]
    with binding.Engine(schedule=schedule) as eng:
        items = []
        for i, (w, h, n) in enumerate(shapes):
            m = synth.scramble_nonzero(synth.random_masks(120 + i, n, h, w, density=0.3), i)
            p = eng.add_plane(w, h, count_bits)
            items.append((m, p, outputs(w, h, count_bits)))
        ops = []
        for i, (m, p, _) in enumerate(items):
            half = m.shape[0] // 2
            ops.append(eng.op(p, padded_bits(m[:half]), mask_format="bits"))
            ops.append(eng.op(p, padded(m[half:])))
        eng.submit(ops)
        # remove a gathered subset again, bit-packed, then re-add it as bytes
        m0, p0, _ = items[0]
        idx = torch.arange(0, m0.shape[0] // 2, 3, dtype=torch.int32, device="cuda")
        bits0 = padded_bits(m0[: m0.shape[0] // 2])
        eng.submit([eng.op(p0, bits0, -1, idx, mask_format="bits")])
        eng.submit([eng.op(p0, padded(m0[: m0.shape[0] // 2]), 1, idx)])
        eng.render([eng.render_op(p, *o) for _, p, o in items])
        eng.sync()
        for m, p, o in items:
            check(o, m)


def pinned_padded(m: np.ndarray, extra_rows: int = 0):
    """Pinned host copy of uint8[n, H, W], rows padded to 16 bytes and each
    raster followed by extra_rows rows of nonzero padding (stride > pitch*H)."""
    n, h, w = m.shape
    pitch = (w + 15) // 16 * 16
    buf = torch.full((n, h + extra_rows, pitch), 255, dtype=torch.uint8).pin_memory()
    buf[:, :h, :w] = torch.from_numpy(m)
    return buf[:, :h, :w]


@pytest.mark.parametrize("count_bits", [32, 16])
@pytest.mark.parametrize("stage_mib", [1, 256])
def test_host_ops_stream_through_staging(count_bits, stage_mib):
    # ops on pinned host members, mixed with device ops in one submit; a 1 MiB
    # staging buffer cuts the host rasters into many chunks that split ops
    with binding.Engine(staging_bytes=stage_mib << 20, staging_buffers=3) as eng:
        ops, rops, outs, kept = [], [], [], []
        for i, (w, h, n) in enumerate([(1024, 1024, 6), (257, 131, 300), (13, 7, 5), (4096, 3, 9), (100, 37, 40)]):
            m = synth.scramble_nonzero(synth.random_masks(80 + i, n, h, w, density=0.4), 80 + i)
            p = eng.add_plane(w, h, count_bits)
            half = n // 2
            host = pinned_padded(m[:half], extra_rows=i % 2)
            dev = padded(m[half:])
            ops += [eng.op(p, host), eng.op(p, dev)]
            o = outputs(w, h, count_bits)
            outs.append(o)
            rops.append(eng.render_op(p, *o))
            kept.append((m, host, p))
        eng.submit(ops)
        # remove the host half again, then add it back, through the staging
        eng.submit([eng.op(p, host, sign=-1) for _, host, p in kept])
        eng.submit([eng.op(p, host) for _, host, p in kept])
        eng.render(rops)
        eng.sync()
        for (m, _, p), o in zip(kept, outs):
            assert eng.member_count(p) == m.shape[0]
            check(o, m)


def test_host_ops_rejections():
    with binding.Engine() as eng:
        p = eng.add_plane(64, 8)
        host = pinned_padded(synth.random_masks(90, 4, 8, 64))
        idx = torch.arange(2, dtype=torch.int32, device="cuda")
        for bad in (eng.op(p, host, index=idx), eng.op(p, synth.random_masks(91, 2, 8, 64))):
            with pytest.raises(binding.CompositeError) as e:
                eng.submit([bad])
            assert e.value.code == binding.CPT_EINVAL
        assert eng.member_count(p) == 0
    with binding.Engine(staging_bytes=1 << 20) as eng:
        p = eng.add_plane(2048, 1024)      # a 2 MiB raster cannot fit a 1 MiB buffer
        big = pinned_padded(np.ones((1, 1024, 2048), np.uint8))
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, big)])
        assert e.value.code == binding.CPT_EINVAL and "staging" in str(e.value)


def test_tuner_with_host_ops_reports_every_dimension():
    with binding.Engine() as eng:
        data, ops = [], []
        for i, (w, h, n) in enumerate([(512, 512, 64), (256, 1024, 40)]):
            m = synth.random_masks(95 + i, n, h, w)
            p = eng.add_plane(w, h)
            host = pinned_padded(m)
            data.append((m, p))
            ops.append(eng.op(p, host))
        slab, ctas = eng.tune(ops, repeats=1)
        cfg = eng.config()
        assert cfg["slab_members"] == slab and cfg["item_member_groups"] in (256, 512, 1024, 2048)
        assert cfg["staging_buffers"] in (2, 3, 4) and cfg["staging_bytes"] in [m << 20 for m in (64, 128, 256, 512)]
        outs = [outputs(512, 512), outputs(256, 1024)]
        eng.render([eng.render_op(p, *o) for (_, p), o in zip(data, outs)])
        eng.sync()
        for (m, _), o in zip(data, outs):
            check(o, m)


def test_host_chunk_failure_poisons_the_submit_planes(monkeypatch):
    with binding.Engine(staging_bytes=1 << 20) as eng:
        m = synth.random_masks(97, 8, 256, 1024)          # 256 KiB rasters: 4 per chunk
        p = eng.add_plane(1024, 256)
        q = eng.add_plane(64, 8)
        other = synth.random_masks(98, 3, 8, 64)
        eng.submit([eng.op(q, padded(other))])
        host = pinned_padded(m)
        monkeypatch.setenv("CPT_FAULT_INJECT", "engine_chunk_fail=1")
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, host)])
        assert e.value.code == binding.CPT_ECUDA
        monkeypatch.delenv("CPT_FAULT_INJECT")
        assert eng.member_count(p) == 0
        with pytest.raises(binding.CompositeError) as e:
            eng.submit([eng.op(p, host)])
        assert e.value.code == binding.CPT_ESTATE
        with pytest.raises(binding.CompositeError) as e:
            eng.render([eng.render_op(p, *outputs(1024, 256))])
        assert e.value.code == binding.CPT_ESTATE
        eng.clear(p)
        eng.submit([eng.op(p, host)])
        o, oq = outputs(1024, 256), outputs(64, 8)
        eng.render([eng.render_op(p, *o), eng.render_op(q, *oq)])
        eng.sync()
    check(o, m)
    check(oq, other)


@pytest.mark.parametrize("count_bits", [32, 16])
def test_clear_many_in_one_launch(count_bits):
    shapes = [(1024, 1024, 12), (13, 7, 5), (257, 131, 40), (4096, 3, 9)]
    with binding.Engine() as eng:
        planes, data = [], []
        for i, (w, h, n) in enumerate(shapes):
            m = synth.random_masks(300 + i, n, h, w)
            p = eng.add_plane(w, h, count_bits)
            dev = padded(m)
            eng.submit([eng.op(p, dev), eng.op(p, dev)])
            planes.append(p)
            data.append((m, dev))
        eng.clear_many(planes[:3] + [planes[0]])        # a repeated id is cleared once
        assert [eng.member_count(p) for p in planes] == [0, 0, 0, 2 * shapes[3][2]]
        eng.submit([eng.op(p, dev) for p, (_, dev) in zip(planes[:3], data[:3])])
        outs = [outputs(w, h, count_bits) for w, h, _ in shapes]
        eng.render([eng.render_op(p, *o) for p, o in zip(planes, outs)])
        eng.sync()
        for (m, _), o in zip(data[:3], outs[:3]):
            check(o, m)
        np.testing.assert_array_equal(outs[3][0].cpu().numpy().astype(np.int64) & 0xFFFF,
                                      2 * oracle.count(data[3][0]))
        with pytest.raises(binding.CompositeError) as e:
            eng.clear_many([planes[0], 999])
        assert e.value.code == binding.CPT_EINVAL


def test_host_ops_bit_packed_through_staging():
    w, h, n = 512, 96, 30
    m = synth.scramble_nonzero(synth.random_masks(310, n, h, w, density=0.4), 310)
    packed = synth.pack_masks(m)                    # rows of 64 bytes: 16-byte aligned
    host = torch.from_numpy(packed).pin_memory()
    with binding.Engine(staging_bytes=1 << 20) as eng:
        p = eng.add_plane(w, h)
        eng.submit([eng.op(p, host, mask_format="bits"), eng.op(p, padded(m[:10]))])
        eng.submit([eng.op(p, host[:10], sign=-1, mask_format="bits")])
        o = outputs(w, h)
        eng.render([eng.render_op(p, *o)])
        eng.sync()
    check(o, np.concatenate([m[10:], m[:10]]))


@pytest.mark.parametrize("hist", [False, True])
def test_op_lists_longer_than_the_shared_memory_index(hist):
    # 2500 planes, one op each, and 2500 render ops in one launch: more than
    # the 2048 first items the kernels keep in shared memory, so the clear,
    # accumulate and render launches look the ops up in global memory
    n_planes, w, h = 2500, 24, 3
    m = synth.scramble_nonzero(synth.random_masks(300, 5, h, w, density=0.4), 300)
    dev = padded(m)
    with binding.Engine() as eng:
        planes = [eng.add_plane(w, h, 16 if i % 2 else 32) for i in range(n_planes)]
        eng.clear_many(planes)
        eng.submit([eng.op(p, dev[: 1 + i % 5]) for i, p in enumerate(planes)])
        buckets = torch.empty((n_planes, h, w), dtype=torch.uint8, device="cuda")
        hists = torch.empty((n_planes, 256), dtype=torch.int64, device="cuda") if hist else None
        eng.render([eng.render_op(p, None, buckets[i], None, hists[i] if hist else None)
                    for i, p in enumerate(planes)])
        eng.sync()
        got_b = buckets.cpu().numpy()
        got_h = hists.cpu().numpy() if hist else None
    for k in range(1, 6):
        b = oracle.bucket(oracle.count(m[:k]), k)
        for i in range(k - 1, n_planes, 5):
            np.testing.assert_array_equal(got_b[i], b, err_msg=f"plane {i}")
            if hist:
                np.testing.assert_array_equal(got_h[i], oracle.histogram(b).astype(np.int64), err_msg=f"plane {i}")


def test_index_lists_are_checked_by_the_binding():
    w, h = 64, 8
    dev = padded(synth.random_masks(92, 6, h, w))
    with binding.Engine() as eng:
        p = eng.add_plane(w, h)
        for bad in (torch.tensor([0, 6], dtype=torch.int32, device="cuda"),     # past the last member
                    torch.tensor([-1], dtype=torch.int32, device="cuda"),
                    torch.tensor([0, 1], dtype=torch.int64, device="cuda"),     # wrong type
                    torch.tensor([0, 1], dtype=torch.int32)):                   # host memory
            with pytest.raises(ValueError):
                eng.op(p, dev, index=bad)
        eng.submit([eng.op(p, dev, index=torch.tensor([5, 0, 5], dtype=torch.int32, device="cuda"))])
        eng.sync()
        assert eng.member_count(p) == 3
