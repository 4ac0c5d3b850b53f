"""Parity of the CUDA composite (through the C ABI) with the CPU oracle.

Counts, overlap classes and colours must match bit for bit; the float32 mean
depth must lie within 1e-5 * N of the FP64 oracle (max abs error).  Every read
path (linear, texture, TMA) and every input memory kind (device, pinned host,
pageable host) is covered, with ragged shapes, several staging-buffer counts
and chunk depths, incremental add/remove, underflow, N = 0 and custom tables.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu

PATHS = ["linear", "texture", "tma"]
KINDS = ["device", "pinned", "pageable"]


def as_kind(a: np.ndarray, kind: str):
    if kind == "pageable":
        return a
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if kind == "pinned" else t.cuda()


def expected(masks_np, lut=None, n=None):
    c = oracle.count(masks_np)
    n = masks_np.shape[0] if n is None else n
    b = oracle.bucket(c, n)
    return c, b, oracle.rgba(b, lut)


def check_counts(comp, masks_np, lut=None, n=None):
    got = comp.render_host(lut=lut)
    c, b, rgba = expected(masks_np, lut, n)
    np.testing.assert_array_equal(got["counts"].astype(np.int64), c)
    np.testing.assert_array_equal(got["bucket"], b)
    np.testing.assert_array_equal(got["rgba"], rgba)


SHAPES = [(1024, 1024, 16), (13, 7, 5), (1, 1, 3), (4097, 3, 9), (100, 37, 40), (48, 33, 300)]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("w,h,n", SHAPES)
def test_count_parity(path, kind, w, h, n):
    m = synth.masks(synth.ensemble(100 + w + h + n, w, h, n)) if w * h > 64 else synth.random_masks(7, n, h, w)
    with binding.Composite(w, h, read_path=path, staging_buffers=2, chunk_members=16) as comp:
        comp.add(as_kind(m, kind))
        assert comp.n == n
        check_counts(comp, m)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("k,c", [(1, 1), (1, 16), (2, 7), (3, 5), (4, 255), (8, 64)])
def test_staging_and_chunk_depths(path, k, c):
    w, h, n = 77, 45, 131
    m = synth.scramble_nonzero(synth.masks(synth.ensemble(9, w, h, n)), 9)
    with binding.Composite(w, h, read_path=path, staging_buffers=k, chunk_members=c) as comp:
        comp.add(as_kind(m, "pinned"))
        check_counts(comp, m)


@pytest.mark.parametrize("path", PATHS)
def test_device_rasters_read_in_place_with_padded_rows(path):
    # rows padded to 64 bytes, members padded by one extra row: aligned, so
    # the linear and TMA paths read the caller's memory directly
    w, h, n = 50, 29, 21
    m = synth.random_masks(21, n, h, w, density=0.4)
    big = torch.zeros((n, h + 1, 64), dtype=torch.uint8, device="cuda")
    big[:, :h, :w] = torch.from_numpy(m).cuda()
    view = big[:, :h, :w]
    with binding.Composite(w, h, read_path=path) as comp:
        comp.add(view)
        check_counts(comp, m)


@pytest.mark.parametrize("kind", KINDS)
def test_strided_host_rasters(kind):
    w, h, n = 31, 17, 12
    m = synth.random_masks(22, n, h, w)
    big = np.full((n, h + 2, 40), 255, np.uint8)   # padding bytes are nonzero on purpose
    big[:, :h, :w] = m
    if kind == "pageable":
        src = big[:, :h, :w]
    else:
        t = torch.from_numpy(big)
        t = t.pin_memory() if kind == "pinned" else t.cuda()
        src = t[:, :h, :w]
    with binding.Composite(w, h, read_path="linear") as comp:
        comp.add(src)
        check_counts(comp, m)


@pytest.mark.parametrize("path", PATHS)
def test_nonzero_bytes_and_32bit_counts(path):
    w, h, n = 96, 40, 70
    m = synth.scramble_nonzero(synth.random_masks(23, n, h, w), 23)
    with binding.Composite(w, h, read_path=path, count_bits=32) as comp:
        comp.add(as_kind(m, "device"))
        got = comp.render_host()
        assert got["counts"].dtype == np.uint32
        check_counts(comp, m)


@pytest.mark.parametrize("path", PATHS)
def test_add_remove_sequence_equals_recompute(path):
    w, h = 70, 33
    a = synth.random_masks(24, 20, h, w)
    b = synth.random_masks(25, 11, h, w)
    with binding.Composite(w, h, read_path=path, chunk_members=8) as comp:
        comp.add(as_kind(a, "device"))
        comp.add(as_kind(b, "pinned"))
        comp.remove(as_kind(a[:10], "pageable"))
        comp.remove(as_kind(a[10:], "device"))
        assert comp.n == 11
        check_counts(comp, b)


def test_empty_composite_renders_white():
    with binding.Composite(20, 10) as comp:
        got = comp.render_host()
        assert not got["counts"].any() and not got["bucket"].any()
        assert (got["rgba"] == 255).all()
        comp.add(as_kind(synth.random_masks(1, 3, 10, 20), "device"))
        comp.remove(as_kind(synth.random_masks(1, 3, 10, 20), "pinned"))
        assert comp.n == 0
        got = comp.render_host()
        assert not got["counts"].any() and (got["rgba"] == 255).all()


@pytest.mark.parametrize("path", PATHS)
def test_underflow_poisons_until_clear(path):
    w, h = 40, 20
    a = synth.random_masks(26, 2, h, w, density=0.5)
    with binding.Composite(w, h, read_path=path) as comp:
        comp.add(as_kind(a[:1], "device"))
        comp.remove(as_kind(a[1:], "device"))
        with pytest.raises(binding.CompositeError) as e:
            comp.render_host()
        assert e.value.code == binding.CPT_EUNDERFLOW
        with pytest.raises(binding.CompositeError) as e:
            comp.add(as_kind(a, "device"))
        assert e.value.code == binding.CPT_ESTATE
        comp.clear()
        comp.add(as_kind(a, "device"))
        check_counts(comp, a)


def test_member_limits_rejected_on_host():
    with binding.Composite(16, 1) as comp:
        with pytest.raises(binding.CompositeError) as e:
            comp.remove(np.zeros((1, 1, 16), np.uint8))
        assert e.value.code == binding.CPT_EINVAL
        ones = torch.ones((65535, 1, 16), dtype=torch.uint8, device="cuda")
        comp.add(ones)
        with pytest.raises(binding.CompositeError) as e:
            comp.add(ones[:1])
        assert e.value.code == binding.CPT_EINVAL
        assert comp.n == 65535
        got = comp.render_host()
        assert (got["counts"] == 65535).all() and (got["bucket"] == 255).all()


def test_custom_lut():
    w, h, n = 33, 9, 6
    m = synth.random_masks(27, n, h, w)
    lut = np.random.default_rng(5).integers(0, 256, (256, 4), dtype=np.uint8)
    with binding.Composite(w, h) as comp:
        comp.add(as_kind(m, "device"))
        check_counts(comp, m, lut=lut)


def test_render_to_device_outputs_matches_host():
    w, h, n = 64, 48, 25
    m = synth.random_masks(28, n, h, w)
    with binding.Composite(w, h) as comp:
        comp.add(as_kind(m, "pinned"))
        counts = torch.empty((h, w), dtype=torch.int16, device="cuda")
        bucket = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        rgba = torch.empty((h, w, 4), dtype=torch.uint8, device="cuda")
        comp.render(counts, bucket, rgba)
        comp.sync()
        c, b, col = expected(m)
        np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint16).astype(np.int64), c)
        np.testing.assert_array_equal(bucket.cpu().numpy(), b)
        np.testing.assert_array_equal(rgba.cpu().numpy(), col)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("w,h,n", [(256, 256, 256), (13, 7, 5), (37, 129, 19)])
def test_mean_depth_parity(path, kind, w, h, n):
    d = synth.depths(synth.ensemble(200 + w + n, w, h, n)) if w * h > 100 else synth.random_depths(3, n, h, w)
    with binding.Composite(w, h, read_path=path, mode="mean_depth", chunk_members=16) as comp:
        comp.add(as_kind(d, kind))
        got = comp.render_host()["mean"]
    ref = oracle.mean_depth(d)
    assert np.abs(got.astype(np.float64) - ref).max() <= 1e-5 * n


def test_mean_depth_single_member_exact_and_remove():
    w, h = 45, 21
    d = synth.random_depths(4, 6, h, w)
    with binding.Composite(w, h, mode="mean_depth") as comp:
        comp.add(as_kind(d[:1], "device"))
        np.testing.assert_array_equal(comp.render_host()["mean"], d[0])
        comp.add(as_kind(d[1:], "pinned"))
        comp.remove(as_kind(d[:3], "pageable"))
        got = comp.render_host()["mean"]
    ref = oracle.mean_depth(d[3:])
    assert np.abs(got.astype(np.float64) - ref).max() <= 1e-5 * 6


def test_trace_records_upload_and_kernel_intervals():
    w, h, n = 256, 128, 64
    m = synth.random_masks(29, n, h, w)
    with binding.Composite(w, h, chunk_members=8, staging_buffers=2, trace=True) as comp:
        comp.add(as_kind(m, "pinned"))
        rec = comp.trace()
        check_counts(comp, m)
    kinds = rec[:, 0].astype(int)
    assert (kinds == 0).sum() == 8 and (kinds == 2).sum() == 8
    assert np.all(rec[:, 2] >= rec[:, 1]) and rec[:, 1].min() >= 0.0


def test_nested_threshold_identity_at_streaming_size():
    # 4096 x 4096, 64 members streamed from pinned host memory through two
    # staging buffers of 32 members: every pixel against the independent
    # binary-search count, sampled rows against the oracle
    w = h = 4096
    n = 64
    ens = synth.ensemble(2, w, h, n)
    host = torch.empty((n, h, w), dtype=torch.uint8).pin_memory()
    synth.fill_masks(ens, host.numpy())
    with binding.Composite(w, h, chunk_members=32, staging_buffers=2) as comp:
        comp.add(host)
        got = comp.render_host()
    sorted_w = np.sort(ens.levels)
    ident = n - np.searchsorted(sorted_w, ens.terrain.ravel(), side="right").reshape(h, w)
    np.testing.assert_array_equal(got["counts"].astype(np.int64), ident)
    rows = [0, 1, 2047, 4095]
    sample = host.numpy()[:, rows, :]
    c = oracle.count(sample)
    b = oracle.bucket(c, n)
    np.testing.assert_array_equal(got["counts"][rows].astype(np.int64), c)
    np.testing.assert_array_equal(got["bucket"][rows], b)
    np.testing.assert_array_equal(got["rgba"][rows], oracle.rgba(b))


@pytest.mark.parametrize("w,h,n", [(1024, 1024, 16), (48, 33, 300), (13, 7, 5), (4097, 3, 9)])
def test_host_read_in_place(w, h, n):
    # pinned rasters read by the kernel over the host link; unaligned
    # layouts fall back to the staging pipeline
    m = synth.scramble_nonzero(synth.random_masks(30 + w, n, h, w), 30)
    with binding.Composite(w, h, host_read=True) as comp:
        comp.add(as_kind(m, "pinned"))
        comp.remove(as_kind(m[: n // 2], "pinned"))
        check_counts(comp, m[n // 2:])


@pytest.mark.parametrize("box", [64, 128, 256])
@pytest.mark.parametrize("mode", ["count", "mean_depth"])
@pytest.mark.parametrize("w,h,n", [(1000, 37, 19), (13, 200, 9), (257, 129, 270)])
def test_tma_box_widths(box, mode, w, h, n):
    if mode == "count":
        m = synth.scramble_nonzero(synth.random_masks(40 + box, n, h, w), 40)
    else:
        m = synth.random_depths(41 + box, n, h, w)
    with binding.Composite(w, h, read_path="tma", tma_box_bytes=box, mode=mode) as comp:
        comp.add(as_kind(m, "pinned"))
        if mode == "count":
            check_counts(comp, m)
        else:
            got = comp.render_host()["mean"]
            assert np.abs(got.astype(np.float64) - oracle.mean_depth(m)).max() <= 1e-5 * n


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("w,h,n", [(1024, 1024, 16), (13, 7, 5), (33, 9, 40), (100, 37, 300), (4097, 3, 9), (1, 1, 3)])
def test_bit_packed_masks(kind, w, h, n):
    m = synth.scramble_nonzero(synth.random_masks(90 + w, n, h, w, density=0.4), 90)
    packed = synth.pack_masks(m)
    assert packed.shape == (n, h, (w + 7) // 8)
    with binding.Composite(w, h, mask_format="bits", chunk_members=16) as comp:
        comp.add(as_kind(packed, kind))
        check_counts(comp, m)


@pytest.mark.parametrize("kind", ["device", "pinned"])
@pytest.mark.parametrize("w,h,n", [(256, 96, 300), (64, 4, 20), (128, 64, 7), (2048, 2, 33), (4096, 32, 1000)])
def test_bit_packed_bulk_copy_layouts(kind, w, h, n):
    # width a multiple of 32 and unpadded rows: the rasters reach the kernel
    # by bulk copies into shared memory (partial last tiles and stages, one
    # member slab folded in place, several folded by atomics)
    m = synth.scramble_nonzero(synth.random_masks(140 + w + n, n, h, w, density=0.3), 140)
    packed = synth.pack_masks(m)
    with binding.Composite(w, h, mask_format="bits", chunk_members=255) as comp:
        comp.add(as_kind(packed, kind))
        check_counts(comp, m)


@pytest.mark.parametrize("count_bits", [16, 32])
def test_bit_packed_bulk_copy_remove_and_underflow(count_bits):
    w, h = 320, 40
    a = synth.random_masks(150, 250, h, w)
    b = synth.random_masks(151, 9, h, w)
    with binding.Composite(w, h, mask_format="bits", chunk_members=255, count_bits=count_bits) as comp:
        comp.add(as_kind(synth.pack_masks(a), "device"))
        comp.add(as_kind(synth.pack_masks(b), "device"))
        comp.remove(as_kind(synth.pack_masks(a), "device"))
        check_counts(comp, b)
        comp.clear()
        comp.add(as_kind(synth.pack_masks(synth.random_masks(152, 3, h, w, density=0.05)), "device"))
        comp.remove(as_kind(synth.pack_masks(a[:1]), "device"))
        with pytest.raises(binding.CompositeError) as e:
            comp.render_host()
        assert e.value.code == binding.CPT_EUNDERFLOW


@pytest.mark.parametrize("k,c", [(1, 3), (2, 255), (3, 16)])
def test_bit_packed_add_remove_and_32bit(k, c):
    w, h = 77, 45
    a = synth.random_masks(95, 120, h, w)
    b = synth.random_masks(96, 30, h, w)
    with binding.Composite(w, h, mask_format="bits", staging_buffers=k, chunk_members=c, count_bits=32) as comp:
        comp.add(as_kind(synth.pack_masks(a), "pinned"))
        comp.add(as_kind(synth.pack_masks(b), "device"))
        comp.remove(as_kind(synth.pack_masks(a), "pageable"))
        check_counts(comp, b)
        # a sparse composite: removing a dense member that was never added underflows
        comp.clear()
        comp.add(as_kind(synth.pack_masks(synth.random_masks(97, 3, h, w, density=0.05)), "device"))
        comp.remove(as_kind(synth.pack_masks(a[:1]), "device"))
        with pytest.raises(binding.CompositeError) as e:
            comp.render_host()
        assert e.value.code == binding.CPT_EUNDERFLOW


@pytest.mark.parametrize("w,h,n", [(1024, 1024, 16), (13, 7, 5), (100, 37, 300), (48, 33, 2)])
@pytest.mark.parametrize("on_device", [False, True])
def test_histogram_of_overlap_classes(w, h, n, on_device):
    m = synth.masks(synth.ensemble(300 + w, w, h, n)) if w * h > 64 else synth.random_masks(8, n, h, w)
    with binding.Composite(w, h) as comp:
        comp.add(as_kind(m, "device"))
        if on_device:
            hist = torch.empty(256, dtype=torch.int64, device="cuda")
            bucket = torch.empty((h, w), dtype=torch.uint8, device="cuda")
            comp.render_histogram(hist, bucket_out=bucket)
            comp.sync()
            got_hist, got_bucket = hist.cpu().numpy().view(np.uint64), bucket.cpu().numpy()
        else:
            got_hist = np.empty(256, np.uint64)
            got_bucket = np.empty((h, w), np.uint8)
            comp.render_histogram(got_hist, bucket_out=got_bucket)
    b = oracle.bucket(oracle.count(m), n)
    np.testing.assert_array_equal(got_bucket, b)
    np.testing.assert_array_equal(got_hist, oracle.histogram(b))


@pytest.mark.parametrize("converter", ["copy", "kernel"])
@pytest.mark.parametrize("mode", ["count", "mean_depth"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("w,h,n", [(256, 64, 40), (13, 7, 5), (100, 37, 19)])
def test_texture_layout_converters(converter, mode, kind, w, h, n):
    if mode == "count":
        m = synth.scramble_nonzero(synth.random_masks(110 + w, n, h, w), 110)
    else:
        m = synth.random_depths(111 + w, n, h, w)
    with binding.Composite(w, h, read_path="texture", layout_converter=converter, mode=mode, chunk_members=8) as comp:
        comp.add(as_kind(m, kind))
        if mode == "count":
            check_counts(comp, m)
        else:
            got = comp.render_host()["mean"]
            assert np.abs(got.astype(np.float64) - oracle.mean_depth(m)).max() <= 1e-5 * n


def _nested_masks(n, targets):
    """uint8[n, 1, W] on the device: member m floods pixel x when m <
    targets[x], so the composite's counts are exactly `targets`."""
    t = torch.as_tensor(np.asarray(targets, np.int64), device="cuda")
    return (torch.arange(n, device="cuda")[:, None] < t[None, :]).to(torch.uint8)[:, None, :].contiguous()


def _class_targets(n):
    if n <= 4097:
        return np.arange(n + 1)
    return np.unique(np.round(np.linspace(0, n, 4097)).astype(np.int64))


CLASS_NS = list(range(1, 130)) + [255, 256, 257, 1000, 4095, 4096, 4097, 65535]


@pytest.mark.parametrize("count_bits", [16, 32])
def test_overlap_class_for_every_count(count_bits):
    # the render's floor(255 c / N) (a multiply-high by an invariant divisor)
    # against the oracle for every count of every listed N; widths both
    # multiples of 16 (16-pixel kernel) and not (per-pixel kernel)
    for n in CLASS_NS:
        targets = _class_targets(n)
        masks = _nested_masks(n, targets)
        with binding.Composite(len(targets), 1, count_bits=count_bits) as comp:
            comp.add(masks)
            got = comp.render_host()
            hist = np.empty(256, np.uint64)
            comp.render_histogram(hist)   # host output: synchronous
        c = np.asarray(targets, np.int64)[None, :]
        b = oracle.bucket(c, n)
        np.testing.assert_array_equal(hist, oracle.histogram(b), err_msg=f"N={n}")
        np.testing.assert_array_equal(got["counts"].astype(np.int64), c, err_msg=f"N={n}")
        np.testing.assert_array_equal(got["bucket"], b, err_msg=f"N={n}")
        np.testing.assert_array_equal(got["rgba"], oracle.rgba(b), err_msg=f"N={n}")


@pytest.mark.parametrize("count_bits", [16, 32])
def test_engine_overlap_class_for_every_count(count_bits):
    ns = [1, 2, 3, 7, 16, 17, 100, 255, 256, 1000, 4097] + ([65535] if count_bits == 16 else [65535, 70001])
    with binding.Engine() as eng:
        for n in ns:
            targets = _class_targets(n)
            w = len(targets)
            buf = torch.zeros((n, 1, (w + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
            buf[:, :, :w] = _nested_masks(n, targets)
            p = eng.add_plane(w, 1, count_bits)
            counts = torch.empty((1, w), dtype=torch.int32 if count_bits == 32 else torch.int16, device="cuda")
            bucket = torch.empty((1, w), dtype=torch.uint8, device="cuda")
            hist = torch.empty(256, dtype=torch.int64, device="cuda")
            eng.submit([eng.op(p, buf[:, :, :w])])
            eng.render([eng.render_op(p, counts, bucket, None)])
            eng.render([eng.render_op(p, histogram_out=hist)])   # the histogram launch's class path too
            eng.sync()
            got = counts.cpu().numpy()
            if got.dtype == np.int16:
                got = got.view(np.uint16)
            c = np.asarray(targets, np.int64)[None, :]
            np.testing.assert_array_equal(got.astype(np.int64), c, err_msg=f"N={n}")
            np.testing.assert_array_equal(bucket.cpu().numpy(), oracle.bucket(c, n), err_msg=f"N={n}")
            np.testing.assert_array_equal(hist.cpu().numpy(), oracle.histogram(oracle.bucket(c, n)).astype(np.int64),
                                          err_msg=f"N={n}")
            eng.free_plane(p)


def test_overlap_class_past_two_to_the_24_members():
    # N >= 2^24 members: the 64-bit division path of the class
    n = (1 << 24) + 3
    targets = np.array([0, 1, 2, n // 3, n // 2, n - 2, n - 1, n] + [0] * 8, np.int64)
    masks = _nested_masks(n, targets)           # n x 1 x 16 bytes, read in place
    with binding.Composite(16, 1, count_bits=32) as comp:
        comp.add(masks)
        got = comp.render_host()
    c = targets[None, :]
    np.testing.assert_array_equal(got["counts"].astype(np.int64), c)
    np.testing.assert_array_equal(got["bucket"], oracle.bucket(c, n))


@pytest.mark.parametrize("threads", [1, 3, 0])
@pytest.mark.parametrize("w,h,n", [(1024, 1024, 40), (100, 37, 300), (13, 7, 5)])
def test_pageable_ingest_threads(threads, w, h, n):
    # pageable rasters through the pinned ring, copied by 1, 3 or the default
    # number of host threads; a strided view forces row-by-row pieces
    m = synth.scramble_nonzero(synth.random_masks(160 + w + threads, n, h, w), 160)
    big = np.zeros((n, h, w + 9), np.uint8)
    big[:, :, :w] = m
    with binding.Composite(w, h, ingest_threads=threads, chunk_members=16, pageable_ingest="ring") as comp:
        comp.add(m)
        comp.remove(big[: n // 3, :, :w])
        comp.add(big[: n // 3, :, :w])
        check_counts(comp, m)


@pytest.mark.parametrize("mode", ["register", "auto"])
@pytest.mark.parametrize("path", PATHS)
def test_pageable_batches_registered_for_the_call(mode, path):
    # register: every pageable batch is page-locked in place for the call;
    # auto: batches of 64 MiB and more (here 80 rasters of 1 MiB) are, and
    # smaller ones take the ring.  The caller may overwrite a batch as soon
    # as the call returns, so the call must not return before its uploads.
    w, h, n = 1024, 1024, 80
    m = synth.scramble_nonzero(synth.random_masks(170, n, h, w, density=0.3), 170)
    strided = np.zeros((n, h, w + 32), np.uint8)
    strided[:, :, :w] = m
    with binding.Composite(w, h, read_path=path, pageable_ingest=mode) as comp:
        batch = m.copy()
        comp.add(batch)
        batch[:] = 0                      # reused right after the call
        comp.remove(strided[:10, :, :w])  # a strided view, registered or ringed
        comp.add(m[:10])                  # small: the ring in auto mode
        check_counts(comp, m)


def test_registration_refused_falls_back_to_the_ring(monkeypatch):
    # host_register: the driver's page-locking refused, as for a batch that
    # overlaps memory registered elsewhere
    w, h, n = 512, 256, 20
    m = synth.random_masks(171, n, h, w)
    monkeypatch.setenv("CPT_FAULT_INJECT", "host_register")
    with binding.Composite(w, h, pageable_ingest="register") as comp:
        comp.add(m)
        check_counts(comp, m)


@pytest.mark.parametrize("count_bits", [16, 32])
@pytest.mark.parametrize("source", ["pageable", "pinned", "device"])
def test_checkpoint_and_resume(count_bits, source):
    # save: the rendered counts and N; resume: load them into a fresh context,
    # then keep adding and removing -- the same as one context all along
    w, h = 100, 37
    a = synth.scramble_nonzero(synth.random_masks(180, 60, h, w), 180)
    b = synth.random_masks(181, 25, h, w)
    dtype = np.uint16 if count_bits == 16 else np.uint32
    with binding.Composite(w, h, count_bits=count_bits) as first:
        first.add(a)
        saved = first.render_host()["counts"].astype(dtype)
        n = first.n
    if source == "pageable":
        counts = saved
    else:
        t = torch.from_numpy(saved.view(np.int16 if count_bits == 16 else np.int32))
        counts = t.pin_memory() if source == "pinned" else t.cuda()
    with binding.Composite(w, h, count_bits=count_bits) as resumed:
        resumed.load_counts(counts, n)
        assert resumed.n == n
        check_counts(resumed, a)
        resumed.add(b)
        resumed.remove(a[:20])
        check_counts(resumed, np.concatenate([a[20:], b]))


def test_resume_rejects_counts_above_n():
    w, h = 16, 4
    bad = np.full((h, w), 3, np.uint16)
    with binding.Composite(w, h) as comp:
        with pytest.raises(binding.CompositeError) as e:
            comp.load_counts(bad, 2)
        assert e.value.code == binding.CPT_EINVAL
        with pytest.raises(binding.CompositeError) as e:
            comp.load_counts(bad, 70000)
        assert e.value.code == binding.CPT_EINVAL
        comp.load_counts(bad, 3)
        assert (comp.render_host()["bucket"] == 255).all()


@pytest.mark.parametrize("w,h,n,path,kind", [(1024, 1024, 100, "linear", "pinned"), (64, 48, 300, "linear", "pinned"),
                                             (1024, 1024, 40, "texture", "pinned"),
                                             (1024, 1024, 40, "texture", "device"),
                                             (2048, 512, 70, "tma", "pinned"), (512, 256, 600, "linear", "pageable")])
def test_automatic_chunk_depth(w, h, n, path, kind):
    # chunk_members 0: a staging buffer holds up to 256 MiB of rasters (512
    # MiB on the texture path), and a call of n rasters goes in chunks of
    # max(16 MiB, min(cap, ceil(n/32)))
    m = synth.scramble_nonzero(synth.random_masks(60 + n, n, h, w, density=0.3), 60)
    row = (w + 15) // 16 * 16
    member = row * h
    cap = max(1, min(255, ((512 if path == "texture" else 256) << 20) // member))
    c = max(min(cap, -(-(16 << 20) // member)), min(cap, -(-n // 32)))
    with binding.Composite(w, h, read_path=path, chunk_members=0, trace=True, pageable_ingest="ring") as comp:
        comp.add(as_kind(m, kind))
        rec = comp.trace()
        check_counts(comp, m)
    # one upload per chunk (the texture path's direct conversion from device
    # memory uploads nothing: one conversion per chunk instead)
    kinds = rec[:, 0].astype(int)
    per_chunk = (kinds == 1).sum() if kind == "device" else (kinds == 0).sum()
    assert int(per_chunk) == -(-n // c)


@pytest.mark.parametrize("what", ["mean_depth", "bits"])
def test_registered_ingest_depths_and_bit_packed(what):
    # page-locked in place for the call: float32 depths and bit-packed masks
    w, h, n = 1024, 512, 40
    if what == "mean_depth":
        d = synth.random_depths(172, n, h, w)            # 84 MB: above the 64 MiB threshold
        with binding.Composite(w, h, mode="mean_depth", pageable_ingest="register") as comp:
            comp.add(d)
            comp.remove(d[:5])
            got = comp.render_host()["mean"]
        assert np.abs(got.astype(np.float64) - oracle.mean_depth(d[5:])).max() <= 1e-5 * n
    else:
        m = synth.random_masks(173, n, h, w)
        packed = synth.pack_masks(m)
        with binding.Composite(w, h, mask_format="bits", pageable_ingest="register") as comp:
            comp.add(packed)
            check_counts(comp, m)
