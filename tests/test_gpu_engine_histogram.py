"""Class histograms of the batched engine's render (Fig. 1 caption: the
frequency of the overlap classes) against the CPU oracle: bin k = pixels of a
plane whose class floor(255 c / N) is k, counted in the render launch itself,
for ragged and padded planes, 16- and 32-bit counts, shared histograms,
captured graphs (zeroed on every replay) and a full-size terrain ensemble."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402
from tests.identities import count_identity  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(1024, 1024, 16), (13, 7, 5), (100, 37, 40), (257, 131, 300), (4096, 3, 9), (1, 1, 2), (48, 600, 1),
          (33, 17, 255)]


def padded(m: np.ndarray):
    n, h, w = m.shape
    pitch = (w + 15) // 16 * 16
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(m).cuda()
    return buf[:, :, :w]


def new_hist():
    # filled with a pattern: the render must zero it first
    return torch.full((256,), 0x5A5A5A5A, dtype=torch.int64, device="cuda")


def expected_hist(masks_np):
    return oracle.histogram(oracle.bucket(oracle.count(masks_np), masks_np.shape[0])).astype(np.int64)


def ensemble(seed, n, h, w, density):
    return synth.scramble_nonzero(synth.random_masks(seed, n, h, w, density=density), seed)


@pytest.mark.parametrize("count_bits", [32, 16])
@pytest.mark.parametrize("with_images", [True, False])
def test_histograms_of_many_planes_in_one_launch(count_bits, with_images):
    with binding.Engine() as eng:
        data, ops, rops, hists, buckets = [], [], [], [], []
        for i, (w, h, n) in enumerate(SHAPES):
            m = ensemble(80 + i, n, h, w, 0.2 + 0.07 * i)
            p = eng.add_plane(w, h, count_bits)
            dev = padded(m)
            hist = new_hist()
            bucket = torch.empty((h, w), dtype=torch.uint8, device="cuda") if with_images else None
            data.append((m, dev))
            hists.append(hist)
            buckets.append(bucket)
            ops.append(eng.op(p, dev))
            rops.append(eng.render_op(p, None, bucket, None, hist))
        eng.submit(ops)
        eng.render(rops)
        eng.sync()
        for (m, _), hist, bucket in zip(data, hists, buckets):
            want = expected_hist(m)
            np.testing.assert_array_equal(hist.cpu().numpy(), want)
            assert int(want.sum()) == m.shape[1] * m.shape[2]
            if bucket is not None:
                np.testing.assert_array_equal(bucket.cpu().numpy(), oracle.bucket(oracle.count(m), m.shape[0]))


def test_some_ops_with_histograms_and_one_shared():
    shapes = [(300, 70, 50), (64, 64, 8), (129, 33, 200)]
    with binding.Engine() as eng:
        ms, ops = [], []
        planes = []
        for i, (w, h, n) in enumerate(shapes):
            m = ensemble(90 + i, n, h, w, 0.35)
            p = eng.add_plane(w, h)
            dev = padded(m)
            ms.append((m, dev))
            planes.append(p)
            ops.append(eng.op(p, dev))
        eng.submit(ops)
        shared = new_hist()
        own = new_hist()
        rgba = torch.empty((shapes[1][1], shapes[1][0], 4), dtype=torch.uint8, device="cuda")
        eng.render([eng.render_op(planes[0], histogram_out=shared),
                    eng.render_op(planes[1], None, None, rgba),            # no histogram
                    eng.render_op(planes[2], histogram_out=shared),
                    eng.render_op(planes[1], histogram_out=own)])
        eng.sync()
        np.testing.assert_array_equal(shared.cpu().numpy(), expected_hist(ms[0][0]) + expected_hist(ms[2][0]))
        np.testing.assert_array_equal(own.cpu().numpy(), expected_hist(ms[1][0]))
        b1 = oracle.bucket(oracle.count(ms[1][0]), shapes[1][2])
        np.testing.assert_array_equal(rgba.cpu().numpy(), oracle.rgba(b1))


def test_histogram_is_zeroed_on_every_render_and_replay():
    w, h, total = 200, 90, 120
    ens = ensemble(95, total, h, w, 0.4)
    dev = padded(ens)
    with binding.Engine() as eng:
        p = eng.add_plane(w, h, 16)
        q = eng.add_plane(w, h, 32)
        hist_p, hist_q = new_hist(), new_hist()
        eng.submit([eng.op(p, dev[:70])])
        for _ in range(3):   # the direct render, repeated
            eng.render([eng.render_op(p, histogram_out=hist_p)])
        eng.sync()
        np.testing.assert_array_equal(hist_p.cpu().numpy(), expected_hist(ens[:70]))
        eng.capture([eng.op(p, dev[:40]), eng.op(q, dev[40:])],
                    [eng.render_op(p, histogram_out=hist_p), eng.render_op(q, histogram_out=hist_q)],
                    keep=(dev,))
        for _ in range(3):
            eng.replay()
        eng.sync()
        np.testing.assert_array_equal(hist_p.cpu().numpy(), expected_hist(ens[:40]))
        np.testing.assert_array_equal(hist_q.cpu().numpy(), expected_hist(ens[40:]))


def test_histogram_output_checks():
    with binding.Engine() as eng:
        p = eng.add_plane(64, 8)
        eng.submit([eng.op(p, padded(ensemble(97, 4, 8, 64, 0.5)))])
        eng.sync()
        raw = torch.zeros(256 + 2, dtype=torch.int64, device="cuda")
        with pytest.raises(binding.CompositeError) as ei:
            eng.render([eng.render_op(p, histogram_out=raw[1:257])])   # 8 bytes off a 16-byte boundary
        assert ei.value.code == binding.CPT_EINVAL
        host = np.zeros(256, dtype=np.int64)   # pageable host memory
        with pytest.raises(binding.CompositeError) as ei:
            eng.render([eng.render_op(p, histogram_out=host)])
        assert ei.value.code == binding.CPT_EINVAL
        eng.sync()
        assert not raw.any()


def test_full_size_terrain_histogram():
    """4096 x 4096 with 64 members of one terrain ensemble: large flat regions
    of one class (long runs, byte counters folded many times) and every class
    boundary of the terrain; counts from the closed form k(p) = #{w_m > t(p)}."""
    w = h = 4096
    n = 64
    ens = synth.ensemble(11, w, h, n)
    masks = torch.empty((n, h, w), dtype=torch.uint8, device="cuda")
    synth.fill_masks_torch(ens, masks)
    want = oracle.histogram(oracle.bucket(count_identity(ens.terrain, ens.levels), n)).astype(np.int64)
    with binding.Engine() as eng:
        p16 = eng.add_plane(w, h, 16)
        p32 = eng.add_plane(w, h, 32)
        h16, h32 = new_hist(), new_hist()
        bucket = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        eng.submit([eng.op(p16, masks), eng.op(p32, masks)])
        eng.render([eng.render_op(p16, None, bucket, None, h16), eng.render_op(p32, histogram_out=h32)])
        eng.sync()
    np.testing.assert_array_equal(h16.cpu().numpy(), want)
    np.testing.assert_array_equal(h32.cpu().numpy(), want)
    got = np.bincount(bucket.cpu().numpy().ravel(), minlength=256)
    np.testing.assert_array_equal(got, want)
    assert (want > 0).sum() > 32   # the ensemble spans many classes


def test_short_outputs_are_refused_before_any_launch():
    # the binding checks that every output holds what the render writes: the
    # C ABI takes plain pointers, and a kernel would overrun a short one
    w, h = 64, 8
    masks = padded(ensemble(98, 3, h, w, 0.5))
    short = {"counts_out": torch.empty((h, w - 1), dtype=torch.int32, device="cuda"),
             "bucket_out": torch.empty((h - 1, w), dtype=torch.uint8, device="cuda"),
             "rgba_out": torch.empty((h, w, 3), dtype=torch.uint8, device="cuda"),
             "histogram_out": torch.empty(255, dtype=torch.int64, device="cuda")}
    with binding.Engine() as eng:
        p = eng.add_plane(w, h)
        eng.submit([eng.op(p, masks)])
        for name, t in short.items():
            with pytest.raises(ValueError, match=name):
                eng.render_op(p, **{name: t})
        eng.sync()
    with binding.Composite(w, h, count_bits=32) as comp:
        comp.add(masks)
        for name, t in short.items():
            with pytest.raises(ValueError, match=name):
                if name == "histogram_out":
                    comp.render_histogram(t)
                else:
                    comp.render(**{name: t})
        with pytest.raises(ValueError, match="counts_out"):
            comp.render(counts_out=np.empty((h, w), np.uint16))   # 16-bit host counts for 32-bit ones
        comp.sync()


@pytest.mark.parametrize("count_bits", [32, 16])
def test_empty_plane_is_all_class_zero(count_bits):
    # N = 0: every pixel is class 0 (the divisor's empty case), in the same
    # launch as a plane with members
    w, h = 40, 9
    m = ensemble(99, 3, h, w, 0.5)
    with binding.Engine() as eng:
        empty, full = eng.add_plane(w, h, count_bits), eng.add_plane(w, h, count_bits)
        eng.submit([eng.op(full, padded(m))])
        he, hf = new_hist(), new_hist()
        bucket = torch.full((h, w), 7, dtype=torch.uint8, device="cuda")
        eng.render([eng.render_op(empty, None, bucket, None, he), eng.render_op(full, histogram_out=hf)])
        eng.sync()
    want = np.zeros(256, np.int64)
    want[0] = w * h
    np.testing.assert_array_equal(he.cpu().numpy(), want)
    assert not bucket.any()
    np.testing.assert_array_equal(hf.cpu().numpy(), expected_hist(m))
