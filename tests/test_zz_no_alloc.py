"""composite_oneshot_static: the entry point for callers that cannot call
cudaMalloc (a render callback that must not stall on an allocation's implicit
device synchronisation, or a host application that owns all device memory).
Its scratch is a fixed device array shared by every call, so calls in a row
must each match the CPU oracle and the context path (composite_begin / add /
render) bit for bit: a later call must not see an earlier call's counts.
The file runs last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402


def _padded_device_masks(m: np.ndarray):
    n, h, w = m.shape
    pitch = (w + 15) // 16 * 16
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(m).cuda()
    return buf[:, :, :w]


def _outputs(h, w):
    return (torch.full((h, w), -1, dtype=torch.int32, device="cuda"),
            torch.full((h, w), 7, dtype=torch.uint8, device="cuda"),
            torch.full((h, w, 4), 7, dtype=torch.uint8, device="cuda"))


def _custom_lut():
    b = np.arange(256)
    return np.stack([b, (b * 7) % 256, 255 - b, np.full(256, 200)], axis=1).astype(np.uint8)


# (width, height, members, seed, lut): the 16-wide output path (width % 16 ==
# 0) and the multi-slab accumulation (N > 255) included; N = 0 renders class 0
CASES = [(300, 200, 40, 31, None), (512, 256, 300, 33, "custom"), (1000, 500, 7, 32, None),
         (64, 48, 0, 34, "custom")]


@pytest.mark.gpu
def test_oneshot_static_matches_oracle_and_context_path_in_a_row():
    stream = torch.cuda.Stream()
    for w, h, n, seed, lut_kind in CASES:
        lut = _custom_lut() if lut_kind else None
        if n:
            m = synth.scramble_nonzero(synth.masks(synth.ensemble(seed, w, h, n)), seed)
        else:
            m = np.zeros((0, h, w), np.uint8)
        dev = _padded_device_masks(m) if n else torch.zeros((0, h, w), dtype=torch.uint8, device="cuda")
        counts, bucket, rgba = _outputs(h, w)
        binding.composite_oneshot_static(dev, counts, bucket, rgba, lut=lut, stream=stream.cuda_stream)
        stream.synchronize()
        c = oracle.count(m) if n else np.zeros((h, w), np.int64)
        b = oracle.bucket(c, n)
        np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32).astype(np.int64), c)
        np.testing.assert_array_equal(bucket.cpu().numpy(), b)
        np.testing.assert_array_equal(rgba.cpu().numpy(), oracle.rgba(b, lut))
        if n:
            with binding.Composite(w, h, count_bits=32) as comp:
                comp.add(dev)
                ref = comp.render_host(lut=lut)
            np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32), ref["counts"])
            np.testing.assert_array_equal(rgba.cpu().numpy(), ref["rgba"])


@pytest.mark.gpu
def test_oneshot_static_rejects_oversize_host_memory_and_bad_outputs():
    big = torch.zeros((1, 2049, 2048), dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_oneshot_static(big, bucket_out=torch.empty((2049, 2048), dtype=torch.uint8, device="cuda"))
    assert e.value.code == binding.CPT_EINVAL and "static scratch" in str(e.value)
    host = np.zeros((1, 16, 16), np.uint8)
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_oneshot_static(host, bucket_out=torch.empty((16, 16), dtype=torch.uint8, device="cuda"))
    assert e.value.code == binding.CPT_EINVAL
    dev = torch.zeros((2, 16, 16), dtype=torch.uint8, device="cuda")
    for bad in (dict(bucket_out=np.zeros((16, 16), np.uint8)),                                # host array
                dict(counts_out=torch.empty((16, 8), dtype=torch.int32, device="cuda")),       # undersized
                dict(counts_out=torch.empty((16, 16), dtype=torch.int16, device="cuda")),      # wrong type
                dict(rgba_out=torch.empty((16, 16), dtype=torch.uint8, device="cuda"))):       # not (h, w, 4)
        with pytest.raises(ValueError):
            binding.composite_oneshot_static(dev, **bad)
    # through the C ABI itself, past the binding's checks: an output in host
    # memory is refused before anything is queued (pinned, so that even a
    # missed check could not fault the GPU)
    lib = binding.load()
    pinned = torch.zeros((16, 16), dtype=torch.uint8).pin_memory()
    rc = lib.composite_oneshot_static(dev.data_ptr(), 2, 256, 16, 16, 16, None, pinned.data_ptr(), None, None, None)
    assert rc == binding.CPT_EINVAL and "current device" in binding.composite_last_error(None)
    assert int(pinned.sum()) == 0
    rc = lib.composite_oneshot_static(ctypes.c_void_p(pinned.data_ptr()), 1, 256, 16, 16, 16, None,
                                      torch.empty((16, 16), dtype=torch.uint8, device="cuda").data_ptr(),
                                      None, None, None)
    assert rc == binding.CPT_EINVAL
