"""composite_oneshot_static: the entry point for callers that cannot call
cudaMalloc (a render callback that must not stall on an allocation's implicit
device synchronisation, or a host application that owns all device memory).
Its scratch is a fixed device array shared by every call; two calls in a row
must each match the context path (composite_begin / add / render) bit for bit,
so the second call must not see the first call's counts."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402


def _padded_device_masks(m: np.ndarray):
    n, h, w = m.shape
    pitch = (w + 15) // 16 * 16
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(m).cuda()
    return buf[:, :, :w]


@pytest.mark.gpu
def test_oneshot_static_matches_context_path_twice():
    cases = [(300, 200, 40, 31), (1000, 500, 7, 32)]   # second call: smaller N, larger raster
    stream = torch.cuda.Stream()
    for w, h, n, seed in cases:
        m = synth.scramble_nonzero(synth.masks(synth.ensemble(seed, w, h, n)), seed)
        dev = _padded_device_masks(m)
        counts = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
        bucket = torch.full((h, w), 7, dtype=torch.uint8, device="cuda")
        rgba = torch.full((h, w, 4), 7, dtype=torch.uint8, device="cuda")
        binding.composite_oneshot_static(dev, counts, bucket, rgba, stream=stream.cuda_stream)
        stream.synchronize()
        with binding.Composite(w, h, count_bits=32) as comp:
            comp.add(dev)
            ref = comp.render_host()
        np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32), ref["counts"])
        np.testing.assert_array_equal(bucket.cpu().numpy(), ref["bucket"])
        np.testing.assert_array_equal(rgba.cpu().numpy(), ref["rgba"])


@pytest.mark.gpu
def test_oneshot_static_rejects_oversize_and_host_memory():
    big = torch.zeros((1, 2049, 2048), dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_oneshot_static(big, bucket_out=torch.empty((2049, 2048), dtype=torch.uint8, device="cuda"))
    assert e.value.code == binding.CPT_EINVAL and "static scratch" in str(e.value)
    host = np.zeros((1, 16, 16), np.uint8)
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_oneshot_static(host, bucket_out=torch.empty((16, 16), dtype=torch.uint8, device="cuda"))
    assert e.value.code == binding.CPT_EINVAL
