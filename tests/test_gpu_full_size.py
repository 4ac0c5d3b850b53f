"""Parity at the benchmark's full size: 1024 flood masks of 4096 x 4096 from
the terrain generator (seed 2), in the launch configurations bench.py times.

Every pixel is checked against the nested-threshold identity (all members
threshold one terrain, so count(p) = #{m : w_m > terrain(p)}, a binary search
over the sorted water levels that sums no mask), and sampled rows against the
CPU oracle (counts, overlap classes, colours)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu

W = H = 4096
N = 1024
ROWS = [0, 1, 1234, 2047, 4095]


@pytest.fixture(scope="module")
def ensemble():
    ens = synth.ensemble(2, W, H, N)
    dev = torch.empty((N, H, W), dtype=torch.uint8, device="cuda")
    synth.fill_masks_torch(ens, dev)
    ident = N - np.searchsorted(np.sort(ens.levels), ens.terrain.ravel(), side="right").reshape(H, W)
    sample = dev[:, ROWS, :].cpu().numpy()
    c = oracle.count(sample)
    b = oracle.bucket(c, N)
    yield ens, dev, ident, (c, b, oracle.rgba(b))
    del dev
    torch.cuda.empty_cache()


def check(got, ident, sample):
    c, b, rgba = sample
    np.testing.assert_array_equal(got["counts"].astype(np.int64), ident)
    np.testing.assert_array_equal(got["counts"][ROWS].astype(np.int64), c)
    np.testing.assert_array_equal(got["bucket"][ROWS], b)
    np.testing.assert_array_equal(got["rgba"][ROWS], rgba)
    np.testing.assert_array_equal(got["bucket"], oracle.bucket(ident, N))


@pytest.mark.parametrize("path", ["linear", "tma", "texture"])
def test_device_resident_one_launch(ensemble, path):
    # the bench's device-resident pass: clear, one accumulate over all 1024
    # members read in place, render (the texture path converts chunks of 16
    # members into its layered arrays first)
    _, dev, ident, sample = ensemble
    with binding.Composite(W, H, read_path=path) as comp:
        comp.add(dev)
        check(comp.render_host(), ident, sample)


def test_staged_from_pinned_host(ensemble):
    # the bench's end-to-end leg: pinned host rasters through two staging
    # buffers of 32 members
    _, dev, ident, sample = ensemble
    host = torch.empty((N, H, W), dtype=torch.uint8, pin_memory=True)
    host.copy_(dev)
    with binding.Composite(W, H, chunk_members=32, staging_buffers=2) as comp:
        comp.add(host)
        check(comp.render_host(), ident, sample)


def test_bit_packed_device_resident(ensemble):
    # the compressed form at the same size (the bulk-copy kernel)
    _, dev, ident, sample = ensemble
    packed = torch.empty((N, H, W // 8), dtype=torch.uint8, device="cuda")
    for m0 in range(0, N, 64):
        packed[m0:m0 + 64] = synth.pack_masks_torch(dev[m0:m0 + 64])
    with binding.Composite(W, H, mask_format="bits") as comp:
        comp.add(packed)
        half = packed[: N // 2]
        comp.remove(half)
        comp.add(half)
        check(comp.render_host(), ident, sample)
