"""Parity of the float32 mean-depth composite at the read-path workload's full
size: 256 water-depth rasters of 4096 x 4096 float32 (17.2 GB, device
resident) from the terrain generator (seed 3), through the linear, texture
and TMA read paths in the launch configurations the read-path sweep times.

Every pixel is checked against the closed form of the mean depth over one
ensemble (a sum of the highest water levels minus k * t, FP64; no raster is
summed), and sampled rows against the FP64 CPU oracle, with the tolerance
max |error| <= 1e-5 * N.  A TMA case with many more 2 KiB tiles than SMs
runs every persistent CTA through several tiles of the ring."""
import numpy as np
import pytest

import oracle
import synth
from tests.identities import count_identity, mean_depth_identity

torch = pytest.importorskip("torch")
from paper_2104_14667_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu

W = H = 4096
N = 256
ROWS = [0, 1, 1777, 2048, 4095]
TOL = 1e-5 * N


@pytest.fixture(scope="module")
def depths():
    ens = synth.ensemble(3, W, H, N)
    dev = torch.empty((N, H, W), dtype=torch.float32, device="cuda")
    synth.fill_depths_torch(ens, dev)
    ident = mean_depth_identity(ens.terrain, ens.levels)
    sample = oracle.mean_depth(dev[:, ROWS, :].cpu().numpy())
    yield ens, dev, ident, sample
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("path,box", [("linear", 0), ("texture", 0), ("tma", 256), ("tma", 64)])
def test_mean_depth_full_size(depths, path, box):
    ens, dev, ident, sample = depths
    with binding.Composite(W, H, read_path=path, mode="mean_depth", tma_box_bytes=box) as comp:
        comp.add(dev)
        got = comp.render_host()["mean"].astype(np.float64)
    assert np.abs(got[ROWS] - sample).max() <= TOL
    assert np.abs(got - ident).max() <= TOL
    # dry exactly where no member floods
    np.testing.assert_array_equal(got == 0.0, count_identity(ens.terrain, ens.levels) == 0)


def test_mean_depth_full_size_remove_half(depths):
    ens, dev, _, _ = depths
    with binding.Composite(W, H, read_path="linear", mode="mean_depth") as comp:
        comp.add(dev)
        comp.remove(dev[: N // 2])
        got = comp.render_host()["mean"].astype(np.float64)
    ref = mean_depth_identity(ens.terrain, ens.levels[N // 2:])
    # float32 sums of 256 depths then 128 taken away: the rounding of the
    # larger sum stays in the result, still far inside 1e-5 * N
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("box", [64, 256])
def test_tma_depth_many_tiles_per_cta(box):
    # 2048 x 1024 floats: 4096 tiles of 2 KiB rows with 256-byte boxes and
    # 4096 with 64-byte boxes (x 16-member groups), against 152 persistent CTAs
    w, h, n = 2048, 1024, 40
    ens = synth.ensemble(31, w, h, n)
    d = synth.depths(ens)
    pinned = torch.from_numpy(d).pin_memory()
    with binding.Composite(w, h, read_path="tma", mode="mean_depth", tma_box_bytes=box) as comp:
        comp.add(pinned.cuda())
        comp.add(pinned)
        comp.remove(pinned[: n // 2].cuda())
        got = comp.render_host()["mean"].astype(np.float64)
    ref = oracle.Composite(w, h, mode="mean_depth")
    ref.add(d)
    ref.add(d)
    ref.remove(d[: n // 2])
    assert np.abs(got - ref.render()["mean"]).max() <= 1e-5 * (2 * n)
