"""Host-side measurement formulas against the paper's printed tables, and the
synthetic generator's determinism."""
import os

import numpy as np
import pytest

import synth
from paper_2104_14667_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_streaming_tables.txt")


def _rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, w, h, alg, n, t_us, rate, eff = line.split()
            rows.append((s, int(w), int(h), alg, int(n), float(t_us), float(rate), float(eff)))
    return rows


def test_golden_has_every_printed_row():
    assert len(_rows()) == 32


def test_transfer_rate_reproduces_paper_tables():
    # 1 byte per pixel: raster bytes x N / wall time gives the printed GB/s
    for s, w, h, alg, n, t_us, rate, _ in _rows():
        got = metrics.transfer_gbs(w * h * n, t_us * 1e-6)
        assert abs(got - rate) <= 0.0015, (s, alg, n, got, rate)
        assert metrics.member_pixels_per_s(n, w, h, t_us * 1e-6) == pytest.approx(rate * 1e9, rel=4e-4)


def test_efficiency_is_rate_over_one_copy_rate_per_set():
    # efficiency = rate / plain-copy rate; the implied copy rate is one
    # number per raster size, whatever the algorithm or N
    by_set = {}
    for s, _, _, _, _, _, rate, eff in _rows():
        by_set.setdefault(s, []).append(rate / (eff / 100.0))
    for s, vals in by_set.items():
        assert max(vals) / min(vals) < 1.005, (s, vals)      # the ~2k N=10 row is 0.3 % off
    copy = {s: float(np.mean(v)) for s, v in by_set.items()}
    assert copy["~4k"] == pytest.approx(5.285, abs=0.005)
    for s, _, _, _, _, _, rate, eff in _rows():
        assert metrics.efficiency(rate, copy[s]) * 100 == pytest.approx(eff, abs=0.2)


def test_pipeline_model_closed_forms():
    n = 10
    # copy-bound: n copies plus the last transform and process
    assert metrics.pipeline_wall([3.0] * n, [0.5] * n, [1.0] * n) == pytest.approx(n * 3.0 + 1.5)
    # compute-bound: the first copy plus every transform and process
    assert metrics.pipeline_wall([1.0] * n, [2.0] * n, [1.5] * n) == pytest.approx(1.0 + n * 3.5)
    assert metrics.pipeline_ratio([2.0] * n, [0.0] * n, [0.0] * n) == pytest.approx(1.0)
    assert metrics.pipeline_ratio([1.0] * n, [0.0] * n, [0.1] * n) >= 1.0


def test_overlap_fraction():
    assert metrics.overlap_fraction([(0, 10)], [(2, 8)]) == pytest.approx(1.0)
    assert metrics.overlap_fraction([(0, 5)], [(5, 10)]) == pytest.approx(0.0)
    # both busy 8 of a 10-long wall: 6 of the 8 overlap
    assert metrics.overlap_fraction([(0, 4), (4, 8)], [(2, 6), (6, 10)]) == pytest.approx(0.75)
    assert metrics.overlap_fraction([], [(0, 1)]) is None


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert metrics.percentile(v, 50) == 50
    assert metrics.percentile(v, 99) == 99
    assert metrics.percentile([7.0], 99) == 7.0


def test_splitmix64_published_vectors():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014)
    got = [int(x) for x in synth.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_counter_based():
    a = synth.splitmix64(42, 100)
    np.testing.assert_array_equal(synth.splitmix64(42, 30, start=70), a[70:])
    u = synth.uniforms(42, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_ensemble_is_deterministic_and_shaped():
    e1 = synth.ensemble(5, 64, 40, 9)
    e2 = synth.ensemble(5, 64, 40, 9)
    np.testing.assert_array_equal(e1.terrain, e2.terrain)
    np.testing.assert_array_equal(e1.levels, e2.levels)
    m = synth.masks(e1)
    assert m.dtype == np.uint8 and m.shape == (9, 40, 64) and set(np.unique(m)) <= {0, 1}
    frac = m.reshape(9, -1).mean(axis=1)
    assert np.all(frac >= 0.09) and np.all(frac <= 0.51)
    np.testing.assert_array_equal(m.reshape(9, -1).sum(axis=1), e1.flooded)
    tail = synth.ensemble(5, 64, 40, 4, member_offset=5)
    np.testing.assert_array_equal(tail.levels, e1.levels[5:])


def test_terrain_row_band_matches_whole():
    whole = synth.terrain(7, 50, 30)
    band = synth.terrain(7, 50, 30, rows=slice(10, 20))
    np.testing.assert_array_equal(band, whole[10:20])


def test_torch_fills_match_numpy_generator():
    torch = __import__("pytest").importorskip("torch")
    ens = synth.ensemble(6, 70, 50, 5)
    m = torch.empty((5, 50, 70), dtype=torch.uint8)
    synth.fill_masks_torch(ens, m)
    np.testing.assert_array_equal(m.numpy(), synth.masks(ens))
    d = torch.empty((5, 50, 70), dtype=torch.float32)
    synth.fill_depths_torch(ens, d)
    np.testing.assert_array_equal(d.numpy(), synth.depths(ens))


def test_pack_masks_round_trip_and_bit_order():
    m = synth.scramble_nonzero(synth.random_masks(3, 4, 5, 19), 3)
    p = synth.pack_masks(m)
    assert p.shape == (4, 5, 3)
    np.testing.assert_array_equal(np.unpackbits(p, axis=-1, bitorder="little")[..., :19], (m != 0).astype(np.uint8))
    one = np.zeros((1, 1, 9), np.uint8)
    one[0, 0, 8] = 7          # pixel 8 -> bit 0 of byte 1
    np.testing.assert_array_equal(synth.pack_masks(one)[0, 0], [0, 1])


def test_pack_masks_torch_matches_numpy():
    torch = __import__("pytest").importorskip("torch")
    m = synth.scramble_nonzero(synth.random_masks(4, 3, 6, 24), 4)
    np.testing.assert_array_equal(synth.pack_masks_torch(torch.from_numpy(m)).numpy(), synth.pack_masks(m))


def test_bench_identity_check_accepts_exact_and_rejects_off_by_one():
    # the sweeps' sampled-row check: counts from the oracle pass, a count
    # one off in a sampled row fails, members cycling through a pool count
    # once per use
    import bench
    import oracle

    ens = synth.ensemble(21, 40, 12, 9)
    masks = synth.masks(ens)

    class Fake:
        def __init__(self, counts):
            self.counts = counts

        def render_host(self):
            return {"counts": self.counts.astype(np.uint16)}

    exact = oracle.count(masks)
    assert bench.identity_rows_exact(Fake(exact), ens.terrain, ens.levels)
    off = exact.copy()
    off[-1, 7] += 1
    assert not bench.identity_rows_exact(Fake(off), ens.terrain, ens.levels)
    cycled = oracle.count(np.concatenate([masks, masks[:4]]))
    assert bench.identity_rows_exact(Fake(cycled), ens.terrain, [ens.levels[m % 9] for m in range(13)])


def test_ncu_traffic_record_scales_member_bytes_only(tmp_path):
    # the summariser reads ncu's CSV log (one row per metric) and scales a
    # small capture to the full workload: member bytes grow with the members,
    # the plane's bytes do not
    from paper_2104_14667_gb300 import ncu_traffic
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",' \
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [("dram__bytes_read.sum", "byte", "1,000,000"), ("dram__bytes_write.sum", "Kbyte", "20"),
            ("gpu__time_duration.sum", "ns", "5000")]
    body = "".join(f'"0","1","p","h","void count_linear_kernel<unsigned short>(X)","1","13","(256, 1, 1)",'
                   f'"(64, 1, 1)","0","10.3","Command line profiler metrics","{m}","{u}","{v}"\n' for m, u, v in rows)
    other = '"1","1","p","h","render_counts_vec_kernel","1","13","(256, 1, 1)","(64, 1, 1)","0","10.3",' \
            '"Command line profiler metrics","dram__bytes_read.sum","byte","7"\n'
    path = tmp_path / "m.csv"
    path.write_text("==PROF== Connected\n" + head + body + other)
    rec = ncu_traffic.summarize(str(path), "count_linear", 100, 10, captured_members=4, members=64, command="c")
    assert rec["captured_dram_bytes"] == 1_000_000 + 20_000
    assert rec["captured_duration_us"] == 5.0
    assert rec["dram_bytes_per_launch"] == 1_020_000 - 4 * 1000 + 64 * 1000
    assert rec["workload"] == "100x10x64" and len(rec["kernel_source_sha256_16"]) == 16


class _OracleComposite:
    """Stands in for a GPU composite in the bench's check helpers: renders the
    oracle's counts and mean depth of the members given."""

    def __init__(self, masks=None, depths=None):
        self.masks, self.depths = masks, depths

    def render_host(self):
        import oracle
        if self.depths is not None:
            return {"mean": oracle.mean_depth(self.depths).astype(np.float32)}
        return {"counts": oracle.count(self.masks)}


def test_bench_identity_checks_accept_the_oracle_and_reject_a_mistake():
    import bench
    ens = synth.ensemble(41, 96, 40, 12)
    masks, depths = synth.masks(ens), synth.depths(ens)
    assert bench.identity_rows_exact(_OracleComposite(masks=masks), ens.terrain, ens.levels)
    assert not bench.identity_rows_exact(_OracleComposite(masks=masks[1:]), ens.terrain, ens.levels)
    err = bench.depth_identity_max_error(_OracleComposite(depths=depths), ens.terrain, ens.levels)
    assert err <= 1e-5
    bad = bench.depth_identity_max_error(_OracleComposite(depths=depths[1:]), ens.terrain, ens.levels)
    assert bad > 1e-3
