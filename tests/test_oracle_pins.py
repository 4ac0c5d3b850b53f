"""Pins of the CPU oracle to facts that do not come from the oracle itself.

The paper prints no composite values, so the oracle is pinned by the
mathematics of the problem:

* the nested-threshold identity: every member of one ensemble thresholds the
  same terrain, so count(p) = #{m : w_m > terrain(p)}, computed here by a
  binary search over the sorted water levels (no mask is summed at all);
* invariants: 0 <= count <= N and sum_p count(p) = sum_m F_m, with F_m taken
  from the sorted terrain by the generator;
* order independence, the single-member case, closed forms (all dry, all
  flooded, N copies of one mask, complementary pairs), bytes other than 0/1;
* the incremental semantics of the interactive list (Fig. 1): add-then-remove
  equals a recompute;
* the overlap class floor(255 c / N), checked for every (c, N) with N <= 4096
  by the inequality that defines a floor, b*N <= 255c < (b+1)*N;
* the colour map at its ends (white, saturated blue) and its monotone
  saturation;
* the mean depth against exact rational arithmetic, and against its closed
  form over one ensemble (a sum of the highest water levels minus k * t).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests.identities import depth_rounding_bound, mean_depth_identity


def nested_threshold_counts(ens: synth.Ensemble) -> np.ndarray:
    w = np.sort(ens.levels)
    below_or_equal = np.searchsorted(w, ens.terrain.ravel(), side="right")
    return (ens.n - below_or_equal).reshape(ens.height, ens.width)


@pytest.mark.parametrize("seed,w,h,n", [(1, 64, 48, 7), (11, 257, 131, 37), (3, 96, 96, 1)])
def test_count_matches_nested_threshold_identity(seed, w, h, n):
    ens = synth.ensemble(seed, w, h, n)
    counts = oracle.count(synth.masks(ens))
    np.testing.assert_array_equal(counts, nested_threshold_counts(ens))


def test_count_nested_threshold_at_tiny_config_size():
    # the 1024x1024, N=16 workload, whole
    ens = synth.ensemble(1, 1024, 1024, 16)
    counts = oracle.count(synth.masks(ens))
    np.testing.assert_array_equal(counts, nested_threshold_counts(ens))


@pytest.mark.parametrize("seed", [2, 5])
def test_count_range_and_sum_invariants(seed):
    ens = synth.ensemble(seed, 200, 120, 23)
    counts = oracle.count(synth.masks(ens))
    assert counts.min() >= 0 and counts.max() <= ens.n
    assert int(counts.sum()) == int(ens.flooded.sum())


def test_count_order_independent():
    m = synth.random_masks(4, 9, 33, 47, density=0.3)
    base = oracle.count(m)
    rng = np.random.default_rng(0)
    for _ in range(5):
        np.testing.assert_array_equal(oracle.count(m[rng.permutation(9)]), base)


def test_single_member_is_its_own_mask():
    m = synth.scramble_nonzero(synth.random_masks(6, 1, 17, 29), 6)
    np.testing.assert_array_equal(oracle.count(m), (m[0] != 0).astype(np.int64))


def test_closed_forms():
    h, w, n = 13, 21, 6
    zero = np.zeros((n, h, w), np.uint8)
    np.testing.assert_array_equal(oracle.count(zero), np.zeros((h, w), np.int64))
    full = synth.scramble_nonzero(np.ones((n, h, w), np.uint8), 1)
    np.testing.assert_array_equal(oracle.count(full), np.full((h, w), n, np.int64))
    one = synth.random_masks(7, 1, h, w)
    copies = np.repeat(one, n, axis=0)
    np.testing.assert_array_equal(oracle.count(copies), n * one[0].astype(np.int64))
    pair = np.stack([one[0], 1 - one[0]])
    np.testing.assert_array_equal(oracle.count(pair), np.ones((h, w), np.int64))


def test_nonzero_bytes_count_once():
    m = synth.random_masks(8, 11, 19, 23)
    np.testing.assert_array_equal(oracle.count(synth.scramble_nonzero(m, 8)), oracle.count(m))


def test_strided_members_read_correctly():
    m = synth.random_masks(9, 5, 10, 14)
    big = np.full((5, 13, 32), 7, np.uint8)      # padding bytes are nonzero on purpose
    big[:, :10, :14] = m
    view = big[:, :10, :14]
    assert view.strides == (13 * 32, 32, 1)
    np.testing.assert_array_equal(oracle.count(view), oracle.count(m))


def test_exhaustive_two_by_two_up_to_three_members():
    # every ensemble of up to 3 masks over 2x2 pixels, against numpy's
    # boolean reduction
    for n in range(1, 4):
        for bits in itertools.product((0, 1), repeat=4 * n):
            m = np.array(bits, np.uint8).reshape(n, 2, 2)
            np.testing.assert_array_equal(oracle.count(m), np.add.reduce(m.astype(bool), axis=0))


def test_add_then_remove_equals_recompute():
    a = synth.random_masks(10, 6, 24, 40)
    b = synth.random_masks(11, 4, 24, 40)
    c = oracle.Composite(40, 24)
    c.add(a)
    c.add(b)
    c.remove(a[::2])
    c.remove(a[1::2])
    np.testing.assert_array_equal(c.counts, oracle.count(b))
    assert c.n == 4
    r = c.render()
    np.testing.assert_array_equal(r["bucket"], oracle.bucket(oracle.count(b), 4))


def test_remove_of_unadded_member_is_underflow():
    a = synth.random_masks(12, 2, 8, 8, density=0.6)
    c = oracle.Composite(8, 8)
    c.add(a[:1])
    c.remove(a[1:])
    assert c.underflow
    with pytest.raises(ValueError):
        c.render()


def test_remove_below_zero_members_rejected():
    c = oracle.Composite(4, 4)
    with pytest.raises(ValueError):
        c.remove(np.zeros((1, 4, 4), np.uint8))


def test_bucket_floor_characterisation_exhaustive():
    for n in range(1, 4097):
        c = np.arange(n + 1, dtype=np.int64)
        b = oracle.bucket(c, n).astype(np.int64)
        assert np.all(b * n <= 255 * c) and np.all(255 * c < (b + 1) * n), n
        assert b[-1] == 255 and np.all(b[:-1] < 255)
        assert np.all(np.diff(b) >= 0)


def test_bucket_large_counts_and_zero_members():
    n = 4_000_000_000
    c = np.array([0, 1, n // 2, n - 1, n], np.int64)
    b = oracle.bucket(c, n).astype(np.int64)
    assert np.all(b * n <= 255 * c) and np.all(255 * c < (b + 1) * n)
    np.testing.assert_array_equal(oracle.bucket(np.zeros(5, np.int64), 0), np.zeros(5, np.uint8))
    with pytest.raises(ValueError):
        oracle.bucket(np.array([3], np.int64), 2)


def test_default_lut_is_white_to_saturated_blue():
    lut = oracle.default_lut().astype(np.int64)
    assert tuple(lut[0]) == (255, 255, 255, 255)
    assert tuple(lut[255]) == (0, 0, 255, 255)
    sat = lut[:, 2] - np.minimum(lut[:, 0], lut[:, 1])     # blue minus the grey floor
    assert np.all(np.diff(sat) > 0)
    assert np.all(lut[:, 2] == 255) and np.all(lut[:, 3] == 255)


def test_rgba_is_a_table_lookup():
    rng = np.random.default_rng(3)
    lut = rng.integers(0, 256, (256, 4), dtype=np.uint8)
    b = rng.integers(0, 256, (7, 9), dtype=np.uint8)
    np.testing.assert_array_equal(oracle.rgba(b, lut), np.take(lut, b, axis=0))


def test_mean_depth_against_exact_rationals():
    d = synth.random_depths(13, 9, 5, 6)
    got = oracle.mean_depth(d)
    for y in range(5):
        for x in range(6):
            exact = sum(Fraction(float(v)) for v in d[:, y, x]) / 9
            assert abs(Fraction(got[y, x]) - exact) <= Fraction(1, 2 ** 50) * (1 + abs(exact))


@pytest.mark.parametrize("seed,w,h,n", [(6, 64, 48, 9), (12, 131, 77, 40)])
def test_mean_depth_matches_threshold_closed_form(seed, w, h, n):
    # an independent algorithm: the depths of one ensemble are w_m - t where
    # positive, so their sum is a sum of the highest levels minus k * t
    ens = synth.ensemble(seed, w, h, n)
    got = oracle.mean_depth(synth.depths(ens))
    ref = mean_depth_identity(ens.terrain, ens.levels)
    assert np.abs(got - ref).max() <= depth_rounding_bound(ens.terrain, ens.levels)
    assert np.abs(ref).max() > 0.01


def test_mean_depth_special_cases():
    d = synth.random_depths(14, 1, 7, 8)
    np.testing.assert_array_equal(oracle.mean_depth(d), d[0].astype(np.float64))
    copies = np.repeat(d, 5, axis=0)
    np.testing.assert_array_equal(oracle.mean_depth(copies), d[0].astype(np.float64))
    ens = synth.ensemble(15, 40, 30, 6)
    dep = synth.depths(ens)
    np.testing.assert_array_equal(dep > 0, synth.masks(ens).astype(bool))


def test_mean_depth_add_then_remove():
    a = synth.random_depths(16, 5, 6, 7)
    b = synth.random_depths(17, 3, 6, 7)
    c = oracle.Composite(7, 6, mode="mean_depth")
    c.add(a)
    c.add(b)
    c.remove(a)
    np.testing.assert_allclose(c.render()["mean"], oracle.mean_depth(b), rtol=0, atol=1e-12)
    empty = oracle.Composite(7, 6, mode="mean_depth")
    np.testing.assert_array_equal(empty.render()["mean"], np.zeros((6, 7)))


def test_histogram_counts_every_pixel_once():
    rng = np.random.default_rng(9)
    b = rng.integers(0, 256, (37, 53), dtype=np.uint8)
    h = oracle.histogram(b)
    assert int(h.sum()) == b.size
    np.testing.assert_array_equal(h, np.bincount(b.ravel(), minlength=256))


def test_histogram_closed_forms():
    h, w, n = 11, 17, 5
    zero = oracle.Composite(w, h)
    assert zero.render()["histogram"][0] == h * w and zero.render()["histogram"][1:].sum() == 0
    full = oracle.Composite(w, h)
    full.add(np.ones((n, h, w), np.uint8))
    hist = full.render()["histogram"]
    assert hist[255] == h * w and hist[:255].sum() == 0
    half = oracle.Composite(w, h)
    m = synth.random_masks(5, 1, h, w)
    half.add(np.concatenate([m, np.ones((1, h, w), np.uint8)]))     # counts 1 or 2 of N = 2
    hist = half.render()["histogram"]
    assert hist[255] == int(m.sum()) and hist[127] == h * w - int(m.sum())


def test_brute_force_on_random_8x8_inputs():
    # 10^4 random 8x8 ensembles of 1..12 members with arbitrary byte values
    # (about half of them zero): counts by walking every member and pixel,
    # classes by Python integers
    rng = np.random.default_rng(12)
    for case in range(10_000):
        n = int(rng.integers(1, 13))
        m = (rng.integers(0, 256, (n, 8, 8)) * rng.integers(0, 2, (n, 8, 8))).astype(np.uint8)
        got = oracle.count(m)
        if case < 300:
            want = np.zeros((8, 8), np.int64)
            for k in range(n):
                for y in range(8):
                    for x in range(8):
                        want[y, x] += 1 if m[k, y, x] else 0
            b = oracle.bucket(got, n)
            for y in range(8):
                for x in range(8):
                    assert b[y, x] == (255 * int(want[y, x])) // n
        else:
            want = np.count_nonzero(m, axis=0)
        np.testing.assert_array_equal(got, want)
