"""The render's one-multiply overlap class for N < 2^16 (every 16-bit
plane): class = umulhi(min(c, N) << (32 - k), M) with M = ceil(255 2^k / N),
k = 32 for N >= 256 and k = 16 below.  The kernels rely on this identity
with floor(255 c / N) for every count 0 <= c <= N; here it is checked
exhaustively for every N < 2048 and for a spread of larger N up to 65535
(the exactness condition c r < 2^k, r = M N - 255 2^k, for every N), in plain
integer arithmetic.  The GPU parity tests check the kernels themselves."""
import numpy as np


def magic(n: int):
    k = 32 if n >= 256 else 16
    return ((255 << k) + n - 1) // n, 32 - k, k


def narrow_class(c: np.ndarray, n: int) -> np.ndarray:
    m, shift, _ = magic(n)
    x = np.minimum(c.astype(np.uint64), np.uint64(n)) << np.uint64(shift)
    return ((x * np.uint64(m)) >> np.uint64(32)).astype(np.int64)


def test_multiplier_fits_and_error_term_is_below_one_for_every_n():
    for n in range(1, 1 << 16):
        m, shift, k = magic(n)
        assert m < 1 << 32
        r = m * n - (255 << k)
        assert 0 <= r < n
        assert n * r < 1 << k          # c r < 2^k for every c <= N
        assert (n << shift) < 1 << 32  # the shifted count fits 32 bits


def test_exhaustive_small_and_sampled_large_n():
    ns = list(range(1, 2048)) + list(range(2048, 1 << 16, 251)) + [4095, 4096, 4097, 32767, 32768, 65534, 65535]
    for n in ns:
        c = np.arange(0, n + 1, dtype=np.int64)
        np.testing.assert_array_equal(narrow_class(c, n), (255 * c) // n, err_msg=f"N={n}")


def test_counts_above_n_are_held_at_class_255():
    for n in (1, 2, 255, 256, 1000, 65535):
        c = np.array([n, n + 1, 2 * n, (1 << 16) - 1], dtype=np.int64)
        assert (narrow_class(c, n) == 255).all()
