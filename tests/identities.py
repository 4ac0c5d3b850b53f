"""Closed forms that hold for every ensemble from the terrain generator, used
to check composites of any size without summing a single raster.

Every member m of one ensemble thresholds the same terrain t at its water
level w_m: mask_m(p) = [t(p) < w_m] and depth_m(p) = max(w_m - t(p), 0).
With the levels sorted and k(p) = #{m : w_m > t(p)} found by a binary search:

  count(p)     = k(p)
  sum_m d_m(p) = (sum of the k(p) highest levels) - k(p) * t(p)

so the mean depth is that sum over N, in FP64 (levels and terrain are float32
values, so w - t is exact in FP64; the generator's float32 depth differs from
it by at most 2^-24 of itself per member)."""
import numpy as np


def count_identity(terrain: np.ndarray, levels) -> np.ndarray:
    lv = np.sort(np.asarray(levels, np.float32))
    t = np.asarray(terrain, np.float32)
    return len(lv) - np.searchsorted(lv, t.ravel(), side="right").reshape(t.shape)


def mean_depth_identity(terrain: np.ndarray, levels) -> np.ndarray:
    lv = np.sort(np.asarray(levels, np.float32)).astype(np.float64)
    n = len(lv)
    suffix = np.zeros(n + 1)
    suffix[:n] = np.cumsum(lv[::-1])[::-1]          # suffix[i] = sum of lv[i:]
    t = np.asarray(terrain, np.float32).astype(np.float64)
    i = np.searchsorted(lv, t.ravel(), side="right").reshape(t.shape)
    k = n - i
    return (suffix[i] - k * t) / n if n else np.zeros_like(t)


def depth_rounding_bound(terrain: np.ndarray, levels) -> float:
    """Largest gap between the identity and an exact mean of the float32
    depths: half an ulp of the deepest depth per member, averaged."""
    return float(np.max(levels) - np.min(terrain)) * 2.0 ** -24
