"""Throughput, efficiency and overlap arithmetic for the streamed composite.

These are host-side formulas used to report measurements; they follow the
paper's own definitions so the numbers read the same way as its tables.

* Transfer rate (Section 6.1, Figs. 6 and 9): raster bytes moved ÷ wall time,
  in GB/s with GB = 1e9 B.  The paper's rasters are 1 byte per pixel, so the
  rate is also member-pixels per nanosecond.
* Efficiency (Section 6.1 and the captions of Figs. 6 and 9): the time of a
  plain host-to-device copy of the same bytes ÷ the algorithm's wall time,
  i.e. achieved rate ÷ copy rate, at most 1.
* Pipelined wall-time model (Section 7.1): with c_i, m_i, p_i the copy,
  layout-transform and processing times of member i, the streamed algorithm
  takes max(c_1 + sum(m) + sum(p), sum(c) + m_n + p_n).  The paper prints this
  divided by sum(c); the subscript "1-n" is read as the sum over 1..n.
* Overlap fraction (not in the paper): 1 - (wall - max(C, K)) / min(C, K) with
  C and K the busy time of the copy and compute engines, clamped to [0, 1]:
  1 when the shorter one hides completely under the longer, 0 when they run
  strictly one after the other.
"""
from __future__ import annotations

from typing import Iterable, Sequence


def member_pixels_per_s(n_members: int, width: int, height: int, seconds: float) -> float:
    return float(n_members) * width * height / seconds


def transfer_gbs(n_bytes: float, seconds: float) -> float:
    return float(n_bytes) / seconds / 1e9


def efficiency(rate_gbs: float, copy_rate_gbs: float) -> float:
    """Achieved rate as a fraction of the plain-copy rate (the tables' sense)."""
    return rate_gbs / copy_rate_gbs


def pipeline_wall(copy: Sequence[float], transform: Sequence[float],
                  process: Sequence[float]) -> float:
    """Wall time of the multi-buffer pipeline predicted by Section 7.1."""
    if not (len(copy) == len(transform) == len(process)) or not copy:
        raise ValueError("need one copy, transform and process time per member")
    head = copy[0] + sum(transform) + sum(process)
    tail = sum(copy) + transform[-1] + process[-1]
    return max(head, tail)


def pipeline_ratio(copy: Sequence[float], transform: Sequence[float],
                   process: Sequence[float]) -> float:
    """The paper's e: predicted wall time over pure copy time (>= 1)."""
    return pipeline_wall(copy, transform, process) / sum(copy)


def _union_length(intervals: Iterable[tuple[float, float]]) -> float:
    total, end = 0.0, None
    for a, b in sorted(intervals):
        if b <= a:
            continue
        if end is None or a > end:
            total += b - a
            end = b
        elif b > end:
            total += b - end
            end = b
    return total


def overlap_fraction(copy_intervals: Sequence[tuple[float, float]],
                     compute_intervals: Sequence[tuple[float, float]]) -> float | None:
    """Fraction of the shorter engine's busy time hidden under the longer one."""
    c = _union_length(copy_intervals)
    k = _union_length(compute_intervals)
    if min(c, k) <= 0.0:
        return None
    ends = [b for _, b in copy_intervals] + [b for _, b in compute_intervals]
    starts = [a for a, _ in copy_intervals] + [a for a, _ in compute_intervals]
    wall = max(ends) - min(starts)
    f = 1.0 - (wall - max(c, k)) / min(c, k)
    return min(1.0, max(0.0, f))


def percentile(values: Sequence[float], q: float) -> float:
    """Nearest-rank percentile, q in (0, 100]."""
    if not values:
        raise ValueError("no values")
    s = sorted(values)
    k = max(1, -(-len(s) * q // 100))
    return float(s[int(k) - 1])
