"""CPU oracle of the iterative ensemble composite -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``composite_oracle.c`` (plain C, built with
gcc on first use) and this module only marshals numpy arrays.

Definitions (Johnson & Jankun-Kelly; Fig. 1 caption, Figs. 2-3, Section 4):

* ``count(p) = sum_m [mask_m(p) != 0]``  -- the per-member accumulation
* ``bucket(p) = floor(255 * count(p) / N)`` (0 when N = 0)  -- overlap class
* ``rgba(p) = LUT[bucket(p)]``  -- blue saturation colour map
* ``hist[b] = #{p : bucket(p) = b}``  -- frequency of overlap classes
* ``mean(p) = sum_m d_m(p) / N`` in FP64  -- mean-depth composite

Parity pins (tests/test_oracle_pins.py): nested-threshold identity against
the terrain's water levels, sum and range invariants, order independence,
single-member and closed-form cases, add-then-remove, the exhaustive
bucket characterisation and exact rational means.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "composite_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compiles the C oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_count_apply.restype = ctypes.c_int64
            lib.oracle_count_apply.argtypes = [_i64p, _u8p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int32]
            lib.oracle_bucket.restype = ctypes.c_int32
            lib.oracle_bucket.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64, _u8p]
            lib.oracle_rgba.restype = None
            lib.oracle_rgba.argtypes = [_u8p, _u8p, ctypes.c_int64, _u8p]
            lib.oracle_histogram.restype = None
            lib.oracle_histogram.argtypes = [_u8p, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_default_lut.restype = None
            lib.oracle_default_lut.argtypes = [_u8p]
            lib.oracle_depth_apply.restype = None
            lib.oracle_depth_apply.argtypes = [_f64p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int32]
            lib.oracle_mean.restype = None
            lib.oracle_mean.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, _f64p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as_members(members: np.ndarray, dtype) -> np.ndarray:
    a = np.asarray(members)
    if a.ndim == 2:
        a = a[None]
    if a.ndim != 3 or a.dtype != dtype:
        raise ValueError(f"members must be {np.dtype(dtype).name}[n, H, W]")
    return a


def _strides(a: np.ndarray) -> tuple[int, int]:
    """(row pitch, member stride) in elements; the innermost axis is dense."""
    item = a.itemsize
    if a.strides[2] != item or a.strides[1] % item or a.strides[0] % item:
        raise ValueError("rows must be contiguous")
    return a.strides[1] // item, a.strides[0] // item


def count_apply(counts: np.ndarray, members: np.ndarray, sign: int = 1) -> int:
    """counts (int64[H, W], in place) += sign * flood masks; returns #negative pixels."""
    a = _as_members(members, np.uint8)
    n, h, w = a.shape
    if counts.dtype != np.int64 or counts.shape != (h, w) or not counts.flags.c_contiguous:
        raise ValueError("counts must be C-contiguous int64[H, W]")
    if sign not in (1, -1):
        raise ValueError("sign must be +1 or -1")
    pitch, stride = _strides(a)
    return int(_load().oracle_count_apply(_ptr(counts, ctypes.c_int64), _ptr(a, ctypes.c_uint8), n,
                                          w, h, pitch, stride, sign))


def count(members: np.ndarray) -> np.ndarray:
    """int64[H, W] number of members whose mask byte is nonzero."""
    a = _as_members(members, np.uint8)
    out = np.zeros(a.shape[1:], dtype=np.int64)
    count_apply(out, a, 1)
    return out


def bucket(counts: np.ndarray, n_members: int) -> np.ndarray:
    """uint8 overlap class floor(255 * count / N); 0 everywhere when N == 0."""
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.empty(c.shape, dtype=np.uint8)
    if _load().oracle_bucket(_ptr(c, ctypes.c_int64), int(n_members), c.size,
                             _ptr(out, ctypes.c_uint8)) != 0:
        raise ValueError("a count lies outside [0, N]")
    return out


def histogram(buckets: np.ndarray) -> np.ndarray:
    """uint64[256] number of pixels in every overlap class (Fig. 1 caption:
    the histogram of overlap-class frequencies)."""
    b = np.ascontiguousarray(buckets, dtype=np.uint8)
    out = np.empty(256, dtype=np.uint64)
    _load().oracle_histogram(_ptr(b, ctypes.c_uint8), b.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def default_lut() -> np.ndarray:
    """uint8[256, 4] white-to-blue ramp: b -> (255-b, 255-b, 255, 255)."""
    lut = np.empty((256, 4), dtype=np.uint8)
    _load().oracle_default_lut(_ptr(lut, ctypes.c_uint8))
    return lut


def rgba(buckets: np.ndarray, lut: np.ndarray | None = None) -> np.ndarray:
    """uint8[..., 4] colour of every bucket through the 256-entry table."""
    b = np.ascontiguousarray(buckets, dtype=np.uint8)
    t = default_lut() if lut is None else np.ascontiguousarray(lut, dtype=np.uint8).reshape(256, 4)
    out = np.empty(b.shape + (4,), dtype=np.uint8)
    _load().oracle_rgba(_ptr(b, ctypes.c_uint8), _ptr(t, ctypes.c_uint8), b.size,
                        _ptr(out, ctypes.c_uint8))
    return out


def depth_apply(sums: np.ndarray, depths: np.ndarray, sign: int = 1) -> None:
    """sums (float64[H, W], in place) += sign * depths, summed in FP64."""
    a = _as_members(depths, np.float32)
    n, h, w = a.shape
    if sums.dtype != np.float64 or sums.shape != (h, w) or not sums.flags.c_contiguous:
        raise ValueError("sums must be C-contiguous float64[H, W]")
    pitch, stride = _strides(a)
    _load().oracle_depth_apply(_ptr(sums, ctypes.c_double), _ptr(a, ctypes.c_float), n, w, h,
                               pitch, stride, int(sign))


def mean(sums: np.ndarray, n_members: int) -> np.ndarray:
    """float64 mean depth sums / N (0 when N == 0)."""
    s = np.ascontiguousarray(sums, dtype=np.float64)
    out = np.empty(s.shape, dtype=np.float64)
    _load().oracle_mean(_ptr(s, ctypes.c_double), int(n_members), s.size, _ptr(out, ctypes.c_double))
    return out


def mean_depth(depths: np.ndarray) -> np.ndarray:
    a = _as_members(depths, np.float32)
    s = np.zeros(a.shape[1:], dtype=np.float64)
    depth_apply(s, a, 1)
    return mean(s, a.shape[0])


class Composite:
    """Incremental composite over a multiset of members (the interactive list
    of Fig. 1): add and remove in any order, render at any time."""

    def __init__(self, width: int, height: int, mode: str = "count"):
        if width <= 0 or height <= 0:
            raise ValueError("raster sides must be positive")
        if mode not in ("count", "mean_depth"):
            raise ValueError("mode is 'count' or 'mean_depth'")
        self.width, self.height, self.mode = width, height, mode
        self.n = 0
        self.counts = np.zeros((height, width), dtype=np.int64)
        self.sums = np.zeros((height, width), dtype=np.float64)
        self.underflow = False

    def add(self, members: np.ndarray) -> None:
        self._apply(members, 1)

    def remove(self, members: np.ndarray) -> None:
        self._apply(members, -1)

    def _apply(self, members: np.ndarray, sign: int) -> None:
        if self.mode == "count":
            a = _as_members(members, np.uint8)
            if self.n + sign * a.shape[0] < 0:
                raise ValueError("cannot remove more members than were added")
            if count_apply(self.counts, a, sign):
                self.underflow = True
        else:
            a = _as_members(members, np.float32)
            if self.n + sign * a.shape[0] < 0:
                raise ValueError("cannot remove more members than were added")
            depth_apply(self.sums, a, sign)
        self.n += sign * a.shape[0]

    def render(self, lut: np.ndarray | None = None) -> dict:
        if self.mode == "mean_depth":
            return {"mean": mean(self.sums, self.n)}
        if self.underflow:
            raise ValueError("a remove took away a member that was never added")
        b = bucket(self.counts, self.n)
        return {"counts": self.counts.copy(), "bucket": b, "rgba": rgba(b, lut), "histogram": histogram(b)}
