"""Thin ctypes binding of include/composite.h.

Argument marshalling only: every step of the composite runs in
libcomposite.so.  Functions keep the C names; arrays may be torch tensors
(CUDA, pinned or pageable CPU) or numpy arrays, passed by pointer with their
strides.  There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

CPT_OK = 0
CPT_EINVAL = -1
CPT_ENOMEM = -2
CPT_ECUDA = -3
CPT_ESTATE = -4
CPT_EUNDERFLOW = -5
CPT_ETIMEOUT = -6
STATUS_NAMES = {0: "CPT_OK", -1: "CPT_EINVAL", -2: "CPT_ENOMEM", -3: "CPT_ECUDA",
                -4: "CPT_ESTATE", -5: "CPT_EUNDERFLOW", -6: "CPT_ETIMEOUT"}

CPT_READ_LINEAR, CPT_READ_TEXTURE, CPT_READ_TMA = 0, 1, 2
READ_PATHS = {"linear": CPT_READ_LINEAR, "texture": CPT_READ_TEXTURE, "tma": CPT_READ_TMA}
CPT_MODE_COUNT, CPT_MODE_MEAN_DEPTH = 0, 1
CPT_MASK_BYTES, CPT_MASK_BITS = 0, 1
CPT_CONVERT_COPY, CPT_CONVERT_KERNEL = 0, 1

HEADER = os.path.join(_build.INCLUDE, "composite.h")
HEADERS = [os.path.join(_build.INCLUDE, h) for h in ("composite.h", "composite_engine.h", "composite_server.h")]


class CompositeError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {message}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("read_path", ctypes.c_int32),
        ("staging_buffers", ctypes.c_int32),
        ("chunk_members", ctypes.c_int32),
        ("count_bits", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("trace", ctypes.c_int32),
        ("pinned_ring_bytes", ctypes.c_int64),
        ("cuda_stream", ctypes.c_void_p),
        ("wait_timeout_ms", ctypes.c_int64),
        ("host_read", ctypes.c_int32),
        ("tma_box_bytes", ctypes.c_int32),
        ("mask_format", ctypes.c_int32),
        ("layout_converter", ctypes.c_int32),
        ("ingest_threads", ctypes.c_int32),
        ("pageable_ingest", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Loads libcomposite.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB_PATH):
            raise RuntimeError(f"{_build.LIB_PATH} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "composite_default_config": (ctypes.c_int, [ctypes.POINTER(Config)]),
            "composite_begin": (ctypes.c_int, [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(Config)]),
            "composite_clear": (ctypes.c_int, [vp]),
            "composite_add_members": (ctypes.c_int, [vp, vp, i32, i64, i32]),
            "composite_remove_members": (ctypes.c_int, [vp, vp, i32, i64, i32]),
            "composite_render": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, vp]),
            "composite_render_histogram": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, vp]),
            "composite_sync": (ctypes.c_int, [vp]),
            "composite_member_count": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
            "composite_load_counts": (ctypes.c_int, [vp, vp, i64]),
            "composite_trace_read": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), i32,
                                                    ctypes.POINTER(i32)]),
            "composite_end": (ctypes.c_int, [vp]),
            "composite_last_error": (ctypes.c_char_p, [vp]),
            "composite_oneshot_static": (ctypes.c_int, [vp, i32, i64, i32, i32, i32, vp, vp, vp, vp, vp]),
            "composite_selftest_bounded_wait": (ctypes.c_int, [i64, ctypes.POINTER(i32), ctypes.POINTER(i64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def declared_functions() -> list[str]:
    """Every function the public headers declare."""
    text = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(composite_\w+)\s*\(", text, re.M)))


# --- marshalling helpers ----------------------------------------------------

def _raster_view(a):
    """(pointer, n, height, width, member_stride_bytes, row_pitch_bytes, dtype, keepalive)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        t = a if a.dim() == 3 else a.unsqueeze(0)
        if t.dim() != 3 or t.stride(2) != 1:
            raise ValueError("rasters must be [n, H, W] (or [H, W]) with contiguous rows")
        item = t.element_size()
        dtype = {torch.uint8: np.uint8, torch.float32: np.float32}.get(t.dtype)
        if dtype is None:
            raise ValueError("rasters must be uint8 masks or float32 depths")
        return (t.data_ptr(), t.shape[0], t.shape[1], t.shape[2], t.stride(0) * item,
                t.stride(1) * item, dtype, t)
    arr = np.asarray(a)
    if arr.ndim == 2:
        arr = arr[None]
    if arr.ndim != 3 or arr.strides[2] != arr.itemsize:
        raise ValueError("rasters must be [n, H, W] (or [H, W]) with contiguous rows")
    if arr.dtype not in (np.uint8, np.float32):
        raise ValueError("rasters must be uint8 masks or float32 depths")
    return (arr.ctypes.data, arr.shape[0], arr.shape[1], arr.shape[2], arr.strides[0],
            arr.strides[1], arr.dtype.type, arr)


def _ptr(a):
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("outputs must be contiguous")
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    if not a.flags.c_contiguous:
        raise ValueError("outputs must be contiguous")
    return a.ctypes.data


def _nbytes(a) -> int:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.numel() * a.element_size()
    except ImportError:  # pragma: no cover
        pass
    return int(a.nbytes)


def _check_room(**outs):
    """Every output must hold what the library writes into it: the C ABI
    takes plain pointers and cannot check sizes, and a short device output
    would be overrun by a kernel."""
    for name, (a, need) in outs.items():
        if a is not None and _nbytes(a) < need:
            raise ValueError(f"{name} holds {_nbytes(a)} bytes; the render writes {need}")


def _on_device(*arrays) -> int:
    dev = None
    for a in arrays:
        if a is None:
            continue
        is_dev = bool(getattr(a, "is_cuda", False))
        if dev is None:
            dev = is_dev
        elif dev != is_dev:
            raise ValueError("outputs must all be device tensors or all host arrays")
    return 1 if dev else 0


def _check(lib, ctx, rc):
    if rc != CPT_OK:
        msg = lib.composite_last_error(ctx)
        raise CompositeError(rc, msg.decode() if msg else "")
    return rc


# --- the C functions, same names ---------------------------------------------

def composite_default_config() -> Config:
    cfg = Config()
    lib = load()
    _check(lib, None, lib.composite_default_config(ctypes.byref(cfg)))
    return cfg


def composite_begin(width: int, height: int, cfg: Config | None = None) -> ctypes.c_void_p:
    lib = load()
    ctx = ctypes.c_void_p()
    rc = lib.composite_begin(ctypes.byref(ctx), int(width), int(height),
                             ctypes.byref(cfg) if cfg is not None else None)
    _check(lib, None, rc)
    return ctx


def composite_clear(ctx) -> None:
    lib = load()
    _check(lib, ctx, lib.composite_clear(ctx))


def _apply(fn_name, ctx, members):
    lib = load()
    ptr, n, _, _, stride, pitch, _, _ = _raster_view(members)
    _check(lib, ctx, getattr(lib, fn_name)(ctx, ptr, n, stride, pitch))


def composite_add_members(ctx, members) -> None:
    _apply("composite_add_members", ctx, members)


def composite_remove_members(ctx, members) -> None:
    _apply("composite_remove_members", ctx, members)


def composite_render(ctx, counts_out=None, bucket_out=None, rgba_out=None, mean_out=None,
                     lut=None) -> None:
    lib = load()
    on_dev = _on_device(counts_out, bucket_out, rgba_out, mean_out)
    lut_arr = None
    if lut is not None:
        lut_arr = np.ascontiguousarray(np.asarray(lut, dtype=np.uint8).reshape(256, 4))
    rc = lib.composite_render(ctx, _ptr(counts_out), _ptr(bucket_out), _ptr(rgba_out), _ptr(mean_out),
                              on_dev, lut_arr.ctypes.data if lut_arr is not None else None)
    _check(lib, ctx, rc)


def composite_render_histogram(ctx, histogram_out, counts_out=None, bucket_out=None, rgba_out=None,
                               lut=None) -> None:
    lib = load()
    on_dev = _on_device(histogram_out, counts_out, bucket_out, rgba_out)
    lut_arr = None
    if lut is not None:
        lut_arr = np.ascontiguousarray(np.asarray(lut, dtype=np.uint8).reshape(256, 4))
    rc = lib.composite_render_histogram(ctx, _ptr(counts_out), _ptr(bucket_out), _ptr(rgba_out),
                                        _ptr(histogram_out), on_dev,
                                        lut_arr.ctypes.data if lut_arr is not None else None)
    _check(lib, ctx, rc)


def composite_sync(ctx) -> None:
    lib = load()
    _check(lib, ctx, lib.composite_sync(ctx))


def composite_member_count(ctx) -> int:
    lib = load()
    n = ctypes.c_int64()
    _check(lib, ctx, lib.composite_member_count(ctx, ctypes.byref(n)))
    return n.value


def composite_trace_read(ctx) -> np.ndarray:
    """float32[n, 3] records {kind, start_ms, end_ms}."""
    lib = load()
    n = ctypes.c_int32()
    _check(lib, ctx, lib.composite_trace_read(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 3), dtype=np.float32)
    _check(lib, ctx, lib.composite_trace_read(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              n.value, ctypes.byref(n)))
    return out[: n.value]


def composite_end(ctx) -> None:
    lib = load()
    _check(lib, None, lib.composite_end(ctx))


def composite_last_error(ctx=None) -> str:
    lib = load()
    msg = lib.composite_last_error(ctx)
    return msg.decode() if msg else ""


def _check_static_outputs(members, h, w, counts_out, bucket_out, rgba_out):
    """The allocation-free entry point writes its outputs straight from the
    GPU: they must be CUDA tensors of exactly the raster's shape and type, on
    the members' device (the C side checks memory kinds, not sizes)."""
    import torch
    want = {"counts_out": (counts_out, (h, w), (torch.int32,)),
            "bucket_out": (bucket_out, (h, w), (torch.uint8,)),
            "rgba_out": (rgba_out, (h, w, 4), (torch.uint8,))}
    if hasattr(torch, "uint32"):
        want["counts_out"] = (counts_out, (h, w), (torch.int32, torch.uint32))
    dev = members.device if isinstance(members, torch.Tensor) else None
    for name, (t, shape, dtypes) in want.items():
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if tuple(t.shape) != shape or t.dtype not in dtypes or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {shape} tensor of {dtypes[0]}")
        if dev is not None and t.device != dev:
            raise ValueError(f"{name} must be on the members' device {dev}")


def composite_oneshot_static(members, counts_out=None, bucket_out=None, rgba_out=None, lut=None,
                             stream=None) -> None:
    """One-shot composite of device-resident masks with no allocation in the
    library (scratch in a fixed device array); queued on ``stream``."""
    lib = load()
    ptr, n, h, w, stride, pitch, dtype, _ = _raster_view(members)
    if dtype is not np.uint8:
        raise ValueError("composite_oneshot_static takes uint8 masks")
    _check_static_outputs(members, h, w, counts_out, bucket_out, rgba_out)
    lut_arr = None
    if lut is not None:
        lut_arr = np.ascontiguousarray(np.asarray(lut, dtype=np.uint8).reshape(256, 4))
    rc = lib.composite_oneshot_static(ptr, n, stride, pitch, w, h, _ptr(counts_out), _ptr(bucket_out),
                                      _ptr(rgba_out), lut_arr.ctypes.data if lut_arr is not None else None,
                                      stream)
    _check(lib, None, rc)


def composite_selftest_bounded_wait(timeout_us: int) -> tuple[bool, int]:
    """(gave_up, waited_us) of a device wait on a barrier nothing arrives at."""
    lib = load()
    gave, waited = ctypes.c_int32(), ctypes.c_int64()
    _check(lib, None, lib.composite_selftest_bounded_wait(int(timeout_us), ctypes.byref(gave), ctypes.byref(waited)))
    return bool(gave.value), waited.value


def caller_stream():
    """The caller's current torch CUDA stream handle (0 = the legacy default
    stream), so the library's work is ordered after torch's work that
    produced its inputs; None without a usable CUDA torch."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
    except Exception:  # pragma: no cover
        pass
    return None


PAGEABLE_INGEST = {"auto": 0, "ring": 1, "register": 2}


def make_config(read_path="linear", staging_buffers=2, chunk_members=0, count_bits=16,
                mode="count", trace=False, pinned_ring_bytes=0, stream=None,
                wait_timeout_ms=0, host_read=False, tma_box_bytes=0, mask_format="bytes",
                layout_converter="kernel", ingest_threads=0, pageable_ingest="auto") -> Config:
    cfg = composite_default_config()
    cfg.read_path = READ_PATHS[read_path] if isinstance(read_path, str) else int(read_path)
    cfg.staging_buffers = staging_buffers
    cfg.chunk_members = chunk_members
    cfg.count_bits = count_bits
    cfg.mode = {"count": CPT_MODE_COUNT, "mean_depth": CPT_MODE_MEAN_DEPTH}[mode] if isinstance(mode, str) else int(mode)
    cfg.trace = 1 if trace else 0
    cfg.pinned_ring_bytes = pinned_ring_bytes
    cfg.cuda_stream = stream if stream is not None else caller_stream()
    cfg.wait_timeout_ms = wait_timeout_ms
    cfg.host_read = 1 if host_read else 0
    cfg.tma_box_bytes = tma_box_bytes
    cfg.mask_format = {"bytes": CPT_MASK_BYTES, "bits": CPT_MASK_BITS}[mask_format] \
        if isinstance(mask_format, str) else int(mask_format)
    cfg.layout_converter = {"copy": CPT_CONVERT_COPY, "kernel": CPT_CONVERT_KERNEL}[layout_converter] \
        if isinstance(layout_converter, str) else int(layout_converter)
    cfg.ingest_threads = ingest_threads
    cfg.pageable_ingest = PAGEABLE_INGEST[pageable_ingest] if isinstance(pageable_ingest, str) \
        else int(pageable_ingest)
    return cfg


class Composite:
    """A composite context as a Python object.  Keeps every borrowed raster
    alive until the next render to host, sync or close, as the C ABI asks."""

    def __init__(self, width: int, height: int, **config):
        self.width, self.height = int(width), int(height)
        self.config = make_config(**config)
        self.ctx = composite_begin(width, height, self.config)
        self._borrowed = []

    def clear(self):
        composite_clear(self.ctx)

    def add(self, members):
        composite_add_members(self.ctx, members)
        self._borrowed.append(members)

    def remove(self, members):
        composite_remove_members(self.ctx, members)
        self._borrowed.append(members)

    @property
    def n(self) -> int:
        return composite_member_count(self.ctx)

    def _check_outputs(self, counts_out, bucket_out, rgba_out, mean_out=None, histogram_out=None):
        px = self.width * self.height
        _check_room(counts_out=(counts_out, px * ((self.config.count_bits or 16) // 8)),
                    bucket_out=(bucket_out, px), rgba_out=(rgba_out, 4 * px), mean_out=(mean_out, 4 * px),
                    histogram_out=(histogram_out, 256 * 8))

    def render(self, counts_out=None, bucket_out=None, rgba_out=None, mean_out=None, lut=None):
        self._check_outputs(counts_out, bucket_out, rgba_out, mean_out)
        composite_render(self.ctx, counts_out, bucket_out, rgba_out, mean_out, lut)
        if not _on_device(counts_out, bucket_out, rgba_out, mean_out):
            self._borrowed.clear()

    def render_histogram(self, histogram_out, counts_out=None, bucket_out=None, rgba_out=None, lut=None):
        self._check_outputs(counts_out, bucket_out, rgba_out, histogram_out=histogram_out)
        composite_render_histogram(self.ctx, histogram_out, counts_out, bucket_out, rgba_out, lut)
        if not _on_device(histogram_out, counts_out, bucket_out, rgba_out):
            self._borrowed.clear()

    def render_host(self, lut=None) -> dict:
        """Renders into fresh numpy arrays."""
        h, w = self.height, self.width
        if self.config.mode == CPT_MODE_MEAN_DEPTH:
            mean = np.empty((h, w), np.float32)
            self.render(mean_out=mean)
            return {"mean": mean}
        counts = np.empty((h, w), np.uint16 if self.config.count_bits == 16 else np.uint32)
        bucket = np.empty((h, w), np.uint8)
        rgba = np.empty((h, w, 4), np.uint8)
        self.render(counts, bucket, rgba, lut=lut)
        return {"counts": counts, "bucket": bucket, "rgba": rgba}

    def load_counts(self, counts, n_members: int):
        """Resumes from a checkpoint: the composite becomes `counts` (a dense
        [H, W] array of the count type, host or device) with N members."""
        lib = load()
        item = self.config.count_bits // 8
        if hasattr(counts, "data_ptr"):
            if not counts.is_contiguous() or counts.element_size() != item or tuple(counts.shape) != (self.height, self.width):
                raise ValueError(f"counts must be a contiguous [{self.height}, {self.width}] tensor of {8 * item}-bit counts")
            ptr = counts.data_ptr()
        else:
            counts = np.ascontiguousarray(counts)
            if counts.itemsize != item or counts.shape != (self.height, self.width):
                raise ValueError(f"counts must be [{self.height}, {self.width}] of {8 * item}-bit counts")
            ptr = counts.ctypes.data
        _check(lib, self.ctx, lib.composite_load_counts(self.ctx, ctypes.c_void_p(ptr), int(n_members)))

    def sync(self):
        composite_sync(self.ctx)
        self._borrowed.clear()

    def trace(self) -> np.ndarray:
        return composite_trace_read(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ctx, self.ctx = self.ctx, None
            composite_end(ctx)
            self._borrowed.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- the batched engine (include/composite_engine.h) -------------------------

class EngineConfig(ctypes.Structure):
    _fields_ = [
        ("cuda_stream", ctypes.c_void_p),
        ("slab_members", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("wait_timeout_ms", ctypes.c_int64),
        ("schedule", ctypes.c_int32),
        ("upload_stream", ctypes.c_void_p),
        ("item_member_groups", ctypes.c_int32),
        ("staging_buffers", ctypes.c_int32),
        ("staging_bytes", ctypes.c_int64),
    ]


CPT_SCHEDULE_PERSISTENT, CPT_SCHEDULE_GRID = 0, 1


class Op(ctypes.Structure):
    _fields_ = [
        ("plane", ctypes.c_int32),
        ("sign", ctypes.c_int32),
        ("members", ctypes.c_void_p),
        ("member_index", ctypes.c_void_p),
        ("n_members", ctypes.c_int32),
        ("row_pitch_bytes", ctypes.c_int32),
        ("member_stride_bytes", ctypes.c_int64),
        ("mask_format", ctypes.c_int32),
    ]


class RenderOp(ctypes.Structure):
    _fields_ = [
        ("plane", ctypes.c_int32),
        ("counts_out", ctypes.c_void_p),
        ("bucket_out", ctypes.c_void_p),
        ("rgba_out", ctypes.c_void_p),
        ("histogram_out", ctypes.c_void_p),
    ]


_engine_sig_done = False


def _engine_lib():
    global _engine_sig_done
    lib = load()
    if not _engine_sig_done:
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        p32, p64 = ctypes.POINTER(i32), ctypes.POINTER(i64)
        sig = {
            "composite_engine_default_config": (ctypes.c_int, [ctypes.POINTER(EngineConfig)]),
            "composite_engine_begin": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(EngineConfig)]),
            "composite_engine_add_plane": (ctypes.c_int, [vp, i32, i32, p32]),
            "composite_engine_add_plane_bits": (ctypes.c_int, [vp, i32, i32, i32, p32]),
            "composite_engine_free_plane": (ctypes.c_int, [vp, i32]),
            "composite_engine_clear": (ctypes.c_int, [vp, i32]),
            "composite_engine_clear_many": (ctypes.c_int, [vp, p32, i32]),
            "composite_engine_submit": (ctypes.c_int, [vp, ctypes.POINTER(Op), i32]),
            "composite_engine_render": (ctypes.c_int, [vp, ctypes.POINTER(RenderOp), i32, vp]),
            "composite_engine_member_count": (ctypes.c_int, [vp, i32, p64]),
            "composite_engine_sync": (ctypes.c_int, [vp, p32]),
            "composite_engine_capture": (ctypes.c_int, [vp, ctypes.POINTER(Op), i32, ctypes.POINTER(RenderOp),
                                                        i32, vp]),
            "composite_engine_replay": (ctypes.c_int, [vp]),
            "composite_engine_tune": (ctypes.c_int, [vp, ctypes.POINTER(Op), i32, i32, p32, p32]),
            "composite_engine_get_tuning": (ctypes.c_int, [vp, p32, p32]),
            "composite_engine_get_config": (ctypes.c_int, [vp, ctypes.POINTER(EngineConfig)]),
            "composite_engine_end": (ctypes.c_int, [vp]),
            "composite_engine_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _engine_sig_done = True
    return lib


def _echeck(lib, eng, rc):
    if rc != CPT_OK:
        msg = lib.composite_engine_last_error(eng)
        raise CompositeError(rc, msg.decode() if msg else "")


def _lut_ptr(lut):
    if lut is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(lut, dtype=np.uint8).reshape(256, 4))
    return arr, arr.ctypes.data


class Engine:
    """Many composite planes on one GPU; ops on all of them run in one
    persistent launch (include/composite_engine.h)."""

    def __init__(self, stream=None, slab_members=0, ctas_per_sm=0, wait_timeout_ms=0, schedule="persistent",
                 item_member_groups=0, staging_buffers=0, staging_bytes=0):
        self.lib = _engine_lib()
        cfg = EngineConfig()
        self.lib.composite_engine_default_config(ctypes.byref(cfg))
        cfg.cuda_stream = stream if stream is not None else caller_stream()
        cfg.slab_members = slab_members
        cfg.ctas_per_sm = ctas_per_sm
        cfg.wait_timeout_ms = wait_timeout_ms
        cfg.schedule = {"persistent": CPT_SCHEDULE_PERSISTENT, "grid": CPT_SCHEDULE_GRID}[schedule]
        cfg.item_member_groups = item_member_groups
        cfg.staging_buffers = staging_buffers
        cfg.staging_bytes = staging_bytes
        h = ctypes.c_void_p()
        _echeck(self.lib, None, self.lib.composite_engine_begin(ctypes.byref(h), ctypes.byref(cfg)))
        self.h = h
        self._keep = []
        self.shapes = {}        # plane -> (width, height)
        self.count_bytes = {}   # plane -> bytes per count

    def add_plane(self, width: int, height: int, count_bits: int = 32) -> int:
        """A zeroed plane of uint32 (or, count_bits=16, uint16) counts; its id."""
        pid = ctypes.c_int32()
        _echeck(self.lib, self.h, self.lib.composite_engine_add_plane_bits(self.h, width, height, count_bits,
                                                                          ctypes.byref(pid)))
        self.shapes[pid.value] = (width, height)
        self.count_bytes[pid.value] = count_bits // 8
        return pid.value

    def free_plane(self, plane: int):
        _echeck(self.lib, self.h, self.lib.composite_engine_free_plane(self.h, plane))
        self.shapes.pop(plane, None)
        self.count_bytes.pop(plane, None)

    def clear(self, plane: int):
        _echeck(self.lib, self.h, self.lib.composite_engine_clear(self.h, plane))

    def clear_many(self, planes):
        """Clears every listed plane in one launch."""
        arr = (ctypes.c_int32 * len(planes))(*planes)
        _echeck(self.lib, self.h, self.lib.composite_engine_clear_many(self.h, arr, len(planes)))

    def op(self, plane: int, members, sign: int = 1, index=None, mask_format: str = "bytes") -> Op:
        """An op from a tensor of masks [n, H, W] (bit-packed: [n, H,
        ceil(W/8)]) in device or pinned host memory, or the whole ensemble
        when an int32 device index tensor selects members (device members
        only).  The engine keeps the tensors alive until sync."""
        ptr, n, _, _, stride, pitch, _, _ = _raster_view(members)
        self._keep.extend([members, index])
        o = Op()
        o.plane, o.sign, o.members = plane, sign, ptr
        o.mask_format = {"bytes": CPT_MASK_BYTES, "bits": CPT_MASK_BITS}[mask_format]
        o.row_pitch_bytes, o.member_stride_bytes = pitch, stride
        if index is not None:
            # the kernel reads members + index[i] * stride: every id must name
            # a raster of `members` (checked here, on the device values)
            import torch
            if not (isinstance(index, torch.Tensor) and index.is_cuda and index.dtype == torch.int32
                    and index.is_contiguous()):
                raise ValueError("index must be a contiguous int32 CUDA tensor")
            if index.numel() and (int(index.min()) < 0 or int(index.max()) >= n):
                raise ValueError(f"index holds member ids outside [0, {n})")
            o.member_index = index.data_ptr()
            o.n_members = int(index.numel())
        else:
            o.member_index = None
            o.n_members = n
        return o

    def render_op(self, plane: int, counts_out=None, bucket_out=None, rgba_out=None, histogram_out=None) -> RenderOp:
        if plane in self.shapes:   # an unknown plane is the library's to reject
            w, h = self.shapes[plane]
            _check_room(counts_out=(counts_out, w * h * self.count_bytes[plane]), bucket_out=(bucket_out, w * h),
                        rgba_out=(rgba_out, 4 * w * h), histogram_out=(histogram_out, 256 * 8))
        r = RenderOp()
        r.plane = plane
        r.counts_out, r.bucket_out, r.rgba_out = _ptr(counts_out), _ptr(bucket_out), _ptr(rgba_out)
        r.histogram_out = _ptr(histogram_out)
        return r

    def submit(self, ops, keep=()):
        arr = (Op * len(ops))(*ops)
        self._keep.extend(keep)
        _echeck(self.lib, self.h, self.lib.composite_engine_submit(self.h, arr, len(ops)))

    def render(self, rops, lut=None, keep=()):
        arr = (RenderOp * len(rops))(*rops)
        l, lp = _lut_ptr(lut)
        self._keep.extend(keep)
        _echeck(self.lib, self.h, self.lib.composite_engine_render(self.h, arr, len(rops), lp))

    def member_count(self, plane: int) -> int:
        n = ctypes.c_int64()
        _echeck(self.lib, self.h, self.lib.composite_engine_member_count(self.h, plane, ctypes.byref(n)))
        return n.value

    def sync(self):
        bad = ctypes.c_int32()
        rc = self.lib.composite_engine_sync(self.h, ctypes.byref(bad))
        self._keep.clear()
        if rc != CPT_OK:
            msg = self.lib.composite_engine_last_error(self.h)
            err = CompositeError(rc, msg.decode() if msg else "")
            err.plane = bad.value
            raise err

    def capture(self, ops, rops, lut=None, keep=()):
        a = (Op * len(ops))(*ops)
        r = (RenderOp * len(rops))(*rops)
        l, lp = _lut_ptr(lut)
        self._graph_keep = list(keep)
        _echeck(self.lib, self.h, self.lib.composite_engine_capture(self.h, a, len(ops), r, len(rops), lp))

    def replay(self):
        _echeck(self.lib, self.h, self.lib.composite_engine_replay(self.h))

    def tune(self, ops, repeats: int = 2):
        a = (Op * len(ops))(*ops)
        s, c = ctypes.c_int32(), ctypes.c_int32()
        _echeck(self.lib, self.h, self.lib.composite_engine_tune(self.h, a, len(ops), repeats,
                                                                  ctypes.byref(s), ctypes.byref(c)))
        return s.value, c.value

    def tuning(self):
        s, c = ctypes.c_int32(), ctypes.c_int32()
        _echeck(self.lib, self.h, self.lib.composite_engine_get_tuning(self.h, ctypes.byref(s), ctypes.byref(c)))
        return s.value, c.value

    def config(self) -> dict:
        """Every field of the engine's current configuration (after tuning:
        the tuned values)."""
        cfg = EngineConfig()
        _echeck(self.lib, self.h, self.lib.composite_engine_get_config(self.h, ctypes.byref(cfg)))
        return {name: getattr(cfg, name) for name, _ in EngineConfig._fields_
                if name not in ("cuda_stream", "upload_stream")}

    def close(self):
        if getattr(self, "h", None) is not None:
            h, self.h = self.h, None
            self.lib.composite_engine_end(h)
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- the interactive server (include/composite_server.h) ---------------------

class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("resident", ctypes.c_void_p),
        ("n_resident", ctypes.c_int32),
        ("overflow", ctypes.c_void_p),
        ("n_overflow", ctypes.c_int32),
        ("row_pitch_bytes", ctypes.c_int32),
        ("member_stride_bytes", ctypes.c_int64),
        ("max_sessions", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("staging_members", ctypes.c_int32),
        ("max_cycles_in_flight", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_int64),
        ("cuda_stream", ctypes.c_void_p),
        ("wait_timeout_ms", ctypes.c_int64),
        ("mask_format", ctypes.c_int32),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("requests_done", "cycles", "members_added", "members_removed", "recomputes",
                 "overflow_uploads", "queued", "in_flight", "cycle_device_us", "enqueue_host_us")]


_server_sig_done = False


def _server_lib():
    global _server_sig_done
    lib = load()
    if not _server_sig_done:
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "composite_server_default_config": (ctypes.c_int, [ctypes.POINTER(ServerConfig)]),
            "composite_server_begin": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig)]),
            "composite_server_open_session": (ctypes.c_int, [vp, ctypes.POINTER(i32)]),
            "composite_server_close_session": (ctypes.c_int, [vp, i32]),
            "composite_server_request": (ctypes.c_int, [vp, i32, vp, i32, vp, vp, vp, ctypes.POINTER(i64)]),
            "composite_server_request_histogram": (ctypes.c_int, [vp, i32, vp, i32, vp, vp, vp, vp,
                                                                  ctypes.POINTER(i64)]),
            "composite_server_pump": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
            "composite_server_drain": (ctypes.c_int, [vp]),
            "composite_server_session_members": (ctypes.c_int, [vp, i32, ctypes.POINTER(i64)]),
            "composite_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
            "composite_server_end": (ctypes.c_int, [vp]),
            "composite_server_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _server_sig_done = True
    return lib


def _scheck(lib, srv, rc):
    if rc != CPT_OK:
        msg = lib.composite_server_last_error(srv)
        raise CompositeError(rc, msg.decode() if msg else "")


class Server:
    """Sessions, requests and continuous batching (include/composite_server.h).
    ``resident``: device uint8[n_r, H, W]; ``overflow``: pinned host uint8[n_o, H, W]
    with the same row pitch and member stride, or None."""

    def __init__(self, resident, overflow=None, max_sessions=64, max_batch=64, staging_members=64,
                 max_cycles_in_flight=4, hbm_budget_bytes=0, stream=None, wait_timeout_ms=0,
                 mask_format="bytes", width=None):
        self.lib = _server_lib()
        rptr, rn, h, w, rstride, rpitch, _, _ = _raster_view(resident)
        if mask_format == "bits":
            if width is None or (width + 7) // 8 != w:
                raise ValueError("bit-packed ensembles need the raster width (rows of ceil(width / 8) bytes)")
            w = width
        cfg = ServerConfig()
        self.lib.composite_server_default_config(ctypes.byref(cfg))
        cfg.width, cfg.height = w, h
        cfg.resident, cfg.n_resident = rptr, rn
        cfg.row_pitch_bytes, cfg.member_stride_bytes = rpitch, rstride
        if overflow is not None:
            optr, on, oh, ow, ostride, opitch, _, _ = _raster_view(overflow)
            if (oh, ostride, opitch) != (h, rstride, rpitch):
                raise ValueError("overflow must have the resident part's layout")
            cfg.overflow, cfg.n_overflow = optr, on
        cfg.max_sessions, cfg.max_batch = max_sessions, max_batch
        cfg.staging_members, cfg.max_cycles_in_flight = staging_members, max_cycles_in_flight
        cfg.hbm_budget_bytes, cfg.wait_timeout_ms = hbm_budget_bytes, wait_timeout_ms
        cfg.cuda_stream = stream if stream is not None else caller_stream()
        cfg.mask_format = {"bytes": CPT_MASK_BYTES, "bits": CPT_MASK_BITS}[mask_format]
        srv = ctypes.c_void_p()
        _scheck(self.lib, None, self.lib.composite_server_begin(ctypes.byref(srv), ctypes.byref(cfg)))
        self.h = srv
        self.width, self.height = w, h
        self._members = (resident, overflow)
        self._pending = {}

    def open_session(self) -> int:
        s = ctypes.c_int32()
        _scheck(self.lib, self.h, self.lib.composite_server_open_session(self.h, ctypes.byref(s)))
        return s.value

    def close_session(self, session: int):
        _scheck(self.lib, self.h, self.lib.composite_server_close_session(self.h, session))

    def request(self, session: int, toggle, counts_out=None, bucket_out=None, rgba_out=None,
                histogram_out=None) -> int:
        px = self.width * self.height
        _check_room(counts_out=(counts_out, 4 * px), bucket_out=(bucket_out, px), rgba_out=(rgba_out, 4 * px),
                    histogram_out=(histogram_out, 256 * 8))
        ids = np.ascontiguousarray(np.asarray(toggle, dtype=np.int32))
        rid = ctypes.c_int64()
        if histogram_out is None:
            rc = self.lib.composite_server_request(
                self.h, session, ids.ctypes.data if ids.size else None, int(ids.size), _ptr(counts_out),
                _ptr(bucket_out), _ptr(rgba_out), ctypes.byref(rid))
        else:
            rc = self.lib.composite_server_request_histogram(
                self.h, session, ids.ctypes.data if ids.size else None, int(ids.size), _ptr(counts_out),
                _ptr(bucket_out), _ptr(rgba_out), _ptr(histogram_out), ctypes.byref(rid))
        _scheck(self.lib, self.h, rc)
        self._pending[rid.value] = (counts_out, bucket_out, rgba_out, histogram_out)
        return rid.value

    def pump(self, capacity: int = 4096) -> list:
        buf = (ctypes.c_int64 * capacity)()
        n = ctypes.c_int32()
        _scheck(self.lib, self.h, self.lib.composite_server_pump(self.h, buf, capacity, ctypes.byref(n)))
        done = list(buf[: n.value])
        for rid in done:
            self._pending.pop(rid, None)
        return done

    def drain(self):
        _scheck(self.lib, self.h, self.lib.composite_server_drain(self.h))
        self._pending.clear()

    def session_members(self, session: int) -> int:
        n = ctypes.c_int64()
        _scheck(self.lib, self.h, self.lib.composite_server_session_members(self.h, session, ctypes.byref(n)))
        return n.value

    def stats(self) -> dict:
        st = ServerStats()
        _scheck(self.lib, self.h, self.lib.composite_server_get_stats(self.h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) is not None:
            h, self.h = self.h, None
            self.lib.composite_server_end(h)
            self._pending.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
