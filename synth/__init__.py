"""Seeded synthetic flood ensembles: the one input source shared by the tests,
the oracle checks and the benchmark.

The paper composites ensembles of simulated and observed flood-extent rasters
(Section 2, "Motivation"; Fig. 1).  Those datasets are not public, so the
inputs here are synthetic, shaped like the paper's workloads: 1 byte per pixel
flood masks (the transfer-rate tables of Section 6.1, Figs. 6 and 9, balance
only at 1 B/pixel), square or rectangular rasters, member counts from 1 to
thousands.

Recipe (fixed here, consumed as bytes by both sides):

* PRNG: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter based:
  draw i of a stream seeded s is ``mix(s + (i+1)*0x9E3779B97F4A7C15)``.
  Uniforms are ``(x >> 11) * 2**-53``; normal i is Box-Muller over
  uniforms 2i and 2i+1.
* Terrain: the sum of 64 Gaussian bumps (centre uniform over the raster,
  sigma uniform in [20, 200] px, amplitude uniform in [0, 1]) plus 0.01 white
  normal noise per pixel, accumulated in float64 and rounded once to float32.
* Member m: flooded fraction f_m ~ U[0.1, 0.5] from its own stream
  (seed ^ (m+1)*gamma), k_m = floor(f_m * W * H), water level
  w_m = sorted(terrain)[k_m], and mask_m(p) = 1 iff terrain(p) < w_m.
  F_m, the number of flooded pixels, is recorded from the sorted terrain.
* Depth of member m: max(w_m - terrain(p), 0) in float32 (positive exactly
  where the mask is 1).

This module holds none of the compositing arithmetic: it produces inputs and
their metadata only.  Values are bit-reproducible on one platform; across
platforms the terrain may differ in the last ulp of ``exp``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

N_BUMPS = 64
SIGMA_RANGE = (20.0, 200.0)
NOISE_STD = 0.01
FLOOD_FRACTION_RANGE = (0.1, 0.5)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream for ``seed``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals; normal i is Box-Muller (cosine branch) over uniform
    draws 2i and 2i+1, so any range of normals can be drawn on its own."""
    u = uniforms(seed, 2 * count, 2 * start)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _substream(seed: int, tag: int) -> int:
    """Seed of an independent stream: seed xor tag * golden gamma (mod 2**64)."""
    mask = 0xFFFFFFFFFFFFFFFF
    return (seed & mask) ^ ((tag * int(GAMMA)) & mask)


def terrain(seed: int, width: int, height: int, rows: slice | None = None) -> np.ndarray:
    """float32[height, width] terrain; ``rows`` restricts to a band of rows."""
    if width <= 0 or height <= 0:
        raise ValueError("raster sides must be positive")
    bump = uniforms(_substream(seed, 0xB0B), 4 * N_BUMPS).reshape(N_BUMPS, 4)
    y0, y1 = (0, height) if rows is None else (rows.start or 0, rows.stop if rows.stop is not None else height)
    xs = np.arange(width, dtype=np.float64)
    ys = np.arange(y0, y1, dtype=np.float64)
    acc = np.zeros((y1 - y0, width), dtype=np.float64)
    for cx_u, cy_u, s_u, amp in bump:
        cx, cy = cx_u * width, cy_u * height
        sigma = SIGMA_RANGE[0] + s_u * (SIGMA_RANGE[1] - SIGMA_RANGE[0])
        gx = np.exp(-((xs - cx) ** 2) / (2.0 * sigma * sigma))
        gy = np.exp(-((ys - cy) ** 2) / (2.0 * sigma * sigma))
        acc += amp * np.outer(gy, gx)
    noise = normals(_substream(seed, 0x5EED), (y1 - y0) * width, y0 * width)
    acc += NOISE_STD * noise.reshape(y1 - y0, width)
    return acc.astype(np.float32)


@dataclass
class Ensemble:
    """Metadata of a synthetic ensemble over one terrain."""

    seed: int
    width: int
    height: int
    terrain: np.ndarray       # float32[H, W]
    levels: np.ndarray        # float32[N] water level w_m
    flooded: np.ndarray       # int64[N]  F_m = #{p : terrain(p) < w_m}

    @property
    def n(self) -> int:
        return int(self.levels.shape[0])

    @property
    def pixels(self) -> int:
        return self.width * self.height


def ensemble(seed: int, width: int, height: int, n_members: int,
             member_offset: int = 0) -> Ensemble:
    """Water levels for members ``member_offset .. member_offset+n-1``."""
    return ensemble_from_terrain(seed, terrain(seed, width, height), n_members, member_offset)


def ensemble_from_terrain(seed: int, t: np.ndarray, n_members: int, member_offset: int = 0,
                          flat_sorted: np.ndarray | None = None) -> Ensemble:
    """As ensemble, over a terrain already computed (and optionally sorted)."""
    height, width = t.shape
    if flat_sorted is None:
        flat_sorted = np.sort(t, axis=None)
    p = width * height
    levels = np.empty(n_members, dtype=np.float32)
    flooded = np.empty(n_members, dtype=np.int64)
    lo, hi = FLOOD_FRACTION_RANGE
    for i in range(n_members):
        m = member_offset + i
        f = lo + (hi - lo) * uniforms(_substream(seed, m + 1), 1)[0]
        k = min(int(math.floor(f * p)), p - 1)
        levels[i] = flat_sorted[k]
        flooded[i] = int(np.searchsorted(flat_sorted, levels[i], side="left"))
    return Ensemble(seed, width, height, t, levels, flooded)


BATCH_SIDES = (256, 512, 1024, 2048, 4096)


def batched_requests(seed: int, count: int, n_range=(8, 2048), sides=BATCH_SIDES):
    """(width, height, members) of `count` composite requests: members
    log-uniform in n_range, width and height drawn independently from
    `sides` (so shapes are often not square)."""
    u = uniforms(_substream(seed, 0xBA7C4), 3 * count).reshape(count, 3)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    out = []
    for a, b, c in u:
        n = int(math.floor(math.exp(lo + a * (hi - lo))))
        n = min(max(n, n_range[0]), n_range[1])
        out.append((sides[int(b * len(sides))], sides[int(c * len(sides))], n))
    return out


def serving_trace(seed: int, n_requests: int, rate_per_s: float, n_sessions: int, n_members: int,
                  size_range=(8, 4096)):
    """Requests of an interactive session mix: Poisson arrivals at rate_per_s
    (exponential gaps), a uniform session, and a toggle set whose size is
    log-uniform in size_range, drawn uniformly from all members.
    Returns [(arrival_s, session, int32 ids)]."""
    u = uniforms(_substream(seed, 0x5E7E), 3 * n_requests).reshape(n_requests, 3)
    lo, hi = math.log(size_range[0]), math.log(size_range[1])
    t = 0.0
    out = []
    for r, (a, b, c) in enumerate(u):
        t += -math.log1p(-a) / rate_per_s
        k = min(max(int(math.exp(lo + c * (hi - lo))), size_range[0]), size_range[1], n_members)
        ids = (splitmix64(_substream(seed, 0x70661E + r), k) % np.uint64(n_members)).astype(np.int32)
        out.append((t, int(b * n_sessions), ids))
    return out


def fill_masks(ens: Ensemble, out: np.ndarray, members: range | None = None) -> np.ndarray:
    """Writes uint8 {0,1} masks of ``members`` into ``out`` (uint8[n, H, W])."""
    idx = range(ens.n) if members is None else members
    if out.dtype != np.uint8 or out.shape[1:] != (ens.height, ens.width) or out.shape[0] < len(idx):
        raise ValueError("out must be uint8[n, H, W] with room for every member")
    flat_t = ens.terrain
    for j, m in enumerate(idx):
        np.less(flat_t, ens.levels[m], out=out[j].view(np.bool_))
    return out


def fill_masks_torch(ens: Ensemble, out, members: range | None = None, terrain_t=None):
    """As fill_masks, into a torch uint8[n, H, W] tensor on any device: the
    same float32 comparison terrain < w_m, so the bytes are identical."""
    import torch
    idx = range(ens.n) if members is None else members
    if out.dtype != torch.uint8 or tuple(out.shape[1:]) != (ens.height, ens.width) or out.shape[0] < len(idx):
        raise ValueError("out must be uint8[n, H, W] with room for every member")
    t = terrain_t if terrain_t is not None else torch.from_numpy(ens.terrain).to(out.device)
    for j, m in enumerate(idx):
        torch.lt(t, float(ens.levels[m]), out=out[j].view(torch.bool))
    return out


def fill_depths_torch(ens: Ensemble, out, members: range | None = None, terrain_t=None):
    """As depths, into a torch float32[n, H, W] tensor on any device: the same
    float32 subtraction w_m - terrain, clipped at 0, so the values are identical."""
    import torch
    idx = range(ens.n) if members is None else members
    if out.dtype != torch.float32 or tuple(out.shape[1:]) != (ens.height, ens.width) or out.shape[0] < len(idx):
        raise ValueError("out must be float32[n, H, W] with room for every member")
    t = terrain_t if terrain_t is not None else torch.from_numpy(ens.terrain).to(out.device)
    for j, m in enumerate(idx):
        torch.sub(torch.tensor(float(ens.levels[m]), dtype=torch.float32, device=t.device), t, out=out[j])
        out[j].clamp_(min=0.0)
    return out


def pack_masks(m: np.ndarray) -> np.ndarray:
    """Bit-packed copy of uint8[..., H, W] masks: uint8[..., H, ceil(W/8)],
    pixel x in bit (x & 7) of byte x >> 3, any nonzero byte a 1 bit."""
    return np.packbits(np.asarray(m) != 0, axis=-1, bitorder="little")


def pack_masks_torch(m):
    """pack_masks for a torch uint8[n, H, W] tensor with W a multiple of 8, on
    its own device: the same bit layout."""
    import torch
    n, h, w = m.shape
    if w % 8:
        raise ValueError("width must be a multiple of 8")
    shifts = torch.arange(8, device=m.device, dtype=torch.uint8)
    bits = (m.reshape(n, h, w // 8, 8) != 0).to(torch.uint8) << shifts
    return bits.sum(dim=-1, dtype=torch.uint8)


def masks(ens: Ensemble) -> np.ndarray:
    """uint8[N, H, W] masks with values in {0, 1}."""
    return fill_masks(ens, np.empty((ens.n, ens.height, ens.width), dtype=np.uint8))


def depths(ens: Ensemble, members: range | None = None) -> np.ndarray:
    """float32[n, H, W] water depths max(w_m - terrain, 0)."""
    idx = range(ens.n) if members is None else members
    out = np.empty((len(idx), ens.height, ens.width), dtype=np.float32)
    for j, m in enumerate(idx):
        np.maximum(ens.levels[m] - ens.terrain, np.float32(0.0), out=out[j])
    return out


def scramble_nonzero(m: np.ndarray, seed: int) -> np.ndarray:
    """Replaces every nonzero byte by a random byte in 1..255 (keeps zeros)."""
    r = (splitmix64(_substream(seed, 0xACE), m.size) % np.uint64(255)).astype(np.uint8) + np.uint8(1)
    return np.where(m != 0, r.reshape(m.shape), np.uint8(0)).astype(np.uint8)


def random_masks(seed: int, n: int, height: int, width: int, density: float = 0.5) -> np.ndarray:
    """Independent Bernoulli masks (no shared terrain): uint8[n, H, W] in {0,1}."""
    u = uniforms(_substream(seed, 0xD1CE), n * height * width)
    return (u < density).astype(np.uint8).reshape(n, height, width)


def random_depths(seed: int, n: int, height: int, width: int, scale: float = 4.0) -> np.ndarray:
    """Independent non-negative float32 depths with about half the pixels dry."""
    u = uniforms(_substream(seed, 0xDEE9), 2 * n * height * width)
    wet = u[0::2] < 0.5
    d = np.where(wet, scale * u[1::2], 0.0).astype(np.float32)
    return d.reshape(n, height, width)
