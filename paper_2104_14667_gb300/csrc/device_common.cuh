// device_common.cuh -- device helpers shared by the accumulation kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cpt {

// 1 in every byte of x that is nonzero, 0 elsewhere.  A mask byte counts as
// flooded when it is nonzero (any value, not only 1).  SWAR: adding 0x7F to
// the low seven bits of a byte sets its bit 7 exactly when those bits are not
// all zero, without carrying into the next byte; or-ing x back in adds the
// byte 0x80.  Bit 7 is then moved down to bit 0.
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t x) {
    uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    return (t >> 7) & 0x01010101u;
}

// Keeps the per-byte ones of word `word` (bytes 4*word .. 4*word+3 of a
// 16-byte group) that lie in the first `valid` bytes of the group.
__device__ __forceinline__ uint32_t valid_byte_mask(int word, int valid) {
    int k = valid - 4 * word;
    if (k >= 4) return 0x01010101u;
    if (k <= 0) return 0u;
    return 0x01010101u & ((1u << (8 * k)) - 1u);
}

// Adds four packed byte counters (16 pixels, pixel 4i+b in byte b of word i)
// into 16 wide counters.
__device__ __forceinline__ void widen16(uint32_t (&wide)[16], uint32_t p0, uint32_t p1,
                                        uint32_t p2, uint32_t p3) {
    const uint32_t p[4] = {p0, p1, p2, p3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int b = 0; b < 4; ++b) wide[4 * i + b] += (p[i] >> (8 * b)) & 0xFFu;
    }
}

__device__ __forceinline__ void flag_set(int *flags, int index) {
    atomicOr(flags + index, 1);
}

// Read-modify-write of one group of 16 composite counts: dst[j] += wide[j]
// (sign > 0) or dst[j] -= wide[j] (sign < 0) for j < valid.  A subtraction
// below zero raises the underflow flag (the composite is then invalid).
template <typename CountT>
__device__ __forceinline__ void apply_count_group(CountT *dst, int valid,
                                                  const uint32_t (&wide)[16], int sign,
                                                  int *flags) {
    bool under = false;
    if (valid == 16) {
        if constexpr (sizeof(CountT) == 2) {
            uint4 *d = reinterpret_cast<uint4 *>(dst);
            uint4 a = d[0], b = d[1];
            uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t lo = w[k] & 0xFFFFu, hi = w[k] >> 16;
                uint32_t dl = wide[2 * k], dh = wide[2 * k + 1];
                if (sign > 0) {
                    lo += dl;
                    hi += dh;
                } else {
                    under |= (dl > lo) | (dh > hi);
                    lo -= dl;
                    hi -= dh;
                }
                w[k] = (lo & 0xFFFFu) | (hi << 16);
            }
            d[0] = make_uint4(w[0], w[1], w[2], w[3]);
            d[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
            uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 v = d[q];
                uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t dv = wide[4 * q + k];
                    if (sign > 0) {
                        w[k] += dv;
                    } else {
                        under |= dv > w[k];
                        w[k] -= dv;
                    }
                }
                d[q] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < valid) {
                uint32_t old = dst[j];
                if (sign > 0) {
                    dst[j] = static_cast<CountT>(old + wide[j]);
                } else {
                    under |= wide[j] > old;
                    dst[j] = static_cast<CountT>(old - wide[j]);
                }
            }
        }
    }
    if (under) flag_set(flags, kFlagUnderflow);
}

// The same update as apply_count_group, by atomic adds (or subtractions) on
// the 32-bit words of the group, for launches where several threads fold
// different member slabs into the same pixels.  Pixels past the raster's edge
// carry a zero delta.  uint16 counts are updated two to a word: an add cannot
// carry into the upper half because no count exceeds N <= 65535, and a
// subtraction that would borrow is itself an underflow, caught from the
// returned old value (subtractions only decrease a count, so a count that
// ends below zero makes some subtraction see an old value below its delta).
template <typename CountT>
__device__ __forceinline__ void atomic_count_group(CountT *dst, const uint32_t (&wide)[16], int sign,
                                                   int *flags) {
    bool under = false;
    uint32_t *w = reinterpret_cast<uint32_t *>(dst);
    if constexpr (sizeof(CountT) == 2) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t dl = wide[2 * k], dh = wide[2 * k + 1];
            const uint32_t d = dl | (dh << 16);
            if (d == 0) continue;
            if (sign > 0) {
                atomicAdd(w + k, d);
            } else {
                const uint32_t old = atomicSub(w + k, d);
                under |= (dl > (old & 0xFFFFu)) | (dh > (old >> 16));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (wide[j] == 0) continue;
            if (sign > 0) {
                atomicAdd(w + j, wide[j]);
            } else {
                const uint32_t old = atomicSub(w + j, wide[j]);
                under |= wide[j] > old;
            }
        }
    }
    if (under) flag_set(flags, kFlagUnderflow);
}

// dst[j] (+|-)= acc[j] for the first `valid` of four float32 sums.
__device__ __forceinline__ void apply_depth_group(float *dst, int valid, const float (&acc)[4],
                                                  int sign) {
    if (valid == 4) {
        float4 *d = reinterpret_cast<float4 *>(dst);
        float4 v = *d;
        if (sign > 0) {
            v.x += acc[0]; v.y += acc[1]; v.z += acc[2]; v.w += acc[3];
        } else {
            v.x -= acc[0]; v.y -= acc[1]; v.z -= acc[2]; v.w -= acc[3];
        }
        *d = v;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < valid) dst[j] = sign > 0 ? dst[j] + acc[j] : dst[j] - acc[j];
    }
}

}  // namespace cpt
