// bit_count.cuh -- counting bit-packed masks: carry-save (Harley-Seal)
// accumulators over 32-pixel words, the transpose out of the bit-sliced form,
// and folding the counts into a composite.
#pragma once

#include "device_common.cuh"

namespace cpt {

// Counts of 32 pixels at once from bit-packed masks (one bit per pixel), kept
// bit-sliced as carry-save accumulators in the manner of the Harley-Seal
// population count:
// bit i of `ones`, `twos`, `fours`, `eights` holds one bit of weight 1, 2, 4,
// 8 of pixel i's count, and every 16 members the weight-16 carries ripple
// into a 4-level counter `hi` (counts stay below 256, one slab).  Sixteen
// members cost 15 carry-save adders (5 logic operations each) plus the
// ripple, about 5 operations per word instead of 16 for a plain ripple-carry
// counter.
struct BitCounter {
    uint32_t ones = 0, twos = 0, fours = 0, eights = 0;
    uint32_t hi[4] = {0u, 0u, 0u, 0u};
};

// Carry-save adder: a + b + c = 2 * h + l, bitwise.
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

__device__ __forceinline__ void bitcount_add16(BitCounter &s, const uint32_t (&w)[16]) {
    uint32_t twos_a, twos_b, fours_a, fours_b, eights_a, eights_b, sixteens;
    csa(twos_a, s.ones, s.ones, w[0], w[1]);
    csa(twos_b, s.ones, s.ones, w[2], w[3]);
    csa(fours_a, s.twos, s.twos, twos_a, twos_b);
    csa(twos_a, s.ones, s.ones, w[4], w[5]);
    csa(twos_b, s.ones, s.ones, w[6], w[7]);
    csa(fours_b, s.twos, s.twos, twos_a, twos_b);
    csa(eights_a, s.fours, s.fours, fours_a, fours_b);
    csa(twos_a, s.ones, s.ones, w[8], w[9]);
    csa(twos_b, s.ones, s.ones, w[10], w[11]);
    csa(fours_a, s.twos, s.twos, twos_a, twos_b);
    csa(twos_a, s.ones, s.ones, w[12], w[13]);
    csa(twos_b, s.ones, s.ones, w[14], w[15]);
    csa(fours_b, s.twos, s.twos, twos_a, twos_b);
    csa(eights_b, s.fours, s.fours, fours_a, fours_b);
    csa(sixteens, s.eights, s.eights, eights_a, eights_b);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t carry = s.hi[j] & sixteens;
        s.hi[j] ^= sixteens;
        sixteens = carry;
    }
}

// Count of pixel i (0..31).
__device__ __forceinline__ uint32_t bitcount_get(const BitCounter &s, int i) {
    uint32_t v = ((s.ones >> i) & 1u) | (((s.twos >> i) & 1u) << 1) | (((s.fours >> i) & 1u) << 2) |
                 (((s.eights >> i) & 1u) << 3);
#pragma unroll
    for (int j = 0; j < 4; ++j) v += ((s.hi[j] >> i) & 1u) << (4 + j);
    return v;
}

// The 32 counts of a BitCounter as 16 words of two 16-bit counts (pixel 2i in
// the low half of pairs[i], pixel 2i+1 in the high half).  Four pixels at a
// time, each bit-slice's 4-bit field is spread into byte lanes -- a 4-bit
// field times 0x00204081 puts its bit k at bit 8k, and the four shifted
// copies do not overlap -- weighted by the slice's power of two and summed
// (the counts are below 256, so no byte carries into the next); the bytes
// are then moved into 16-bit lanes.  About 270 operations for 32 pixels,
// against ~20 per pixel for bitcount_get.
__device__ __forceinline__ void bitcount_pairs(const BitCounter &s, uint32_t (&pairs)[16]) {
    const uint32_t slice[8] = {s.ones, s.twos, s.fours, s.eights, s.hi[0], s.hi[1], s.hi[2], s.hi[3]};
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        uint32_t bytes = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t field = (slice[j] >> (4 * n)) & 0xFu;
            bytes += ((field * 0x00204081u) & 0x01010101u) << j;
        }
        pairs[2 * n] = __byte_perm(bytes, 0u, 0x4140);       // pixels 4n, 4n + 1
        pairs[2 * n + 1] = __byte_perm(bytes, 0u, 0x4342);   // pixels 4n + 2, 4n + 3
    }
}

// A group of 16 counts given as 8 pair words (see bitcount_pairs) folded into
// dst: a read-modify-write of the group's first `valid` pixels, or (atomic)
// atomic adds/subtractions as in atomic_count_group, uint16 counts a pair per
// 32-bit atomic.
template <typename CountT>
__device__ __forceinline__ void apply_pair_group(CountT *dst, int valid, const uint32_t *pairs, int sign,
                                                 int *flags) {
    uint32_t wide[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        wide[2 * k] = pairs[k] & 0xFFFFu;
        wide[2 * k + 1] = pairs[k] >> 16;
    }
    apply_count_group<CountT>(dst, valid, wide, sign, flags);
}

template <typename CountT>
__device__ __forceinline__ void atomic_pair_group(CountT *dst, const uint32_t *pairs, int sign, int *flags) {
    if constexpr (sizeof(CountT) == 2) {
        bool under = false;
        uint32_t *w = reinterpret_cast<uint32_t *>(dst);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t d = pairs[k];
            if (d == 0) continue;
            if (sign > 0) {
                atomicAdd(w + k, d);
            } else {
                const uint32_t old = atomicSub(w + k, d);
                under |= ((d & 0xFFFFu) > (old & 0xFFFFu)) | ((d >> 16) > (old >> 16));
            }
        }
        if (under) flag_set(flags, kFlagUnderflow);
    } else {
        uint32_t wide[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            wide[2 * k] = pairs[k] & 0xFFFFu;
            wide[2 * k + 1] = pairs[k] >> 16;
        }
        atomic_count_group<CountT>(dst, wide, sign, flags);
    }
}

}  // namespace cpt
