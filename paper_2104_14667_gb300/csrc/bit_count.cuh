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

// The 32 counts of a BitCounter as 16 words of two 16-bit counts (pixel 2i in
// the low half of pairs[i], pixel 2i+1 in the high half).  Eight pixels at a
// time, byte b of each of the eight bit-slices becomes row j of an 8 x 8 bit
// matrix held in one 64-bit word; transposing it (three delta swaps of 1-,
// 2- and 4-bit blocks across the diagonal, the 8 x 8 bit-matrix transpose of
// Warren's "Hacker's Delight", section 7-3) makes byte i the count of pixel
// 8b + i with bit j weighted 2^j (counts are below 256), and the bytes are
// then moved into 16-bit lanes.  About 40 operations per 8 pixels (a
// nibble-spreading multiply per slice and 4 pixels took ~70, a per-pixel
// extraction ~160).
__device__ __forceinline__ void bitcount_pairs(const BitCounter &s, uint32_t (&pairs)[16]) {
    const uint32_t sl[8] = {s.ones, s.twos, s.fours, s.eights, s.hi[0], s.hi[1], s.hi[2], s.hi[3]};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t sel = (uint32_t)b | ((uint32_t)(b + 4) << 4);      // byte b of x, byte b of y
        const uint32_t lo = __byte_perm(__byte_perm(sl[0], sl[1], sel), __byte_perm(sl[2], sl[3], sel), 0x5410);
        const uint32_t hi = __byte_perm(__byte_perm(sl[4], sl[5], sel), __byte_perm(sl[6], sl[7], sel), 0x5410);
        uint64_t x = (uint64_t)lo | ((uint64_t)hi << 32);
        uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
        x = x ^ t ^ (t << 7);
        t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
        x = x ^ t ^ (t << 14);
        t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
        x = x ^ t ^ (t << 28);
        const uint32_t c_lo = (uint32_t)x, c_hi = (uint32_t)(x >> 32);    // counts of pixels 8b .. 8b + 7
        pairs[4 * b] = __byte_perm(c_lo, 0u, 0x4140);
        pairs[4 * b + 1] = __byte_perm(c_lo, 0u, 0x4342);
        pairs[4 * b + 2] = __byte_perm(c_hi, 0u, 0x4140);
        pairs[4 * b + 3] = __byte_perm(c_hi, 0u, 0x4342);
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
