// bits_kernels.cu -- the accumulation step over bit-packed masks (one bit
// per pixel) for layouts the bulk-copy kernel of tma_kernels.cu does not take:
// padded or unaligned rows, and pinned host memory read in place.
#include <algorithm>

#include "bit_count.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;
constexpr int kPackedLimit = 255;   // members a bit-sliced counter can hold

// Bit-packed masks (one bit per pixel, pixel x at bit x & 7 of byte x >> 3 of
// the row).  A thread owns kWords 32-pixel words of a composite row (with
// kWords = 2 a warp reads 256 contiguous bytes per member, 8 per lane) and
// keeps the slab's counts in BitCounters (carry-save accumulators, see
// bit_count.cuh); whole steps of 16 members load without predicates, and
// the counts leave the bit-sliced form through bitcount_pairs.
template <typename CountT, int kWords>
__global__ void __launch_bounds__(kThreads, 4)
count_bits_kernel(RasterBatch b, Plane p, int sign, int *flags, int64_t units, int units_per_row,
                  int slab, int slabs) {
    constexpr int kPix = 32 * kWords;
    CountT *plane = static_cast<CountT *>(p.data);
    const int64_t stride = b.member_stride;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units * slabs;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int sl = (int)(u / units);
        const int64_t g = u - (int64_t)sl * units;
        const int y = (int)(g / units_per_row);
        const int gx = (int)(g - (int64_t)y * units_per_row);
        const int x0 = gx * kPix;
        const int valid = min(kPix, p.width - x0);
        const int m0 = sl * slab;
        const int m1 = min(b.n, m0 + slab);
        const uint8_t *q = static_cast<const uint8_t *>(b.base) + (int64_t)y * b.row_pitch + gx * 4 * kWords +
                           (int64_t)m0 * stride;
        BitCounter acc[kWords];
        int m = m0;
        if (valid == kPix) {
            for (; m + 16 <= m1; m += 16) {
                uint32_t w[kWords][16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if constexpr (kWords == 2) {
                        const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(q + k * stride));
                        w[0][k] = v.x;
                        w[1][k] = v.y;
                    } else {
                        w[0][k] = __ldcs(reinterpret_cast<const uint32_t *>(q + k * stride));
                    }
                }
#pragma unroll
                for (int j = 0; j < kWords; ++j) bitcount_add16(acc[j], w[j]);
                q += 16 * stride;
            }
        }
        // the slab's last (< 16) members, and every member at a ragged right
        // edge: word by word, bits past the width dropped
        for (; m < m1; m += 16) {
            const int take = min(16, m1 - m);
#pragma unroll
            for (int j = 0; j < kWords; ++j) {
                const int vj = min(32, max(0, valid - 32 * j));
                const int nbytes = (vj + 7) / 8;
                const uint32_t keep = vj == 32 ? 0xFFFFFFFFu : ((1u << vj) - 1u);
                uint32_t w[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    uint32_t v = 0;
                    if (k < take) {
                        const uint8_t *r = q + k * stride + 4 * j;
                        if (vj == 32)
                            v = __ldcs(reinterpret_cast<const uint32_t *>(r));
                        else
                            for (int i = 0; i < nbytes; ++i) v |= (uint32_t)r[i] << (8 * i);
                    }
                    w[k] = v & keep;
                }
                bitcount_add16(acc[j], w);
            }
            q += 16 * stride;
        }
        CountT *dst = plane + (int64_t)y * p.pitch + x0;
#pragma unroll
        for (int j = 0; j < kWords; ++j) {
            if (valid <= 32 * j) break;
            uint32_t pairs[16];
            bitcount_pairs(acc[j], pairs);
#pragma unroll
            for (int h = 0; h < 2; ++h) {           // two 16-pixel groups per word
                const int v = min(16, valid - 32 * j - 16 * h);
                if (v <= 0) break;
                if (slabs == 1)
                    apply_pair_group<CountT>(dst + 32 * j + 16 * h, v, pairs + 8 * h, sign, flags);
                else
                    atomic_pair_group<CountT>(dst + 32 * j + 16 * h, pairs + 8 * h, sign, flags);
            }
        }
    }
}

inline int64_t blocks_for(int64_t groups) {
    int64_t blocks = (groups + kThreads - 1) / kThreads;
    return blocks < 1 ? 1 : (blocks > 0x7FFFFFFF ? 0x7FFFFFFF : blocks);
}

}  // namespace

cudaError_t launch_count_bits(const RasterBatch &b, const Plane &p, int sign, int *flags,
                              const DeviceCaps &caps, cudaStream_t s) {
    const int wpr = (p.width + 31) / 32;
    if (b.n <= 0 || wpr == 0 || p.height == 0) return cudaSuccess;
    // two words (8 bytes) per thread and member where every row start is 8-byte aligned
    const bool wide = wpr >= 2 && reinterpret_cast<uintptr_t>(b.base) % 8 == 0 && b.row_pitch % 8 == 0 &&
                      b.member_stride % 8 == 0;
    const int per_row = wide ? (wpr + 1) / 2 : wpr;
    const int64_t units = (int64_t)per_row * p.height;
    // member slabs of at most 255 (eight counter levels); more only to fill
    // about four waves of four 256-thread CTAs per SM, since every slab pays
    // the bit-sliced epilogue and its atomics
    const int64_t target_units = 4ll * caps.num_sms * 4 * kThreads;
    int64_t slabs = (b.n + kPackedLimit - 1) / kPackedLimit;
    const int64_t want = std::min<int64_t>((target_units + units - 1) / units, (b.n + 31) / 32);
    slabs = std::max<int64_t>(std::max<int64_t>(slabs, want), 1);
    const int slab = (int)((b.n + slabs - 1) / slabs);
    slabs = (b.n + slab - 1) / slab;
    const unsigned grid = (unsigned)blocks_for(units * slabs);
    if (p.count_bits == 16) {
        if (wide)
            count_bits_kernel<uint16_t, 2><<<grid, kThreads, 0, s>>>(b, p, sign, flags, units, per_row, slab, (int)slabs);
        else
            count_bits_kernel<uint16_t, 1><<<grid, kThreads, 0, s>>>(b, p, sign, flags, units, per_row, slab, (int)slabs);
    } else {
        if (wide)
            count_bits_kernel<uint32_t, 2><<<grid, kThreads, 0, s>>>(b, p, sign, flags, units, per_row, slab, (int)slabs);
        else
            count_bits_kernel<uint32_t, 1><<<grid, kThreads, 0, s>>>(b, p, sign, flags, units, per_row, slab, (int)slabs);
    }
    return cudaGetLastError();
}

}  // namespace cpt
