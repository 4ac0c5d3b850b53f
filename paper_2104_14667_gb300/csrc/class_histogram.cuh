// class_histogram.cuh -- the class histogram of a render (Fig. 1 caption:
// the frequency of the overlap classes), counted by warps in shared memory
// while they classify: the counters every warp keeps, how its lanes add to
// them, and how the warp folds them into totals and hands those on.
#pragma once

#include <stdint.h>

namespace cpt {

// A warp's slice (kHistWarpBytes): kHistRows rows of byte counters, one per
// class, four to a 32-bit word, then 256 32-bit totals.  Every
// kHistLanesPerRow lanes share a row and add to it with shared atomics whose
// result they never wait for; lanes of different rows never touch one word.
// Four neighbouring pixels of one class are added at once.  Row r's 64 words
// are stored with the word index XORed with r, so that one class of all rows
// lies in different banks.  A byte gains at most 16 per item from each of the
// kHistLanesPerRow lanes of its row (one group of 16 pixels per lane), so
// after kHistFoldItems items it is still below 256: the warp
// then folds the bytes into the totals (hist_fold; lane L owns classes
// 4L..4L+3 and 128+4L..128+4L+3, stored at [class slot][lane] so that the
// lanes' accesses never share a bank).  The totals go to the 64-bit
// histogram in global memory per warp (hist_emit) or per block
// (hist_emit_block).
constexpr int kHistLanesPerRow = 2;
constexpr int kHistRows = 32 / kHistLanesPerRow;
constexpr int kHistCounterBytes = kHistRows * 256;
constexpr int kHistWarpBytes = kHistCounterBytes + 256 * 4;   // counters, then the totals
constexpr int kHistFoldItems = 255 / (16 * kHistLanesPerRow);

// row: the lane's row of 256 counter bytes; key: the row index << 2, which
// XORs the word index (class >> 2) with the row index
__device__ __forceinline__ void hist_add(uint8_t *row, uint32_t key, uint32_t cls, uint32_t n) {
    atomicAdd(reinterpret_cast<uint32_t *>(row + ((cls ^ key) & 0xFCu)), n << ((cls & 3u) << 3));
}

// Four pixels' classes: one add when they agree.
__device__ __forceinline__ void hist_count_quarter(uint8_t *row, uint32_t key, uint32_t b0, uint32_t b1, uint32_t b2,
                                                   uint32_t b3) {
    if (b0 == b1 && b1 == b2 && b2 == b3) {
        hist_add(row, key, b0, 4u);
    } else {
        hist_add(row, key, b0, 1u);
        hist_add(row, key, b1, 1u);
        hist_add(row, key, b2, 1u);
        hist_add(row, key, b3, 1u);
    }
}

__device__ __forceinline__ void hist_fold(uint8_t *cnt, uint32_t *tot, int lane) {
    __syncwarp();
    uint32_t *w = reinterpret_cast<uint32_t *>(cnt);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t k = (uint32_t)lane + 32u * h;   // the word of classes 4k..4k+3
        uint32_t lo = 0, hi = 0;                      // bytes 0, 2 and 1, 3 as 16-bit sums
#pragma unroll 8
        for (int r = 0; r < kHistRows; ++r) {
            uint32_t *at = w + r * 64 + (k ^ (uint32_t)r);
            const uint32_t v = *at;
            *at = 0u;
            lo += v & 0x00FF00FFu;
            hi += (v >> 8) & 0x00FF00FFu;
        }
        tot[(4 * h + 0) * 32 + lane] += lo & 0xFFFFu;
        tot[(4 * h + 1) * 32 + lane] += hi & 0xFFFFu;
        tot[(4 * h + 2) * 32 + lane] += lo >> 16;
        tot[(4 * h + 3) * 32 + lane] += hi >> 16;
    }
    __syncwarp();
}

__device__ __forceinline__ void hist_emit(uint32_t *tot, unsigned long long *hist, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t &t = tot[(4 * h + j) * 32 + lane];
            if (t) atomicAdd(hist + 4 * lane + 128 * h + j, (unsigned long long)t);
            t = 0u;
        }
}

// Adds the totals of every warp of the block (each warp's kHistWarpBytes
// slice of `hist`) into the 64-bit histogram: thread t sums class t over the
// warps.  Call after every warp's last hist_fold and a __syncthreads; needs
// at least 256 threads.
__device__ __forceinline__ void hist_emit_block(const uint8_t *hist, int n_warps, unsigned long long *out) {
    const int cls = threadIdx.x;
    if (cls >= 256) return;
    const int slot = (cls >> 7) * 4 + (cls & 3), lane = (cls & 127) >> 2;
    uint32_t t = 0;
    for (int w = 0; w < n_warps; ++w)
        t += reinterpret_cast<const uint32_t *>(hist + w * kHistWarpBytes + kHistCounterBytes)[slot * 32 + lane];
    if (t) atomicAdd(out + cls, (unsigned long long)t);
}

}  // namespace cpt
