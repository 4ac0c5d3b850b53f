// engine.cu -- the batched composite engine of include/composite_engine.h.
//
// A submit turns every op (add/remove a member set to one plane) into work
// items (op, member slab, chunk of 16-pixel groups), numbered op after op,
// slab after slab, chunk after chunk.  One persistent launch of
// num_SMs x ctas_per_sm CTAs runs warps that each pull item numbers from a
// device counter; the op owning an item is found by binary search over the
// ops' first items.  Each lane folds its groups of one slab's members into
// packed byte counters (member i of the op read at base + idx(i) * stride,
// the slab's indices staged in the warp's shared memory) and adds the counts
// into the op's plane (uint32, or uint16 for a 16-bit plane): with L2
// atomics, or with a plain read-modify-write when the op is alone on its
// plane and has a single slab.  The render launch deals warp-level (plane,
// chunk) items round robin to its warps.  Consecutive
// items are neighbouring chunks of the same slab, so concurrently running
// warps read neighbouring bytes of the same members.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "composite_engine.h"
#include "bit_count.cuh"
#include "internal.cuh"
#include "overlap_class.cuh"
#include "class_histogram.cuh"

namespace {

using cpt::DeviceCaps;
using cpt::Lut;

constexpr int kThreads = 256;          // threads per CTA = 16-pixel groups per tile
constexpr int kMaxPlanes = 1 << 16;
constexpr int kMaxSlab = 255;          // packed byte counters
constexpr int kUploadRing = 64;        // descriptor uploads in flight before the host waits

struct OpDesc {
    const uint8_t *base;
    const int32_t *index;
    uint32_t *plane;
    int64_t stride;
    int64_t plane_pitch;   // elements
    int64_t item_start;
    int32_t pitch;
    int32_t n;
    int32_t width;
    int32_t height;
    int32_t groups_per_row;
    int32_t tiles;
    int32_t slab;
    int32_t sign;
    int32_t plane_id;
    int32_t groups_per_thread;   // groups per lane per item (short slabs take several)
    int32_t exclusive;           // the only op on its plane, one slab: plain read-modify-write
    int32_t bits;                // bit-packed masks: a group is a 32-pixel word
    int32_t words_per_row;       // bits: ceil(width / 32)
    int32_t u16;                 // the plane holds uint16 counts (else uint32)
    int32_t pad;
};

// One render op.  The plane's pitch is groups_per_row x 16 pixels, so group g of the plane holds
// the counts of pixels 16 g .. 16 g + 15 in memory order.
struct RenderDesc {
    const uint32_t *plane;
    void *counts_out;
    uint8_t *bucket_out;
    uint32_t *rgba_out;
    int64_t item_start;
    int32_t width;
    int32_t height;
    int32_t groups_per_row;
    int32_t vec;           // 16-byte stores allowed
    int32_t u16;           // the plane holds uint16 counts (else uint32)
    int32_t dense;         // width == plane pitch: group g's outputs start at 16 g
    cpt::ClassDivisor div; // floor(255 c / n_members) by multiplication
    unsigned long long *hist;   // 256 class counts, zeroed before the launch, or NULL
};

// One plane of a batched clear: its bytes as 16-byte words, in items of
// 32 lanes x kClearWords words.
struct ClearDesc {
    uint4 *data;
    int64_t words;
    int64_t item_start;
    int32_t plane_id;
    int32_t pad;
};

constexpr int kSmemStarts = 2048;      // ops whose first items fit in shared memory
constexpr int kClearWords = 8;         // 16-byte words per lane per clear item
constexpr int kClearCtasPerSm = 4;
constexpr int kRenderCtasPerSm = 4;    // render launch: CTAs per SM, grid-stride over items
constexpr int kRenderHistCtasPerSm = 4;   // with histograms: 32 KB of counters per CTA

template <typename Desc>
__device__ __forceinline__ int find_desc(const Desc *d, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].item_start <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The op owning `item`: binary search over the first items, in shared memory
// when the op list is short enough, else over the descriptors themselves.
template <typename Desc>
__device__ __forceinline__ int find_op(const Desc *d, int n, const uint32_t *starts, uint32_t item) {
    if (n > kSmemStarts) return find_desc(d, n, item);
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// First item of op i (from shared memory when the list fits there).
template <typename Desc>
__device__ __forceinline__ uint32_t op_start(const Desc *d, int n, const uint32_t *starts, int i) {
    return n <= kSmemStarts ? starts[i] : (uint32_t)d[i].item_start;
}

template <typename Desc>
__device__ __forceinline__ void load_starts(const Desc *d, int n, uint32_t *starts) {
    if (n <= kSmemStarts)
        for (int i = threadIdx.x; i < n; i += blockDim.x) starts[i] = (uint32_t)d[i].item_start;
}

// One warp item: (op, member slab, chunk of 32 x groups_per_thread groups).
// The slab's member indices are staged in the warp's slice of shared memory.
__device__ __forceinline__ void process_item(const OpDesc &op, uint32_t item, int lane, int32_t *index,
                                             int *flags) {
    const uint32_t local = item - (uint32_t)op.item_start;
    const int sl = (int)(local / (uint32_t)op.tiles);
    const int chunk = (int)(local - (uint32_t)sl * op.tiles);
    const int m0 = sl * op.slab;
    const int cnt = min(op.n - m0, op.slab);
    const bool gather = op.index != nullptr;
    if (gather) {
        for (int i = lane; i < cnt; i += 32) index[i] = op.index[m0 + i];
        __syncwarp();
    }
    const int64_t groups = (int64_t)op.groups_per_row * op.height;
    const int gpt = op.groups_per_thread;
    for (int j = 0; j < gpt; ++j) {
        const int64_t g = ((int64_t)chunk * gpt + j) * 32 + lane;
        if (g >= groups) break;
        const int y = (int)(g / op.groups_per_row);
        const int x0 = (int)(g - (int64_t)y * op.groups_per_row) * 16;
        const int valid = min(16, op.width - x0);
        const uint8_t *row = op.base + (int64_t)y * op.pitch + x0;
        const int64_t stride = op.stride;
        uint32_t k[4] = {0u, 0u, 0u, 0u};
        if (valid == 16 && !gather) {
            const uint8_t *q = row + (int64_t)m0 * stride;
#pragma unroll 8
            for (int i = 0; i < cnt; ++i) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(q));
                q += stride;
                k[0] += cpt::nonzero_bytes(v.x);
                k[1] += cpt::nonzero_bytes(v.y);
                k[2] += cpt::nonzero_bytes(v.z);
                k[3] += cpt::nonzero_bytes(v.w);
            }
        } else if (valid == 16) {
#pragma unroll 8
            for (int i = 0; i < cnt; ++i) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(row + (int64_t)index[i] * stride));
                k[0] += cpt::nonzero_bytes(v.x);
                k[1] += cpt::nonzero_bytes(v.y);
                k[2] += cpt::nonzero_bytes(v.z);
                k[3] += cpt::nonzero_bytes(v.w);
            }
        } else {
            for (int i = 0; i < cnt; ++i) {
                const int64_t mi = gather ? index[i] : (int64_t)(m0 + i);
                const uint8_t *q = row + mi * stride;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if (jj < valid) k[jj / 4] += (uint32_t)(q[jj] != 0) << (8 * (jj % 4));
            }
        }
        uint32_t wide[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) wide[jj] = 0;
        cpt::widen16(wide, k[0], k[1], k[2], k[3]);
        const int64_t at = (int64_t)y * op.plane_pitch + x0;
        if (op.u16) {
            uint16_t *dst = reinterpret_cast<uint16_t *>(op.plane) + at;
            if (op.exclusive)
                cpt::apply_count_group<uint16_t>(dst, valid, wide, op.sign, flags + op.plane_id);
            else
                cpt::atomic_count_group<uint16_t>(dst, wide, op.sign, flags + op.plane_id);
        } else {
            uint32_t *dst = op.plane + at;
            if (op.exclusive)
                cpt::apply_count_group<uint32_t>(dst, valid, wide, op.sign, flags + op.plane_id);
            else
                cpt::atomic_count_group<uint32_t>(dst, wide, op.sign, flags + op.plane_id);
        }
    }
    if (gather) __syncwarp();
}

// The same for bit-packed masks: a lane owns 32-pixel words and keeps their
// counts in carry-save accumulators (BitCounter), 16 members per step.
__device__ __forceinline__ void process_bits_item(const OpDesc &op, uint32_t item, int lane, int32_t *index,
                                                  int *flags) {
    const uint32_t local = item - (uint32_t)op.item_start;
    const int sl = (int)(local / (uint32_t)op.tiles);
    const int chunk = (int)(local - (uint32_t)sl * op.tiles);
    const int m0 = sl * op.slab;
    const int cnt = min(op.n - m0, op.slab);
    const bool gather = op.index != nullptr;
    if (gather) {
        for (int i = lane; i < cnt; i += 32) index[i] = op.index[m0 + i];
        __syncwarp();
    }
    const int64_t words = (int64_t)op.words_per_row * op.height;
    const int gpt = op.groups_per_thread;
    const int64_t stride = op.stride;
    for (int j = 0; j < gpt; ++j) {
        const int64_t g = ((int64_t)chunk * gpt + j) * 32 + lane;
        if (g >= words) break;
        const int y = (int)(g / op.words_per_row);
        const int gx = (int)(g - (int64_t)y * op.words_per_row);
        const int x0 = gx * 32;
        const int valid = min(32, op.width - x0);
        const int nbytes = (valid + 7) / 8;
        const uint32_t keep = valid == 32 ? 0xFFFFFFFFu : ((1u << valid) - 1u);
        const uint8_t *row = op.base + (int64_t)y * op.pitch + gx * 4;
        cpt::BitCounter acc;
        for (int i = 0; i < cnt; i += 16) {
            const int take = min(16, cnt - i);
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint32_t v = 0;
                if (k < take) {
                    const int64_t mi = gather ? index[i + k] : (int64_t)(m0 + i + k);
                    const uint8_t *q = row + mi * stride;
                    if (valid == 32) {
                        v = __ldcs(reinterpret_cast<const uint32_t *>(q));
                    } else {
                        for (int b = 0; b < nbytes; ++b) v |= (uint32_t)q[b] << (8 * b);
                        v &= keep;
                    }
                }
                w[k] = v;
            }
            cpt::bitcount_add16(acc, w);
        }
        const int64_t at = (int64_t)y * op.plane_pitch + x0;
        uint32_t pairs[16];
        cpt::bitcount_pairs(acc, pairs);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = min(16, valid - 16 * h);
            if (v <= 0) break;
            if (op.u16) {
                uint16_t *dst = reinterpret_cast<uint16_t *>(op.plane) + at + 16 * h;
                if (op.exclusive)
                    cpt::apply_pair_group<uint16_t>(dst, v, pairs + 8 * h, op.sign, flags + op.plane_id);
                else
                    cpt::atomic_pair_group<uint16_t>(dst, pairs + 8 * h, op.sign, flags + op.plane_id);
            } else {
                uint32_t *dst = op.plane + at + 16 * h;
                if (op.exclusive)
                    cpt::apply_pair_group<uint32_t>(dst, v, pairs + 8 * h, op.sign, flags + op.plane_id);
                else
                    cpt::atomic_pair_group<uint32_t>(dst, pairs + 8 * h, op.sign, flags + op.plane_id);
            }
        }
    }
    if (gather) __syncwarp();
}

__device__ __forceinline__ void run_item(const OpDesc &op, uint32_t item, int lane, int32_t *index, int *flags) {
    if (op.bits)
        process_bits_item(op, item, lane, index, flags);
    else
        process_item(op, item, lane, index, flags);
}

// Persistent schedule: warps claim items from the counter one ahead (lane 0
// asks for the next while the warp works on the current one), so warps
// never wait for one another and uneven items balance across the GPU.
// Two register budgets: launched with four or five CTAs per SM, 48 registers
// (a few spill; four such CTAs still leave a quarter of the register file to
// a kernel on another stream); with three or fewer, 64 and no spills (three
// such CTAs leave the same quarter).
template <int kCtasPerSm>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
engine_accumulate_kernel(const OpDesc *ops, int n_ops, uint32_t n_items, uint32_t *counter, int *flags) {
    __shared__ int32_t s_index[kThreads / 32][kMaxSlab + 1];
    __shared__ uint32_t s_starts[kSmemStarts];
    load_starts(ops, n_ops, s_starts);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int32_t *index = s_index[threadIdx.x >> 5];
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(counter, 1u);
    next = __shfl_sync(0xFFFFFFFFu, next, 0);
    while (next < n_items) {
        const uint32_t item = next;
        if (lane == 0) next = atomicAdd(counter, 1u);
        run_item(ops[find_op(ops, n_ops, s_starts, item)], item, lane, index, flags);
        next = __shfl_sync(0xFFFFFFFFu, next, 0);
    }
}

// Grid schedule: one launch of ceil(items / 8) CTAs, warp w of CTA b takes
// item 8b + w; the hardware block scheduler balances the CTAs.
__global__ void __launch_bounds__(kThreads)
engine_accumulate_grid_kernel(const OpDesc *ops, int n_ops, uint32_t n_items, int *flags) {
    __shared__ int32_t s_index[kThreads / 32][kMaxSlab + 1];
    const int lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (item >= n_items) return;
    run_item(ops[find_desc(ops, n_ops, item)], item, lane, s_index[threadIdx.x >> 5], flags);
}

// Clear of many planes in one launch (counts to zero, the planes' underflow
// flags too): warp-level items (plane, 32 x kClearWords words) dealt round
// robin.  A CUDA graph that clears its planes this way has one node for all
// of them instead of two memset nodes per plane, which run one after another.
__global__ void __launch_bounds__(kThreads)
engine_clear_kernel(const ClearDesc *ops, int n_ops, uint32_t n_items, int *flags) {
    __shared__ uint32_t s_starts[kSmemStarts];
    load_starts(ops, n_ops, s_starts);
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n_ops; i += blockDim.x)
            if (ops[i].plane_id >= 0) flags[ops[i].plane_id] = 0;   // -1: a histogram, no flag
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (kThreads / 32);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t item = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); item < n_items; item += warps) {
        const ClearDesc op = ops[find_op(ops, n_ops, s_starts, item)];   // by value: the stores may alias
        const int64_t w0 = (int64_t)(item - (uint32_t)op.item_start) * (32 * kClearWords) + lane;
#pragma unroll
        for (int k = 0; k < kClearWords; ++k) {
            const int64_t wi = w0 + 32 * k;
            if (wi < op.words) op.data[wi] = zero;
        }
    }
}

// Classify and store one lane's group of 16 pixels (counts c, as loaded in
// v); row: the lane's histogram counters, or NULL.
template <bool kHist, bool kNarrow>
__device__ __forceinline__ void render_group(const RenderDesc &op, const uint4 (&v)[4], const uint32_t (&c)[16], int valid,
                                             int64_t out, int pieces, const uint32_t *table, uint8_t *row,
                                             uint32_t key) {
    auto cls = [&](uint32_t x) {
        return kNarrow ? cpt::overlap_class_narrow(x, op.div) : cpt::overlap_class(x, op.div);
    };
    if (op.vec && valid == 16) {
        if (op.counts_out) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < pieces)   // 'pieces' bytes per count
                    reinterpret_cast<uint4 *>(static_cast<uint8_t *>(op.counts_out) + out * pieces)[q] = v[q];
        }
        // a quarter of the group at a time: classes, their colours, the packed classes
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t b0 = cls(c[4 * q]), b1 = cls(c[4 * q + 1]);
            const uint32_t b2 = cls(c[4 * q + 2]), b3 = cls(c[4 * q + 3]);
            w[q] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
            if (kHist && row) cpt::hist_count_quarter(row, key, b0, b1, b2, b3);
            if (op.rgba_out)
                reinterpret_cast<uint4 *>(op.rgba_out + out)[q] = make_uint4(table[b0], table[b1], table[b2], table[b3]);
        }
        if (op.bucket_out) *reinterpret_cast<uint4 *>(op.bucket_out + out) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < valid) {
                const uint32_t b = cls(c[j]);
                if (op.counts_out) {
                    if (op.u16)
                        reinterpret_cast<uint16_t *>(op.counts_out)[out + j] = (uint16_t)c[j];
                    else
                        reinterpret_cast<uint32_t *>(op.counts_out)[out + j] = c[j];
                }
                if (op.bucket_out) op.bucket_out[out + j] = (uint8_t)b;
                if (op.rgba_out) op.rgba_out[out + j] = table[b];
                if (kHist && row) cpt::hist_add(row, key, b, 1u);
            }
        }
    }
}

// Render: warp-level items (render op, 32 16-pixel groups of its plane, one
// per lane) dealt round robin to every warp of the launch -- items are all
// the same size, so no counter is needed.  With histograms (kHist; 5 KB of
// dynamic shared memory per warp) every CTA takes one contiguous range of
// items instead, so that a warp's items span one or two ops and its totals
// go to global memory once or twice.  A plane's pitch is a whole number of
// groups, so group g holds the counts of pixels 16 g .. 16 g + 15 in memory
// order; when the outputs are dense at that pitch too (width a multiple of
// 16) they start at 16 g as well and no row division is needed.
template <bool kHist>
__global__ void __launch_bounds__(kThreads, kHist ? kRenderHistCtasPerSm : kRenderCtasPerSm)
engine_render_kernel(const RenderDesc *__restrict__ ops, int n_ops, uint32_t n_items, Lut lut) {
    __shared__ uint32_t table[256];
    __shared__ uint32_t s_starts[kSmemStarts];
    extern __shared__ __align__(16) uint8_t s_hist[];
    const int lane = threadIdx.x & 31;
    uint8_t *cnt = s_hist + (kHist ? (threadIdx.x >> 5) * cpt::kHistWarpBytes : 0);
    uint8_t *row = cnt + (kHist ? (lane / cpt::kHistLanesPerRow) * 256 : 0);
    const uint32_t key = (uint32_t)(lane / cpt::kHistLanesPerRow) << 2;
    for (int i = threadIdx.x; i < 256; i += kThreads) table[i] = lut.rgba[i];
    if (kHist)
        for (int i = lane; i < cpt::kHistWarpBytes / 16; i += 32) reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0, 0, 0, 0);
    load_starts(ops, n_ops, s_starts);
    __syncthreads();
    unsigned long long *hist_at = nullptr;   // the histogram the warp's counts belong to
    uint32_t *tot = reinterpret_cast<uint32_t *>(cnt + cpt::kHistCounterBytes);
    int since_fold = 0;
    uint32_t first, last, stride;
    if (kHist) {
        const uint32_t per = (n_items + gridDim.x - 1) / gridDim.x;
        first = blockIdx.x * per + (threadIdx.x >> 5);
        last = min(n_items, (blockIdx.x + 1) * per);
        stride = kThreads / 32;
    } else {
        first = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
        last = n_items;
        stride = gridDim.x * (kThreads / 32);
    }
    // the op of the warp's current item: without histograms the next item's
    // op is looked up while the current item's counts are on their way; with
    // them (contiguous items, few op changes) only when an item passes the
    // current op's end
    int idx = first < last ? find_op(ops, n_ops, s_starts, first) : 0;
    uint32_t op_end = kHist && first < last && idx + 1 < n_ops ? op_start(ops, n_ops, s_starts, idx + 1) : n_items;
    for (uint32_t item = first; item < last; item += stride) {
        if (kHist && item >= op_end) {
            idx = find_op(ops, n_ops, s_starts, item);
            op_end = idx + 1 < n_ops ? op_start(ops, n_ops, s_starts, idx + 1) : n_items;
        }
        // restrict: the outputs are plain pointers, and without it every
        // store would force the descriptor's fields to be reloaded
        const RenderDesc &op = ops[idx];
        if (kHist) {
            if (op.hist != hist_at) {
                if (hist_at) {
                    cpt::hist_fold(cnt, tot, lane);
                    cpt::hist_emit(tot, hist_at, lane);
                }
                hist_at = op.hist;
                since_fold = 0;
            } else if (hist_at && since_fold == cpt::kHistFoldItems) {
                cpt::hist_fold(cnt, tot, lane);
                since_fold = 0;
            }
            ++since_fold;
        }
        const int64_t groups = (int64_t)op.groups_per_row * op.height;
        const int64_t g = (int64_t)(item - (uint32_t)op.item_start) * 32 + lane;
        const int pieces = op.u16 ? 2 : 4;   // 16-byte pieces of a group's counts
        const uint4 *src = reinterpret_cast<const uint4 *>(op.plane) + g * pieces;
        uint4 v[4];
        if (g < groups) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < pieces) v[q] = src[q];
        }
        const uint32_t next = item + stride;
        if (!kHist && next < last && idx + 1 < n_ops && next >= op_start(ops, n_ops, s_starts, idx + 1))
            idx = find_op(ops, n_ops, s_starts, next);
        if (g >= groups) continue;
        uint32_t c[16];
        if (op.u16) {
            const uint32_t w[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[2 * q] = w[q] & 0xFFFFu;
                c[2 * q + 1] = w[q] >> 16;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c[4 * q] = v[q].x; c[4 * q + 1] = v[q].y; c[4 * q + 2] = v[q].z; c[4 * q + 3] = v[q].w;
            }
        }
        int valid = 16;
        int64_t out = g * 16;
        if (!op.dense) {
            const int y = (int)(g / op.groups_per_row);
            const int x0 = (int)(g - (int64_t)y * op.groups_per_row) * 16;
            valid = min(16, op.width - x0);
            out = (int64_t)y * op.width + x0;
        }
        // one multiply-high per class for N < 2^16 (every 16-bit plane), the
        // general division otherwise: a branch per item, so that each
        // specialisation keeps only its own divisor fields live
        if (op.div.narrow)
            render_group<kHist, true>(op, v, c, valid, out, pieces, table, hist_at ? row : nullptr, key);
        else
            render_group<kHist, false>(op, v, c, valid, out, pieces, table, hist_at ? row : nullptr, key);
    }
    if (kHist && hist_at) {
        cpt::hist_fold(cnt, tot, lane);
        cpt::hist_emit(tot, hist_at, lane);
    }
}

struct PlaneRec {
    int32_t width = 0, height = 0;
    int64_t pitch_px = 0;
    uint32_t *data = nullptr;    // uint16 counts when count_bits is 16
    int32_t count_bits = 32;
    int64_t n = 0;
    bool alive = false;
    bool poisoned = false;       // a submit failed after its launch may have begun

    size_t bytes() const { return (size_t)pitch_px * height * (count_bits / 8); }
    int64_t max_members() const { return count_bits == 16 ? 0xFFFFll : 0xFFFFFFFFll; }
};

// A device buffer of descriptors with its pinned host mirror.
struct Upload {
    void *d = nullptr;
    void *h = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;      // the upload out of h finished (upload stream)
    cudaEvent_t consumed = nullptr;  // the launch that read d finished (engine stream)
    bool used = false;
};

// A staging buffer for ops on pinned host members.
struct StageSlot {
    uint8_t *d = nullptr;
    cudaEvent_t ready = nullptr;     // its upload finished (copy stream)
    cudaEvent_t consumed = nullptr;  // the launch that read it finished (engine stream)
    bool used = false;
};

constexpr int64_t kDefaultStageBytes = 256ll << 20;
constexpr int kDefaultItemMemberGroups = 512;

thread_local std::string g_engine_error;

}  // namespace

struct composite_engine {
    composite_engine_config cfg{};
    int device = 0;
    DeviceCaps caps{};
    cudaStream_t stream = nullptr;
    std::vector<PlaneRec> planes;
    int *d_flags = nullptr;
    int *h_flags = nullptr;
    uint32_t *d_counter = nullptr;
    Upload up_ops[kUploadRing], up_render[kUploadRing];
    int up_i = 0, rup_i = 0;
    cudaEvent_t done_ev = nullptr;
    Lut default_lut{};
    // captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    void *graph_ops = nullptr;
    void *graph_rops = nullptr;
    void *graph_clears = nullptr;
    uint32_t *graph_counters = nullptr;
    std::vector<std::pair<int32_t, int64_t>> graph_n;   // plane -> N after a replay
    std::vector<int32_t> graph_planes;                  // every plane the graph touches
    cudaStream_t capture_stream = nullptr;              // private stream for graph capture
    // ops on pinned host members
    std::vector<StageSlot> stage;
    int64_t stage_bytes = 0;       // bytes per allocated staging buffer
    uint64_t stage_next = 0;
    cudaStream_t copy = nullptr;   // their uploads
    cudaEvent_t caller_ready = nullptr;
    std::string err;
};

namespace {

int efail(composite_engine *e, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (e)
        e->err = buf;
    else
        g_engine_error = buf;
    return code;
}

int ecuda(composite_engine *e, cudaError_t err, const char *what) {
    return efail(e, err == cudaErrorMemoryAllocation ? CPT_ENOMEM : CPT_ECUDA, "%s: %s", what,
                 cudaGetErrorString(err));
}

#define ECK(e, call)                                      \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ecuda(e, e_, #call); \
    } while (0)

int64_t etimeout(const composite_engine *e) { return e->cfg.wait_timeout_ms > 0 ? e->cfg.wait_timeout_ms : 10000; }

int ewait(composite_engine *e, cudaEvent_t ev) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(etimeout(e));
    for (unsigned spin = 0;; ++spin) {
        const cudaError_t r = cudaEventQuery(ev);
        if (r == cudaSuccess) return CPT_OK;
        if (r != cudaErrorNotReady) return ecuda(e, r, "cudaEventQuery");
        if (std::chrono::steady_clock::now() > deadline)
            return efail(e, CPT_ETIMEOUT, "wait exceeded %lld ms", (long long)etimeout(e));
        if (spin < 200)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int drain(composite_engine *e) {
    ECK(e, cudaEventRecord(e->done_ev, e->stream));
    return ewait(e, e->done_ev);
}

Lut make_lut(const uint8_t *rgba) {
    Lut l;
    for (int b = 0; b < 256; ++b) {
        const uint32_t r = rgba ? rgba[4 * b] : 255u - b, g = rgba ? rgba[4 * b + 1] : 255u - b;
        const uint32_t bl = rgba ? rgba[4 * b + 2] : 255u, a = rgba ? rgba[4 * b + 3] : 255u;
        l.rgba[b] = r | (g << 8) | (bl << 16) | (a << 24);
    }
    return l;
}

// Copies `bytes` of descriptors into the next slot of the upload ring
// and queues their upload, on the upload stream when the engine has one (so
// that small uploads follow the caller's own uploads in order instead of
// waiting behind them on a copy engine); returns the slot.  The caller
// records slot->consumed on the engine stream after the launch that reads it.
int upload(composite_engine *e, Upload *ring, int *idx, const void *src, size_t bytes, Upload **slot,
           cudaStream_t on = nullptr) {
    Upload &u = ring[*idx];
    *idx = (*idx + 1) % kUploadRing;
    if (u.used) {
        int rc = ewait(e, u.done);
        if (rc) return rc;
    }
    cudaStream_t us = on ? on : e->cfg.upload_stream ? static_cast<cudaStream_t>(e->cfg.upload_stream) : e->stream;
    if (u.cap < bytes) {
        if (u.d) cudaFree(u.d);
        if (u.h) cudaFreeHost(u.h);
        u.d = u.h = nullptr;
        u.cap = 0;
        const size_t cap = std::max<size_t>(bytes, 4096);
        ECK(e, cudaMalloc(&u.d, cap));
        ECK(e, cudaHostAlloc(&u.h, cap, cudaHostAllocDefault));
        u.cap = cap;
    }
    memcpy(u.h, src, bytes);
    if (us != e->stream && u.used) ECK(e, cudaStreamWaitEvent(us, u.consumed, 0));
    ECK(e, cudaMemcpyAsync(u.d, u.h, bytes, cudaMemcpyHostToDevice, us));
    ECK(e, cudaEventRecord(u.done, us));
    if (us != e->stream) ECK(e, cudaStreamWaitEvent(e->stream, u.done, 0));
    u.used = true;
    *slot = &u;
    return CPT_OK;
}

// Memory kind of an op's members as seen from `device`: 1 = pinned host,
// 0 = device (this device's, or managed), -1 = neither (pageable host, or
// another GPU's memory, which a kernel here cannot be assumed to reach).
int member_kind(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type == cudaMemoryTypeManaged) return 0;
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? 0 : -1;
    return a.type == cudaMemoryTypeHost ? 1 : -1;
}

// Whether a kernel on `device` may read or write p in place: this device's
// memory, managed memory, or pinned host memory mapped for the device.
bool device_reachable(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type == cudaMemoryTypeDevice) return a.device == device;
    return a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
}

bool plane_ok(const composite_engine *e, int32_t p) {
    return p >= 0 && p < (int32_t)e->planes.size() && e->planes[p].alive;
}

// Validates ops and builds their descriptors.  n_after holds, per plane
// touched, the member count after the ops starting from `start` counts.
int plan_ops(composite_engine *e, const composite_op *ops, int32_t n_ops, std::vector<OpDesc> *descs,
             int64_t *n_items, std::vector<std::pair<int32_t, int64_t>> *n_after, bool from_zero,
             bool check_n = true) {
    if (n_ops < 0 || (n_ops > 0 && !ops)) return efail(e, CPT_EINVAL, "bad op list");
    descs->clear();
    n_after->clear();
    std::vector<int64_t> n(e->planes.size(), -1);
    int64_t items = 0;
    const int slab = e->cfg.slab_members;
    for (int32_t i = 0; i < n_ops; ++i) {
        const composite_op &o = ops[i];
        if (!plane_ok(e, o.plane)) return efail(e, CPT_EINVAL, "op %d: no plane %d", i, o.plane);
        if (o.sign != 1 && o.sign != -1) return efail(e, CPT_EINVAL, "op %d: sign must be +1 or -1", i);
        if (o.n_members < 0) return efail(e, CPT_EINVAL, "op %d: n_members < 0", i);
        const PlaneRec &p = e->planes[o.plane];
        if (n[o.plane] < 0) n[o.plane] = from_zero ? 0 : p.n;
        n[o.plane] += (int64_t)o.sign * o.n_members;
        if (check_n && n[o.plane] < 0)
            return efail(e, CPT_EINVAL, "op %d: plane %d would hold fewer than 0 members", i, o.plane);
        if (check_n && n[o.plane] > p.max_members())
            return efail(e, CPT_EINVAL, "op %d: plane %d would exceed %lld members (%d-bit counts)", i, o.plane,
                         (long long)p.max_members(), p.count_bits);
        if (o.n_members == 0) continue;
        if (!o.members) return efail(e, CPT_EINVAL, "op %d: members is NULL", i);
        if ((reinterpret_cast<uintptr_t>(o.members) % 16) || (o.row_pitch_bytes % 16) || (o.member_stride_bytes % 16))
            return efail(e, CPT_EINVAL, "op %d: members, row pitch and stride must be 16-byte aligned", i);
        if (o.mask_format != CPT_MASK_BYTES && o.mask_format != CPT_MASK_BITS)
            return efail(e, CPT_EINVAL, "op %d: mask_format %d out of range", i, o.mask_format);
        const bool bits = o.mask_format == CPT_MASK_BITS;
        const int64_t row_bytes = bits ? ((int64_t)p.width + 7) / 8 : p.width;
        if (o.row_pitch_bytes < row_bytes || o.member_stride_bytes < (int64_t)o.row_pitch_bytes * p.height)
            return efail(e, CPT_EINVAL, "op %d: row pitch or member stride too small", i);
        OpDesc d{};
        d.base = static_cast<const uint8_t *>(o.members);
        d.index = o.member_index;
        d.plane = p.data;
        d.stride = o.member_stride_bytes;
        d.plane_pitch = p.pitch_px;
        d.item_start = items;
        d.pitch = o.row_pitch_bytes;
        d.n = o.n_members;
        d.width = p.width;
        d.height = p.height;
        d.groups_per_row = (int32_t)(p.pitch_px / 16);
        d.bits = bits ? 1 : 0;
        d.u16 = p.count_bits == 16 ? 1 : 0;
        d.words_per_row = (int32_t)(((int64_t)p.width + 31) / 32);
        const int64_t groups = bits ? (int64_t)d.words_per_row * p.height : (int64_t)d.groups_per_row * p.height;
        // a warp item: 32 lanes x groups_per_thread groups, so that a lane
        // streams about item_member_groups member-groups per item whatever
        // the slab length
        const int first_slab = std::min(o.n_members, slab);
        d.groups_per_thread = std::max(1, e->cfg.item_member_groups / first_slab);
        const int64_t per_item = 32ll * d.groups_per_thread;
        d.tiles = (int32_t)((groups + per_item - 1) / per_item);
        d.slab = slab;
        d.sign = o.sign;
        d.plane_id = o.plane;
        d.exclusive = 0;
        const int64_t slabs = (o.n_members + slab - 1) / slab;
        items += slabs * d.tiles;
        descs->push_back(d);
    }
    // An op that is alone on its plane in this submit and has a single slab
    // owns every pixel it touches: no atomics needed.
    std::vector<int> ops_on_plane(e->planes.size(), 0);
    for (const OpDesc &d : *descs) ++ops_on_plane[d.plane_id];
    for (OpDesc &d : *descs) d.exclusive = (ops_on_plane[d.plane_id] == 1 && d.n <= d.slab) ? 1 : 0;
    if (items >= (int64_t)1 << 31) return efail(e, CPT_EINVAL, "too many work items in one submit");
    for (size_t p = 0; p < n.size(); ++p)
        if (n[p] >= 0) n_after->push_back({(int32_t)p, n[p]});
    *n_items = items;
    return CPT_OK;
}

int plan_render(composite_engine *e, const composite_render_op *ops, int32_t n_ops, std::vector<RenderDesc> *descs,
                int64_t *n_items, const std::vector<std::pair<int32_t, int64_t>> *n_override) {
    if (n_ops < 0 || (n_ops > 0 && !ops)) return efail(e, CPT_EINVAL, "bad render list");
    descs->clear();
    int64_t items = 0;
    for (int32_t i = 0; i < n_ops; ++i) {
        const composite_render_op &o = ops[i];
        if (!plane_ok(e, o.plane)) return efail(e, CPT_EINVAL, "render %d: no plane %d", i, o.plane);
        const PlaneRec &p = e->planes[o.plane];
        if ((reinterpret_cast<uintptr_t>(o.counts_out) % (p.count_bits / 8)) || (reinterpret_cast<uintptr_t>(o.rgba_out) % 4))
            return efail(e, CPT_EINVAL, "render %d: counts_out must be aligned to its count type, rgba_out to 4 bytes", i);
        if (reinterpret_cast<uintptr_t>(o.histogram_out) % 16)
            return efail(e, CPT_EINVAL, "render %d: histogram_out must be 16-byte aligned", i);
        const void *outs[4] = {o.counts_out, o.bucket_out, o.rgba_out, o.histogram_out};
        for (const void *q : outs)
            if (q && !device_reachable(q, e->device))
                return efail(e, CPT_EINVAL, "render %d: outputs must be device memory of device %d (or mapped pinned "
                                            "host memory)", i, e->device);
        int64_t n = p.n;
        bool refolded = false;   // a captured graph clears and refolds the plane first
        if (n_override)
            for (const auto &pn : *n_override)
                if (pn.first == o.plane) {
                    n = pn.second;
                    refolded = true;
                }
        if (p.poisoned && !refolded)
            return efail(e, CPT_ESTATE, "render %d: plane %d: an earlier submit failed part-way; clear it", i, o.plane);
        RenderDesc d{};
        d.plane = p.data;
        d.counts_out = o.counts_out;
        d.bucket_out = o.bucket_out;
        d.rgba_out = reinterpret_cast<uint32_t *>(o.rgba_out);
        d.item_start = items;
        d.div = cpt::class_divisor((uint64_t)n);
        d.width = p.width;
        d.height = p.height;
        d.groups_per_row = (int32_t)(p.pitch_px / 16);
        const int64_t groups = (int64_t)d.groups_per_row * p.height;
        const int64_t tiles = (groups + 31) / 32;   // warp items: one 16-pixel group per lane
        const uintptr_t a = reinterpret_cast<uintptr_t>(o.counts_out) | reinterpret_cast<uintptr_t>(o.bucket_out) |
                            reinterpret_cast<uintptr_t>(o.rgba_out);
        d.vec = (p.width % 16 == 0) && (a % 16 == 0);
        d.u16 = p.count_bits == 16 ? 1 : 0;
        d.dense = p.pitch_px == p.width ? 1 : 0;
        d.hist = reinterpret_cast<unsigned long long *>(o.histogram_out);
        items += tiles;
        descs->push_back(d);
    }
    if (items >= (int64_t)1 << 31) return efail(e, CPT_EINVAL, "too many render items");
    *n_items = items;
    return CPT_OK;
}

unsigned persistent_grid(const composite_engine *e, int64_t items) {
    const int64_t cap = (int64_t)e->caps.num_sms * e->cfg.ctas_per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(cap, items));
}

int launch_accumulate(composite_engine *e, const void *d_ops, int n_ops, int64_t n_items, uint32_t *counter) {
    if (e->cfg.schedule == CPT_SCHEDULE_GRID) {
        const int64_t ctas = (n_items + kThreads / 32 - 1) / (kThreads / 32);
        engine_accumulate_grid_kernel<<<(unsigned)ctas, kThreads, 0, e->stream>>>(
            static_cast<const OpDesc *>(d_ops), n_ops, (uint32_t)n_items, e->d_flags);
    } else {
        ECK(e, cudaMemsetAsync(counter, 0, sizeof(uint32_t), e->stream));
        const int64_t warps_needed = (n_items + kThreads / 32 - 1) / (kThreads / 32);
        const unsigned grid = (unsigned)std::min<int64_t>(persistent_grid(e, n_items), warps_needed);
        const OpDesc *ops = static_cast<const OpDesc *>(d_ops);
        if (e->cfg.ctas_per_sm >= 4)
            engine_accumulate_kernel<5><<<grid, kThreads, 0, e->stream>>>(ops, n_ops, (uint32_t)n_items, counter,
                                                                          e->d_flags);
        else
            engine_accumulate_kernel<4><<<grid, kThreads, 0, e->stream>>>(ops, n_ops, (uint32_t)n_items, counter,
                                                                          e->d_flags);
    }
    ECK(e, cudaGetLastError());
    return CPT_OK;
}

// True when some render op asks for a class histogram.
bool any_histogram(const std::vector<RenderDesc> &descs) {
    for (const RenderDesc &d : descs)
        if (d.hist) return true;
    return false;
}

// Clear entries (plane_id -1, no flag) for the histograms of a render, each
// 256 x uint64 = 128 16-byte words, one clear item.
void plan_histogram_clears(const std::vector<RenderDesc> &rdescs, std::vector<ClearDesc> *cdescs, int64_t *citems) {
    for (const RenderDesc &r : rdescs) {
        if (!r.hist) continue;
        ClearDesc d{};
        d.data = reinterpret_cast<uint4 *>(r.hist);
        d.words = 256 * sizeof(uint64_t) / 16;
        d.item_start = *citems;
        d.plane_id = -1;
        *citems += (d.words + 32 * kClearWords - 1) / (32 * kClearWords);
        cdescs->push_back(d);
    }
}

constexpr int kRenderHistSmem = (kThreads / 32) * cpt::kHistWarpBytes;   // dynamic: the warps' counters

// The histogram render's dynamic shared memory (40 KB, beside 9 KB static):
// allowed explicitly, and the largest carveout asked for, so that four such
// CTAs fit on an SM.
int prepare_render_kernels(composite_engine *e) {
    ECK(e, cudaFuncSetAttribute(engine_render_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kRenderHistSmem));
    ECK(e, cudaFuncSetAttribute(engine_render_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
    return CPT_OK;
}

int launch_render(composite_engine *e, const void *d_ops, int n_ops, int64_t n_items, bool hist, const Lut &lut) {
    const int64_t ctas = std::min<int64_t>((int64_t)e->caps.num_sms * (hist ? kRenderHistCtasPerSm : kRenderCtasPerSm),
                                           (n_items + kThreads / 32 - 1) / (kThreads / 32));
    const unsigned grid = (unsigned)std::max<int64_t>(1, ctas);
    if (hist)
        engine_render_kernel<true><<<grid, kThreads, kRenderHistSmem, e->stream>>>(
            static_cast<const RenderDesc *>(d_ops), n_ops, (uint32_t)n_items, lut);
    else
        engine_render_kernel<false><<<grid, kThreads, 0, e->stream>>>(static_cast<const RenderDesc *>(d_ops), n_ops,
                                                                       (uint32_t)n_items, lut);
    ECK(e, cudaGetLastError());
    return CPT_OK;
}

int clear_plane(composite_engine *e, int32_t p) {
    PlaneRec &r = e->planes[p];
    ECK(e, cudaMemsetAsync(r.data, 0, r.bytes(), e->stream));
    ECK(e, cudaMemsetAsync(e->d_flags + p, 0, sizeof(int), e->stream));
    r.n = 0;
    r.poisoned = false;
    return CPT_OK;
}

// Descriptors of one clear launch over the listed planes (each once).
int plan_clears(composite_engine *e, const int32_t *planes, int32_t n, std::vector<ClearDesc> *descs,
                int64_t *n_items) {
    if (n < 0 || (n > 0 && !planes)) return efail(e, CPT_EINVAL, "bad plane list");
    descs->clear();
    std::vector<char> seen(e->planes.size(), 0);
    int64_t items = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t p = planes[i];
        if (!plane_ok(e, p)) return efail(e, CPT_EINVAL, "clear %d: no plane %d", i, p);
        if (seen[p]) continue;
        seen[p] = 1;
        const PlaneRec &r = e->planes[p];
        ClearDesc d{};
        d.data = reinterpret_cast<uint4 *>(r.data);
        d.words = (int64_t)(r.bytes() / 16);   // plane rows are whole 16-pixel groups
        d.item_start = items;
        d.plane_id = p;
        items += (d.words + 32 * kClearWords - 1) / (32 * kClearWords);
        descs->push_back(d);
    }
    if (items >= (int64_t)1 << 31) return efail(e, CPT_EINVAL, "too many clear items");
    *n_items = items;
    return CPT_OK;
}

int launch_clear(composite_engine *e, const void *d_ops, int n_ops, int64_t n_items) {
    const int64_t ctas = std::min<int64_t>((int64_t)e->caps.num_sms * kClearCtasPerSm,
                                           (n_items + kThreads / 32 - 1) / (kThreads / 32));
    engine_clear_kernel<<<(unsigned)std::max<int64_t>(1, ctas), kThreads, 0, e->stream>>>(
        static_cast<const ClearDesc *>(d_ops), n_ops, (uint32_t)n_items, e->d_flags);
    ECK(e, cudaGetLastError());
    return CPT_OK;
}

// Clears the listed planes in one launch (their counts, N and underflow and
// failure marks).
int clear_many(composite_engine *e, const int32_t *planes, int32_t n) {
    std::vector<ClearDesc> descs;
    int64_t items = 0;
    int rc = plan_clears(e, planes, n, &descs, &items);
    if (rc || descs.empty()) return rc;
    Upload *u = nullptr;
    rc = upload(e, e->up_render, &e->rup_i, descs.data(), descs.size() * sizeof(ClearDesc), &u);
    if (rc) return rc;
    rc = launch_clear(e, u->d, (int)descs.size(), items);
    if (rc) return rc;
    ECK(e, cudaEventRecord(u->consumed, e->stream));
    for (const ClearDesc &d : descs) {
        e->planes[d.plane_id].n = 0;
        e->planes[d.plane_id].poisoned = false;
    }
    return CPT_OK;
}

void free_stage(composite_engine *e) {
    for (StageSlot &s : e->stage) {
        if (s.d) cudaFree(s.d);
        if (s.ready) cudaEventDestroy(s.ready);
        if (s.consumed) cudaEventDestroy(s.consumed);
    }
    e->stage.clear();
    e->stage_bytes = 0;
    e->stage_next = 0;
}

// Staging buffers of the configured count and size, allocated at the first
// host op and again whenever the configuration changed (after the engine's
// queued work, which may still read the old ones).
int ensure_stage(composite_engine *e) {
    const int k = e->cfg.staging_buffers;
    const int64_t bytes = e->cfg.staging_bytes;
    if ((int)e->stage.size() == k && e->stage_bytes == bytes) return CPT_OK;
    int rc = drain(e);
    if (rc) return rc;
    free_stage(e);
    if (!e->copy) ECK(e, cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking));
    if (!e->caller_ready) ECK(e, cudaEventCreateWithFlags(&e->caller_ready, cudaEventDisableTiming));
    e->stage.resize(k);
    for (StageSlot &s : e->stage) {
        cudaError_t err = cudaMalloc(&s.d, (size_t)bytes);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s.consumed, cudaEventDisableTiming);
        if (err != cudaSuccess) {
            free_stage(e);
            return ecuda(e, err, "staging buffer allocation");
        }
    }
    e->stage_bytes = bytes;
    return CPT_OK;
}

// Launches the accumulate kernel over ops (already validated as a whole).
// desc_stream: where the descriptors are uploaded (NULL = the usual upload
// stream); the launch waits for them either way.
int launch_ops(composite_engine *e, const composite_op *ops, int32_t n_ops, bool *launched,
               cudaStream_t desc_stream = nullptr) {
    std::vector<OpDesc> descs;
    std::vector<std::pair<int32_t, int64_t>> n_after;
    int64_t items = 0;
    int rc = plan_ops(e, ops, n_ops, &descs, &items, &n_after, false, false);
    if (rc || items == 0) return rc;
    Upload *u = nullptr;
    rc = upload(e, e->up_ops, &e->up_i, descs.data(), descs.size() * sizeof(OpDesc), &u, desc_stream);
    if (rc) return rc;
    if (cpt::fault_injected("engine_submit")) return efail(e, CPT_ECUDA, "submit refused before its launch (injected)");
    *launched = true;   // from here on the launch may have begun
    rc = launch_accumulate(e, u->d, (int)descs.size(), items, e->d_counter);
    if (rc) return rc;
    ECK(e, cudaEventRecord(u->consumed, e->stream));
    return CPT_OK;
}

// Ops on pinned host members: their rasters are packed, op after op, into
// staging buffers of stage_bytes; a full buffer is uploaded on the copy
// stream (after the launch that last read it) and folded by one accumulate
// launch on the engine stream (after the upload), so the upload of one
// buffer overlaps the fold of the previous one.
int stream_host_ops(composite_engine *e, const std::vector<composite_op> &hops, bool *launched) {
    int rc = ensure_stage(e);
    if (rc) return rc;
    // uploads start after the caller's earlier work on the engine stream
    ECK(e, cudaEventRecord(e->caller_ready, e->stream));
    ECK(e, cudaStreamWaitEvent(e->copy, e->caller_ready, 0));
    struct Run {
        size_t op;
        int32_t m0, cnt;
        int64_t offset;
    };
    std::vector<Run> runs;
    int64_t used = 0;
    int64_t chunk = 0;
    const int64_t inject_at = cpt::fault_injected_value("engine_chunk_fail");
    auto flush = [&]() -> int {
        if (runs.empty()) return CPT_OK;
        if (inject_at == chunk) return efail(e, CPT_ECUDA, "upload of staging chunk %lld refused (injected)", (long long)chunk);
        ++chunk;
        StageSlot &slot = e->stage[e->stage_next++ % e->stage.size()];
        if (slot.used) ECK(e, cudaStreamWaitEvent(e->copy, slot.consumed, 0));
        std::vector<composite_op> cops;
        cops.reserve(runs.size());
        for (const Run &r : runs) {
            const composite_op &o = hops[r.op];
            const int64_t rb = (int64_t)o.row_pitch_bytes * e->planes[o.plane].height;
            const uint8_t *src = static_cast<const uint8_t *>(o.members) + (int64_t)r.m0 * o.member_stride_bytes;
            if (o.member_stride_bytes == rb)
                ECK(e, cudaMemcpyAsync(slot.d + r.offset, src, (size_t)(r.cnt * rb), cudaMemcpyHostToDevice, e->copy));
            else
                ECK(e, cudaMemcpy2DAsync(slot.d + r.offset, (size_t)rb, src, (size_t)o.member_stride_bytes, (size_t)rb,
                                         (size_t)r.cnt, cudaMemcpyHostToDevice, e->copy));
            composite_op c = o;
            c.members = slot.d + r.offset;
            c.member_index = nullptr;
            c.n_members = r.cnt;
            c.member_stride_bytes = rb;
            cops.push_back(c);
        }
        ECK(e, cudaEventRecord(slot.ready, e->copy));
        ECK(e, cudaStreamWaitEvent(e->stream, slot.ready, 0));
        // the chunk's descriptors follow its rasters on the copy stream: on the
        // engine stream they would queue on a copy engine behind the next
        // chunk's rasters, and the fold would wait one upload longer
        int r = launch_ops(e, cops.data(), (int32_t)cops.size(), launched, e->copy);
        if (r) return r;
        ECK(e, cudaEventRecord(slot.consumed, e->stream));
        slot.used = true;
        runs.clear();
        used = 0;
        return CPT_OK;
    };
    for (size_t i = 0; i < hops.size(); ++i) {
        const composite_op &o = hops[i];
        const int64_t rb = (int64_t)o.row_pitch_bytes * e->planes[o.plane].height;
        for (int32_t m = 0; m < o.n_members;) {
            const int64_t fit = (e->stage_bytes - used) / rb;
            if (fit <= 0) {
                if ((rc = flush())) return rc;
                continue;
            }
            const int32_t take = (int32_t)std::min<int64_t>(fit, o.n_members - m);
            runs.push_back({i, m, take, used});
            used += take * rb;
            m += take;
        }
    }
    return flush();
}

int submit_internal(composite_engine *e, const composite_op *ops, int32_t n_ops) {
    const cpt::TraceRange range("composite_engine_submit");
    std::vector<OpDesc> descs;
    std::vector<std::pair<int32_t, int64_t>> n_after;
    int64_t items = 0;
    int rc = plan_ops(e, ops, n_ops, &descs, &items, &n_after, false);
    if (rc) return rc;
    for (const auto &pn : n_after)
        if (e->planes[pn.first].poisoned)
            return efail(e, CPT_ESTATE, "plane %d: an earlier submit failed part-way; clear it", pn.first);
    // device ops fold in one launch; ops on pinned host members stream
    std::vector<composite_op> dev_ops, host_ops;
    for (int32_t i = 0; i < n_ops; ++i) {
        const composite_op &o = ops[i];
        if (o.n_members == 0) continue;
        const int kind = member_kind(o.members, e->device);
        if (kind < 0)
            return efail(e, CPT_EINVAL, "op %d: members must be device memory of device %d or pinned host memory", i,
                         e->device);
        if (kind == 0) {
            if (o.member_index && !device_reachable(o.member_index, e->device))
                return efail(e, CPT_EINVAL, "op %d: member_index must be device memory of device %d", i, e->device);
            dev_ops.push_back(o);
            continue;
        }
        if (o.member_index) return efail(e, CPT_EINVAL, "op %d: an index list needs device members", i);
        if ((int64_t)o.row_pitch_bytes * e->planes[o.plane].height > e->cfg.staging_bytes)
            return efail(e, CPT_EINVAL, "op %d: a raster is larger than staging_bytes", i);
        host_ops.push_back(o);
    }
    bool launched = false;
    if (host_ops.empty()) {
        if (items > 0) {
            Upload *u = nullptr;
            rc = upload(e, e->up_ops, &e->up_i, descs.data(), descs.size() * sizeof(OpDesc), &u);
            if (rc) return rc;   // nothing launched: every plane is as before
            if (cpt::fault_injected("engine_submit"))
                return efail(e, CPT_ECUDA, "submit refused before its launch (injected)");
            launched = true;
            rc = launch_accumulate(e, u->d, (int)descs.size(), items, e->d_counter);
            if (!rc) {
                for (const auto &pn : n_after) e->planes[pn.first].n = pn.second;
                ECK(e, cudaEventRecord(u->consumed, e->stream));
                return CPT_OK;
            }
        }
    } else {
        rc = launch_ops(e, dev_ops.data(), (int32_t)dev_ops.size(), &launched);
        if (!rc) rc = stream_host_ops(e, host_ops, &launched);
    }
    if (rc) {
        // a launch may have begun: the planes of the submit hold an unknown
        // part of the ops until they are cleared
        if (launched)
            for (const auto &pn : n_after) e->planes[pn.first].poisoned = true;
        return rc;
    }
    for (const auto &pn : n_after) e->planes[pn.first].n = pn.second;
    return CPT_OK;
}

void destroy_graph(composite_engine *e) {
    if (e->graph_exec) cudaGraphExecDestroy(e->graph_exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->graph_ops) cudaFree(e->graph_ops);
    if (e->graph_rops) cudaFree(e->graph_rops);
    if (e->graph_clears) cudaFree(e->graph_clears);
    if (e->graph_counters) cudaFree(e->graph_counters);
    e->graph_exec = nullptr;
    e->graph = nullptr;
    e->graph_ops = e->graph_rops = e->graph_clears = nullptr;
    e->graph_counters = nullptr;
    e->graph_n.clear();
    e->graph_planes.clear();
}

void destroy_engine(composite_engine *e) {
    destroy_graph(e);
    for (PlaneRec &p : e->planes)
        if (p.data) cudaFree(p.data);
    for (Upload *ring : {e->up_ops, e->up_render})
        for (int i = 0; i < kUploadRing; ++i) {
            if (ring[i].d) cudaFree(ring[i].d);
            if (ring[i].h) cudaFreeHost(ring[i].h);
            if (ring[i].done) cudaEventDestroy(ring[i].done);
            if (ring[i].consumed) cudaEventDestroy(ring[i].consumed);
        }
    if (e->d_flags) cudaFree(e->d_flags);
    if (e->h_flags) cudaFreeHost(e->h_flags);
    if (e->d_counter) cudaFree(e->d_counter);
    if (e->done_ev) cudaEventDestroy(e->done_ev);
    if (e->capture_stream) cudaStreamDestroy(e->capture_stream);
    free_stage(e);
    if (e->copy) cudaStreamDestroy(e->copy);
    if (e->caller_ready) cudaEventDestroy(e->caller_ready);
    delete e;
}

}  // namespace

extern "C" {

int composite_engine_default_config(composite_engine_config *cfg) try {
    if (!cfg) return CPT_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->slab_members = 128;
    cfg->ctas_per_sm = 5;
    cfg->schedule = CPT_SCHEDULE_PERSISTENT;
    cfg->item_member_groups = kDefaultItemMemberGroups;
    cfg->staging_buffers = 2;
    cfg->staging_bytes = kDefaultStageBytes;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_begin(composite_engine **out, const composite_engine_config *cfg) try {
    g_engine_error.clear();
    if (!out) return efail(nullptr, CPT_EINVAL, "out is NULL");
    *out = nullptr;
    composite_engine_config c;
    composite_engine_default_config(&c);
    if (cfg) {
        c.cuda_stream = cfg->cuda_stream;
        c.wait_timeout_ms = cfg->wait_timeout_ms;
        if (cfg->slab_members) c.slab_members = cfg->slab_members;
        if (cfg->ctas_per_sm) c.ctas_per_sm = cfg->ctas_per_sm;
        c.schedule = cfg->schedule;
        c.upload_stream = cfg->upload_stream;
        if (cfg->item_member_groups) c.item_member_groups = cfg->item_member_groups;
        if (cfg->staging_buffers) c.staging_buffers = cfg->staging_buffers;
        if (cfg->staging_bytes) c.staging_bytes = cfg->staging_bytes;
    }
    if (c.schedule != CPT_SCHEDULE_PERSISTENT && c.schedule != CPT_SCHEDULE_GRID)
        return efail(nullptr, CPT_EINVAL, "schedule must be CPT_SCHEDULE_PERSISTENT or CPT_SCHEDULE_GRID");
    if (c.slab_members < 1 || c.slab_members > kMaxSlab) return efail(nullptr, CPT_EINVAL, "slab_members not in 1..255");
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 8) return efail(nullptr, CPT_EINVAL, "ctas_per_sm not in 1..8");
    if (c.wait_timeout_ms < 0) return efail(nullptr, CPT_EINVAL, "negative timeout");
    if (c.item_member_groups < 16 || c.item_member_groups > 8192)
        return efail(nullptr, CPT_EINVAL, "item_member_groups not in 16..8192");
    if (c.staging_buffers < 2 || c.staging_buffers > 8) return efail(nullptr, CPT_EINVAL, "staging_buffers not in 2..8");
    if (c.staging_bytes < (1ll << 20)) return efail(nullptr, CPT_EINVAL, "staging_bytes below 1 MiB");
    composite_engine *e = new composite_engine();
    e->cfg = c;
    auto setup = [&]() -> int {
        ECK(e, cudaGetDevice(&e->device));
        ECK(e, cudaDeviceGetAttribute(&e->caps.num_sms, cudaDevAttrMultiProcessorCount, e->device));
        e->stream = static_cast<cudaStream_t>(c.cuda_stream);   // NULL: the legacy default stream
        ECK(e, cudaMalloc(&e->d_flags, kMaxPlanes * sizeof(int)));
        ECK(e, cudaMemsetAsync(e->d_flags, 0, kMaxPlanes * sizeof(int), e->stream));
        ECK(e, cudaHostAlloc(&e->h_flags, kMaxPlanes * sizeof(int), cudaHostAllocDefault));
        ECK(e, cudaMalloc(&e->d_counter, sizeof(uint32_t)));
        ECK(e, cudaEventCreateWithFlags(&e->done_ev, cudaEventDisableTiming));
        for (Upload *ring : {e->up_ops, e->up_render})
            for (int i = 0; i < kUploadRing; ++i) {
                ECK(e, cudaEventCreateWithFlags(&ring[i].done, cudaEventDisableTiming));
                ECK(e, cudaEventCreateWithFlags(&ring[i].consumed, cudaEventDisableTiming));
            }
        e->default_lut = make_lut(nullptr);
        return prepare_render_kernels(e);
    };
    const int rc = setup();
    if (rc) {
        g_engine_error = e->err;
        destroy_engine(e);
        return rc;
    }
    *out = e;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_add_plane(composite_engine *e, int32_t width, int32_t height, int32_t *plane_out) try {
    return composite_engine_add_plane_bits(e, width, height, 32, plane_out);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_add_plane_bits(composite_engine *e, int32_t width, int32_t height, int32_t count_bits,
                                    int32_t *plane_out) try {
    if (!e || !plane_out) return CPT_EINVAL;
    e->err.clear();
    if (width <= 0 || height <= 0) return efail(e, CPT_EINVAL, "plane %d x %d is empty", width, height);
    if (count_bits != 16 && count_bits != 32) return efail(e, CPT_EINVAL, "count_bits must be 16 or 32");
    if ((int)e->planes.size() >= kMaxPlanes) return efail(e, CPT_EINVAL, "at most %d planes", kMaxPlanes);
    PlaneRec r;
    r.width = width;
    r.height = height;
    r.pitch_px = ((int64_t)width + 15) / 16 * 16;
    r.count_bits = count_bits;
    if (cpt::fault_injected("engine_plane")) return efail(e, CPT_ENOMEM, "plane allocation refused (injected)");
    ECK(e, cudaMalloc(&r.data, r.bytes()));
    r.alive = true;
    e->planes.push_back(r);
    const int32_t id = (int32_t)e->planes.size() - 1;
    const int rc = clear_plane(e, id);
    if (rc) return rc;
    *plane_out = id;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_free_plane(composite_engine *e, int32_t plane) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    if (!plane_ok(e, plane)) return efail(e, CPT_EINVAL, "no plane %d", plane);
    int rc = drain(e);
    if (rc) return rc;
    cudaFree(e->planes[plane].data);
    e->planes[plane] = PlaneRec();
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_clear(composite_engine *e, int32_t plane) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    if (!plane_ok(e, plane)) return efail(e, CPT_EINVAL, "no plane %d", plane);
    return clear_plane(e, plane);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_clear_many(composite_engine *e, const int32_t *planes, int32_t n_planes) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    return clear_many(e, planes, n_planes);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_submit(composite_engine *e, const composite_op *ops, int32_t n_ops) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    return submit_internal(e, ops, n_ops);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_render(composite_engine *e, const composite_render_op *ops, int32_t n_ops,
                            const uint8_t *lut_rgba) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    std::vector<RenderDesc> descs;
    int64_t items = 0;
    int rc = plan_render(e, ops, n_ops, &descs, &items, nullptr);
    if (rc || items == 0) return rc;
    const bool hist = any_histogram(descs);
    std::vector<ClearDesc> cdescs;
    int64_t citems = 0;
    if (hist) plan_histogram_clears(descs, &cdescs, &citems);
    // one upload: the histograms' clear entries, then the render descriptors
    std::vector<unsigned char> blob(cdescs.size() * sizeof(ClearDesc) + descs.size() * sizeof(RenderDesc));
    if (!cdescs.empty()) memcpy(blob.data(), cdescs.data(), cdescs.size() * sizeof(ClearDesc));
    memcpy(blob.data() + cdescs.size() * sizeof(ClearDesc), descs.data(), descs.size() * sizeof(RenderDesc));
    Upload *u = nullptr;
    rc = upload(e, e->up_render, &e->rup_i, blob.data(), blob.size(), &u);
    if (rc) return rc;
    if (citems > 0) {
        rc = launch_clear(e, u->d, (int)cdescs.size(), citems);
        if (rc) return rc;
    }
    rc = launch_render(e, static_cast<unsigned char *>(u->d) + cdescs.size() * sizeof(ClearDesc), (int)descs.size(),
                       items, hist, lut_rgba ? make_lut(lut_rgba) : e->default_lut);
    if (rc) return rc;
    ECK(e, cudaEventRecord(u->consumed, e->stream));
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_member_count(const composite_engine *e, int32_t plane, int64_t *n_out) try {
    if (!e || !n_out || !plane_ok(e, plane)) return CPT_EINVAL;
    *n_out = e->planes[plane].n;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_sync(composite_engine *e, int32_t *bad_plane_out) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    if (bad_plane_out) *bad_plane_out = -1;
    const size_t n = e->planes.size();
    if (n) ECK(e, cudaMemcpyAsync(e->h_flags, e->d_flags, n * sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    int rc = drain(e);
    if (rc) return rc;
    for (size_t p = 0; p < n; ++p)
        if (e->planes[p].alive && e->h_flags[p]) {
            if (bad_plane_out) *bad_plane_out = (int32_t)p;
            return efail(e, CPT_EUNDERFLOW, "plane %zu: a remove took away a member that was never added", p);
        }
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_capture(composite_engine *e, const composite_op *ops, int32_t n_ops,
                             const composite_render_op *rops, int32_t n_rops, const uint8_t *lut_rgba) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    std::vector<OpDesc> descs;
    std::vector<RenderDesc> rdescs;
    std::vector<std::pair<int32_t, int64_t>> n_after;
    int64_t items = 0, ritems = 0;
    int rc = plan_ops(e, ops, n_ops, &descs, &items, &n_after, true);
    if (rc) return rc;
    for (int32_t i = 0; i < n_ops; ++i) {
        if (ops[i].n_members == 0) continue;
        if (member_kind(ops[i].members, e->device) != 0)
            return efail(e, CPT_EINVAL, "op %d: a captured graph reads members of device %d only", i, e->device);
        if (ops[i].member_index && !device_reachable(ops[i].member_index, e->device))
            return efail(e, CPT_EINVAL, "op %d: member_index must be device memory of device %d", i, e->device);
    }
    rc = plan_render(e, rops, n_rops, &rdescs, &ritems, &n_after);
    if (rc) return rc;
    std::vector<int32_t> cleared;
    for (const auto &pn : n_after) cleared.push_back(pn.first);
    std::vector<ClearDesc> cdescs;
    int64_t citems = 0;
    rc = plan_clears(e, cleared.data(), (int32_t)cleared.size(), &cdescs, &citems);
    if (rc) return rc;
    const bool hist = any_histogram(rdescs);
    plan_histogram_clears(rdescs, &cdescs, &citems);   // zeroed in the same clear node
    rc = drain(e);
    if (rc) return rc;
    destroy_graph(e);
    ECK(e, cudaMalloc(&e->graph_counters, 2 * sizeof(uint32_t)));
    if (!cdescs.empty()) {
        ECK(e, cudaMalloc(&e->graph_clears, cdescs.size() * sizeof(ClearDesc)));
        ECK(e, cudaMemcpy(e->graph_clears, cdescs.data(), cdescs.size() * sizeof(ClearDesc), cudaMemcpyHostToDevice));
    }
    if (!descs.empty()) {
        ECK(e, cudaMalloc(&e->graph_ops, descs.size() * sizeof(OpDesc)));
        ECK(e, cudaMemcpy(e->graph_ops, descs.data(), descs.size() * sizeof(OpDesc), cudaMemcpyHostToDevice));
    }
    if (!rdescs.empty()) {
        ECK(e, cudaMalloc(&e->graph_rops, rdescs.size() * sizeof(RenderDesc)));
        ECK(e, cudaMemcpy(e->graph_rops, rdescs.data(), rdescs.size() * sizeof(RenderDesc), cudaMemcpyHostToDevice));
    }
    const Lut lut = lut_rgba ? make_lut(lut_rgba) : e->default_lut;
    // Capture happens on a private stream (the legacy default stream cannot
    // be captured); the graph is launched on the engine's stream.
    if (!e->capture_stream) ECK(e, cudaStreamCreateWithFlags(&e->capture_stream, cudaStreamNonBlocking));
    cudaStream_t engine_stream = e->stream;
    e->stream = e->capture_stream;
    struct Restore {
        composite_engine *e;
        cudaStream_t s;
        ~Restore() { e->stream = s; }
    } restore{e, engine_stream};
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> int {
        if (citems > 0) {   // every target plane and its flag in one node
            int r = launch_clear(e, e->graph_clears, (int)cdescs.size(), citems);
            if (r) return r;
        }
        if (items > 0) {
            int r = launch_accumulate(e, e->graph_ops, (int)descs.size(), items, e->graph_counters);
            if (r) return r;
        }
        if (ritems > 0) {
            int r = launch_render(e, e->graph_rops, (int)rdescs.size(), ritems, hist, lut);
            if (r) return r;
        }
        return CPT_OK;
    };
    const int brc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(e->stream, &g);
    if (brc) {
        if (g) cudaGraphDestroy(g);
        return brc;
    }
    if (ec != cudaSuccess) return ecuda(e, ec, "cudaStreamEndCapture");
    e->graph = g;
    ECK(e, cudaGraphInstantiate(&e->graph_exec, e->graph, 0));
    e->graph_n = n_after;
    for (const auto &pn : n_after) e->graph_planes.push_back(pn.first);
    for (int32_t i = 0; i < n_rops; ++i) e->graph_planes.push_back(rops[i].plane);
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_replay(composite_engine *e) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    if (!e->graph_exec) return efail(e, CPT_ESTATE, "nothing captured");
    for (const int32_t p : e->graph_planes)
        if (!plane_ok(e, p)) return efail(e, CPT_ESTATE, "a captured plane was freed");
    ECK(e, cudaGraphLaunch(e->graph_exec, e->stream));
    // the graph clears every plane it folds into before folding
    for (const auto &pn : e->graph_n) {
        e->planes[pn.first].n = pn.second;
        e->planes[pn.first].poisoned = false;
    }
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_tune(composite_engine *e, const composite_op *ops, int32_t n_ops, int32_t repeats,
                          int32_t *slab_out, int32_t *ctas_out) try {
    if (!e) return CPT_EINVAL;
    e->err.clear();
    if (repeats < 1) return efail(e, CPT_EINVAL, "repeats < 1");
    std::vector<OpDesc> descs;
    std::vector<std::pair<int32_t, int64_t>> n_after;
    int64_t items = 0;
    int rc = plan_ops(e, ops, n_ops, &descs, &items, &n_after, true);
    if (rc) return rc;
    bool any_host = false;
    for (int32_t i = 0; i < n_ops; ++i)
        if (ops[i].n_members > 0 && member_kind(ops[i].members, e->device) == 1) any_host = true;
    cudaEvent_t a = nullptr, b = nullptr;
    ECK(e, cudaEventCreate(&a));
    cudaError_t ce = cudaEventCreate(&b);
    if (ce != cudaSuccess) {
        cudaEventDestroy(a);
        return ecuda(e, ce, "cudaEventCreate");
    }
    std::vector<int32_t> cleared;
    for (const auto &pn : n_after) cleared.push_back(pn.first);
    auto run = [&]() -> int {
        const int r = clear_many(e, cleared.data(), (int32_t)cleared.size());
        return r ? r : submit_internal(e, ops, n_ops);
    };
    // Best of `repeats` timed runs (each after an untimed one) of the current
    // configuration, in ms; < 0 on error (rc set).
    auto time_config = [&]() -> float {
        float t_best = 1e30f;
        for (int r = 0; r < repeats; ++r) {
            if ((rc = run())) return -1.f;             // warm and measure alike: clear + submit
            if (cudaEventRecord(a, e->stream) != cudaSuccess) { rc = efail(e, CPT_ECUDA, "cudaEventRecord"); return -1.f; }
            if ((rc = run())) return -1.f;
            if (cudaEventRecord(b, e->stream) != cudaSuccess) { rc = efail(e, CPT_ECUDA, "cudaEventRecord"); return -1.f; }
            if ((rc = ewait(e, b))) return -1.f;
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            t_best = std::min(t_best, ms);
        }
        return t_best;
    };
    composite_engine_config best = e->cfg;
    float best_ms = 1e30f;
    auto consider = [&]() -> bool {
        const float ms = time_config();
        if (ms < 0) return false;
        if (ms < best_ms) {
            best_ms = ms;
            best = e->cfg;
        }
        return true;
    };
    // pass 1: slab depth x schedule (ctas_per_sm 0 stands for the grid schedule)
    static const int slabs[] = {32, 64, 128, 255};
    static const int ctas[] = {0, 3, 4, 5};
    const int ctas_before = e->cfg.ctas_per_sm;
    for (int sl : slabs)
        for (int c : ctas) {
            if (rc) break;
            e->cfg.slab_members = sl;
            e->cfg.schedule = c ? CPT_SCHEDULE_PERSISTENT : CPT_SCHEDULE_GRID;
            e->cfg.ctas_per_sm = c ? c : ctas_before;
            if (!consider()) break;
        }
    // pass 2: the work item's tile of groups
    static const int item_groups[] = {256, 512, 1024, 2048};
    if (!rc) {
        e->cfg = best;
        for (int g : item_groups) {
            e->cfg.item_member_groups = g;
            if (!consider()) break;
        }
    }
    // pass 3: staging buffers for host members
    static const int stage_counts[] = {2, 3, 4};
    static const int stage_mib[] = {64, 128, 256, 512};
    if (!rc && any_host) {
        int64_t largest = 0;
        for (int32_t i = 0; i < n_ops; ++i)
            largest = std::max<int64_t>(largest, (int64_t)ops[i].row_pitch_bytes * e->planes[ops[i].plane].height);
        e->cfg = best;
        for (int k : stage_counts)
            for (int mib : stage_mib) {
                if (rc || ((int64_t)mib << 20) < largest) continue;
                e->cfg.staging_buffers = k;
                e->cfg.staging_bytes = (int64_t)mib << 20;
                if (!consider()) break;
            }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e->cfg = best;
    if (rc) return rc;
    rc = run();
    if (rc) return rc;
    if (slab_out) *slab_out = best.slab_members;
    if (ctas_out) *ctas_out = best.schedule == CPT_SCHEDULE_GRID ? 0 : best.ctas_per_sm;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_get_tuning(const composite_engine *e, int32_t *slab_out, int32_t *ctas_out) try {
    if (!e) return CPT_EINVAL;
    if (slab_out) *slab_out = e->cfg.slab_members;
    if (ctas_out) *ctas_out = e->cfg.schedule == CPT_SCHEDULE_GRID ? 0 : e->cfg.ctas_per_sm;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_get_config(const composite_engine *e, composite_engine_config *cfg_out) try {
    if (!e || !cfg_out) return CPT_EINVAL;
    *cfg_out = e->cfg;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_engine_end(composite_engine *e) try {
    if (!e) return CPT_OK;
    const int rc = drain(e);
    destroy_engine(e);
    return rc;
} catch (...) {
    return cpt::abi_exception_status();
}

const char *composite_engine_last_error(const composite_engine *e) try {
    return e ? e->err.c_str() : g_engine_error.c_str();
} catch (...) {
    return "internal error (exception)";
}

}  // extern "C"
