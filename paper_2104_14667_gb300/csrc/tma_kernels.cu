// tma_kernels.cu -- the accumulation step over the TMA read path.
//
// The batch is described to the tensor memory accelerator as a 3-D tensor
// (x = pixel within a row, y = row, z = member).  A persistent CTA walks its
// composite tiles (64, 128 or 256 bytes wide, 2 KiB per member); for every
// tile one producer thread streams boxes of that tile x 16 members through a
// ring of shared-memory stages with cp.async.bulk.tensor, and four consumer
// warps fold each box into registers, one 16-byte group per thread.  Boxes
// past the raster's edge or the last member are zero filled by the hardware,
// which counts as "not flooded" and adds 0.0 to a depth sum.  Every mbarrier wait is bounded
// in time; a wait that runs out raises the timeout flag and the CTA leaves
// after draining its own copies in flight.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include <cudaTypedefs.h>

#include "bit_count.cuh"

namespace cpt {
namespace {

// A box is kBoxX bytes x (2048 / kBoxX) rows x kBoxMembers members: 2 KiB
// per member, 32 KiB per box, one 16-byte group per consumer thread and
// member; four stages, one CTA per SM.  Measured on 256 members at 4096^2
// (256-byte boxes, ms per pass, masks / depths): 16 x 4 x 1 CTA 0.639-0.649 /
// 2.36-2.39; 16 x 5 x 1 0.648 / 2.45; 16 x 3 x 1 0.661 / 2.47; 32 x 2 x 1
// 0.648 / 2.40; 8 x 6 x 2 CTAs 0.680 / 2.48; 8 x 13 x 1 0.650 / 2.50.
constexpr int kMemberPlaneBytes = 2048;
constexpr int kBoxMembers = 16;                      // z extent
constexpr int kBoxBytes = kMemberPlaneBytes * kBoxMembers;   // 32 KiB
constexpr int kStages = 4;
constexpr int kConsumers = 128;                      // one 16-byte group each
constexpr int kThreads = kConsumers + 32;            // + one producer warp
constexpr int kCtasPerSm = 1;

struct alignas(128) TmaShared {
    uint8_t stage[kStages][kBoxBytes];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    int abort;
};
constexpr size_t kSmemBytes = sizeof(TmaShared) + 128;   // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `bar` with the given parity to complete, for at most
// timeout_ns, or until another thread of the CTA has given up.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, uint64_t timeout_ns,
                                             volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t deadline = global_ns() + timeout_ns;
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 31u) == 0u && (*abort || global_ns() > deadline)) return false;
    }
}

__device__ __forceinline__ void tma_load_box(void *dst, const CUtensorMap *map, int x, int y,
                                             int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint4 lds16(const uint8_t *p) {
    return *reinterpret_cast<const uint4 *>(p);
}

// The producer role: one thread issues every box of the CTA's tiles.
__device__ void produce(TmaShared &sh, const CUtensorMap *map, int tiles, int tiles_x,
                        int slabs, int box_x_elems, int box_rows, uint64_t timeout_ns, int *flags) {
    uint32_t it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < tiles; tile += gridDim.x) {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        for (int slab = 0; slab < slabs; ++slab, ++it) {
            const int s = it % kStages;
            const uint32_t phase = (it / kStages) & 1u;
            if (!wait_bounded(&sh.empty[s], phase ^ 1u, timeout_ns, &sh.abort)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&sh.full[s], kBoxBytes);
            tma_load_box(sh.stage[s], map, tx * box_x_elems, ty * box_rows, slab * kBoxMembers,
                         &sh.full[s]);
        }
    }
    if (!ok) {
        flag_set(flags, kFlagTimeout);
        sh.abort = 1;
        // Drain: every box still in flight lands before the CTA may exit.
        const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0u;
        for (uint32_t j = first; j < it; ++j) {
            int dummy = 0;
            wait_bounded(&sh.full[j % kStages], (j / kStages) & 1u, timeout_ns, &dummy);
        }
    }
}

template <typename CountT, int kBoxX>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
count_tma_kernel(const __grid_constant__ CUtensorMap map, Plane p, int n_members, int sign,
                 int *flags, uint64_t timeout_ns) {
    constexpr int kRows = kMemberPlaneBytes / kBoxX;
    constexpr int kGroupsPerRow = kBoxX / 16;
    extern __shared__ uint8_t smem_raw[];
    TmaShared &sh = *reinterpret_cast<TmaShared *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tiles_x = (p.width + kBoxX - 1) / kBoxX;
    const int tiles = tiles_x * ((p.height + kRows - 1) / kRows);
    const int slabs = (n_members + kBoxMembers - 1) / kBoxMembers;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], kConsumers);
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= kConsumers) {
        if (threadIdx.x == kConsumers)
            produce(sh, &map, tiles, tiles_x, slabs, kBoxX, kRows, timeout_ns, flags);
        return;
    }

    CountT *plane = static_cast<CountT *>(p.data);
    const int row = threadIdx.x / kGroupsPerRow, grp = threadIdx.x % kGroupsPerRow;
    const int offset = row * kBoxX + grp * 16;
    uint32_t it = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        uint32_t wide[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) wide[j] = 0;
        uint32_t k0 = 0, k1 = 0, k2 = 0, k3 = 0;
        int packed_members = 0;
        for (int slab = 0; slab < slabs; ++slab, ++it) {
            const int s = it % kStages;
            if (!wait_bounded(&sh.full[s], (it / kStages) & 1u, timeout_ns, &sh.abort)) {
                flag_set(flags, kFlagTimeout);
                sh.abort = 1;
                return;
            }
            const uint8_t *box = sh.stage[s] + offset;
#pragma unroll
            for (int m = 0; m < kBoxMembers; ++m) {
                const uint4 v = lds16(box + m * kMemberPlaneBytes);
                k0 += nonzero_bytes(v.x);
                k1 += nonzero_bytes(v.y);
                k2 += nonzero_bytes(v.z);
                k3 += nonzero_bytes(v.w);
            }
            mbar_arrive(&sh.empty[s]);
            packed_members += kBoxMembers;
            if (packed_members > 255 - kBoxMembers) {
                widen16(wide, k0, k1, k2, k3);
                k0 = k1 = k2 = k3 = 0;
                packed_members = 0;
            }
        }
        widen16(wide, k0, k1, k2, k3);
        const int y = ty * kRows + row;
        const int x0 = tx * kBoxX + grp * 16;
        if (y < p.height && x0 < p.width)
            apply_count_group<CountT>(plane + (int64_t)y * p.pitch + x0, min(16, p.width - x0),
                                      wide, sign, flags);
    }
}

template <int kBoxX>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
depth_tma_kernel(const __grid_constant__ CUtensorMap map, Plane p, int n_members, int sign,
                 int *flags, uint64_t timeout_ns) {
    constexpr int kRows = kMemberPlaneBytes / kBoxX;
    constexpr int kGroupsPerRow = kBoxX / 16;
    constexpr int kBoxXElems = kBoxX / 4;      // float32 pixels per box row
    extern __shared__ uint8_t smem_raw[];
    TmaShared &sh = *reinterpret_cast<TmaShared *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tiles_x = (p.width + kBoxXElems - 1) / kBoxXElems;
    const int tiles = tiles_x * ((p.height + kRows - 1) / kRows);
    const int slabs = (n_members + kBoxMembers - 1) / kBoxMembers;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], kConsumers);
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= kConsumers) {
        if (threadIdx.x == kConsumers)
            produce(sh, &map, tiles, tiles_x, slabs, kBoxXElems, kRows, timeout_ns, flags);
        return;
    }

    float *plane = static_cast<float *>(p.data);
    const int row = threadIdx.x / kGroupsPerRow, grp = threadIdx.x % kGroupsPerRow;
    const int offset = row * kBoxX + grp * 16;
    uint32_t it = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int slab = 0; slab < slabs; ++slab, ++it) {
            const int s = it % kStages;
            if (!wait_bounded(&sh.full[s], (it / kStages) & 1u, timeout_ns, &sh.abort)) {
                flag_set(flags, kFlagTimeout);
                sh.abort = 1;
                return;
            }
            const uint8_t *box = sh.stage[s] + offset;
#pragma unroll
            for (int m = 0; m < kBoxMembers; ++m) {
                const float4 v = *reinterpret_cast<const float4 *>(box + m * kMemberPlaneBytes);
                acc[0] += v.x;
                acc[1] += v.y;
                acc[2] += v.z;
                acc[3] += v.w;
            }
            mbar_arrive(&sh.empty[s]);
        }
        const int y = ty * kRows + row;
        const int x0 = tx * kBoxXElems + grp * 4;
        if (y < p.height && x0 < p.width)
            apply_depth_group(plane + (int64_t)y * p.pitch + x0, min(4, p.width - x0), acc, sign);
    }
}

// ---- bit-packed masks through bulk copies -----------------------------------
//
// With unpadded bit rows (width a multiple of 32, row pitch width / 8) a
// member's raster is one run of 32-pixel words, so a tile of kBitsTileWords
// consecutive words is one contiguous 2 KiB piece of every member.  The
// producer warp streams the pieces of 16 members per stage with cp.async.bulk
// (no tensor map: one lane per member) into a ring of seven 32 KiB
// shared-memory stages; four consumer warps keep the counts of 128 pixels per
// thread in carry-save accumulators, four independent chains per thread.
// The bytes in flight wait in shared memory instead of registers, which is
// what limits the register kernel (launch_count_bits).  Measured shapes
// (4096^2 x 1024, ms per pass): 4 warps x 128 pixels 0.371 with a 192 KiB
// ring, 0.367 with 224 KiB, 0.398 with 128 KiB; 8 x 64 0.378; 16 x 64
// 0.404; 4 x 64 (1 KiB pieces) 0.613; two or three CTAs per SM with smaller
// rings 0.403.
// Work items are (tile, member slab).  They are numbered in blocks of one
// tile per CTA, slab after slab within a block, and dealt to the persistent
// CTAs round robin, so CTA c takes tile c of the block through all its slabs
// in turn: no two CTAs fold into one tile at the same time, and the tile's
// counts stay in L2 between its slabs.  (Slab-major numbering streamed the
// whole mask set between two visits of a tile and re-read the count plane
// from DRAM once per slab; tile-major numbering had up to 18 CTAs folding
// atomics into the same tile.)  A slab is at most 15 stages (240 members):
// the counters hold 255.
constexpr int kBitsConsumerWarps = 4;
constexpr int kBitsWordsPerThread = 4;
constexpr int kBitsConsumers = kBitsConsumerWarps * 32;
constexpr int kBitsThreads = kBitsConsumers + 32;                    // + the producer warp
constexpr int kBitsTileWords = kBitsConsumers * kBitsWordsPerThread;
constexpr int kBitsTileBytes = kBitsTileWords * 4;
constexpr int kBitsStageMembers = 16;
constexpr int kBitsStageBytes = kBitsTileBytes * kBitsStageMembers;
constexpr int kBitsRingBytes = 224 * 1024;
constexpr int kBitsStages = kBitsRingBytes / kBitsStageBytes;
constexpr int kBitsCtasPerSm = 1;
constexpr int kBitsSlabStages = 15;
static_assert(kBitsStages >= 2, "the ring needs two stages");
static_assert(kBitsWordsPerThread == 1 || kBitsWordsPerThread == 2 || kBitsWordsPerThread == 4,
              "a consumer reads 4, 8 or 16 bytes per member");

struct alignas(128) BitsShared {
    uint8_t stage[kBitsStages][kBitsStageBytes];
    uint64_t full[kBitsStages];
    uint64_t empty[kBitsStages];
    int abort;
};
constexpr size_t kBitsSmemBytes = sizeof(BitsShared) + 128;
static_assert(kBitsSmemBytes <= 227 * 1024, "shared memory per CTA");

struct BitsWork {
    const uint8_t *base;
    int64_t stride;          // member stride, bytes
    int64_t words;           // 32-pixel words per member
    int words_per_row;
    int tiles;
    int slabs;
    int slab_stages;
    int n;
    int block_tiles;         // tiles per block of items (the grid size)
};

// The (tile, slab) of work item `item`.
__device__ __forceinline__ void bits_item(const BitsWork &w, int item, int &tile, int &slab) {
    const int per_block = w.block_tiles * w.slabs;
    const int block = item / per_block;
    const int r = item - block * per_block;
    const int first = block * w.block_tiles;
    const int in_block = min(w.block_tiles, w.tiles - first);
    slab = r / in_block;
    tile = first + (r - slab * in_block);
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// The producer warp: lane 0 waits for a free stage and announces its bytes,
// then lane k copies member k's piece.  (One tensor-map box per stage --
// {256 words, 2 rows, 16 members} -- was slower: 0.381 against 0.367 ms.)
__device__ void produce_bits(BitsShared &sh, const BitsWork &w, uint64_t timeout_ns, int *flags) {
    const int lane = threadIdx.x & 31;
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < w.slabs * w.tiles; item += gridDim.x) {
        int tile, slab;
        bits_item(w, item, tile, slab);
        const int m0 = slab * w.slab_stages * kBitsStageMembers;
        const int m1 = min(w.n, m0 + w.slab_stages * kBitsStageMembers);
        const int64_t word0 = (int64_t)tile * kBitsTileWords;
        const uint32_t bytes = (uint32_t)(min((int64_t)kBitsTileWords, w.words - word0) * 4);
        for (int ms = m0; ms < m1; ms += kBitsStageMembers, ++it) {
            const int s = it % kBitsStages;
            const int cnt = min(kBitsStageMembers, m1 - ms);
            bool got = true;
            if (lane == 0) {
                got = wait_bounded(&sh.empty[s], ((it / kBitsStages) & 1u) ^ 1u, timeout_ns, &sh.abort);
                if (got) mbar_arrive_expect_tx(&sh.full[s], bytes * (uint32_t)cnt);
            }
            ok = __shfl_sync(0xFFFFFFFFu, got, 0);
            if (!ok) break;
            if (lane < cnt)
                bulk_load(sh.stage[s] + lane * kBitsTileBytes, w.base + (int64_t)(ms + lane) * w.stride + word0 * 4,
                          bytes, &sh.full[s]);
        }
    }
    if (!ok && lane == 0) {
        flag_set(flags, kFlagTimeout);
        sh.abort = 1;
        // Drain: every piece still in flight lands before the CTA may exit.
        const uint32_t first = it > (uint32_t)kBitsStages ? it - kBitsStages : 0u;
        for (uint32_t j = first; j < it; ++j) {
            int dummy = 0;
            wait_bounded(&sh.full[j % kBitsStages], (j / kBitsStages) & 1u, timeout_ns, &dummy);
        }
    }
}

template <typename CountT>
__global__ void __launch_bounds__(kBitsThreads, kBitsCtasPerSm)
count_bits_bulk_kernel(BitsWork w, Plane p, int sign, int *flags, uint64_t timeout_ns) {
    extern __shared__ uint8_t smem_raw[];
    BitsShared &sh = *reinterpret_cast<BitsShared *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBitsStages; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], kBitsConsumerWarps);
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= kBitsConsumers) {
        produce_bits(sh, w, timeout_ns, flags);
        return;
    }

    CountT *plane = static_cast<CountT *>(p.data);
    const int tid = threadIdx.x;
    uint32_t it = 0;
    for (int item = blockIdx.x; item < w.slabs * w.tiles; item += gridDim.x) {
        int tile, slab;
        bits_item(w, item, tile, slab);
        const int m0 = slab * w.slab_stages * kBitsStageMembers;
        const int m1 = min(w.n, m0 + w.slab_stages * kBitsStageMembers);
        BitCounter acc[kBitsWordsPerThread];
        for (int ms = m0; ms < m1; ms += kBitsStageMembers, ++it) {
            const int s = it % kBitsStages;
            const int cnt = min(kBitsStageMembers, m1 - ms);
            if (!wait_bounded(&sh.full[s], (it / kBitsStages) & 1u, timeout_ns, &sh.abort)) {
                flag_set(flags, kFlagTimeout);
                sh.abort = 1;
                return;
            }
            const uint8_t *src = sh.stage[s] + 4 * kBitsWordsPerThread * tid;
            uint32_t wv[kBitsWordsPerThread][16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint32_t v[4] = {0u, 0u, 0u, 0u};
                if (k < cnt) {
                    const uint8_t *q = src + k * kBitsTileBytes;
                    if constexpr (kBitsWordsPerThread == 4) {
                        const uint4 t = *reinterpret_cast<const uint4 *>(q);
                        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
                    } else if constexpr (kBitsWordsPerThread == 2) {
                        const uint2 t = *reinterpret_cast<const uint2 *>(q);
                        v[0] = t.x, v[1] = t.y;
                    } else {
                        v[0] = *reinterpret_cast<const uint32_t *>(q);
                    }
                }
#pragma unroll
                for (int j = 0; j < kBitsWordsPerThread; ++j) wv[j][k] = v[j];
            }
#pragma unroll
            for (int j = 0; j < kBitsWordsPerThread; ++j) bitcount_add16(acc[j], wv[j]);
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&sh.empty[s]);
        }
        // words past the raster's last (a partial tile) hold stale bytes and are skipped
        const int64_t word0 = (int64_t)tile * kBitsTileWords + kBitsWordsPerThread * tid;
#pragma unroll
        for (int j = 0; j < kBitsWordsPerThread; ++j) {
            const int64_t g = word0 + j;
            if (g >= w.words) break;
            const int y = (int)(g / w.words_per_row);
            const int x0 = 32 * (int)(g - (int64_t)y * w.words_per_row);
            CountT *dst = plane + (int64_t)y * p.pitch + x0;
            uint32_t pairs[16];
            bitcount_pairs(acc[j], pairs);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (w.slabs == 1)
                    apply_pair_group<CountT>(dst + 16 * h, 16, pairs + 8 * h, sign, flags);
                else
                    atomic_pair_group<CountT>(dst + 16 * h, pairs + 8 * h, sign, flags);
            }
        }
    }
}

// Runs the bounded wait of the TMA kernels on an mbarrier that nothing
// arrives at: it must give up after timeout_ns and report it.  status[0] =
// 1 if the wait gave up, status[1] = nanoseconds it waited.
__global__ void bounded_wait_selftest_kernel(uint64_t timeout_ns, unsigned long long *status) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_ns();
        const bool ok = wait_bounded(&bar, 0u, timeout_ns, &abort);
        status[0] = ok ? 0ull : 1ull;
        status[1] = global_ns() - t0;
    }
}

// Raises a kernel's dynamic shared-memory limit to `bytes`, once per
// (kernel, device): the attribute belongs to the device that is current when
// it is set, so a process that drives several GPUs sets it on each.
cudaError_t allow_smem(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        return nullptr;
    }();
    return fn;
}

unsigned grid_for(int tiles, const DeviceCaps &caps) {
    const int cap = caps.num_sms * kCtasPerSm;
    return (unsigned)(tiles < cap ? tiles : cap);
}

}  // namespace

cudaError_t launch_bounded_wait_selftest(uint64_t timeout_ns, unsigned long long *status, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(timeout_ns, status);
    return cudaGetLastError();
}

bool tma_box_supported(int box_bytes) {
    return box_bytes == 64 || box_bytes == 128 || box_bytes == 256;
}

int encode_tma_map(CUtensorMap *map, const RasterBatch &b, int width, int height, int elem_bytes,
                   int box_bytes) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
    if (!enc) return CUDA_ERROR_NOT_FOUND;
    if (!tma_box_supported(box_bytes)) return CUDA_ERROR_INVALID_VALUE;
    cuuint64_t dims[3] = {(cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)b.n};
    cuuint64_t strides[2] = {(cuuint64_t)b.row_pitch, (cuuint64_t)b.member_stride};
    cuuint32_t box[3] = {(cuuint32_t)(box_bytes / elem_bytes), (cuuint32_t)(kMemberPlaneBytes / box_bytes),
                         kBoxMembers};
    cuuint32_t estrides[3] = {1, 1, 1};
    CUresult r = enc(map,
                     elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     3, const_cast<void *>(b.base), dims, strides, box, estrides,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (int)r;
}

template <typename CountT, int kBoxX>
cudaError_t launch_count_tma_t(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                               int *flags, uint64_t timeout_ns, const DeviceCaps &caps, cudaStream_t s) {
    constexpr int kRows = kMemberPlaneBytes / kBoxX;
    const cudaError_t prep = allow_smem(reinterpret_cast<const void *>(count_tma_kernel<CountT, kBoxX>), kSmemBytes);
    if (prep != cudaSuccess) return prep;
    const int tiles = ((p.width + kBoxX - 1) / kBoxX) * ((p.height + kRows - 1) / kRows);
    count_tma_kernel<CountT, kBoxX><<<grid_for(tiles, caps), kThreads, kSmemBytes, s>>>(
        map, p, b.n, sign, flags, timeout_ns);
    return cudaGetLastError();
}

template <int kBoxX>
cudaError_t launch_depth_tma_t(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                               int *flags, uint64_t timeout_ns, const DeviceCaps &caps, cudaStream_t s) {
    constexpr int kRows = kMemberPlaneBytes / kBoxX;
    const cudaError_t prep = allow_smem(reinterpret_cast<const void *>(depth_tma_kernel<kBoxX>), kSmemBytes);
    if (prep != cudaSuccess) return prep;
    const int tiles = ((p.width + kBoxX / 4 - 1) / (kBoxX / 4)) * ((p.height + kRows - 1) / kRows);
    depth_tma_kernel<kBoxX><<<grid_for(tiles, caps), kThreads, kSmemBytes, s>>>(map, p, b.n, sign, flags,
                                                                                 timeout_ns);
    return cudaGetLastError();
}

cudaError_t launch_count_tma(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                             int *flags, uint64_t timeout_ns, int box_bytes, const DeviceCaps &caps,
                             cudaStream_t s) {
    if (b.n <= 0) return cudaSuccess;
    const bool u16 = p.count_bits == 16;
    switch (box_bytes) {
        case 64:
            return u16 ? launch_count_tma_t<uint16_t, 64>(map, b, p, sign, flags, timeout_ns, caps, s)
                       : launch_count_tma_t<uint32_t, 64>(map, b, p, sign, flags, timeout_ns, caps, s);
        case 128:
            return u16 ? launch_count_tma_t<uint16_t, 128>(map, b, p, sign, flags, timeout_ns, caps, s)
                       : launch_count_tma_t<uint32_t, 128>(map, b, p, sign, flags, timeout_ns, caps, s);
        case 256:
            return u16 ? launch_count_tma_t<uint16_t, 256>(map, b, p, sign, flags, timeout_ns, caps, s)
                       : launch_count_tma_t<uint32_t, 256>(map, b, p, sign, flags, timeout_ns, caps, s);
        default:
            return cudaErrorInvalidValue;
    }
}

bool bits_bulk_compatible(const RasterBatch &b, int width, int height) {
    return width % 32 == 0 && b.row_pitch == width / 8 && reinterpret_cast<uintptr_t>(b.base) % 16 == 0 &&
           b.member_stride % 16 == 0 && ((int64_t)(width / 32) * height) % 4 == 0;
}

template <typename CountT>
cudaError_t launch_bits_bulk_t(const BitsWork &w, unsigned grid, const Plane &p, int sign, int *flags,
                               uint64_t timeout_ns, cudaStream_t s) {
    const cudaError_t prep = allow_smem(reinterpret_cast<const void *>(count_bits_bulk_kernel<CountT>), kBitsSmemBytes);
    if (prep != cudaSuccess) return prep;
    count_bits_bulk_kernel<CountT><<<grid, kBitsThreads, kBitsSmemBytes, s>>>(w, p, sign, flags, timeout_ns);
    return cudaGetLastError();
}

cudaError_t launch_count_bits_bulk(const RasterBatch &b, const Plane &p, int sign, int *flags, uint64_t timeout_ns,
                                   const DeviceCaps &caps, cudaStream_t s) {
    if (b.n <= 0 || p.width == 0 || p.height == 0) return cudaSuccess;
    if (!bits_bulk_compatible(b, p.width, p.height)) return cudaErrorInvalidValue;
    BitsWork w;
    w.base = static_cast<const uint8_t *>(b.base);
    w.stride = b.member_stride;
    w.words_per_row = p.width / 32;
    w.words = (int64_t)w.words_per_row * p.height;
    const int64_t tiles = (w.words + kBitsTileWords - 1) / kBitsTileWords;
    if (tiles > (1 << 24)) return cudaErrorInvalidValue;
    w.tiles = (int)tiles;
    w.n = b.n;
    // slabs of at most 15 stages; more if needed for about eight items per CTA
    const int stages = (b.n + kBitsStageMembers - 1) / kBitsStageMembers;
    int slabs = (stages + kBitsSlabStages - 1) / kBitsSlabStages;
    const int want = (int)std::min<int64_t>((8ll * kBitsCtasPerSm * caps.num_sms + tiles - 1) / tiles, stages);
    slabs = std::max(slabs, want);
    w.slab_stages = (stages + slabs - 1) / slabs;
    w.slabs = (stages + w.slab_stages - 1) / w.slab_stages;
    const int64_t items = (int64_t)w.slabs * w.tiles;
    if (items > INT32_MAX) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)kBitsCtasPerSm * caps.num_sms);
    w.block_tiles = (int)std::min<int64_t>(grid, w.tiles);
    return p.count_bits == 16 ? launch_bits_bulk_t<uint16_t>(w, grid, p, sign, flags, timeout_ns, s)
                              : launch_bits_bulk_t<uint32_t>(w, grid, p, sign, flags, timeout_ns, s);
}

cudaError_t launch_depth_tma(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                             int *flags, uint64_t timeout_ns, int box_bytes, const DeviceCaps &caps,
                             cudaStream_t s) {
    if (b.n <= 0) return cudaSuccess;
    switch (box_bytes) {
        case 64: return launch_depth_tma_t<64>(map, b, p, sign, flags, timeout_ns, caps, s);
        case 128: return launch_depth_tma_t<128>(map, b, p, sign, flags, timeout_ns, caps, s);
        case 256: return launch_depth_tma_t<256>(map, b, p, sign, flags, timeout_ns, caps, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cpt
