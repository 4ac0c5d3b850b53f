// count_kernels.cu -- the accumulation step (Fig. 3, step 4: fold member i
// into the composite) over the linear read path, mask bytes and float32
// depths.
//
// One thread owns one 16-byte group of a composite row (16 mask pixels, or
// 4 float32 depth pixels) and walks the members of the batch, so every
// member byte is read once with a 16-byte load and the composite is read and
// written once per launch instead of once per member (the paper's kernel
// reads and writes the accumulator per member, Fig. 2 step 4).  Mask bytes
// are turned into per-byte ones and summed four to a 32-bit word, in slabs of
// at most 255 members so the packed byte counters cannot overflow.
#include <algorithm>

#include "device_common.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;
constexpr int kPackedLimit = 255;   // members a packed byte counter can hold

__device__ __forceinline__ uint4 load_stream16(const uint8_t *p) {
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}

// Work unit = (member slab, 16-byte group).  A slab holds at most 255
// members, so four packed byte counters never overflow inside a unit; with
// more than one slab the unit's counts go into the composite by atomics.
// Splitting the members gives many small units, so the last wave of a large
// launch is as full as the others.
template <typename CountT>
__global__ void __launch_bounds__(kThreads)
count_linear_kernel(RasterBatch b, Plane p, int sign, int *flags, int64_t groups,
                    int groups_per_row, int slab, int slabs) {
    CountT *plane = static_cast<CountT *>(p.data);
    const int64_t stride = b.member_stride;
    const int64_t units = groups * slabs;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int sl = (int)(u / groups);
        const int64_t g = u - (int64_t)sl * groups;
        const int y = (int)(g / groups_per_row);
        const int x0 = (int)(g - (int64_t)y * groups_per_row) * 16;
        const int valid = min(16, p.width - x0);
        const int m0 = sl * slab;
        const int m1 = min(b.n, m0 + slab);
        const uint8_t *q = static_cast<const uint8_t *>(b.base) + y * b.row_pitch + x0 + (int64_t)m0 * stride;
        uint32_t k[4] = {0u, 0u, 0u, 0u};
        if (valid == 16) {
#pragma unroll 8
            for (int m = m0; m < m1; ++m) {
                const uint4 v = load_stream16(q);
                q += stride;
                k[0] += nonzero_bytes(v.x);
                k[1] += nonzero_bytes(v.y);
                k[2] += nonzero_bytes(v.z);
                k[3] += nonzero_bytes(v.w);
            }
        } else {
            // ragged right edge: scalar loads, never past the row's last pixel
            for (int m = m0; m < m1; ++m, q += stride) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < valid) k[j / 4] += (uint32_t)(q[j] != 0) << (8 * (j % 4));
            }
        }
        uint32_t wide[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) wide[j] = 0;
        widen16(wide, k[0], k[1], k[2], k[3]);
        CountT *dst = plane + (int64_t)y * p.pitch + x0;
        if (slabs == 1)
            apply_count_group<CountT>(dst, valid, wide, sign, flags);
        else
            atomic_count_group<CountT>(dst, wide, sign, flags);
    }
}

__global__ void __launch_bounds__(kThreads)
depth_linear_kernel(RasterBatch b, Plane p, int sign, int64_t groups, int groups_per_row) {
    float *plane = static_cast<float *>(p.data);
    const int64_t stride = b.member_stride;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(g / groups_per_row);
        const int x0 = (int)(g - (int64_t)y * groups_per_row) * 4;
        const int valid = min(4, p.width - x0);
        const uint8_t *src = static_cast<const uint8_t *>(b.base) + y * b.row_pitch + x0 * 4;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid == 4) {
            const uint8_t *q = src;
#pragma unroll 8
            for (int m = 0; m < b.n; ++m) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(q));
                q += stride;
                acc[0] += v.x;
                acc[1] += v.y;
                acc[2] += v.z;
                acc[3] += v.w;
            }
        } else {
            for (int m = 0; m < b.n; ++m) {
                const float *q = reinterpret_cast<const float *>(src + (int64_t)m * stride);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < valid) acc[j] += q[j];
            }
        }
        apply_depth_group(plane + (int64_t)y * p.pitch + x0, valid, acc, sign);
    }
}

inline int64_t blocks_for(int64_t groups) {
    int64_t blocks = (groups + kThreads - 1) / kThreads;
    return blocks < 1 ? 1 : (blocks > 0x7FFFFFFF ? 0x7FFFFFFF : blocks);
}

}  // namespace

cudaError_t launch_count_linear(const RasterBatch &b, const Plane &p, int sign, int *flags,
                                const DeviceCaps &caps, cudaStream_t s) {
    const int gpr = (p.width + 15) / 16;
    const int64_t groups = (int64_t)gpr * p.height;
    if (b.n <= 0 || groups == 0) return cudaSuccess;
    // Member slabs: at most kPackedLimit members each; more slabs (down to 32
    // members each) when the groups alone fill fewer than eight waves.
    const int64_t target_units = 8ll * caps.num_sms * 2048;
    int64_t slabs = (b.n + kPackedLimit - 1) / kPackedLimit;
    const int64_t want = std::min<int64_t>((target_units + groups - 1) / groups, (b.n + 31) / 32);
    slabs = std::max<int64_t>(std::max<int64_t>(slabs, want), 1);
    const int slab = (int)((b.n + slabs - 1) / slabs);
    slabs = (b.n + slab - 1) / slab;
    const unsigned grid = (unsigned)blocks_for(groups * slabs);
    if (p.count_bits == 16)
        count_linear_kernel<uint16_t><<<grid, kThreads, 0, s>>>(b, p, sign, flags, groups, gpr, slab, (int)slabs);
    else
        count_linear_kernel<uint32_t><<<grid, kThreads, 0, s>>>(b, p, sign, flags, groups, gpr, slab, (int)slabs);
    return cudaGetLastError();
}

cudaError_t launch_depth_linear(const RasterBatch &b, const Plane &p, int sign, int *,
                                const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 3) / 4;
    const int64_t groups = (int64_t)gpr * p.height;
    if (b.n <= 0 || groups == 0) return cudaSuccess;
    depth_linear_kernel<<<(unsigned)blocks_for(groups), kThreads, 0, s>>>(b, p, sign, groups, gpr);
    return cudaGetLastError();
}

}  // namespace cpt
