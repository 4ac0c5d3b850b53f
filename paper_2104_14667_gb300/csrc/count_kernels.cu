// count_kernels.cu -- the accumulation step (Fig. 3, step 4: fold member i
// into the composite) over the linear and texture read paths.
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

// Bit-packed masks (one bit per pixel, pixel x at bit x & 7 of byte x >> 3 of
// the row).  A thread owns kWords 32-pixel words of a composite row (with
// kWords = 2 a warp reads 256 contiguous bytes per member, 8 per lane) and
// keeps the slab's counts in BitCounters (carry-save accumulators, see
// device_common.cuh); whole steps of 16 members load without predicates, and
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

// Texture path: member `layer` of the batch is layer `layer` of a layered
// cudaArray whose texels are 16 bytes (16 mask pixels).  Texels past the
// raster's right edge hold padding and are masked off.
template <typename CountT>
__global__ void __launch_bounds__(kThreads)
count_texture_kernel(cudaTextureObject_t tex, int n_layers, Plane p, int sign, int *flags,
                     int64_t groups, int groups_per_row) {
    CountT *plane = static_cast<CountT *>(p.data);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(g / groups_per_row);
        const int gx = (int)(g - (int64_t)y * groups_per_row);
        const int x0 = gx * 16;
        const int valid = min(16, p.width - x0);
        const uint32_t m0 = valid_byte_mask(0, valid), m1 = valid_byte_mask(1, valid);
        const uint32_t m2 = valid_byte_mask(2, valid), m3 = valid_byte_mask(3, valid);
        const float u = gx + 0.5f, v = y + 0.5f;
        uint32_t k0 = 0, k1 = 0, k2 = 0, k3 = 0;
#pragma unroll 8
        for (int layer = 0; layer < n_layers; ++layer) {
            const uint4 t = tex2DLayered<uint4>(tex, u, v, layer);
            k0 += nonzero_bytes(t.x) & m0;
            k1 += nonzero_bytes(t.y) & m1;
            k2 += nonzero_bytes(t.z) & m2;
            k3 += nonzero_bytes(t.w) & m3;
        }
        uint32_t wide[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) wide[j] = 0;
        widen16(wide, k0, k1, k2, k3);
        apply_count_group<CountT>(plane + (int64_t)y * p.pitch + x0, valid, wide, sign, flags);
    }
}

__global__ void __launch_bounds__(kThreads)
depth_texture_kernel(cudaTextureObject_t tex, int n_layers, Plane p, int sign, int64_t groups,
                     int groups_per_row) {
    float *plane = static_cast<float *>(p.data);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(g / groups_per_row);
        const int gx = (int)(g - (int64_t)y * groups_per_row);
        const int x0 = gx * 4;
        const int valid = min(4, p.width - x0);
        const float u = gx + 0.5f, v = y + 0.5f;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int layer = 0; layer < n_layers; ++layer) {
            const float4 t = tex2DLayered<float4>(tex, u, v, layer);
            acc[0] += t.x;
            acc[1] += valid > 1 ? t.y : 0.f;
            acc[2] += valid > 2 ? t.z : 0.f;
            acc[3] += valid > 3 ? t.w : 0.f;
        }
        apply_depth_group(plane + (int64_t)y * p.pitch + x0, valid, acc, sign);
    }
}

// Layout conversion by hand (the buffer-to-image transform of Section 4):
// one thread per 16-byte texel reads the linear raster with a 16-byte load
// and stores the texel into the layered cudaArray through a surface object.
__global__ void __launch_bounds__(kThreads)
convert_to_array_kernel(const uint8_t *src, int64_t pitch, int64_t member_stride, cudaSurfaceObject_t surf,
                        int texels_per_row, int height, int64_t texels) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < texels;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / texels_per_row;
        const int x = (int)(t - row * texels_per_row);
        const int layer = (int)(row / height);
        const int y = (int)(row - (int64_t)layer * height);
        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src + layer * member_stride + y * pitch + x * 16));
        surf2DLayeredwrite(v, surf, x * 16, y, layer);
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

cudaError_t launch_depth_linear(const RasterBatch &b, const Plane &p, int sign, int *,
                                const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 3) / 4;
    const int64_t groups = (int64_t)gpr * p.height;
    if (b.n <= 0 || groups == 0) return cudaSuccess;
    depth_linear_kernel<<<(unsigned)blocks_for(groups), kThreads, 0, s>>>(b, p, sign, groups, gpr);
    return cudaGetLastError();
}

cudaError_t launch_count_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *flags, const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 15) / 16;
    const int64_t groups = (int64_t)gpr * p.height;
    if (n_layers <= 0 || groups == 0) return cudaSuccess;
    if (n_layers > kPackedLimit) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)blocks_for(groups);
    if (p.count_bits == 16)
        count_texture_kernel<uint16_t><<<grid, kThreads, 0, s>>>(tex, n_layers, p, sign, flags, groups, gpr);
    else
        count_texture_kernel<uint32_t><<<grid, kThreads, 0, s>>>(tex, n_layers, p, sign, flags, groups, gpr);
    return cudaGetLastError();
}

cudaError_t launch_convert_to_array(const void *src, int64_t pitch, int64_t member_stride,
                                    cudaSurfaceObject_t surf, int texels_per_row, int height, int n_layers,
                                    cudaStream_t s) {
    const int64_t texels = (int64_t)texels_per_row * height * n_layers;
    if (texels == 0) return cudaSuccess;
    convert_to_array_kernel<<<(unsigned)blocks_for(texels), kThreads, 0, s>>>(
        static_cast<const uint8_t *>(src), pitch, member_stride, surf, texels_per_row, height, texels);
    return cudaGetLastError();
}

cudaError_t launch_depth_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *, const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 3) / 4;
    const int64_t groups = (int64_t)gpr * p.height;
    if (n_layers <= 0 || groups == 0) return cudaSuccess;
    depth_texture_kernel<<<(unsigned)blocks_for(groups), kThreads, 0, s>>>(tex, n_layers, p, sign, groups, gpr);
    return cudaGetLastError();
}

}  // namespace cpt
