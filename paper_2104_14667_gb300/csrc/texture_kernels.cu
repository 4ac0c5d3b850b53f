// texture_kernels.cu -- the texture (image) read path: the accumulation
// step over members held as layers of a cudaArray, and the hand-written
// buffer-to-array conversion (Section 4's layout transform) through a
// surface object.
#include <algorithm>

#include "device_common.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;
constexpr int kPackedLimit = 255;   // members a packed byte counter can hold

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
// and stores the texel into the layered cudaArray through a surface object,
// a warp taking 32 consecutive texels of a row.  (Warps over 4 x 8 texel
// blocks converted 1.9 TB/s of source against 2.1 for rows; four texels per
// thread with every load issued first gave 2.16 / 1.75 TB/s for masks /
// depths against 2.16 / 2.18: the surface stores, not the loads in flight,
// set the rate.)
__global__ void __launch_bounds__(kThreads)
convert_to_array_kernel(const uint8_t *src, int64_t pitch, int64_t member_stride, cudaSurfaceObject_t surf,
                        int texels_per_row, int height, int64_t texels) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < texels;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / texels_per_row;
        const int x = (int)(t - row * texels_per_row);
        const int layer = (int)(row / height);
        const int y = (int)(row - (int64_t)layer * height);
        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src + layer * member_stride + (int64_t)y * pitch + x * 16));
        surf2DLayeredwrite(v, surf, x * 16, y, layer);
    }
}

inline int64_t blocks_for(int64_t groups) {
    int64_t blocks = (groups + kThreads - 1) / kThreads;
    return blocks < 1 ? 1 : (blocks > 0x7FFFFFFF ? 0x7FFFFFFF : blocks);
}

}  // namespace

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
