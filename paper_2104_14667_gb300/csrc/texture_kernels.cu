// texture_kernels.cu -- the texture (image) read path: the accumulation
// step over members held as layers of a cudaArray, and the hand-written
// buffer-to-array conversion (Section 4's layout transform) through a
// surface object.
#include <algorithm>

#include "device_common.cuh"

namespace cpt {
namespace {

constexpr int kPackedLimit = 255;   // members a packed byte counter can hold

// Both texture-path kernels walk the layered array in 2-D tiles of texels
// rather than along rows: the array is stored in tiles of rows (block
// linear), and a CTA that covers a few texels of many rows reads and writes
// whole tiles.  Measured at 4096 x 4096 x 32 layers, alone on the GPU: the
// texture count moved 5.44 TB/s of member bytes with 4 x 32 tiles against
// 4.78 with a CTA per row, and the conversion 3.19 TB/s of source (6.4 TB/s
// of DRAM traffic, read plus write) with 16 x 8 tiles against 2.60 for a
// flat, row-ordered index.  Several layers per conversion thread were slower
// (1.8-2.4 TB/s): the stores, not the loads in flight, set the pace.
constexpr int kCountTileW = 4, kCountTileH = 32;
constexpr int kConvertTileW = 16, kConvertTileH = 8;
constexpr int kTileThreads = 128;
static_assert(kCountTileW * kCountTileH == kTileThreads && kConvertTileW * kConvertTileH == kTileThreads,
              "tiles fill a CTA");

// Texture path: member `layer` of the batch is layer `layer` of a layered
// cudaArray whose texels are 16 bytes (16 mask pixels).  Texels past the
// raster's right edge hold padding and are masked off.  One thread per texel
// column (x, y), over every layer.
template <typename CountT>
__global__ void __launch_bounds__(kTileThreads)
count_texture_kernel(cudaTextureObject_t tex, int n_layers, Plane p, int sign, int *flags, int groups_per_row) {
    const int gx = blockIdx.x * kCountTileW + (int)(threadIdx.x % kCountTileW);
    const int y = blockIdx.y * kCountTileH + (int)(threadIdx.x / kCountTileW);
    if (gx >= groups_per_row || y >= p.height) return;
    CountT *plane = static_cast<CountT *>(p.data);
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

__global__ void __launch_bounds__(kTileThreads)
depth_texture_kernel(cudaTextureObject_t tex, int n_layers, Plane p, int sign, int groups_per_row) {
    const int gx = blockIdx.x * kCountTileW + (int)(threadIdx.x % kCountTileW);
    const int y = blockIdx.y * kCountTileH + (int)(threadIdx.x / kCountTileW);
    if (gx >= groups_per_row || y >= p.height) return;
    float *plane = static_cast<float *>(p.data);
    const int x0 = gx * 4;
    const int valid = min(4, p.width - x0);
    const float u = gx + 0.5f, v = y + 0.5f;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int layer = 0; layer < n_layers; ++layer) {
        const float4 t = tex2DLayered<float4>(tex, u, v, layer);
        acc[0] += t.x;
        acc[1] += valid > 1 ? t.y : 0.f;
        acc[2] += valid > 2 ? t.z : 0.f;
        acc[3] += valid > 3 ? t.w : 0.f;
    }
    apply_depth_group(plane + (int64_t)y * p.pitch + x0, valid, acc, sign);
}

// Layout conversion by hand (the buffer-to-image transform of Section 4):
// one thread per 16-byte texel of one layer, a 16-byte streaming load from
// the linear raster and a surface store into the layered array, over a grid
// of (tile column, tile row, layer).
__global__ void __launch_bounds__(kTileThreads)
convert_to_array_kernel(const uint8_t *src, int64_t pitch, int64_t member_stride, cudaSurfaceObject_t surf,
                        int texels_per_row, int height) {
    const int x = blockIdx.x * kConvertTileW + (int)(threadIdx.x % kConvertTileW);
    const int y = blockIdx.y * kConvertTileH + (int)(threadIdx.x / kConvertTileW);
    const int layer = blockIdx.z;
    if (x >= texels_per_row || y >= height) return;
    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src + layer * member_stride + (int64_t)y * pitch + x * 16));
    surf2DLayeredwrite(v, surf, x * 16, y, layer);
}

// Grid of (tile columns, tile rows[, layers]); false when a dimension is
// beyond the launch limits (never for arrays within the texture limits).
inline bool tile_grid(dim3 *g, int cols, int rows, int tw, int th, int layers) {
    *g = dim3((unsigned)((cols + tw - 1) / tw), (unsigned)((rows + th - 1) / th), (unsigned)layers);
    return g->y <= 65535 && g->z <= 65535;
}

}  // namespace

cudaError_t launch_count_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *flags, const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 15) / 16;
    if (n_layers <= 0 || p.height <= 0 || gpr == 0) return cudaSuccess;
    if (n_layers > kPackedLimit) return cudaErrorInvalidValue;
    dim3 grid;
    if (!tile_grid(&grid, gpr, p.height, kCountTileW, kCountTileH, 1)) return cudaErrorInvalidValue;
    if (p.count_bits == 16)
        count_texture_kernel<uint16_t><<<grid, kTileThreads, 0, s>>>(tex, n_layers, p, sign, flags, gpr);
    else
        count_texture_kernel<uint32_t><<<grid, kTileThreads, 0, s>>>(tex, n_layers, p, sign, flags, gpr);
    return cudaGetLastError();
}

cudaError_t launch_convert_to_array(const void *src, int64_t pitch, int64_t member_stride,
                                    cudaSurfaceObject_t surf, int texels_per_row, int height, int n_layers,
                                    cudaStream_t s) {
    if (texels_per_row <= 0 || height <= 0 || n_layers <= 0) return cudaSuccess;
    dim3 grid;
    if (!tile_grid(&grid, texels_per_row, height, kConvertTileW, kConvertTileH, n_layers)) return cudaErrorInvalidValue;
    convert_to_array_kernel<<<grid, kTileThreads, 0, s>>>(static_cast<const uint8_t *>(src), pitch, member_stride,
                                                          surf, texels_per_row, height);
    return cudaGetLastError();
}

cudaError_t launch_depth_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *, const DeviceCaps &, cudaStream_t s) {
    const int gpr = (p.width + 3) / 4;
    if (n_layers <= 0 || p.height <= 0 || gpr == 0) return cudaSuccess;
    dim3 grid;
    if (!tile_grid(&grid, gpr, p.height, kCountTileW, kCountTileH, 1)) return cudaErrorInvalidValue;
    depth_texture_kernel<<<grid, kTileThreads, 0, s>>>(tex, n_layers, p, sign, gpr);
    return cudaGetLastError();
}

}  // namespace cpt
