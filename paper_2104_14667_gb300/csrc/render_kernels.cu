// render_kernels.cu -- the display step: composite counts to overlap classes
// and colours (Fig. 1 caption: a blue saturation map where high overlap is
// high saturation, and the frequency of overlap classes), or depth sums to a
// mean depth.  One thread per output pixel; outputs are dense row-major.
#include "device_common.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;

// floor(255 * c / n) for 0 <= c <= n, exact.  With n < 2^24 the product fits
// in 32 bits; larger n take the 64-bit path.
__device__ __forceinline__ uint32_t overlap_class(uint32_t c, uint64_t n) {
    if (n == 0) return 0;
    if (n < (1u << 24)) return (255u * c) / (uint32_t)n;
    return (uint32_t)((255ull * c) / n);
}

template <typename CountT>
__global__ void __launch_bounds__(kThreads)
render_counts_kernel(Plane p, uint64_t n_members, CountT *counts_out, uint8_t *bucket_out,
                     uint32_t *rgba_out, Lut lut) {
    __shared__ uint32_t table[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) table[i] = lut.rgba[i];
    __syncthreads();
    const CountT *plane = static_cast<const CountT *>(p.data);
    const int64_t total = (int64_t)p.width * p.height;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / p.width);
        const int x = (int)(i - (int64_t)y * p.width);
        const uint32_t c = plane[(int64_t)y * p.pitch + x];
        const uint32_t b = overlap_class(c, n_members);
        if (counts_out) counts_out[i] = (CountT)c;
        if (bucket_out) bucket_out[i] = (uint8_t)b;
        if (rgba_out) rgba_out[i] = table[b & 0xFFu];
    }
}

__global__ void __launch_bounds__(kThreads)
render_mean_kernel(Plane p, uint64_t n_members, float *mean_out) {
    const float *plane = static_cast<const float *>(p.data);
    const int64_t total = (int64_t)p.width * p.height;
    const float n = (float)n_members;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / p.width);
        const int x = (int)(i - (int64_t)y * p.width);
        mean_out[i] = n_members == 0 ? 0.0f : plane[(int64_t)y * p.pitch + x] / n;
    }
}

unsigned grid_for(int64_t total, const DeviceCaps &caps) {
    int64_t blocks = (total + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)caps.num_sms * 16;
    if (blocks > cap) blocks = cap;
    return (unsigned)(blocks < 1 ? 1 : blocks);
}

}  // namespace

cudaError_t launch_render_counts(const Plane &p, uint64_t n_members, void *counts_out,
                                 uint8_t *bucket_out, uint32_t *rgba_out, const Lut &lut,
                                 const DeviceCaps &caps, cudaStream_t s) {
    const int64_t total = (int64_t)p.width * p.height;
    if (!counts_out && !bucket_out && !rgba_out) return cudaSuccess;
    if (p.count_bits == 16)
        render_counts_kernel<uint16_t><<<grid_for(total, caps), kThreads, 0, s>>>(
            p, n_members, static_cast<uint16_t *>(counts_out), bucket_out, rgba_out, lut);
    else
        render_counts_kernel<uint32_t><<<grid_for(total, caps), kThreads, 0, s>>>(
            p, n_members, static_cast<uint32_t *>(counts_out), bucket_out, rgba_out, lut);
    return cudaGetLastError();
}

cudaError_t launch_render_mean(const Plane &p, uint64_t n_members, float *mean_out,
                               const DeviceCaps &caps, cudaStream_t s) {
    if (!mean_out) return cudaSuccess;
    const int64_t total = (int64_t)p.width * p.height;
    render_mean_kernel<<<grid_for(total, caps), kThreads, 0, s>>>(p, n_members, mean_out);
    return cudaGetLastError();
}

}  // namespace cpt
