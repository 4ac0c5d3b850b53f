// render_kernels.cu -- the display step: composite counts to overlap classes
// and colours (Fig. 1 caption: a blue saturation map where high overlap is
// high saturation, and the frequency of overlap classes), or depth sums to a
// mean depth.  One thread per output pixel; outputs are dense row-major.
#include "device_common.cuh"
#include "overlap_class.cuh"
#include "class_histogram.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;
constexpr int kHistCtasPerSm = 4;   // resident CTAs of the histogram render (64 registers, 41 KB of shared memory)

// Histogram of overlap classes (Fig. 1 caption): every warp counts into its
// own 256 bins in shared memory, a thread adds runs of equal classes at once,
// and each block adds its bins into the 64-bit global histogram at the end.
struct HistBins {
    uint32_t warp[kThreads / 32][256];
};

__device__ __forceinline__ void hist_init(HistBins &h) {
    for (int i = threadIdx.x; i < (kThreads / 32) * 256; i += blockDim.x) (&h.warp[0][0])[i] = 0;
}

__device__ __forceinline__ void hist_flush(HistBins &h, unsigned long long *hist_out) {
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += h.warp[w][b];
        if (t) atomicAdd(hist_out + b, (unsigned long long)t);
    }
}

template <typename CountT, bool kHist>
__global__ void __launch_bounds__(kThreads)
render_counts_kernel(Plane p, ClassDivisor div, CountT *counts_out, uint8_t *bucket_out,
                     uint32_t *rgba_out, Lut lut, unsigned long long *hist_out) {
    __shared__ uint32_t table[256];
    __shared__ HistBins bins;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) table[i] = lut.rgba[i];
    if (kHist) hist_init(bins);
    __syncthreads();
    uint32_t *my_bins = bins.warp[threadIdx.x / 32];
    const CountT *plane = static_cast<const CountT *>(p.data);
    const int64_t total = (int64_t)p.width * p.height;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / p.width);
        const int x = (int)(i - (int64_t)y * p.width);
        const uint32_t c = plane[(int64_t)y * p.pitch + x];
        const uint32_t b = overlap_class(c, div);
        if (counts_out) counts_out[i] = (CountT)c;
        if (bucket_out) bucket_out[i] = (uint8_t)b;
        if (rgba_out) rgba_out[i] = table[b];
        if (kHist) atomicAdd(my_bins + b, 1u);
    }
    if (kHist) hist_flush(bins, hist_out);
}

// 16 pixels of one row per thread, 16-byte stores; used when the width is a
// multiple of 16 and every output is 16-byte aligned, so every dense output
// row starts on a 16-byte boundary.
template <typename CountT>
__global__ void __launch_bounds__(kThreads)
render_counts_vec_kernel(Plane p, ClassDivisor div, CountT *counts_out, uint8_t *bucket_out,
                         uint32_t *rgba_out, Lut lut) {
    __shared__ uint32_t table[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) table[i] = lut.rgba[i];
    __syncthreads();
    const CountT *plane = static_cast<const CountT *>(p.data);
    const int gpr = p.width / 16;
    const int64_t groups = (int64_t)gpr * p.height;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(g / gpr);
        const int x0 = (int)(g - (int64_t)y * gpr) * 16;
        const int64_t out = (int64_t)y * p.width + x0;
        uint32_t c[16];
        const uint4 *src = reinterpret_cast<const uint4 *>(plane + (int64_t)y * p.pitch + x0);
        if constexpr (sizeof(CountT) == 2) {
            const uint4 a = src[0], b = src[1];
            const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c[2 * k] = w[k] & 0xFFFFu;
                c[2 * k + 1] = w[k] >> 16;
            }
            if (counts_out) {
                uint4 *d = reinterpret_cast<uint4 *>(counts_out + out);
                d[0] = a;
                d[1] = b;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = src[q];
                c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
                if (counts_out) reinterpret_cast<uint4 *>(counts_out + out)[q] = v;
            }
        }
        uint32_t b[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) b[j] = overlap_class(c[j], div);
        if (bucket_out) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                w[q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | (b[4 * q + 3] << 24);
            *reinterpret_cast<uint4 *>(bucket_out + out) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (rgba_out) {
            uint4 *d = reinterpret_cast<uint4 *>(rgba_out + out);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                d[q] = make_uint4(table[b[4 * q]], table[b[4 * q + 1]], table[b[4 * q + 2]], table[b[4 * q + 3]]);
        }
    }
}

// render_counts_vec_kernel with the class histogram: the loop runs over warp
// items (32 consecutive groups, one per lane) so that every lane of a warp
// takes part in the folds of its counters (class_histogram.cuh); a group is
// classified, coloured and counted a quarter at a time.  The grid is one
// wave of resident CTAs, so that the per-block hand-over of the totals stays
// short.
template <typename CountT>
__global__ void __launch_bounds__(kThreads, kHistCtasPerSm)
render_counts_vec_hist_kernel(Plane p, ClassDivisor div, CountT *counts_out, uint8_t *bucket_out,
                              uint32_t *rgba_out, Lut lut, unsigned long long *hist_out) {
    __shared__ uint32_t table[256];
    __shared__ __align__(16) uint8_t s_hist[(kThreads / 32) * kHistWarpBytes];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *cnt = s_hist + warp * kHistWarpBytes;
    uint8_t *row = cnt + (lane / kHistLanesPerRow) * 256;
    const uint32_t key = (uint32_t)(lane / kHistLanesPerRow) << 2;
    uint32_t *tot = reinterpret_cast<uint32_t *>(cnt + kHistCounterBytes);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) table[i] = lut.rgba[i];
    for (int i = threadIdx.x; i < (kThreads / 32) * kHistWarpBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(s_hist)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const CountT *plane = static_cast<const CountT *>(p.data);
    const int gpr = p.width / 16;
    const int64_t groups = (int64_t)gpr * p.height;
    const bool packed = p.pitch == p.width;   // group g's counts at 16 g
    int since_fold = 0;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + warp * 32; base < groups;
         base += (int64_t)gridDim.x * blockDim.x) {
        if (since_fold == kHistFoldItems) {
            hist_fold(cnt, tot, lane);
            since_fold = 0;
        }
        ++since_fold;
        const int64_t g = base + lane;
        if (g >= groups) continue;
        const int64_t out = g * 16;   // the width is a multiple of 16: dense outputs
        const CountT *at = plane + out;
        if (!packed) {
            const int y = (int)(g / gpr);
            at = plane + (int64_t)y * p.pitch + (int)(g - (int64_t)y * gpr) * 16;
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(at);
        uint32_t c[16];
        if constexpr (sizeof(CountT) == 2) {
            const uint4 a = src[0], b = src[1];
            const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c[2 * k] = w[k] & 0xFFFFu;
                c[2 * k + 1] = w[k] >> 16;
            }
            if (counts_out) {
                uint4 *d = reinterpret_cast<uint4 *>(counts_out + out);
                d[0] = a;
                d[1] = b;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = src[q];
                c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
                if (counts_out) reinterpret_cast<uint4 *>(counts_out + out)[q] = v;
            }
        }
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t b0 = overlap_class(c[4 * q], div), b1 = overlap_class(c[4 * q + 1], div);
            const uint32_t b2 = overlap_class(c[4 * q + 2], div), b3 = overlap_class(c[4 * q + 3], div);
            w[q] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
            hist_count_quarter(row, key, b0, b1, b2, b3);
            if (rgba_out)
                reinterpret_cast<uint4 *>(rgba_out + out)[q] = make_uint4(table[b0], table[b1], table[b2], table[b3]);
        }
        if (bucket_out) *reinterpret_cast<uint4 *>(bucket_out + out) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    hist_fold(cnt, tot, lane);
    __syncthreads();
    hist_emit_block(s_hist, kThreads / 32, hist_out);
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

template <bool kHist>
cudaError_t render_counts_t(const Plane &p, uint64_t n_members, void *counts_out, uint8_t *bucket_out,
                            uint32_t *rgba_out, const Lut &lut, unsigned long long *hist_out,
                            const DeviceCaps &caps, cudaStream_t s) {
    const ClassDivisor div = class_divisor(n_members);
    const int64_t total = (int64_t)p.width * p.height;
    const bool aligned = ((reinterpret_cast<uintptr_t>(counts_out) | reinterpret_cast<uintptr_t>(bucket_out) |
                           reinterpret_cast<uintptr_t>(rgba_out)) % 16) == 0;
    const bool vec = p.width % 16 == 0 && aligned;
    const int64_t groups = total / 16;
    if (kHist && vec) {
        const unsigned grid = std::min<unsigned>(grid_for(groups, caps), (unsigned)caps.num_sms * kHistCtasPerSm);
        if (p.count_bits == 16)
            render_counts_vec_hist_kernel<uint16_t><<<grid, kThreads, 0, s>>>(
                p, div, static_cast<uint16_t *>(counts_out), bucket_out, rgba_out, lut, hist_out);
        else
            render_counts_vec_hist_kernel<uint32_t><<<grid, kThreads, 0, s>>>(
                p, div, static_cast<uint32_t *>(counts_out), bucket_out, rgba_out, lut, hist_out);
    } else if (!kHist && vec) {
        if (p.count_bits == 16)
            render_counts_vec_kernel<uint16_t><<<grid_for(groups, caps), kThreads, 0, s>>>(
                p, div, static_cast<uint16_t *>(counts_out), bucket_out, rgba_out, lut);
        else
            render_counts_vec_kernel<uint32_t><<<grid_for(groups, caps), kThreads, 0, s>>>(
                p, div, static_cast<uint32_t *>(counts_out), bucket_out, rgba_out, lut);
    } else if (p.count_bits == 16) {
        render_counts_kernel<uint16_t, kHist><<<grid_for(total, caps), kThreads, 0, s>>>(
            p, div, static_cast<uint16_t *>(counts_out), bucket_out, rgba_out, lut, hist_out);
    } else {
        render_counts_kernel<uint32_t, kHist><<<grid_for(total, caps), kThreads, 0, s>>>(
            p, div, static_cast<uint32_t *>(counts_out), bucket_out, rgba_out, lut, hist_out);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_counts(const Plane &p, uint64_t n_members, void *counts_out,
                                 uint8_t *bucket_out, uint32_t *rgba_out, const Lut &lut,
                                 const DeviceCaps &caps, cudaStream_t s, uint64_t *hist_out) {
    if (hist_out) {
        cudaError_t e = cudaMemsetAsync(hist_out, 0, 256 * sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
        return render_counts_t<true>(p, n_members, counts_out, bucket_out, rgba_out, lut,
                                     reinterpret_cast<unsigned long long *>(hist_out), caps, s);
    }
    if (!counts_out && !bucket_out && !rgba_out) return cudaSuccess;
    return render_counts_t<false>(p, n_members, counts_out, bucket_out, rgba_out, lut, nullptr, caps, s);
}

cudaError_t launch_render_mean(const Plane &p, uint64_t n_members, float *mean_out,
                               const DeviceCaps &caps, cudaStream_t s) {
    if (!mean_out) return cudaSuccess;
    const int64_t total = (int64_t)p.width * p.height;
    render_mean_kernel<<<grid_for(total, caps), kThreads, 0, s>>>(p, n_members, mean_out);
    return cudaGetLastError();
}

}  // namespace cpt
