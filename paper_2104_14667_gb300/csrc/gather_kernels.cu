// gather_kernels.cu -- the server's overflow upload: a cycle's distinct
// overflow rasters, scattered over the pinned host part, gathered into one
// device staging half by a single launch on the copy stream.  The kernel
// reads host memory through its device mapping over the host link, so one
// launch replaces one copy call per raster (a cycle moves about a thousand).
#include <algorithm>

#include "internal.cuh"

namespace cpt {
namespace {

constexpr int kThreads = 256;

// dst + i * stride <- src + ids[i] * stride, vecs_per_raster 16-byte vectors
// each; consecutive threads take consecutive vectors of one raster.
__global__ void __launch_bounds__(kThreads)
gather_rasters_kernel(uint8_t *dst, const uint8_t *src, const int32_t *ids, int n, int64_t stride,
                      int64_t vecs_per_raster) {
    const int64_t total = vecs_per_raster * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / vecs_per_raster);
        const int64_t v = t - (int64_t)i * vecs_per_raster;
        const uint4 x = __ldcs(reinterpret_cast<const uint4 *>(src + (int64_t)ids[i] * stride) + v);
        reinterpret_cast<uint4 *>(dst + (int64_t)i * stride)[v] = x;
    }
}

}  // namespace

cudaError_t launch_gather_rasters(void *dst, const void *src, const int32_t *ids, int n, int64_t stride,
                                  int64_t raster_bytes, const DeviceCaps &caps, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t vecs = raster_bytes / 16;
    // two CTAs per SM: enough loads in flight for the link, and room left for
    // the compute kernels it overlaps
    const int64_t blocks = std::min<int64_t>((vecs * n + kThreads - 1) / kThreads, (int64_t)caps.num_sms * 2);
    gather_rasters_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(
        static_cast<uint8_t *>(dst), static_cast<const uint8_t *>(src), ids, n, stride, vecs);
    return cudaGetLastError();
}

}  // namespace cpt
