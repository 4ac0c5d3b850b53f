// static_scratch.cu -- composite_oneshot_static: a one-shot composite of
// device-resident rasters that allocates nothing.
//
// Some callers cannot call cudaMalloc: an interactive viewer's per-frame
// render callback must not risk the implicit device synchronisation an
// allocation can bring, and a host application that owns all device memory
// through its own pool may forbid libraries from allocating at all.  This
// entry point runs the same accumulation and render kernels as the context
// path, but its composite plane and device flags live in file-scope
// __device__ arrays of a fixed size instead of memory the library allocates.
//
// In host code the names g_static_plane / g_static_flags are host-side
// stand-ins, not device addresses; the device addresses are looked up once
// per device with cudaGetSymbolAddress (with that device current) on the
// first call made on that device, and passed to the kernels.
#include <mutex>

#include "composite.h"
#include "internal.cuh"

namespace {

constexpr int64_t kMaxPlanePixels = CPT_ONESHOT_MAX_PIXELS;
constexpr int kMaxDevices = 64;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) uint32_t g_static_plane[kMaxPlanePixels];
static __device__ __align__(256) int g_static_flags[cpt::kFlagCount];

struct DeviceScratch {
    bool ready = false;
    uint32_t *plane = nullptr;
    int *flags = nullptr;
    int num_sms = 0;
    int device = 0;
};

std::mutex g_mutex;
DeviceScratch g_scratch[kMaxDevices];

int reject(int code, const char *message) {
    cpt::set_thread_error(message);
    return code;
}

// True when p is device (or managed) memory the current device can address
// as its own: kernels here read and write these pointers directly, so host
// memory or another GPU's memory must be turned away before any launch.
bool on_current_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device addresses of the static scratch on the current device.
int resolve(DeviceScratch *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(CPT_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(CPT_EINVAL, "device ordinal beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceScratch &s = g_scratch[dev];
    if (!s.ready) {
        void *plane = nullptr, *flags = nullptr;
        e = cudaGetSymbolAddress(&plane, g_static_plane);
        if (e != cudaSuccess) return reject(CPT_ECUDA, cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&flags, g_static_flags);
        if (e != cudaSuccess) return reject(CPT_ECUDA, cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return reject(CPT_ECUDA, cudaGetErrorString(e));
        s.plane = static_cast<uint32_t *>(plane);
        s.flags = static_cast<int *>(flags);
        s.device = dev;
        s.ready = true;
    }
    *out = s;
    return CPT_OK;
}

}  // namespace

extern "C" int composite_oneshot_static(const void *members, int32_t n_members,
                                        int64_t member_stride_bytes, int32_t row_pitch_bytes,
                                        int32_t width, int32_t height, uint32_t *counts_out,
                                        uint8_t *bucket_out, uint8_t *rgba_out,
                                        const uint8_t *lut_rgba, void *cuda_stream) try {
    if (width <= 0 || height <= 0) return reject(CPT_EINVAL, "raster is empty");
    if (n_members < 0) return reject(CPT_EINVAL, "n_members < 0");
    const int64_t pitch_px = ((int64_t)width + 15) / 16 * 16;
    if (pitch_px * height > kMaxPlanePixels)
        return reject(CPT_EINVAL, "raster exceeds the static scratch: roundup(width, 16) * height must be "
                                  "at most CPT_ONESHOT_MAX_PIXELS");
    if (n_members > 0) {
        if (!members) return reject(CPT_EINVAL, "members is NULL");
        if (row_pitch_bytes < width || member_stride_bytes < (int64_t)row_pitch_bytes * height)
            return reject(CPT_EINVAL, "row pitch or member stride too small");
        if ((reinterpret_cast<uintptr_t>(members) % 16) || (row_pitch_bytes % 16) || (member_stride_bytes % 16))
            return reject(CPT_EINVAL, "members, row pitch and member stride must be 16-byte aligned");
    }
    if ((reinterpret_cast<uintptr_t>(counts_out) % 4) || (reinterpret_cast<uintptr_t>(rgba_out) % 4))
        return reject(CPT_EINVAL, "counts_out and rgba_out must be 4-byte aligned");

    DeviceScratch s;
    int rc = resolve(&s);
    if (rc) return rc;
    if (n_members > 0 && !on_current_device(members, s.device))
        return reject(CPT_EINVAL, "members must be device memory of the current device");
    const void *outs[3] = {counts_out, bucket_out, rgba_out};
    for (const void *o : outs)
        if (o && !on_current_device(o, s.device))
            return reject(CPT_EINVAL, "outputs must be device memory of the current device");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    cpt::Lut lut;
    for (int b = 0; b < 256; ++b) {
        const uint8_t *e = lut_rgba ? lut_rgba + 4 * b : nullptr;
        const uint32_t r = e ? e[0] : 255u - b, g = e ? e[1] : 255u - b, bl = e ? e[2] : 255u, al = e ? e[3] : 255u;
        lut.rgba[b] = r | (g << 8) | (bl << 16) | (al << 24);
    }
    cpt::Plane plane{s.plane, pitch_px, width, height, 32};
    cpt::DeviceCaps caps{s.num_sms};
    // The scratch keeps the previous call's contents: clear the part in use.
    cudaError_t e = cudaMemsetAsync(s.plane, 0, (size_t)pitch_px * height * sizeof(uint32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.flags, 0, cpt::kFlagCount * sizeof(int), stream);
    if (e == cudaSuccess && n_members > 0) {
        cpt::RasterBatch batch{members, member_stride_bytes, row_pitch_bytes, n_members};
        e = cpt::launch_count_linear(batch, plane, +1, s.flags, caps, stream);
    }
    if (e == cudaSuccess)
        e = cpt::launch_render_counts(plane, (uint64_t)n_members, counts_out, bucket_out,
                                      reinterpret_cast<uint32_t *>(rgba_out), lut, caps, stream);
    if (e != cudaSuccess) return reject(CPT_ECUDA, cudaGetErrorString(e));
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}
