// internal.cuh -- declarations shared by the library's translation units.
// Not installed; the public interface is include/composite.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

namespace cpt {

// Device error flags (int32 each), cleared by composite_clear.
enum FlagIndex { kFlagUnderflow = 0, kFlagTimeout = 1, kFlagCount = 4 };

// A raster batch as a kernel sees it: n rasters of height rows, row y of
// member m at base + m * member_stride + y * row_pitch (bytes).
struct RasterBatch {
    const void *base;
    int64_t member_stride;
    int64_t row_pitch;
    int32_t n;
};

// The composite plane: height rows of `pitch` elements (pitch is width
// rounded up to one 16-byte vector), element uint16/uint32 counts or float32
// depth sums.
struct Plane {
    void *data;
    int64_t pitch;      // elements
    int32_t width;
    int32_t height;
    int32_t count_bits; // 16, 32, or 0 for float32 sums
};

struct DeviceCaps {
    int num_sms;
};

// Linear read path: 16-byte loads straight from the batch (device memory).
cudaError_t launch_count_linear(const RasterBatch &b, const Plane &p, int sign, int *flags,
                                const DeviceCaps &caps, cudaStream_t s);
cudaError_t launch_depth_linear(const RasterBatch &b, const Plane &p, int sign, int *flags,
                                const DeviceCaps &caps, cudaStream_t s);
// Bit-packed masks (pixel x = bit x & 7 of byte x >> 3 of its row); the
// plane pitch must be a multiple of 32 pixels.
cudaError_t launch_count_bits(const RasterBatch &b, const Plane &p, int sign, int *flags,
                              const DeviceCaps &caps, cudaStream_t s);

// Texture read path: a layered cudaArray with 16-byte texels (uint4 for
// masks, float4 for depths); n_layers members.
cudaError_t launch_count_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *flags, const DeviceCaps &caps, cudaStream_t s);
cudaError_t launch_depth_texture(cudaTextureObject_t tex, int n_layers, const Plane &p, int sign,
                                 int *flags, const DeviceCaps &caps, cudaStream_t s);
// dst + i * stride <- src + ids[i] * stride, raster_bytes (a multiple of 16)
// each, i < n; src may be host-mapped pinned memory.  16-byte aligned.
cudaError_t launch_gather_rasters(void *dst, const void *src, const int32_t *ids, int n, int64_t stride,
                                  int64_t raster_bytes, const DeviceCaps &caps, cudaStream_t s);
// Linear rasters (16-byte aligned base, pitch and stride) -> the layers of a
// cudaArray of 16-byte texels, through a surface object.
cudaError_t launch_convert_to_array(const void *src, int64_t pitch, int64_t member_stride,
                                    cudaSurfaceObject_t surf, int texels_per_row, int height, int n_layers,
                                    cudaStream_t s);

// TMA read path: tensor map over the batch, tiles staged in shared memory.
// The tensor map must come from encode_tma_map for the same batch.
// box_bytes: the x extent of a box in bytes (64, 128 or 256); a box is always
// 2 KiB per member (box_bytes x 2048/box_bytes rows) x 16 members.
cudaError_t launch_count_tma(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                             int *flags, uint64_t timeout_ns, int box_bytes, const DeviceCaps &caps,
                             cudaStream_t s);
cudaError_t launch_depth_tma(const CUtensorMap &map, const RasterBatch &b, const Plane &p, int sign,
                             int *flags, uint64_t timeout_ns, int box_bytes, const DeviceCaps &caps,
                             cudaStream_t s);
bool tma_box_supported(int box_bytes);
// Bit-packed masks through cp.async.bulk copies of contiguous 2 KiB pieces
// into a shared-memory ring (device memory only).  Needs unpadded rows (width
// a multiple of 32, row pitch width / 8), a 16-byte aligned base and member
// stride, and width / 32 * height a multiple of 4; bits_bulk_compatible says.
bool bits_bulk_compatible(const RasterBatch &b, int width, int height);
cudaError_t launch_count_bits_bulk(const RasterBatch &b, const Plane &p, int sign, int *flags, uint64_t timeout_ns,
                                   const DeviceCaps &caps, cudaStream_t s);
// One thread waits, bounded by timeout_ns, on an mbarrier nothing arrives at
// (the same wait the TMA kernels use); status[0] = gave up, status[1] = ns.
cudaError_t launch_bounded_wait_selftest(uint64_t timeout_ns, unsigned long long *status, cudaStream_t s);
// Returns 0 on success; a CUresult otherwise.  elem_bytes 1 (masks) or 4.
int encode_tma_map(CUtensorMap *map, const RasterBatch &b, int width, int height, int elem_bytes,
                   int box_bytes);

// Render: counts -> dense counts / bucket / rgba, or sums -> mean.
struct Lut {
    uint32_t rgba[256];
};
// hist_out (device, 256 x uint64, may be NULL): zeroed, then the number of
// pixels in every overlap class, counted in the same pass.
cudaError_t launch_render_counts(const Plane &p, uint64_t n_members, void *counts_out,
                                 uint8_t *bucket_out, uint32_t *rgba_out, const Lut &lut,
                                 const DeviceCaps &caps, cudaStream_t s, uint64_t *hist_out = nullptr);
cudaError_t launch_render_mean(const Plane &p, uint64_t n_members, float *mean_out,
                               const DeviceCaps &caps, cudaStream_t s);

// Sets the calling thread's context-free error message (the one that
// composite_last_error(NULL) returns).
void set_thread_error(const char *message);

// Host-side fault injection for tests: the environment variable
// CPT_FAULT_INJECT holds a comma-separated list of sites -- staging_alloc,
// pinned_ring, ingest_threads, host_register, engine_plane, server_stage --
// and a listed site behaves as if its host-side request (a device or pinned
// allocation, the ingest threads, the page-locking of a pageable batch) had
// been refused; engine_submit makes every engine submit fail after its
// descriptors are uploaded and before its launch.  Nothing on the device is
// affected.
bool fault_injected(const char *site);
// Indexed sites in the same list, written "site=K": returns K when the site
// is listed, -1 otherwise.  chunk_fail=K makes chunk K (from 0) of every add
// or remove fail as if its upload had been refused, after chunks 0..K-1 were
// queued; server_chunk_fail=K does the same to overflow chunk K of every
// server cycle, engine_chunk_fail=K to staging chunk K of an engine submit's
// host ops.  Each fails on the host, before that chunk's work is queued.
int64_t fault_injected_value(const char *site);

// NVTX range around a host-side phase (a call, a pipeline chunk), for
// timeline profilers; a no-op call when no profiler is attached.
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Status for a C++ exception caught at an entry point of the C ABI (none may
// cross it), called from the catch handler: CPT_ENOMEM for a failed host
// allocation, CPT_EINVAL for anything else; the message goes to
// set_thread_error.
int abi_exception_status() noexcept;

}  // namespace cpt
