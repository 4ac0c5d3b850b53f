// api.cu -- the C ABI of include/composite.h: contexts, the upload pipeline
// and the dispatch to the accumulation and render kernels.
//
// Pipeline (Section 4, Figs. 3 and 4, generalised from two receiving buffers
// to k): member chunk j goes to staging slot s = j mod k.  The copy stream
// waits for slot s to be released by the kernel that last read it, uploads
// the chunk, and records `ready`; the compute stream waits for `ready`,
// converts the layout if the read path needs it, runs the accumulation
// kernel and records `consumed`.  No host synchronisation sits between
// chunks: the ordering is all CUDA events, the remedy the paper gives for
// synchronisation stalls (Section 7.1).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "composite.h"
#include "copy_pool.cuh"
#include "internal.cuh"

using cpt::DeviceCaps;
using cpt::Lut;
using cpt::Plane;
using cpt::RasterBatch;

namespace {

thread_local std::string g_begin_error;

enum MemKind { kPageable = 0, kPinned = 1, kDevice = 2, kForeignDevice = 3 };
constexpr int kDefaultTmaBoxBytes = 256;
enum TraceKind { kTraceUpload = 0, kTraceConvert = 1, kTraceKernel = 2 };

struct Slot {
    uint8_t *stage = nullptr;         // device receiving buffer, C rasters
    cudaArray_t array = nullptr;      // texture path: the slot's layered array
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;     // the same array, written by the layout kernel
    cudaEvent_t ready = nullptr;      // upload (or conversion) into the slot done
    cudaEvent_t consumed = nullptr;   // the kernel that read the slot done
    uint8_t *ring = nullptr;          // pinned host ring slot (pageable inputs)
    cudaEvent_t ring_free = nullptr;  // upload out of the ring slot done
    bool ring_used = false;
};

struct TraceRec {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace

struct composite_ctx {
    int32_t width = 0, height = 0;
    composite_config cfg{};
    int elem = 1;              // bytes per raster element
    int vec_px = 16;           // pixels per 16-byte group
    int64_t pitch_px = 0;      // plane row pitch, elements
    int64_t row_bytes = 0;     // bytes of one raster row as the caller lays it out (unpadded)
    int64_t stage_pitch = 0;   // staging row pitch, bytes (a multiple of 16)
    int64_t member_bytes = 0;  // staging raster stride, bytes
    int slot_members = 0;      // rasters a staging slot holds: chunk_members, or the automatic depth's cap
    int call_chunk = 0;        // C of the current add/remove
    bool bits = false;         // masks are bit-packed
    Plane plane{};
    int *flags = nullptr;      // device flags
    int *h_flags = nullptr;    // pinned copy of the flags
    int64_t n_members = 0;
    bool poisoned = false;
    std::string poison_reason;   // why the context refuses work until a clear
    int64_t call_chunks = 0;     // chunks of the current add/remove queued so far
    int device = 0;
    DeviceCaps caps{};
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<Slot> slots;
    uint64_t next_slot = 0;
    int64_t ring_chunk = 0;
    std::unique_ptr<cpt::CopyPool> ingest;   // step a2 copy threads (pageable inputs)
    std::vector<void *> pending_unregister;  // registered batches whose uploads outlived their call
    uint8_t *out_scratch = nullptr;
    size_t out_scratch_bytes = 0;
    cudaEvent_t done_compute = nullptr, done_copy = nullptr;
    cudaEvent_t caller_ready = nullptr;   // the caller's work queued before a call
    std::vector<TraceRec> trace;
    std::vector<cudaEvent_t> trace_pool;
    size_t trace_used = 0;
    Lut default_lut{};
    std::string err;
};

namespace {

int fail(composite_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_begin_error = buf;
    return code;
}

int cuda_fail(composite_ctx *ctx, cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? CPT_ENOMEM : CPT_ECUDA;
    return fail(ctx, code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(ctx, call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int64_t timeout_ms(const composite_ctx *ctx) {
    return ctx->cfg.wait_timeout_ms > 0 ? ctx->cfg.wait_timeout_ms : 10000;
}

// Polls an event until it completes or the context's timeout runs out; after
// a short spin it sleeps between polls (tight polling loops were measured to
// slow host-to-device copies over the host link).
int wait_event(composite_ctx *ctx, cudaEvent_t ev) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms(ctx));
    for (unsigned spin = 0;; ++spin) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return CPT_OK;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "cudaEventQuery");
        if (std::chrono::steady_clock::now() > deadline)
            return fail(ctx, CPT_ETIMEOUT, "wait exceeded %lld ms", (long long)timeout_ms(ctx));
        if (spin < 200)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int trace_event(composite_ctx *ctx, cudaEvent_t *out) {
    if (ctx->trace_used == ctx->trace_pool.size()) {
        cudaEvent_t ev;
        CK(ctx, cudaEventCreate(&ev));
        ctx->trace_pool.push_back(ev);
    }
    *out = ctx->trace_pool[ctx->trace_used++];
    return CPT_OK;
}

// Opens a traced interval on stream s; close it with trace_close.
int trace_open(composite_ctx *ctx, int kind, cudaStream_t s) {
    if (!ctx->cfg.trace) return CPT_OK;
    TraceRec r{kind, nullptr, nullptr};
    int rc = trace_event(ctx, &r.a);
    if (rc) return rc;
    rc = trace_event(ctx, &r.b);
    if (rc) return rc;
    CK(ctx, cudaEventRecord(r.a, s));
    ctx->trace.push_back(r);
    return CPT_OK;
}

int trace_close(composite_ctx *ctx, cudaStream_t s) {
    if (!ctx->cfg.trace) return CPT_OK;
    CK(ctx, cudaEventRecord(ctx->trace.back().b, s));
    return CPT_OK;
}

// Poisons the context: every call but clear, load_counts, sync, trace_read
// and end returns CPT_ESTATE until composite_clear or composite_load_counts.
void poison(composite_ctx *ctx, const char *reason) {
    ctx->poisoned = true;
    ctx->poison_reason = reason;
}

int refuse_poisoned(composite_ctx *ctx) {
    return fail(ctx, CPT_ESTATE, "context poisoned: %s; clear it", ctx->poison_reason.c_str());
}

// Automatic chunk depth (chunk_members = 0).  A staging slot holds up to
// kAutoSlotBytes of rasters.  Each call is cut into about kAutoChunksPerCall
// chunks, no smaller than kAutoMinChunkBytes: the kernel of a call's last
// chunk has no later upload to hide under, so the share of kernel time left
// exposed is about one chunk in the number of chunks, while chunks too small
// pay a fixed cost per copy and launch.  The texture path's slots hold twice
// as much: each chunk is a conversion launch and a texture-fold launch over a
// layered array, and device-resident masks go through the slots too (4096^2 x
// 1024 resident: 2.09-2.10e12 member-px/s with 32 layers per chunk against
// 1.97-2.00e12 with 16; streamed, both at 0.985-0.991 of the link).
constexpr int64_t kAutoSlotBytes = 256ll << 20;
constexpr int64_t kAutoSlotBytesTexture = 512ll << 20;
constexpr int64_t kAutoMinChunkBytes = 16ll << 20;
constexpr int kAutoChunksPerCall = 32;

int auto_slot_members(int64_t member_bytes, int32_t read_path) {
    const int64_t slot = read_path == CPT_READ_TEXTURE ? kAutoSlotBytesTexture : kAutoSlotBytes;
    return (int)std::max<int64_t>(1, std::min<int64_t>(255, slot / member_bytes));
}

int chunk_for_call(const composite_ctx *ctx, int n) {
    if (ctx->cfg.chunk_members > 0) return ctx->cfg.chunk_members;
    const int cap = ctx->slot_members;
    const int floor_c = (int)std::min<int64_t>(cap, std::max<int64_t>(1, (kAutoMinChunkBytes + ctx->member_bytes - 1) / ctx->member_bytes));
    const int want = (n + kAutoChunksPerCall - 1) / kAutoChunksPerCall;
    return std::max(floor_c, std::min(cap, want));
}

// Called before the work of each chunk of an add or remove is queued.  From
// then on a failure leaves part of the call's rasters folded in, which
// apply() turns into a poisoned context.
int begin_chunk(composite_ctx *ctx) {
    if (cpt::fault_injected_value("chunk_fail") == ctx->call_chunks)
        return fail(ctx, CPT_ECUDA, "upload of chunk %lld refused (injected)", (long long)ctx->call_chunks);
    ++ctx->call_chunks;
    return CPT_OK;
}

// Memory kind of p as seen from `device`: device memory of another GPU is
// kForeignDevice (a kernel here cannot be assumed to reach it).
MemKind memory_kind(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kPageable;
    }
    switch (a.type) {
        case cudaMemoryTypeDevice:
            return a.device == device ? kDevice : kForeignDevice;
        case cudaMemoryTypeManaged:
            return kDevice;
        case cudaMemoryTypeHost:
            return kPinned;
        default:
            return kPageable;
    }
}

// Whether a kernel on `device` may write p: device memory of that device,
// managed memory, or pinned host memory mapped for the device.  Pageable
// host memory or another GPU's memory is turned away before any launch.
bool device_writable(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type == cudaMemoryTypeDevice) return a.device == device;
    return a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
}

Lut pack_lut(const uint8_t *rgba) {
    Lut l;
    for (int b = 0; b < 256; ++b)
        l.rgba[b] = (uint32_t)rgba[4 * b] | ((uint32_t)rgba[4 * b + 1] << 8) |
                    ((uint32_t)rgba[4 * b + 2] << 16) | ((uint32_t)rgba[4 * b + 3] << 24);
    return l;
}

int check_config(const composite_config &c) {
    if (c.read_path < CPT_READ_LINEAR || c.read_path > CPT_READ_TMA) return fail(nullptr, CPT_EINVAL, "read_path %d out of range", c.read_path);
    if (c.staging_buffers < 1 || c.staging_buffers > 8) return fail(nullptr, CPT_EINVAL, "staging_buffers %d not in 1..8", c.staging_buffers);
    if (c.chunk_members < 0 || c.chunk_members > 255) return fail(nullptr, CPT_EINVAL, "chunk_members %d not in 0..255", c.chunk_members);
    if (c.count_bits != 16 && c.count_bits != 32) return fail(nullptr, CPT_EINVAL, "count_bits %d is not 16 or 32", c.count_bits);
    if (c.mode != CPT_MODE_COUNT && c.mode != CPT_MODE_MEAN_DEPTH) return fail(nullptr, CPT_EINVAL, "mode %d out of range", c.mode);
    if (c.trace != 0 && c.trace != 1) return fail(nullptr, CPT_EINVAL, "trace must be 0 or 1");
    if (c.pinned_ring_bytes < 0 || c.wait_timeout_ms < 0) return fail(nullptr, CPT_EINVAL, "negative ring budget or timeout");
    if (c.host_read != 0 && c.host_read != 1) return fail(nullptr, CPT_EINVAL, "host_read must be 0 or 1");
    if (c.layout_converter != CPT_CONVERT_COPY && c.layout_converter != CPT_CONVERT_KERNEL)
        return fail(nullptr, CPT_EINVAL, "layout_converter %d out of range", c.layout_converter);
    if (c.mask_format != CPT_MASK_BYTES && c.mask_format != CPT_MASK_BITS)
        return fail(nullptr, CPT_EINVAL, "mask_format %d out of range", c.mask_format);
    if (c.mask_format == CPT_MASK_BITS && (c.mode != CPT_MODE_COUNT || c.read_path != CPT_READ_LINEAR))
        return fail(nullptr, CPT_EINVAL, "bit-packed masks need CPT_MODE_COUNT and CPT_READ_LINEAR");
    if (c.tma_box_bytes != 0 && !cpt::tma_box_supported(c.tma_box_bytes))
        return fail(nullptr, CPT_EINVAL, "tma_box_bytes %d is not 0, 64, 128 or 256", c.tma_box_bytes);
    if (c.ingest_threads < 0 || c.ingest_threads > 64)
        return fail(nullptr, CPT_EINVAL, "ingest_threads %d not in 0..64", c.ingest_threads);
    if (c.pageable_ingest < CPT_INGEST_AUTO || c.pageable_ingest > CPT_INGEST_REGISTER)
        return fail(nullptr, CPT_EINVAL, "pageable_ingest %d out of range", c.pageable_ingest);
    return CPT_OK;
}

void destroy(composite_ctx *ctx) {
    for (Slot &s : ctx->slots) {
        if (s.tex) cudaDestroyTextureObject(s.tex);
        if (s.surf) cudaDestroySurfaceObject(s.surf);
        if (s.array) cudaFreeArray(s.array);
        if (s.stage) cudaFree(s.stage);
        if (s.ring) cudaFreeHost(s.ring);
        if (s.ready) cudaEventDestroy(s.ready);
        if (s.consumed) cudaEventDestroy(s.consumed);
        if (s.ring_free) cudaEventDestroy(s.ring_free);
    }
    for (cudaEvent_t e : ctx->trace_pool) cudaEventDestroy(e);
    if (ctx->done_compute) cudaEventDestroy(ctx->done_compute);
    if (ctx->done_copy) cudaEventDestroy(ctx->done_copy);
    if (ctx->caller_ready) cudaEventDestroy(ctx->caller_ready);
    if (ctx->out_scratch) cudaFree(ctx->out_scratch);
    if (ctx->plane.data) cudaFree(ctx->plane.data);
    if (ctx->flags) cudaFree(ctx->flags);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    if (ctx->copy) cudaStreamDestroy(ctx->copy);
    delete ctx;
}

int setup(composite_ctx *ctx) {
    composite_config &c = ctx->cfg;
    CK(ctx, cudaGetDevice(&ctx->device));
    CK(ctx, cudaDeviceGetAttribute(&ctx->caps.num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    // NULL is the legacy default stream: the library's work is then ordered
    // with everything else the caller issues to it
    ctx->compute = static_cast<cudaStream_t>(c.cuda_stream);
    CK(ctx, cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    CK(ctx, cudaEventCreateWithFlags(&ctx->caller_ready, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&ctx->done_compute, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&ctx->done_copy, cudaEventDisableTiming));

    const int64_t groups = ctx->pitch_px / ctx->vec_px;
    if (c.read_path == CPT_READ_TEXTURE) {
        int maxw = 0, maxh = 0, maxl = 0;
        CK(ctx, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLayeredWidth, ctx->device));
        CK(ctx, cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLayeredHeight, ctx->device));
        CK(ctx, cudaDeviceGetAttribute(&maxl, cudaDevAttrMaxTexture2DLayeredLayers, ctx->device));
        if (groups > maxw || ctx->height > maxh || ctx->slot_members > maxl)
            return fail(ctx, CPT_EINVAL, "raster %dx%d with %d layers exceeds the layered texture limits (%d texels, %d rows, %d layers)",
                        ctx->width, ctx->height, ctx->slot_members, maxw, maxh, maxl);
    }

    const int count_bytes = c.mode == CPT_MODE_COUNT ? c.count_bits / 8 : 4;
    const size_t plane_bytes = (size_t)ctx->pitch_px * ctx->height * count_bytes;
    CK(ctx, cudaMalloc(&ctx->plane.data, plane_bytes));
    ctx->plane.pitch = ctx->pitch_px;
    ctx->plane.width = ctx->width;
    ctx->plane.height = ctx->height;
    ctx->plane.count_bits = c.mode == CPT_MODE_COUNT ? c.count_bits : 0;
    CK(ctx, cudaMalloc(&ctx->flags, cpt::kFlagCount * sizeof(int)));
    CK(ctx, cudaHostAlloc(&ctx->h_flags, cpt::kFlagCount * sizeof(int), cudaHostAllocDefault));
    memset(ctx->h_flags, 0, cpt::kFlagCount * sizeof(int));

    ctx->slots.resize(c.staging_buffers);
    for (Slot &s : ctx->slots) {
        if (cpt::fault_injected("staging_alloc")) return fail(ctx, CPT_ENOMEM, "staging buffer allocation refused (injected)");
        CK(ctx, cudaMalloc(&s.stage, (size_t)ctx->slot_members * ctx->member_bytes));
        CK(ctx, cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming));
        CK(ctx, cudaEventCreateWithFlags(&s.consumed, cudaEventDisableTiming));
        CK(ctx, cudaEventCreateWithFlags(&s.ring_free, cudaEventDisableTiming));
        if (c.read_path == CPT_READ_TEXTURE) {
            cudaChannelFormatDesc desc =
                c.mode == CPT_MODE_COUNT
                    ? cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindUnsigned)
                    : cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindFloat);
            CK(ctx, cudaMalloc3DArray(&s.array, &desc,
                                      make_cudaExtent((size_t)groups, ctx->height, ctx->slot_members),
                                      cudaArrayLayered | cudaArraySurfaceLoadStore));
            cudaResourceDesc rd{};
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = s.array;
            CK(ctx, cudaCreateSurfaceObject(&s.surf, &rd));
            cudaTextureDesc td{};
            td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            CK(ctx, cudaCreateTextureObject(&s.tex, &rd, &td, nullptr));
        }
    }
    uint8_t def[1024];
    for (int b = 0; b < 256; ++b) {
        def[4 * b] = (uint8_t)(255 - b);
        def[4 * b + 1] = (uint8_t)(255 - b);
        def[4 * b + 2] = 255;
        def[4 * b + 3] = 255;
    }
    ctx->default_lut = pack_lut(def);
    CK(ctx, cudaMemsetAsync(ctx->plane.data, 0, plane_bytes, ctx->compute));
    CK(ctx, cudaMemsetAsync(ctx->flags, 0, cpt::kFlagCount * sizeof(int), ctx->compute));
    return CPT_OK;
}

// The accumulation kernel over one batch already in device memory (a staging
// slot, or the caller's own rasters when they can be read in place), or in
// pinned host memory read through its device mapping (host_mapped: only the
// plain load kernels read it there, never a bulk or tensor copy).
int accumulate(composite_ctx *ctx, const RasterBatch &b, int sign, bool host_mapped = false) {
    const bool count = ctx->cfg.mode == CPT_MODE_COUNT;
    const uint64_t tns = (uint64_t)timeout_ms(ctx) * 1000000ull;
    int rc = trace_open(ctx, kTraceKernel, ctx->compute);
    if (rc) return rc;
    cudaError_t e;
    if (ctx->cfg.read_path == CPT_READ_TMA) {
        CUtensorMap map;
        const int box = ctx->cfg.tma_box_bytes;
        const int r = cpt::encode_tma_map(&map, b, ctx->width, ctx->height, ctx->elem, box);
        if (r != 0) return fail(ctx, CPT_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", r);
        e = count ? cpt::launch_count_tma(map, b, ctx->plane, sign, ctx->flags, tns, box, ctx->caps, ctx->compute)
                  : cpt::launch_depth_tma(map, b, ctx->plane, sign, ctx->flags, tns, box, ctx->caps, ctx->compute);
    } else if (ctx->bits) {
        e = !host_mapped && cpt::bits_bulk_compatible(b, ctx->width, ctx->height)
                ? cpt::launch_count_bits_bulk(b, ctx->plane, sign, ctx->flags, tns, ctx->caps, ctx->compute)
                : cpt::launch_count_bits(b, ctx->plane, sign, ctx->flags, ctx->caps, ctx->compute);
    } else {
        e = count ? cpt::launch_count_linear(b, ctx->plane, sign, ctx->flags, ctx->caps, ctx->compute)
                  : cpt::launch_depth_linear(b, ctx->plane, sign, ctx->flags, ctx->caps, ctx->compute);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "accumulation kernel launch");
    return trace_close(ctx, ctx->compute);
}

int accumulate_texture(composite_ctx *ctx, Slot &s, int n_layers, int sign) {
    int rc = trace_open(ctx, kTraceKernel, ctx->compute);
    if (rc) return rc;
    const cudaError_t e =
        ctx->cfg.mode == CPT_MODE_COUNT
            ? cpt::launch_count_texture(s.tex, n_layers, ctx->plane, sign, ctx->flags, ctx->caps, ctx->compute)
            : cpt::launch_depth_texture(s.tex, n_layers, ctx->plane, sign, ctx->flags, ctx->caps, ctx->compute);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "texture kernel launch");
    return trace_close(ctx, ctx->compute);
}

// Layout conversion into the slot's cudaArray (the buffer-to-image copy of
// Section 4), from `src` rasters with row pitch `pitch` and raster stride
// pitch * height, on stream st.
int convert_to_array(composite_ctx *ctx, Slot &s, const void *src, int64_t pitch, int n_layers,
                     cudaStream_t st) {
    int rc = trace_open(ctx, kTraceConvert, st);
    if (rc) return rc;
    const int texels = (int)(ctx->pitch_px / ctx->vec_px);
    const bool aligned = (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (pitch % 16 == 0);
    if (ctx->cfg.layout_converter == CPT_CONVERT_KERNEL && aligned) {
        const cudaError_t e = cpt::launch_convert_to_array(src, pitch, pitch * ctx->height, s.surf, texels,
                                                           ctx->height, n_layers, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "layout conversion kernel launch");
        return trace_close(ctx, st);
    }
    cudaMemcpy3DParms p{};
    p.srcPtr = make_cudaPitchedPtr(const_cast<void *>(src), (size_t)pitch, (size_t)pitch, ctx->height);
    p.dstArray = s.array;
    p.extent = make_cudaExtent((size_t)(ctx->pitch_px / ctx->vec_px), ctx->height, n_layers);
    p.kind = cudaMemcpyDeviceToDevice;
    CK(ctx, cudaMemcpy3DAsync(&p, st));
    return trace_close(ctx, st);
}

// Consumes one staged chunk on the compute stream.
int consume_slot(composite_ctx *ctx, Slot &s, int c, int sign) {
    if (ctx->cfg.read_path == CPT_READ_TEXTURE) {
        int rc = convert_to_array(ctx, s, s.stage, ctx->stage_pitch, c, ctx->compute);
        if (rc) return rc;
        return accumulate_texture(ctx, s, c, sign);
    }
    RasterBatch b{s.stage, ctx->member_bytes, ctx->stage_pitch, c};
    return accumulate(ctx, b, sign);
}

// Uploads c rasters (any memory kind) into a staging buffer laid out with
// row pitch pitch_px * elem and raster stride member_bytes.
int upload(composite_ctx *ctx, uint8_t *dst, const uint8_t *src, int c, int64_t stride,
           int64_t pitch) {
    const int64_t row = ctx->row_bytes;
    const int64_t dpitch = ctx->stage_pitch;
    const int64_t h = ctx->height;
    if (pitch == row && row == dpitch && stride == pitch * h) {
        CK(ctx, cudaMemcpyAsync(dst, src, (size_t)c * ctx->member_bytes, cudaMemcpyDefault, ctx->copy));
    } else if (stride == pitch * h) {
        CK(ctx, cudaMemcpy2DAsync(dst, dpitch, src, pitch, row, (size_t)c * h, cudaMemcpyDefault, ctx->copy));
    } else {
        for (int i = 0; i < c; ++i)
            CK(ctx, cudaMemcpy2DAsync(dst + (int64_t)i * ctx->member_bytes, dpitch, src + i * stride, pitch,
                                      row, h, cudaMemcpyDefault, ctx->copy));
    }
    return CPT_OK;
}

Slot &next_slot(composite_ctx *ctx) {
    return ctx->slots[ctx->next_slot++ % ctx->slots.size()];
}

// Pinned-host or device rasters: upload chunk by chunk through the slots.
int run_staged(composite_ctx *ctx, const uint8_t *src, int n, int64_t stride, int64_t pitch, int sign) {
    const int C = ctx->call_chunk;
    for (int m0 = 0; m0 < n; m0 += C) {
        const cpt::TraceRange chunk_range("composite chunk");
        const int c = n - m0 < C ? n - m0 : C;
        int rc = begin_chunk(ctx);
        if (rc) return rc;
        Slot &s = next_slot(ctx);
        CK(ctx, cudaStreamWaitEvent(ctx->copy, s.consumed, 0));
        rc = trace_open(ctx, kTraceUpload, ctx->copy);
        if (rc) return rc;
        rc = upload(ctx, s.stage, src + (int64_t)m0 * stride, c, stride, pitch);
        if (rc) return rc;
        rc = trace_close(ctx, ctx->copy);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.ready, ctx->copy));
        CK(ctx, cudaStreamWaitEvent(ctx->compute, s.ready, 0));
        rc = consume_slot(ctx, s, c, sign);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.consumed, ctx->compute));
    }
    return CPT_OK;
}

// Device rasters on the texture path, converted straight from the caller's
// memory into the slot arrays on the copy stream.
int run_texture_from_device(composite_ctx *ctx, const uint8_t *src, int n, int64_t stride, int64_t pitch, int sign) {
    const int C = ctx->call_chunk;
    for (int m0 = 0; m0 < n; m0 += C) {
        const cpt::TraceRange chunk_range("composite chunk");
        const int c = n - m0 < C ? n - m0 : C;
        int rc = begin_chunk(ctx);
        if (rc) return rc;
        Slot &s = next_slot(ctx);
        CK(ctx, cudaStreamWaitEvent(ctx->copy, s.consumed, 0));
        rc = convert_to_array(ctx, s, src + (int64_t)m0 * stride, pitch, c, ctx->copy);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.ready, ctx->copy));
        CK(ctx, cudaStreamWaitEvent(ctx->compute, s.ready, 0));
        rc = accumulate_texture(ctx, s, c, sign);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.consumed, ctx->compute));
    }
    return CPT_OK;
}

// Pageable host rasters: host copy into the pinned ring, then as run_staged.
constexpr int64_t kIngestPiece = 4 << 20;   // bytes per ring-copy piece

int run_ring(composite_ctx *ctx, const uint8_t *src, int n, int64_t stride, int64_t pitch, int sign) {
    const int k = (int)ctx->slots.size();
    if (ctx->ring_chunk == 0) {
        int64_t chunk = ctx->slot_members;
        if (ctx->cfg.pinned_ring_bytes > 0) {
            const int64_t fit = ctx->cfg.pinned_ring_bytes / ((int64_t)k * ctx->member_bytes);
            if (fit < 1)
                return fail(ctx, CPT_EINVAL, "pinned_ring_bytes %lld holds fewer than %d rasters",
                            (long long)ctx->cfg.pinned_ring_bytes, k);
            if (fit < chunk) chunk = fit;
        }
        for (Slot &s : ctx->slots) {
            const cudaError_t e = cpt::fault_injected("pinned_ring")
                                      ? cudaErrorMemoryAllocation
                                      : cudaHostAlloc(&s.ring, (size_t)chunk * ctx->member_bytes, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                // all or nothing: a later call starts the ring afresh
                for (Slot &t : ctx->slots)
                    if (t.ring) {
                        cudaFreeHost(t.ring);
                        t.ring = nullptr;
                    }
                cudaGetLastError();
                return fail(ctx, CPT_ENOMEM, "pinned ring allocation failed: %s", cudaGetErrorString(e));
            }
        }
        ctx->ring_chunk = chunk;
        int threads = ctx->cfg.ingest_threads;
        if (threads == 0) threads = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
        if (threads > 1) {
            // no exception may cross the C ABI: a host that refuses the threads
            // gets the copy on the calling thread
            try {
                if (cpt::fault_injected("ingest_threads")) throw std::runtime_error("ingest threads refused (injected)");
                ctx->ingest.reset(new cpt::CopyPool(threads - 1));
            } catch (...) {
                ctx->ingest.reset();
            }
        }
    }
    const int C = (int)std::min<int64_t>(ctx->ring_chunk, ctx->call_chunk);
    const int64_t row = ctx->row_bytes;
    const int64_t dpitch = ctx->stage_pitch;
    for (int m0 = 0; m0 < n; m0 += C) {
        const cpt::TraceRange chunk_range("composite chunk");
        const int c = n - m0 < C ? n - m0 : C;
        int rc = begin_chunk(ctx);
        if (rc) return rc;
        Slot &s = next_slot(ctx);
        if (s.ring_used) {
            rc = wait_event(ctx, s.ring_free);
            if (rc) return rc;
        }
        // the chunk's rasters into the ring slot: pieces of about kIngestPiece
        // bytes (whole rows), copied by the ingest threads at once
        const int64_t rows_per_piece = std::max<int64_t>(1, kIngestPiece / std::max<int64_t>(1, row));
        const int64_t pieces_per_member = (ctx->height + rows_per_piece - 1) / rows_per_piece;
        const uint8_t *base = src + (int64_t)m0 * stride;
        uint8_t *ring = s.ring;
        const int64_t member_bytes = ctx->member_bytes, height = ctx->height;
        auto piece = [&](int p) {
            const int64_t i = p / pieces_per_member;
            const int64_t y0 = (p - i * pieces_per_member) * rows_per_piece;
            const int64_t y1 = std::min(height, y0 + rows_per_piece);
            const uint8_t *from = base + i * stride;
            uint8_t *to = ring + i * member_bytes;
            if (pitch == dpitch && row == dpitch) {
                memcpy(to + y0 * dpitch, from + y0 * pitch, (size_t)((y1 - y0) * row));
            } else {
                for (int64_t y = y0; y < y1; ++y) memcpy(to + y * dpitch, from + y * pitch, (size_t)row);
            }
        };
        const int n_pieces = (int)(c * pieces_per_member);
        if (ctx->ingest) {
            ctx->ingest->run(n_pieces, piece);
        } else {
            for (int p = 0; p < n_pieces; ++p) piece(p);
        }
        CK(ctx, cudaStreamWaitEvent(ctx->copy, s.consumed, 0));
        rc = trace_open(ctx, kTraceUpload, ctx->copy);
        if (rc) return rc;
        CK(ctx, cudaMemcpyAsync(s.stage, s.ring, (size_t)c * ctx->member_bytes, cudaMemcpyHostToDevice, ctx->copy));
        rc = trace_close(ctx, ctx->copy);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.ring_free, ctx->copy));
        CK(ctx, cudaEventRecord(s.ready, ctx->copy));
        s.ring_used = true;
        CK(ctx, cudaStreamWaitEvent(ctx->compute, s.ready, 0));
        rc = consume_slot(ctx, s, c, sign);
        if (rc) return rc;
        CK(ctx, cudaEventRecord(s.consumed, ctx->compute));
    }
    return CPT_OK;
}

// Pageable rasters registered with the driver for the call (page-locked in
// place, cudaHostRegister): uploaded straight from the caller's memory like
// pinned rasters, then -- since the caller may reuse a pageable batch once
// the call returns -- the call waits for its uploads and unregisters the
// batch.  A wait that fails leaves the batch registered until the copy
// stream is known idle (the next successful sync, render to host or end).
// On a 16-core Grace host with a GB300, page-locking a batch in place was
// faster than any number of host threads copying it (109-145 GB/s end to end
// for 4.3 GB, against 78-100 through the ring; the host's own pageable-to-
// pinned copy tops out at 88-106 GB/s).
constexpr int64_t kRegisterMinBytes = 64ll << 20;

int run_registered(composite_ctx *ctx, const uint8_t *src, int n, int64_t stride, int64_t pitch, int sign) {
    const int rc = run_staged(ctx, src, n, stride, pitch, sign);
    const cudaError_t e = cudaEventRecord(ctx->done_copy, ctx->copy);
    const int wrc = e == cudaSuccess ? wait_event(ctx, ctx->done_copy) : cuda_fail(ctx, e, "cudaEventRecord");
    if (wrc == CPT_OK)
        cudaHostUnregister(const_cast<uint8_t *>(src));
    else
        ctx->pending_unregister.push_back(const_cast<uint8_t *>(src));
    return rc ? rc : wrc;
}

void unregister_pending(composite_ctx *ctx) {
    for (void *p : ctx->pending_unregister) cudaHostUnregister(p);
    ctx->pending_unregister.clear();
}

int apply(composite_ctx *ctx, const void *members, int32_t n, int64_t stride, int32_t pitch, int sign) {
    const cpt::TraceRange range(sign > 0 ? "composite_add_members" : "composite_remove_members");
    if (!ctx) return CPT_EINVAL;
    ctx->err.clear();
    if (ctx->poisoned) return refuse_poisoned(ctx);
    if (n < 0) return fail(ctx, CPT_EINVAL, "n_members %d < 0", n);
    if (n == 0) return CPT_OK;
    if (!members) return fail(ctx, CPT_EINVAL, "members is NULL");
    const int64_t row = ctx->row_bytes;
    if (pitch < row) return fail(ctx, CPT_EINVAL, "row_pitch_bytes %d < the row's %lld bytes", pitch, (long long)row);
    if (stride < (int64_t)pitch * ctx->height)
        return fail(ctx, CPT_EINVAL, "member_stride_bytes %lld < row_pitch_bytes * height", (long long)stride);
    if (ctx->elem == 4 && ((reinterpret_cast<uintptr_t>(members) | (uintptr_t)pitch | (uintptr_t)stride) & 3))
        return fail(ctx, CPT_EINVAL, "float32 rasters need 4-byte aligned pointer, pitch and stride");
    const int64_t after = ctx->n_members + (int64_t)sign * n;
    if (after < 0) return fail(ctx, CPT_EINVAL, "removing %d members from a composite of %lld", n, (long long)ctx->n_members);
    if (ctx->cfg.mode == CPT_MODE_COUNT && ctx->cfg.count_bits == 16 && after > 65535)
        return fail(ctx, CPT_EINVAL, "16-bit counts hold at most 65535 members");
    if (ctx->cfg.mode == CPT_MODE_COUNT && after > 0xFFFFFFFFll)
        return fail(ctx, CPT_EINVAL, "32-bit counts hold at most 2^32-1 members");

    const uint8_t *src = static_cast<const uint8_t *>(members);
    const MemKind kind = memory_kind(members, ctx->device);
    if (kind == kForeignDevice)
        return fail(ctx, CPT_EINVAL, "members are device memory of another GPU (the context runs on device %d)", ctx->device);
    ctx->call_chunks = 0;
    ctx->call_chunk = chunk_for_call(ctx, n);
    // uploads on the copy stream start after the caller's earlier work on the
    // compute stream (which may have produced the rasters)
    CK(ctx, cudaEventRecord(ctx->caller_ready, ctx->compute));
    CK(ctx, cudaStreamWaitEvent(ctx->copy, ctx->caller_ready, 0));
    int rc;
    if (kind == kDevice) {
        const bool aligned = (reinterpret_cast<uintptr_t>(members) % 16 == 0) && (pitch % 16 == 0) && (stride % 16 == 0);
        if (ctx->cfg.read_path == CPT_READ_TEXTURE) {
            const bool direct = (ctx->width % ctx->vec_px == 0) && stride == (int64_t)pitch * ctx->height;
            rc = direct ? run_texture_from_device(ctx, src, n, stride, pitch, sign)
                        : run_staged(ctx, src, n, stride, pitch, sign);
        } else if (aligned) {
            RasterBatch b{members, stride, pitch, n};
            rc = begin_chunk(ctx);
            if (!rc) rc = accumulate(ctx, b, sign);
        } else {
            rc = run_staged(ctx, src, n, stride, pitch, sign);
        }
    } else if (kind == kPinned) {
        const bool aligned = (reinterpret_cast<uintptr_t>(members) % 16 == 0) && (pitch % 16 == 0) && (stride % 16 == 0);
        if (ctx->cfg.host_read && ctx->cfg.read_path == CPT_READ_LINEAR && aligned) {
            // the kernel loads the pinned rasters over the host link itself
            void *dptr = nullptr;
            CK(ctx, cudaHostGetDevicePointer(&dptr, const_cast<void *>(members), 0));
            RasterBatch b{dptr, stride, pitch, n};
            rc = begin_chunk(ctx);
            if (!rc) rc = accumulate(ctx, b, sign, true);
        } else {
            rc = run_staged(ctx, src, n, stride, pitch, sign);
        }
    } else {
        // the bytes the batch spans, from its first row to the end of its last
        const int64_t span = (int64_t)(n - 1) * stride + pitch * (int64_t)(ctx->height - 1) + row;
        const int mode = ctx->cfg.pageable_ingest;
        bool registered = false;
        if ((mode == CPT_INGEST_REGISTER || (mode == CPT_INGEST_AUTO && span >= kRegisterMinBytes)) &&
            !cpt::fault_injected("host_register")) {
            registered = cudaHostRegister(const_cast<void *>(members), (size_t)span, cudaHostRegisterDefault) == cudaSuccess;
            if (!registered) cudaGetLastError();   // e.g. already registered: use the ring
        }
        rc = registered ? run_registered(ctx, src, n, stride, pitch, sign) : run_ring(ctx, src, n, stride, pitch, sign);
    }
    if (rc) {
        // Chunks queued before the failure still fold into the composite, so
        // it holds an unknown part of this call's rasters while N is that of
        // the call before: refuse further work until a clear.
        if (ctx->call_chunks > 0) poison(ctx, "an add or remove failed part-way; the composite holds part of its rasters");
        return rc;
    }
    ctx->n_members = after;
    return CPT_OK;
}

// Reads the device flags (already copied into h_flags by stream order).
int check_flags(composite_ctx *ctx) {
    if (ctx->h_flags[cpt::kFlagTimeout]) return fail(ctx, CPT_ETIMEOUT, "a device-side wait ran out");
    if (ctx->h_flags[cpt::kFlagUnderflow]) {
        poison(ctx, "a remove took away a member that was never added");
        return fail(ctx, CPT_EUNDERFLOW, "a remove took away a member that was never added");
    }
    return CPT_OK;
}

int wait_all(composite_ctx *ctx) {
    CK(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->flags, cpt::kFlagCount * sizeof(int), cudaMemcpyDeviceToHost, ctx->compute));
    CK(ctx, cudaEventRecord(ctx->done_compute, ctx->compute));
    CK(ctx, cudaEventRecord(ctx->done_copy, ctx->copy));
    int rc = wait_event(ctx, ctx->done_copy);
    if (rc) return rc;
    unregister_pending(ctx);   // the copy stream is idle
    return wait_event(ctx, ctx->done_compute);
}

}  // namespace

void cpt::set_thread_error(const char *message) { g_begin_error = message; }

int64_t cpt::fault_injected_value(const char *site) {
    const char *v = std::getenv("CPT_FAULT_INJECT");
    if (!v || !*v) return -1;
    const size_t n = strlen(site);
    for (const char *p = v;;) {
        const char *q = strchr(p, ',');
        const size_t len = q ? (size_t)(q - p) : strlen(p);
        if (len > n + 1 && strncmp(p, site, n) == 0 && p[n] == '=') {
            int64_t k = 0;
            for (size_t i = n + 1; i < len; ++i) {
                if (p[i] < '0' || p[i] > '9') return -1;
                k = k * 10 + (p[i] - '0');
            }
            return k;
        }
        if (!q) return -1;
        p = q + 1;
    }
}

bool cpt::fault_injected(const char *site) {
    const char *v = std::getenv("CPT_FAULT_INJECT");
    if (!v || !*v) return false;
    const size_t n = strlen(site);
    for (const char *p = v;;) {
        const char *q = strchr(p, ',');
        const size_t len = q ? (size_t)(q - p) : strlen(p);
        if (len == n && strncmp(p, site, n) == 0) return true;
        if (!q) return false;
        p = q + 1;
    }
}

cpt::TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
cpt::TraceRange::~TraceRange() { nvtxRangePop(); }

int cpt::abi_exception_status() noexcept {
    int rc = CPT_EINVAL;
    const char *what = "internal error (exception)";
    try {
        throw;
    } catch (const std::bad_alloc &) {
        rc = CPT_ENOMEM;
        what = "out of host memory";
    } catch (...) {
    }
    try {
        cpt::set_thread_error(what);
    } catch (...) {
    }
    return rc;
}

extern "C" {

int composite_default_config(composite_config *cfg) try {
    if (!cfg) return CPT_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->read_path = CPT_READ_LINEAR;
    cfg->staging_buffers = 2;
    cfg->chunk_members = 0;
    cfg->count_bits = 16;
    cfg->mode = CPT_MODE_COUNT;
    cfg->trace = 0;
    cfg->pinned_ring_bytes = 0;
    cfg->cuda_stream = nullptr;
    cfg->wait_timeout_ms = 0;
    cfg->host_read = 0;
    cfg->tma_box_bytes = 0;
    cfg->mask_format = CPT_MASK_BYTES;
    cfg->layout_converter = CPT_CONVERT_KERNEL;
    cfg->ingest_threads = 0;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_begin(composite_ctx **out, int32_t width, int32_t height, const composite_config *cfg) try {
    g_begin_error.clear();
    if (!out) return fail(nullptr, CPT_EINVAL, "out is NULL");
    *out = nullptr;
    if (width <= 0 || height <= 0) return fail(nullptr, CPT_EINVAL, "raster %d x %d is empty", width, height);
    composite_config c;
    if (cfg)
        c = *cfg;
    else
        composite_default_config(&c);
    int rc = check_config(c);
    if (rc) return rc;
    if (c.tma_box_bytes == 0) c.tma_box_bytes = kDefaultTmaBoxBytes;
    composite_ctx *ctx = new composite_ctx();
    ctx->width = width;
    ctx->height = height;
    ctx->cfg = c;
    ctx->elem = c.mode == CPT_MODE_COUNT ? 1 : 4;
    ctx->vec_px = 16 / ctx->elem;
    ctx->pitch_px = ((int64_t)width + ctx->vec_px - 1) / ctx->vec_px * ctx->vec_px;
    ctx->bits = c.mask_format == CPT_MASK_BITS;
    ctx->row_bytes = ctx->bits ? ((int64_t)width + 7) / 8 : (int64_t)width * ctx->elem;
    ctx->stage_pitch = (ctx->row_bytes + 15) / 16 * 16;
    ctx->member_bytes = ctx->stage_pitch * height;
    ctx->slot_members = c.chunk_members > 0 ? c.chunk_members : auto_slot_members(ctx->member_bytes, c.read_path);
    rc = setup(ctx);
    if (rc) {
        g_begin_error = ctx->err;
        destroy(ctx);
        return rc;
    }
    *out = ctx;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_load_counts(composite_ctx *ctx, const void *counts, int64_t n_members) try {
    if (!ctx) return CPT_EINVAL;
    ctx->err.clear();
    if (ctx->cfg.mode != CPT_MODE_COUNT) return fail(ctx, CPT_EINVAL, "counts can be loaded only in CPT_MODE_COUNT");
    if (!counts) return fail(ctx, CPT_EINVAL, "counts is NULL");
    const int64_t limit = ctx->cfg.count_bits == 16 ? 0xFFFFll : 0xFFFFFFFFll;
    if (n_members < 0 || n_members > limit)
        return fail(ctx, CPT_EINVAL, "n_members %lld outside 0..%lld", (long long)n_members, (long long)limit);
    const size_t elem = (size_t)ctx->cfg.count_bits / 8;
    if (reinterpret_cast<uintptr_t>(counts) % elem) return fail(ctx, CPT_EINVAL, "counts not aligned to its element");
    const MemKind kind = memory_kind(counts, ctx->device);
    if (kind == kForeignDevice)
        return fail(ctx, CPT_EINVAL, "counts are device memory of another GPU (the context runs on device %d)", ctx->device);
    const int64_t px = (int64_t)ctx->width * ctx->height;
    if (kind != kDevice) {
        // host counts are checked against N before anything changes
        for (int64_t i = 0; i < px; ++i) {
            const uint64_t c = elem == 2 ? static_cast<const uint16_t *>(counts)[i] : static_cast<const uint32_t *>(counts)[i];
            if (c > (uint64_t)n_members)
                return fail(ctx, CPT_EINVAL, "count %llu at pixel %lld exceeds N = %lld", (unsigned long long)c,
                            (long long)i, (long long)n_members);
        }
    }
    CK(ctx, cudaMemcpy2DAsync(ctx->plane.data, (size_t)ctx->pitch_px * elem, counts, (size_t)ctx->width * elem,
                              (size_t)ctx->width * elem, (size_t)ctx->height, cudaMemcpyDefault, ctx->compute));
    CK(ctx, cudaMemsetAsync(ctx->flags, 0, cpt::kFlagCount * sizeof(int), ctx->compute));
    if (kind != kDevice) {
        // host counts: the caller may reuse them as soon as the call returns
        cudaEvent_t copied = nullptr;
        CK(ctx, cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(copied, ctx->compute);
        const int rc = e == cudaSuccess ? wait_event(ctx, copied) : cuda_fail(ctx, e, "cudaEventRecord");
        cudaEventDestroy(copied);
        if (rc) return rc;
    }
    ctx->n_members = n_members;
    ctx->poisoned = false;
    memset(ctx->h_flags, 0, cpt::kFlagCount * sizeof(int));
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_clear(composite_ctx *ctx) try {
    if (!ctx) return CPT_EINVAL;
    ctx->err.clear();
    const size_t bytes = (size_t)ctx->pitch_px * ctx->height *
                         (ctx->cfg.mode == CPT_MODE_COUNT ? ctx->cfg.count_bits / 8 : 4);
    ctx->trace.clear();
    ctx->trace_used = 0;
    CK(ctx, cudaMemsetAsync(ctx->plane.data, 0, bytes, ctx->compute));
    CK(ctx, cudaMemsetAsync(ctx->flags, 0, cpt::kFlagCount * sizeof(int), ctx->compute));
    ctx->n_members = 0;
    ctx->poisoned = false;
    memset(ctx->h_flags, 0, cpt::kFlagCount * sizeof(int));
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_add_members(composite_ctx *ctx, const void *members, int32_t n_members,
                          int64_t member_stride_bytes, int32_t row_pitch_bytes) try {
    return apply(ctx, members, n_members, member_stride_bytes, row_pitch_bytes, +1);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_remove_members(composite_ctx *ctx, const void *members, int32_t n_members,
                             int64_t member_stride_bytes, int32_t row_pitch_bytes) try {
    return apply(ctx, members, n_members, member_stride_bytes, row_pitch_bytes, -1);
} catch (...) {
    return cpt::abi_exception_status();
}

}  // extern "C"

namespace {

int render(composite_ctx *ctx, void *counts_out, uint8_t *bucket_out, uint8_t *rgba_out, float *mean_out,
           uint64_t *hist_out, int32_t out_on_device, const uint8_t *lut_rgba) {
    const cpt::TraceRange range("composite_render");
    if (!ctx) return CPT_EINVAL;
    ctx->err.clear();
    if (ctx->poisoned) return refuse_poisoned(ctx);
    const bool count = ctx->cfg.mode == CPT_MODE_COUNT;
    if (count && mean_out) return fail(ctx, CPT_EINVAL, "mean_out needs CPT_MODE_MEAN_DEPTH");
    if (!count && (counts_out || bucket_out || rgba_out || hist_out))
        return fail(ctx, CPT_EINVAL, "counts, buckets, colours and histograms need CPT_MODE_COUNT");
    if (out_on_device != 0 && out_on_device != 1) return fail(ctx, CPT_EINVAL, "out_on_device must be 0 or 1");
    if (out_on_device) {
        const uintptr_t cbytes = count ? (uintptr_t)(ctx->cfg.count_bits / 8) : 1;
        if ((reinterpret_cast<uintptr_t>(counts_out) % cbytes) || (reinterpret_cast<uintptr_t>(rgba_out) % 4) ||
            (reinterpret_cast<uintptr_t>(mean_out) % 4) || (reinterpret_cast<uintptr_t>(hist_out) % 8))
            return fail(ctx, CPT_EINVAL, "device outputs must be aligned to their element size");
        // the render kernel writes them directly
        const void *outs[5] = {counts_out, bucket_out, rgba_out, mean_out, hist_out};
        for (const void *o : outs)
            if (o && !device_writable(o, ctx->device))
                return fail(ctx, CPT_EINVAL, "out_on_device = 1 needs device memory of device %d (or mapped pinned "
                                             "host memory) for every output", ctx->device);
    }
    const Lut lut = lut_rgba ? pack_lut(lut_rgba) : ctx->default_lut;
    const int64_t px = (int64_t)ctx->width * ctx->height;
    const uint64_t n = (uint64_t)ctx->n_members;
    const int cb = count ? ctx->cfg.count_bits / 8 : 0;

    if (out_on_device) {
        cudaError_t e = count ? cpt::launch_render_counts(ctx->plane, n, counts_out, bucket_out,
                                                          reinterpret_cast<uint32_t *>(rgba_out), lut, ctx->caps,
                                                          ctx->compute, hist_out)
                              : cpt::launch_render_mean(ctx->plane, n, mean_out, ctx->caps, ctx->compute);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "render kernel launch");
        return CPT_OK;
    }

    // scratch regions start on 256-byte boundaries (uint32 colour stores)
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = count ? up((size_t)px * cb) + up((size_t)px) + up((size_t)px * 4) + 256 * sizeof(uint64_t)
                              : up((size_t)px * 4);
    if (ctx->out_scratch_bytes < need) {
        if (ctx->out_scratch) {
            CK(ctx, cudaStreamSynchronize(ctx->compute));
            cudaFree(ctx->out_scratch);
            ctx->out_scratch = nullptr;
            ctx->out_scratch_bytes = 0;
        }
        CK(ctx, cudaMalloc(&ctx->out_scratch, need));
        ctx->out_scratch_bytes = need;
    }
    if (count) {
        uint8_t *d_counts = ctx->out_scratch;
        uint8_t *d_bucket = d_counts + up((size_t)px * cb);
        uint8_t *d_rgba = d_bucket + up((size_t)px);
        uint64_t *d_hist = reinterpret_cast<uint64_t *>(d_rgba + up((size_t)px * 4));
        cudaError_t e = cpt::launch_render_counts(ctx->plane, n, counts_out ? d_counts : nullptr,
                                                  bucket_out ? d_bucket : nullptr,
                                                  rgba_out ? reinterpret_cast<uint32_t *>(d_rgba) : nullptr,
                                                  lut, ctx->caps, ctx->compute, hist_out ? d_hist : nullptr);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "render kernel launch");
        if (hist_out) CK(ctx, cudaMemcpyAsync(hist_out, d_hist, 256 * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->compute));
        if (counts_out) CK(ctx, cudaMemcpyAsync(counts_out, d_counts, (size_t)px * cb, cudaMemcpyDeviceToHost, ctx->compute));
        if (bucket_out) CK(ctx, cudaMemcpyAsync(bucket_out, d_bucket, (size_t)px, cudaMemcpyDeviceToHost, ctx->compute));
        if (rgba_out) CK(ctx, cudaMemcpyAsync(rgba_out, d_rgba, (size_t)px * 4, cudaMemcpyDeviceToHost, ctx->compute));
    } else if (mean_out) {
        float *d_mean = reinterpret_cast<float *>(ctx->out_scratch);
        cudaError_t e = cpt::launch_render_mean(ctx->plane, n, d_mean, ctx->caps, ctx->compute);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "render kernel launch");
        CK(ctx, cudaMemcpyAsync(mean_out, d_mean, (size_t)px * 4, cudaMemcpyDeviceToHost, ctx->compute));
    }
    int rc = wait_all(ctx);
    if (rc) return rc;
    return check_flags(ctx);
}

}  // namespace

extern "C" {

int composite_render(composite_ctx *ctx, void *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                     float *mean_out, int32_t out_on_device, const uint8_t *lut_rgba) try {
    return render(ctx, counts_out, bucket_out, rgba_out, mean_out, nullptr, out_on_device, lut_rgba);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_render_histogram(composite_ctx *ctx, void *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                               uint64_t *histogram_out, int32_t out_on_device, const uint8_t *lut_rgba) try {
    if (ctx && !histogram_out) return fail(ctx, CPT_EINVAL, "histogram_out is NULL");
    return render(ctx, counts_out, bucket_out, rgba_out, nullptr, histogram_out, out_on_device, lut_rgba);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_sync(composite_ctx *ctx) try {
    if (!ctx) return CPT_EINVAL;
    ctx->err.clear();
    int rc = wait_all(ctx);
    if (rc) return rc;
    return check_flags(ctx);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_member_count(const composite_ctx *ctx, int64_t *n_out) try {
    if (!ctx || !n_out) return CPT_EINVAL;
    *n_out = ctx->n_members;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_trace_read(composite_ctx *ctx, float *records, int32_t capacity, int32_t *n_out) try {
    if (!ctx || !n_out || capacity < 0 || (capacity > 0 && !records)) return CPT_EINVAL;
    ctx->err.clear();
    int rc = wait_all(ctx);
    if (rc) return rc;
    const int32_t n = (int32_t)ctx->trace.size();
    *n_out = n;
    if (n == 0) return CPT_OK;
    // origin: the earliest start among the records
    cudaEvent_t origin = ctx->trace[0].a;
    for (const TraceRec &r : ctx->trace) {
        float d;
        CK(ctx, cudaEventElapsedTime(&d, origin, r.a));
        if (d < 0) origin = r.a;
    }
    for (int32_t i = 0; i < n && i < capacity; ++i) {
        float a, b;
        CK(ctx, cudaEventElapsedTime(&a, origin, ctx->trace[i].a));
        CK(ctx, cudaEventElapsedTime(&b, origin, ctx->trace[i].b));
        records[3 * i] = (float)ctx->trace[i].kind;
        records[3 * i + 1] = a;
        records[3 * i + 2] = b;
    }
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_end(composite_ctx *ctx) try {
    if (!ctx) return CPT_OK;
    int rc = wait_all(ctx);
    destroy(ctx);
    return rc == CPT_EUNDERFLOW ? CPT_OK : rc;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_selftest_bounded_wait(int64_t timeout_us, int32_t *gave_up_out, int64_t *waited_us_out) try {
    g_begin_error.clear();
    if (timeout_us <= 0 || timeout_us > 10000000 || !gave_up_out)
        return fail(nullptr, CPT_EINVAL, "timeout_us must be in 1..1e7 and gave_up_out not NULL");
    unsigned long long *d = nullptr, h[2] = {0, 0};
    cudaError_t e = cudaMalloc(&d, sizeof h);
    if (e == cudaSuccess) e = cpt::launch_bounded_wait_selftest((uint64_t)timeout_us * 1000ull, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounded-wait self-test");
    *gave_up_out = (int32_t)h[0];
    if (waited_us_out) *waited_us_out = (int64_t)(h[1] / 1000ull);
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

const char *composite_last_error(const composite_ctx *ctx) try {
    return ctx ? ctx->err.c_str() : g_begin_error.c_str();
} catch (...) {
    return "internal error (exception)";
}

}  // extern "C"
