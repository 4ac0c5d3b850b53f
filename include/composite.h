/*
 * composite.h -- C ABI of the GB300 iterative ensemble compositor.
 *
 * The operation (Johnson & Jankun-Kelly, "Efficacy of Images Versus Data
 * Buffers", Section 2 and Fig. 1): N flood-extent rasters are combined into
 * one composite image, the users add or remove rasters in real time, and the
 * composite is shown as a blue saturation map of the overlap.  The
 * accumulation streams the rasters from host memory through two or more
 * device receiving buffers so that the upload of one overlaps the processing
 * of another (Section 4, Figs. 2-4).
 *
 * Per pixel p, over the current multiset S of members, N = |S|:
 *   count(p)  = #{m in S : mask_m(p) != 0}
 *   bucket(p) = N == 0 ? 0 : floor(255 * count(p) / N)     (exact integers)
 *   rgba(p)   = lut[bucket(p)]                            (256 x RGBA8 table)
 *   mean(p)   = N == 0 ? 0 : sum_{m in S} d_m(p) / N      (mean-depth mode)
 *
 * Conventions for every call:
 *   - Return value: CPT_OK (0) or a negative composite_status.  On error the
 *     message is available from composite_last_error(ctx) until the next call
 *     on that context.
 *   - A raster is `height` rows of `width` elements; element type uint8 in
 *     CPT_MODE_COUNT (or one bit per pixel with CPT_MASK_BITS), float32 in
 *     CPT_MODE_MEAN_DEPTH.  Row y of member m starts at members +
 *     m * member_stride_bytes + y * row_pitch_bytes.
 *   - Memory kind of `members` is detected (cudaPointerGetAttributes); device
 *     memory of another GPU than the context's is rejected (CPT_EINVAL):
 *       pageable host  -> copied through the library's pinned ring; the
 *                         caller may reuse the memory as soon as the call
 *                         returns;
 *       pinned host    -> uploaded straight from it (cudaMemcpyAsync on the
 *       or device         copy stream) or read in place; BORROWED until the
 *                         next composite_render/composite_sync/composite_end
 *                         returns: do not modify or free it before then.
 *   - Work is queued on the context's compute stream (config.cuda_stream, by
 *     default the legacy default stream) and a copy stream the library owns,
 *     ordered by events, never by host synchronisation; uploads wait for the
 *     caller's earlier work on the compute stream.  Host waits that do
 *     happen (ring reuse, render to host, sync, end) are bounded by
 *     config.wait_timeout_ms and return CPT_ETIMEOUT when exceeded.
 *   - One context per host thread; contexts are independent.
 *   - The library never falls back to a CPU implementation: without a usable
 *     CUDA device every compute call returns CPT_ECUDA.
 *   - No C++ exception crosses this interface (nor those of composite_engine.h
 *     and composite_server.h): a failed host allocation inside a call returns
 *     CPT_ENOMEM, with its message in composite_last_error(NULL).
 */
#ifndef COMPOSITE_H
#define COMPOSITE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct composite_ctx composite_ctx;   /* opaque, owned by the library */

typedef enum composite_status {
    CPT_OK = 0,
    CPT_EINVAL = -1,      /* bad argument; the context is unchanged            */
    CPT_ENOMEM = -2,      /* device, pinned or host allocation failed          */
    CPT_ECUDA = -3,       /* CUDA runtime/driver error (message in last_error) */
    CPT_ESTATE = -4,      /* context poisoned by an earlier underflow or by an
                             add/remove that failed part-way                   */
    CPT_EUNDERFLOW = -5,  /* a remove took away a member that was never added  */
    CPT_ETIMEOUT = -6     /* a bounded wait (host or device) ran out           */
} composite_status;

/* How the accumulation kernel reads a member raster (the paper's images
 * versus buffers question, Sections 5.3 and 6.3, re-asked for sm_103a). */
enum {
    CPT_READ_LINEAR = 0,   /* 16-byte vector loads from linear device memory     */
    CPT_READ_TEXTURE = 1,  /* texture object over a layered, block-tiled cudaArray
                              filled by a buffer-to-array copy (the image path)  */
    CPT_READ_TMA = 2       /* TMA tensor tiles staged into shared memory         */
};

/* The buffer-to-image transform of the texture path (Section 4). */
enum {
    CPT_CONVERT_COPY = 0,     /* cudaMemcpy3DAsync into the array (the driver's copy)      */
    CPT_CONVERT_KERNEL = 1    /* a kernel: 16-byte loads, surface stores into the array;
                                 unaligned sources fall back to the copy                */
};

/* How pageable host rasters reach the device (step a2). */
enum {
    CPT_INGEST_AUTO = 0,      /* register batches of at least 64 MiB, copy smaller ones
                                 through the ring                                         */
    CPT_INGEST_RING = 1,      /* copy into the library's pinned ring on host threads, then
                                 upload from the ring                                    */
    CPT_INGEST_REGISTER = 2   /* page-lock the caller's batch in place for the call
                                 (cudaHostRegister), upload straight from it, wait for the
                                 uploads and unregister it before returning; a batch the
                                 driver will not register (already registered, say) goes
                                 through the ring.  While the call runs the batch is
                                 pinned memory to every other caller too: it must not be
                                 handed to another call (another context, another
                                 thread) at the same time                                */
};

enum {
    CPT_MODE_COUNT = 0,       /* uint8 masks -> per-pixel member counts      */
    CPT_MODE_MEAN_DEPTH = 1   /* float32 depths -> per-pixel mean (float32)   */
};

/* How a mask raster is stored (CPT_MODE_COUNT).  Bit-packed masks are the
 * compressed upload the paper proposes (Section 7.1: compress the input and
 * decompress it on the GPU): 8 times fewer bytes over the host link and in
 * device memory, decoded inside the accumulation kernel. */
enum {
    CPT_MASK_BYTES = 0,       /* one byte per pixel, nonzero = flooded                  */
    CPT_MASK_BITS = 1         /* one bit per pixel: pixel x is bit (x & 7) of byte x >> 3
                                 of its row; a row is ceil(width / 8) bytes            */
};

typedef struct composite_config {
    int32_t read_path;          /* CPT_READ_*; default CPT_READ_LINEAR                    */
    int32_t staging_buffers;    /* k device receiving buffers, 1..8; 1 is the paper's
                                   single-buffer control ("1b"), 2 its dual buffer ("2b");
                                   default 2                                              */
    int32_t chunk_members;      /* C members per upload and per kernel launch, 1..255, or
                                   0 = automatic (the default): a staging buffer holds up
                                   to 256 MiB of rasters (512 MiB on the texture path;
                                   at most 255 rasters), and each add or
                                   remove of n rasters is cut into chunks of
                                   max(16 MiB of rasters, min(that cap, ceil(n / 32)))
                                   members, so that a call has about 32 chunks: the
                                   kernel of a call's last chunk has no upload left to
                                   hide under                                             */
    int32_t count_bits;         /* 16 (N <= 65535) or 32; default 16                      */
    int32_t mode;               /* CPT_MODE_*; default CPT_MODE_COUNT                     */
    int32_t trace;              /* 1 = time every copy and kernel with CUDA events
                                   (composite_trace_read); default 0                      */
    int64_t pinned_ring_bytes;  /* cap on the pinned ring used for pageable inputs;
                                   0 = k * C rasters                                      */
    void *cuda_stream;          /* compute stream (a cudaStream_t); NULL = the legacy
                                   default stream.  The library's work is ordered after
                                   the caller's earlier work on this stream.              */
    int64_t wait_timeout_ms;    /* bound on every wait, host and device; 0 = 10000        */
    int32_t host_read;          /* 1 = with CPT_READ_LINEAR, pinned host rasters with 16-byte
                                   aligned base, pitch and stride are read in place by the
                                   accumulation kernel over the host link (no copy engine,
                                   no staging); 0 = upload through the staging buffers
                                   (the paper's pipeline); default 0                      */
    int32_t tma_box_bytes;      /* CPT_READ_TMA box width in bytes: 64, 128 or 256 (a box is
                                   2 KiB per member: width x 2048/width rows, x 16 members);
                                   0 = 256                                                */
    int32_t mask_format;        /* CPT_MASK_*; CPT_MASK_BITS needs CPT_MODE_COUNT and
                                   CPT_READ_LINEAR; default CPT_MASK_BYTES                */
    int32_t layout_converter;   /* CPT_READ_TEXTURE: how rasters reach the cudaArray;
                                   default CPT_CONVERT_KERNEL                             */
    int32_t ingest_threads;     /* host threads, the calling thread included, that copy
                                   pageable rasters into the pinned ring (step a2), each
                                   chunk cut into pieces copied at once; 1 = the calling
                                   thread alone; 0 = min(16, the host's hardware threads);
                                   at most 64.  The threads start at the first pageable
                                   add and end with the context.                          */
    int32_t pageable_ingest;    /* CPT_INGEST_*; default CPT_INGEST_AUTO.  Either way the
                                   caller may reuse a pageable batch once the call returns */
} composite_config;

/* Fills *cfg with the defaults listed above.  CPT_EINVAL if cfg is NULL. */
int composite_default_config(composite_config *cfg);

/* Creates a context for width x height rasters and clears its composite
 * (Fig. 3, step 1: clear the accumulation buffers).  Allocates the device
 * composite plane, the k staging buffers (and, for CPT_READ_TEXTURE, their
 * k layered cudaArrays), the streams and events.  cfg NULL = defaults.
 * Errors: CPT_EINVAL (out NULL, width/height <= 0, a config field out of
 * range), CPT_ENOMEM, CPT_ECUDA.  On error *out is set to NULL. */
int composite_begin(composite_ctx **out, int32_t width, int32_t height,
                    const composite_config *cfg);

/* Resets the composite to the empty multiset (counts and sums to zero,
 * N = 0) and clears the underflow state, stream-ordered after every earlier
 * call (Fig. 3, step 1; the paper's timing starts right after this). */
int composite_clear(composite_ctx *ctx);

/* Adds n_members rasters to the multiset: count(p) += [mask(p) != 0], or in
 * mean-depth mode sum(p) += d(p) (Fig. 3, steps 3-7: upload into receiving
 * buffer slot i mod k, accumulate, advance).
 * member_stride_bytes >= row_pitch_bytes * height; row_pitch_bytes >= the
 * row's bytes (width x element size, or ceil(width / 8) for bit-packed
 * masks); float32 rasters need 4-byte aligned pointer, pitch and stride.
 * n_members == 0 is a no-op.  Errors: CPT_EINVAL (NULL members with n > 0,
 * bad strides, N would exceed 65535 with count_bits 16; nothing changed),
 * CPT_ESTATE, CPT_ECUDA, CPT_ENOMEM, CPT_ETIMEOUT.
 * A call that fails after the work of its first chunk was queued (a CUDA
 * error, a ring wait that ran out) leaves the composite holding an unknown
 * part of its rasters while N stays that of the call before: the context is
 * then poisoned -- add, remove and render return CPT_ESTATE -- until
 * composite_clear or composite_load_counts.  A failure before any chunk
 * leaves the context unchanged. */
int composite_add_members(composite_ctx *ctx, const void *members, int32_t n_members,
                          int64_t member_stride_bytes, int32_t row_pitch_bytes);

/* Removes n_members rasters from the multiset (the interactive list of
 * Fig. 1).  The state afterwards equals a recompute over what is left.
 * CPT_EINVAL, with nothing changed, if N would become negative.  If a pixel
 * count would go below zero (a raster removed that was never added), the
 * device records it, the next render or sync returns CPT_EUNDERFLOW and the
 * context is poisoned (CPT_ESTATE) until composite_clear. */
int composite_remove_members(composite_ctx *ctx, const void *members, int32_t n_members,
                             int64_t member_stride_bytes, int32_t row_pitch_bytes);

/* Renders the composite (Fig. 1 caption: overlap classes and the blue
 * saturation map).  Every output is dense row-major, width x height, caller
 * owned, and may be NULL to skip it:
 *   counts_out  uint16 or uint32 per pixel (count_bits)      COUNT mode
 *   bucket_out  uint8 overlap class per pixel                COUNT mode
 *   rgba_out    4 x uint8 per pixel, lut[bucket]             COUNT mode
 *   mean_out    float32 mean depth per pixel                 MEAN_DEPTH mode
 * lut_rgba: 256 x 4 bytes in host memory, or NULL for the default ramp
 * b -> (255-b, 255-b, 255, 255).
 * out_on_device = 1: the outputs are device pointers (device memory of the
 * context's device, or mapped pinned host memory; anything else is rejected
 * with CPT_EINVAL before anything is queued); the render is queued on
 * the compute stream and the call returns without waiting (an underflow is
 * then reported by composite_sync).  out_on_device = 0: host pointers; the
 * call waits (bounded) until they are written and reports an underflow.
 * Ends the borrow of every member passed so far when out_on_device = 0. */
int composite_render(composite_ctx *ctx, void *counts_out, uint8_t *bucket_out,
                     uint8_t *rgba_out, float *mean_out, int32_t out_on_device,
                     const uint8_t *lut_rgba);

/* As composite_render (COUNT mode), and in the same pass the histogram of
 * overlap classes (Fig. 1 caption: the frequency of the overlap classes,
 * the distribution of flood occurrences): histogram_out[b] = number of
 * pixels whose class is b, b = 0..255, 256 x uint64, in device memory when
 * out_on_device = 1 (8-byte aligned) else host memory.  histogram_out must
 * not be NULL; the other outputs may be. */
int composite_render_histogram(composite_ctx *ctx, void *counts_out, uint8_t *bucket_out,
                               uint8_t *rgba_out, uint64_t *histogram_out, int32_t out_on_device,
                               const uint8_t *lut_rgba);

/* Waits (bounded) until every queued copy and kernel of the context has
 * finished; returns CPT_EUNDERFLOW if a remove underflowed, CPT_ETIMEOUT if
 * the wait ran out, and ends the borrow of every member passed so far. */
int composite_sync(composite_ctx *ctx);

/* *n_out = N, the number of members in the multiset. */
int composite_member_count(const composite_ctx *ctx, int64_t *n_out);

/* Resume from a checkpoint: replaces the composite by the given per-pixel
 * counts and member count N, as if the members behind them had been added to
 * an empty composite.  The other half of the checkpoint is composite_render
 * with counts_out plus composite_member_count (a composite is fully described
 * by its counts and N; Section 2's interactive list may then go on adding and
 * removing).  CPT_MODE_COUNT only (a mean-depth composite renders means, not
 * its sums).
 *   counts: width x height dense rows of the context's count type (uint16 or
 *           uint32), host (pageable or pinned) or device memory, aligned to
 *           its element; copied, not borrowed, stream-ordered after earlier
 *           work.
 *   n_members: 0 <= N <= the count type's limit.  Every count must be <= N;
 *           host counts are checked (CPT_EINVAL, nothing changed), device
 *           counts are the caller's responsibility (a count above N renders
 *           as class 255).
 * Clears the underflow state like composite_clear. */
int composite_load_counts(composite_ctx *ctx, const void *counts, int64_t n_members);

/* With config.trace = 1: copies up to `capacity` records of 3 floats
 * {kind, start_ms, end_ms} into `records` (host memory), kind 0 = upload,
 * 1 = layout conversion, 2 = accumulation kernel, times relative to the
 * first traced event since the last composite_clear.  Waits (bounded) for
 * the traced work.  *n_out = records available (may exceed capacity). */
int composite_trace_read(composite_ctx *ctx, float *records, int32_t capacity, int32_t *n_out);

/* Waits (bounded) for the context's work and frees everything it owns.
 * NULL is accepted.  The context pointer is invalid afterwards. */
int composite_end(composite_ctx *ctx);

/* Message of the last error on ctx (or of the last failed composite_begin
 * or composite_oneshot_static on this thread when ctx is NULL).  Owned by
 * the library; valid until the next call on the same context. */
const char *composite_last_error(const composite_ctx *ctx);

/* Self-test of the device-side bounded wait used by the TMA kernels: one
 * thread waits on a shared-memory mbarrier that nothing ever arrives at, for
 * at most timeout_us (1..1e7), then gives up, exactly as a stuck TMA kernel
 * would, and the host reads the outcome.  *gave_up_out = 1 when the wait
 * gave up (the expected result), *waited_us_out (may be NULL) = how long it
 * waited.  No GPU fault is involved; the context-free error message is in
 * composite_last_error(NULL). */
int composite_selftest_bounded_wait(int64_t timeout_us, int32_t *gave_up_out, int64_t *waited_us_out);

/* Largest composite plane of composite_oneshot_static, in padded pixels:
 * roundup(width, 16) * height must not exceed it (2048 x 2048). */
#define CPT_ONESHOT_MAX_PIXELS 4194304

/* One-shot composite that allocates nothing.  The paper has no counterpart:
 * it exists for callers that cannot call cudaMalloc, such as a per-frame
 * render callback that must not risk the implicit device synchronisation an
 * allocation can bring, or a host application that owns all device memory
 * through its own pool and forbids libraries from allocating.
 * Computes, over the n_members device-resident uint8 masks, uint32 counts,
 * overlap classes and colours exactly as composite_begin + add_members +
 * render would (same kernels), writing every non-NULL output: dense
 * row-major width x height, counts_out uint32 and rgba_out 4 x uint8 per
 * pixel (both 4-byte aligned), bucket_out uint8 per pixel, each in device
 * memory of the current device and large enough (the library cannot check
 * sizes).  members, row_pitch_bytes and member_stride_bytes must be 16-byte
 * aligned and members in device memory of the current device (or managed
 * memory); host memory or another GPU's memory is rejected with CPT_EINVAL
 * before anything is queued.  lut_rgba is a host table or NULL for the
 * default.
 * The work is queued on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting.
 * Scratch: a file-scope __device__ array of CPT_ONESHOT_MAX_PIXELS uint32
 * counts (16 MiB, plus 16 bytes of flags) that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up its
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * Every call on a device shares that array and clears the part it uses, so
 * calls whose work overlaps on the GPU (different streams, or host threads)
 * race and must be serialised by the caller.
 * Errors: CPT_EINVAL (empty raster, raster larger than the scratch,
 * unaligned members or outputs, members or outputs not in the current
 * device's memory, bad strides), CPT_ECUDA; the message is in
 * composite_last_error(NULL). */
int composite_oneshot_static(const void *members, int32_t n_members, int64_t member_stride_bytes,
                             int32_t row_pitch_bytes, int32_t width, int32_t height,
                             uint32_t *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                             const uint8_t *lut_rgba, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* COMPOSITE_H */
