/*
 * composite_engine.h -- C ABI of the batched composite engine.
 *
 * Many composites at once (the batched and interactive uses of the paper's
 * flood-analysis program, Section 2 and Fig. 1: several member selections,
 * each folded into its own composite and shown as its own saturation map).
 * The engine holds composite planes in device memory (uint32 or uint16 counts, one per
 * plane) and applies "ops" to them: add or remove a set of device-resident
 * uint8 masks to one plane.  All ops of one submit call run in ONE persistent
 * kernel launch whose warps pull work items (op, member slab, chunk of
 * 16-pixel groups) from a device counter, so small and large composites share
 * the GPU without one launch per composite; one render call likewise renders
 * many planes in one launch.  A submit + render sequence can be captured in a
 * CUDA graph and replayed, and an autotuner picks the slab depth and the CTAs
 * per SM by timing candidates on the caller's ops.
 *
 * Per pixel p of plane P (members S_P, N_P = |S_P|), exactly as composite.h:
 *   count(p) = #{m in S_P : mask_m(p) != 0}
 *   bucket(p) = N_P == 0 ? 0 : floor(255 count(p) / N_P); rgba(p) = lut[bucket(p)]
 *
 * Conventions: every call returns CPT_OK (0) or a negative composite_status
 * (composite.h); the message is in composite_engine_last_error.  Members are
 * device memory of the engine's device or pinned host memory; index lists and
 * outputs are device memory of that device (outputs may also be mapped pinned
 * host memory); anything else is rejected with CPT_EINVAL before anything is
 * queued.  Rasters need 16-byte aligned base, row pitch and member stride.
 * Ops on pinned host members stream through the engine's own staging
 * buffers (the dual-buffer pipeline of Section 4, Figs. 3-4): rasters of
 * consecutive host ops are packed into a buffer of staging_bytes, uploaded on
 * a copy stream while the previous buffer is folded, one accumulate launch
 * per buffer.  Work is queued on the engine's stream; host waits are bounded
 * by wait_timeout_ms.  Members and index lists are borrowed until the next
 * composite_engine_sync returns.
 */
#ifndef COMPOSITE_ENGINE_H
#define COMPOSITE_ENGINE_H

#include <stdint.h>

#include "composite.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct composite_engine composite_engine;

/* How the accumulate launch hands work items to warps. */
enum {
    CPT_SCHEDULE_PERSISTENT = 0,  /* num_SMs x ctas_per_sm CTAs; warps claim items from a counter */
    CPT_SCHEDULE_GRID = 1         /* one CTA per 8 items; the hardware schedules the CTAs        */
};

typedef struct composite_engine_config {
    void *cuda_stream;        /* cudaStream_t for all engine work, NULL = the legacy
                                 default stream (ordered with the caller's work there) */
    int32_t slab_members;     /* members per work item, 1..255; 0 = 128               */
    int32_t ctas_per_sm;      /* persistent CTAs of 256 threads per SM, 1..8; 0 = 5   */
    int64_t wait_timeout_ms;  /* bound on host waits; 0 = 10000                        */
    int32_t schedule;         /* CPT_SCHEDULE_*; default CPT_SCHEDULE_PERSISTENT       */
    void *upload_stream;      /* cudaStream_t for the engine's small host-to-device
                                 uploads (op descriptors), NULL = cuda_stream; a caller
                                 that streams its own rasters on a copy stream passes
                                 it here so the small uploads queue behind its uploads
                                 in order instead of competing for a copy engine      */
    int32_t item_member_groups; /* work item size: a lane folds about this many
                                 (member, 16-pixel group) pairs per item, so an item
                                 covers 32 x (item_member_groups / slab) groups of one
                                 slab; 16..8192, 0 = 512                                */
    int32_t staging_buffers;  /* staging buffers for host ops, 2..8; 0 = 2           */
    int64_t staging_bytes;    /* bytes per staging buffer, >= 1 MiB (and >= the largest
                                 host raster); 0 = 256 MiB.  Allocated at the first
                                 host op.                                              */
} composite_engine_config;

/* One add or remove of n_members masks to one plane.  Member i of the op is
 * the raster at members + idx(i) * member_stride_bytes, idx(i) =
 * member_index[i] (a device int32 array) or i when member_index is NULL.
 * The raster's width and height are the plane's.  members is device memory,
 * or pinned host memory (then member_index must be NULL).  The library does
 * not know how many rasters the allocation holds: every member_index entry
 * must name one of them (the Python binding checks this on the device
 * values). */
typedef struct composite_op {
    int32_t plane;
    int32_t sign;                 /* +1 add, -1 remove */
    const void *members;          /* device or pinned host, 16-byte aligned */
    const int32_t *member_index;  /* device, n_members entries, or NULL */
    int32_t n_members;
    int32_t row_pitch_bytes;      /* multiple of 16, >= the row's bytes (width, or
                                     ceil(width / 8) for bit-packed masks) */
    int64_t member_stride_bytes;  /* multiple of 16, >= row_pitch_bytes * height */
    int32_t mask_format;          /* CPT_MASK_BYTES or CPT_MASK_BITS (composite.h) */
} composite_op;

/* Render of one plane into dense row-major device outputs (each may be NULL). */
typedef struct composite_render_op {
    int32_t plane;
    void *counts_out;       /* width x height counts of the plane's type (uint32, or
                               uint16 for a 16-bit plane), aligned to it */
    uint8_t *bucket_out;    /* width x height */
    uint8_t *rgba_out;      /* width x height x 4, 4-byte aligned */
    uint64_t *histogram_out; /* 256 x uint64, 16-byte aligned, or NULL: the number of
                               pixels of the plane in every overlap class (Fig. 1
                               caption: the frequency of the overlap classes),
                               counted in the same launch */
} composite_render_op;

int composite_engine_default_config(composite_engine_config *cfg);

/* Creates an engine (no planes yet).  cfg NULL = defaults. */
int composite_engine_begin(composite_engine **out, const composite_engine_config *cfg);

/* Allocates a zeroed width x height uint32 plane (N = 0); *plane_out is its id. */
int composite_engine_add_plane(composite_engine *eng, int32_t width, int32_t height, int32_t *plane_out);

/* The same with the count width chosen: count_bits 32, or 16 for a plane that
 * will never hold more than 65535 members (half the plane's bytes in every
 * clear, fold and render; a submit that would exceed 65535 is rejected with
 * CPT_EINVAL).  count_bits other than 16 or 32: CPT_EINVAL. */
int composite_engine_add_plane_bits(composite_engine *eng, int32_t width, int32_t height, int32_t count_bits,
                                    int32_t *plane_out);

/* Frees a plane after the engine's queued work; its id is not reused. */
int composite_engine_free_plane(composite_engine *eng, int32_t plane);

/* Queues a clear of the plane (counts 0, N = 0, underflow state and a
 * failed submit's mark cleared). */
int composite_engine_clear(composite_engine *eng, int32_t plane);

/* Queues a clear of every listed plane (ids may repeat) in ONE launch, as
 * composite_engine_clear does for one: counts 0, N = 0, underflow state and
 * failure marks cleared.  CPT_EINVAL, nothing queued, for an unknown plane. */
int composite_engine_clear_many(composite_engine *eng, const int32_t *planes, int32_t n_planes);

/* Queues every op in one persistent accumulate launch.  Validates all ops on
 * the host first (CPT_EINVAL and nothing queued if one is bad: unknown plane,
 * sign not +-1, N of a plane would go negative or above its count type's
 * maximum (2^32-1, or 65535 for a 16-bit plane), bad strides).
 * A pixel count that would go below zero raises the plane's underflow state
 * (reported by composite_engine_sync).
 * A failure before the launch (descriptor upload) leaves every plane and N
 * as they were.  A failure of the launch itself (CPT_ECUDA) marks every plane
 * of the submit as failed: they may hold part of the ops, so submits and
 * renders naming them return CPT_ESTATE until composite_engine_clear (or a
 * captured graph that refolds them). */
int composite_engine_submit(composite_engine *eng, const composite_op *ops, int32_t n_ops);

/* Queues the render of every listed plane in one persistent launch.
 * lut_rgba: 256 x 4 host bytes or NULL for the default white-to-blue ramp.
 * An op's histogram_out (if not NULL) is zeroed and then filled in the same
 * call: bin k = the number of the plane's width x height pixels whose
 * overlap class is k; it must not overlap another output of the call unless
 * it is the same histogram, in which case the ops' pixels add up in it.
 * CPT_EINVAL, nothing queued, for an unaligned or unreachable output. */
int composite_engine_render(composite_engine *eng, const composite_render_op *ops, int32_t n_ops,
                            const uint8_t *lut_rgba);

/* *n_out = N of the plane (host bookkeeping, exact). */
int composite_engine_member_count(const composite_engine *eng, int32_t plane, int64_t *n_out);

/* Waits (bounded) for the engine's queued work.  CPT_EUNDERFLOW if some
 * plane underflowed since its last clear; *bad_plane_out (may be NULL) then
 * holds the first such plane. */
int composite_engine_sync(composite_engine *eng, int32_t *bad_plane_out);

/* Captures "clear every target plane, submit ops, render rops" as a CUDA
 * graph held by the engine (replacing any earlier one): three kernel nodes,
 * the clear of all target planes (and of the render ops' histograms, so
 * that every replay starts them from zero) in one of them.  The ops' member
 * sets, index lists and outputs are fixed by the capture.  Does not run it.
 * Device members only (CPT_EINVAL for an op on host memory). */
int composite_engine_capture(composite_engine *eng, const composite_op *ops, int32_t n_ops,
                             const composite_render_op *rops, int32_t n_rops, const uint8_t *lut_rgba);

/* Launches the captured graph once on the engine's stream. */
int composite_engine_replay(composite_engine *eng);

/* Autotuner: times "clear the ops' planes + submit ops", `repeats` runs per
 * candidate, in three passes, each keeping the fastest: (1) slab_members in
 * {32, 64, 128, 255} x schedule {grid, persistent with ctas_per_sm 3, 4, 5};
 * (2) item_member_groups in {256, 512, 1024, 2048} (the work item's tile of
 * groups); (3) when some op reads pinned host members, staging_buffers in
 * {2, 3, 4} x staging_bytes in {64, 128, 256, 512} MiB.  The winner becomes
 * the engine's configuration (composite_engine_get_config reports every
 * field); slab and schedule are also reported here (either pointer may be
 * NULL; *ctas_per_sm_out = 0 means the grid schedule won).  The planes end
 * holding the result of the ops applied once to cleared planes. */
int composite_engine_tune(composite_engine *eng, const composite_op *ops, int32_t n_ops, int32_t repeats,
                          int32_t *slab_out, int32_t *ctas_per_sm_out);

/* Current (slab_members, ctas_per_sm); ctas_per_sm 0 = grid schedule. */
int composite_engine_get_tuning(const composite_engine *eng, int32_t *slab_out, int32_t *ctas_per_sm_out);

/* The engine's whole current configuration (defaults filled in, tuned values
 * after composite_engine_tune). */
int composite_engine_get_config(const composite_engine *eng, composite_engine_config *cfg_out);

/* Waits (bounded) and frees everything.  NULL is accepted. */
int composite_engine_end(composite_engine *eng);

const char *composite_engine_last_error(const composite_engine *eng);

#ifdef __cplusplus
}
#endif

#endif /* COMPOSITE_ENGINE_H */
