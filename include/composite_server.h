/*
 * composite_server.h -- C ABI of the interactive composite server.
 *
 * The paper's use: users of the flood-analysis program vary the set of
 * selected members in real time and the composite follows (Section 2 and
 * Fig. 1: the member list where surfaces are added or removed, the composite
 * and its overlap-class view updated from it).  The server keeps an ensemble
 * of uint8 masks (a resident part in device memory, an overflow part in pinned
 * host memory), sessions that each hold a member set and its uint32
 * composite plane in device memory, and a queue of requests.  A request
 * toggles a set of member ids in one session (selected ones are removed,
 * unselected ones added) and asks for the session's composite rendered into
 * caller-owned device outputs.
 *
 * Scheduling (continuous batching): composite_server_pump admits every queued
 * request whose session has no request in flight, up to max_batch requests
 * and within the device-memory budget, and turns the admitted requests into
 * one "cycle" of device work queued without waiting for earlier cycles:
 *   - per request, the toggle becomes adds and removes of members, or, when
 *     that is cheaper, a clear and a re-add of the new member set;
 *   - resident members of every admitted request: one engine submit (a
 *     single persistent launch, members gathered by index lists);
 *   - overflow members: each distinct one uploaded once per cycle from pinned
 *     host memory into one of two device staging halves, alternating, by one
 *     gather kernel per half on a copy stream (it reads the pinned rasters
 *     through their device mapping), members ordered by the set of requests
 *     that toggle them so that each request's members lie in few runs; each
 *     half is followed by one engine submit for all requests' members in it
 *     (the paper's dual-buffer upload, Section 4, shared by the requests of
 *     the cycle);
 *   - one render launch for all admitted sessions.
 * The overflow part must be pinned host memory (or device memory) whose
 * device address is 16-byte aligned.
 * A request completes when its cycle's event has completed; pump reports
 * completed request ids.  Requests that arrive while cycles run are admitted
 * into the next cycle; cycles run back to back on the device, the copy stream
 * overlapping uploads of one with kernels of another.
 *
 * Results are exact: the composite of a session after a request equals the
 * oracle count over the session's member set, independent of what else was
 * in the cycle.  Every call returns CPT_OK or a negative composite_status
 * (composite.h); the message is in composite_server_last_error.
 */
#ifndef COMPOSITE_SERVER_H
#define COMPOSITE_SERVER_H

#include <stdint.h>

#include "composite.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct composite_server composite_server;

typedef struct composite_server_config {
    int32_t width, height;         /* raster size of every member                        */
    const void *resident;          /* device: n_resident masks (member ids 0..n_resident-1) */
    int32_t n_resident;
    const void *overflow;          /* pinned host: n_overflow masks (ids n_resident..), may be NULL */
    int32_t n_overflow;
    int32_t row_pitch_bytes;       /* layout of both parts: multiple of 16, >= width       */
    int64_t member_stride_bytes;   /* multiple of 16, >= row_pitch_bytes * height          */
    int32_t max_sessions;          /* 1..65536                                            */
    int32_t max_batch;             /* requests per cycle, 1..4096; 1 = one request at a time */
    int32_t staging_members;       /* overflow rasters per staging half, 1..4096; 0 = 64   */
    int32_t max_cycles_in_flight;  /* 1..16; 0 = 4                                         */
    int64_t hbm_budget_bytes;      /* cap on planes + staging + index buffers; 0 = no cap  */
    void *cuda_stream;             /* compute stream, NULL = the legacy default stream    */
    int64_t wait_timeout_ms;       /* bound on host waits; 0 = 10000                      */
    int32_t mask_format;           /* CPT_MASK_BYTES or CPT_MASK_BITS (both parts): bit-packed
                                      rows are ceil(width / 8) bytes, 8x fewer bytes resident
                                      and over the host link                             */
} composite_server_config;

typedef struct composite_server_stats {
    int64_t requests_done;
    int64_t cycles;
    int64_t members_added;
    int64_t members_removed;
    int64_t recomputes;            /* requests served by clear + re-add                   */
    int64_t overflow_uploads;      /* overflow rasters uploaded                           */
    int64_t queued;                /* requests waiting now                                 */
    int64_t in_flight;             /* requests in cycles not yet completed                 */
    int64_t cycle_device_us;       /* sum over completed cycles of the time from the cycle's
                                      first queued operation to its completion (events)  */
    int64_t enqueue_host_us;       /* host time spent building and queueing cycles         */
} composite_server_stats;

int composite_server_default_config(composite_server_config *cfg);

/* Creates the server; allocates the staging halves and the per-cycle index
 * buffers.  CPT_EINVAL for a bad layout or limits, CPT_ENOMEM if the budget
 * cannot hold the staging halves. */
int composite_server_begin(composite_server **out, const composite_server_config *cfg);

/* Opens a session with an empty member set; allocates its plane (CPT_ENOMEM
 * if that would exceed the budget or max_sessions). */
int composite_server_open_session(composite_server *srv, int32_t *session_out);

/* Closes a session once its requests are done (CPT_ESTATE while some are
 * queued or in flight); frees its plane. */
int composite_server_close_session(composite_server *srv, int32_t session);

/* Queues a request: toggle the n member ids in `toggle` (host array, ids in
 * [0, n_resident + n_overflow), duplicates toggle twice) in the session, then
 * render its composite into the device outputs (each may be NULL; width x
 * height, dense; counts uint32 4-byte aligned, rgba 4-byte aligned; device
 * memory of the server's device or mapped pinned host memory, else
 * CPT_EINVAL).  The outputs are written when the request completes.  *request_id_out gets an
 * id that increases with every request. */
int composite_server_request(composite_server *srv, int32_t session, const int32_t *toggle, int32_t n,
                             uint32_t *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                             int64_t *request_id_out);

/* As composite_server_request, and also the class histogram of the request's
 * composite (Fig. 1 caption: the frequency of the overlap classes) into
 * histogram_out: 256 x uint64, bin k = the pixels whose overlap class is k,
 * 16-byte aligned, device memory of the server's device or mapped pinned host
 * memory (else CPT_EINVAL), zeroed and filled when the request completes.  A
 * histogram must not be shared by two requests in flight.  NULL = none. */
int composite_server_request_histogram(composite_server *srv, int32_t session, const int32_t *toggle, int32_t n,
                                       uint32_t *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                                       uint64_t *histogram_out, int64_t *request_id_out);

/* Makes progress without blocking: collects completed cycles (their request
 * ids go to `completed`, up to `capacity`; *n_completed = how many were
 * written) and queues new cycles for admissible requests.
 * If a cycle fails after admission (an engine error, a refused upload), its
 * sessions may hold part of its work: every request of those sessions in the
 * cycle or still queued is dropped (it never completes), the error names the
 * sessions, and further requests on them return CPT_ESTATE until they are
 * closed.  Other sessions are unaffected. */
int composite_server_pump(composite_server *srv, int64_t *completed, int32_t capacity, int32_t *n_completed);

/* Pumps until nothing is queued or in flight (bounded by wait_timeout_ms per
 * cycle); completed ids are dropped. */
int composite_server_drain(composite_server *srv);

/* Member count of a session after every queued request (host bookkeeping). */
int composite_server_session_members(const composite_server *srv, int32_t session, int64_t *n_out);

int composite_server_get_stats(const composite_server *srv, composite_server_stats *out);

/* Drains (bounded), then frees everything.  NULL is accepted. */
int composite_server_end(composite_server *srv);

const char *composite_server_last_error(const composite_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* COMPOSITE_SERVER_H */
