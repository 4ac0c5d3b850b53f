// server.cu -- the interactive composite server of include/composite_server.h:
// sessions, the request queue and the continuous-batching scheduler, built on
// the batched engine (include/composite_engine.h).
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <unordered_set>
#include <utility>
#include <vector>

#include "composite_engine.h"
#include "composite_server.h"
#include "internal.cuh"

namespace {

struct Session {
    bool open = false;
    int32_t plane = -1;
    std::vector<uint64_t> bits;    // member set after every admitted request
    std::vector<uint64_t> view;    // member set after every queued request
    int64_t n = 0;
    int64_t n_view = 0;
    int pending = 0;               // queued + in flight
    bool busy = false;             // a request in flight
    bool failed = false;           // a cycle failed part-way over this session's plane
};

struct Request {
    int64_t id;
    int32_t session;
    std::vector<int32_t> toggle;
    uint32_t *counts_out;
    uint8_t *bucket_out;
    uint8_t *rgba_out;
    uint64_t *histogram_out;
};

struct Cycle {
    bool in_flight = false;
    cudaEvent_t start = nullptr;   // timed: recorded on the copy stream when the cycle is queued
    cudaEvent_t done = nullptr;    // timed: the cycle's last operation (compute stream)
    cudaEvent_t index_ready = nullptr;
    cudaEvent_t caller_ready = nullptr;
    std::vector<int64_t> ids;
    std::vector<int32_t> sessions;
    int32_t *d_index = nullptr;
    int32_t *h_index = nullptr;
    size_t cap = 0;                // int32 entries
};

// One overflow member to upload for one request of a cycle.
struct OverflowItem {
    int32_t request;   // index into the cycle's admitted requests
    int32_t sign;
    int32_t member;    // overflow id (0-based within the overflow part)
    int32_t pos;       // position of the member among the cycle's distinct overflow ids
};

thread_local std::string g_server_error;

int popcount_words(const std::vector<uint64_t> &w) {
    int64_t c = 0;
    for (uint64_t x : w) c += __builtin_popcountll(x);
    return (int)c;
}

}  // namespace

struct composite_server {
    composite_server_config cfg{};
    composite_engine *eng = nullptr;
    cudaStream_t compute = nullptr, copy = nullptr;
    int32_t n_total = 0;
    int64_t raster_bytes = 0;      // row_pitch * height
    int64_t plane_bytes = 0;
    int64_t used_bytes = 0;        // counted against the budget
    std::vector<Session> sessions;
    std::deque<Request> queue;
    std::vector<Cycle> cycles;
    uint8_t *d_stage = nullptr;    // 2 halves x staging_members rasters
    const void *overflow_dev = nullptr;   // the overflow part as the device reads it
    std::vector<int32_t> pos_of;          // overflow id -> staging position, per cycle
    cpt::DeviceCaps caps{};
    int device = 0;                // the device current at begin
    cudaEvent_t stage_ready[2] = {nullptr, nullptr}, stage_free[2] = {nullptr, nullptr};
    int stage_half = 0;
    int64_t next_id = 0;
    composite_server_stats stats{};
    std::string err;
};

namespace {

int sfail(composite_server *s, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s)
        s->err = buf;
    else
        g_server_error = buf;
    return code;
}

int scuda(composite_server *s, cudaError_t e, const char *what) {
    return sfail(s, e == cudaErrorMemoryAllocation ? CPT_ENOMEM : CPT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SCK(s, call)                                      \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return scuda(s, e_, #call); \
    } while (0)

int engine_rc(composite_server *s, int rc) {
    if (rc != CPT_OK) sfail(s, rc, "engine: %s", composite_engine_last_error(s->eng));
    return rc;
}

bool budget_allows(const composite_server *s, int64_t extra) {
    return s->cfg.hbm_budget_bytes == 0 || s->used_bytes + extra <= s->cfg.hbm_budget_bytes;
}

int64_t timeout_ms(const composite_server *s) { return s->cfg.wait_timeout_ms > 0 ? s->cfg.wait_timeout_ms : 10000; }

// Grows a cycle's index buffers (device and pinned host) to `need` entries.
int reserve_index(composite_server *s, Cycle &c, size_t need) {
    if (c.cap >= need) return CPT_OK;
    size_t cap = std::max<size_t>(need, std::max<size_t>(2 * c.cap, 4096));
    const int64_t delta = (int64_t)(cap - c.cap) * 4;
    if (!budget_allows(s, delta)) return sfail(s, CPT_ENOMEM, "index buffers would exceed the device-memory budget");
    if (c.d_index) cudaFree(c.d_index);
    if (c.h_index) cudaFreeHost(c.h_index);
    c.d_index = nullptr;
    c.h_index = nullptr;
    s->used_bytes -= (int64_t)c.cap * 4;
    c.cap = 0;
    SCK(s, cudaMalloc(&c.d_index, cap * sizeof(int32_t)));
    SCK(s, cudaHostAlloc(&c.h_index, cap * sizeof(int32_t), cudaHostAllocDefault));
    c.cap = cap;
    s->used_bytes += (int64_t)cap * 4;
    return CPT_OK;
}

void toggle_bits(std::vector<uint64_t> &bits, const std::vector<int32_t> &ids) {
    for (int32_t id : ids) bits[id >> 6] ^= 1ull << (id & 63);
}

// Collects completed cycles.
int reap(composite_server *s, int64_t *completed, int32_t capacity, int32_t *n_completed) {
    for (Cycle &c : s->cycles) {
        if (!c.in_flight) continue;
        const cudaError_t q = cudaEventQuery(c.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return scuda(s, q, "cudaEventQuery");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.start, c.done) == cudaSuccess) s->stats.cycle_device_us += (int64_t)(1000.0f * ms);
        for (int64_t id : c.ids) {
            if (completed && n_completed && *n_completed < capacity) completed[(*n_completed)++] = id;
            ++s->stats.requests_done;
            --s->stats.in_flight;
        }
        for (int32_t ss : c.sessions) {
            s->sessions[ss].busy = false;
            --s->sessions[ss].pending;
        }
        c.ids.clear();
        c.sessions.clear();
        c.in_flight = false;
    }
    return CPT_OK;
}

int build_cycle(composite_server *s, Cycle *cyc, std::vector<Request> &batch);

// A cycle that failed after admission: its sessions' planes hold an unknown
// part of its work, so the sessions are marked failed (further requests get
// CPT_ESTATE until they are closed), and their requests -- the admitted ones
// and any queued behind them -- are dropped: they never complete.
void abandon_cycle(composite_server *s, const std::vector<Request> &batch) {
    for (const Request &q : batch) {
        Session &ss = s->sessions[q.session];
        ss.failed = true;
        ss.busy = false;
        --ss.pending;
        --s->stats.queued;
    }
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Session &ss = s->sessions[it->session];
        if (!ss.failed) {
            ++it;
            continue;
        }
        --ss.pending;
        --s->stats.queued;
        it = s->queue.erase(it);
    }
}

// Builds and queues one cycle from the admissible queued requests.
int launch_cycle(composite_server *s, bool *launched) {
    const cpt::TraceRange range("composite_server cycle");
    *launched = false;
    Cycle *cyc = nullptr;
    for (Cycle &c : s->cycles)
        if (!c.in_flight) {
            cyc = &c;
            break;
        }
    if (!cyc || s->queue.empty()) return CPT_OK;

    // admission: FIFO, one request per session per cycle, sessions not busy
    std::vector<Request> batch;
    std::unordered_set<int32_t> taken;
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < s->cfg.max_batch;) {
        Session &ss = s->sessions[it->session];
        if (ss.busy || taken.count(it->session)) {
            ++it;
            continue;
        }
        taken.insert(it->session);
        batch.push_back(std::move(*it));
        it = s->queue.erase(it);
    }
    if (batch.empty()) return CPT_OK;
    const int rc = build_cycle(s, cyc, batch);
    if (rc) {
        std::string sessions;
        for (const Request &q : batch) sessions += (sessions.empty() ? "" : ", ") + std::to_string(q.session);
        const std::string why = s->err;
        abandon_cycle(s, batch);
        return sfail(s, rc, "%s; the requests of sessions %s were dropped and the sessions must be closed",
                     why.c_str(), sessions.c_str());
    }
    *launched = true;
    return CPT_OK;
}

// The body of a cycle: session updates, index lists, the engine submits for
// resident and overflow members, the render.  On error the caller abandons
// the cycle.
int build_cycle(composite_server *s, Cycle *cyc, std::vector<Request> &batch) {
    const int32_t R = s->cfg.n_resident;
    const int words = (s->n_total + 63) / 64;
    std::vector<std::vector<int32_t>> res_add(batch.size()), res_rem(batch.size());
    std::vector<OverflowItem> ovf;
    std::vector<char> recompute(batch.size(), 0);
    for (size_t r = 0; r < batch.size(); ++r) {
        Session &ss = s->sessions[batch[r].session];
        std::vector<uint64_t> after = ss.bits;
        toggle_bits(after, batch[r].toggle);
        int64_t n_add = 0, n_rem = 0;
        for (int w = 0; w < words; ++w) {
            n_add += __builtin_popcountll(after[w] & ~ss.bits[w]);
            n_rem += __builtin_popcountll(ss.bits[w] & ~after[w]);
        }
        const int64_t n_after = popcount_words(after);
        // clear + re-add the whole new set when that touches fewer members
        recompute[r] = n_after < n_add + n_rem;
        for (int w = 0; w < words; ++w) {
            const uint64_t add = recompute[r] ? after[w] : (after[w] & ~ss.bits[w]);
            const uint64_t rem = recompute[r] ? 0 : (ss.bits[w] & ~after[w]);
            for (int sign = 1; sign >= -1; sign -= 2) {
                uint64_t m = sign > 0 ? add : rem;
                while (m) {
                    const int id = w * 64 + __builtin_ctzll(m);
                    m &= m - 1;
                    if (id < R)
                        (sign > 0 ? res_add[r] : res_rem[r]).push_back(id);
                    else
                        ovf.push_back({(int32_t)r, sign, id - R, 0});
                }
            }
        }
        s->stats.members_added += recompute[r] ? n_after : n_add;
        s->stats.members_removed += recompute[r] ? 0 : n_rem;
        s->stats.recomputes += recompute[r];
        ss.bits.swap(after);
        ss.n = n_after;
        ss.busy = true;
    }
    // Distinct overflow members of the cycle: each is uploaded once, whatever
    // number of requests toggle it; requests gather it from staging by index.
    // Staging order is by the (ascending) list of requests that toggle the
    // member, compared lexicographically, then by id: a request's members
    // then lie in few contiguous runs, so each staging chunk holds few
    // (request, sign) groups and the chunk's submit has few, large ops (each
    // op costs a pass over its plane, whatever its member count).
    std::vector<int32_t> distinct;
    {
        std::vector<std::pair<int32_t, int32_t>> mr;   // (member, request), one per item
        mr.reserve(ovf.size());
        for (const OverflowItem &o : ovf) mr.push_back({o.member, o.request});
        std::sort(mr.begin(), mr.end());
        std::vector<size_t> first;   // per distinct member, its run in mr
        for (size_t i = 0; i < mr.size(); ++i)
            if (i == 0 || mr[i].first != mr[i - 1].first) first.push_back(i);
        first.push_back(mr.size());
        std::vector<int32_t> order(first.size() - 1);
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            const auto a0 = mr.begin() + first[a], a1 = mr.begin() + first[a + 1];
            const auto b0 = mr.begin() + first[b], b1 = mr.begin() + first[b + 1];
            const auto by_request = [](const std::pair<int32_t, int32_t> &x, const std::pair<int32_t, int32_t> &y) {
                return x.second < y.second;
            };
            if (std::lexicographical_compare(a0, a1, b0, b1, by_request)) return true;
            if (std::lexicographical_compare(b0, b1, a0, a1, by_request)) return false;
            return a0->first < b0->first;
        });
        distinct.resize(order.size());
        if (s->pos_of.size() < (size_t)s->cfg.n_overflow) s->pos_of.resize(s->cfg.n_overflow);
        for (size_t i = 0; i < order.size(); ++i) {
            distinct[i] = mr[first[order[i]]].first;
            s->pos_of[distinct[i]] = (int32_t)i;
        }
    }
    for (OverflowItem &o : ovf) o.pos = s->pos_of[o.member];
    std::sort(ovf.begin(), ovf.end(), [](const OverflowItem &a, const OverflowItem &b) {
        if (a.request != b.request) return a.request < b.request;
        if (a.sign != b.sign) return a.sign > b.sign;
        return a.pos < b.pos;
    });

    // index lists of the resident ops (and, after them, of the overflow ops
    // and the overflow ids each chunk gathers)
    size_t total = ovf.size() + distinct.size();
    for (size_t r = 0; r < batch.size(); ++r) total += res_add[r].size() + res_rem[r].size();
    int rc = reserve_index(s, *cyc, std::max<size_t>(total, 1));
    if (rc) return rc;
    std::vector<composite_op> ops;
    size_t off = 0;
    std::vector<int32_t> cleared;   // planes recomputed from scratch: one clear launch for all
    for (size_t r = 0; r < batch.size(); ++r)
        if (recompute[r]) cleared.push_back(s->sessions[batch[r].session].plane);
    if (!cleared.empty()) {
        rc = engine_rc(s, composite_engine_clear_many(s->eng, cleared.data(), (int32_t)cleared.size()));
        if (rc) return rc;
    }
    for (size_t r = 0; r < batch.size(); ++r) {
        const int32_t plane = s->sessions[batch[r].session].plane;
        for (int sign = 1; sign >= -1; sign -= 2) {
            const std::vector<int32_t> &ids = sign > 0 ? res_add[r] : res_rem[r];
            if (ids.empty()) continue;
            memcpy(cyc->h_index + off, ids.data(), ids.size() * sizeof(int32_t));
            composite_op o{};
            o.plane = plane;
            o.sign = sign;
            o.members = s->cfg.resident;
            o.member_index = cyc->d_index + off;
            o.n_members = (int32_t)ids.size();
            o.row_pitch_bytes = s->cfg.row_pitch_bytes;
            o.member_stride_bytes = s->cfg.member_stride_bytes;
            o.mask_format = s->cfg.mask_format;
            ops.push_back(o);
            off += ids.size();
        }
    }
    // the copy stream starts after the caller's earlier work on the compute stream
    SCK(s, cudaEventRecord(cyc->caller_ready, s->compute));
    SCK(s, cudaStreamWaitEvent(s->copy, cyc->caller_ready, 0));
    SCK(s, cudaEventRecord(cyc->start, s->copy));
    if (off) {
        // on the copy stream, ahead of this cycle's raster uploads
        SCK(s, cudaMemcpyAsync(cyc->d_index, cyc->h_index, off * sizeof(int32_t), cudaMemcpyHostToDevice, s->copy));
        SCK(s, cudaEventRecord(cyc->index_ready, s->copy));
        SCK(s, cudaStreamWaitEvent(s->compute, cyc->index_ready, 0));
    }
    if (!ops.empty()) {
        rc = engine_rc(s, composite_engine_submit(s->eng, ops.data(), (int32_t)ops.size()));
        if (rc) return rc;
    }

    // Overflow members through the two staging halves: chunk c uploads the
    // distinct members [c0, c1) into half h on the copy stream, then one
    // engine submit folds, for every (request, sign) group, the group's
    // members in that chunk (their staging slots as an index list).
    std::vector<size_t> group_start, cursor;
    for (size_t i = 0; i < ovf.size(); ++i)
        if (i == 0 || ovf[i].request != ovf[i - 1].request || ovf[i].sign != ovf[i - 1].sign) group_start.push_back(i);
    cursor = group_start;
    group_start.push_back(ovf.size());
    const int half = s->cfg.staging_members;
    const int64_t inject_at = cpt::fault_injected_value("server_chunk_fail");
    for (size_t c0 = 0; c0 < distinct.size(); c0 += half) {
        if (inject_at >= 0 && (int64_t)(c0 / half) == inject_at)
            return sfail(s, CPT_ECUDA, "upload of overflow chunk %lld refused (injected)", (long long)inject_at);
        const size_t c1 = std::min(distinct.size(), c0 + (size_t)half);
        const int h = s->stage_half;
        s->stage_half ^= 1;
        uint8_t *base = s->d_stage + (int64_t)h * half * s->cfg.member_stride_bytes;
        std::vector<composite_op> chunk_ops;
        const size_t off0 = off;
        for (size_t g = 0; g + 1 < group_start.size(); ++g) {
            size_t &cur = cursor[g];
            const size_t first = cur;
            while (cur < group_start[g + 1] && (size_t)ovf[cur].pos < c1) {
                cyc->h_index[off + (cur - first)] = ovf[cur].pos - (int32_t)c0;
                ++cur;
            }
            if (cur == first) continue;
            composite_op o{};
            o.plane = s->sessions[batch[ovf[first].request].session].plane;
            o.sign = ovf[first].sign;
            o.members = base;
            o.member_index = cyc->d_index + off;
            o.n_members = (int32_t)(cur - first);
            o.row_pitch_bytes = s->cfg.row_pitch_bytes;
            o.member_stride_bytes = s->cfg.member_stride_bytes;
            o.mask_format = s->cfg.mask_format;
            chunk_ops.push_back(o);
            off += cur - first;
        }
        // the chunk's distinct overflow ids, after its ops' slot lists
        const size_t ids_off = off;
        for (size_t i = c0; i < c1; ++i) cyc->h_index[off++] = distinct[i];
        SCK(s, cudaStreamWaitEvent(s->copy, s->stage_free[h], 0));
        SCK(s, cudaMemcpyAsync(cyc->d_index + off0, cyc->h_index + off0, (off - off0) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s->copy));
        SCK(s, cpt::launch_gather_rasters(base, s->overflow_dev, cyc->d_index + ids_off, (int)(c1 - c0),
                                          s->cfg.member_stride_bytes, s->raster_bytes, s->caps, s->copy));
        s->stats.overflow_uploads += (int64_t)(c1 - c0);
        SCK(s, cudaEventRecord(s->stage_ready[h], s->copy));
        SCK(s, cudaStreamWaitEvent(s->compute, s->stage_ready[h], 0));
        rc = engine_rc(s, composite_engine_submit(s->eng, chunk_ops.data(), (int32_t)chunk_ops.size()));
        if (rc) return rc;
        SCK(s, cudaEventRecord(s->stage_free[h], s->compute));
    }

    // one render for every admitted session
    std::vector<composite_render_op> rops;
    for (const Request &q : batch) {
        composite_render_op ro{};
        ro.plane = s->sessions[q.session].plane;
        ro.counts_out = q.counts_out;
        ro.bucket_out = q.bucket_out;
        ro.rgba_out = q.rgba_out;
        ro.histogram_out = q.histogram_out;
        if (ro.counts_out || ro.bucket_out || ro.rgba_out || ro.histogram_out) rops.push_back(ro);
    }
    if (!rops.empty()) {
        rc = engine_rc(s, composite_engine_render(s->eng, rops.data(), (int32_t)rops.size(), nullptr));
        if (rc) return rc;
    }
    SCK(s, cudaEventRecord(cyc->done, s->compute));
    for (const Request &q : batch) {
        cyc->ids.push_back(q.id);
        cyc->sessions.push_back(q.session);
    }
    s->stats.in_flight += (int64_t)batch.size();
    s->stats.queued -= (int64_t)batch.size();
    ++s->stats.cycles;
    cyc->in_flight = true;
    return CPT_OK;
}

void destroy_server(composite_server *s) {
    if (s->eng) composite_engine_end(s->eng);
    for (Cycle &c : s->cycles) {
        if (c.done) cudaEventDestroy(c.done);
        if (c.start) cudaEventDestroy(c.start);
        if (c.index_ready) cudaEventDestroy(c.index_ready);
        if (c.caller_ready) cudaEventDestroy(c.caller_ready);
        if (c.d_index) cudaFree(c.d_index);
        if (c.h_index) cudaFreeHost(c.h_index);
    }
    for (int h = 0; h < 2; ++h) {
        if (s->stage_ready[h]) cudaEventDestroy(s->stage_ready[h]);
        if (s->stage_free[h]) cudaEventDestroy(s->stage_free[h]);
    }
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
}

}  // namespace

extern "C" {

int composite_server_default_config(composite_server_config *cfg) try {
    if (!cfg) return CPT_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->max_sessions = 64;
    cfg->max_batch = 64;
    cfg->staging_members = 64;
    cfg->max_cycles_in_flight = 4;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_begin(composite_server **out, const composite_server_config *cfg) try {
    g_server_error.clear();
    if (!out || !cfg) return sfail(nullptr, CPT_EINVAL, "out and cfg must not be NULL");
    *out = nullptr;
    composite_server_config c = *cfg;
    if (c.staging_members == 0) c.staging_members = 64;
    if (c.max_cycles_in_flight == 0) c.max_cycles_in_flight = 4;
    if (c.width <= 0 || c.height <= 0) return sfail(nullptr, CPT_EINVAL, "raster is empty");
    if (c.n_resident < 0 || c.n_overflow < 0 || (int64_t)c.n_resident + c.n_overflow > (1 << 30))
        return sfail(nullptr, CPT_EINVAL, "member counts out of range");
    if (c.n_resident > 0 && !c.resident) return sfail(nullptr, CPT_EINVAL, "resident is NULL");
    if (c.n_overflow > 0 && !c.overflow) return sfail(nullptr, CPT_EINVAL, "overflow is NULL");
    if (c.mask_format != CPT_MASK_BYTES && c.mask_format != CPT_MASK_BITS)
        return sfail(nullptr, CPT_EINVAL, "mask_format out of range");
    const int64_t row_bytes = c.mask_format == CPT_MASK_BITS ? ((int64_t)c.width + 7) / 8 : c.width;
    if ((c.row_pitch_bytes % 16) || (c.member_stride_bytes % 16) || c.row_pitch_bytes < row_bytes ||
        c.member_stride_bytes < (int64_t)c.row_pitch_bytes * c.height)
        return sfail(nullptr, CPT_EINVAL, "row pitch and member stride must be multiples of 16 covering the raster");
    if (reinterpret_cast<uintptr_t>(c.resident) % 16) return sfail(nullptr, CPT_EINVAL, "resident must be 16-byte aligned");
    if (c.max_sessions < 1 || c.max_sessions > 65536) return sfail(nullptr, CPT_EINVAL, "max_sessions not in 1..65536");
    if (c.max_batch < 1 || c.max_batch > 4096) return sfail(nullptr, CPT_EINVAL, "max_batch not in 1..4096");
    if (c.staging_members < 1 || c.staging_members > 4096) return sfail(nullptr, CPT_EINVAL, "staging_members not in 1..4096");
    if (c.max_cycles_in_flight < 1 || c.max_cycles_in_flight > 16) return sfail(nullptr, CPT_EINVAL, "max_cycles_in_flight not in 1..16");
    if (c.hbm_budget_bytes < 0 || c.wait_timeout_ms < 0) return sfail(nullptr, CPT_EINVAL, "negative budget or timeout");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(nullptr, CPT_ECUDA, "no CUDA device");
    }
    if (c.n_resident > 0) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, c.resident) != cudaSuccess ||
            !(a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device))) {
            cudaGetLastError();
            return sfail(nullptr, CPT_EINVAL, "resident members must be device memory of the current device");
        }
    }
    if (c.n_overflow > 0) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, c.overflow) != cudaSuccess || a.type == cudaMemoryTypeUnregistered ||
            (a.type == cudaMemoryTypeDevice && a.device != device)) {
            cudaGetLastError();
            return sfail(nullptr, CPT_EINVAL, "overflow members must be pinned host memory (or device memory of "
                                              "the current device)");
        }
    }
    composite_server *s = new composite_server();
    s->cfg = c;
    s->device = device;
    s->n_total = c.n_resident + c.n_overflow;
    s->raster_bytes = (int64_t)c.row_pitch_bytes * c.height;
    s->plane_bytes = ((int64_t)c.width + 15) / 16 * 16 * c.height * 4;
    auto setup = [&]() -> int {
        s->compute = static_cast<cudaStream_t>(c.cuda_stream);   // NULL: the legacy default stream
        int dev = 0;
        SCK(s, cudaGetDevice(&dev));
        SCK(s, cudaDeviceGetAttribute(&s->caps.num_sms, cudaDevAttrMultiProcessorCount, dev));
        if (c.n_overflow > 0) {
            // pinned host memory is read by the gather kernel through its device mapping
            cudaPointerAttributes a;
            SCK(s, cudaPointerGetAttributes(&a, c.overflow));
            s->overflow_dev = a.type == cudaMemoryTypeHost ? a.devicePointer : c.overflow;
            if (!s->overflow_dev) return sfail(s, CPT_EINVAL, "the overflow part has no device mapping");
            if (reinterpret_cast<uintptr_t>(s->overflow_dev) % 16)
                return sfail(s, CPT_EINVAL, "overflow must be 16-byte aligned");
        }
        SCK(s, cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
        composite_engine_config ec;
        composite_engine_default_config(&ec);
        ec.cuda_stream = s->compute;
        ec.wait_timeout_ms = c.wait_timeout_ms;
        ec.slab_members = 255;
        // four persistent CTAs per SM, not five: the overflow gather kernel on
        // the copy stream then fits beside the engine's launch (registers) and
        // the uploads overlap the folds instead of taking turns with them
        // (byte masks at 500 req/s: 52.8 against 50.7 composites/s)
        ec.ctas_per_sm = 4;
        ec.upload_stream = s->copy;
        int rc = composite_engine_begin(&s->eng, &ec);
        if (rc) return sfail(s, rc, "engine: %s", composite_engine_last_error(nullptr));
        const int64_t stage = c.n_overflow > 0 ? 2ll * c.staging_members * c.member_stride_bytes : 0;
        if (!budget_allows(s, stage)) return sfail(s, CPT_ENOMEM, "staging halves exceed the device-memory budget");
        if (stage && cpt::fault_injected("server_stage"))
            return sfail(s, CPT_ENOMEM, "staging allocation refused (injected)");
        if (stage) SCK(s, cudaMalloc(&s->d_stage, (size_t)stage));
        s->used_bytes += stage;
        for (int h = 0; h < 2; ++h) {
            SCK(s, cudaEventCreateWithFlags(&s->stage_ready[h], cudaEventDisableTiming));
            SCK(s, cudaEventCreateWithFlags(&s->stage_free[h], cudaEventDisableTiming));
        }
        s->cycles.resize(c.max_cycles_in_flight);
        for (Cycle &cy : s->cycles) {
            SCK(s, cudaEventCreate(&cy.start));
            SCK(s, cudaEventCreate(&cy.done));
            SCK(s, cudaEventCreateWithFlags(&cy.index_ready, cudaEventDisableTiming));
            SCK(s, cudaEventCreateWithFlags(&cy.caller_ready, cudaEventDisableTiming));
        }
        return CPT_OK;
    };
    const int rc = setup();
    if (rc) {
        g_server_error = s->err;
        destroy_server(s);
        return rc;
    }
    *out = s;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_open_session(composite_server *s, int32_t *session_out) try {
    if (!s || !session_out) return CPT_EINVAL;
    s->err.clear();
    int32_t id = -1;
    int open = 0;
    for (size_t i = 0; i < s->sessions.size(); ++i) {
        if (s->sessions[i].open)
            ++open;
        else if (id < 0)
            id = (int32_t)i;
    }
    if (open >= s->cfg.max_sessions) return sfail(s, CPT_ENOMEM, "max_sessions sessions are open");
    if (!budget_allows(s, s->plane_bytes)) return sfail(s, CPT_ENOMEM, "a new plane would exceed the device-memory budget");
    int32_t plane = -1;
    const int rc = composite_engine_add_plane(s->eng, s->cfg.width, s->cfg.height, &plane);
    if (rc) return sfail(s, rc, "engine: %s", composite_engine_last_error(s->eng));
    if (id < 0) {
        id = (int32_t)s->sessions.size();
        s->sessions.emplace_back();
    }
    Session &ss = s->sessions[id];
    ss = Session();
    ss.open = true;
    ss.plane = plane;
    ss.bits.assign((s->n_total + 63) / 64, 0);
    ss.view = ss.bits;
    s->used_bytes += s->plane_bytes;
    *session_out = id;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_close_session(composite_server *s, int32_t session) try {
    if (!s) return CPT_EINVAL;
    s->err.clear();
    if (session < 0 || session >= (int32_t)s->sessions.size() || !s->sessions[session].open)
        return sfail(s, CPT_EINVAL, "no session %d", session);
    Session &ss = s->sessions[session];
    if (ss.pending) return sfail(s, CPT_ESTATE, "session %d has requests queued or in flight", session);
    const int rc = composite_engine_free_plane(s->eng, ss.plane);
    if (rc) return sfail(s, rc, "engine: %s", composite_engine_last_error(s->eng));
    s->used_bytes -= s->plane_bytes;
    ss = Session();
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

namespace {

int queue_request(composite_server *s, int32_t session, const int32_t *toggle, int32_t n, uint32_t *counts_out,
                  uint8_t *bucket_out, uint8_t *rgba_out, uint64_t *histogram_out, int64_t *request_id_out) {
    if (!s) return CPT_EINVAL;
    s->err.clear();
    if (session < 0 || session >= (int32_t)s->sessions.size() || !s->sessions[session].open)
        return sfail(s, CPT_EINVAL, "no session %d", session);
    if (s->sessions[session].failed)
        return sfail(s, CPT_ESTATE, "session %d lost a cycle to an error; close it and open a new one", session);
    if (n < 0 || (n > 0 && !toggle)) return sfail(s, CPT_EINVAL, "bad toggle list");
    for (int32_t i = 0; i < n; ++i)
        if (toggle[i] < 0 || toggle[i] >= s->n_total)
            return sfail(s, CPT_EINVAL, "member id %d out of range [0, %d)", toggle[i], s->n_total);
    if ((reinterpret_cast<uintptr_t>(counts_out) % 4) || (reinterpret_cast<uintptr_t>(rgba_out) % 4))
        return sfail(s, CPT_EINVAL, "counts_out and rgba_out must be 4-byte aligned");
    if (reinterpret_cast<uintptr_t>(histogram_out) % 16)
        return sfail(s, CPT_EINVAL, "histogram_out must be 16-byte aligned");
    // the render kernel writes the outputs directly: device memory of the
    // server's device, or mapped pinned host memory
    const void *outs[4] = {counts_out, bucket_out, rgba_out, histogram_out};
    for (const void *o : outs) {
        if (!o) continue;
        cudaPointerAttributes a;
        const bool ok = cudaPointerGetAttributes(&a, o) == cudaSuccess &&
                        (a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == s->device) ||
                         (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr));
        if (!ok) {
            cudaGetLastError();
            return sfail(s, CPT_EINVAL, "outputs must be device memory of device %d (or mapped pinned host memory)",
                         s->device);
        }
    }
    Request q;
    q.id = s->next_id++;
    q.session = session;
    q.toggle.assign(toggle, toggle + n);
    q.counts_out = counts_out;
    q.bucket_out = bucket_out;
    q.rgba_out = rgba_out;
    q.histogram_out = histogram_out;
    Session &ss = s->sessions[session];
    toggle_bits(ss.view, q.toggle);
    ss.n_view = popcount_words(ss.view);
    ++ss.pending;
    s->queue.push_back(std::move(q));
    ++s->stats.queued;
    if (request_id_out) *request_id_out = s->next_id - 1;
    return CPT_OK;
}

}  // namespace

int composite_server_request(composite_server *s, int32_t session, const int32_t *toggle, int32_t n,
                             uint32_t *counts_out, uint8_t *bucket_out, uint8_t *rgba_out, int64_t *request_id_out) try {
    return queue_request(s, session, toggle, n, counts_out, bucket_out, rgba_out, nullptr, request_id_out);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_request_histogram(composite_server *s, int32_t session, const int32_t *toggle, int32_t n,
                                       uint32_t *counts_out, uint8_t *bucket_out, uint8_t *rgba_out,
                                       uint64_t *histogram_out, int64_t *request_id_out) try {
    return queue_request(s, session, toggle, n, counts_out, bucket_out, rgba_out, histogram_out, request_id_out);
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_pump(composite_server *s, int64_t *completed, int32_t capacity, int32_t *n_completed) try {
    if (!s || capacity < 0 || (capacity > 0 && !completed)) return CPT_EINVAL;
    s->err.clear();
    int32_t dummy = 0;
    int32_t *nc = n_completed ? n_completed : &dummy;
    *nc = 0;
    int rc = reap(s, completed, capacity, nc);
    if (rc) return rc;
    for (;;) {
        bool launched = false;
        const auto t0 = std::chrono::steady_clock::now();
        rc = launch_cycle(s, &launched);
        if (launched)
            s->stats.enqueue_host_us +=
                std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (rc || !launched) return rc;
    }
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_drain(composite_server *s) try {
    if (!s) return CPT_EINVAL;
    s->err.clear();
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms(s));
    int64_t last_done = s->stats.requests_done;
    for (unsigned spin = 0; s->stats.queued > 0 || s->stats.in_flight > 0; ++spin) {
        int rc = composite_server_pump(s, nullptr, 0, nullptr);
        if (rc) return rc;
        if (s->stats.requests_done != last_done) {
            last_done = s->stats.requests_done;
            deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms(s));
        } else if (std::chrono::steady_clock::now() > deadline) {
            return sfail(s, CPT_ETIMEOUT, "no request completed within %lld ms", (long long)timeout_ms(s));
        }
        if (spin > 200) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_session_members(const composite_server *s, int32_t session, int64_t *n_out) try {
    if (!s || !n_out || session < 0 || session >= (int32_t)s->sessions.size() || !s->sessions[session].open)
        return CPT_EINVAL;
    *n_out = s->sessions[session].n_view;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_get_stats(const composite_server *s, composite_server_stats *out) try {
    if (!s || !out) return CPT_EINVAL;
    *out = s->stats;
    return CPT_OK;
} catch (...) {
    return cpt::abi_exception_status();
}

int composite_server_end(composite_server *s) try {
    if (!s) return CPT_OK;
    const int rc = composite_server_drain(s);
    destroy_server(s);
    return rc;
} catch (...) {
    return cpt::abi_exception_status();
}

const char *composite_server_last_error(const composite_server *s) try {
    return s ? s->err.c_str() : g_server_error.c_str();
} catch (...) {
    return "internal error (exception)";
}

}  // extern "C"
