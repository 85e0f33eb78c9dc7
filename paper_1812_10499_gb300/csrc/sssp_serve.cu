// sssp_serve.cu -- continuous-batching query server of the GB300 bound-based
// SSSP library (Garg, arXiv 1812.10499).
//
// All admitted queries share one multi-query solve context.  Their records
// live in a paged pool (1024 records per page, each query a contiguous page
// range) sized from the device-memory budget; a page table maps a record to
// its query slot.  A server step (1) admits queued queries into free slots
// and pages, initialises their records and puts their sources into the
// current round's frontier; (2) runs a few rounds of the shared loop (the
// CUDA graph with the device-side while node, as a single solve); (3) copies
// out every query that finished and frees its slot and pages.  Each query
// keeps its own thresholds and round counter, so its rounds -- and its
// result -- do not depend on the other queries in flight.
//
// A server thread runs the steps while any query is queued or in flight, so
// queries complete without the client calling in; with SSSP_SERVE_MANUAL the
// client's poll / wait / drain calls run them instead.  Host bookkeeping
// (queue, tickets, query states, counters) is guarded by `mu`; the device
// state (slots, pages, the context) is touched only by the step that holds
// `step_mu`.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "sssp_engine.h"

using namespace sssp;
using namespace sssp::engine;

namespace {

constexpr u32 kServeVbits = 32;            // parent ids up to 2^32 - 1, distances below 2^32
// Device bytes per record: record, fixing round, distance staging, the
// small lists (4 x 4 B), the hub lists (4 x 8 B), the chunk maps (4 x 4 B)
// and the hub reduction slots (8 B + 4 B).
constexpr u64 kBytesPerRecordCommon = 4 + 8 + 16 + 32 + 16 + 12;
// The compact layout adds the relaxation filter word (8 B).

enum QState { kQueued = 0, kInFlight = 1, kComplete = 2 };

u64 now_ns() {
    return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Query {
    u64 ticket = 0;
    sssp_graph* g = nullptr;
    u32 source = 0;
    u64* out = nullptr;
    u32 slot = 0;
    u32 first_page = 0, npages = 0;
    u32 rounds = 0;
    QState state = kQueued;
    u64 submit_ns = 0, admit_ns = 0, done_ns = 0;
    u64 first_step = 0, last_step = 0;
};

}  // namespace

struct sssp_server {
    int device = 0;
    sssp_serve_cfg cfg{};
    bool narrow = true;                 // 16-byte records
    Context ctx;
    cudaStream_t stream = nullptr;
    u32 round_host = 1;
    u32* h_stop = nullptr;              // pinned staging for the stop round
    // Device-side bookkeeping: only the step holding step_mu touches it.
    std::mutex step_mu;
    std::vector<unsigned char> page_used;
    std::vector<u32> free_slots;
    std::vector<Query*> slot_query;
    u32 inflight = 0;
    // Finished queries whose distances wait in the page-locked staging h_out
    // (at the given offsets) to be copied into their output arrays.
    u64* h_out = nullptr;
    u64 h_out_n = 0;
    std::vector<std::pair<Query*, u64>> deliver;
    // Host-side bookkeeping, guarded by mu.
    std::mutex mu;
    std::condition_variable cv_work;    // a query was queued, or the server closes
    std::condition_variable cv_done;    // a step finished (queries may have completed)
    std::deque<Query*> pending;
    std::unordered_map<u64, Query*> tickets;
    u64 next_ticket = 0;
    u64 steps = 0, rounds = 0, submitted = 0, completed = 0;
    u32 inflight_seen = 0, max_inflight = 0;
    int error = SSSP_OK;                // the error that stopped the server
    bool stop = false;
    bool stuck = false;                 // queued queries, none in flight, none admissible
    std::thread worker;
};

namespace {

int open_impl(sssp_server* s) {
    Context& c = s->ctx;
    const sssp_serve_cfg& cfg = s->cfg;
    c.pool.al = Allocator{cfg.alloc, cfg.free, cfg.alloc_ctx};
    c.multi = true;
    c.narrow = s->narrow;
    const u64 per_rec =
        kBytesPerRecordCommon + (s->narrow ? sizeof(VRecN) + sizeof(uint2) : sizeof(VRec));
    u64 nrec = cfg.budget_bytes / per_rec;
    // Record ids are 32-bit list entries.
    nrec = std::min<u64>(nrec, 0xFFFFFF00ull);
    nrec = (nrec >> kPageShift) << kPageShift;
    if (nrec < (1u << kPageShift)) return SSSP_E_NOMEM;
    c.nrec = nrec;
    c.nslots = cfg.max_slots;
    c.npages = (u32)(nrec >> kPageShift);
    CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    c.grid = std::max(1, sms) * std::max(1, round_blocks_per_sm(kThreads));
    c.grid_cup = std::max(1, sms) * std::max(1, cupdate_blocks_per_sm(kThreads));
    c.grid_solve = std::max(1, sms) * std::max(1, solve_blocks_per_sm(kThreads));
    c.tail_ctas = tail_cluster_ctas();
    RoundParams& P = c.P;
    P.tail_items = kDefaultTailItems;
    if (s->narrow) {
        // Records, then (when the records fit the persisting L2) the
        // relaxation filter words.
        const bool filt = records_fit_l2((size_t)nrec * sizeof(VRecN), s->device);
        unsigned char* buf = nullptr;
        RC(c.pool.get(&buf, (size_t)nrec * (sizeof(VRecN) + (filt ? sizeof(uint2) : 0))));
        P.recn = reinterpret_cast<VRecN*>(buf);
        P.gf = filt ? reinterpret_cast<uint2*>(buf + (size_t)nrec * sizeof(VRecN)) : nullptr;
    } else {
        RC(c.pool.get(&P.rec, nrec));
    }
    RC(c.pool.get(&P.fround, nrec));
    set_l2_window(c, s->device);
    RC(alloc_hot(c, c.nslots, s->stream));
    InstDesc* idesc = nullptr;
    u32* pages = nullptr;
    RC(c.pool.get(&idesc, c.nslots));
    RC(c.pool.get(&pages, c.npages));
    P.idesc = idesc;
    P.page_owner = pages;
    RC(c.pool.get(&c.stage, nrec));
    // Chunk maps sized like the record pool; chunks beyond are found by search.
    RC(alloc_lists(c, nrec, nrec, nrec));
    P.page_shift = kPageShift;
    P.hub = kDefaultHub;
    P.chunk = kDefaultChunk;
    P.rule = SSSP_RULE_THRESHOLD;
    P.vbits = kServeVbits;
    P.dinf = (~0ull) >> kServeVbits;
    RC(alloc_pinned(c, c.nslots));
    CK(cudaHostAlloc((void**)&c.h_desc, sizeof(InstDesc) * c.nslots, cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&c.h_pages, sizeof(u32) * c.npages, cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&s->h_stop, sizeof(u32), cudaHostAllocDefault));
    s->h_out_n = 1u << 23;
    CK(cudaHostAlloc((void**)&s->h_out, sizeof(u64) * s->h_out_n, cudaHostAllocDefault));
    CK(cudaMemsetAsync(P.L.hubmin, 0xFF, sizeof(u64) * c.capH, s->stream));
    CK(cudaMemsetAsync(P.L.hubcnt, 0, sizeof(u32) * c.capH, s->stream));
    CK(cudaMemsetAsync(P.ivar, 0, sizeof(InstVar) * c.nslots, s->stream));
    CK(cudaMemsetAsync((void*)P.page_owner, 0xFF, sizeof(u32) * c.npages, s->stream));
    k_reset_ctl<<<1, 32, 0, s->stream>>>(P.ctl, c.nslots, 0xFFFFFFF0u);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    s->page_used.assign(c.npages, 0);
    s->slot_query.assign(c.nslots, nullptr);
    for (u32 i = c.nslots; i > 0; --i) s->free_slots.push_back(i - 1);
    return SSSP_OK;
}

// First fit over the page map; returns false when no run of `np` pages is free.
bool find_pages(const sssp_server* s, u32 np, u32* first) {
    u32 run = 0;
    for (u32 p = 0; p < (u32)s->page_used.size(); ++p) {
        run = s->page_used[p] ? 0 : run + 1;
        if (run == np) {
            *first = p + 1 - np;
            return true;
        }
    }
    return false;
}

// Admits queued queries that fit (in queue order, skipping those that do
// not fit yet).  Caller holds step_mu; takes mu for the queue.
int admit(sssp_server* s, u64 step) {
    Context& c = s->ctx;
    std::vector<Query*> take;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            if (s->free_slots.size() <= take.size()) break;
            Query* q = *it;
            u32 first = 0;
            if (!find_pages(s, q->npages, &first)) {
                ++it;
                continue;
            }
            for (u32 p = 0; p < q->npages; ++p) s->page_used[first + p] = 1;
            q->first_page = first;
            take.push_back(q);
            it = s->pending.erase(it);
        }
        // Counted as in flight from the moment they leave the queue, so that a
        // waiter never sees a query neither queued nor in flight before it is
        // complete.
        s->inflight_seen += (u32)take.size();
    }
    for (Query* q : take) {
        const u32 slot = s->free_slots.back();
        s->free_slots.pop_back();
        q->slot = slot;
        const u32 first = q->first_page;
        for (u32 p = 0; p < q->npages; ++p) c.h_pages[first + p] = slot;
        const sssp_graph* g = q->g;
        c.h_desc[slot] = InstDesc{g->out_off, g->out_adj, g->in_off, g->in_adj,
                                  s->narrow ? g->outw_pack : g->outw, g->inw,
                                  (u64)first << kPageShift, g->n, q->source};
        CK(cudaMemcpyAsync((void*)(c.P.idesc + slot), c.h_desc + slot, sizeof(InstDesc),
                           cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync((void*)(c.P.page_owner + first), c.h_pages + first,
                           sizeof(u32) * q->npages, cudaMemcpyHostToDevice, s->stream));
        k_init_records_multi<<<c.grid, kThreads, 0, s->stream>>>(c.P, c.nrec, first, q->npages);
        CK(cudaGetLastError());
        CK(launch_start(true, s->narrow, c.P, slot, 1, 0, s->stream));
        s->slot_query[slot] = q;
        s->inflight++;
    }
    if (!take.empty()) {
        const u64 t = now_ns();
        std::lock_guard<std::mutex> lk(s->mu);
        for (Query* q : take) {
            q->state = kInFlight;
            q->admit_ns = t;
            q->first_step = step;
        }
    }
    return SSSP_OK;
}

// Reads the per-query status after the step's rounds and writes out every
// finished query.  Caller holds step_mu.
int retire(sssp_server* s, u64 step, u32* rounds_run) {
    Context& c = s->ctx;
    CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(c.h_ivar, c.P.ivar, sizeof(InstVar) * c.nslots, cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (c.h_ctl->error & 4u) return SSSP_E_DEVICE_TIMEOUT;
    if (c.h_ctl->error) return SSSP_E_INTERNAL;
    if (c.h_ctl->status == kErrRounds) return SSSP_E_ROUND_LIMIT;
    *rounds_run = c.h_ctl->round - s->round_host;
    s->round_host = c.h_ctl->round;
    std::vector<Query*> done;
    u64 total = 0;
    for (u32 slot = 0; slot < c.nslots; ++slot) {
        Query* q = s->slot_query[slot];
        if (!q || c.h_ivar[slot].status != kDone) continue;
        done.push_back(q);
        total += q->g->n;
    }
    // The staging is free here: the previous step's results were delivered
    // before this step's status read.
    if (total > s->h_out_n) {
        cudaFreeHost(s->h_out);
        s->h_out = nullptr;
        s->h_out_n = 0;
        const u64 n = std::max<u64>(total, 2 * (u64)(1u << 23));
        CK(cudaHostAlloc((void**)&s->h_out, sizeof(u64) * n, cudaHostAllocDefault));
        s->h_out_n = n;
    }
    u64 off = 0;
    for (Query* q : done) {
        const u32 slot = q->slot;
        const u64 base = (u64)q->first_page << kPageShift;
        k_finalize<<<c.grid, kThreads, 0, s->stream>>>(c.P.rec, c.P.recn, c.P.fround, base,
                                                       q->g->n, c.P.vbits, c.P.ivar + slot,
                                                       c.stage + base, nullptr, nullptr, nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(s->h_out + off, c.stage + base, sizeof(u64) * q->g->n,
                           cudaMemcpyDeviceToHost, s->stream));
        q->rounds = c.h_ivar[slot].rounds;
        q->last_step = step;
        s->deliver.emplace_back(q, off);
        off += q->g->n;
    }
    if (!done.empty()) CK(cudaStreamSynchronize(s->stream));
    // The distances are on the host: the slots and pages take new queries.
    for (Query* q : done) {
        for (u32 p = 0; p < q->npages; ++p) s->page_used[q->first_page + p] = 0;
        s->slot_query[q->slot] = nullptr;
        s->free_slots.push_back(q->slot);
        s->inflight--;
    }
    return SSSP_OK;
}

// Copies the finished queries' distances from the staging into their output
// arrays and completes them.  A step does this after it has launched its
// rounds, so the copies overlap the device's work.  Caller holds step_mu.
void deliver(sssp_server* s) {
    if (s->deliver.empty()) return;
    for (const auto& d : s->deliver)
        memcpy(d.first->out, s->h_out + d.second, sizeof(u64) * d.first->g->n);
    const u64 t = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    for (const auto& d : s->deliver) {
        d.first->state = kComplete;
        d.first->done_ns = t;
    }
    s->completed += s->deliver.size();
    s->deliver.clear();
}

// One server step: admission, a few rounds of every query in flight,
// retirement.  Caller holds step_mu (not mu).
int step(sssp_server* s) {
    u64 step_no;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != SSSP_OK) return s->error;
        step_no = s->steps + 1;
    }
    int rc = admit(s, step_no);
    u32 ran = 0, inflight = s->inflight;
    bool stuck = false;
    if (rc == SSSP_OK && s->inflight > 0) {
        Context& c = s->ctx;
        *s->h_stop = s->round_host + s->cfg.rounds_per_step - 1;
        cudaError_t e = cudaMemcpyAsync(&c.P.ctl->stop_round, s->h_stop, sizeof(u32),
                                        cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            rc = SSSP_E_CUDA;
        }
        if (rc == SSSP_OK) rc = run_loop(c, SSSP_LOOP_GRAPH, s->stream);
        deliver(s);    // the previous step's results, while the rounds run
        if (rc == SSSP_OK) rc = retire(s, step_no, &ran);
    } else if (rc == SSSP_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        stuck = !s->pending.empty();   // nothing on the device and nothing admissible
    }
    // With nothing left on the device no step may follow soon: deliver now.
    if (s->inflight == 0) deliver(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (inflight > 0) {
            s->steps = step_no;
            s->rounds += ran;
            s->max_inflight = std::max(s->max_inflight, inflight);
        }
        s->inflight_seen = s->inflight + (u32)s->deliver.size();
        s->stuck = stuck;
        if (rc != SSSP_OK && s->error == SSSP_OK) s->error = rc;
    }
    s->cv_done.notify_all();
    return rc;
}

// The server thread: steps while queries are queued or in flight.
void worker_main(sssp_server* s) {
    DeviceGuard dg(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [s] {
                return s->stop || s->error != SSSP_OK ||
                       (!s->pending.empty() && !s->stuck) || s->inflight_seen > 0;
            });
            if (s->stop || s->error != SSSP_OK) break;
        }
        std::lock_guard<std::mutex> slk(s->step_mu);
        step(s);
    }
    s->cv_done.notify_all();
}

bool manual(const sssp_server* s) { return (s->cfg.flags & SSSP_SERVE_MANUAL) != 0; }

// Manual mode: one step on the caller's thread.
int manual_step(sssp_server* s) {
    DeviceGuard dg(s->device);
    std::lock_guard<std::mutex> slk(s->step_mu);
    return step(s);
}

// Reports a completed query and releases its ticket (caller holds mu).
void take_result(sssp_server* s, std::unordered_map<u64, Query*>::iterator it, uint32_t* rounds,
                 sssp_query_info* info) {
    Query* q = it->second;
    if (rounds) *rounds = q->rounds;
    if (info) {
        info->rounds = q->rounds;
        info->reserved = 0;
        info->submit_ns = q->submit_ns;
        info->admit_ns = q->admit_ns;
        info->done_ns = q->done_ns;
        info->first_step = q->first_step;
        info->last_step = q->last_step;
    }
    s->tickets.erase(it);
    delete q;
}

}  // namespace

extern "C" {

int sssp_serve_open(const sssp_serve_cfg* cfg, sssp_server** out) {
    if (!out) return SSSP_E_INVAL;
    sssp_serve_cfg c{};
    if (cfg) c = *cfg;
    if (c.budget_bytes == 0) c.budget_bytes = 32ull << 30;
    if (c.max_slots == 0) c.max_slots = 1024;
    if (c.rounds_per_step == 0) c.rounds_per_step = 8;
    if ((c.alloc == nullptr) != (c.free == nullptr)) return SSSP_E_INVAL;
    if (c.flags & ~(SSSP_SERVE_MANUAL | SSSP_SERVE_WIDE)) return SSSP_E_INVAL;
    int dev = c.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SSSP_E_CUDA;
    }
    sssp_server* s = new (std::nothrow) sssp_server();
    if (!s) return SSSP_E_NOMEM;
    s->device = dev;
    s->cfg = c;
    s->narrow = (c.flags & SSSP_SERVE_WIDE) == 0;
    int rc;
    {
        DeviceGuard dg(dev);
        rc = open_impl(s);
        if (rc != SSSP_OK) {
            s->ctx.destroy();
            if (s->h_stop) cudaFreeHost(s->h_stop);
            if (s->h_out) cudaFreeHost(s->h_out);
            if (s->stream) cudaStreamDestroy(s->stream);
        }
    }
    if (rc != SSSP_OK) {
        delete s;
        return rc;
    }
    if (!manual(s)) {
        try {
            s->worker = std::thread(worker_main, s);
        } catch (...) {
            DeviceGuard dg(dev);
            s->ctx.destroy();
            cudaFreeHost(s->h_stop);
            if (s->h_out) cudaFreeHost(s->h_out);
            cudaStreamDestroy(s->stream);
            delete s;
            return SSSP_E_NOMEM;
        }
    }
    *out = s;
    return SSSP_OK;
}

int sssp_serve_submit(sssp_server* s, sssp_handle g, uint32_t source, uint64_t* dist_out,
                      uint64_t* ticket) {
    if (!s || !g || !dist_out || !ticket) return SSSP_E_INVAL;
    if (source >= g->n) return SSSP_E_SOURCE_RANGE;
    // Any hub degree and chunk size: a graph's in-hub flags (built for its
    // own hub degree) only place vertices in one work list or the other.
    if (g->device != s->device || g->opt.rule != s->ctx.P.rule) return SSSP_E_INVAL;
    if (s->narrow && !g->narrow) return SSSP_E_OVERFLOW;   // needs 32-byte records
    if (g->vbits > kServeVbits ||
        (g->wmax && (unsigned __int128)g->n * g->wmax >= (unsigned __int128)s->ctx.P.dinf))
        return SSSP_E_OVERFLOW;
    const u32 np = (u32)(((u64)g->n + (1u << kPageShift) - 1) >> kPageShift);
    if (np > s->ctx.npages) return SSSP_E_BUSY;
    Query* q = new (std::nothrow) Query();
    if (!q) return SSSP_E_NOMEM;
    q->g = g;
    q->source = source;
    q->out = reinterpret_cast<u64*>(dist_out);
    q->npages = np;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != SSSP_OK) {
            delete q;
            return s->error;
        }
        q->ticket = ++s->next_ticket;
        q->submit_ns = now_ns();
        s->pending.push_back(q);
        s->tickets[q->ticket] = q;
        s->submitted++;
        s->stuck = false;
        *ticket = q->ticket;
    }
    s->cv_work.notify_one();
    return SSSP_OK;
}

int sssp_serve_poll(sssp_server* s, uint64_t ticket, uint32_t* rounds_out) {
    if (!s) return SSSP_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return SSSP_E_NOT_FOUND;
        if (it->second->state == kComplete) {
            take_result(s, it, rounds_out, nullptr);
            return SSSP_OK;
        }
        if (s->error != SSSP_OK) return s->error;
    }
    if (!manual(s)) return SSSP_PENDING;
    RC(manual_step(s));
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOT_FOUND;
    if (it->second->state != kComplete) return SSSP_PENDING;
    take_result(s, it, rounds_out, nullptr);
    return SSSP_OK;
}

int sssp_serve_wait(sssp_server* s, uint64_t ticket, uint32_t timeout_ms, sssp_query_info* info) {
    if (!s) return SSSP_E_INVAL;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto it = s->tickets.find(ticket);
            if (it == s->tickets.end()) return SSSP_E_NOT_FOUND;
            if (!manual(s)) {
                s->cv_done.wait_until(lk, deadline, [s, ticket] {
                    auto jt = s->tickets.find(ticket);
                    return jt == s->tickets.end() || jt->second->state == kComplete ||
                           s->error != SSSP_OK;
                });
                it = s->tickets.find(ticket);
                if (it == s->tickets.end()) return SSSP_E_NOT_FOUND;
            }
            if (it->second->state == kComplete) {
                take_result(s, it, nullptr, info);
                return SSSP_OK;
            }
            if (s->error != SSSP_OK) return s->error;
            if (std::chrono::steady_clock::now() >= deadline) return SSSP_PENDING;
            if (!manual(s)) continue;
            if (s->stuck && s->inflight_seen == 0) return SSSP_E_BUSY;
        }
        RC(manual_step(s));
    }
}

int sssp_serve_drain(sssp_server* s) {
    if (!s) return SSSP_E_INVAL;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!manual(s)) {
                s->cv_done.wait(lk, [s] {
                    return s->error != SSSP_OK || s->stuck ||
                           (s->pending.empty() && s->inflight_seen == 0);
                });
            }
            if (s->error != SSSP_OK) return s->error;
            if (s->pending.empty() && s->inflight_seen == 0) return SSSP_OK;
            if (s->stuck && s->inflight_seen == 0) return SSSP_E_BUSY;   // nothing admissible
            if (!manual(s)) continue;
        }
        RC(manual_step(s));
    }
}

int sssp_serve_stats_get(sssp_server* s, sssp_serve_stats* out) {
    if (!s || !out) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->steps = s->steps;
    out->rounds = s->rounds;
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queued = (u32)s->pending.size();
    out->inflight = s->inflight_seen;
    out->max_inflight = s->max_inflight;
    out->layout = s->narrow ? SSSP_LAYOUT_COMPACT : SSSP_LAYOUT_WIDE;
    return SSSP_OK;
}

void sssp_serve_close(sssp_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        DeviceGuard dg(s->device);
        if (s->stream) cudaStreamSynchronize(s->stream);
        s->ctx.destroy();
        if (s->h_stop) cudaFreeHost(s->h_stop);
        if (s->h_out) cudaFreeHost(s->h_out);
        if (s->stream) cudaStreamDestroy(s->stream);
    }
    for (auto& kv : s->tickets) delete kv.second;
    delete s;
}

}  // extern "C"
