// sssp_serve.cu -- continuous-batching query server of the GB300 bound-based
// SSSP library (Garg, arXiv 1812.10499).
//
// All admitted queries share one multi-query solve context.  Their records
// live in a paged pool (1024 records per page, each query a contiguous page
// range) sized from the device-memory budget; a page table maps a record to
// its query slot.  A server step (1) admits queued queries into free slots
// and pages, initialises their records and puts their sources into the
// current round's frontier; (2) runs a few rounds of the shared loop; (3)
// copies out every query that finished and frees its slot and pages.  Each
// query keeps its own thresholds and round counter, so its rounds -- and its
// result -- do not depend on the other queries in flight.
#include <deque>
#include <unordered_map>

#include "sssp_engine.h"

namespace sssp {
}  // namespace sssp

using namespace sssp;
using namespace sssp::engine;

namespace {

constexpr u32 kServeVbits = 32;            // parent ids up to 2^32 - 1, distances below 2^32
constexpr u64 kBytesPerRecord = 32 + 16 + 32 + 8 + 4 + 8;

enum QState { kQueued = 0, kInFlight = 1, kComplete = 2 };

struct Query {
    u64 ticket = 0;
    sssp_graph* g = nullptr;
    u32 source = 0;
    u64* out = nullptr;
    u32 slot = 0;
    u32 first_page = 0, npages = 0;
    u32 rounds = 0;
    QState state = kQueued;
};

}  // namespace

struct sssp_server {
    int device = 0;
    sssp_serve_cfg cfg{};
    Context ctx;
    cudaStream_t stream = nullptr;
    u32 round_host = 1;
    u32* h_stop = nullptr;              // pinned staging for the stop round
    std::vector<unsigned char> page_used;
    std::vector<u32> free_slots;
    std::vector<Query*> slot_query;
    std::deque<Query*> pending;
    std::unordered_map<u64, Query*> tickets;
    u64 next_ticket = 0;
    u32 inflight = 0;
};

namespace {

int open_impl(sssp_server* s) {
    Context& c = s->ctx;
    const sssp_serve_cfg& cfg = s->cfg;
    c.pool.al = Allocator{cfg.alloc, cfg.free, cfg.alloc_ctx};
    c.multi = true;
    u64 nrec = cfg.budget_bytes / kBytesPerRecord;
    // Record ids are 32-bit list entries.
    nrec = std::min<u64>(nrec, 0xFFFFFFFFull);
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
    RoundParams& P = c.P;
    RC(c.pool.get(&P.rec, nrec));
    RC(c.pool.get(&P.fround, nrec));
    RC(c.pool.get(&P.ctl, 1));
    RC(c.pool.get(&P.ivar, c.nslots));
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

int admit(sssp_server* s) {
    Context& c = s->ctx;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        Query* q = *it;
        u32 first = 0;
        if (s->free_slots.empty()) break;
        if (!find_pages(s, q->npages, &first)) {
            ++it;
            continue;
        }
        const u32 slot = s->free_slots.back();
        s->free_slots.pop_back();
        q->slot = slot;
        q->first_page = first;
        for (u32 p = 0; p < q->npages; ++p) {
            s->page_used[first + p] = 1;
            c.h_pages[first + p] = slot;
        }
        const sssp_graph* g = q->g;
        c.h_desc[slot] = InstDesc{g->out_off, g->out_adj, g->in_off, g->in_adj, g->outw, g->inw,
                                  (u64)first << kPageShift, g->n, q->source};
        CK(cudaMemcpyAsync((void*)(c.P.idesc + slot), c.h_desc + slot, sizeof(InstDesc),
                           cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync((void*)(c.P.page_owner + first), c.h_pages + first,
                           sizeof(u32) * q->npages, cudaMemcpyHostToDevice, s->stream));
        k_init_records_multi<<<c.grid, kThreads, 0, s->stream>>>(c.P, c.nrec, first, q->npages);
        CK(cudaGetLastError());
        CK(launch_start(true, false, c.P, slot, 1, 0, s->stream));
        q->state = kInFlight;
        s->slot_query[slot] = q;
        s->inflight++;
        it = s->pending.erase(it);
    }
    return SSSP_OK;
}

int retire(sssp_server* s) {
    Context& c = s->ctx;
    CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(c.h_ivar, c.P.ivar, sizeof(InstVar) * c.nslots, cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (c.h_ctl->error & 4u) return SSSP_E_DEVICE_TIMEOUT;
    if (c.h_ctl->error) return SSSP_E_INTERNAL;
    if (c.h_ctl->status == kErrRounds) return SSSP_E_ROUND_LIMIT;
    s->round_host = c.h_ctl->round;
    bool any = false;
    for (u32 slot = 0; slot < c.nslots; ++slot) {
        Query* q = s->slot_query[slot];
        if (!q || c.h_ivar[slot].status != kDone) continue;
        const u64 base = (u64)q->first_page << kPageShift;
        k_finalize<<<c.grid, kThreads, 0, s->stream>>>(c.P.rec, nullptr, c.P.fround, base, q->g->n,
                                                       c.P.vbits,
                                                       c.P.ivar + slot, c.stage + base, nullptr,
                                                       nullptr, nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(q->out, c.stage + base, sizeof(u64) * q->g->n, cudaMemcpyDeviceToHost,
                           s->stream));
        q->rounds = c.h_ivar[slot].rounds;
        any = true;
    }
    if (any) CK(cudaStreamSynchronize(s->stream));
    for (u32 slot = 0; slot < c.nslots; ++slot) {
        Query* q = s->slot_query[slot];
        if (!q || c.h_ivar[slot].status != kDone) continue;
        q->state = kComplete;
        for (u32 p = 0; p < q->npages; ++p) s->page_used[q->first_page + p] = 0;
        s->slot_query[slot] = nullptr;
        s->free_slots.push_back(slot);
        s->inflight--;
    }
    return SSSP_OK;
}

int step(sssp_server* s) {
    RC(admit(s));
    if (s->inflight == 0) return SSSP_OK;
    Context& c = s->ctx;
    const u32 k = s->cfg.rounds_per_step;
    *s->h_stop = s->round_host + k - 1;
    CK(cudaMemcpyAsync(&c.P.ctl->stop_round, s->h_stop, sizeof(u32), cudaMemcpyHostToDevice,
                       s->stream));
    RC(run_loop(c, SSSP_LOOP_PERSISTENT, s->stream));
    return retire(s);
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
    int dev = c.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SSSP_E_CUDA;
    }
    sssp_server* s = new (std::nothrow) sssp_server();
    if (!s) return SSSP_E_NOMEM;
    s->device = dev;
    s->cfg = c;
    int rc;
    {
        DeviceGuard dg(dev);
        rc = open_impl(s);
        if (rc != SSSP_OK) {
            s->ctx.destroy();
            if (s->h_stop) cudaFreeHost(s->h_stop);
            if (s->stream) cudaStreamDestroy(s->stream);
        }
    }
    if (rc != SSSP_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return SSSP_OK;
}

int sssp_serve_submit(sssp_server* s, sssp_handle g, uint32_t source, uint64_t* dist_out,
                      uint64_t* ticket) {
    if (!s || !g || !dist_out || !ticket) return SSSP_E_INVAL;
    if (source >= g->n) return SSSP_E_SOURCE_RANGE;
    if (g->device != s->device || g->opt.hub_degree != s->ctx.P.hub ||
        g->opt.chunk_edges != s->ctx.P.chunk || g->opt.rule != s->ctx.P.rule)
        return SSSP_E_INVAL;
    if (g->vbits > kServeVbits ||
        (g->wmax && (unsigned __int128)g->n * g->wmax >= (unsigned __int128)s->ctx.P.dinf))
        return SSSP_E_OVERFLOW;
    const u32 np = (u32)(((u64)g->n + (1u << kPageShift) - 1) >> kPageShift);
    if (np > s->ctx.npages) return SSSP_E_BUSY;
    Query* q = new (std::nothrow) Query();
    if (!q) return SSSP_E_NOMEM;
    q->ticket = ++s->next_ticket;
    q->g = g;
    q->source = source;
    q->out = reinterpret_cast<u64*>(dist_out);
    q->npages = np;
    s->pending.push_back(q);
    s->tickets[q->ticket] = q;
    *ticket = q->ticket;
    return SSSP_OK;
}

int sssp_serve_poll(sssp_server* s, uint64_t ticket, uint32_t* rounds_out) {
    if (!s) return SSSP_E_INVAL;
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOT_FOUND;
    Query* q = it->second;
    if (q->state != kComplete) {
        DeviceGuard dg(s->device);
        RC(step(s));
    }
    if (q->state != kComplete) return SSSP_PENDING;
    if (rounds_out) *rounds_out = q->rounds;
    s->tickets.erase(it);
    delete q;
    return SSSP_OK;
}

int sssp_serve_drain(sssp_server* s) {
    if (!s) return SSSP_E_INVAL;
    DeviceGuard dg(s->device);
    while (!s->pending.empty() || s->inflight > 0) {
        const u32 before = s->inflight + (u32)s->pending.size();
        RC(step(s));
        if (s->inflight == 0 && !s->pending.empty() &&
            s->inflight + (u32)s->pending.size() == before)
            return SSSP_E_BUSY;   // nothing can be admitted
    }
    return SSSP_OK;
}

void sssp_serve_close(sssp_server* s) {
    if (!s) return;
    {
        DeviceGuard dg(s->device);
        if (s->stream) cudaStreamSynchronize(s->stream);
        s->ctx.destroy();
        if (s->h_stop) cudaFreeHost(s->h_stop);
        if (s->stream) cudaStreamDestroy(s->stream);
    }
    for (auto& kv : s->tickets) delete kv.second;
    delete s;
}

}  // extern "C"
