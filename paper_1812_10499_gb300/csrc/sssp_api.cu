// sssp_api.cu -- host engine and C ABI (include/sssp.h) of the GB300
// bound-based SSSP library (Garg, arXiv 1812.10499).
//
// A handle owns the device-resident graph (CSR out-edges, CSC in-edges,
// outWeight) and a single-query solve context.  Solving launches three setup
// kernels, the round loop, and one output kernel; the loop is a CUDA graph
// with a device-side while node whose condition the last CTA of each round
// sets, so a solve costs one graph launch whatever its round count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sssp_engine.h"

using namespace sssp;
using namespace sssp::engine;

namespace sssp {
namespace engine {

// Grid of a round kernel: SMs x CTAs per SM (the option, else occupancy).
int occupancy_grid(int device, const sssp_options& o, bool cupdate) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per = (int)o.ctas_per_sm;
    if (per <= 0)
        per = std::max(1, cupdate ? cupdate_blocks_per_sm(kThreads) : round_blocks_per_sm(kThreads));
    return std::max(1, sms) * per;
}

int scan_excl(u64* in, u64 cnt, u64* out, u64* tmp, cudaStream_t st) {
    const u32 tiles = (u32)((cnt + kScanTile - 1) / kScanTile);
    k_scan_tiles<<<tiles, kThreads, 0, st>>>(in, cnt, tmp);
    k_scan_sums<<<1, kThreads, 0, st>>>(tmp, tiles);
    k_scan_apply<<<tiles, kThreads, 0, st>>>(in, cnt, tmp, out);
    CK(cudaGetLastError());
    return SSSP_OK;
}

// L2 residency of the per-vertex records, the target of the lower-bound
// gathers and the relaxation's atomics: when the records fit the device's
// persisting L2 capacity, an access-policy window over them marks all their
// lines persisting, so the streamed adjacency and the relaxation filter words
// do not evict them.  (Measured on R-MAT scale 22: a window larger than the
// capacity, whose excess lines then stream, is slower than none, and so are
// the filter words without the window: the relaxation then no longer keeps
// the records warm for the lower-bound gathers.)  SSSP_L2_PERSIST=0 turns
// the window, and with it the filter words, off.
bool records_fit_l2(size_t bytes, int device) {
    if (const char* v = getenv("SSSP_L2_PERSIST"))
        if (strtoul(v, nullptr, 10) == 0) return false;
    int max_win = 0, max_persist = 0;
    if (cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, device) !=
            cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return bytes > 0 && bytes <= (size_t)max_win && bytes <= (size_t)max_persist;
}

// Sets the window over the context's records when they fit (the context's
// persisting L2 limit is raised to their size); otherwise clears it.
void set_l2_window(Context& c, int device) {
    c.l2win = cudaAccessPolicyWindow{};
    void* base = c.narrow ? (void*)c.P.recn : (void*)c.P.rec;
    const size_t bytes = c.nrec * (c.narrow ? sizeof(VRecN) : sizeof(VRec));
    if (!base || !records_fit_l2(bytes, device)) return;
    size_t limit = 0;
    if (cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (limit < bytes &&
        (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess ||
         cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize) != cudaSuccess)) {
        (void)cudaGetLastError();
        return;
    }
    if (limit < bytes) return;
    c.l2win.base_ptr = base;
    c.l2win.num_bytes = bytes;
    c.l2win.hitRatio = 1.0f;
    c.l2win.hitProp = cudaAccessPropertyPersisting;
    c.l2win.missProp = cudaAccessPropertyNormal;
}

// Builds the device-side while loop: body = relax -> cupdate -> tail (the
// cluster kernel that runs the following rounds while they are small).
int build_loop(Context& c) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        CK(e);
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        CK(e);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    RoundParams P = c.P;
    P.cond = h;
    void* args[] = {&P};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(relax_fn(c.multi, c.narrow, c.P.pcnt != nullptr));
    kp.gridDim = dim3(c.grid);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = (unsigned)relax_smem_bytes(c.narrow);
    kp.kernelParams = args;
    cudaGraphNode_t n1, n2;
    e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp);
    if (e == cudaSuccess) {
        kp.func = const_cast<void*>(cupdate_fn(c.multi, c.narrow, c.P.pcnt != nullptr));
        kp.gridDim = dim3(c.grid_cup);
        kp.sharedMemBytes = (unsigned)cupdate_smem_bytes(c.narrow);
        e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp);
    }
    if (e == cudaSuccess && c.tail_ctas) {
        cudaGraphNode_t n3;
        kp.func = const_cast<void*>(tail_fn(c.multi, c.narrow, c.P.pcnt != nullptr));
        kp.gridDim = dim3(c.tail_ctas);
        kp.sharedMemBytes = (unsigned)solve_smem_bytes(c.narrow);
        e = cudaGraphAddKernelNode(&n3, body, &n2, 1, &kp);
        if (e == cudaSuccess) {
            cudaLaunchAttributeValue v{};
            v.clusterDim.x = c.tail_ctas;
            v.clusterDim.y = 1;
            v.clusterDim.z = 1;
            e = cudaGraphKernelNodeSetAttribute(n3, cudaLaunchAttributeClusterDimension, &v);
        }
    }
    // The records' lines persist in L2 (see set_l2_window).
    if (e == cudaSuccess && c.l2win.num_bytes) {
        cudaLaunchAttributeValue v{};
        v.accessPolicyWindow = c.l2win;
        e = cudaGraphKernelNodeSetAttribute(n1, cudaLaunchAttributeAccessPolicyWindow, &v);
        if (e == cudaSuccess)
            e = cudaGraphKernelNodeSetAttribute(n2, cudaLaunchAttributeAccessPolicyWindow, &v);
        if (e == cudaSuccess && c.tail_ctas) {
            cudaGraphNode_t nodes[3];
            size_t cnt = 3;
            e = cudaGraphGetNodes(body, nodes, &cnt);
            if (e == cudaSuccess && cnt == 3)
                e = cudaGraphKernelNodeSetAttribute(nodes[2], cudaLaunchAttributeAccessPolicyWindow,
                                                    &v);
        }
    }
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        CK(e);
    }
    c.graph = g;
    c.exec = x;
    return SSSP_OK;
}

// A profiled solve in the device loop's schedule: each iteration launches
// k_relax, k_cupdate and the cluster tail kernel from the host, with events
// around each launch, and snapshots of the control block after k_cupdate and
// after k_tail that split the work counters by the kernel that did the work.
int profile_graph_schedule(Context& c, cudaStream_t st) {
    const void* fr = relax_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
    const void* fc = cupdate_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
    const void* ft = tail_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
    const size_t smr = relax_smem_bytes(c.narrow), smc = cupdate_smem_bytes(c.narrow);
    RoundParams P = c.P;
    P.cond = 0;
    void* args[] = {&P};
    while (c.ev.size() < 5) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c.ev.push_back(e);
    }
    if (!c.h_snap) CK(cudaHostAlloc((void**)&c.h_snap, 2 * sizeof(Ctl), cudaHostAllocDefault));
    // Launch attributes as in the device loop: the records' L2 window on
    // every kernel, the cluster shape on the tail kernel.
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeAccessPolicyWindow;
    at[0].val.accessPolicyWindow = c.l2win;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = c.tail_ctas;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    const unsigned nwin = c.l2win.num_bytes ? 1u : 0u;
    cudaLaunchConfig_t rcfg = {}, ccfg = {}, tcfg = {};
    rcfg.gridDim = dim3(c.grid);
    rcfg.blockDim = dim3(kThreads);
    rcfg.dynamicSmemBytes = smr;
    rcfg.stream = st;
    rcfg.attrs = at;
    rcfg.numAttrs = nwin;
    ccfg = rcfg;
    ccfg.gridDim = dim3(c.grid_cup);
    ccfg.dynamicSmemBytes = smc;
    tcfg.gridDim = dim3(c.tail_ctas);
    tcfg.blockDim = dim3(kThreads);
    tcfg.dynamicSmemBytes = solve_smem_bytes(c.narrow);
    tcfg.stream = st;
    tcfg.attrs = at + 1 - nwin;
    tcfg.numAttrs = 1 + nwin;
    CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    Ctl prev = *c.h_ctl;
    c.prof_round_relax.clear();
    c.prof_round_cup.clear();
    c.prof_round_tail.clear();
    c.prof_round_tail_rounds.clear();
    c.prof_round_ctr.clear();
    while (prev.status == kRunning && prev.round <= prev.stop_round) {
        CK(cudaEventRecord(c.ev[0], st));
        CK(cudaLaunchKernelExC(&rcfg, fr, args));
        CK(cudaEventRecord(c.ev[1], st));
        CK(cudaLaunchKernelExC(&ccfg, fc, args));
        CK(cudaEventRecord(c.ev[2], st));
        CK(cudaMemcpyAsync(&c.h_snap[0], c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(c.ev[3], st));
        CK(cudaLaunchKernelExC(&tcfg, ft, args));
        CK(cudaEventRecord(c.ev[4], st));
        CK(cudaMemcpyAsync(&c.h_snap[1], c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float a = 0, b = 0, t = 0;
        CK(cudaEventElapsedTime(&a, c.ev[0], c.ev[1]));
        CK(cudaEventElapsedTime(&b, c.ev[1], c.ev[2]));
        CK(cudaEventElapsedTime(&t, c.ev[3], c.ev[4]));
        const Ctl& A = c.h_snap[0];
        const Ctl& B = c.h_snap[1];
        for (int i = 0; i < 4; ++i) {
            c.prof_grid_ctr[i] += A.stats[i] - prev.stats[i];
            c.prof_tail_ctr[i] += B.stats[i] - A.stats[i];
            c.prof_round_ctr.push_back(A.stats[i] - prev.stats[i]);
        }
        const u32 tr = B.round - A.round;
        c.prof_relax_ms += a;
        c.prof_cup_ms += b;
        c.prof_tail_ms += t;
        c.prof_relax_n++;
        c.prof_cup_n++;
        c.prof_tail_n++;
        c.prof_tail_rounds += tr;
        c.prof_round_relax.push_back(a);
        c.prof_round_cup.push_back(b);
        c.prof_round_tail.push_back(t);
        c.prof_round_tail_rounds.push_back(tr);
        prev = B;
    }
    *c.h_ctl = prev;
    return SSSP_OK;
}

// Runs rounds until the device loop stops (all queries done, stop round hit,
// or an error).
int run_loop(Context& c, u32 loop_mode, cudaStream_t st) {
    // Round kernels per loop iteration (for the launch count of a solve).
    const bool graph = loop_mode == SSSP_LOOP_GRAPH && !c.prof;
    c.last_loop = graph ? SSSP_LOOP_GRAPH : (loop_mode == SSSP_LOOP_PERSISTENT ? loop_mode
                                                                               : SSSP_LOOP_HOST);
    // Profiling in the device loop's schedule launches its three kernels.
    const bool prof_graph = c.prof && loop_mode == SSSP_LOOP_GRAPH && c.tail_ctas;
    if (prof_graph) c.last_loop = SSSP_LOOP_GRAPH;
    c.launches_per_iter = c.last_loop == SSSP_LOOP_PERSISTENT
                              ? 0
                              : ((graph || prof_graph) && c.tail_ctas ? 3 : 2);
    if (prof_graph) return profile_graph_schedule(c, st);
    if (loop_mode == SSSP_LOOP_PERSISTENT) {
        RoundParams P = c.P;
        P.cond = 0;
        if (c.prof) {
            // Device trace: globaltimer at launch and at the end of every phase.
            if (!c.trace) {
                c.trace_cap = 2 * 65536 + 1;
                RC(c.pool.get(&c.trace, c.trace_cap));
            }
            CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            P.trace = c.trace;
            P.trace_cap = c.trace_cap;
            P.trace_base = c.h_ctl->round;
            for (int i = 0; i < 4; ++i) c.prof_grid_ctr[i] -= c.h_ctl->stats[i];
        }
        void* args[] = {&P};
        const void* fs = solve_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
        CK(cudaLaunchCooperativeKernel(fs, dim3(c.grid_solve), dim3(kThreads), args,
                                       solve_smem_bytes(c.narrow), st));
        if (c.prof) {
            CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int i = 0; i < 4; ++i) c.prof_grid_ctr[i] += c.h_ctl->stats[i];
            const u32 rounds = std::min<u32>(c.h_ctl->round - P.trace_base, (c.trace_cap - 1) / 2);
            std::vector<u64> t(2 * rounds + 1);
            CK(cudaMemcpy(t.data(), c.trace, sizeof(u64) * t.size(), cudaMemcpyDeviceToHost));
            c.prof_round_relax.clear();
            c.prof_round_cup.clear();
            c.prof_round_tail.clear();
            c.prof_round_tail_rounds.clear();
            c.prof_round_ctr.clear();
            for (u32 i = 0; i < rounds; ++i) {
                const float a = (float)((t[2 * i + 1] - t[2 * i]) * 1e-6);
                const float b = (float)((t[2 * i + 2] - t[2 * i + 1]) * 1e-6);
                c.prof_round_relax.push_back(a);
                c.prof_round_cup.push_back(b);
                c.prof_round_tail.push_back(0.f);
                c.prof_round_tail_rounds.push_back(0);
                c.prof_round_ctr.insert(c.prof_round_ctr.end(), 4, 0ull);
                c.prof_relax_ms += a;
                c.prof_cup_ms += b;
            }
            c.prof_relax_n += rounds;
            c.prof_cup_n += rounds;
        }
        return SSSP_OK;
    }
    if (loop_mode == SSSP_LOOP_GRAPH && !c.prof) {
        if (!c.exec) RC(build_loop(c));
        CK(cudaGraphLaunch(c.exec, st));
        return SSSP_OK;
    }
    // Host-launched rounds, 16 per group, then a status check.  With
    // profiling, events bracket every launch: ev[3i] | relax | ev[3i+1] |
    // cupdate | ev[3i+2].
    constexpr int kGroup = 16;
    const void* fr = relax_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
    const void* fc = cupdate_fn(c.multi, c.narrow, c.P.pcnt != nullptr);
    const size_t smr = relax_smem_bytes(c.narrow), smc = cupdate_smem_bytes(c.narrow);
    RoundParams P = c.P;
    P.cond = 0;
    void* args[] = {&P};
    if (c.prof && c.ev.empty()) {
        c.ev.resize(3 * kGroup);
        for (auto& e : c.ev) CK(cudaEventCreate(&e));
    }
    CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    u32 round_before = c.h_ctl->round;
    if (c.prof) {
        c.prof_round_relax.clear();
        c.prof_round_cup.clear();
        c.prof_round_tail.clear();
        c.prof_round_tail_rounds.clear();
        c.prof_round_ctr.clear();
    }
    const Ctl start_ctl = *c.h_ctl;
    for (;;) {
        for (int i = 0; i < kGroup; ++i) {
            if (c.prof) CK(cudaEventRecord(c.ev[3 * i], st));
            CK(cudaLaunchKernel(fr, dim3(c.grid), dim3(kThreads), args, smr, st));
            if (c.prof) CK(cudaEventRecord(c.ev[3 * i + 1], st));
            CK(cudaLaunchKernel(fc, dim3(c.grid_cup), dim3(kThreads), args, smc, st));
            if (c.prof) CK(cudaEventRecord(c.ev[3 * i + 2], st));
        }
        CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (c.prof) {
            const u32 ran = std::min<u32>(kGroup, c.h_ctl->round - round_before);
            for (u32 i = 0; i < ran; ++i) {
                float a = 0, b = 0;
                CK(cudaEventElapsedTime(&a, c.ev[3 * i], c.ev[3 * i + 1]));
                CK(cudaEventElapsedTime(&b, c.ev[3 * i + 1], c.ev[3 * i + 2]));
                c.prof_relax_ms += a;
                c.prof_cup_ms += b;
                c.prof_round_relax.push_back(a);
                c.prof_round_cup.push_back(b);
                c.prof_round_tail.push_back(0.f);
                c.prof_round_tail_rounds.push_back(0);
                c.prof_round_ctr.insert(c.prof_round_ctr.end(), 4, 0ull);
            }
            c.prof_relax_n += ran;
            c.prof_cup_n += ran;
        }
        round_before = c.h_ctl->round;
        if (c.h_ctl->status != kRunning || c.h_ctl->round > c.h_ctl->stop_round) break;
    }
    if (c.prof)
        for (int i = 0; i < 4; ++i) c.prof_grid_ctr[i] += c.h_ctl->stats[i] - start_ctl.stats[i];
    return SSSP_OK;
}

int alloc_lists(Context& c, u64 capS, u64 capH, u64 capC) {
    capH = std::max<u64>(capH, 1);
    capC = std::min<u64>(std::max<u64>(capC, 1), 0xFFFFFFFFull);
    for (int i = 0; i < 2; ++i) {
        RC(c.pool.get(&c.P.L.FS[i], capS));
        RC(c.pool.get(&c.P.L.AS[i], capS));
        RC(c.pool.get(&c.P.L.FH[i], capH));
        RC(c.pool.get(&c.P.L.AH[i], capH));
        RC(c.pool.get(&c.P.L.FC[i], capC));
        RC(c.pool.get(&c.P.L.AC[i], capC));
    }
    c.P.L.capC = (u32)capC;
    RC(c.pool.get(&c.P.L.hubmin, capH));
    RC(c.pool.get(&c.P.L.hubcnt, capH));
    c.P.L.capS = (u32)std::min<u64>(capS, 0xFFFFFFFFull);
    c.P.L.capH = (u32)std::min<u64>(capH, 0xFFFFFFFFull);
    c.capH = c.P.L.capH;
    return SSSP_OK;
}

// The control block and, when they fit beside it, the per-query scalars go in
// one of kHotSlots candidate slots, kHotStride bytes apart, of one allocation:
// the slot that the tail kernel's cluster reaches with the shortest chain of
// atomics (k_place_probe).  Which slot that is depends on where the
// allocation lands in physical memory, and the latency-bound rounds -- each
// a chain of waits on these words -- differ by up to 14% between a good slot
// and a bad one.  SSSP_HOT_SLOT=<i> forces slot i (for measurements).
int alloc_hot(Context& c, u32 nivar, cudaStream_t st) {
    constexpr u32 kHotSlots = 16, kHotStride = 4096;
    const size_t bytes = (size_t)kHotSlots * kHotStride;
    unsigned char* hot = nullptr;
    RC(c.pool.get(&hot, bytes + 256));
    auto* cyc = reinterpret_cast<unsigned long long*>(hot + bytes);
    CK(launch_place_probe(reinterpret_cast<u32*>(hot), kHotSlots, kHotStride / 4, cyc,
                          c.tail_ctas, solve_smem_bytes(c.narrow), st));
    unsigned long long h[kHotSlots];
    CK(cudaMemcpyAsync(h, cyc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(hot, 0, bytes + 256, st));
    CK(cudaStreamSynchronize(st));
    int best = 0;
    for (u32 i = 1; i < kHotSlots; ++i)
        if (h[i] < h[best]) best = (int)i;
    if (const char* e = getenv("SSSP_HOT_SLOT")) {
        const int f = atoi(e);
        if (f >= 0 && f < (int)kHotSlots) best = f;
    }
    c.hot_slot = best;
    unsigned char* slot = hot + (size_t)best * kHotStride;
    c.P.ctl = reinterpret_cast<Ctl*>(slot);
    const size_t ivoff = (sizeof(Ctl) + 255) & ~(size_t)255;
    if (ivoff + (size_t)nivar * sizeof(InstVar) <= kHotStride)
        c.P.ivar = reinterpret_cast<InstVar*>(slot + ivoff);
    else
        RC(c.pool.get(&c.P.ivar, nivar));
    return SSSP_OK;
}

int alloc_pinned(Context& c, u32 slots) {
    CK(cudaHostAlloc((void**)&c.h_ctl, sizeof(Ctl), cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&c.h_ivar, sizeof(InstVar) * slots, cudaHostAllocDefault));
    return SSSP_OK;
}

// Hub chunks a list can hold: at most m / chunk plus one partial chunk per
// hub, in either direction.
u64 hub_chunks(const sssp_graph* h) {
    return h->m / h->opt.chunk_edges + std::max(h->hubs_in, h->hubs_out) + 1;
}

int init_single_context(sssp_graph* h) {
    Context& c = h->single;
    c.pool.al = Allocator{h->opt.alloc, h->opt.free, h->opt.alloc_ctx};
    c.multi = false;
    c.nrec = h->n;
    c.nslots = 1;
    c.grid = h->grid;
    c.grid_cup = h->grid_cup;
    c.grid_solve = h->grid_solve;
    c.tail_ctas = h->tail_ctas;
    RoundParams& P = c.P;
    P.tail_items = h->tail_items;
    P.g.out_off = h->out_off;
    P.g.out_adj = h->out_adj;
    P.g.in_off = h->in_off;
    P.g.in_adj = h->in_adj;
    P.g.outw = h->narrow ? h->outw_pack : h->outw;
    P.g.inw = h->inw;
    P.g.base = 0;
    P.g.n = h->n;
    P.g.source = 0;
    c.narrow = h->narrow;
    if (c.narrow) {
        // Compact records, then (label-setting rounds, records held in L2)
        // the relaxation filter words right after them.
        const bool filt = (h->opt.rule & (SSSP_RULE_LABEL_CORRECTING | SSSP_RULE_WINDOWED)) == 0 &&
                          records_fit_l2((size_t)h->n * sizeof(VRecN), h->device);
        unsigned char* buf = nullptr;
        RC(c.pool.get(&buf, (size_t)h->n * (sizeof(VRecN) + (filt ? sizeof(uint2) : 0))));
        P.recn = reinterpret_cast<VRecN*>(buf);
        P.gf = filt ? reinterpret_cast<uint2*>(buf + (size_t)h->n * sizeof(VRecN)) : nullptr;
    } else {
        RC(c.pool.get(&P.rec, h->n));
    }
    RC(c.pool.get(&P.fround, h->n));
    RC(alloc_hot(c, 1, h->stream));
    RC(c.pool.get(&c.stage, h->n));
    RC(alloc_lists(c, h->n, std::max(h->hubs_in, h->hubs_out), hub_chunks(h)));
    P.dinf = h->dinf;
    P.vbits = h->vbits;
    P.hub = h->opt.hub_degree;
    P.chunk = h->opt.chunk_edges;
    P.rule = h->opt.rule & SSSP_RULE_MIND;
    P.lc = (h->opt.rule & SSSP_RULE_LABEL_CORRECTING) ? 1u : 0u;
    P.cheap = (h->opt.rule & SSSP_RULE_CHEAP_FIRST) ? 1u : 0u;
    P.win = (h->opt.rule & SSSP_RULE_WINDOWED) ? 1u : 0u;
    P.delta = h->opt.delta;
    if (h->opt.rule & SSSP_RULE_PRED_COUNT) {
        CK(pred_kernels_init());
        RC(c.pool.get(&P.pcnt, h->n));
    }
    if (P.lc || P.win) {
        RC(c.pool.get(&P.snap, h->n));
        RC(c.pool.get(&P.chg, h->n));
        RC(c.pool.get(&P.L.FX[0], h->n));
        RC(c.pool.get(&P.L.FX[1], h->n));
    }
    P.page_shift = kPageShift;
    set_l2_window(c, h->device);
    RC(alloc_pinned(c, 1));
    CK(cudaMemsetAsync(P.L.hubmin, 0xFF, sizeof(u64) * c.capH, h->stream));
    CK(cudaMemsetAsync(P.L.hubcnt, 0, sizeof(u32) * c.capH, h->stream));
    return SSSP_OK;
}

int validate_csr(u32 n, u64 m, const u64* off, const u32* idx, const u32* w, u32* wmax) {
    if (!off || (m && (!idx || !w))) return SSSP_E_INVAL;
    if (off[0] != 0 || off[n] != m) return SSSP_E_INVAL;
    u32 mx = 0;
    for (u32 u = 0; u < n; ++u)
        if (off[u + 1] < off[u]) return SSSP_E_INVAL;
    for (u64 k = 0; k < m; ++k) {
        if (idx[k] >= n) return SSSP_E_INVAL;
        if (w[k] == 0) return SSSP_E_ZERO_WEIGHT;
        mx = std::max(mx, w[k]);
    }
    *wmax = mx;
    return SSSP_OK;
}

// Copies a CSR without its self-loops (Sec. II: the graph is loop-free).
// `src_of_row` is true for CSR (row = source), false for CSC (row = target);
// the loop test is the same either way.
void strip_loops(u32 n, const u64* off, const u32* idx, const u32* w, std::vector<u64>& o2,
                 std::vector<u32>& i2, std::vector<u32>& w2) {
    o2.assign((size_t)n + 1, 0);
    i2.clear();
    w2.clear();
    i2.reserve(off[n]);
    w2.reserve(off[n]);
    for (u32 u = 0; u < n; ++u) {
        o2[u] = i2.size();
        for (u64 k = off[u]; k < off[u + 1]; ++k) {
            if (idx[k] == u) continue;
            i2.push_back(idx[k]);
            w2.push_back(w[k]);
        }
    }
    o2[n] = i2.size();
}

bool has_loop(u32 n, const u64* off, const u32* idx) {
    for (u32 u = 0; u < n; ++u)
        for (u64 k = off[u]; k < off[u + 1]; ++k)
            if (idx[k] == u) return true;
    return false;
}

int upload_adj(sssp_graph* h, const u32* idx, const u32* w, u64 m, uint2* adj) {
    if (m == 0) return SSSP_OK;
    Pool tmp;
    tmp.al = h->gpool.al;
    u32 *d_i = nullptr, *d_w = nullptr;
    int rc = tmp.get(&d_i, m);
    if (rc == SSSP_OK) rc = tmp.get(&d_w, m);
    if (rc == SSSP_OK) {
        cudaError_t e = cudaMemcpyAsync(d_i, idx, sizeof(u32) * m, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_w, w, sizeof(u32) * m, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) {
            k_interleave<<<h->grid, kThreads, 0, h->stream>>>(d_i, d_w, m, adj);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            rc = SSSP_E_CUDA;
        }
    }
    tmp.release();
    return rc;
}

int create_impl(sssp_graph* h, u32 n, u64 m, const u64* row_ptr, const u32* col, const u32* w,
                const u64* col_ptr, const u32* row, const u32* w_in) {
    u32 wmax = 0;
    RC(validate_csr(n, m, row_ptr, col, w, &wmax));
    const bool csc_given = col_ptr || row || w_in;
    if (csc_given) {
        if (!(col_ptr && (m == 0 || (row && w_in)))) return SSSP_E_INVAL;
        u32 wmax2 = 0;
        RC(validate_csr(n, m, col_ptr, row, w_in, &wmax2));
        if (wmax2 != wmax) return SSSP_E_INVAL;
    }
    h->vbits = std::max<u32>(1, bits_for((u64)n - 1));
    h->dinf = (~0ull) >> h->vbits;
    // Every finite quantity of a round (D, C, lb + w, D + outWeight) stays
    // below n * wmax; it must stay below the infinity of the packed word.
    if (wmax && (unsigned __int128)n * wmax >= (unsigned __int128)h->dinf) return SSSP_E_OVERFLOW;
    h->wmax = wmax;
    // Compact records hold 31-bit lower bounds: every finite distance
    // (at most (n - 1) * wmax) must stay below 2^31 - 1.
    const bool fits = (unsigned __int128)n * wmax < kNarrowLimit;
    if (h->opt.layout == SSSP_LAYOUT_COMPACT && !fits) return SSSP_E_OVERFLOW;
    h->narrow = fits && h->opt.layout != SSSP_LAYOUT_WIDE;
    if (h->narrow) {
        // The compact kernels keep the distance in the upper half of the
        // packed D word.
        h->vbits = 32;
        h->dinf = (~0ull) >> 32;
    }

    std::vector<u64> o2, c2;
    std::vector<u32> i2, w2, r2, wi2;
    if (has_loop(n, row_ptr, col)) {
        strip_loops(n, row_ptr, col, w, o2, i2, w2);
        row_ptr = o2.data();
        col = i2.data();
        w = w2.data();
        m = o2[n];
        if (csc_given) {
            strip_loops(n, col_ptr, row, w_in, c2, r2, wi2);
            col_ptr = c2.data();
            row = r2.data();
            w_in = wi2.data();
            if (c2[n] != m) return SSSP_E_INVAL;
        }
    }
    h->n = n;
    h->m = m;

    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->grid = occupancy_grid(h->device, h->opt);
    h->grid_cup = occupancy_grid(h->device, h->opt, true);
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        h->grid_solve = std::max(1, sms) * std::max(1, solve_blocks_per_sm(kThreads));
        h->tail_items = kDefaultTailItems;
    }
    Pool& gp = h->gpool;
    RC(gp.get(&h->out_off, (size_t)n + 1));
    RC(gp.get(&h->in_off, (size_t)n + 1));
    RC(gp.get(&h->out_adj, std::max<u64>(m, 1)));
    RC(gp.get(&h->in_adj, std::max<u64>(m, 1)));
    RC(gp.get(&h->outw, n));
    CK(cudaMemcpyAsync(h->out_off, row_ptr, sizeof(u64) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                       h->stream));
    RC(upload_adj(h, col, w, m, h->out_adj));
    if (csc_given) {
        CK(cudaMemcpyAsync(h->in_off, col_ptr, sizeof(u64) * ((size_t)n + 1),
                           cudaMemcpyHostToDevice, h->stream));
        RC(upload_adj(h, row, w_in, m, h->in_adj));
    } else {
        // K0: transpose on the device (histogram, exclusive scan, scatter).
        Pool tmp;
        tmp.al = gp.al;
        u64 *cnt = nullptr, *cursor = nullptr, *sums = nullptr;
        const u64 cntn = (u64)n + 1;
        int rc = tmp.get(&cnt, cntn);
        if (rc == SSSP_OK) rc = tmp.get(&cursor, cntn);
        if (rc == SSSP_OK) rc = tmp.get(&sums, (cntn + kScanTile - 1) / kScanTile + 1);
        cudaError_t e = cudaSuccess;
        if (rc == SSSP_OK) {
            e = cudaMemsetAsync(cnt, 0, sizeof(u64) * cntn, h->stream);
            if (e == cudaSuccess && m) {
                k_count_in<<<h->grid, kThreads, 0, h->stream>>>(h->out_adj, m, cnt);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) rc = scan_excl(cnt, cntn, h->in_off, sums, h->stream);
            if (rc == SSSP_OK && e == cudaSuccess)
                e = cudaMemcpyAsync(cursor, h->in_off, sizeof(u64) * cntn, cudaMemcpyDeviceToDevice,
                                    h->stream);
            if (rc == SSSP_OK && e == cudaSuccess && m) {
                k_scatter_in<<<h->grid, kThreads, 0, h->stream>>>(h->out_off, h->out_adj, n, cursor,
                                                                  h->in_adj);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        }
        tmp.release();
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return SSSP_E_CUDA;
        }
        RC(rc);
    }
    k_outw<<<h->grid, kThreads, 0, h->stream>>>(h->out_off, h->out_adj, n, h->outw);
    CK(cudaGetLastError());
    RC(gp.get(&h->inw, n));   // inWeight: the same reduction over the in-edges
    k_outw<<<h->grid, kThreads, 0, h->stream>>>(h->in_off, h->in_adj, n, h->inw);
    CK(cudaGetLastError());
    // The graph's degree statistics (its class in the tuning cache), then
    // the state that depends on the tuning.
    RC(count_hubs(h, h->opt.hub_degree, &h->hubs_out, &h->hubs_in, &h->max_out, &h->max_in));
    resolve_tuning(h);
    RC(apply_tuning(h));
    return SSSP_OK;
}

// Hub counts by direction for hub degree `hub` (list capacities), and the
// largest out- and in-degree (nullable outputs).
int count_hubs(sssp_graph* h, u32 hub, u32* hubs_out, u32* hubs_in, u32* max_out, u32* max_in) {
    Pool tmp;
    tmp.al = h->gpool.al;
    u32* cnt = nullptr;
    RC(tmp.get(&cnt, 4));
    u32 hc[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(hc), h->stream);
    if (e == cudaSuccess) {
        k_count_hubs<<<h->grid, kThreads, 0, h->stream>>>(h->out_off, h->in_off, h->n, hub, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    tmp.release();
    CK(e);
    *hubs_out = hc[0];
    *hubs_in = hc[1];
    if (max_out) *max_out = hc[2];
    if (max_in) *max_in = hc[3];
    return SSSP_OK;
}

// State that depends on the tuning (hub degree, chunk size, CTAs per SM,
// cluster-tail thresholds): the round kernels' grids, the compact layout's
// in-hub flags, the hub counts, and the solve contexts (rebuilt).
int apply_tuning(sssp_graph* h) {
    const u32 n = h->n;
    CK(cudaStreamSynchronize(h->stream));
    h->grid = occupancy_grid(h->device, h->opt);
    h->grid_cup = occupancy_grid(h->device, h->opt, true);
    h->tail_ctas = h->tail_items ? tail_cluster_ctas() : 0;
    if (h->narrow) {
        if (!h->outw_pack) RC(h->gpool.get(&h->outw_pack, n));
        k_pack_outw<<<h->grid, kThreads, 0, h->stream>>>(h->outw, h->in_off, n, h->opt.hub_degree,
                                                         h->outw_pack);
        CK(cudaGetLastError());
    }
    RC(count_hubs(h, h->opt.hub_degree, &h->hubs_out, &h->hubs_in, nullptr, nullptr));
    h->single.destroy();
    h->single = Context();
    if (h->batch) {
        h->batch->destroy();
        delete h->batch;
        h->batch = nullptr;
    }
    RC(init_single_context(h));
    CK(cudaStreamSynchronize(h->stream));
    return SSSP_OK;
}

void destroy_impl(sssp_graph* h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->single.destroy();
    if (h->batch) {
        h->batch->destroy();
        delete h->batch;
        h->batch = nullptr;
    }
    h->gpool.release();
    if (h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
}

// The device address of a page-locked host allocation mapped into the
// device's address space, or nullptr (pageable memory, or not mapped).
u64* mapped_device_ptr(void* host) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<u64*>(at.devicePointer);
}

int read_status(Context& c, cudaStream_t st, u32 ninst) {
    CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c.h_ivar, c.P.ivar, sizeof(InstVar) * ninst, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (c.h_ctl->error & 4u) return SSSP_E_DEVICE_TIMEOUT;
    if (c.h_ctl->error & 8u) return SSSP_E_OVERFLOW;
    if (c.h_ctl->error) return SSSP_E_INTERNAL;
    if (c.h_ctl->status == kErrRounds) return SSSP_E_ROUND_LIMIT;
    return SSSP_OK;
}

// Enqueues one single-query solve on `st` (no synchronisation).
int enqueue_single(sssp_graph* h, u32 source, u32 max_rounds, cudaStream_t st, u64* dist_dev,
                   u32* parent_dev, int* fround_dev, u64* lower_dev, u32 target) {
    Context& c = h->single;
    RoundParams P = c.P;
    P.g.source = source;
    c.P.g.source = source;
    k_init_records<<<c.grid, kThreads, 0, st>>>(P.rec, P.recn, P.fround, h->outw, h->in_off, h->n,
                                                P.chg, P.gf, h->outw_pack, P.pcnt);
    k_reset_ctl<<<1, 32, 0, st>>>(P.ctl, 1, h->n + 2);
    CK(launch_start(false, c.narrow, P, 0, 1, max_rounds, st, target));
    RC(run_loop(c, h->opt.loop_mode, st));
    k_finalize<<<c.grid, kThreads, 0, st>>>(P.rec, P.recn, P.fround, 0, h->n, h->vbits, P.ivar,
                                            dist_dev,
                                            parent_dev, fround_dev, lower_dev);
    CK(cudaGetLastError());
    return SSSP_OK;
}

// ----------------------------------------------------------- multi-query

int ensure_batch(sssp_graph* h0, u64 nrec, u32 nslots, u32 npages, u64 capH, u64 capC) {
    Context* c = h0->batch;
    if (c && c->nrec >= nrec && c->nslots >= nslots && c->npages >= npages && c->capH >= capH &&
        c->P.L.capC >= capC)
        return SSSP_OK;
    if (c) {
        c->destroy();
        delete c;
        h0->batch = nullptr;
    }
    c = new (std::nothrow) Context();
    if (!c) return SSSP_E_NOMEM;
    h0->batch = c;
    c->pool.al = Allocator{h0->opt.alloc, h0->opt.free, h0->opt.alloc_ctx};
    c->multi = true;
    c->nrec = nrec;
    c->nslots = nslots;
    c->npages = npages;
    c->grid = h0->grid;
    c->grid_cup = h0->grid_cup;
    c->grid_solve = h0->grid_solve;
    c->tail_ctas = h0->tail_ctas;
    RoundParams& P = c->P;
    P.tail_items = h0->tail_items;
    RC(c->pool.get(&c->rec_store, nrec));   // 32-byte slots; the compact layout uses half
    RC(c->pool.get(&P.fround, nrec));
    RC(alloc_hot(*c, nslots, h0->stream));
    InstDesc* idesc = nullptr;
    u32* pages = nullptr;
    RC(c->pool.get(&idesc, nslots));
    RC(c->pool.get(&pages, npages));
    P.idesc = idesc;
    P.page_owner = pages;
    RC(c->pool.get(&c->stage, nrec));
    RC(alloc_lists(*c, nrec, capH, capC));
    P.page_shift = kPageShift;
    P.hub = h0->opt.hub_degree;
    P.chunk = h0->opt.chunk_edges;
    P.rule = h0->opt.rule & SSSP_RULE_MIND;
    P.lc = (h0->opt.rule & SSSP_RULE_LABEL_CORRECTING) ? 1u : 0u;
    P.cheap = (h0->opt.rule & SSSP_RULE_CHEAP_FIRST) ? 1u : 0u;
    P.win = (h0->opt.rule & SSSP_RULE_WINDOWED) ? 1u : 0u;
    P.delta = h0->opt.delta;
    if (h0->opt.rule & SSSP_RULE_PRED_COUNT) {
        CK(pred_kernels_init());
        RC(c->pool.get(&P.pcnt, nrec));
    }
    if (P.lc || P.win) {
        RC(c->pool.get(&P.snap, nrec));
        RC(c->pool.get(&P.chg, nrec));
        RC(c->pool.get(&P.L.FX[0], nrec));
        RC(c->pool.get(&P.L.FX[1], nrec));
    }
    RC(alloc_pinned(*c, nslots));
    CK(cudaHostAlloc((void**)&c->h_desc, sizeof(InstDesc) * nslots, cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&c->h_pages, sizeof(u32) * npages, cudaHostAllocDefault));
    CK(cudaMemsetAsync(P.L.hubmin, 0xFF, sizeof(u64) * c->capH, h0->stream));
    CK(cudaMemsetAsync(P.L.hubcnt, 0, sizeof(u32) * c->capH, h0->stream));
    CK(cudaStreamSynchronize(h0->stream));
    return SSSP_OK;
}

int batch_impl(const sssp_handle* g, const u32* sources, u32 k, u64* const* dist, bool dev,
               u32* rounds_out, cudaStream_t st_user, bool use_user_stream,
               const sssp_tuning* tune) {
    if (!g || !sources || !dist || k == 0) return SSSP_E_INVAL;
    sssp_graph* h0 = g[0];
    if (!h0) return SSSP_E_INVAL;
    for (u32 i = 0; i < k; ++i) {
        if (!g[i] || !dist[i]) return SSSP_E_INVAL;
        if (g[i]->device != h0->device || g[i]->opt.rule != h0->opt.rule ||
            g[i]->opt.delta != h0->opt.delta)
            return SSSP_E_INVAL;
        if (sources[i] >= g[i]->n) return SSSP_E_SOURCE_RANGE;
    }
    // The batch's tuning: the one given (autotuner), else the cache's entry
    // for the batch's class, else the first graph's.  The graphs' own hub
    // degrees may differ from it: a graph's in-hub flags (compact layout)
    // then place some vertices in the other list, which changes no result.
    sssp_tuning bt{};
    if (tune) {
        bt = *tune;
    } else {
        char key[96];
        batch_key(g, k, key, sizeof(key));
        if (tune_cache_find(key, &bt) != SSSP_OK) {
            bt.hub_degree = h0->opt.hub_degree;
            bt.chunk_edges = h0->opt.chunk_edges;
            bt.ctas_per_sm = h0->opt.ctas_per_sm;
            bt.tail_items = h0->tail_items;
        }
    }
    u32 vbits = 1;
    bool narrow = true;
    u64 npages = 0, capH = 0, capC = 0;
    for (u32 i = 0; i < k; ++i) {
        vbits = std::max(vbits, std::max<u32>(1, bits_for((u64)g[i]->n - 1)));
        narrow = narrow && g[i]->narrow;
        npages += ((u64)g[i]->n + (1u << kPageShift) - 1) >> kPageShift;
        // Hub entries: flagged in-hubs of the graph's own hub degree, and at
        // most m / (hub + 1) vertices above the batch's hub degree.
        const u64 above = std::min<u64>(g[i]->n, g[i]->m / ((u64)bt.hub_degree + 1));
        const u64 hi = std::max<u64>(std::max(g[i]->hubs_in, g[i]->hubs_out), above) + 1;
        capH += hi;
        capC += g[i]->m / bt.chunk_edges + hi;
    }
    const u64 nrec = npages << kPageShift;
    if (nrec >= 0xFFFFFFFFull) return SSSP_E_NOMEM;   // list entries are 32-bit record ids
    if (narrow) vbits = 32;                           // compact kernels: distance in the upper half
    const u64 dinf = (~0ull) >> vbits;
    for (u32 i = 0; i < k; ++i)
        if (g[i]->wmax && (unsigned __int128)g[i]->n * g[i]->wmax >= (unsigned __int128)dinf)
            return SSSP_E_OVERFLOW;
    DeviceGuard dg(h0->device);
    std::lock_guard<std::mutex> lk(h0->mu);
    RC(ensure_batch(h0, nrec, k, (u32)npages, capH, capC));
    Context& c = *h0->batch;
    cudaStream_t st = use_user_stream ? st_user : h0->stream;
    RoundParams& P = c.P;
    sssp_options bo = h0->opt;
    bo.ctas_per_sm = bt.ctas_per_sm;
    const int grid = occupancy_grid(h0->device, bo), grid_cup = occupancy_grid(h0->device, bo, true);
    const u32 tail_ctas = bt.tail_items ? tail_cluster_ctas() : 0;
    // The loop graph bakes the params in; rebuild it when they change.
    if (c.exec && (P.vbits != vbits || c.narrow != narrow || P.hub != bt.hub_degree ||
                   P.chunk != bt.chunk_edges || P.tail_items != bt.tail_items ||
                   c.grid != grid || c.grid_cup != grid_cup || c.tail_ctas != tail_ctas)) {
        cudaGraphExecDestroy(c.exec);
        cudaGraphDestroy(c.graph);
        c.exec = nullptr;
        c.graph = nullptr;
    }
    P.hub = bt.hub_degree;
    P.chunk = bt.chunk_edges;
    P.tail_items = bt.tail_items;
    c.grid = grid;
    c.grid_cup = grid_cup;
    c.tail_ctas = tail_ctas;
    P.vbits = vbits;
    P.dinf = dinf;
    c.narrow = narrow;
    P.rec = narrow ? nullptr : c.rec_store;
    P.recn = narrow ? reinterpret_cast<VRecN*>(c.rec_store) : nullptr;
    // Compact label-setting batches whose records fit the persisting L2 keep
    // the relaxation filter words in the second half of the 32-byte record
    // slots (right after the records).
    P.gf = (narrow && !P.lc && !P.win && records_fit_l2(c.nrec * sizeof(VRecN), h0->device))
               ? reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(c.rec_store) +
                                          c.nrec * sizeof(VRecN))
               : nullptr;
    if (!c.exec) set_l2_window(c, h0->device);   // baked into the loop graph built next
    P.g = InstDesc{g[0]->out_off, g[0]->out_adj, g[0]->in_off, g[0]->in_adj,
                   narrow ? g[0]->outw_pack : g[0]->outw, g[0]->inw, 0, g[0]->n, sources[0]};
    u64 page = 0;
    for (u32 i = 0; i < k; ++i) {
        const sssp_graph* gi = g[i];
        c.h_desc[i] = InstDesc{gi->out_off, gi->out_adj, gi->in_off, gi->in_adj,
                               narrow ? gi->outw_pack : gi->outw, gi->inw, page << kPageShift,
                               gi->n, sources[i]};
        const u64 np = ((u64)gi->n + (1u << kPageShift) - 1) >> kPageShift;
        for (u64 p = 0; p < np; ++p) c.h_pages[page + p] = i;
        page += np;
    }
    CK(cudaMemcpyAsync((void*)P.idesc, c.h_desc, sizeof(InstDesc) * k, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync((void*)P.page_owner, c.h_pages, sizeof(u32) * npages, cudaMemcpyHostToDevice,
                       st));
    u32 max_n = 0;
    for (u32 i = 0; i < k; ++i) max_n = std::max(max_n, g[i]->n);
    k_init_records_multi<<<c.grid, kThreads, 0, st>>>(P, nrec, 0, (u32)npages);
    k_reset_ctl<<<1, 32, 0, st>>>(P.ctl, k, max_n + 2);
    CK(launch_start(true, c.narrow, P, 0, k, 0, st));
    RC(run_loop(c, h0->opt.loop_mode, st));
    k_finalize_multi<<<c.grid, kThreads, 0, st>>>(P, nrec, c.stage);
    CK(cudaGetLastError());
    for (u32 i = 0; i < k; ++i) {
        const u64 base = c.h_desc[i].base;
        if (dev) {
            CK(cudaMemcpyAsync(dist[i], c.stage + base, sizeof(u64) * g[i]->n,
                               cudaMemcpyDeviceToDevice, st));
        }
    }
    if (!dev) {
        if (c.h_stage_n < nrec) {
            if (c.h_stage) cudaFreeHost(c.h_stage);
            c.h_stage = nullptr;
            c.h_stage_n = 0;
            CK(cudaHostAlloc((void**)&c.h_stage, sizeof(u64) * nrec, cudaHostAllocDefault));
            c.h_stage_n = nrec;
        }
        CK(cudaMemcpyAsync(c.h_stage, c.stage, sizeof(u64) * nrec, cudaMemcpyDeviceToHost, st));
    }
    RC(read_status(c, st, k));
    for (u32 i = 0; i < k; ++i) {
        if (c.h_ivar[i].status != kDone) return SSSP_E_ROUND_LIMIT;
        if (rounds_out) rounds_out[i] = c.h_ivar[i].rounds;
        if (!dev) memcpy(dist[i], c.h_stage + c.h_desc[i].base, sizeof(u64) * g[i]->n);
    }
    return SSSP_OK;
}

}  // namespace engine
}  // namespace sssp

// ================================================================= C ABI

extern "C" {

void sssp_options_default(sssp_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->rule = SSSP_RULE_THRESHOLD;
    opt->loop_mode = SSSP_LOOP_GRAPH;
    opt->hub_degree = 0;      // the library chooses (see sssp_tuning)
    opt->chunk_edges = 0;
    opt->block_threads = kThreads;
    opt->ctas_per_sm = 0;
    opt->device = -1;
}

int sssp_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                const uint32_t* w, const uint64_t* col_ptr, const uint32_t* row,
                const uint32_t* w_in, const sssp_options* opt, sssp_handle* out) {
    if (!out || n == 0 || n == 0xFFFFFFFFu || !row_ptr) return SSSP_E_INVAL;
    sssp_options o;
    sssp_options_default(&o);
    if (opt) o = *opt;
    // Hub degree and chunk size both left 0: the library chooses the tuning.
    const bool tune_auto = o.hub_degree == 0 && o.chunk_edges == 0;
    if (o.hub_degree == 0) o.hub_degree = kDefaultHub;
    if (o.chunk_edges == 0) o.chunk_edges = kDefaultChunk;
    if (o.block_threads == 0) o.block_threads = kThreads;
    if ((o.rule & ~(SSSP_RULE_MIND | SSSP_RULE_LABEL_CORRECTING | SSSP_RULE_CHEAP_FIRST |
                    SSSP_RULE_WINDOWED | SSSP_RULE_PRED_COUNT)) != 0 ||
        ((o.rule & SSSP_RULE_LABEL_CORRECTING) && (o.rule & SSSP_RULE_WINDOWED)) ||
        ((o.rule & SSSP_RULE_PRED_COUNT) &&
         (o.rule & (SSSP_RULE_LABEL_CORRECTING | SSSP_RULE_WINDOWED))) ||
        o.loop_mode > SSSP_LOOP_PERSISTENT || o.chunk_edges % 32 != 0 ||
        o.layout > SSSP_LAYOUT_COMPACT ||
        o.hub_degree > (1u << 20) || o.chunk_edges > (1u << 20) ||
        o.block_threads != kThreads || (o.alloc == nullptr) != (o.free == nullptr))
        return SSSP_E_INVAL;
    {
        // Host-side checks first: no device is touched for a malformed graph.
        u32 wmax = 0, wmax2 = 0;
        RC(validate_csr(n, m, reinterpret_cast<const u64*>(row_ptr), col, w, &wmax));
        if (col_ptr || row || w_in) {
            if (!(col_ptr && (m == 0 || (row && w_in)))) return SSSP_E_INVAL;
            RC(validate_csr(n, m, reinterpret_cast<const u64*>(col_ptr), row, w_in, &wmax2));
            if (wmax2 != wmax) return SSSP_E_INVAL;
        }
        const u32 vb = std::max<u32>(1, bits_for((u64)n - 1));
        if (wmax && (unsigned __int128)n * wmax >= (unsigned __int128)((~0ull) >> vb))
            return SSSP_E_OVERFLOW;
        if (o.layout == SSSP_LAYOUT_COMPACT && (unsigned __int128)n * wmax >= kNarrowLimit)
            return SSSP_E_OVERFLOW;
    }
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SSSP_E_CUDA;
    }
    sssp_graph* h = new (std::nothrow) sssp_graph();
    if (!h) return SSSP_E_NOMEM;
    h->device = dev;
    h->opt = o;
    h->opt.device = dev;
    h->tune_auto = tune_auto;
    h->gpool.al = Allocator{o.alloc, o.free, o.alloc_ctx};
    int rc;
    {
        DeviceGuard dg(dev);
        rc = create_impl(h, n, m, reinterpret_cast<const u64*>(row_ptr), col, w,
                         reinterpret_cast<const u64*>(col_ptr), row, w_in);
        if (rc != SSSP_OK) destroy_impl(h);
    }
    if (rc != SSSP_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return SSSP_OK;
}

void sssp_destroy(sssp_handle h) {
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        destroy_impl(h);
    }
    delete h;
}

int sssp_host_alloc(size_t bytes, void** out) {
    if (!out || bytes == 0) return SSSP_E_INVAL;
    *out = nullptr;
    if (cudaHostAlloc(out, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();   // clear the runtime's last-error state
        *out = nullptr;
        return SSSP_E_NOMEM;
    }
    return SSSP_OK;
}

void sssp_host_free(void* p) {
    if (p) cudaFreeHost(p);
}

uint32_t sssp_num_vertices(sssp_handle h) { return h ? h->n : 0; }
uint64_t sssp_num_edges(sssp_handle h) { return h ? h->m : 0; }
int sssp_solve_to(sssp_handle h, uint32_t source, uint32_t target, uint64_t* dist_target,
                  uint32_t* rounds_out) {
    if (!h || !dist_target) return SSSP_E_INVAL;
    if (source >= h->n || target >= h->n) return SSSP_E_SOURCE_RANGE;
    DeviceGuard dg(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    Context& c = h->single;
    cudaStream_t st = h->stream;
    RC(enqueue_single(h, source, 0, st, c.stage, nullptr, nullptr, nullptr, target));
    u64 d = 0;
    CK(cudaMemcpyAsync(&d, c.stage + target, sizeof(u64), cudaMemcpyDeviceToHost, st));
    RC(read_status(c, st, 1));
    const InstVar& v = c.h_ivar[0];
    if (v.status != kDone && v.status != kStopped) return SSSP_E_ROUND_LIMIT;
    *dist_target = d;
    if (rounds_out) *rounds_out = v.rounds;
    return SSSP_OK;
}

int sssp_selftest_barrier_timeout(uint32_t timeout_ms) {
    if (timeout_ms == 0 || timeout_ms > 10000) return SSSP_E_INVAL;
    Ctl* ctl = nullptr;
    CK(cudaMalloc(&ctl, sizeof(Ctl)));
    int rc = SSSP_OK;
    cudaError_t e = cudaMemset(ctl, 0, sizeof(Ctl));
    if (e == cudaSuccess) {
        RoundParams P{};
        P.ctl = ctl;
        P.barrier_ns = (unsigned long long)timeout_ms * 1000000ull;
        u32 absent = 1;
        void* args[] = {&P, &absent};
        // Four co-resident CTAs of one warp; CTA 1 never arrives.
        e = cudaLaunchCooperativeKernel(barrier_selftest_fn(), dim3(4), dim3(32), args, 0, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    Ctl h{};
    if (e == cudaSuccess) e = cudaMemcpy(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        rc = SSSP_E_CUDA;
    } else {
        rc = (h.error & 4u) ? SSSP_E_DEVICE_TIMEOUT : SSSP_E_INTERNAL;
    }
    cudaFree(ctl);
    return rc;
}

uint32_t sssp_layout(sssp_handle h) {
    return h ? (h->narrow ? SSSP_LAYOUT_COMPACT : SSSP_LAYOUT_WIDE) : 0u;
}

int sssp_solve_ex(sssp_handle h, uint32_t source, const sssp_solve_args* args,
                  sssp_solve_info* info) {
    if (!h) return SSSP_E_INVAL;
    if (source >= h->n) return SSSP_E_SOURCE_RANGE;
    sssp_solve_args a{};
    if (args) a = *args;
    if (a.has_target && a.target >= h->n) return SSSP_E_SOURCE_RANGE;
    DeviceGuard dg(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = a.cuda_stream ? (cudaStream_t)a.cuda_stream : h->stream;
    Context& c = h->single;
    u64* const a_dist = reinterpret_cast<u64*>(a.dist);
    u64* const a_lower = reinterpret_cast<u64*>(a.lower);
    // A page-locked, device-mapped host array (sssp_host_alloc) takes the
    // distances straight from the output kernel; any other host array gets
    // them by a copy from device scratch.
    u64* const dist_mapped = (!a.dev && a_dist) ? mapped_device_ptr(a_dist) : nullptr;
    u64* dist_dev = a.dev ? a_dist : (dist_mapped ? dist_mapped : (a_dist ? c.stage : nullptr));
    // Host outputs other than dist go through device scratch in the lists
    // (free after the solve): parent / fround use FS, lower uses AS.
    u32* parent_dev = a.parent ? (a.dev ? a.parent : c.P.L.FS[0]) : nullptr;
    int* fround_dev = a.fixed_round ? (a.dev ? a.fixed_round : (int*)c.P.L.FS[1]) : nullptr;
    u64* lower_dev = (a_lower && a.dev) ? a_lower : nullptr;
    Pool tmp;
    tmp.al = c.pool.al;
    if (a.lower && !a.dev) RC(tmp.get(&lower_dev, h->n));
    int rc = enqueue_single(h, source, a.max_rounds, st, dist_dev, parent_dev, fround_dev, lower_dev,
                            a.has_target ? a.target : kNoTarget);
    // The host copies go on the stream before the status read, so that one
    // synchronisation covers the solve, the outputs and the status (outputs
    // are unspecified when the solve fails).
    if (rc == SSSP_OK && !a.dev) {
        cudaError_t e = cudaSuccess;
        if (a.dist && !dist_mapped)
            e = cudaMemcpyAsync(a.dist, dist_dev, sizeof(u64) * h->n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && a.parent)
            e = cudaMemcpyAsync(a.parent, parent_dev, sizeof(u32) * h->n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && a.fixed_round)
            e = cudaMemcpyAsync(a.fixed_round, fround_dev, sizeof(int) * h->n,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && a.lower)
            e = cudaMemcpyAsync(a.lower, lower_dev, sizeof(u64) * h->n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            rc = SSSP_E_CUDA;
        }
    }
    if (rc == SSSP_OK) rc = read_status(c, st, 1);
    else cudaStreamSynchronize(st);   // nothing enqueued may outlive the scratch below
    tmp.release();
    if (rc != SSSP_OK) return rc;
    const InstVar& v = c.h_ivar[0];
    if (v.status != kDone && v.status != kStopped) return SSSP_E_ROUND_LIMIT;
    if (info) {
        info->rounds = v.rounds;
        info->finished = v.status == kDone;
        info->out_scanned = c.h_ctl->stats[0];
        info->in_scanned = c.h_ctl->stats[1];
        info->active_visits = c.h_ctl->stats[2];
        info->front_visits = c.h_ctl->stats[3];
        info->reached = c.h_ctl->stats[4];
        info->kernel_launches = 4 + c.launches_per_iter * (u64)c.h_ctl->body_iters +
                                (c.last_loop == SSSP_LOOP_PERSISTENT ? 1 : 0);
    }
    return SSSP_OK;
}

int sssp_solve(sssp_handle h, uint32_t source, uint64_t* dist_out, uint32_t* rounds_out) {
    if (!h || !dist_out) return SSSP_E_INVAL;
    sssp_solve_args a{};
    a.dist = dist_out;
    sssp_solve_info info{};
    RC(sssp_solve_ex(h, source, &a, &info));
    if (rounds_out) *rounds_out = info.rounds;
    return SSSP_OK;
}

int sssp_solve_device(sssp_handle h, uint32_t source, uint64_t* dist_dev, uint32_t* rounds_out,
                      void* cuda_stream) {
    if (!h || !dist_dev) return SSSP_E_INVAL;
    if (source >= h->n) return SSSP_E_SOURCE_RANGE;
    DeviceGuard dg(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    RC(enqueue_single(h, source, 0, st, reinterpret_cast<u64*>(dist_dev), nullptr, nullptr,
                      nullptr, kNoTarget));
    if (rounds_out) {
        RC(read_status(h->single, st, 1));
        if (h->single.h_ivar[0].status != kDone) return SSSP_E_ROUND_LIMIT;
        *rounds_out = h->single.h_ivar[0].rounds;
    }
    return SSSP_OK;
}

int sssp_solve_batch(const sssp_handle* g, const uint32_t* sources, uint32_t k,
                     uint64_t* const* dist_out, uint32_t* rounds_out) {
    return batch_impl(g, sources, k, reinterpret_cast<u64* const*>(dist_out), false, rounds_out,
                      nullptr, false, nullptr);
}

int sssp_solve_batch_device(const sssp_handle* g, const uint32_t* sources, uint32_t k,
                            uint64_t* const* dist_dev, uint32_t* rounds_out, void* cuda_stream) {
    return batch_impl(g, sources, k, reinterpret_cast<u64* const*>(dist_dev), true, rounds_out,
                      (cudaStream_t)cuda_stream, true, nullptr);
}

int sssp_profile(sssp_handle h, int enable, sssp_kernel_profile* out) {
    if (!h || (enable != 0 && enable != 1)) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    Context& c = h->single;
    if (out) {
        out->relax_launches = c.prof_relax_n;
        out->cupdate_launches = c.prof_cup_n;
        out->relax_ms = c.prof_relax_ms;
        out->cupdate_ms = c.prof_cup_ms;
        out->tail_launches = c.prof_tail_n;
        out->tail_ms = c.prof_tail_ms;
        out->tail_rounds = c.prof_tail_rounds;
        for (int i = 0; i < 4; ++i) {
            out->grid_counters[i] = c.prof_grid_ctr[i];
            out->tail_counters[i] = c.prof_tail_ctr[i];
        }
    }
    c.prof_relax_n = c.prof_cup_n = c.prof_tail_n = c.prof_tail_rounds = 0;
    c.prof_relax_ms = c.prof_cup_ms = c.prof_tail_ms = 0;
    for (int i = 0; i < 4; ++i) c.prof_grid_ctr[i] = c.prof_tail_ctr[i] = 0;
    c.prof = enable != 0;
    return SSSP_OK;
}

int sssp_profile_rounds(sssp_handle h, float* relax_ms, float* cupdate_ms, float* tail_ms,
                        uint32_t* tail_rounds, uint64_t* grid_counters, uint32_t cap,
                        uint32_t* count) {
    if (!h || !count || (cap && (!relax_ms || !cupdate_ms))) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    const Context& c = h->single;
    const u32 n = (u32)c.prof_round_cup.size();
    for (u32 i = 0; i < n && i < cap; ++i) {
        relax_ms[i] = c.prof_round_relax[i];
        cupdate_ms[i] = c.prof_round_cup[i];
        if (tail_ms) tail_ms[i] = c.prof_round_tail[i];
        if (tail_rounds) tail_rounds[i] = c.prof_round_tail_rounds[i];
        if (grid_counters)
            for (u32 k = 0; k < 4; ++k) grid_counters[4 * i + k] = c.prof_round_ctr[4 * i + k];
    }
    *count = n;
    return SSSP_OK;
}

const char* sssp_strerror(int code) {
    switch (code) {
        case SSSP_OK: return "ok";
        case SSSP_PENDING: return "pending";
        case SSSP_E_INVAL: return "invalid argument";
        case SSSP_E_ZERO_WEIGHT: return "edge weight must be strictly positive";
        case SSSP_E_SOURCE_RANGE: return "source vertex out of range";
        case SSSP_E_OVERFLOW: return "n * max weight does not fit the packed distance word";
        case SSSP_E_NOMEM: return "out of device memory or budget";
        case SSSP_E_DEVICE_TIMEOUT: return "device-side wait timed out";
        case SSSP_E_CUDA: return "CUDA runtime error";
        case SSSP_E_ROUND_LIMIT: return "round limit exceeded";
        case SSSP_E_BUSY: return "server busy";
        case SSSP_E_NOT_FOUND: return "unknown ticket";
        case SSSP_E_INTERNAL: return "internal consistency guard tripped";
        case SSSP_E_NOALLOC_LIMIT:
            return "graph exceeds the fixed scratch of sssp_solve_noalloc "
                   "(SSSP_NOALLOC_MAX_VERTICES vertices)";
        default: return "unknown status";
    }
}

}  // extern "C"
