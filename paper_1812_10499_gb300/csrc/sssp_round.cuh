// sssp_round.cuh -- sm_103a kernels of the SP_3/SP_4 round (Garg, arXiv
// 1812.10499, Sec. V-VI), as templates.  sssp_round.cu instantiates them for
// the two state layouts, sssp_round_pred.cu for the same layouts with SP_1's
// predecessor counts; the two compile in parallel.
//
// One round r is two phases:
//   relax   : SP_4 step 3, label-setting (as SP_3 explores only fixed
//             vertices): every out-edge (x, y, w) of a vertex x fixed in
//             round r - 1 lowers D[y] by a 64-bit atomicMin on the packed
//             (distance, parent) word when y is not fixed.  A y whose D was
//             infinite joins the active (discovered, unfixed) set.  The
//             minima of D and D + outWeight over the active set (SP_4 step
//             1; Lemmas 7 and 8) are folded in as relaxations succeed.
//   cupdate : SP_4 steps 4 and 5 for every active y, reading the lower
//             bounds of the previous round (Jacobi):
//               lb(x) = max(C[x], min(D[x], threshold))
//               C'[y] = max(C[y], min(D[y], threshold),
//                           min over in-edges (x, y) of lb(x) + w)   (Eq. 1)
//             y is fixed iff C'[y] = D[y]; fixed vertices form the next
//             frontier, the others stay active and seed the next round's
//             minima.
// The phases run as two kernels per round (k_relax, k_cupdate, driven by a
// CUDA graph or the host) or inside one persistent cooperative kernel
// (k_solve).  Work is pulled per warp: 32 list entries with a warp-local
// load balance over their edges, or one chunk of a hub vertex.  Edges go
// through a per-warp three-stage cp.async pipeline in shared memory:
// adjacency two batches ahead, neighbour states one batch ahead, compute on
// the current batch.  List appends go through warp-private buffers flushed
// 32 entries per atomic.  Every kernel is templated on the state layout:
// 32-byte records (WideL) or 16-byte records (NarrowL), either of them
// with predecessor counts (PredL).
#pragma once
#include "sssp_dev.cuh"

namespace sssp {

constexpr u32 kFull = 0xFFFFFFFFu;
constexpr u32 kWarps = 8;       // warps per CTA (256 threads)
constexpr u32 kSmallGrid = 32;  // grids up to this many CTAs run latency-bound rounds
constexpr u32 kQCap = 64;       // entries of a warp append buffer
// Build-time tuning: CTAs per SM the round kernels are compiled for, and
// edges per warp batch of the copy pipeline.
#ifndef SSSP_MIN_CTAS
#define SSSP_MIN_CTAS 3
#endif
#ifndef SSSP_CUP_MIN_CTAS
#define SSSP_CUP_MIN_CTAS 3
#endif
#ifndef SSSP_BATCH
#define SSSP_BATCH 64
#endif
constexpr u32 kB = SSSP_BATCH;  // edges per warp batch
constexpr u32 kBI = kB / 32;    // batch edges per lane
constexpr u32 kAS = 3;          // adjacency slots: batches b, b + 1, b + 2 in flight
constexpr u32 kDS = 2;          // neighbour-state slots: batches b, b + 1

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a > b ? a : b; }
__device__ __forceinline__ u32 ld_volatile(const u32* p) { return *(volatile const u32*)p; }
__device__ __forceinline__ u64 ld_volatile(const u64* p) { return *(volatile const u64*)p; }
__device__ __forceinline__ u32 lanemask_le(u32 lane) { return 0xFFFFFFFFu >> (31 - lane); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async_8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cp_async_16(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g)
                 : "memory");
}
// L2 policy for data read once per visit (adjacency): evicted first, so the
// per-vertex state stays resident in L2.
__device__ __forceinline__ u64 policy_evict_first() {
    u64 pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void cp_async_8_stream(void* s, const void* g, u64 pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(
                     smem_addr(s)),
                 "l"(g), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ----------------------------------------------------------- state layouts

// A lower-bound word is handled in the wide form: value | kFixed (bit 63).
__device__ __forceinline__ u64 widen_c(u32 c) {
    return (u64)(c & ~kFixedN) | ((u64)(c & kFixedN) << 32);
}
__device__ __forceinline__ u32 narrow_c(u64 c) {
    return (u32)(c & kCMask) | (u32)((c >> 32) & kFixedN);
}

// Staged neighbour state.  d() is the packed D word, c(cur) the wide-form
// lower-bound word of round parity cur.
struct DcSlot {                         // wide, k_cupdate: (D, C[cur])
    ulonglong2 v;
    __device__ __forceinline__ void issue(const VRec* p, u32 cur) {
        if (cur == 0) {
            cp_async_16(&v, p);
        } else {
            cp_async_8(&v.x, &p->dp);
            cp_async_8(&v.y, &p->cf[1]);
        }
    }
    __device__ __forceinline__ u64 d() const { return v.x; }
    __device__ __forceinline__ u64 c(u32) const { return v.y; }
    __device__ __forceinline__ bool fixed(u32) const { return (v.y & kFixed) != 0; }
};
struct RecSlot {                        // wide, k_relax: the whole record
    ulonglong2 lo, hi;
    __device__ __forceinline__ void issue(const VRec* p, u32) {
        cp_async_16(&lo, p);
        cp_async_16(&hi, reinterpret_cast<const char*>(p) + 16);
    }
    __device__ __forceinline__ u64 d() const { return lo.x; }
    __device__ __forceinline__ u64 c(u32 cur) const { return cur ? hi.x : lo.y; }
    __device__ __forceinline__ bool fixed(u32 cur) const { return (c(cur) & kFixed) != 0; }
    __device__ __forceinline__ u32 outw() const { return (u32)hi.y; }
    __device__ __forceinline__ u32 indeg() const { return (u32)(hi.y >> 32); }
};
struct NSlot {                          // compact: the whole 16-byte record
    ulonglong2 v;
    __device__ __forceinline__ void issue(const VRecN* p, u32) { cp_async_16(&v, p); }
    __device__ __forceinline__ u64 d() const { return v.x; }
    __device__ __forceinline__ u32 c32(u32 cur) const {
        return cur ? (u32)(v.y >> 32) : (u32)v.y;
    }
    __device__ __forceinline__ u64 c(u32 cur) const { return widen_c(c32(cur)); }
    __device__ __forceinline__ bool fixed(u32 cur) const { return (c32(cur) & kFixedN) != 0; }
};

// Clamps an in-neighbour bound term can take: lb(x) uses threshold (rule 0)
// or minD (rule 1) of the in-neighbour's query.
struct Bounds64 {
    u64 thr, minD;
};
struct Bounds32 {
    u32 thr, minD;
};
constexpr u32 kInf31 = kFixedN - 1;     // compact-layout term infinity

// lb(x): the lower bound an in-neighbour contributes (Lemmas 7 and 8); with
// rule 1 the printed SP_4 step 4 clamp (minD for unfixed vertices).
template <class S>
__device__ __forceinline__ u64 lb_of(const RoundParams& P, const S& v, u32 cur, u64 thr,
                                     u64 minD) {
    const u64 dx = v.d() >> P.vbits;          // infinity maps to dinf
    const u64 cw = v.c(cur);
    const u64 cx = cw & kCMask;
    if (P.rule == 0) return umax64(cx, umin64(dx, thr));
    return (cw & kFixed) ? cx : umax64(cx, minD);
}

struct WideL {
    typedef VRec Rec;
    typedef RecSlot RSlot;
    typedef DcSlot CSlot;
    static constexpr bool kNarrow = false;
    static constexpr bool kPred = false;
    // Eq. (1) term lb(x) + w of one in-edge, clamped to the distance infinity.
    typedef u64 Term;
    typedef Bounds64 Bounds;
    static constexpr u64 kTermInf = kInf64;
    __device__ static Bounds bounds(u64 thr, u64 minD) { return Bounds64{thr, minD}; }
    __device__ static Term term(const RoundParams& P, const CSlot& v, u32 cur, u32 w, Bounds b) {
        return umin64(lb_of(P, v, cur, b.thr, b.minD) + w, P.dinf);
    }
    __device__ static Rec* rec(const RoundParams& P) { return P.rec; }
    // (D word, wide C word of parity cur)
    __device__ static ulonglong2 ld_dc(const Rec* p, u32 cur) {
        if (cur == 0) return *reinterpret_cast<const ulonglong2*>(p);
        return make_ulonglong2(p->dp, p->cf[1]);
    }
    __device__ static void set_c(Rec* p, u32 slot, u64 c) { p->cf[slot] = c; }
};
struct NarrowL {
    typedef VRecN Rec;
    typedef NSlot RSlot;
    typedef NSlot CSlot;
    static constexpr bool kNarrow = true;
    static constexpr bool kPred = false;
    // The same term in 32-bit arithmetic.  Here the packed D word holds the
    // distance in its upper half (32 parent bits) and every finite value is
    // below 2^31 - 1, so lb(x) <= kInf31 and lb(x) + w cannot wrap.  Terms are
    // clamped to kInf31; a clamped term never decides the minimum, because an
    // active vertex y always has a fixed in-neighbour whose term is exactly
    // D[y] < kInf31 (D[y] is the least D[x] + w over the fixed in-neighbours,
    // all of which have relaxed their edges into y).
    typedef u32 Term;
    typedef Bounds32 Bounds;
    static constexpr u32 kTermInf = kInf31;
    __device__ static Bounds bounds(u64 thr, u64 minD) {
        return Bounds32{(u32)umin64(thr, kInf31), (u32)umin64(minD, kInf31)};
    }
    __device__ static Term term(const RoundParams& P, const CSlot& v, u32 cur, u32 w, Bounds b) {
        const u32 d = (u32)(v.v.x >> 32);
        const u32 cw = v.c32(cur);
        const u32 c = cw & ~kFixedN;
        u32 lb;
        if (P.rule == 0) lb = max(c, min(d, b.thr));
        else lb = (cw & kFixedN) ? c : max(c, b.minD);
        return min(lb + w, kInf31);
    }
    __device__ static Rec* rec(const RoundParams& P) { return P.recn; }
    __device__ static ulonglong2 ld_dc(const Rec* p, u32 cur) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
        return make_ulonglong2(v.x, widen_c((u32)(v.y >> (32 * cur))));
    }
    __device__ static void set_c(Rec* p, u32 slot, u64 c) { p->cf[slot] = narrow_c(c); }
};

// A layout with SP_1's predecessor counts (Sec. III): the relaxation
// decrements the count of every unfixed target, and the lower-bound phase
// fixes an active vertex whose count is 0 without reading its in-edges.
// The counting kernels are separate instantiations (compiled in their own
// translation unit), so the default kernels carry none of it.
template <class Base>
struct PredL : Base {
    static constexpr bool kPred = true;
};

// Shared-memory pipeline of one warp: adjacency of three batches and
// neighbour states of two; nz lists the lanes of the current tile with edges.
template <class S>
struct __align__(16) WarpStage {
    S dc[kDS][kB];
    uint2 adj[kAS][kB];                 // {neighbour, weight}
    unsigned char own[kAS][kB];         // lane owning the edge (small tiles)
    unsigned char nz[32];
};

__device__ __forceinline__ u32 warp_incl_scan(u32 x, u32 lane) {
#pragma unroll
    for (u32 d = 1; d < 32; d <<= 1) {
        u32 y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

__device__ __forceinline__ u64 warp_min64(u64 v) {
#pragma unroll
    for (u32 d = 16; d >= 1; d >>= 1) v = umin64(v, __shfl_xor_sync(kFull, v, d));
    return v;
}
__device__ __forceinline__ u64 warp_sum64(u64 v) {
#pragma unroll
    for (u32 d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ void put_small(const RoundParams& P, u32* list, u32 idx, u32 g) {
    if (idx < P.L.capS) list[idx] = g;
    else atomicOr(&P.ctl->error, 1u);
}
__device__ __forceinline__ void put_hub(const RoundParams& P, u64* pk, uint2* list, u32* cmap,
                                        u32 g, u64 deg) {
    const u32 nch = (u32)((deg + P.chunk - 1) / P.chunk);
    const u64 old = atomicAdd(pk, (1ull << 32) | nch);
    const u32 idx = (u32)(old >> 32), first = (u32)old;
    if (idx < P.L.capH) list[idx] = make_uint2(g, first);
    else atomicOr(&P.ctl->error, 2u);
    // Chunk -> entry map, so that a chunk finds its vertex with one load.
    const u32 end = min(first + nch, P.L.capC);
    for (u32 k = first; k < end; ++k) cmap[k] = idx;
}

// Entry of hub list `list` (n entries) that chunk c belongs to: from the
// chunk map, else by binary search over the entries' first chunks.
__device__ __forceinline__ u32 hub_entry(const RoundParams& P, const uint2* list, const u32* cmap,
                                         u32 n, u32 c) {
    if (c < P.L.capC) return min(cmap[c], n - 1);
    u32 lo = 0, hi = n;
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (list[mid].y <= c) lo = mid; else hi = mid;
    }
    return lo;
}

// Warp-private append buffer of one small list (in shared memory); the
// count is warp-uniform.  32 entries leave per global atomicAdd.
struct WarpQueue {
    u32* buf;
    u32 cnt;
};

__device__ __forceinline__ void wq_push(const RoundParams& P, WarpQueue& q, u32* counter,
                                        u32* list, bool pred, u32 g, u32 lane) {
    const u32 mask = __ballot_sync(kFull, pred);
    if (mask == 0) return;
    if (pred) q.buf[q.cnt + __popc(mask & ((1u << lane) - 1u))] = g;
    q.cnt += __popc(mask);
    __syncwarp();
    if (q.cnt >= 32) {
        u32 base = 0;
        if (lane == 0) base = atomicAdd(counter, 32u);
        base = __shfl_sync(kFull, base, 0);
        put_small(P, list, base + lane, q.buf[lane]);
        const u32 rest = q.cnt - 32;
        const u32 v = (lane < rest) ? q.buf[32 + lane] : 0u;
        __syncwarp();
        if (lane < rest) q.buf[lane] = v;
        __syncwarp();
        q.cnt = rest;
    }
}

__device__ __forceinline__ void wq_flush(const RoundParams& P, WarpQueue& q, u32* counter,
                                         u32* list, u32 lane) {
    if (q.cnt == 0) return;
    u32 base = 0;
    if (lane == 0) base = atomicAdd(counter, q.cnt);
    base = __shfl_sync(kFull, base, 0);
    if (lane < q.cnt) put_small(P, list, base + lane, q.buf[lane]);
    __syncwarp();
    q.cnt = 0;
}

// Flushes two queues; both counter atomics are in flight together.
__device__ __forceinline__ void wq_flush2(const RoundParams& P, WarpQueue& q1, u32* c1, u32* l1,
                                          WarpQueue& q2, u32* c2, u32* l2, u32 lane) {
    u32 b1 = 0, b2 = 0;
    if (lane == 0) {
        if (q1.cnt) b1 = atomicAdd(c1, q1.cnt);
        if (q2.cnt) b2 = atomicAdd(c2, q2.cnt);
    }
    b1 = __shfl_sync(kFull, b1, 0);
    b2 = __shfl_sync(kFull, b2, 0);
    if (lane < q1.cnt) put_small(P, l1, b1 + lane, q1.buf[lane]);
    if (lane < q2.cnt) put_small(P, l2, b2 + lane, q2.buf[lane]);
    __syncwarp();
    q1.cnt = 0;
    q2.cnt = 0;
}

// Appends g (where pred holds) to a small list with one atomic per warp.
__device__ __forceinline__ void warp_append(const RoundParams& P, u32* counter, u32* list,
                                            bool pred, u32 g, u32 lane) {
    const u32 mask = __ballot_sync(kFull, pred);
    if (mask == 0) return;
    u32 base = 0;
    if (lane == 0) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(kFull, base, 0);
    if (pred) put_small(P, list, base + __popc(mask & ((1u << lane) - 1u)), g);
}

// The static first work item of warp wib of this CTA.  Items are dealt
// round-robin over the CTAs, starting with CTA 1 and ending with CTA 0: a
// small list spreads over many SMs, and CTA 0 -- which runs the end-of-round
// epilogue right before the cluster tail kernel's next relaxation -- gets an
// item only when every other CTA has one.
__device__ __forceinline__ u32 static_item(u32 wib) {
    const u32 rank = blockIdx.x == 0 ? gridDim.x - 1 : blockIdx.x - 1;
    return wib * gridDim.x + rank;
}

// Accumulators a thread carries through one phase.
struct Acc {
    u64 fmin_d, fmin_t;     // folds of minD / threshold (single-query mode)
    u64 edges, visits;
    u32 nfix;               // vertices fixed (single-query mode)
};

__device__ __forceinline__ void atomic_min_checked(u64* p, u64 v) {
    if (v < ld_volatile(p)) atomicMin(p, v);
}

// Fold one unfixed vertex's (D, D + outWeight) into the minima of `slot`.
template <bool MULTI>
__device__ __forceinline__ void fold(const RoundParams& P, u32 inst, u32 slot, u64 d, u64 t,
                                     Acc& a) {
    if (MULTI) {
        atomic_min_checked(&P.ivar[inst].minD[slot], d);
        atomic_min_checked(&P.ivar[inst].thr[slot], t);
    } else {
        a.fmin_d = umin64(a.fmin_d, d);
        a.fmin_t = umin64(a.fmin_t, t);
    }
}

// Flush register folds and counters at the end of a phase (all lanes).
template <bool MULTI, bool NARROW = false>
__device__ __forceinline__ void flush(const RoundParams& P, u32 slot, u32 nfix_slot, Acc& a,
                                      u32 lane, int stat_edges, int stat_visits) {
    if (NARROW && gridDim.x <= kSmallGrid) {
        // Cluster-sized grid, compact layout: every sum and minimum fits 32
        // bits (distances below 2^31, D + outWeight below 2^32 - 2), so one
        // warp reduction each instead of shuffle trees.
        const u32 e32 = __reduce_add_sync(kFull, (u32)a.edges);
        const u32 v32 = __reduce_add_sync(kFull, (u32)a.visits);
        const u32 nf32 = __reduce_add_sync(kFull, (u32)a.nfix);
        if (!MULTI) {
            const u32 d32 = __reduce_min_sync(kFull, a.fmin_d == kInf64 ? kFull : (u32)a.fmin_d);
            const u32 t32 = __reduce_min_sync(kFull, a.fmin_t == kInf64 ? kFull : (u32)a.fmin_t);
            if (lane == 0) {
                if (d32 != kFull) atomicMin(&P.ivar[0].minD[slot], (u64)d32);
                if (t32 != kFull) atomicMin(&P.ivar[0].thr[slot], (u64)t32);
                if (nf32) atomicAdd(&P.ivar[0].nfix[nfix_slot], nf32);
            }
        }
        if (lane == 0) {
            if (e32) atomicAdd(&P.ctl->stats[stat_edges], (u64)e32);
            if (v32) atomicAdd(&P.ctl->stats[stat_visits], (u64)v32);
        }
        return;
    }
    const u64 e = warp_sum64(a.edges), v = warp_sum64(a.visits);
    const u64 nf = warp_sum64(a.nfix);
    if (!MULTI) {
        const u64 d = warp_min64(a.fmin_d), t = warp_min64(a.fmin_t);
        if (lane == 0) {
            // A large grid first reads the minimum, so that most warps skip
            // the atomic on this one address; a cluster-sized grid (few
            // warps, latency-bound rounds) fires the atomics without waiting.
            if (gridDim.x > kSmallGrid) {
                if (d != kInf64) atomic_min_checked(&P.ivar[0].minD[slot], d);
                if (t != kInf64) atomic_min_checked(&P.ivar[0].thr[slot], t);
            } else {
                if (d != kInf64) atomicMin(&P.ivar[0].minD[slot], d);
                if (t != kInf64) atomicMin(&P.ivar[0].thr[slot], t);
            }
            if (nf) atomicAdd(&P.ivar[0].nfix[nfix_slot], (u32)nf);
        }
    }
    if (lane == 0) {
        if (e) atomicAdd(&P.ctl->stats[stat_edges], e);
        if (v) atomicAdd(&P.ctl->stats[stat_visits], v);
    }
}

// Graph of the list entry g (local id, descriptor) in either mode.
template <bool MULTI>
__device__ __forceinline__ const InstDesc& desc_of(const RoundParams& P, u32 g, u32& inst) {
    if (MULTI) {
        inst = P.page_owner[g >> P.page_shift];
        return P.idesc[inst];
    }
    inst = 0;
    return P.g;
}

// outWeight of local vertex v: from the record (wide) or the graph (compact).
__device__ __forceinline__ u32 outw_rec(const InstDesc&, const VRec* r, u32) { return r->outw; }
__device__ __forceinline__ u32 outw_rec(const InstDesc& d, const VRecN*, u32 v) {
    const u32 ow = d.outw[v] & kInf31;            // bit 31: in-hub flag
    return ow == kInf31 ? kNoOutW : ow;
}
template <class L>
__device__ __forceinline__ u32 outw_of(const InstDesc& d, const typename L::Rec* r, u32 v) {
    return outw_rec(d, r, v);
}

// ------------------------------------------------------------- pipeline

// Drives batches 0 .. nbat-1 through the pipeline.  issue_adj(b, slot) and
// issue_dc(b, aslot, dslot) start cp.async copies (no wait); compute(b,
// aslot, dslot) consumes a batch.  Commit groups, in order: A0 A1 D0, then
// per batch b: A(b+2) D(b+1); so waiting for all but the newest group
// completes A(b+1), and all but the newest two completes D(b).  Batches are
// issued in increasing order.
template <class IA, class ID, class CO>
__device__ __forceinline__ void run_pipeline(u32 nbat, IA issue_adj, ID issue_dc, CO compute) {
    if (nbat == 0) return;
    issue_adj(0u, 0u);
    cp_async_commit();
    if (nbat > 1) issue_adj(1u, 1u);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    issue_dc(0u, 0u, 0u);
    cp_async_commit();
    for (u32 b = 0; b < nbat; ++b) {
        cp_async_wait<1>();
        __syncwarp();
        if (b + 2 < nbat) issue_adj(b + 2, (b + 2) % kAS);
        cp_async_commit();
        if (b + 1 < nbat) issue_dc(b + 1, (b + 1) % kAS, (b + 1) % kDS);
        cp_async_commit();
        cp_async_wait<2>();
        __syncwarp();
        compute(b, b % kAS, b % kDS);
        __syncwarp();
    }
    cp_async_wait<0>();
}

// A small tile: 32 list entries, lane i with deg_i edges starting at
// position excl_i of the tile's concatenated edge space.
struct Tile {
    u32 excl, total, nzmask;
    u32 hc;                              // segment heads in positions already issued
    u64 eaddr;                           // lane's first edge (uint2*)
    u64 pol;                             // L2 policy of the adjacency copies
};

template <class S>
__device__ __forceinline__ Tile make_tile(WarpStage<S>& st, u32 deg, u64 eaddr, u32 lane) {
    Tile t;
    const u32 incl = warp_incl_scan(deg, lane);
    t.total = __shfl_sync(kFull, incl, 31);
    t.excl = incl - deg;
    t.eaddr = eaddr;
    t.pol = policy_evict_first();
    t.nzmask = __ballot_sync(kFull, deg > 0);
    t.hc = 0;
    if (deg > 0) st.nz[__popc(t.nzmask & ((1u << lane) - 1u))] = (unsigned char)lane;
    __syncwarp();
    return t;
}

// Owner lane of position j0 + lane of a tile.  Rows are issued in order, so
// the owner's rank among the lanes with edges is the number of segment
// heads (an owner's first edge) at positions up to j0 + lane, minus one:
// the heads before j0 are carried in t.hc, those in the row come from one
// OR-reduction.  Position 0 is always a head.
template <class S>
__device__ __forceinline__ u32 row_owner(const WarpStage<S>& st, Tile& t, u32 j0, u32 deg,
                                         u32 lane) {
    const bool hd = deg > 0 && t.excl >= j0 && t.excl < j0 + 32;
    const u32 heads = __reduce_or_sync(kFull, hd ? (1u << (t.excl - j0)) : 0u);
    const u32 rank = t.hc + __popc(heads & lanemask_le(lane)) - 1u;
    t.hc += __popc(heads);
    return st.nz[rank & 31u];
}

// Starts copying edges [b0, b0 + kB) of a tile into adjacency slot s.
template <class S>
__device__ __forceinline__ void issue_tile_adj(WarpStage<S>& st, Tile& t, u32 s, u32 b0,
                                               u32 deg, u32 lane) {
#pragma unroll
    for (u32 i = 0; i < kBI; ++i) {
        const u32 j0 = b0 + 32 * i;
        if (j0 >= t.total) break;                 // warp-uniform
        const u32 own = row_owner(st, t, j0, deg, lane);
        const u32 j = j0 + lane;
        const u32 k = j - __shfl_sync(kFull, t.excl, own);
        const uint2* ep = reinterpret_cast<const uint2*>(__shfl_sync(kFull, t.eaddr, own)) + k;
        if (j < t.total) {
            cp_async_8_stream(&st.adj[s][32 * i + lane], ep, t.pol);
            st.own[s][32 * i + lane] = (unsigned char)own;
        }
    }
}

// Starts copying contiguous edges [e0, e1) (at most kB) into slot s.
template <class S>
__device__ __forceinline__ void issue_range_adj(WarpStage<S>& st, u32 s, const uint2* adj, u64 e0,
                                                u64 e1, u32 lane) {
    const u64 pol = policy_evict_first();
#pragma unroll
    for (u32 i = 0; i < kBI; ++i) {
        const u64 e = e0 + 32 * i + lane;
        if (e < e1) cp_async_8_stream(&st.adj[s][32 * i + lane], adj + e, pol);
    }
}

// Starts gathering the neighbour states of the nb edges in adjacency slot
// as into state slot ds.  `base` is the record base of the edge's graph,
// taken from the owning lane in multi-query mode.
template <bool MULTI, class L, bool RELAX = false, class S>
__device__ __forceinline__ void issue_dc(const RoundParams& P, WarpStage<S>& st, u32 as, u32 ds,
                                         u32 nb, u32 cur, u64 base, bool per_owner, u32 lane) {
    typename L::Rec* rec = L::rec(P);
    // The relaxation of the compact label-setting round stages the 8-byte
    // filter word (relaxation bound, outWeight) instead of the record.
    const bool filt = RELAX && L::kNarrow && P.gf != nullptr;
#pragma unroll
    for (u32 i = 0; i < kBI; ++i) {
        if (32 * i >= nb) break;                   // warp-uniform
        const u32 idx = 32 * i + lane;
        const bool ev = idx < nb;
        u64 ob = base;
        if (MULTI && per_owner) ob = __shfl_sync(kFull, base, ev ? st.own[as][idx] : 0u);
        if (!ev) continue;
        const u32 gy = (u32)(ob + st.adj[as][idx].x);
        if (filt) cp_async_8(&st.dc[ds][idx], P.gf + gy);
        else st.dc[ds][idx].issue(rec + gy, cur);
    }
}

// ------------------------------------------------------------------ relax

// Relaxations whose atomicMin results are still in flight.  A batch's
// results are consumed while the next batch is handled, so a warp does not
// wait for the atomics' round trip; the last batch of a phase is consumed
// at its end.
struct Pend {
    u64 cand[kBI], old[kBI];        // old = 0: nothing was tried
    u32 gy[kBI], yl[kBI];           // target record / local id
    u32 ow[kBI];                    // target outWeight (compact: | in-hub flag in bit 31)
    u32 deg[kBI];                   // target in-degree (wide layout)
    u32 inst[kBI];                  // target's query (multi-query mode)
    u32 r;                          // the round (label-correcting change marks)
    bool any;                       // a batch is pending (warp-uniform)
};

// Issues the relaxations of the staged edges [0, nb) (SP_4 step 3): per edge
// the owner's distance dx and id xloc.  A target that is fixed, or whose
// staged D is already no larger, is skipped.
template <bool MULTI, class L>
__device__ __forceinline__ void relax_issue(const RoundParams& P,
                                            WarpStage<typename L::RSlot>& st, u32 as, u32 ds,
                                            u32 nb, u32 cur, bool per_owner, u64 dx, u32 xloc,
                                            u64 gbase, u32 inst, Acc& a, Pend& pd, u32 lane) {
    typename L::Rec* rec = L::rec(P);
#pragma unroll
    for (u32 i = 0; i < kBI; ++i) {
        pd.cand[i] = 0;
        pd.old[i] = 0;
        if (32 * i >= nb) continue;                // warp-uniform
        const u32 idx = 32 * i + lane;
        const bool ev = idx < nb;
        const u32 own = (per_owner && ev) ? st.own[as][idx] : lane;
        u64 odx = dx;
        if (per_owner) {
            // Compact layout: distances are below 2^31, one 32-bit shuffle.
            if (L::kNarrow) odx = __shfl_sync(kFull, (u32)dx, own);
            else odx = __shfl_sync(kFull, dx, own);
        }
        const u32 ox = per_owner ? __shfl_sync(kFull, xloc, own) : xloc;
        u64 ob = gbase;
        u32 oi = inst;                             // an edge's target is in its source's query
        if (MULTI && per_owner) {
            ob = __shfl_sync(kFull, gbase, own);
            oi = __shfl_sync(kFull, inst, own);
        }
        if (!ev) continue;
        const uint2 e = st.adj[as][idx];
        const typename L::RSlot& v = st.dc[ds][idx];
        const u64 dd = odx + e.y;
        // A distance at the layout's limit cannot come from a graph whose
        // n * max weight fits it (checked when the graph is created); it
        // means an edge heavier than the declared maximum weight.
        if (dd >= (L::kNarrow ? kNarrowLimit : P.dinf)) {
            atomicOr(&P.ctl->error, 8u);
            continue;
        }
        const u64 cand = (dd << (L::kNarrow ? 32u : P.vbits)) | ox;
        pd.yl[i] = e.x;
        pd.gy[i] = (u32)(ob + e.x);
        pd.inst[i] = oi;
        if (L::kNarrow && P.gf) {
            // Filter word: bound 0 (fixed) rejects every candidate, a larger
            // distance cannot lower D; an equal one may (smaller parent).
            const uint2 fw = *reinterpret_cast<const uint2*>(&v);
            // SP_1's predecessor count: this edge into an unfixed y is relaxed.
            if (L::kPred && fw.x != 0u) atomicSub(&P.pcnt[pd.gy[i]], 1u);
            if (dd <= fw.x) {
                pd.cand[i] = cand;
                if (fw.x == kRelaxUnseen) pd.old[i] = atomicMin(&rec[pd.gy[i]].dp, cand);
                else atomicMin(&rec[pd.gy[i]].dp, cand);
                pd.ow[i] = fw.y;
            }
            a.edges++;
            continue;
        }
        if (L::kPred && !v.fixed(cur)) atomicSub(&P.pcnt[pd.gy[i]], 1u);
        if (!v.fixed(cur) && cand < v.d()) {
            pd.cand[i] = cand;
            // Windowed: D[y] changes this round (it ends at most cand, below the
            // D staged during this phase), so y must relax again.
            if (P.win) P.chg[pd.gy[i]] = 1u;
            // The old value is needed only to detect a first discovery (staged D
            // infinite) or, label-correcting, a change; otherwise the atomic is a
            // reduction whose result the warp never waits for.
            if (P.lc || v.d() == kInf64) pd.old[i] = atomicMin(&rec[pd.gy[i]].dp, cand);
            else atomicMin(&rec[pd.gy[i]].dp, cand);
            if (L::kNarrow) {
                const InstDesc& d = MULTI ? P.idesc[oi] : P.g;
                pd.ow[i] = d.outw[e.x];
            } else {
                const RecSlot& w = reinterpret_cast<const RecSlot&>(v);
                pd.ow[i] = w.outw();
                pd.deg[i] = w.indeg();
            }
        }
        a.edges++;
    }
    pd.any = true;
}

// Consumes a pending batch.  Every candidate that was issued folds its
// distance and distance + outWeight of the target into the minima of the
// round (Lemmas 7 and 8): the minimum over candidates into an active y is
// D[y] after the relaxation or more, and D[y] itself is folded (by its own
// winning candidate, or as a survivor of the previous round), so the minima
// are exact without knowing which candidate won.  A target whose D was
// infinite is newly discovered and joins the active set.
template <bool MULTI, class L>
__device__ __forceinline__ void relax_consume(const RoundParams& P, u32 cur, Acc& a, WarpQueue& q,
                                              WarpQueue& qf, Pend& pd, u32 lane) {
    if (!pd.any) return;
    pd.any = false;
    const u32 nxt = cur ^ 1u;
#pragma unroll
    for (u32 i = 0; i < kBI; ++i) {
        const bool issued = pd.cand[i] != 0;            // candidates are never 0
        const bool ok = pd.cand[i] < pd.old[i];         // old = 0 unless returned
        const bool fresh = ok && pd.old[i] == kInf64;
        bool hub = false;
        if (issued) {
            u32 ow = pd.ow[i];
            bool none;
            if (L::kNarrow) {
                hub = (ow >> 31) != 0;
                ow &= kInf31;
                none = ow == kInf31;
            } else {
                hub = pd.deg[i] > P.hub;
                none = ow == kNoOutW;
            }
            const u64 dd = pd.cand[i] >> (L::kNarrow ? 32u : P.vbits);
            fold<MULTI>(P, pd.inst[i], cur, dd, none ? P.dinf : dd + ow, a);
        }
        const bool sm = fresh && !hub;
        wq_push(P, q, &P.ctl->nAS[cur], P.L.AS[cur], sm, pd.gy[i], lane);
        if (fresh && hub) {
            u64 deg;
            if (L::kNarrow) {
                const InstDesc& d = MULTI ? P.idesc[pd.inst[i]] : P.g;
                deg = d.in_off[pd.yl[i] + 1] - d.in_off[pd.yl[i]];
            } else {
                deg = pd.deg[i];
            }
            put_hub(P, &P.ctl->AHpk[cur], P.L.AH[cur], P.L.AC[cur], pd.gy[i], deg);
        }
        if (P.lc) {
            // Label-correcting: a target whose D changed is relaxed again in
            // the next round (once, however often it changed in this one).
            const bool chg = ok && atomicExch(&P.chg[pd.gy[i]], pd.r) != pd.r;
            u64 odeg = 0;
            if (chg) {
                const InstDesc& d = MULTI ? P.idesc[pd.inst[i]] : P.g;
                odeg = d.out_off[pd.yl[i] + 1] - d.out_off[pd.yl[i]];
                if (MULTI) atomicAdd(&P.ivar[pd.inst[i]].nfix[nxt], 1u);
                else a.nfix++;
            }
            const bool fs = chg && odeg <= P.hub;
            wq_push(P, qf, &P.ctl->nFS[nxt], P.L.FS[nxt], fs, pd.gy[i], lane);
            if (chg && !fs) put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], P.L.FC[nxt], pd.gy[i], odeg);
        }
    }
}

template <bool MULTI, class L>
__device__ void relax_small(const RoundParams& P, WarpStage<typename L::RSlot>& st, u32 t,
                            u32 nfs, u32 cur, u32 lane, Acc& a, WarpQueue& q, WarpQueue& qf,
                            Pend& pd, bool has_pre, u32 gpre) {
    const u32 idx = t * 32 + lane;
    const bool valid = idx < nfs;
    u32 g = 0, xloc = 0, inst = 0, deg = 0;
    u64 gbase = 0, b = 0, dx = 0;
    const uint2* adj = P.g.out_adj;
    if (valid) {
        g = has_pre ? gpre : P.L.FS[cur][idx];
        const InstDesc& d = desc_of<MULTI>(P, g, inst);
        gbase = d.base;
        adj = d.out_adj;
        xloc = g - (u32)gbase;
        b = d.out_off[xloc];
        deg = (u32)(d.out_off[xloc + 1] - b);
        typename L::Rec* rx = L::rec(P) + g;
        rx->cf[cur ^ 1] = rx->cf[cur];              // keep both copies "fixed"
        // Label-setting: C = D for a fixed vertex.  Label-correcting and
        // windowed: the distance at the start of this relaxation step.
        dx = (P.lc || P.win) ? P.snap[g] : (L::ld_dc(rx, cur).y & kCMask);
        a.visits++;
    }
    Tile tl = make_tile(st, deg, (u64)(adj + b), lane);
    run_pipeline(
        (tl.total + kB - 1) / kB,
        [&](u32 bb, u32 s) { issue_tile_adj(st, tl, s, bb * kB, deg, lane); },
        [&](u32 bb, u32 as, u32 ds) {
            issue_dc<MULTI, L, true>(P, st, as, ds, min(kB, tl.total - bb * kB), cur, gbase, true,
                                     lane);
        },
        [&](u32 bb, u32 as, u32 ds) {
            relax_consume<MULTI, L>(P, cur, a, q, qf, pd, lane);
            relax_issue<MULTI, L>(P, st, as, ds, min(kB, tl.total - bb * kB), cur, true, dx, xloc,
                                  gbase, inst, a, pd, lane);
        });
}

template <bool MULTI, class L>
__device__ void relax_hub(const RoundParams& P, WarpStage<typename L::RSlot>& st, u32 c, u32 nfh,
                          u32 cur, u32 lane, Acc& a, WarpQueue& q, WarpQueue& qf, Pend& pd) {
    const uint2* FH = P.L.FH[cur];
    const uint2 ent = FH[hub_entry(P, FH, P.L.FC[cur], nfh, c)];
    const u32 g = ent.x, k = c - ent.y;
    u32 inst;
    const InstDesc& d = desc_of<MULTI>(P, g, inst);
    const u32 xloc = g - (u32)d.base;
    const u64 b = d.out_off[xloc], e_end = d.out_off[xloc + 1];
    const u64 cb = b + (u64)k * P.chunk;
    const u64 ce = umin64(cb + P.chunk, e_end);
    typename L::Rec* rx = L::rec(P) + g;
    const u64 dx = (P.lc || P.win) ? P.snap[g] : (L::ld_dc(rx, cur).y & kCMask);
    if (k == 0 && lane == 0) {
        rx->cf[cur ^ 1] = rx->cf[cur];
        a.visits++;
    }
    const u32 n = ce > cb ? (u32)(ce - cb) : 0u;
    run_pipeline(
        (n + kB - 1) / kB,
        [&](u32 bb, u32 s) { issue_range_adj(st, s, d.out_adj, cb + bb * kB, ce, lane); },
        [&](u32 bb, u32 as, u32 ds) {
            issue_dc<MULTI, L, true>(P, st, as, ds, min(kB, n - bb * kB), cur, d.base, false, lane);
        },
        [&](u32 bb, u32 as, u32 ds) {
            relax_consume<MULTI, L>(P, cur, a, q, qf, pd, lane);
            relax_issue<MULTI, L>(P, st, as, ds, min(kB, n - bb * kB), cur, false, dx, xloc,
                                  d.base, inst, a, pd, lane);
        });
}

template <class L>
constexpr size_t relax_smem() {
    return sizeof(WarpStage<typename L::RSlot>) * kWarps + 2 * sizeof(u32) * kWarps * kQCap;
}
template <class L>
constexpr size_t cupdate_smem() {
    return sizeof(WarpStage<typename L::CSlot>) * kWarps + sizeof(u64) * kWarps * 32 +
           2 * sizeof(u32) * kWarps * kQCap;
}

// Step (a) of round r over the whole frontier (all CTAs of the grid).
template <bool MULTI, class L>
__device__ void relax_phase(const RoundParams& P, unsigned char* s_dyn, u32 r) {
    typedef WarpStage<typename L::RSlot> Stage;
    Stage* s_st = reinterpret_cast<Stage*>(s_dyn);
    u32* s_q = reinterpret_cast<u32*>(s_dyn + sizeof(Stage) * kWarps);
    Ctl* ctl = P.ctl;
    const u32 cur = r & 1u, nxt = cur ^ 1u;
    const u32 lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    // The static item's small-list entry, loaded beside the list counts (one
    // memory round trip fewer); it is used only if the item is a small tile.
    const u32 item0 = static_item(wib);
    const u32 pidx = item0 * 32 + lane;
    const u32 gpre = pidx < P.L.capS ? P.L.FS[cur][pidx] : 0u;

    if (blockIdx.x == 0) {
        // Open the slots of round r + 1 (last read in round r - 1).
        // (Label-correcting: this relaxation appends the next frontier, so
        // its lists and counts were cleared by the previous round's end.)
        if (threadIdx.x == 0) {
            // Watchdog: every round advances ctl->round, so more loop bodies
            // than the round limit means the epilogue stopped running.
            if (++ctl->loop_iters > ctl->round_limit) ctl->status = kErrRounds;
            if (!P.lc) {
                ctl->nFS[nxt] = 0;
                ctl->FHpk[nxt] = 0;
            }
            ctl->nAS[nxt] = 0;
            ctl->AHpk[nxt] = 0;
            ctl->nFX[nxt] = 0;
            ctl->work[1] = 0;
            ctl->done_ctas = 0;
        }
        for (u32 i = threadIdx.x; i < ctl->ninst; i += blockDim.x) {
            P.ivar[i].thr[nxt] = kInf64;
            P.ivar[i].minD[nxt] = kInf64;
            if (!P.lc) P.ivar[i].nfix[nxt] = 0;
        }
    }

    // Counts are clamped to the list capacities (an overflow is flagged in
    // ctl->error by the writer and can only come from a library bug).
    const u32 nfs = min(ctl->nFS[cur], P.L.capS);
    const u64 fhpk = ctl->FHpk[cur];
    const u32 nfh = min((u32)(fhpk >> 32), P.L.capH), fh_chunks = (u32)fhpk;
    const u32 tiles = (nfs + 31) >> 5;
    // Label-correcting and windowed: copy the fixed lower-bound word of the
    // vertices fixed last round into the other parity slot (32 per item).
    const u32 nfx = (P.lc || P.win) ? min(ctl->nFX[cur], P.L.capS) : 0u;
    const u32 total = tiles + fh_chunks + ((nfx + 31) >> 5);

    Acc a = {kInf64, kInf64, 0, 0, 0};
    WarpQueue q = {s_q + wib * kQCap, 0};
    WarpQueue qf = {s_q + (kWarps + wib) * kQCap, 0};   // label-correcting next frontier
    Pend pd;
    pd.any = false;
    pd.r = r;
    // First item per warp is static (no atomic); the rest are pulled.
    const u32 nwarps = gridDim.x * kWarps;
    for (u32 item = item0; item < total;) {
        if (item < tiles) {
            relax_small<MULTI, L>(P, s_st[wib], item, nfs, cur, lane, a, q, qf, pd,
                                  item == item0, gpre);
        } else if (item < tiles + fh_chunks) {
            relax_hub<MULTI, L>(P, s_st[wib], item - tiles, nfh, cur, lane, a, q, qf, pd);
        } else {
            const u32 idx = (item - tiles - fh_chunks) * 32 + lane;
            if (idx < nfx) {
                typename L::Rec* rx = L::rec(P) + P.L.FX[cur][idx];
                rx->cf[nxt] = rx->cf[cur];
            }
        }
        if (total <= nwarps) break;                // the static items were all
        u32 next = 0;
        if (lane == 0) next = atomicAdd(&ctl->work[0], 1u) + nwarps;
        item = __shfl_sync(kFull, next, 0);
    }
    relax_consume<MULTI, L>(P, cur, a, q, qf, pd, lane);
    wq_flush2(P, q, &ctl->nAS[cur], P.L.AS[cur], qf, &ctl->nFS[nxt], P.L.FS[nxt], lane);
    flush<MULTI, L::kNarrow>(P, cur, nxt, a, lane, 0, 3);
}

template <bool MULTI, class L>
__global__ void __launch_bounds__(256, SSSP_MIN_CTAS) k_relax(RoundParams P) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->body_iters++;   // launch count
    if (ld_volatile(&P.ctl->status) != kRunning) return;
    if (ld_volatile(&P.ctl->cup_only)) return;     // relaxed already (tail kernel)
    relax_phase<MULTI, L>(P, s_dyn, P.ctl->round);
}

// ---------------------------------------------------------------- cupdate

// Segment minimum: brk has a bit at the first lane of every segment of
// contiguous lanes.  An inclusive segmented scan, exact at the segment's last
// lane.  (A warp reduction with each segment's lane mask gives every lane the
// minimum too, but it made the latency-bound rounds 9-13% slower.)
template <class T>
__device__ __forceinline__ T seg_min(T v, u32 brk, u32 lane) {
    const u32 span = lane - (31 - __clz(brk & lanemask_le(lane)));
#pragma unroll
    for (u32 dd = 1; dd < 32; dd <<= 1) {
        const T ov = __shfl_up_sync(kFull, v, dd);
        if (dd <= span) v = ov < v ? ov : v;
    }
    return v;
}

// The cheaper fixing rules tried before the in-edge scan: SP_2's in-version
// rule D[y] <= minD + inWeight[y] (Sec. IV) and D[y] <= threshold (Lemma 8).
// Each implies that Eq. (1) gives C[y] = D[y]: a fixed in-neighbour x gives
// D[x] + w >= D[y], an unfixed one lb(x) + w >= minD + inWeight[y].
__device__ __forceinline__ bool cheap_rules_fix(u64 dy, u32 inw, u64 thr, u64 minD) {
    return (inw != kNoOutW && dy <= minD + inw) || dy <= thr;
}

// Windowed relaxation: the bound below which a changed active vertex relaxes
// before it is fixed (minD of this round + delta, saturating).
__device__ __forceinline__ u64 win_limit(u64 minD, u64 delta) {
    const u64 l = minD + delta;
    return l < minD ? kInf64 : l;
}

// Decision for one active vertex after its Eq. (1) minimum m is known.
__device__ __forceinline__ u64 decide(const RoundParams& P, u64 dy, u64 cy, u64 m, u64 thr,
                                      u64 minD, bool& fix) {
    u64 self = (P.rule == 0) ? umax64(cy, umin64(dy, thr)) : umax64(cy, minD);
    u64 cn = umax64(self, m);
    fix = (cn == dy) || (P.rule == 1 && dy <= thr);
    return fix ? dy : cn;
}

// SHATOM (the cluster tail kernel): with the compact layout each edge's
// 32-bit term goes into its owner's slot by a shared-memory atomicMin
// instead of the segmented scan -- fewer dependent instructions per batch,
// which is what the small rounds wait on (random n = 4096 -15%, R-MAT 22
// +3%).  In large rounds, where many lanes share an owner, the scan is
// faster, and with the wide layout's 64-bit terms the atomics cost 1.4% on
// the 4096^2 grid, so both keep the scan.
template <bool MULTI, class L, bool SHATOM = false>
__device__ void cup_small(const RoundParams& P, WarpStage<typename L::CSlot>& st, u32 t, u32 nas,
                          u32 r, u32 cur, u32 lane, u64* smin, u64 thr0, u64 minD0, Acc& a,
                          Acc& an, WarpQueue& qf, WarpQueue& qa, bool has_pre, u32 gpre) {
    const u32 nxt = cur ^ 1u;
    const u32 idx = t * 32 + lane;
    const bool valid = idx < nas;
    u32 g = 0, yloc = 0, inst = 0, deg = 0, outw = kNoOutW;
    u64 gbase = 0, ib = 0, dy = 0, cy = 0, thr = thr0, minD = minD0, odeg = 0;
    bool fix_now = false;
    const uint2* in_adj = P.g.in_adj;
    typename L::Rec* rec = L::rec(P);
    if (valid) {
        g = has_pre ? gpre : P.L.AS[cur][idx];
        const InstDesc& d = desc_of<MULTI>(P, g, inst);
        gbase = d.base;
        in_adj = d.in_adj;
        if (MULTI) {
            thr = ld_volatile(&P.ivar[inst].thr[cur]);
            minD = ld_volatile(&P.ivar[inst].minD[cur]);
        }
        yloc = g - (u32)gbase;
        ib = d.in_off[yloc];
        deg = (u32)(d.in_off[yloc + 1] - ib);
        // Out-degree now, in the same round trip (needed if y gets fixed).
        odeg = d.out_off[yloc + 1] - d.out_off[yloc];
        const ulonglong2 v = L::ld_dc(rec + g, cur);
        dy = v.x >> P.vbits;
        cy = v.y & kCMask;
        outw = outw_of<L>(d, rec + g, yloc);
        if (P.cheap) fix_now = cheap_rules_fix(dy, d.inw[yloc], thr, minD);
        // SP_1: every in-edge relaxed by a fixed source, so D[y] is final.
        if (L::kPred && !fix_now) fix_now = P.pcnt[g] == 0u;
        if (fix_now) deg = 0;                     // its in-edges are not read
    }
    // The owners' minima: 64-bit slots, or (compact layout, SHATOM) 32-bit
    // slots in their place.
    constexpr bool kAtom = SHATOM && L::kNarrow;
    u32* smin32 = reinterpret_cast<u32*>(smin);
    if (kAtom) smin32[lane] = kInf31;
    else smin[lane] = kInf64;
    const typename L::Bounds bd = L::bounds(thr, minD);
    Tile tl = make_tile(st, deg, (u64)(in_adj + ib), lane);
    run_pipeline(
        (tl.total + kB - 1) / kB,
        [&](u32 b, u32 s) { issue_tile_adj(st, tl, s, b * kB, deg, lane); },
        [&](u32 b, u32 as, u32 ds) {
            issue_dc<MULTI, L>(P, st, as, ds, min(kB, tl.total - b * kB), cur, gbase, true, lane);
        },
        [&](u32 b, u32 as, u32 ds) {
            const u32 nb = min(kB, tl.total - b * kB);
#pragma unroll
            for (u32 i = 0; i < kBI; ++i) {
                if (32 * i >= nb) break;                   // warp-uniform
                const u32 sidx = 32 * i + lane;
                const bool ev = sidx < nb;
                const u32 own = ev ? st.own[as][sidx] : 0u;
                typename L::Bounds ob = bd;
                if (MULTI) {
                    ob.thr = __shfl_sync(kFull, bd.thr, own);
                    ob.minD = __shfl_sync(kFull, bd.minD, own);
                }
                typename L::Term val = L::kTermInf;
                if (ev) val = L::term(P, st.dc[ds][sidx], cur, st.adj[as][sidx].y, ob);
                if (kAtom) {
                    if (ev) atomicMin(smin32 + own, (u32)val);
                    continue;
                }
                // Min over the lanes sharing an owner (contiguous lanes; a
                // segment starts at every owner change).
                const u32 prev = __shfl_up_sync(kFull, own, 1);
                const u32 brk = __ballot_sync(kFull, lane == 0 || !ev || prev != own);
                if (L::kNarrow && brk == 1u) {
                    // The whole row is one owner's: one warp reduction.
                    val = __reduce_min_sync(kFull, (u32)val);
                    if (lane == 0) smin[own] = umin64(smin[own], (u64)val);
                } else {
                    val = seg_min(val, brk, lane);
                    const bool tail = ev && (lane == 31 || ((brk >> (lane + 1)) & 1u));
                    if (tail) smin[own] = umin64(smin[own], (u64)val);
                }
                __syncwarp();
            }
        });
    a.edges += (lane == 0) ? tl.total : 0;
    __syncwarp();

    bool fix = false;
    if (valid) {
        u64 cn = dy;
        if (fix_now) fix = true;
        else cn = decide(P, dy, cy, kAtom ? (u64)smin32[lane] : smin[lane], thr, minD, fix);
        L::set_c(rec + g, nxt, cn | (fix ? kFixed : 0ull));
        if (fix) P.fround[g] = (int)r;
        // Relaxation bound: D is stable until the next relaxation.
        if (L::kNarrow && P.gf) P.gf[g].x = fix ? 0u : (u32)dy;
        a.visits++;
    }
    __syncwarp();
    // Label-setting: the fixed vertices are the next frontier.  (Label-
    // correcting: the relaxation built it; the fixed vertices go to FX.)
    // Windowed: the fixed vertices and, while D < minD + delta, the
    // survivors -- each only if its D changed since it last relaxed; the
    // fixed vertices also go to FX.
    bool fx = valid && fix && !P.lc;
    const bool sv = valid && !fix;
    if (P.win) {
        fx = valid && P.chg[g] != 0 && (fix || dy < win_limit(minD, P.delta));
        if (fx) {
            P.chg[g] = 0;
            P.snap[g] = dy;
        }
        warp_append(P, &P.ctl->nFX[nxt], P.L.FX[nxt], valid && fix, g, lane);
    }
    const bool fs = fx && odeg <= P.hub;
    if (P.lc) wq_push(P, qf, &P.ctl->nFX[nxt], P.L.FX[nxt], valid && fix, g, lane);
    else wq_push(P, qf, &P.ctl->nFS[nxt], P.L.FS[nxt], fs, g, lane);
    if (fx && !fs) put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], P.L.FC[nxt], g, odeg);
    wq_push(P, qa, &P.ctl->nAS[nxt], P.L.AS[nxt], sv, g, lane);
    if (MULTI) {
        if (fx) atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
    } else {
        an.nfix += fx;
    }
    if (sv) fold<MULTI>(P, inst, nxt, dy, outw == kNoOutW ? P.dinf : dy + outw, an);
}

template <bool MULTI, class L>
__device__ void cup_hub(const RoundParams& P, WarpStage<typename L::CSlot>& st, u32 c, u32 nah,
                        u32 r, u32 cur, u32 lane, u64 thr0, u64 minD0, Acc& a, Acc& an) {
    const u32 nxt = cur ^ 1u;
    const uint2* AH = P.L.AH[cur];
    const u32 lo = hub_entry(P, AH, P.L.AC[cur], nah, c);
    const uint2 ent = AH[lo];
    const u32 g = ent.x, k = c - ent.y;
    u32 inst;
    const InstDesc& d = desc_of<MULTI>(P, g, inst);
    u64 thr = thr0, minD = minD0;
    if (MULTI) {
        thr = ld_volatile(&P.ivar[inst].thr[cur]);
        minD = ld_volatile(&P.ivar[inst].minD[cur]);
    }
    const u32 yloc = g - (u32)d.base;
    const u64 ib = d.in_off[yloc], ie = d.in_off[yloc + 1];
    const u32 nch = (u32)((ie - ib + P.chunk - 1) / P.chunk);   // as counted by put_hub
    const u64 cb = ib + (u64)k * P.chunk;
    const u64 ce = umin64(cb + P.chunk, ie);
    const typename L::Bounds bd = L::bounds(thr, minD);
    typename L::Term tv = L::kTermInf;
    // Cheaper rules first: every chunk of y takes the same decision (the
    // predecessor counts do not change during this phase).
    bool fix_now = false;
    if (P.cheap)
        fix_now = cheap_rules_fix(L::ld_dc(L::rec(P) + g, cur).x >> P.vbits, d.inw[yloc], thr,
                                  minD);
    if (L::kPred && !fix_now) fix_now = P.pcnt[g] == 0u;
    const u32 n = (ce > cb && !fix_now) ? (u32)(ce - cb) : 0u;
    run_pipeline(
        (n + kB - 1) / kB,
        [&](u32 b, u32 s) { issue_range_adj(st, s, d.in_adj, cb + b * kB, ce, lane); },
        [&](u32 b, u32 as, u32 ds) {
            issue_dc<MULTI, L>(P, st, as, ds, min(kB, n - b * kB), cur, d.base, false, lane);
        },
        [&](u32 b, u32 as, u32 ds) {
            const u32 nb = min(kB, n - b * kB);
#pragma unroll
            for (u32 i = 0; i < kBI; ++i) {
                const u32 sidx = 32 * i + lane;
                if (sidx < nb) tv = min(tv, L::term(P, st.dc[ds][sidx], cur, st.adj[as][sidx].y, bd));
            }
        });
    const u64 val = warp_min64((u64)tv);
    if (lane != 0) return;
    a.edges += n;
    atomicMin(&P.L.hubmin[lo], val);
    // The arrival count is an acquire-release atomic: it publishes this
    // chunk's minimum and, for the last arrival, makes every other chunk's
    // minimum visible before the vertex is finished.
    u32 arrived;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;\n"
                 : "=r"(arrived)
                 : "l"(&P.L.hubcnt[lo])
                 : "memory");
    if (arrived != nch - 1) return;
    // Last chunk of this hub: finish the vertex.
    const u64 m = atomicExch(&P.L.hubmin[lo], kInf64);
    P.L.hubcnt[lo] = 0;
    typename L::Rec* ry = L::rec(P) + g;
    const ulonglong2 v = L::ld_dc(ry, cur);
    const u64 dy = v.x >> P.vbits;
    const u64 cy = v.y & kCMask;
    const u32 outw = outw_of<L>(d, ry, yloc);
    bool fix = true;
    u64 cn = dy;
    if (!fix_now) cn = decide(P, dy, cy, m, thr, minD, fix);
    L::set_c(ry, nxt, cn | (fix ? kFixed : 0ull));
    if (L::kNarrow && P.gf) P.gf[g].x = fix ? 0u : (u32)dy;
    a.visits++;
    // The next frontier and FX as in cup_small.
    bool front = fix && !P.lc;
    if (fix) {
        P.fround[g] = (int)r;
        if (P.lc || P.win) put_small(P, P.L.FX[nxt], atomicAdd(&P.ctl->nFX[nxt], 1u), g);
    } else {
        put_hub(P, &P.ctl->AHpk[nxt], P.L.AH[nxt], P.L.AC[nxt], g, ie - ib);
        fold<MULTI>(P, inst, nxt, dy, outw == kNoOutW ? P.dinf : dy + outw, an);
    }
    if (P.win) {
        front = P.chg[g] != 0 && (fix || dy < win_limit(minD, P.delta));
        if (front) {
            P.chg[g] = 0;
            P.snap[g] = dy;
        }
    }
    if (front) {
        const u64 odeg = d.out_off[yloc + 1] - d.out_off[yloc];
        if (odeg <= P.hub) put_small(P, P.L.FS[nxt], atomicAdd(&P.ctl->nFS[nxt], 1u), g);
        else put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], P.L.FC[nxt], g, odeg);
        if (MULTI) atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
        else an.nfix++;
    }
}

// Whether query v has rounds left after round r (nxt = the parity of round
// r + 1): a next frontier (counted in nfix) or, windowed, active vertices
// that wait outside the window (their D was folded into minD[nxt]).
__device__ __forceinline__ bool has_next(const RoundParams& P, const InstVar* v, u32 nxt) {
    if (ld_volatile(&v->nfix[nxt]) != 0) return true;
    return P.win && ld_volatile(&v->minD[nxt]) != kInf64;
}

// End of round r, run by the last CTA: retire finished queries, advance the
// round counter and set the device loop's condition.
__device__ inline void round_epilogue(const RoundParams& P, u32 r) {
    __shared__ u32 s_running;
    Ctl* ctl = P.ctl;
    const u32 nxt = (r & 1u) ^ 1u;
    if (threadIdx.x == 0) s_running = 0;
    __syncthreads();
    u32 running = 0;
    const u32 ninst = ctl->ninst;
    for (u32 i = threadIdx.x; i < ninst; i += blockDim.x) {
        InstVar* v = P.ivar + i;
        if (ld_volatile(&v->status) != kRunning) continue;
        const u32 nr = r - v->start_round + 1;
        const u32 tgt = v->target;
        if (!has_next(P, v, nxt)) {
            v->rounds = nr;
            v->status = kDone;
        } else if (tgt != kNoTarget &&
                   *(volatile const int*)&P.fround[(P.idesc ? P.idesc[i].base : P.g.base) + tgt] >=
                       0) {
            v->rounds = nr;                     // the target is fixed: query answered
            v->status = kStopped;
        } else if (v->max_rounds != 0 && nr >= v->max_rounds) {
            v->rounds = nr;
            v->status = kStopped;
        } else {
            running++;
        }
    }
    if (running) atomicAdd(&s_running, running);
    __syncthreads();
    if (threadIdx.x == 0) {
        const u32 total = s_running;
        // Vertices fixed this round (single query): label-setting counts them
        // in nfix, label-correcting and windowed relaxation list them in FX.
        if (ninst == 1) ctl->stats[4] += (P.lc || P.win) ? ctl->nFX[nxt] : P.ivar[0].nfix[nxt];
        ctl->running = total;
        ctl->cup_only = 0;
        ctl->round = r + 1;
        u32 st = kRunning;
        if (total == 0) st = kDone;
        else if (r + 1 > ctl->round_limit) st = kErrRounds;
        ctl->status = st;
        __threadfence();
        if (P.cond)
            cudaGraphSetConditional(P.cond, (st == kRunning && r + 1 <= ctl->stop_round) ? 1u : 0u);
    }
}

// Label-correcting: one item of the next frontier's distance snapshot (32
// entries of the small list, then 32 of the hub list).
template <class L>
__device__ __forceinline__ void snap_frontier(const RoundParams& P, u32 k, u32 nxt, u32 sfs,
                                              u32 sfh, u32 lane) {
    const u32 fs_tiles = (sfs + 31) >> 5;
    u32 g = 0;
    bool ok;
    if (k < fs_tiles) {
        const u32 idx = k * 32 + lane;
        ok = idx < sfs;
        if (ok) g = P.L.FS[nxt][idx];
    } else {
        const u32 idx = (k - fs_tiles) * 32 + lane;
        ok = idx < sfh;
        if (ok) g = P.L.FH[nxt][idx].x;
    }
    if (ok) P.snap[g] = L::rec(P)[g].dp >> P.vbits;
}

// Steps (b) and (c) of round r over the whole active set (all CTAs); TAIL:
// inside the cluster tail kernel.
template <bool MULTI, class L, bool TAIL = false>
__device__ void cupdate_phase(const RoundParams& P, unsigned char* s_dyn, u32 r) {
    typedef WarpStage<typename L::CSlot> Stage;
    Stage* s_st = reinterpret_cast<Stage*>(s_dyn);
    u64* s_min = reinterpret_cast<u64*>(s_dyn + sizeof(Stage) * kWarps);
    u32* s_qf = reinterpret_cast<u32*>(s_min + kWarps * 32);
    u32* s_qa = s_qf + kWarps * kQCap;
    Ctl* ctl = P.ctl;
    const u32 cur = r & 1u, nxt = cur ^ 1u;
    const u32 lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    // The static item's small-list entry, loaded beside the list counts (as
    // in relax_phase).
    const u32 item0 = static_item(wib);
    const u32 pidx = item0 * 32 + lane;
    const u32 gpre = pidx < P.L.capS ? P.L.AS[cur][pidx] : 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->work[0] = 0;
    if (P.lc && blockIdx.x == 0) {
        // Label-correcting: the next relaxation appends the frontier after it
        // into slot cur, whose frontier this round's relaxation has consumed.
        for (u32 i = threadIdx.x; i < ctl->ninst; i += blockDim.x) P.ivar[i].nfix[cur] = 0;
        if (threadIdx.x == 0) {
            ctl->nFS[cur] = 0;
            ctl->FHpk[cur] = 0;
        }
    }

    const u32 nas = min(ctl->nAS[cur], P.L.capS);
    const u64 ahpk = ctl->AHpk[cur];
    const u32 nah = min((u32)(ahpk >> 32), P.L.capH), ah_chunks = (u32)ahpk;
    const u32 tiles = (nas + 31) >> 5;
    // Label-correcting: also record the distance of every next-frontier
    // vertex while D is stable (its relaxation reads it next round).
    u32 sfs = 0, sfh = 0, snap_items = 0;
    if (P.lc) {
        sfs = min(ctl->nFS[nxt], P.L.capS);
        sfh = min((u32)(ctl->FHpk[nxt] >> 32), P.L.capH);
        snap_items = ((sfs + 31) >> 5) + ((sfh + 31) >> 5);
    }
    const u32 total = tiles + ah_chunks + snap_items;
    u64 thr = kInf64, minD = kInf64;
    if (!MULTI) {
        thr = P.ivar[0].thr[cur];
        minD = P.ivar[0].minD[cur];
    }

    Acc a = {kInf64, kInf64, 0, 0, 0};
    Acc an = {kInf64, kInf64, 0, 0, 0};
    WarpQueue qf = {s_qf + wib * kQCap, 0}, qa = {s_qa + wib * kQCap, 0};
    // First item per warp is static (no atomic); the rest are pulled.
    const u32 nwarps = gridDim.x * kWarps;
    for (u32 item = item0; item < total;) {
        if (item < tiles)
            cup_small<MULTI, L, TAIL>(P, s_st[wib], item, nas, r, cur, lane, s_min + wib * 32,
                                      thr, minD, a, an, qf, qa, item == item0, gpre);
        else if (item < tiles + ah_chunks)
            cup_hub<MULTI, L>(P, s_st[wib], item - tiles, nah, r, cur, lane, thr, minD, a, an);
        else
            snap_frontier<L>(P, item - tiles - ah_chunks, nxt, sfs, sfh, lane);
        __syncwarp();
        if (total <= nwarps) break;                // the static items were all
        u32 next = 0;
        if (lane == 0) next = atomicAdd(&ctl->work[1], 1u) + nwarps;
        item = __shfl_sync(kFull, next, 0);
    }
    // (Label-correcting: qf carries the vertices fixed this round, to FX.)
    if (P.lc) wq_flush2(P, qf, &ctl->nFX[nxt], P.L.FX[nxt], qa, &ctl->nAS[nxt], P.L.AS[nxt], lane);
    else wq_flush2(P, qf, &ctl->nFS[nxt], P.L.FS[nxt], qa, &ctl->nAS[nxt], P.L.AS[nxt], lane);
    a.fmin_d = an.fmin_d;
    a.fmin_t = an.fmin_t;
    a.nfix = an.nfix;
    flush<MULTI, L::kNarrow>(P, nxt, nxt, a, lane, 1, 2);
}

template <bool MULTI, class L>
__global__ void __launch_bounds__(256, SSSP_CUP_MIN_CTAS) k_cupdate(RoundParams P) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ u32 s_last;
    Ctl* ctl = P.ctl;
    if (ld_volatile(&ctl->status) != kRunning) {
        // Nothing runs: make sure the device loop ends.
        if (P.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(P.cond, 0u);
        return;
    }
    const u32 r = ctl->round;
    cupdate_phase<MULTI, L>(P, s_dyn, r);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&ctl->done_ctas, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        round_epilogue(P, r);
    }
}

// ------------------------------------------------------- persistent loop

// Grid-wide barrier of the persistent kernel (all CTAs are co-resident:
// cooperative launch).  The last CTA to arrive runs the end-of-round
// epilogue when asked, then releases the others.  A CTA that waits longer
// than kBarrierTimeoutNs sets ctl->error bit 4 and returns false, so the
// kernel ends instead of hanging.
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline bool grid_barrier(const RoundParams& P, bool epilogue, u32 r) {
    __shared__ u32 s_last, s_gen;
    Ctl* ctl = P.ctl;
    const unsigned long long lim = P.barrier_ns ? P.barrier_ns : kBarrierTimeoutNs;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_gen = ld_volatile(&ctl->bar_gen);
        __threadfence();
        s_last = (atomicAdd(&ctl->bar_count, 1u) + 1 == gridDim.x) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (epilogue) round_epilogue(P, r);
        if (threadIdx.x == 0) {
            const u32 ti = 2 * (r - P.trace_base) + (epilogue ? 2u : 1u);
            if (P.trace && ti < P.trace_cap) P.trace[ti] = global_ns();
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        while (ld_volatile(&ctl->bar_gen) == s_gen) {
            if (global_ns() - t0 > lim) {
                atomicOr(&ctl->error, 4u);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
    }
    __syncthreads();
    return (ld_volatile(&ctl->error) & 4u) == 0;
}

// All rounds of the running queries in one launch: relax phase, barrier,
// lower-bound phase, barrier (whose last arriver closes the round), until
// no query runs, the stop round is passed, or a barrier times out.
template <bool MULTI, class L>
__global__ void __launch_bounds__(256, SSSP_MIN_CTAS) k_solve(RoundParams P) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    Ctl* ctl = P.ctl;
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && P.trace_cap) P.trace[0] = global_ns();
    for (;;) {
        if (ld_volatile(&ctl->status) != kRunning) break;
        const u32 r = ld_volatile(&ctl->round);
        if (r > ld_volatile(&ctl->stop_round)) break;
        relax_phase<MULTI, L>(P, s_dyn, r);
        if (!grid_barrier(P, false, r)) break;
        cupdate_phase<MULTI, L>(P, s_dyn, r);
        if (!grid_barrier(P, true, r)) break;
    }
}

// ---------------------------------------------------- cluster tail kernel

// Rounds whose work is small are latency chains: list -> offsets ->
// adjacency -> neighbour states, twice per round.  Two full-grid launches
// and a grid-wide arrival add several microseconds to each.  The tail kernel
// runs such rounds back to back in one thread-block cluster (kTailCTAs CTAs,
// hardware cluster barriers between phases).  Appended to every iteration
// of the device loop, it starts only when the next round is small and hands
// back to the full grid when a round grows.
constexpr u32 kTailCTAs = 16;

// Cluster-wide barrier; its release / acquire semantics order every global
// memory access before it (in any CTA of the cluster) before every access
// after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Whether round ctl->round starts in the tail kernel: the loop is running
// and not past its stop round, and the frontier and the active set known
// before the round each make at most P.tail_items work items (32-entry
// tiles plus hub chunks).  The relaxation may add active vertices: the
// second phase is checked again after it (tail_cup_fits).
__device__ __forceinline__ u32 tail_decide(const RoundParams& P) {
    const Ctl* ctl = P.ctl;
    if (ld_volatile(&ctl->status) != kRunning) return 0;
    const u32 r = ld_volatile(&ctl->round);
    if (r > ld_volatile(&ctl->stop_round)) return 0;
    const u32 cur = r & 1u;
    const u32 fi = ((ld_volatile(&ctl->nFS[cur]) + 31) >> 5) + (u32)ld_volatile(&ctl->FHpk[cur]);
    const u32 ai = ((ld_volatile(&ctl->nAS[cur]) + 31) >> 5) + (u32)ld_volatile(&ctl->AHpk[cur]);
    return (fi <= P.tail_items && ai <= P.tail_items) ? 1u : 0u;
}

__device__ __forceinline__ u32 tail_cup_fits(const RoundParams& P, u32 r) {
    const Ctl* ctl = P.ctl;
    const u32 cur = r & 1u;
    const u32 ai = ((ld_volatile(&ctl->nAS[cur]) + 31) >> 5) + (u32)ld_volatile(&ctl->AHpk[cur]);
    return ai <= P.tail_items ? 1u : 0u;
}

// Whether a single query goes on to round r + 1 in the tail kernel: the
// decision of the end-of-round epilogue (a round that leaves no next frontier
// -- and, windowed, no active vertex -- ends the query; so do the target and
// the round limits) and the frontier's size check.  Every input is final once
// round r's lower-bound phase has passed a cluster barrier and is written by no
// step of round r + 1, so CTAs that already started its relaxation (which
// appends to the active lists: their size is checked after it, tail_cup_fits)
// cannot change another CTA's decision.  The one exception, minD of round r + 1
// (the relaxation folds its candidates into it), is read only when the next
// frontier is empty, and then round r + 1 relaxes nothing.
__device__ __forceinline__ bool tail_next_single(const RoundParams& P, u32 r) {
    const InstVar* v = P.ivar;
    const Ctl* ctl = P.ctl;
    const u32 nxt = (r & 1u) ^ 1u;
    // Every load first (one memory round trip), then the decision.
    const u32 tgt = v->target;
    const u32 nfix = ld_volatile(&v->nfix[nxt]);
    const u64 mind = ld_volatile(&v->minD[nxt]);
    const int tfix = tgt != kNoTarget ? *(volatile const int*)&P.fround[P.g.base + tgt] : -1;
    const u32 stop = ld_volatile(&ctl->stop_round);
    const u32 nfs = ld_volatile(&ctl->nFS[nxt]);
    const u64 fhpk = ld_volatile(&ctl->FHpk[nxt]);
    if (nfix == 0 && !(P.win && mind != kInf64)) return false;   // has_next
    if (tfix >= 0) return false;
    if (v->max_rounds != 0 && r - v->start_round + 1 >= v->max_rounds) return false;
    if (r + 1 > ctl->round_limit || r + 1 > stop) return false;
    return ((nfs + 31) >> 5) + (u32)fhpk <= P.tail_items;
}

// Launched as one cluster of kTailCTAs CTAs.  Every CTA takes the same
// number of cluster barriers: each loop decision is either computed by every
// CTA from the same values, final at the barrier before it, or (several
// queries) written by CTA 0 before a barrier and read by all after it.  CTA 0
// alone writes the end-of-round state; with a single query the other CTAs
// start the next relaxation meanwhile, which reads none of that state (the
// round number is passed along, not read back).
template <bool MULTI, class L>
__global__ void __launch_bounds__(256, 1) k_tail(RoundParams P) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    Ctl* ctl = P.ctl;
    const bool lead = blockIdx.x == 0;
    if (lead && threadIdx.x == 0) ctl->tail_go = tail_decide(P);
    cluster_sync_all();
    bool go = ld_volatile(&ctl->tail_go) != 0;
    u32 r = ld_volatile(&ctl->round);
    while (go) {
        relax_phase<MULTI, L>(P, s_dyn, r);
        cluster_sync_all();
        if (!tail_cup_fits(P, r)) {
            // The relaxation grew the active set: the full grid finishes
            // the round (its relax launch is skipped).
            if (lead && threadIdx.x == 0) ctl->cup_only = 1;
            break;
        }
        cupdate_phase<MULTI, L, true>(P, s_dyn, r);
        cluster_sync_all();
        if (!MULTI) {
            go = tail_next_single(P, r);
            if (lead) round_epilogue(P, r);
            ++r;
        } else {
            if (lead) {
                round_epilogue(P, r);
                if (threadIdx.x == 0) ctl->tail_go = tail_decide(P);
            }
            cluster_sync_all();
            go = ld_volatile(&ctl->tail_go) != 0;
            r = ld_volatile(&ctl->round);
        }
    }
    // The device loop goes on while rounds remain (the epilogue's setting
    // is overridden here because the tail kernel ends the loop body).
    if (lead && threadIdx.x == 0 && P.cond) {
        const u32 st = ld_volatile(&ctl->status);
        const u32 rr = ld_volatile(&ctl->round);
        cudaGraphSetConditional(P.cond,
                                (st == kRunning && rr <= ld_volatile(&ctl->stop_round)) ? 1u : 0u);
    }
}

// -------------------------------------------------- per-query start state

// Starts the queries in slots [first, first + count) at the control block's
// current round: the source is fixed with D = C = 0 and forms the frontier.
// target (single query only, kNoTarget otherwise): stop once it is fixed; a
// target equal to the source is answered without any round.
template <bool MULTI, class L>
__global__ void k_start(RoundParams P, u32 first, u32 count, u32 max_rounds, u32 target) {
    __shared__ u32 s_run;
    Ctl* ctl = P.ctl;
    const u32 r = ctl->round;
    const u32 cur = r & 1u;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (u32 i = threadIdx.x; i < count; i += blockDim.x) {
        const u32 slot = first + i;
        const InstDesc& d = MULTI ? P.idesc[slot] : P.g;
        InstVar* v = P.ivar + slot;
        v->thr[0] = v->thr[1] = kInf64;
        v->minD[0] = v->minD[1] = kInf64;
        v->nfix[0] = v->nfix[1] = 0;
        v->start_round = r;
        v->rounds = 0;
        v->max_rounds = max_rounds;
        v->target = target;
        const u32 s = d.source;
        const u32 g = (u32)(d.base + s);
        typename L::Rec* rs = L::rec(P) + g;
        rs->dp = s;                   // distance 0, parent = itself
        L::set_c(rs, 0, kFixed);
        L::set_c(rs, 1, kFixed);
        if (L::kNarrow && P.gf) P.gf[g].x = 0u;   // fixed: no relaxation into it
        P.fround[g] = 0;
        if (P.snap) P.snap[g] = 0;    // label-correcting: relaxed in round 1 with D = 0
        if (target == s) {            // answered: the source is fixed
            __threadfence();
            v->status = kStopped;
            continue;
        }
        const u64 odeg = d.out_off[s + 1] - d.out_off[s];
        if (odeg <= P.hub) put_small(P, P.L.FS[cur], atomicAdd(&ctl->nFS[cur], 1u), g);
        else put_hub(P, &ctl->FHpk[cur], P.L.FH[cur], P.L.FC[cur], g, odeg);
        __threadfence();
        v->status = kRunning;
        atomicAdd(&s_run, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->stats[4] += count;       // the sources are fixed
        if (s_run) {
            ctl->status = kRunning;
            ctl->running += s_run;
        }
    }
}

// ----------------------------------------------- host access for the engine

enum class RoundKernel { kRelax, kCupdate, kSolve, kTail };

// Address of one round kernel for the layouts W (32-byte records) and N
// (16-byte records); instantiating this instantiates the kernels, so each
// translation unit that includes this header does it for its own layouts.
template <class W, class N>
const void* round_kernel(RoundKernel k, bool multi, bool narrow) {
    switch (k) {
        case RoundKernel::kRelax:
            if (multi) return narrow ? (const void*)k_relax<true, N> : (const void*)k_relax<true, W>;
            return narrow ? (const void*)k_relax<false, N> : (const void*)k_relax<false, W>;
        case RoundKernel::kCupdate:
            if (multi)
                return narrow ? (const void*)k_cupdate<true, N> : (const void*)k_cupdate<true, W>;
            return narrow ? (const void*)k_cupdate<false, N> : (const void*)k_cupdate<false, W>;
        case RoundKernel::kSolve:
            if (multi) return narrow ? (const void*)k_solve<true, N> : (const void*)k_solve<true, W>;
            return narrow ? (const void*)k_solve<false, N> : (const void*)k_solve<false, W>;
        case RoundKernel::kTail:
            if (multi) return narrow ? (const void*)k_tail<true, N> : (const void*)k_tail<true, W>;
            return narrow ? (const void*)k_tail<false, N> : (const void*)k_tail<false, W>;
    }
    return nullptr;
}

// The kernels of the layouts with predecessor counts (sssp_round_pred.cu).
const void* pred_round_kernel(RoundKernel k, bool multi, bool narrow);

}  // namespace sssp
