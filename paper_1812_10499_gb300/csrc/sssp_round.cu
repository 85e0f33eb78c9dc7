// sssp_round.cu -- sm_103a kernels of the SP_3/SP_4 round (Garg, arXiv
// 1812.10499, Sec. V-VI).
//
// One round r is two kernels:
//   k_relax   : SP_4 step 3, label-setting (as SP_3 explores only fixed
//               vertices): every out-edge (x, y, w) of a vertex x fixed in
//               round r - 1 lowers D[y] by a 64-bit atomicMin on the packed
//               (distance, parent) word when y is not fixed.  A y whose D was
//               infinite joins the active (discovered, unfixed) set.  The
//               minima of D and D + outWeight over the active set (SP_4 step
//               1; Lemmas 7 and 8) are folded in as relaxations succeed.
//   k_cupdate : SP_4 steps 4 and 5 for every active y, reading the lower
//               bounds of the previous round (Jacobi):
//                 lb(x) = max(C[x], min(D[x], threshold))
//                 C'[y] = max(C[y], min(D[y], threshold),
//                             min over in-edges (x, y) of lb(x) + w)   (Eq. 1)
//               y is fixed iff C'[y] = D[y]; fixed vertices form the next
//               frontier, the others stay active and seed the next round's
//               minima.  The last CTA to finish closes the round.
// Both kernels pull work dynamically: 32 list entries per warp with a
// warp-local load balance over their edges, or one chunk of a hub vertex.
// Every lane keeps kUnroll edges in flight (independent adjacency loads,
// then independent 32-byte state gathers); the adjacency is streamed with
// an evict-first policy so the state records stay in L2; list appends go
// through warp-private buffers flushed 32 entries per atomic.
#include "sssp_dev.cuh"

namespace sssp {

constexpr u32 kFull = 0xFFFFFFFFu;
constexpr u32 kUnroll = 4;     // edges per lane in flight
constexpr u32 kWarps = 8;      // warps per CTA (256 threads)
constexpr u32 kQCap = 64;      // entries of a warp append buffer

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ ulonglong4_32a ld_rec(const VRec* p) {
    return *reinterpret_cast<const ulonglong4_32a*>(p);
}
// The two words a round reads from a neighbour: packed D and the lower-bound
// word of round parity `cur` (both in the record's 32-byte sector).
struct DC {
    u64 d, c;
};
__device__ __forceinline__ DC ld_dc(const VRec* p, u32 cur) {
    DC r;
    if (cur == 0) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
        r.d = v.x;
        r.c = v.y;
    } else {
        r.d = p->dp;
        r.c = p->cf[1];
    }
    return r;
}
// Adjacency entries are read once per visit: stream them (evict first).
__device__ __forceinline__ uint2 ld_stream(const uint2* p) { return __ldcs(p); }
__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a > b ? a : b; }
__device__ __forceinline__ u32 ld_volatile(const u32* p) { return *(volatile const u32*)p; }
__device__ __forceinline__ u64 ld_volatile(const u64* p) { return *(volatile const u64*)p; }

__device__ __forceinline__ u32 warp_incl_scan(u32 x, u32 lane) {
#pragma unroll
    for (u32 d = 1; d < 32; d <<= 1) {
        u32 y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Largest lane i with excl_i <= j (excl is non-decreasing over lanes).
__device__ __forceinline__ u32 find_owner(u32 excl, u32 j) {
    u32 lo = 0;
#pragma unroll
    for (u32 step = 16; step >= 1; step >>= 1) {
        u32 e = __shfl_sync(kFull, excl, lo + step);
        if (e <= j) lo += step;
    }
    return lo;
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
__device__ __forceinline__ void put_hub(const RoundParams& P, u64* pk, uint2* list, u32 g,
                                        u64 deg) {
    u32 nch = (u32)((deg + P.chunk - 1) / P.chunk);
    u64 old = atomicAdd(pk, (1ull << 32) | nch);
    u32 idx = (u32)(old >> 32);
    if (idx < P.L.capH) list[idx] = make_uint2(g, (u32)old);
    else atomicOr(&P.ctl->error, 2u);
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

// Accumulators a thread carries through one kernel.
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

// Flush register folds and counters at the end of a kernel (all lanes).
template <bool MULTI>
__device__ __forceinline__ void flush(const RoundParams& P, u32 slot, Acc& a, u32 lane,
                                      int stat_edges, int stat_visits) {
    const u64 e = warp_sum64(a.edges), v = warp_sum64(a.visits);
    const u64 nf = warp_sum64(a.nfix);
    if (!MULTI) {
        const u64 d = warp_min64(a.fmin_d), t = warp_min64(a.fmin_t);
        if (lane == 0) {
            if (d != kInf64) atomic_min_checked(&P.ivar[0].minD[slot], d);
            if (t != kInf64) atomic_min_checked(&P.ivar[0].thr[slot], t);
            if (nf) atomicAdd(&P.ivar[0].nfix[slot], (u32)nf);
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

// ---------------------------------------------------------------- k_relax

// Relaxes kUnroll out-edges per lane (SP_4 step 3) and queues newly
// discovered targets.  Call with all lanes of the warp.
template <bool MULTI>
__device__ __forceinline__ void relax_edges(const RoundParams& P, u32 cur, const bool* ev,
                                            const uint2* e, const u64* dx, const u32* xloc,
                                            const u64* gbase, const u64* const* in_off,
                                            const u32* inst, Acc& a, WarpQueue& q, u32 lane) {
    DC v[kUnroll];
    u32 gy[kUnroll];
#pragma unroll
    for (u32 u = 0; u < kUnroll; ++u) {
        gy[u] = (u32)(gbase[u] + e[u].x);
        if (ev[u]) v[u] = ld_dc(P.rec + gy[u], cur);
    }
    bool fresh[kUnroll];
    u64 indeg[kUnroll];
#pragma unroll
    for (u32 u = 0; u < kUnroll; ++u) {
        fresh[u] = false;
        indeg[u] = 0;
        if (!ev[u]) continue;
        const u64 dd = dx[u] + e[u].y;
        const u64 cand = (dd << P.vbits) | xloc[u];
        if ((v[u].c & kFixed) || cand >= v[u].d) continue;
        const u64 old = atomicMin(&P.rec[gy[u]].dp, cand);
        if (cand < old) {
            const u32 ow = P.rec[gy[u]].outw;
            fold<MULTI>(P, inst[u], cur, dd, ow == kNoOutW ? P.dinf : dd + ow, a);
            fresh[u] = (old == kInf64);
        }
    }
#pragma unroll
    for (u32 u = 0; u < kUnroll; ++u)
        if (fresh[u]) indeg[u] = in_off[u][e[u].x + 1] - in_off[u][e[u].x];
#pragma unroll
    for (u32 u = 0; u < kUnroll; ++u) {
        const bool sm = fresh[u] && indeg[u] <= P.hub;
        wq_push(P, q, &P.ctl->nAS[cur], P.L.AS[cur], sm, gy[u], lane);
        if (fresh[u] && !sm) put_hub(P, &P.ctl->AHpk[cur], P.L.AH[cur], gy[u], indeg[u]);
    }
}

template <bool MULTI>
__device__ void relax_small(const RoundParams& P, u32 t, u32 nfs, u32 cur, u32 lane, Acc& a,
                            WarpQueue& q) {
    const u32 idx = t * 32 + lane;
    const bool valid = idx < nfs;
    u32 g = 0, xloc = 0, inst = 0, deg = 0;
    u64 gbase = 0, b = 0, dx = 0;
    const uint2* adj = P.g.out_adj;
    const u64* in_off = P.g.in_off;
    if (valid) {
        g = P.L.FS[cur][idx];
        const InstDesc& d = desc_of<MULTI>(P, g, inst);
        gbase = d.base;
        adj = d.out_adj;
        in_off = d.in_off;
        xloc = g - (u32)gbase;
        b = d.out_off[xloc];
        deg = (u32)(d.out_off[xloc + 1] - b);
        VRec* rx = P.rec + g;
        const u64 cfx = rx->cf[cur];
        rx->cf[cur ^ 1] = cfx;       // keep both copies "fixed" from now on
        dx = cfx & kCMask;           // C = D for a fixed vertex
        a.visits++;
    }
    const u32 incl = warp_incl_scan(deg, lane);
    const u32 total = __shfl_sync(kFull, incl, 31);
    const u32 excl = incl - deg;
    const u64 eaddr = (u64)(adj + b);
    for (u32 j0 = 0; j0 < total; j0 += 32 * kUnroll) {
        bool ev[kUnroll];
        uint2 e[kUnroll];
        u64 odx[kUnroll], ob[kUnroll];
        u32 ox[kUnroll], oinst[kUnroll];
        const u64* oin[kUnroll];
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u) {
            ev[u] = false;
            e[u] = make_uint2(0, 0);
            odx[u] = 0;
            ox[u] = 0;
            ob[u] = 0;
            oinst[u] = 0;
            oin[u] = in_off;
            if (j0 + 32 * u >= total) continue;    // warp-uniform
            const u32 j = j0 + 32 * u + lane;
            ev[u] = j < total;
            const u32 own = find_owner(excl, j);
            const u32 k = j - __shfl_sync(kFull, excl, own);
            const uint2* ep = reinterpret_cast<const uint2*>(__shfl_sync(kFull, eaddr, own)) + k;
            odx[u] = __shfl_sync(kFull, dx, own);
            ox[u] = __shfl_sync(kFull, xloc, own);
            if (MULTI) {
                ob[u] = __shfl_sync(kFull, gbase, own);
                oin[u] = reinterpret_cast<const u64*>(__shfl_sync(kFull, (u64)in_off, own));
                oinst[u] = __shfl_sync(kFull, inst, own);
            }
            if (ev[u]) e[u] = ld_stream(ep);
            a.edges += ev[u];
        }
        relax_edges<MULTI>(P, cur, ev, e, odx, ox, ob, oin, oinst, a, q, lane);
    }
}

template <bool MULTI>
__device__ void relax_hub(const RoundParams& P, u32 c, u32 nfh, u32 cur, u32 lane, Acc& a,
                          WarpQueue& q) {
    const uint2* FH = P.L.FH[cur];
    u32 lo = 0, hi = nfh;
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (FH[mid].y <= c) lo = mid; else hi = mid;
    }
    const uint2 ent = FH[lo];
    const u32 g = ent.x, k = c - ent.y;
    u32 inst;
    const InstDesc& d = desc_of<MULTI>(P, g, inst);
    const u32 xloc = g - (u32)d.base;
    const u64 b = d.out_off[xloc], e_end = d.out_off[xloc + 1];
    const u64 cb = b + (u64)k * P.chunk;
    const u64 ce = umin64(cb + P.chunk, e_end);
    VRec* rx = P.rec + g;
    const u64 cfx = rx->cf[cur];
    if (k == 0 && lane == 0) {
        rx->cf[cur ^ 1] = cfx;
        a.visits++;
    }
    bool ev[kUnroll];
    uint2 e[kUnroll];
    u64 odx[kUnroll], ob[kUnroll];
    u32 ox[kUnroll], oinst[kUnroll];
    const u64* oin[kUnroll];
#pragma unroll
    for (u32 u = 0; u < kUnroll; ++u) {
        odx[u] = cfx & kCMask;
        ox[u] = xloc;
        ob[u] = d.base;
        oinst[u] = inst;
        oin[u] = d.in_off;
    }
    for (u64 e0 = cb; e0 < ce; e0 += 32 * kUnroll) {
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u) {
            const u64 ei = e0 + 32 * u + lane;
            ev[u] = ei < ce;
            e[u] = ev[u] ? ld_stream(d.out_adj + ei) : make_uint2(0, 0);
            a.edges += ev[u];
        }
        relax_edges<MULTI>(P, cur, ev, e, odx, ox, ob, oin, oinst, a, q, lane);
    }
}

template <bool MULTI>
__global__ void __launch_bounds__(256, 2) k_relax(RoundParams P) {
    __shared__ u32 s_q[kWarps][kQCap];
    Ctl* ctl = P.ctl;
    if (ld_volatile(&ctl->status) != kRunning) return;
    const u32 r = ctl->round;
    const u32 cur = r & 1u, nxt = cur ^ 1u;
    const u32 lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;

    if (blockIdx.x == 0) {
        // Open the slots of round r + 1 (last read in round r - 1).
        if (threadIdx.x == 0) {
            // Watchdog: every round advances ctl->round, so more loop bodies
            // than the round limit means the epilogue stopped running.
            if (++ctl->loop_iters > ctl->round_limit) ctl->status = kErrRounds;
            ctl->nFS[nxt] = 0;
            ctl->nAS[nxt] = 0;
            ctl->FHpk[nxt] = 0;
            ctl->AHpk[nxt] = 0;
            ctl->work[1] = 0;
            ctl->done_ctas = 0;
        }
        for (u32 i = threadIdx.x; i < ctl->ninst; i += blockDim.x) {
            P.ivar[i].thr[nxt] = kInf64;
            P.ivar[i].minD[nxt] = kInf64;
            P.ivar[i].nfix[nxt] = 0;
        }
    }

    // Counts are clamped to the list capacities (an overflow is flagged in
    // ctl->error by the writer and can only come from a library bug).
    const u32 nfs = min(ctl->nFS[cur], P.L.capS);
    const u64 fhpk = ctl->FHpk[cur];
    const u32 nfh = min((u32)(fhpk >> 32), P.L.capH), fh_chunks = (u32)fhpk;
    const u32 tiles = (nfs + 31) >> 5;
    const u32 total = tiles + fh_chunks;

    Acc a = {kInf64, kInf64, 0, 0, 0};
    WarpQueue q = {s_q[wib], 0};
    for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&ctl->work[0], 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        if (item < tiles) relax_small<MULTI>(P, item, nfs, cur, lane, a, q);
        else relax_hub<MULTI>(P, item - tiles, nfh, cur, lane, a, q);
    }
    wq_flush(P, q, &ctl->nAS[cur], P.L.AS[cur], lane);
    flush<MULTI>(P, cur, a, lane, 0, 3);
}

// -------------------------------------------------------------- k_cupdate

// lb(x): the lower bound an in-neighbour contributes (Lemmas 7 and 8); with
// rule 1 the printed SP_4 step 4 clamp (minD for unfixed vertices).
__device__ __forceinline__ u64 lb_of(const RoundParams& P, const DC& v, u64 thr, u64 minD) {
    const u64 dx = v.d >> P.vbits;            // infinity maps to dinf
    const u64 cfx = v.c;
    const u64 cx = cfx & kCMask;
    if (P.rule == 0) return umax64(cx, umin64(dx, thr));
    return (cfx & kFixed) ? cx : umax64(cx, minD);
}

// Decision for one active vertex after its Eq. (1) minimum m is known.
__device__ __forceinline__ u64 decide(const RoundParams& P, u64 dy, u64 cy, u64 m, u64 thr,
                                      u64 minD, bool& fix) {
    u64 self = (P.rule == 0) ? umax64(cy, umin64(dy, thr)) : umax64(cy, minD);
    u64 cn = umax64(self, m);
    fix = (cn == dy) || (P.rule == 1 && dy <= thr);
    return fix ? dy : cn;
}

template <bool MULTI>
__device__ void cup_small(const RoundParams& P, u32 t, u32 nas, u32 r, u32 cur, u32 lane,
                          u64* smin, u64 thr0, u64 minD0, Acc& a, Acc& an, WarpQueue& qf,
                          WarpQueue& qa) {
    const u32 nxt = cur ^ 1u;
    const u32 idx = t * 32 + lane;
    const bool valid = idx < nas;
    u32 g = 0, yloc = 0, inst = 0, deg = 0, outw = kNoOutW;
    u64 gbase = 0, ib = 0, dy = 0, cy = 0, thr = thr0, minD = minD0;
    const uint2* in_adj = P.g.in_adj;
    const u64* out_off = P.g.out_off;
    if (valid) {
        g = P.L.AS[cur][idx];
        const InstDesc& d = desc_of<MULTI>(P, g, inst);
        gbase = d.base;
        in_adj = d.in_adj;
        out_off = d.out_off;
        if (MULTI) {
            thr = ld_volatile(&P.ivar[inst].thr[cur]);
            minD = ld_volatile(&P.ivar[inst].minD[cur]);
        }
        yloc = g - (u32)gbase;
        ib = d.in_off[yloc];
        deg = (u32)(d.in_off[yloc + 1] - ib);
        const ulonglong4_32a v = ld_rec(P.rec + g);
        dy = v.x >> P.vbits;
        cy = (cur ? v.z : v.y) & kCMask;
        outw = (u32)v.w;
    }
    smin[lane] = kInf64;
    __syncwarp();
    const u32 incl = warp_incl_scan(deg, lane);
    const u32 total = __shfl_sync(kFull, incl, 31);
    const u32 excl = incl - deg;
    const u64 eaddr = (u64)(in_adj + ib);
    for (u32 j0 = 0; j0 < total; j0 += 32 * kUnroll) {
        bool ev[kUnroll];
        uint2 e[kUnroll];
        u32 own[kUnroll];
        u64 othr[kUnroll], omin[kUnroll], ob[kUnroll];
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u) {
            ev[u] = false;
            own[u] = 0;
            e[u] = make_uint2(0, 0);
            othr[u] = thr;
            omin[u] = minD;
            ob[u] = 0;
            if (j0 + 32 * u >= total) continue;    // warp-uniform
            const u32 j = j0 + 32 * u + lane;
            ev[u] = j < total;
            own[u] = find_owner(excl, j);
            const u32 k = j - __shfl_sync(kFull, excl, own[u]);
            const uint2* ep =
                reinterpret_cast<const uint2*>(__shfl_sync(kFull, eaddr, own[u])) + k;
            if (MULTI) {
                othr[u] = __shfl_sync(kFull, thr, own[u]);
                omin[u] = __shfl_sync(kFull, minD, own[u]);
                ob[u] = __shfl_sync(kFull, gbase, own[u]);
            }
            if (ev[u]) e[u] = ld_stream(ep);
        }
        DC v[kUnroll];
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u)
            if (ev[u]) v[u] = ld_dc(P.rec + (u32)(ob[u] + e[u].x), cur);
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u) {
            if (j0 + 32 * u >= total) continue;    // warp-uniform
            u64 val = kInf64;
            if (ev[u]) val = umin64(lb_of(P, v[u], othr[u], omin[u]) + e[u].y, P.dinf);
            // Segmented min over lanes sharing an owner (contiguous by construction).
            const u32 key = ev[u] ? own[u] : 32u + lane;
#pragma unroll
            for (u32 dd = 1; dd < 32; dd <<= 1) {
                const u64 ov = __shfl_up_sync(kFull, val, dd);
                const u32 ok = __shfl_up_sync(kFull, key, dd);
                if (lane >= dd && ok == key) val = umin64(val, ov);
            }
            const u32 nk = __shfl_down_sync(kFull, key, 1);
            if (ev[u] && (lane == 31 || nk != key)) smin[own[u]] = umin64(smin[own[u]], val);
            __syncwarp();
        }
    }
    a.edges += (lane == 0) ? total : 0;

    bool fix = false;
    if (valid) {
        const u64 cn = decide(P, dy, cy, smin[lane], thr, minD, fix);
        VRec* ry = P.rec + g;
        ry->cf[nxt] = cn | (fix ? kFixed : 0ull);
        if (fix) ry->fround = (int)r;
        a.visits++;
    }
    __syncwarp();
    const bool fx = valid && fix, sv = valid && !fix;
    u64 odeg = 0;
    if (fx) odeg = out_off[yloc + 1] - out_off[yloc];
    const bool fs = fx && odeg <= P.hub;
    wq_push(P, qf, &P.ctl->nFS[nxt], P.L.FS[nxt], fs, g, lane);
    if (fx && !fs) put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], g, odeg);
    wq_push(P, qa, &P.ctl->nAS[nxt], P.L.AS[nxt], sv, g, lane);
    if (MULTI) {
        if (fx) atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
    } else {
        an.nfix += fx;
    }
    if (sv) fold<MULTI>(P, inst, nxt, dy, outw == kNoOutW ? P.dinf : dy + outw, an);
}

template <bool MULTI>
__device__ void cup_hub(const RoundParams& P, u32 c, u32 nah, u32 ah_chunks, u32 r, u32 cur,
                        u32 lane, u64 thr0, u64 minD0, Acc& a, Acc& an) {
    const u32 nxt = cur ^ 1u;
    const uint2* AH = P.L.AH[cur];
    u32 lo = 0, hi = nah;
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (AH[mid].y <= c) lo = mid; else hi = mid;
    }
    const uint2 ent = AH[lo];
    const u32 g = ent.x, k = c - ent.y;
    const u32 nch = ((lo + 1 < nah) ? AH[lo + 1].y : ah_chunks) - ent.y;
    u32 inst;
    const InstDesc& d = desc_of<MULTI>(P, g, inst);
    u64 thr = thr0, minD = minD0;
    if (MULTI) {
        thr = ld_volatile(&P.ivar[inst].thr[cur]);
        minD = ld_volatile(&P.ivar[inst].minD[cur]);
    }
    const u32 yloc = g - (u32)d.base;
    const u64 ib = d.in_off[yloc], ie = d.in_off[yloc + 1];
    const u64 cb = ib + (u64)k * P.chunk;
    const u64 ce = umin64(cb + P.chunk, ie);
    u64 val = kInf64;
    for (u64 e0 = cb + lane; e0 < ce; e0 += 32 * kUnroll) {
        uint2 e[kUnroll];
        bool ev[kUnroll];
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u) {
            ev[u] = e0 + 32 * u < ce;
            e[u] = ev[u] ? ld_stream(d.in_adj + e0 + 32 * u) : make_uint2(0, 0);
        }
        DC v[kUnroll];
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u)
            if (ev[u]) v[u] = ld_dc(P.rec + (u32)(d.base + e[u].x), cur);
#pragma unroll
        for (u32 u = 0; u < kUnroll; ++u)
            if (ev[u]) val = umin64(val, umin64(lb_of(P, v[u], thr, minD) + e[u].y, P.dinf));
    }
    val = warp_min64(val);
    if (lane != 0) return;
    a.edges += ce - cb;
    atomicMin(&P.L.hubmin[lo], val);
    __threadfence();
    if (atomicAdd(&P.L.hubcnt[lo], 1u) != nch - 1) return;
    // Last chunk of this hub: finish the vertex.
    __threadfence();
    const u64 m = atomicExch(&P.L.hubmin[lo], kInf64);
    P.L.hubcnt[lo] = 0;
    VRec* ry = P.rec + g;
    const ulonglong4_32a v = ld_rec(ry);
    const u64 dy = v.x >> P.vbits;
    const u64 cy = (cur ? v.z : v.y) & kCMask;
    const u32 outw = (u32)v.w;
    bool fix;
    const u64 cn = decide(P, dy, cy, m, thr, minD, fix);
    ry->cf[nxt] = cn | (fix ? kFixed : 0ull);
    a.visits++;
    if (fix) {
        ry->fround = (int)r;
        const u64 odeg = d.out_off[yloc + 1] - d.out_off[yloc];
        if (odeg <= P.hub) put_small(P, P.L.FS[nxt], atomicAdd(&P.ctl->nFS[nxt], 1u), g);
        else put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], g, odeg);
        if (MULTI) atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
        else an.nfix++;
    } else {
        put_hub(P, &P.ctl->AHpk[nxt], P.L.AH[nxt], g, ie - ib);
        fold<MULTI>(P, inst, nxt, dy, outw == kNoOutW ? P.dinf : dy + outw, an);
    }
}

// End of round r, run by the last CTA: retire finished queries, advance the
// round counter and set the device loop's condition.
__device__ void round_epilogue(const RoundParams& P, u32 r) {
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
        if (ld_volatile(&v->nfix[nxt]) == 0) {
            v->rounds = nr;
            v->status = kDone;
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
        ctl->running = total;
        ctl->round = r + 1;
        u32 st = kRunning;
        if (total == 0) st = kDone;
        else if (r + 1 > ctl->round_limit) st = kErrRounds;
        ctl->status = st;
        __threadfence();
        if (P.cond) cudaGraphSetConditional(P.cond, (st == kRunning && r + 1 <= ctl->stop_round) ? 1u : 0u);
    }
}

template <bool MULTI>
__global__ void __launch_bounds__(256, 2) k_cupdate(RoundParams P) {
    __shared__ u64 s_min[kWarps][32];
    __shared__ u32 s_qf[kWarps][kQCap];
    __shared__ u32 s_qa[kWarps][kQCap];
    __shared__ u32 s_last;
    Ctl* ctl = P.ctl;
    if (ld_volatile(&ctl->status) != kRunning) {
        // Nothing runs: make sure the device loop ends.
        if (P.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(P.cond, 0u);
        return;
    }
    const u32 r = ctl->round;
    const u32 cur = r & 1u, nxt = cur ^ 1u;
    const u32 lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->work[0] = 0;

    const u32 nas = min(ctl->nAS[cur], P.L.capS);
    const u64 ahpk = ctl->AHpk[cur];
    const u32 nah = min((u32)(ahpk >> 32), P.L.capH), ah_chunks = (u32)ahpk;
    const u32 tiles = (nas + 31) >> 5;
    const u32 total = tiles + ah_chunks;
    u64 thr = kInf64, minD = kInf64;
    if (!MULTI) {
        thr = P.ivar[0].thr[cur];
        minD = P.ivar[0].minD[cur];
    }

    Acc a = {kInf64, kInf64, 0, 0, 0};
    Acc an = {kInf64, kInf64, 0, 0, 0};
    WarpQueue qf = {s_qf[wib], 0}, qa = {s_qa[wib], 0};
    for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&ctl->work[1], 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        if (item < tiles)
            cup_small<MULTI>(P, item, nas, r, cur, lane, s_min[wib], thr, minD, a, an, qf, qa);
        else
            cup_hub<MULTI>(P, item - tiles, nah, ah_chunks, r, cur, lane, thr, minD, a, an);
        __syncwarp();
    }
    wq_flush(P, qf, &ctl->nFS[nxt], P.L.FS[nxt], lane);
    wq_flush(P, qa, &ctl->nAS[nxt], P.L.AS[nxt], lane);
    a.fmin_d = an.fmin_d;
    a.fmin_t = an.fmin_t;
    a.nfix = an.nfix;
    flush<MULTI>(P, nxt, a, lane, 1, 2);

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

// Starts the queries in slots [first, first + count) at the control block's
// current round: the source is fixed with D = C = 0 and forms the frontier.
template <bool MULTI>
__global__ void k_start(RoundParams P, u32 first, u32 count, u32 max_rounds) {
    Ctl* ctl = P.ctl;
    const u32 r = ctl->round;
    const u32 cur = r & 1u;
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
        const u32 s = d.source;
        const u32 g = (u32)(d.base + s);
        VRec rs;
        rs.dp = s;                    // distance 0, parent = itself
        rs.cf[0] = kFixed;
        rs.cf[1] = kFixed;
        rs.outw = d.outw[s];
        rs.fround = 0;
        P.rec[g] = rs;
        const u64 odeg = d.out_off[s + 1] - d.out_off[s];
        if (odeg <= P.hub) put_small(P, P.L.FS[cur], atomicAdd(&ctl->nFS[cur], 1u), g);
        else put_hub(P, &ctl->FHpk[cur], P.L.FH[cur], g, odeg);
        __threadfence();
        v->status = kRunning;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->status = kRunning;
        ctl->running += count;
    }
}

template __global__ void k_relax<false>(RoundParams);
template __global__ void k_relax<true>(RoundParams);
template __global__ void k_cupdate<false>(RoundParams);
template __global__ void k_cupdate<true>(RoundParams);
template __global__ void k_start<false>(RoundParams, u32, u32, u32);
template __global__ void k_start<true>(RoundParams, u32, u32, u32);

// --------------------------------------------- host access for the engine

const void* relax_fn(bool multi) {
    return multi ? (const void*)k_relax<true> : (const void*)k_relax<false>;
}
const void* cupdate_fn(bool multi) {
    return multi ? (const void*)k_cupdate<true> : (const void*)k_cupdate<false>;
}

cudaError_t launch_start(bool multi, const RoundParams& P, u32 first, u32 count, u32 max_rounds,
                         cudaStream_t st) {
    if (multi) k_start<true><<<1, 256, 0, st>>>(P, first, count, max_rounds);
    else k_start<false><<<1, 32, 0, st>>>(P, first, count, max_rounds);
    return cudaGetLastError();
}

int round_blocks_per_sm(int threads) {
    int a = 0, b = 0, c = 0, d = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cupdate<false>, threads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relax<false>, threads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_cupdate<true>, threads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_relax<true>, threads, 0);
    int m = a < b ? a : b;
    m = m < c ? m : c;
    m = m < d ? m : d;
    return m;
}

}  // namespace sssp
