// sssp_round.cu -- sm_103a kernels of the SP_3/SP_4 round (Garg, arXiv
// 1812.10499, Sec. V-VI) and the per-graph setup kernels.
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
#include "sssp_dev.cuh"

namespace sssp {

constexpr u32 kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ ulonglong4_32a ld_rec(const VRec* p) {
    return *reinterpret_cast<const ulonglong4_32a*>(p);
}
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

// Warp-aggregated append: one atomicAdd per warp.  Call with all lanes.
__device__ __forceinline__ u32 warp_append(u32* counter, bool pred, u32 lane) {
    u32 mask = __ballot_sync(kFull, pred);
    if (mask == 0) return 0;
    u32 leader = __ffs(mask) - 1;
    u32 base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(kFull, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
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

// Accumulators a thread carries through one kernel.
struct Acc {
    u64 fmin_d, fmin_t;     // folds of minD / threshold (single-query mode)
    u64 edges, visits;
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
    u64 e = warp_sum64(a.edges), v = warp_sum64(a.visits);
    if (!MULTI) {
        u64 d = warp_min64(a.fmin_d), t = warp_min64(a.fmin_t);
        if (lane == 0) {
            if (d != kInf64) atomic_min_checked(&P.ivar[0].minD[slot], d);
            if (t != kInf64) atomic_min_checked(&P.ivar[0].thr[slot], t);
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

// Relaxes one out-edge (x -> y, w) of a fixed x (SP_4 step 3) and appends a
// newly discovered y to the active lists.  Call with all lanes of the warp.
template <bool MULTI>
__device__ __forceinline__ void relax_edge(const RoundParams& P, u32 cur, bool ev,
                                           const uint2* ep, u64 dx, u32 xloc, u64 gbase,
                                           const u64* in_off, u32 inst, Acc& a, u32 lane) {
    bool fresh = false;
    u32 gy = 0;
    u64 indeg = 0;
    if (ev) {
        uint2 e = *ep;                        // {y, w}
        u64 d = dx + e.y;
        u64 cand = (d << P.vbits) | xloc;
        gy = (u32)(gbase + e.x);
        VRec* ry = P.rec + gy;
        ulonglong4_32a v = ld_rec(ry);
        u64 cf = cur ? v.z : v.y;
        if (!(cf & kFixed) && cand < v.x) {
            u64 old = atomicMin(&ry->dp, cand);
            if (cand < old) {
                u32 ow = (u32)v.w;
                fold<MULTI>(P, inst, cur, d, ow == kNoOutW ? P.dinf : d + ow, a);
                if (old == kInf64) {
                    fresh = true;
                    indeg = in_off[e.x + 1] - in_off[e.x];
                }
            }
        }
    }
    bool sm = fresh && indeg <= P.hub;
    u32 idx = warp_append(&P.ctl->nAS[cur], sm, lane);
    if (sm) put_small(P, P.L.AS[cur], idx, gy);
    if (fresh && !sm) put_hub(P, &P.ctl->AHpk[cur], P.L.AH[cur], gy, indeg);
}

template <bool MULTI>
__device__ void relax_small(const RoundParams& P, u32 t, u32 nfs, u32 cur, u32 lane, Acc& a) {
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
        u64 cfx = rx->cf[cur];
        rx->cf[cur ^ 1] = cfx;       // keep both copies "fixed" from now on
        dx = cfx & kCMask;           // C = D for a fixed vertex
        a.visits++;
    }
    const u32 incl = warp_incl_scan(deg, lane);
    const u32 total = __shfl_sync(kFull, incl, 31);
    const u32 excl = incl - deg;
    const u64 eaddr = (u64)(adj + b);
    for (u32 j0 = 0; j0 < total; j0 += 32) {
        const u32 j = j0 + lane;
        const bool ev = j < total;
        const u32 own = find_owner(excl, j);
        const u32 k = j - __shfl_sync(kFull, excl, own);
        const uint2* ep = reinterpret_cast<const uint2*>(__shfl_sync(kFull, eaddr, own)) + k;
        const u64 odx = __shfl_sync(kFull, dx, own);
        const u32 ox = __shfl_sync(kFull, xloc, own);
        u64 ob = 0;
        const u64* oin = in_off;
        u32 oinst = 0;
        if (MULTI) {
            ob = __shfl_sync(kFull, gbase, own);
            oin = reinterpret_cast<const u64*>(__shfl_sync(kFull, (u64)in_off, own));
            oinst = __shfl_sync(kFull, inst, own);
        }
        relax_edge<MULTI>(P, cur, ev, ep, odx, ox, ob, oin, oinst, a, lane);
        a.edges += ev;
    }
}

template <bool MULTI>
__device__ void relax_hub(const RoundParams& P, u32 c, u32 nfh, u32 cur, u32 lane, Acc& a) {
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
    const u64 b = d.out_off[xloc], e = d.out_off[xloc + 1];
    const u64 cb = b + (u64)k * P.chunk;
    const u64 ce = umin64(cb + P.chunk, e);
    VRec* rx = P.rec + g;
    const u64 cfx = rx->cf[cur];
    const u64 dx = cfx & kCMask;
    if (k == 0 && lane == 0) {
        rx->cf[cur ^ 1] = cfx;
        a.visits++;
    }
    for (u64 e0 = cb; e0 < ce; e0 += 32) {
        const u64 ei = e0 + lane;
        const bool ev = ei < ce;
        relax_edge<MULTI>(P, cur, ev, d.out_adj + ei, dx, xloc, d.base, d.in_off, inst, a, lane);
        a.edges += ev;
    }
}

template <bool MULTI>
__global__ void __launch_bounds__(256) k_relax(RoundParams P) {
    Ctl* ctl = P.ctl;
    if (ld_volatile(&ctl->status) != kRunning) return;
    const u32 r = ctl->round;
    const u32 cur = r & 1u, nxt = cur ^ 1u;
    const u32 lane = threadIdx.x & 31u;

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

    Acc a = {kInf64, kInf64, 0, 0};
    for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&ctl->work[0], 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        if (item < tiles) relax_small<MULTI>(P, item, nfs, cur, lane, a);
        else relax_hub<MULTI>(P, item - tiles, nfh, cur, lane, a);
    }
    flush<MULTI>(P, cur, a, lane, 0, 3);
}

// -------------------------------------------------------------- k_cupdate

// lb(x): the lower bound an in-neighbour contributes (Lemmas 7 and 8); with
// rule 1 the printed SP_4 step 4 clamp (minD for unfixed vertices).
__device__ __forceinline__ u64 lb_of(const RoundParams& P, u32 cur, u32 gx, u64 thr, u64 minD) {
    const ulonglong4_32a v = ld_rec(P.rec + gx);
    const u64 dx = v.x >> P.vbits;            // infinity maps to dinf
    const u64 cfx = cur ? v.z : v.y;
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
                          u64* smin, u64 thr0, u64 minD0, Acc& a, Acc& an) {
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
    for (u32 j0 = 0; j0 < total; j0 += 32) {
        const u32 j = j0 + lane;
        const bool ev = j < total;
        const u32 own = find_owner(excl, j);
        const u32 k = j - __shfl_sync(kFull, excl, own);
        const uint2* ep = reinterpret_cast<const uint2*>(__shfl_sync(kFull, eaddr, own)) + k;
        u64 othr = thr, omin = minD, ob = 0;
        if (MULTI) {
            othr = __shfl_sync(kFull, thr, own);
            omin = __shfl_sync(kFull, minD, own);
            ob = __shfl_sync(kFull, gbase, own);
        }
        u64 val = kInf64;
        if (ev) {
            const uint2 e = *ep;                     // {x, w}
            const u64 lb = lb_of(P, cur, (u32)(ob + e.x), othr, omin);
            val = umin64(lb + e.y, P.dinf);
        }
        // Segmented min over lanes sharing an owner (contiguous by construction).
        const u32 key = ev ? own : 32u + lane;
#pragma unroll
        for (u32 dd = 1; dd < 32; dd <<= 1) {
            const u64 ov = __shfl_up_sync(kFull, val, dd);
            const u32 ok = __shfl_up_sync(kFull, key, dd);
            if (lane >= dd && ok == key) val = umin64(val, ov);
        }
        const u32 nk = __shfl_down_sync(kFull, key, 1);
        if (ev && (lane == 31 || nk != key)) smin[own] = umin64(smin[own], val);
        __syncwarp();
    }
    a.edges += (lane == 0) ? total : 0;

    bool fix = false;
    u64 cn = 0;
    if (valid) {
        cn = decide(P, dy, cy, smin[lane], thr, minD, fix);
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
    u32 pos = warp_append(&P.ctl->nFS[nxt], fs, lane);
    if (fs) put_small(P, P.L.FS[nxt], pos, g);
    if (fx && !fs) put_hub(P, &P.ctl->FHpk[nxt], P.L.FH[nxt], g, odeg);
    pos = warp_append(&P.ctl->nAS[nxt], sv, lane);
    if (sv) put_small(P, P.L.AS[nxt], pos, g);
    if (MULTI) {
        if (fx) atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
    } else {
        const u32 c = __popc(__ballot_sync(kFull, fx));
        if (lane == 0 && c) atomicAdd(&P.ivar[0].nfix[nxt], c);
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
    for (u64 e0 = cb + lane; e0 < ce; e0 += 32) {
        const uint2 e = d.in_adj[e0];
        const u64 lb = lb_of(P, cur, (u32)(d.base + e.x), thr, minD);
        val = umin64(val, umin64(lb + e.y, P.dinf));
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
        atomicAdd(&P.ivar[inst].nfix[nxt], 1u);
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
__global__ void __launch_bounds__(256) k_cupdate(RoundParams P) {
    __shared__ u64 s_min[8][32];
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

    Acc a = {kInf64, kInf64, 0, 0};
    Acc an = {kInf64, kInf64, 0, 0};
    for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&ctl->work[1], 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        if (item < tiles) cup_small<MULTI>(P, item, nas, r, cur, lane, s_min[wib], thr, minD, a, an);
        else cup_hub<MULTI>(P, item - tiles, nah, ah_chunks, r, cur, lane, thr, minD, a, an);
        __syncwarp();
    }
    a.fmin_d = an.fmin_d;
    a.fmin_t = an.fmin_t;
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

// ------------------------------------------------------- start / finalize

// Every record of a single query: D = inf, C = 0 (Fig. SP_4 declarations).
__global__ void k_init_records(VRec* rec, const u32* outw, u32 n) {
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        VRec r;
        r.dp = kInf64;
        r.cf[0] = 0;
        r.cf[1] = 0;
        r.outw = outw[v];
        r.fround = -1;
        rec[v] = r;
    }
}

// Records of all multi-query slots (pages not owned by a slot are skipped).
__global__ void k_init_records_multi(RoundParams P, u64 nrec, u32 first_page, u32 npages) {
    const u64 lo = (u64)first_page << P.page_shift;
    const u64 hi = umin64(nrec, (u64)(first_page + npages) << P.page_shift);
    for (u64 g = lo + blockIdx.x * (u64)blockDim.x + threadIdx.x; g < hi;
         g += (u64)gridDim.x * blockDim.x) {
        const u32 inst = P.page_owner[g >> P.page_shift];
        if (inst == kFull) continue;
        const InstDesc& d = P.idesc[inst];
        const u64 v = g - d.base;
        if (v >= d.n) continue;
        VRec r;
        r.dp = kInf64;
        r.cf[0] = 0;
        r.cf[1] = 0;
        r.outw = d.outw[v];
        r.fround = -1;
        P.rec[g] = r;
    }
}

// Resets the control block for a fresh solve context.
__global__ void k_reset_ctl(Ctl* ctl, u32 ninst, u32 round_limit) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctl c;
    memset(&c, 0, sizeof(c));
    c.round = 1;
    c.status = kDone;
    c.stop_round = 0xFFFFFFFFu;
    c.round_limit = round_limit;
    c.ninst = ninst;
    *ctl = c;
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

// Output of one query (Sec. I: cost[x]; parents as in Sec. I's remark on
// backward parent pointers).
// The lower bounds after the query's last round r sit in cf[(r + 1) & 1].
__global__ void k_finalize(const VRec* rec, u64 base, u32 n, u32 vbits, const InstVar* iv,
                           u64* dist, u32* parent, int* fround, u64* lower) {
    const u64 vmask = (vbits >= 64) ? ~0ull : ((1ull << vbits) - 1);
    const u32 cslot = (iv->start_round + iv->rounds) & 1u;
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        const VRec r = rec[base + v];
        const bool reach = r.dp != kInf64;
        if (dist) dist[v] = reach ? (r.dp >> vbits) : kInf64;
        if (parent) parent[v] = reach ? (u32)(r.dp & vmask) : kFull;
        if (fround) fround[v] = r.fround;
        if (lower) lower[v] = r.cf[cslot] & kCMask;
    }
}

// Distances of every query of a multi-query context into one staging array
// laid out like the records (entry g = record g).
__global__ void k_finalize_multi(RoundParams P, u64 nrec, u64* dist) {
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < nrec;
         g += (u64)gridDim.x * blockDim.x) {
        const u32 inst = P.page_owner[g >> P.page_shift];
        if (inst == kFull) continue;
        const u64 dp = P.rec[g].dp;
        dist[g] = (dp == kInf64) ? kInf64 : (dp >> P.vbits);
    }
}

// ----------------------------------------------------------- graph setup

__global__ void k_interleave(const u32* col, const u32* w, u64 m, uint2* adj) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < m;
         i += (u64)gridDim.x * blockDim.x)
        adj[i] = make_uint2(col[i], w[i]);
}

__global__ void k_count_in(const uint2* adj, u64 m, u64* cnt) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < m;
         i += (u64)gridDim.x * blockDim.x)
        atomicAdd(&cnt[adj[i].x], 1ull);
}

// One warp per source vertex scatters its out-edges into the in-lists.
__global__ void k_scatter_in(const u64* out_off, const uint2* out_adj, u32 n, u64* cursor,
                             uint2* in_adj) {
    const u32 lane = threadIdx.x & 31u;
    for (u64 u = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((u64)gridDim.x * blockDim.x) >> 5) {
        for (u64 k = out_off[u] + lane; k < out_off[u + 1]; k += 32) {
            const uint2 e = out_adj[k];
            const u64 pos = atomicAdd(&cursor[e.x], 1ull);
            in_adj[pos] = make_uint2((u32)u, e.y);
        }
    }
}

// outWeight[u] = min out-edge weight (computed once per graph, Sec. V).
__global__ void k_outw(const u64* out_off, const uint2* out_adj, u32 n, u32* outw) {
    const u32 lane = threadIdx.x & 31u;
    for (u64 u = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((u64)gridDim.x * blockDim.x) >> 5) {
        u32 m = kNoOutW;
        for (u64 k = out_off[u] + lane; k < out_off[u + 1]; k += 32) m = min(m, out_adj[k].y);
#pragma unroll
        for (u32 d = 16; d >= 1; d >>= 1) m = min(m, __shfl_xor_sync(kFull, m, d));
        if (lane == 0) outw[u] = m;
    }
}

// Vertices above the hub degree, by direction (list capacities).
__global__ void k_count_hubs(const u64* out_off, const u64* in_off, u32 n, u32 hub, u32* cnt) {
    u32 a = 0, b = 0;
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        a += (out_off[v + 1] - out_off[v]) > hub;
        b += (in_off[v + 1] - in_off[v]) > hub;
    }
    for (u32 d = 16; d >= 1; d >>= 1) {
        a += __shfl_xor_sync(kFull, a, d);
        b += __shfl_xor_sync(kFull, b, d);
    }
    if ((threadIdx.x & 31u) == 0) {
        if (a) atomicAdd(&cnt[0], a);
        if (b) atomicAdd(&cnt[1], b);
    }
}

// Exclusive scan of u64 counts, three passes (setup only).
constexpr u32 kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ u64 block_excl_scan(u64 x, u64* total) {
    __shared__ u64 s_warp[kScanThreads / 32];
    const u32 lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    u64 incl = x;
#pragma unroll
    for (u32 d = 1; d < 32; d <<= 1) {
        u64 y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        u64 s = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
        u64 si = s;
#pragma unroll
        for (u32 d = 1; d < 32; d <<= 1) {
            u64 y = __shfl_up_sync(kFull, si, d);
            if (lane >= d) si += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    const u64 res = s_warp[wid] + incl - x;
    __syncthreads();
    return res;
}

__global__ void k_scan_tiles(const u64* in, u64 cnt, u64* tile_sums) {
    __shared__ u64 s_tot;
    const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
    u64 s = 0;
    for (u32 i = 0; i < kScanItems; ++i)
        if (base + i < cnt) s += in[base + i];
    block_excl_scan(s, &s_tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s_tot;
}

__global__ void k_scan_sums(u64* tile_sums, u32 ntiles) {
    __shared__ u64 s_tot;
    u64 carry = 0;
    for (u32 base = 0; base < ntiles; base += kScanThreads) {
        const u32 i = base + threadIdx.x;
        const u64 x = (i < ntiles) ? tile_sums[i] : 0;
        const u64 ex = block_excl_scan(x, &s_tot);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += s_tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const u64* in, u64 cnt, const u64* tile_sums, u64* out) {
    __shared__ u64 s_tot;
    const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
    u64 v[kScanItems];
    u64 s = 0;
    for (u32 i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < cnt) ? in[base + i] : 0;
        s += v[i];
    }
    u64 run = tile_sums[blockIdx.x] + block_excl_scan(s, &s_tot);
    for (u32 i = 0; i < kScanItems; ++i) {
        if (base + i < cnt) out[base + i] = run;
        run += v[i];
    }
}

// Explicit instantiations used by the host engine.
template __global__ void k_relax<false>(RoundParams);
template __global__ void k_relax<true>(RoundParams);
template __global__ void k_cupdate<false>(RoundParams);
template __global__ void k_cupdate<true>(RoundParams);
template __global__ void k_start<false>(RoundParams, u32, u32, u32);
template __global__ void k_start<true>(RoundParams, u32, u32, u32);

}  // namespace sssp

// --------------------------------------------- host access for the engine

namespace sssp {

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
