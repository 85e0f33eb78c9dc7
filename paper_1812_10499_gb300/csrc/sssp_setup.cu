// sssp_setup.cu -- per-query start/output kernels and per-graph setup
// kernels (CSC transpose, outWeight, hub counts) of the GB300 bound-based
// SSSP library (Garg, arXiv 1812.10499).
#include "sssp_dev.cuh"

namespace sssp {

namespace {
constexpr u32 kFull = 0xFFFFFFFFu;
__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
}  // namespace

// ------------------------------------------------------- start / finalize

// Every record of a single query: D = inf, C = 0 (Fig. SP_4 declarations).
// Exactly one of rec (32-byte records) and recn (16-byte records) is set.
// gf (nullable, compact layout): the relaxation filter words, from the
// packed outWeight words outw_pack.  pcnt (nullable): SP_1's predecessor
// counts, each vertex's in-degree (Fig. SP_1 declarations).
__global__ void k_init_records(VRec* rec, VRecN* recn, int* fround, const u32* outw,
                               const u64* in_off, u32 n, u32* chg, uint2* gf,
                               const u32* outw_pack, u32* pcnt) {
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        if (recn) {
            VRecN r;
            r.dp = kInf64;
            r.cf[0] = 0;
            r.cf[1] = 0;
            recn[v] = r;
            if (gf) gf[v] = make_uint2(kRelaxUnseen, outw_pack[v]);
        } else {
            VRec r;
            r.dp = kInf64;
            r.cf[0] = 0;
            r.cf[1] = 0;
            r.outw = outw[v];
            r.indeg = (u32)(in_off[v + 1] - in_off[v]);
            rec[v] = r;
        }
        fround[v] = -1;
        if (chg) chg[v] = 0;     // label-correcting change marks (rounds start at 1)
        if (pcnt) pcnt[v] = (u32)(in_off[v + 1] - in_off[v]);
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
        if (P.recn) {
            VRecN r;
            r.dp = kInf64;
            r.cf[0] = 0;
            r.cf[1] = 0;
            P.recn[g] = r;
            if (P.gf) P.gf[g] = make_uint2(kRelaxUnseen, d.outw[v]);
        } else {
            VRec r;
            r.dp = kInf64;
            r.cf[0] = 0;
            r.cf[1] = 0;
            r.outw = d.outw[v];
            r.indeg = (u32)(d.in_off[v + 1] - d.in_off[v]);
            P.rec[g] = r;
        }
        P.fround[g] = -1;
        if (P.chg) P.chg[g] = 0;
        if (P.pcnt) P.pcnt[g] = (u32)(d.in_off[v + 1] - d.in_off[v]);
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

// Output of one query (Sec. I: cost[x]; parents as in Sec. I's remark on
// backward parent pointers).  Exactly one of rec and recn is set.
// The lower bounds after the query's last round r sit in cf[(r + 1) & 1].
__global__ void k_finalize(const VRec* rec, const VRecN* recn, const int* frec, u64 base, u32 n,
                           u32 vbits, const InstVar* iv, u64* dist, u32* parent, int* fround,
                           u64* lower) {
    const u64 vmask = (vbits >= 64) ? ~0ull : ((1ull << vbits) - 1);
    const u32 cslot = (iv->start_round + iv->rounds) & 1u;
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        u64 dp, c;
        if (recn) {
            const VRecN r = recn[base + v];
            dp = r.dp;
            c = (cslot ? r.cf[1] : r.cf[0]) & ~kFixedN;
        } else {
            const VRec r = rec[base + v];
            dp = r.dp;
            c = (cslot ? r.cf[1] : r.cf[0]) & kCMask;
        }
        const bool reach = dp != kInf64;
        if (dist) dist[v] = reach ? (dp >> vbits) : kInf64;
        if (parent) parent[v] = reach ? (u32)(dp & vmask) : kFull;
        if (fround) fround[v] = frec[base + v];
        if (lower) lower[v] = c;
    }
}

// Distances of every query of a multi-query context into one staging array
// laid out like the records (entry g = record g).
__global__ void k_finalize_multi(RoundParams P, u64 nrec, u64* dist) {
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < nrec;
         g += (u64)gridDim.x * blockDim.x) {
        const u32 inst = P.page_owner[g >> P.page_shift];
        if (inst == kFull) continue;
        const u64 dp = P.recn ? P.recn[g].dp : P.rec[g].dp;
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

// outWeight word of the compact layout: the minimum out-weight (below 2^31
// there; 2^31 - 1 when the vertex has no out-edge) with bit 31 set when the
// in-degree is above the hub degree.  May run in place (out == outw).
__global__ void k_pack_outw(const u32* outw, const u64* in_off, u32 n, u32 hub, u32* out) {
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        const u32 ow = outw[v];
        const u32 lo = ow == kNoOutW ? (kFixedN - 1) : ow;
        out[v] = lo | ((in_off[v + 1] - in_off[v] > hub) ? kFixedN : 0u);
    }
}

// Vertices above the hub degree, by direction (list capacities), and the
// largest out- and in-degree (cnt[2], cnt[3]; clamped to 2^32 - 1).
__global__ void k_count_hubs(const u64* out_off, const u64* in_off, u32 n, u32 hub, u32* cnt) {
    u32 a = 0, b = 0;
    u64 mo = 0, mi = 0;
    for (u64 v = blockIdx.x * (u64)blockDim.x + threadIdx.x; v < n;
         v += (u64)gridDim.x * blockDim.x) {
        const u64 od = out_off[v + 1] - out_off[v], id = in_off[v + 1] - in_off[v];
        a += od > hub;
        b += id > hub;
        mo = od > mo ? od : mo;
        mi = id > mi ? id : mi;
    }
    u32 mo32 = (u32)(mo > 0xFFFFFFFFull ? 0xFFFFFFFFull : mo);
    u32 mi32 = (u32)(mi > 0xFFFFFFFFull ? 0xFFFFFFFFull : mi);
    for (u32 d = 16; d >= 1; d >>= 1) {
        a += __shfl_xor_sync(kFull, a, d);
        b += __shfl_xor_sync(kFull, b, d);
        mo32 = max(mo32, __shfl_xor_sync(kFull, mo32, d));
        mi32 = max(mi32, __shfl_xor_sync(kFull, mi32, d));
    }
    if ((threadIdx.x & 31u) == 0) {
        if (a) atomicAdd(&cnt[0], a);
        if (b) atomicAdd(&cnt[1], b);
        if (mo32) atomicMax(&cnt[2], mo32);
        if (mi32) atomicMax(&cnt[3], mi32);
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

// ------------------------------------------------- control-block placement

// Round-trip time, in SM cycles, of a chain of 16 dependent atomics on each
// of nslots candidate words (stride_words apart), the least of three passes
// after one warming pass, from one thread of CTA 0.  Launched like the tail
// kernel (one cluster of its CTAs), so the thread runs where the tail
// kernel's CTA 0 will: the words the tail kernel's rounds wait on (list
// counters, round minima) go in the fastest slot.  Writes cycles[0, nslots);
// the candidate words are left changed (they are reset before any solve).
__global__ void k_place_probe(u32* base, u32 nslots, u32 stride_words,
                              unsigned long long* cycles) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    u32 x = 0;
    for (u32 s = 0; s < nslots; ++s) x = atomicAdd(base + (size_t)s * stride_words, x >> 31);
    for (u32 s = 0; s < nslots; ++s) cycles[s] = ~0ull;
    for (u32 pass = 0; pass < 3; ++pass)
        for (u32 s = 0; s < nslots; ++s) {
            u32* p = base + (size_t)s * stride_words;
            const long long t0 = clock64();
            // Each atomic's operand depends on the previous one's result.
            for (int i = 0; i < 16; ++i) x = atomicAdd(p, x >> 31);
            const unsigned long long dt = (unsigned long long)(clock64() - t0) + (x >> 31);
            if (dt < cycles[s]) cycles[s] = dt;
        }
}

cudaError_t launch_place_probe(u32* base, u32 nslots, u32 stride_words, unsigned long long* cycles,
                               u32 cluster_ctas, size_t smem, cudaStream_t st) {
    if (cluster_ctas == 0) {
        k_place_probe<<<1, 32, 0, st>>>(base, nslots, stride_words, cycles);
        return cudaGetLastError();
    }
    cudaError_t e =
        cudaFuncSetAttribute(k_place_probe, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_place_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster_ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cluster_ctas);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_place_probe, base, nslots, stride_words, cycles);
}

}  // namespace sssp
