// sssp_dev.cuh -- device-side data layout shared by the round kernels and the
// host engine of the GB300 bound-based SSSP library (Garg, arXiv 1812.10499).
//
// Per-query state lives in one 32-byte record per vertex (VRec), so the two
// random accesses of a round -- the relaxation of an out-edge (Sec. VI, SP_4
// step 3) and the lower-bound gather over an in-edge (Eq. 1) -- touch exactly
// one 32-byte DRAM sector each.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sssp {

typedef unsigned long long u64;
typedef unsigned int u32;

// Packed upper bound: D word = (dist << vbits) | parent.  Equal distances keep
// the smaller parent id (64-bit atomicMin).  All ones = infinity.
constexpr u64 kInf64 = ~0ull;
// Lower-bound words carry the "fixed" flag in bit 63 (C < 2^63 always).
constexpr u64 kFixed = 1ull << 63;
constexpr u64 kCMask = kFixed - 1;
constexpr u32 kNoOutW = 0xFFFFFFFFu;   // vertex without out-edges

// One vertex of one query.  cf[] is double-buffered by round parity: round r
// reads cf[r & 1] (the lower bounds before the round: Jacobi update, SP_4
// step 4 "in parallel") and writes cf[(r & 1) ^ 1].
struct __align__(32) VRec {
    u64 dp;        // packed upper bound D (atomicMin target)
    u64 cf[2];     // lower bound C | kFixed
    u32 outw;      // outWeight (Fig. SP_3 / SP_4 declarations), kNoOutW if none
    u32 indeg;     // in-degree (decides the work list of a newly discovered vertex)
};
static_assert(sizeof(VRec) == 32, "VRec must be one 32-byte sector");

// Compact record, used when every finite distance is below 2^31 (checked
// from n * max weight when the graph is created): C words are 31-bit values
// with the fixed flag in bit 31; outWeight and the in-degree are read from
// the graph when needed.  Two records share a 32-byte sector, so the state
// the gathers touch is half as large.
struct __align__(16) VRecN {
    u64 dp;        // packed upper bound D (atomicMin target)
    u32 cf[2];     // lower bound C | kFixedN, double-buffered by round parity
};
static_assert(sizeof(VRecN) == 16, "VRecN must be 16 bytes");
constexpr u32 kFixedN = 1u << 31;
constexpr u64 kNarrowLimit = kFixedN - 1;   // distances must stay below this
constexpr u32 kRelaxUnseen = 0x7FFFFFFFu;   // relaxation bound of an undiscovered vertex

// Read-only description of one query's graph.
struct InstDesc {
    const u64* out_off;     // CSR offsets, n + 1
    const uint2* out_adj;   // {target, weight}
    const u64* in_off;      // CSC offsets, n + 1
    const uint2* in_adj;    // {source, weight}
    const u32* outw;        // min out-weight per vertex
    const u32* inw;         // min in-weight per vertex (kNoOutW: none), for the cheap rules
    u64 base;               // global record index of local vertex 0
    u32 n;
    u32 source;
};

enum : u32 { kIdle = 0, kRunning = 1, kDone = 2, kStopped = 3, kErrRounds = 4 };

// Mutable per-query scalars; slot [r & 1] belongs to round r.
struct __align__(16) InstVar {
    u64 thr[2];         // threshold = min over unfixed discovered of D + outWeight (Lemma 8)
    u64 minD[2];        // min over unfixed discovered of D (Lemma 7)
    u32 nfix[2];        // vertices fixed in the round
    u32 start_round;    // engine round in which the query's round 1 runs
    u32 rounds;         // rounds executed (set when the query stops)
    u32 status;         // kIdle / kRunning / kDone / kStopped
    u32 max_rounds;     // stop after this many rounds (0 = unlimited)
    u32 target;         // single-target query: stop once this local vertex is fixed
};
constexpr u32 kNoTarget = 0xFFFFFFFFu;

// Engine control block (one per solve context).
struct __align__(16) Ctl {
    u32 round;          // next engine round to execute
    u32 status;         // kRunning while any query runs, kDone otherwise, kErrRounds
    u32 running;        // queries still running after the last round
    u32 stop_round;     // device loop stops after this round (serving steps)
    u32 round_limit;    // hard cap; exceeding it is an internal error
    u32 error;          // nonzero: a list capacity was exceeded (bug guard)
    u32 nFS[2];         // frontier, small-degree entries
    u32 nAS[2];         // active, small-degree entries
    u64 FHpk[2];        // frontier hubs: (entries << 32) | chunks
    u64 AHpk[2];        // active hubs: (entries << 32) | chunks
    u32 work[2];        // dynamic work counters of the two round kernels
    u32 done_ctas;      // arrival counter for the end-of-round epilogue
    u32 ninst;          // number of query slots
    u32 loop_iters;     // loop bodies started (watchdog against a stuck loop)
    u32 bar_count;      // grid barrier of the persistent kernel: arrivals
    u32 bar_gen;        // grid barrier generation (bumped on release)
    u32 tail_go;        // cluster tail kernel: run the next step (set before a cluster barrier)
    u32 cup_only;       // the round's relaxation is done (by the tail kernel): the next
                        // full-grid relax launch is skipped
    u32 body_iters;     // launches of the relax kernel (one per loop iteration)
    u32 nFX[2];         // label-correcting: vertices fixed in the round (see Lists::FX)

    u64 stats[5];       // out-edges scanned, in-edges scanned, active visits, frontier
                        // visits, vertices fixed (single query)
};

// Work lists.  Small-degree vertices are processed 32 per warp with a
// warp-local load balance; vertices above the hub degree are split into
// chunks of `chunk` edges handled by many warps.
struct Lists {
    u32* FS[2];
    uint2* FH[2];   // {record index, first chunk}
    u32* AS[2];
    uint2* AH[2];
    u64* hubmin;    // per active-hub entry: running min of Eq. (1) terms
    u32* hubcnt;    // per active-hub entry: chunks finished
    u32* FX[2];     // label-correcting: vertices fixed in the round.  Their lower-bound
                    // word is fixed in one parity slot only; the next round's
                    // relaxation phase copies it to the other (in label-setting mode
                    // the frontier, which is these vertices, does it)
    u32* FC[2];     // chunk -> FH entry, written with the entry (chunks below capC)
    u32* AC[2];     // chunk -> AH entry
    u32 capS, capH; // capacities of the small and hub lists
    u32 capC;       // capacity of the chunk maps (chunks beyond it are found by search)
    u32 pad;
};

struct RoundParams {
    InstDesc g;                 // the graph when a single query runs
    const InstDesc* idesc;      // per-slot graphs (multi-query)
    InstVar* ivar;              // per-slot scalars
    const u32* page_owner;      // record page -> slot (multi-query)
    VRec* rec;                  // wide records (or nullptr)
    VRecN* recn;                // compact records (or nullptr)
    uint2* gf;                  // compact layout, label-setting rounds (or nullptr): per
                                // record {relaxation bound, outWeight word}.  The bound is
                                // 0 once the vertex is fixed, else at least its distance
                                // (kRelaxUnseen before it is discovered); the second word
                                // is its graph's outWeight | in-hub flag.  The relaxation
                                // filters its candidates with it instead of the record.
    int* fround;                // per record: round in which it was fixed, -1 if never
    Ctl* ctl;
    Lists L;
    u64 dinf;                   // distance infinity = 2^(64 - vbits) - 1
    u32 vbits;                  // parent bits of the packed D word
    u32 hub;                    // hub degree threshold
    u32 chunk;                  // edges per hub chunk
    u32 rule;                   // 0: min(D, threshold) clamp; 1: minD clamp
    u32 page_shift;
    u32 trace_cap;              // entries of `trace`
    u32 trace_base;             // round number of the first traced round
    u32 tail_items;             // cluster tail kernel: most work items a round may have
    u32 lc;                     // 1: label-correcting relaxation (SP_4 step 3 as printed):
                                // the frontier is every vertex whose D changed in the
                                // previous round's relaxation
    u32 cheap;                  // 1: fix y without scanning its in-edges when
                                // D[y] <= minD + inWeight[y] or D[y] <= threshold
    u32* pcnt;                  // SP_1's predecessor counts (nullable): per record, the
                                // in-edges not yet relaxed; an active y at 0 is fixed
                                // without scanning its in-edges
    u32 win;                    // 1: windowed relaxation (Delta-stepping's bucket as a
                                // window over D): an active vertex whose D changed since
                                // it last relaxed relaxes while D < minD + delta
    u64 delta;                  // the window's width (windowed relaxation)
    unsigned long long* snap;   // label-correcting / windowed: distance of each frontier
                                // vertex at the start of the relaxation (written the round
                                // before)
    u32* chg;                   // label-correcting: last round in which D changed;
                                // windowed: nonzero while D changed since the last relaxation
    unsigned long long cond;    // cudaGraphConditionalHandle of the device loop, 0 = none
    unsigned long long barrier_ns;  // wait limit of the persistent kernel's grid barrier
                                    // (0 = the default, 20 s)
    u64* trace;                 // persistent kernel: globaltimer at launch, then at the end of
                                // every phase (2 per round); nullable
};

}  // namespace sssp
