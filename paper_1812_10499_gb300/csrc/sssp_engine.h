// sssp_engine.h -- host-side structures shared by the engine translation
// units (sssp_api.cu: graphs, single and batched solves; sssp_serve.cu:
// continuous-batching server).  Internal; not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sssp.h"
#include "sssp_dev.cuh"

namespace sssp {
// narrow: 16-byte records (RoundParams::recn) instead of 32-byte ones (rec);
// pred: the kernels with SP_1's predecessor counts (RoundParams::pcnt set).
const void* relax_fn(bool multi, bool narrow, bool pred);
const void* cupdate_fn(bool multi, bool narrow, bool pred);
const void* solve_fn(bool multi, bool narrow, bool pred);
const void* tail_fn(bool multi, bool narrow, bool pred);
const void* barrier_selftest_fn();
u32 tail_cluster_ctas();
size_t solve_smem_bytes(bool narrow);
int solve_blocks_per_sm(int threads);
size_t relax_smem_bytes(bool narrow);
size_t cupdate_smem_bytes(bool narrow);
cudaError_t round_kernels_init();
cudaError_t pred_kernels_init();   // before the first graph with SSSP_RULE_PRED_COUNT
cudaError_t launch_start(bool multi, bool narrow, const RoundParams& P, u32 first, u32 count,
                         u32 max_rounds, cudaStream_t st, u32 target = kNoTarget);
int round_blocks_per_sm(int threads);
int cupdate_blocks_per_sm(int threads);
__global__ void k_init_records(VRec* rec, VRecN* recn, int* fround, const u32* outw,
                               const u64* in_off, u32 n, u32* chg = nullptr,
                               uint2* gf = nullptr, const u32* outw_pack = nullptr,
                               u32* pcnt = nullptr);
__global__ void k_init_records_multi(RoundParams P, u64 nrec, u32 first_page, u32 npages);
__global__ void k_reset_ctl(Ctl* ctl, u32 ninst, u32 round_limit);
__global__ void k_finalize(const VRec* rec, const VRecN* recn, const int* frec, u64 base, u32 n,
                           u32 vbits, const InstVar* iv, u64* dist, u32* parent, int* fround,
                           u64* lower);
__global__ void k_finalize_multi(RoundParams P, u64 nrec, u64* dist);
__global__ void k_interleave(const u32* col, const u32* w, u64 m, uint2* adj);
__global__ void k_count_in(const uint2* adj, u64 m, u64* cnt);
__global__ void k_scatter_in(const u64* out_off, const uint2* out_adj, u32 n, u64* cursor,
                             uint2* in_adj);
__global__ void k_outw(const u64* out_off, const uint2* out_adj, u32 n, u32* outw);
__global__ void k_pack_outw(const u32* outw, const u64* in_off, u32 n, u32 hub, u32* out);
__global__ void k_count_hubs(const u64* out_off, const u64* in_off, u32 n, u32 hub, u32* cnt);
__global__ void k_scan_tiles(const u64* in, u64 cnt, u64* tile_sums);
__global__ void k_scan_sums(u64* tile_sums, u32 ntiles);
__global__ void k_scan_apply(const u64* in, u64 cnt, const u64* tile_sums, u64* out);
constexpr u32 kScanTile = 2048;
cudaError_t launch_place_probe(u32* base, u32 nslots, u32 stride_words, unsigned long long* cycles,
                               u32 cluster_ctas, size_t smem, cudaStream_t st);
}  // namespace sssp

namespace sssp {
namespace engine {

constexpr u32 kThreads = 256;
constexpr u32 kPageShift = 10;
constexpr u32 kDefaultHub = 256;
constexpr u32 kDefaultChunk = 1024;
constexpr u32 kDefaultTailItems = 512;

#define CK(call)                                       \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            (void)cudaGetLastError();                  \
            return SSSP_E_CUDA;                        \
        }                                              \
    } while (0)

#define RC(call)                      \
    do {                              \
        int r_ = (call);              \
        if (r_ != SSSP_OK) return r_; \
    } while (0)

struct Allocator {
    sssp_alloc_fn fa = nullptr;
    sssp_free_fn ff = nullptr;
    void* ctx = nullptr;
    void* get(size_t bytes) {
        if (bytes == 0) bytes = 256;
        if (fa) return fa(bytes, ctx);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void* p) {
        if (!p) return;
        if (ff) ff(p, ctx);
        else cudaFree(p);
    }
};

// Device allocations of one owner, released together.
struct Pool {
    Allocator al;
    std::vector<void*> ptrs;
    template <class T>
    int get(T** out, size_t count) {
        void* p = al.get(count * sizeof(T));
        if (!p) return SSSP_E_NOMEM;
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return SSSP_OK;
    }
    void release() {
        for (void* p : ptrs) al.put(p);
        ptrs.clear();
    }
};

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (dev != prev_) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev_); }

   private:
    int prev_ = 0;
};

inline u32 bits_for(u64 x) {
    u32 b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

// Solve context: records, work lists, control block, per-query scalars and
// the instantiated round loop.
struct Context {
    Pool pool;
    bool multi = false;
    bool narrow = false;     // 16-byte records (P.recn) in use
    u64 nrec = 0;            // records
    u32 nslots = 0;          // query slots
    u32 npages = 0;
    u32 capH = 0;
    RoundParams P{};
    VRec* rec_store = nullptr;  // record storage of a multi-query context (either layout)
    u64* stage = nullptr;    // device staging (distances)
    Ctl* h_ctl = nullptr;    // pinned
    InstVar* h_ivar = nullptr;
    InstDesc* h_desc = nullptr;
    u32* h_pages = nullptr;
    u64* h_stage = nullptr;  // pinned staging for multi-query host outputs
    u64 h_stage_n = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
    int grid_solve = 0;              // co-resident grid of the persistent kernel
    int grid_cup = 0;                // grid of the lower-bound kernel
    u32 tail_ctas = 0;               // cluster size of the tail kernel, 0 = not in the loop
    u32 last_loop = 0;               // loop mode of the last run_loop
    u32 launches_per_iter = 0;       // round kernels per loop iteration in that mode
    // Per-kernel event timing (sssp_profile).
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    u64 prof_relax_n = 0, prof_cup_n = 0, prof_tail_n = 0, prof_tail_rounds = 0;
    double prof_relax_ms = 0, prof_cup_ms = 0, prof_tail_ms = 0;
    u64 prof_grid_ctr[4] = {}, prof_tail_ctr[4] = {};      // counters by kernel (see sssp.h)
    // Last profiled solve, one entry per loop iteration (host-launched rounds:
    // one round each).
    std::vector<float> prof_round_relax, prof_round_cup, prof_round_tail;
    std::vector<u32> prof_round_tail_rounds;
    std::vector<u64> prof_round_ctr;   // per iteration: the 4 work counters of k_relax +
                                       // k_cupdate (device-loop schedule; 0 otherwise)
    Ctl* h_snap = nullptr;           // pinned control-block snapshots (graph-schedule profile)
    cudaAccessPolicyWindow l2win{};  // L2 window over the records (num_bytes 0: none)
    u64* trace = nullptr;            // device trace of the persistent kernel
    u32 trace_cap = 0;
    int hot_slot = -1;               // slot of the control block in its probed region

    void destroy() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_ivar) cudaFreeHost(h_ivar);
        if (h_desc) cudaFreeHost(h_desc);
        if (h_pages) cudaFreeHost(h_pages);
        if (h_stage) cudaFreeHost(h_stage);
        if (h_snap) cudaFreeHost(h_snap);
        h_snap = nullptr;
        h_ctl = nullptr;
        h_ivar = nullptr;
        h_desc = nullptr;
        h_pages = nullptr;
        h_stage = nullptr;
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        pool.release();
    }
};

}  // namespace engine
}  // namespace sssp

struct sssp_graph {
    typedef sssp::u32 u32;
    typedef sssp::u64 u64;
    int device = 0;
    u32 n = 0;
    u64 m = 0;
    u32 vbits = 1;
    u64 dinf = 0;
    u32 wmax = 0;
    bool narrow = false;             // compact 16-byte records
    u32 hubs_out = 0, hubs_in = 0;
    sssp_options opt{};
    sssp::engine::Pool gpool;        // graph arrays
    u64* out_off = nullptr;
    uint2* out_adj = nullptr;
    u64* in_off = nullptr;
    uint2* in_adj = nullptr;
    u32* outw = nullptr;
    u32* outw_pack = nullptr;        // compact layout: outWeight | in-hub flag (k_pack_outw)
    u32* inw = nullptr;              // inWeight: min in-edge weight (kNoOutW: none)
    cudaStream_t stream = nullptr;   // internal stream for setup and host-pointer solves
    int grid = 0;
    int grid_solve = 0;
    int grid_cup = 0;
    u32 tail_ctas = 0;               // see Context::tail_ctas
    u32 tail_items = 0;
    u32 max_out = 0, max_in = 0;     // largest out- / in-degree (the graph's class)
    bool tune_auto = false;          // the options left the tuning to the library
    sssp::engine::Context single;    // single-query context
    sssp::engine::Context* batch = nullptr;  // multi-query context (grown on demand)
    std::mutex mu;
};


namespace sssp {
namespace engine {
int count_hubs(sssp_graph* h, u32 hub, u32* hubs_out, u32* hubs_in, u32* max_out, u32* max_in);
int apply_tuning(sssp_graph* h);
void resolve_tuning(sssp_graph* h);
int enqueue_single(sssp_graph* h, u32 source, u32 max_rounds, cudaStream_t st, u64* dist_dev,
                   u32* parent_dev, int* fround_dev, u64* lower_dev, u32 target);
int batch_impl(const sssp_handle* g, const u32* sources, u32 k, u64* const* dist, bool dev,
               u32* rounds_out, cudaStream_t st_user, bool use_user_stream,
               const sssp_tuning* tune);
int occupancy_grid(int device, const sssp_options& o, bool cupdate = false);
// Tuning cache (sssp_tune.cu): the class key of a graph / a batch and the
// process-wide cache of tunings by key.
void graph_key(const sssp_graph* h, char* buf, size_t cap);
void batch_key(const sssp_handle* g, u32 k, char* buf, size_t cap);
int tune_cache_find(const char* key, sssp_tuning* out);
int build_loop(Context& c);
int run_loop(Context& c, u32 loop_mode, cudaStream_t st);
int alloc_lists(Context& c, u64 capS, u64 capH, u64 capC);
int alloc_hot(Context& c, u32 nivar, cudaStream_t st);
int alloc_pinned(Context& c, u32 slots);
void set_l2_window(Context& c, int device);
bool records_fit_l2(size_t bytes, int device);
}  // namespace engine
}  // namespace sssp
