// sssp_noalloc.cu -- a single-source solve that allocates no memory.
//
// Some callers cannot allocate device memory at solve time: code that runs
// inside another framework's memory pool (which owns all device memory and
// forbids cudaMalloc), services whose device-memory budget is fixed when
// they start, and latency-critical loops where a cudaMalloc / cudaFree would
// synchronise the device and stall other streams.  sssp_solve_noalloc
// serves them: the caller passes the graph (already in device memory) and
// the output buffer, and every piece of working state -- per-vertex records,
// work lists, control block -- lives in one fixed file-scope device array.
// The array is part of the library image, so every GPU that loads the
// library holds it (kNoAllocBytes) until the process exits.
#include <mutex>

#include "sssp_engine.h"

using namespace sssp;
using namespace sssp::engine;

namespace {

// Largest graph the fixed scratch holds, and the scratch size.  Per vertex:
// 32 B record, 4 B fixing round, 4 B outWeight, 4 x 4 B small lists,
// 4 x 8 B hub lists, 8 B + 4 B hub reduction slots = 100 B.
constexpr u32 kNoAllocMaxVertices = SSSP_NOALLOC_MAX_VERTICES;
constexpr size_t kPerVertex = 100;
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxVertices * kPerVertex + 64 * 1024;

// The scratch.  Host code must not use this name as an address (it is a
// host-side shadow); it takes the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};
int g_grid[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch, the round kernels' shared-memory limit and the persistent grid.
int setup_device(int dev, unsigned char** scratch, int* grid) {
    if (dev < 0 || dev >= kMaxDevices) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        CK(round_kernels_init());
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        g_grid[dev] = std::max(1, sms) * std::max(1, solve_blocks_per_sm(kThreads));
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *scratch = g_scratch_dev[dev];
    *grid = g_grid[dev];
    return SSSP_OK;
}

// Carves `count` objects of T, aligned to 256 bytes, from the scratch.
template <class T>
T* carve(unsigned char* base, size_t& off, size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
}

}  // namespace

extern "C" int sssp_solve_noalloc(uint32_t n, const uint64_t* out_off, const uint32_t* out_adj,
                                  const uint64_t* in_off, const uint32_t* in_adj, uint32_t source,
                                  uint32_t max_weight, uint64_t* dist_dev, uint32_t* rounds_out,
                                  void* cuda_stream) {
    if (n == 0 || !out_off || !in_off || !dist_dev) return SSSP_E_INVAL;
    if (n > kNoAllocMaxVertices) return SSSP_E_NOALLOC_LIMIT;
    if (source >= n) return SSSP_E_SOURCE_RANGE;
    // Compact 16-byte records when every finite distance fits 31 bits; their
    // kernels keep the distance in the upper half of the packed D word.
    const bool narrow = (unsigned __int128)n * max_weight < kNarrowLimit;
    const u32 vbits = narrow ? 32u : std::max<u32>(1, bits_for((u64)n - 1));
    const u64 dinf = (~0ull) >> vbits;
    if ((unsigned __int128)n * max_weight >= (unsigned __int128)dinf) return SSSP_E_OVERFLOW;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    int grid = 0;
    RC(setup_device(dev, &base, &grid));
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // Lay the working state out in the scratch (no allocation).
    size_t off = 0;
    RoundParams P{};
    if (narrow) P.recn = carve<VRecN>(base, off, n);
    else P.rec = carve<VRec>(base, off, n);
    P.fround = carve<int>(base, off, n);
    u32* outw = carve<u32>(base, off, n);
    for (int i = 0; i < 2; ++i) {
        P.L.FS[i] = carve<u32>(base, off, n);
        P.L.AS[i] = carve<u32>(base, off, n);
        P.L.FH[i] = carve<uint2>(base, off, n);
        P.L.AH[i] = carve<uint2>(base, off, n);
    }
    P.L.hubmin = carve<u64>(base, off, n);
    P.L.hubcnt = carve<u32>(base, off, n);
    P.ctl = carve<Ctl>(base, off, 1);
    P.ivar = carve<InstVar>(base, off, 1);
    if (off > kNoAllocBytes) return SSSP_E_INTERNAL;
    P.L.capS = n;
    P.L.capH = n;
    P.L.capC = 0;   // no chunk maps here: hub chunks find their vertex by search
    P.g = InstDesc{reinterpret_cast<const u64*>(out_off), reinterpret_cast<const uint2*>(out_adj),
                   reinterpret_cast<const u64*>(in_off), reinterpret_cast<const uint2*>(in_adj),
                   outw, nullptr, 0, n, source};
    P.dinf = dinf;
    P.vbits = vbits;
    P.hub = kDefaultHub;
    P.chunk = kDefaultChunk;
    P.rule = SSSP_RULE_THRESHOLD;
    P.page_shift = kPageShift;

    // Every call starts from cleared state: the scratch keeps the previous
    // call's contents.  Hub reduction slots start at (infinity, 0).  Once the
    // first command is enqueued, a failure waits for the stream before it
    // returns, so no kernel of a failed call still uses the scratch.
    int rc = SSSP_OK;
    cudaError_t e = cudaMemsetAsync(P.L.hubmin, 0xFF, sizeof(u64) * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.L.hubcnt, 0, sizeof(u32) * n, st);
    if (e == cudaSuccess) {
        k_outw<<<grid, kThreads, 0, st>>>(P.g.out_off, P.g.out_adj, n, outw);
        if (narrow)   // compact kernels read outWeight with the in-hub flag (in place)
            k_pack_outw<<<grid, kThreads, 0, st>>>(outw, P.g.in_off, n, kDefaultHub, outw);
        k_init_records<<<grid, kThreads, 0, st>>>(P.rec, P.recn, P.fround, outw, P.g.in_off, n);
        k_reset_ctl<<<1, 32, 0, st>>>(P.ctl, 1, n + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_start(false, narrow, P, 0, 1, 0, st);
    if (e == cudaSuccess) {
        void* args[] = {&P};
        e = cudaLaunchCooperativeKernel(solve_fn(false, narrow, false), dim3(grid), dim3(kThreads), args,
                                        solve_smem_bytes(narrow), st);
    }
    if (e == cudaSuccess) {
        k_finalize<<<grid, kThreads, 0, st>>>(P.rec, P.recn, P.fround, 0, n, vbits, P.ivar,
                                              reinterpret_cast<u64*>(dist_dev), nullptr, nullptr,
                                              nullptr);
        e = cudaGetLastError();
    }
    // Status and round count into host stack memory.
    Ctl hc;
    InstVar hv;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hv, P.ivar, sizeof(InstVar), cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return SSSP_E_CUDA;
    }
    if (hc.error & 4u) rc = SSSP_E_DEVICE_TIMEOUT;
    else if (hc.error & 8u) rc = SSSP_E_OVERFLOW;   // a weight above max_weight
    else if (hc.error) rc = SSSP_E_INTERNAL;
    else if (hv.status != kDone) rc = SSSP_E_ROUND_LIMIT;
    if (rc != SSSP_OK) return rc;
    if (rounds_out) *rounds_out = hv.rounds;
    return SSSP_OK;
}
