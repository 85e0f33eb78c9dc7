// sssp_round.cu -- the round kernels of sssp_round.cuh for the two state
// layouts, the per-query start kernel and the persistent kernel's barrier
// self-test, with the engine's access to them (kernel addresses, shared
// memory, occupancy, start launches).  The kernels with SP_1's predecessor
// counts come from sssp_round_pred.cu.
#include "sssp_round.cuh"

namespace sssp {

// Self-test of the barrier's wait limit: CTA `absent` never arrives, so the
// others must give up after P.barrier_ns, set ctl->error bit 4 and return.
__global__ void k_barrier_selftest(RoundParams P, u32 absent) {
    if (blockIdx.x == absent) return;
    grid_barrier(P, false, 0);
}

namespace {
const void* kernel_of(RoundKernel k, bool multi, bool narrow, bool pred) {
    return pred ? pred_round_kernel(k, multi, narrow)
                : round_kernel<WideL, NarrowL>(k, multi, narrow);
}
}  // namespace

const void* relax_fn(bool multi, bool narrow, bool pred) {
    return kernel_of(RoundKernel::kRelax, multi, narrow, pred);
}
const void* cupdate_fn(bool multi, bool narrow, bool pred) {
    return kernel_of(RoundKernel::kCupdate, multi, narrow, pred);
}
const void* solve_fn(bool multi, bool narrow, bool pred) {
    return kernel_of(RoundKernel::kSolve, multi, narrow, pred);
}
const void* tail_fn(bool multi, bool narrow, bool pred) {
    return kernel_of(RoundKernel::kTail, multi, narrow, pred);
}
const void* barrier_selftest_fn() { return (const void*)k_barrier_selftest; }

// The counting layouts stage the same slots, so the sizes are the layout's.
size_t relax_smem_bytes(bool narrow) {
    return narrow ? relax_smem<NarrowL>() : relax_smem<WideL>();
}
size_t cupdate_smem_bytes(bool narrow) {
    return narrow ? cupdate_smem<NarrowL>() : cupdate_smem<WideL>();
}
size_t solve_smem_bytes(bool narrow) {
    const size_t a = relax_smem_bytes(narrow), b = cupdate_smem_bytes(narrow);
    return a > b ? a : b;
}

cudaError_t launch_start(bool multi, bool narrow, const RoundParams& P, u32 first, u32 count,
                         u32 max_rounds, cudaStream_t st, u32 target) {
    if (multi) {
        if (narrow) k_start<true, NarrowL><<<1, 256, 0, st>>>(P, first, count, max_rounds, target);
        else k_start<true, WideL><<<1, 256, 0, st>>>(P, first, count, max_rounds, target);
    } else {
        if (narrow) k_start<false, NarrowL><<<1, 32, 0, st>>>(P, first, count, max_rounds, target);
        else k_start<false, WideL><<<1, 32, 0, st>>>(P, first, count, max_rounds, target);
    }
    return cudaGetLastError();
}

namespace {
// Raises the dynamic shared-memory limit of the four round kernels of one
// family (default or counting) and allows the tail kernel's 16-CTA cluster.
cudaError_t set_attributes(bool pred) {
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
        const bool multi = v & 1, narrow = (v >> 1) & 1;
        e = cudaFuncSetAttribute(relax_fn(multi, narrow, pred),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)relax_smem_bytes(narrow));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cupdate_fn(multi, narrow, pred),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cupdate_smem_bytes(narrow));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(solve_fn(multi, narrow, pred),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)solve_smem_bytes(narrow));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tail_fn(multi, narrow, pred),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)solve_smem_bytes(narrow));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tail_fn(multi, narrow, pred),
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    return e;
}

int blocks_per_sm(RoundKernel k, bool multi, bool narrow, bool pred, int threads,
                  size_t smem) {
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kernel_of(k, multi, narrow, pred),
                                                      threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return a;
}

int clusters_per_gpu(bool multi, bool narrow, bool pred) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kTailCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kTailCTAs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = solve_smem_bytes(narrow);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tail_fn(multi, narrow, pred), &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}
}  // namespace

// The default kernels' attributes (every call; cheap).  The counting kernels
// are left alone here: touching them loads their module, and a module loaded
// before a graph's buffers moves where those buffers land, which changes the
// latency-bound rounds of some workloads by up to 14%.
cudaError_t round_kernels_init() { return set_attributes(false); }

// The counting kernels, set up when a graph with SSSP_RULE_PRED_COUNT is
// created.  They are compiled with the default kernels' launch bounds and
// stage the same shared memory, so the occupancy-derived grids and the tail
// cluster of the default kernels fit them; checked here all the same.
cudaError_t pred_kernels_init() {
    cudaError_t e = set_attributes(true);
    if (e != cudaSuccess) return e;
    for (int v = 0; v < 4; ++v) {
        const bool multi = v & 1, narrow = (v >> 1) & 1;
        const RoundKernel ks[3] = {RoundKernel::kRelax, RoundKernel::kCupdate,
                                   RoundKernel::kSolve};
        const size_t sm[3] = {relax_smem_bytes(narrow), cupdate_smem_bytes(narrow),
                              solve_smem_bytes(narrow)};
        for (int i = 0; i < 3; ++i)
            if (blocks_per_sm(ks[i], multi, narrow, true, 256, sm[i]) <
                blocks_per_sm(ks[i], multi, narrow, false, 256, sm[i]))
                return cudaErrorInvalidConfiguration;
        if (clusters_per_gpu(multi, narrow, true) < clusters_per_gpu(multi, narrow, false))
            return cudaErrorInvalidConfiguration;
    }
    return cudaSuccess;
}

// CTAs of the tail kernel's cluster, or 0 when such a cluster cannot be
// scheduled on the current device (the device loop then runs without it).
u32 tail_cluster_ctas() {
    if (round_kernels_init() != cudaSuccess) return 0;
    for (int v = 0; v < 4; ++v)
        if (clusters_per_gpu(v & 1, (v >> 1) & 1, false) < 1) return 0;
    return kTailCTAs;
}

namespace {
// Fewest co-resident CTAs per SM over the default variants of one round
// kernel (the counting variants match them: pred_kernels_init).
int min_blocks_per_sm(RoundKernel k, int threads, size_t (*smem)(bool)) {
    if (round_kernels_init() != cudaSuccess) return 1;
    int best = 1 << 30;
    for (int v = 0; v < 4; ++v) {
        const bool multi = v & 1, narrow = (v >> 1) & 1;
        const int a = blocks_per_sm(k, multi, narrow, false, threads, smem(narrow));
        best = a < best ? a : best;
    }
    return best;
}
}  // namespace

// CTAs per SM of the relax kernel (every variant fits), and of the
// lower-bound kernel, which is compiled for more CTAs per SM.
int round_blocks_per_sm(int threads) {
    return min_blocks_per_sm(RoundKernel::kRelax, threads, relax_smem_bytes);
}
int cupdate_blocks_per_sm(int threads) {
    return min_blocks_per_sm(RoundKernel::kCupdate, threads, cupdate_smem_bytes);
}

// Co-resident CTAs per SM of the persistent kernel (its grid must fit).
int solve_blocks_per_sm(int threads) {
    return min_blocks_per_sm(RoundKernel::kSolve, threads, solve_smem_bytes);
}

}  // namespace sssp
