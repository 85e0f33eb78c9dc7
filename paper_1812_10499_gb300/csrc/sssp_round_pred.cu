// sssp_round_pred.cu -- the round kernels of sssp_round.cuh for the two state
// layouts with SP_1's predecessor counts (Sec. III; SSSP_RULE_PRED_COUNT).
// A translation unit of their own, so that they compile alongside the default
// kernels (sssp_round.cu) instead of after them.
#include "sssp_round.cuh"

namespace sssp {

const void* pred_round_kernel(RoundKernel k, bool multi, bool narrow) {
    return round_kernel<PredL<WideL>, PredL<NarrowL>>(k, multi, narrow);
}

}  // namespace sssp
