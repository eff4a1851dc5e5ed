// Chunked single-problem pipeline, n = 4, m = 2: FP32, FP32 with FP64 tree
// levels, FP64.  At n <= 4 lqt_solve runs the thread-per-step kernels; this
// variant serves the options those kernels do not have (Method 2, and the
// FULL refinement with its Newton step for S, v, K).
#include "lqt_chain_impl.cuh"

namespace lqt {

const ChainVariant* chain_variants_n4(int* count) {
    static const ChainVariant v[] = {LQT_CHAIN_VARIANT(float, float, 4, 2),
                                     LQT_CHAIN_VARIANT(float, double, 4, 2),
                                     LQT_CHAIN_VARIANT(double, double, 4, 2)};
    *count = 3;
    return v;
}

}  // namespace lqt
