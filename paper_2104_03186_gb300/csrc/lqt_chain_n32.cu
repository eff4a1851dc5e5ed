// Chunked single-problem pipeline, n = 32, m = 16: FP32, FP32 with FP64 tree
// levels, FP64.
#include "lqt_chain_impl.cuh"

namespace lqt {

const ChainVariant* chain_variants_n32(int* count) {
    static const ChainVariant v[] = {LQT_CHAIN_VARIANT(float, float, 32, 16),
                                     LQT_CHAIN_VARIANT(float, double, 32, 16),
                                     LQT_CHAIN_VARIANT(double, double, 32, 16)};
    *count = 3;
    return v;
}

}  // namespace lqt
