// Chunked single-problem pipeline, n = 16, m = 8: FP32, FP32 with FP64 tree
// levels, FP64.
#include "lqt_chain_impl.cuh"

namespace lqt {

const ChainVariant* chain_variants_n16(int* count) {
    static const ChainVariant v[] = {LQT_CHAIN_VARIANT(float, float, 16, 8),
                                     LQT_CHAIN_VARIANT(float, double, 16, 8),
                                     LQT_CHAIN_VARIANT(double, double, 16, 8)};
    *count = 3;
    return v;
}

}  // namespace lqt
