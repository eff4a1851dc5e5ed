// Chunked single-problem pipeline, n = 8, m = 4: FP32, FP32 with FP64 tree
// levels, FP64.
#include "lqt_chain_impl.cuh"

namespace lqt {

const ChainVariant* chain_variants_n8(int* count) {
    static const ChainVariant v[] = {LQT_CHAIN_VARIANT(float, float, 8, 4),
                                     LQT_CHAIN_VARIANT(float, double, 8, 4),
                                     LQT_CHAIN_VARIANT(double, double, 8, 4)};
    *count = 3;
    return v;
}

}  // namespace lqt
