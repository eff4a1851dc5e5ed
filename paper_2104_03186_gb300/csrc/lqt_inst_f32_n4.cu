// Kernel instantiations: LQT_VARIANTS_F32_N4 of lqt_variants.h.
#include "lqt_launch_impl.cuh"
#include "lqt_variants.h"

namespace lqt {
LQT_VARIANTS_F32_N4(LQT_INSTANTIATE)
}  // namespace lqt
