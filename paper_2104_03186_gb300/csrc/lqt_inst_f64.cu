// Kernel instantiations: LQT_VARIANTS_F64 of lqt_variants.h.
#include "lqt_launch_impl.cuh"
#include "lqt_variants.h"

namespace lqt {
LQT_VARIANTS_F64(LQT_INSTANTIATE)
}  // namespace lqt
