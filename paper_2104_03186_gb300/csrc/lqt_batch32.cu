// The n = 32 batched variant (its own translation unit: it compiles slowly).
#include "lqt_batch_launch.cuh"

namespace lqt {
template void launch_batch<32, 16, 2>(const BatchDesc*, int, int*, int*, cudaStream_t, cudaError_t*);
}  // namespace lqt
