// Launcher of one batched kernel variant (see lqt_batch.cuh).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>

#include "lqt_batch.cuh"

namespace lqt {

template <int N, int M, int NG>
void launch_batch(const BatchDesc* d, int count, int* ticket, int* status, cudaStream_t s,
                  cudaError_t* err) {
    using Lay = batch::Layout<N, M, NG>;
    static std::atomic<bool> attr[64];
    int dev = 0;
    if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return;
    const size_t smem = Lay::bytes();
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        if ((*err = cudaFuncSetAttribute(batch::k_batch<N, M, NG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem)) != cudaSuccess)
            return;
        attr[dev] = true;
    }
    int sms = 0, per_sm = 0;
    if ((*err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return;
    if ((*err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch::k_batch<N, M, NG>,
                                                              Lay::THREADS, smem)) != cudaSuccess)
        return;
    const int grid = std::max(1, std::min(count, sms * std::max(per_sm, 1)));
    batch::k_batch<N, M, NG><<<grid, Lay::THREADS, smem, s>>>(d, count, ticket, status);
    *err = cudaGetLastError();
}

}  // namespace lqt
