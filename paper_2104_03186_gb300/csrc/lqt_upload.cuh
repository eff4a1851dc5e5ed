// Host -> device upload of small descriptor arrays through kernel parameters.
//
// The batch entry points build their per-problem descriptors on the host.  A
// cudaMemcpyAsync from pageable host memory first synchronises the stream, so
// the host waited for the previous state size's kernels before it could plan
// and launch the next size (the GPU idling in between), and such a copy cannot
// be captured in a CUDA graph.  Here the bytes travel as the parameter block
// of a one-CTA copy kernel instead (kernel parameters may take up to 32 764
// bytes on sm_70 and later): the launch is asynchronous like any other, the
// host buffer may be reused as soon as the call returns, and a captured graph
// keeps the values it was captured with.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace lqt {

constexpr int kParamBlobBytes = 32000;  // a multiple of 16, under the 32 764-byte limit

struct ParamBlob {
    uint4 w[kParamBlobBytes / 16];
};

template <int UNUSED = 0>
__global__ void __launch_bounds__(256) k_param_copy(uint4* dst, const ParamBlob blob, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = blob.w[i];
}

// Copies `bytes` from host memory `src` to the device address `dst` (16-byte
// aligned) on stream `s`, in blocks of kParamBlobBytes.  The last block is
// written in whole 16-byte words, so up to 15 bytes past dst + bytes are
// overwritten: the destination region must be rounded up to 16 bytes.
inline cudaError_t param_upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    static thread_local ParamBlob blob;  // 32 KB: kept off the caller's stack
    for (size_t off = 0; off < bytes; off += kParamBlobBytes) {
        const size_t n = bytes - off < (size_t)kParamBlobBytes ? bytes - off : kParamBlobBytes;
        memcpy(&blob, static_cast<const char*>(src) + off, n);
        k_param_copy<<<1, 256, 0, s>>>(reinterpret_cast<uint4*>(static_cast<char*>(dst) + off),
                                       blob, (int)((n + 15) / 16));
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace lqt
