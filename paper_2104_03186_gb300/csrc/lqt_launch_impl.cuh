// Definitions of the per-instantiation launchers (included by the lqt_inst_*.cu
// translation units only).
#pragma once

#include "lqt_kernels.cuh"
#include "lqt_launch.cuh"

namespace lqt {

// Raise the dynamic shared-memory cap of a kernel once per device.
template <typename Kernel>
static cudaError_t allow_smem(Kernel k, bool* done, size_t bytes) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev] || bytes <= 48 * 1024) return cudaSuccess;
    int optin = 0;
    err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <typename R, int N, int M>
lqt_status launch_solve(const Params<R>& P, const Plan& plan, cudaStream_t stream, Prof* prof) {
    constexpr int W = tile_threads<R, N, M>();
    constexpr int TP = top_threads();
    using SM = Smem<R, N, M, W>;
    static bool done_up[64], done_top[64], done_down[64], done_ftop[64], done_fdown[64];
    const size_t smem_up = SM::bytes(SM::UP_BIG, P.p);
    const size_t smem_top = (size_t)(Dims<N>::ELEM + Dims<N>::VALUE) * TP * sizeof(R);
    const size_t smem_down = SM::bytes(SM::DOWN_BIG, P.p);
    const size_t smem_ftop = (size_t)(Dims<N>::AFFINE + N) * TP * sizeof(R);
    const size_t smem_fdown = SM::bytes(SM::FDOWN_BIG, P.p);
    cudaError_t err;
    if ((err = allow_smem(k_bwd_up<R, N, M, W>, done_up, smem_up)) != cudaSuccess ||
        (err = allow_smem(k_bwd_top<R, N, TP>, done_top, smem_top)) != cudaSuccess ||
        (err = allow_smem(k_bwd_down<R, N, M, W>, done_down, smem_down)) != cudaSuccess ||
        (err = allow_smem(k_fwd_top<R, N, TP>, done_ftop, smem_ftop)) != cudaSuccess ||
        (err = allow_smem(k_fwd_down<R, N, M, W>, done_fdown, smem_fdown)) != cudaSuccess)
        return LQT_ECUDA;
    const int tiles = plan.tiles;
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "bwd_up.refine" : "bwd_up");
        k_bwd_up<R, N, M, W><<<tiles, W, smem_up, stream>>>(P);
    }
    prof_mark(prof, stream, P.refine_add ? "bwd_top.refine" : "bwd_top");
    k_bwd_top<R, N, TP><<<1, TP, smem_top, stream>>>(P);
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "bwd_down.refine" : "bwd_down");
        k_bwd_down<R, N, M, W><<<tiles, W, smem_down, stream>>>(P);
    }
    prof_mark(prof, stream, P.refine_add ? "fwd_top.refine" : "fwd_top");
    k_fwd_top<R, N, TP><<<1, TP, smem_ftop, stream>>>(P);
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "fwd_down.refine" : "fwd_down");
        k_fwd_down<R, N, M, W><<<tiles, W, smem_fdown, stream>>>(P);
    }
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

template <typename R, int N, int M>
lqt_status launch_seq(const Params<R>& P, cudaStream_t stream) {
    static bool done[64];
    const size_t smem = (size_t)ModelLayout<N, M>::size(P.p) * sizeof(R);
    if (allow_smem(k_riccati_seq<R, N, M>, done, smem) != cudaSuccess) return LQT_ECUDA;
    k_riccati_seq<R, N, M><<<1, 32, smem, stream>>>(P);
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

#define LQT_INSTANTIATE(R, N, M)                                                             \
    template lqt_status launch_solve<R, N, M>(const Params<R>&, const Plan&, cudaStream_t, \
                                              Prof*);                                      \
    template lqt_status launch_seq<R, N, M>(const Params<R>&, cudaStream_t);

}  // namespace lqt
