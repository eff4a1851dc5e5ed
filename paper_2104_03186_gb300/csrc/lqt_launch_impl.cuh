// Definitions of the per-instantiation launchers (included by the lqt_inst_*.cu
// translation units only).
#pragma once

#include <atomic>

#include "lqt_kernels.cuh"
#include "lqt_launch.cuh"

namespace lqt {

// Raise the dynamic shared-memory cap of a kernel once per device.
template <typename Kernel>
static cudaError_t allow_smem(Kernel k, std::atomic<bool>* done, size_t bytes) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_relaxed) || bytes <= 48 * 1024) return cudaSuccess;
    int optin = 0;
    err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (err == cudaSuccess) done[dev].store(true, std::memory_order_relaxed);
    return err;
}

// Launch with programmatic stream serialization when `pdl`: the kernel may be
// scheduled while its predecessor in the stream finishes (it waits in
// griddep_wait()).  Measured on one GB300 (vehicle, refined, A/B in one
// session): T = 100 0.101 -> 0.092 ms, T = 1e3 0.138 -> 0.128 ms, T = 1e5
// 0.176 -> 0.174 ms, but T = 1e6 0.365 -> 0.380 ms; so it is used for short
// chunks only (the plan's B <= kPdlMaxChunk).
constexpr int kPdlMaxChunk = 4;

template <typename R>
static cudaError_t launch_pdl(void (*kernel)(const Params<R>), unsigned grid, unsigned block,
                              size_t smem, cudaStream_t stream, const Params<R>& P, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, P);
}

template <typename R, int N, int M>
lqt_status launch_solve(const Params<R>& P, const Plan& plan, cudaStream_t stream, Prof* prof,
                        cudaEvent_t bwd_done) {
    constexpr int W = tile_threads<R, N, M>();
    constexpr int TP = top_threads();
    using SM = Smem<R, N, M, W>;
    static std::atomic<bool> done_up[64], done_top[64], done_top1[64], done_top2[64], done_down[64],
        done_ftop[64], done_fdown[64], done_solo[64];
    if (plan.solo) {
        // one tile: the whole pass in one CTA
        const size_t smem = SoloSmem<R, N, M, W>::bytes(P.p);
        if (plan.tiles != 1 || allow_smem(k_solo<R, N, M, W>, done_solo, smem) != cudaSuccess)
            return plan.tiles != 1 ? LQT_EINVAL : LQT_ECUDA;
        prof_mark(prof, stream, P.refine_add ? "solo.refine" : "solo");
        if (launch_pdl<R>(k_solo<R, N, M, W>, 1, W, smem, stream, P, true) != cudaSuccess)
            return LQT_ECUDA;
        if (bwd_done && cudaEventRecord(bwd_done, stream) != cudaSuccess) return LQT_ECUDA;
        return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
    }
    const size_t smem_up = SM::bytes(SM::UP_BIG, P.p);
    constexpr long long kTopReplay =
        top_smem_bytes(Dims<N>::ELEM, Dims<N>::VALUE, N, TP, (int)sizeof(R), true);
    const size_t smem_top_full = (size_t)top_smem_bytes(Dims<N>::ELEM, Dims<N>::VALUE, N, TP,
                                                        (int)sizeof(R), false);
    const size_t smem_top_max = kTopReplay <= kTopSmemMax ? (size_t)kTopReplay : smem_top_full;
    const size_t smem_top = P.top_mode == 2 ? (size_t)kTopReplay : smem_top_full;
    // recording and replay need one tile per top-scan thread (layout() only
    // reserves the factor store then); k_bwd_top re-checks
    if (smem_top > smem_top_max || (P.top_mode != 0 && plan.tiles > TP)) return LQT_EINVAL;
    const size_t smem_down = SM::bytes(SM::DOWN_BIG, P.p);
    const size_t smem_ftop = (size_t)(Dims<N>::AFFINE + N) * tstride(TP, (int)sizeof(R)) * sizeof(R);
    const size_t smem_fdown = SM::bytes(SM::FDOWN_BIG, P.p);
    cudaError_t err;
    if ((err = allow_smem(k_bwd_up<R, N, M, W>, done_up, smem_up)) != cudaSuccess ||
        (err = allow_smem(k_bwd_top<R, N, TP, 0>, done_top, smem_top_full)) != cudaSuccess ||
        (err = allow_smem(k_bwd_top<R, N, TP, 1>, done_top1, smem_top_full)) != cudaSuccess ||
        (err = allow_smem(k_bwd_top<R, N, TP, 2>, done_top2, smem_top_max)) != cudaSuccess ||
        (err = allow_smem(k_bwd_down<R, N, M, W>, done_down, smem_down)) != cudaSuccess ||
        (err = allow_smem(k_fwd_top<R, N, TP>, done_ftop, smem_ftop)) != cudaSuccess ||
        (err = allow_smem(k_fwd_down<R, N, M, W>, done_fdown, smem_fdown)) != cudaSuccess)
        return LQT_ECUDA;
    const int tiles = plan.tiles;
    const bool pdl = plan.B <= kPdlMaxChunk;
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "bwd_up.refine" : "bwd_up");
        err = launch_pdl<R>(k_bwd_up<R, N, M, W>, tiles, W, smem_up, stream, P, pdl);
        if (err != cudaSuccess) return LQT_ECUDA;
    }
    prof_mark(prof, stream, P.refine_add ? "bwd_top.refine" : "bwd_top");
    err = launch_pdl<R>(P.top_mode == 2   ? k_bwd_top<R, N, TP, 2>
                        : P.top_mode == 1 ? k_bwd_top<R, N, TP, 1>
                                          : k_bwd_top<R, N, TP, 0>,
                        1, TP, smem_top, stream, P, pdl);
    if (err != cudaSuccess) return LQT_ECUDA;
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "bwd_down.refine" : "bwd_down");
        err = launch_pdl<R>(k_bwd_down<R, N, M, W>, tiles, W, smem_down, stream, P, pdl);
        if (err != cudaSuccess) return LQT_ECUDA;
    }
    // S, v and K are final here (a second refinement pass does not write them)
    if (bwd_done && cudaEventRecord(bwd_done, stream) != cudaSuccess) return LQT_ECUDA;
    prof_mark(prof, stream, P.refine_add ? "fwd_top.refine" : "fwd_top");
    err = launch_pdl<R>(k_fwd_top<R, N, TP>, 1, TP, smem_ftop, stream, P, pdl);
    if (err != cudaSuccess) return LQT_ECUDA;
    if (tiles > 0) {
        prof_mark(prof, stream, P.refine_add ? "fwd_down.refine" : "fwd_down");
        err = launch_pdl<R>(k_fwd_down<R, N, M, W>, tiles, W, smem_fdown, stream, P, pdl);
        if (err != cudaSuccess) return LQT_ECUDA;
    }
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

template <typename R, int N, int M>
lqt_status launch_seq(const Params<R>& P, cudaStream_t stream) {
    static std::atomic<bool> done[64];
    const size_t smem = (size_t)ModelLayout<N, M>::size(P.p) * sizeof(R);
    if (allow_smem(k_riccati_seq<R, N, M>, done, smem) != cudaSuccess) return LQT_ECUDA;
    k_riccati_seq<R, N, M><<<1, 32, smem, stream>>>(P);
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

#define LQT_INSTANTIATE(R, N, M)                                                             \
    template lqt_status launch_solve<R, N, M>(const Params<R>&, const Plan&, cudaStream_t, \
                                              Prof*, cudaEvent_t);                         \
    template lqt_status launch_seq<R, N, M>(const Params<R>&, cudaStream_t);

}  // namespace lqt
