// Launch sequence of the chunked single-problem pipeline (lqt_chain.cuh) for
// one (R, RT, N, M) variant; included by the lqt_chain_n*.cu units only.
#pragma once

#include <cuda_runtime.h>

#include "lqt_chain.cuh"
#include "lqt_chain_api.h"
#include "lqt_launch.cuh"

namespace lqt {
namespace chain {

template <typename Kernel>
static cudaError_t chain_allow_smem(Kernel k, bool* done, size_t bytes) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev] || bytes <= 48 * 1024) return cudaSuccess;
    err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <typename R, typename RT, int N, int M>
struct Launcher {
    static constexpr int FOLD_B = FoldSmem<N, M>::SIZE * (int)sizeof(R);
    static constexpr int REFOLD_B = RefoldSmem<N, M>::SIZE * (int)sizeof(R);
    static constexpr int UP_B = UpSmem<N>::SIZE * (int)sizeof(RT);
    static constexpr int DOWN_B = DownSmem<N>::SIZE * (int)sizeof(RT);
    static constexpr int FUP_B = FupSmem<N>::SIZE * (int)sizeof(RT);
    static constexpr int FDOWN_B = FdownSmem<N>::SIZE * (int)sizeof(RT);
    static constexpr int ROLL_B = RollSmem<N, M>::SIZE * (int)sizeof(R);
    static constexpr int NG_FOLD = groups_for<N>(FOLD_B);
    static constexpr int NG_REFOLD = groups_for<N>(REFOLD_B);
    static constexpr int NG_UP = groups_for<N>(UP_B);
    static constexpr int NG_DOWN = groups_for<N>(DOWN_B);
    static constexpr int NG_FUP = groups_for<N>(FUP_B);
    static constexpr int NG_FDOWN = groups_for<N>(FDOWN_B);
    static constexpr int NG_ROLL = groups_for<N>(ROLL_B);
    static constexpr int NG_RESID = 256 / N;

    static cudaError_t prepare() {
        static bool d_fold[64], d_refold[64], d_up[64], d_down[64], d_fup[64], d_fdown[64],
            d_roll[64];
        cudaError_t e;
        if ((e = chain_allow_smem(k_cfold<R, RT, N, M, NG_FOLD>, d_fold,
                                  (size_t)NG_FOLD * FOLD_B)) != cudaSuccess ||
            (e = chain_allow_smem(k_crefold<R, RT, N, M, NG_REFOLD>, d_refold,
                                  (size_t)NG_REFOLD * REFOLD_B)) != cudaSuccess ||
            (e = chain_allow_smem(k_cup<RT, N, NG_UP>, d_up, (size_t)NG_UP * UP_B)) !=
                cudaSuccess ||
            (e = chain_allow_smem(k_cdown<RT, N, NG_DOWN>, d_down, (size_t)NG_DOWN * DOWN_B)) !=
                cudaSuccess ||
            (e = chain_allow_smem(k_cfup<RT, N, NG_FUP>, d_fup, (size_t)NG_FUP * FUP_B)) !=
                cudaSuccess ||
            (e = chain_allow_smem(k_cfdown<R, RT, N, NG_FDOWN>, d_fdown,
                                  (size_t)NG_FDOWN * FDOWN_B)) != cudaSuccess)
            return e;
        return chain_allow_smem(k_croll<R, RT, N, M, NG_ROLL>, d_roll, (size_t)NG_ROLL * ROLL_B);
    }

    static int blocks(long long items, int ng) { return (int)((items + ng - 1) / ng); }

    // One pass: backward scan, re-fold, forward scan, rollout.
    static void pass(const Args<R, RT>& a, bool sequential, bool refine_pass, cudaStream_t s,
                     Prof* prof) {
        const int NC = a.NC;
        if (!sequential) {
            prof_mark(prof, s, refine_pass ? "chain_fold.refine" : "chain_fold");
            k_cfold<R, RT, N, M, NG_FOLD>
                <<<blocks(NC, NG_FOLD), NG_FOLD * N, (size_t)NG_FOLD * FOLD_B, s>>>(a);
            if (NC > 1) prof_mark(prof, s, refine_pass ? "chain_up.refine" : "chain_up");
            for (int h = 1; h < NC; h *= 2)
                k_cup<RT, N, NG_UP><<<blocks(NC / (2 * h), NG_UP), NG_UP * N,
                                      (size_t)NG_UP * UP_B, s>>>(a.E, NC, h, a.status);
        }
        prof_mark(prof, s, refine_pass ? "chain_down.refine" : "chain_down");
        k_cterm<R, RT, N><<<1, N, 0, s>>>(a);
        for (int h = NC / 2; h >= 1; h /= 2)
            k_cdown<RT, N, NG_DOWN><<<blocks(NC / (2 * h), NG_DOWN), NG_DOWN * N,
                                      (size_t)NG_DOWN * DOWN_B, s>>>(a.E, a.V, NC, h, a.status);
        prof_mark(prof, s, refine_pass ? "chain_refold.refine" : "chain_refold");
        k_crefold<R, RT, N, M, NG_REFOLD>
            <<<blocks(NC, NG_REFOLD), NG_REFOLD * N, (size_t)NG_REFOLD * REFOLD_B, s>>>(a);
        if (NC > 1) {
            prof_mark(prof, s, refine_pass ? "chain_fwd.refine" : "chain_fwd");
            for (int h = 1; h < NC; h *= 2)
                k_cfup<RT, N, NG_FUP><<<blocks(NC / (2 * h), NG_FUP), NG_FUP * N,
                                        (size_t)NG_FUP * FUP_B, s>>>(a.FE, NC, h);
            for (int h = NC / 2; h >= 1; h /= 2)
                k_cfdown<R, RT, N, NG_FDOWN><<<blocks(NC / (2 * h), NG_FDOWN), NG_FDOWN * N,
                                               (size_t)NG_FDOWN * FDOWN_B, s>>>(
                    a.FE, a.X, a.D.x0, NC, h, h == NC / 2 ? 1 : 0);
        }
        prof_mark(prof, s, refine_pass ? "chain_roll.refine" : "chain_roll");
        k_croll<R, RT, N, M, NG_ROLL>
            <<<blocks(NC, NG_ROLL), NG_ROLL * N, (size_t)NG_ROLL * ROLL_B, s>>>(a);
    }

    static lqt_status run(const ChainCall& call, cudaStream_t s, Prof* prof) {
        if (prepare() != cudaSuccess) return LQT_ECUDA;
        const lqt_problem* P = call.problem;
        const lqt_solution* sol = call.solution;
        Args<R, RT> a;
        a.D = make_desc<R>(P, sol);
        a.B = call.B;
        a.NC = call.NC;
        a.E = static_cast<RT*>(call.E);
        a.V = static_cast<RT*>(call.V);
        a.FE = static_cast<RT*>(call.FE);
        a.X = static_cast<RT*>(call.X);
        a.status = call.status;
        a.out_mask = 1;
        a.refine_add = 0;
        pass(a, call.sequential, false, s, prof);
        if (call.refine && P->T > 0) {
            R* rp = static_cast<R*>(call.rp);
            R* cp = static_cast<R*>(call.cp);
            R* rTp = static_cast<R*>(call.rTp);
            R* x0p = static_cast<R*>(call.x0p);
            prof_mark(prof, s, "chain_resid");
            const long long items = P->T + 1;
            int grid = blocks(items, NG_RESID);
            if (grid > 4096) grid = 4096;
            k_cresid<R, N, NG_RESID><<<grid, NG_RESID * N, 0, s>>>(a.D, rp, cp, rTp, x0p);
            // the shifted problem: same matrices, r', c', r'_T, x'_0 = 0; S and K
            // do not depend on r or c, so the pass does not write them again
            Args<R, RT> b = a;
            b.D.r = P->p > 0 ? rp : nullptr;
            b.D.sr = P->p;
            b.D.c = cp;
            b.D.sc = N;
            b.D.rT = P->pT > 0 ? rTp : nullptr;
            b.D.x0 = x0p;
            b.out_mask = 0;
            b.refine_add = 1;
            pass(b, call.sequential, true, s, prof);
        }
        prof_end(prof, s);
        return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
    }

    static int fold_groups_per_cta() { return NG_FOLD; }
    static const void* fold_kernel() {
        return reinterpret_cast<const void*>(k_cfold<R, RT, N, M, NG_FOLD>);
    }
    static size_t fold_smem() { return (size_t)NG_FOLD * FOLD_B; }
};

}  // namespace chain

#define LQT_CHAIN_VARIANT(R, RT, N, M)                                                         \
    ChainVariant {                                                                              \
        sizeof(R) == 8 ? LQT_F64 : LQT_F32, N, M, sizeof(RT) == 8 && sizeof(R) == 4,            \
            (int)sizeof(R), (int)sizeof(RT), &chain::Launcher<R, RT, N, M>::run,                \
            &chain::Launcher<R, RT, N, M>::fold_kernel, &chain::Launcher<R, RT, N, M>::fold_smem, \
            &chain::Launcher<R, RT, N, M>::fold_groups_per_cta                                  \
    }

}  // namespace lqt
