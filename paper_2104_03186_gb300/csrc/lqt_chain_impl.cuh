// Launch sequence of the chunked single-problem pipeline (lqt_chain.cuh) for
// one (R, RT, N, M) variant; included by the lqt_chain_n*.cu units only.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string.h>

#include <vector>

#include "lqt_chain.cuh"
#include "lqt_chain_api.h"
#include "lqt_persist.cuh"
#include "lqt_warm.cuh"
#include "lqt_launch.cuh"
#include "lqt_upload.cuh"

namespace lqt {
namespace chain {

// Per host thread and device: the stream on which Method 2's forward element
// scan runs beside the backward scan, and the fork and join events.  Created
// on first use and never destroyed (a thread_local destructor can run after
// the CUDA runtime has shut down at process exit).
struct ForkAux {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static ForkAux* fork_aux() {
    thread_local ForkAux aux[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    ForkAux& a = aux[dev];
    if (!a.s) {
        cudaStream_t s = nullptr;
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) {
            if (e1) cudaEventDestroy(e1);
            cudaStreamDestroy(s);
            return nullptr;
        }
        a.s = s;
        a.fork = e1;
        a.join = e2;
    }
    return &a;
}

template <typename Kernel>
static cudaError_t chain_allow_smem(Kernel k, std::atomic<bool>* done, size_t bytes) {
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
    static constexpr int FOLD_B = gstride<N>(FoldSmem<N, M, R>::SIZE) * (int)sizeof(R);
    static constexpr int REFOLD_B = gstride<N>(RefoldSmem<N, M>::SIZE) * (int)sizeof(R);
    static constexpr int UP_B = gstride<N>(UpSmem<N>::SIZE) * (int)sizeof(RT);
    static constexpr int DOWN_B = gstride<N>(DownSmem<N>::SIZE) * (int)sizeof(RT);
    static constexpr int FUP_B = gstride<N>(FupSmem<N>::SIZE) * (int)sizeof(RT);
    static constexpr int FDOWN_B = gstride<N>(FdownSmem<N>::SIZE) * (int)sizeof(RT);
    static constexpr int ROLL_B = gstride<N>(RollSmem<N, M>::SIZE) * (int)sizeof(R);
    static constexpr int NG_FOLD = groups_for<N>(FOLD_B);
    static constexpr int NG_REFOLD = groups_for<N>(REFOLD_B);
    static constexpr int NG_UP = groups_for<N>(UP_B);
    static constexpr int NG_DOWN = groups_for<N>(DOWN_B);
    static constexpr int NG_FUP = groups_for<N>(FUP_B);
    static constexpr int NG_FDOWN = groups_for<N>(FDOWN_B);
    static constexpr int NG_ROLL = groups_for<N>(ROLL_B);
    static constexpr int RESID_B = ResidSmem<N, M>::template bytes<R>();
    static constexpr int NEWTON_B = gstride<N>(NewtonSmem<N, M>::SIZE) * (int)sizeof(double);
    static constexpr int NG_NEWTON = groups_for<N>(NEWTON_B);
    // FP32 problems: the compensated-FP32 Newton kernels
    static constexpr int NEWTON_C_B = gstride<N>(NewtonCSmem<N, M>::SIZE) * (int)sizeof(float);
    static constexpr int NG_NEWTON_C = groups_for<N>(NEWTON_C_B);
    static constexpr int NEWTON_G_B = gstride<N>(NewtonGSmem<N, M>::SIZE) * (int)sizeof(float);
    static constexpr int NG_NEWTON_G = groups_for<N>(NEWTON_G_B);
    static constexpr bool kCompNewton = sizeof(R) == 4;
    static constexpr int NG_RESID = groups_for<N>(RESID_B);
    static constexpr int M2_B = gstride<N>(M2Smem<N, M>::SIZE) * (int)sizeof(R);
    static constexpr int NG_M2 = groups_for<N>(M2_B);
    static constexpr int WARM_B = gstride<N>(WarmSmem<N, M>::SIZE) * (int)sizeof(R);
    static constexpr int NG_WARM = groups_for<N>(WARM_B);

    static cudaError_t prepare() {
        static std::atomic<bool> d_fold[64], d_refold[64], d_up[64], d_down[64], d_fup[64], d_fdown[64],
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
            (e = chain_allow_smem(k_cfdown<RT, N, NG_FDOWN>, d_fdown,
                                  (size_t)NG_FDOWN * FDOWN_B)) != cudaSuccess)
            return e;
        static std::atomic<bool> d_nres[64], d_ngain[64], d_resid[64], d_m2up[64], d_m2down[64], d_m2roll[64];
        if ((e = chain_allow_smem(k_m2up<RT, N, NG_UP>, d_m2up, (size_t)NG_UP * UP_B)) !=
                cudaSuccess ||
            (e = chain_allow_smem(k_m2down<RT, N, NG_UP>, d_m2down, (size_t)NG_UP * UP_B)) !=
                cudaSuccess ||
            (e = chain_allow_smem(k_m2roll<R, RT, N, M, NG_M2>, d_m2roll, (size_t)NG_M2 * M2_B)) !=
                cudaSuccess)
            return e;
        if ((e = chain_allow_smem(k_cresid<R, N, M, NG_RESID>, d_resid,
                                  (size_t)NG_RESID * RESID_B)) != cudaSuccess)
            return e;
        if constexpr (kCompNewton) {
            static std::atomic<bool> d_nres_c[64], d_ngain_c[64];
            if ((e = chain_allow_smem(k_nresid_c<N, M, NG_NEWTON_C>, d_nres_c,
                                      (size_t)NG_NEWTON_C * NEWTON_C_B)) != cudaSuccess ||
                (e = chain_allow_smem(k_ngains_c<N, M, NG_NEWTON_G>, d_ngain_c,
                                      (size_t)NG_NEWTON_G * NEWTON_G_B)) != cudaSuccess)
                return e;
        }
        if ((e = chain_allow_smem(k_nresid<R, N, M, NG_NEWTON>, d_nres,
                                  (size_t)NG_NEWTON * NEWTON_B)) != cudaSuccess ||
            (e = chain_allow_smem(k_ngains<R, N, M, NG_NEWTON>, d_ngain,
                                  (size_t)NG_NEWTON * NEWTON_B)) != cudaSuccess)
            return e;
        return chain_allow_smem(k_croll<R, RT, N, M, NG_ROLL>, d_roll, (size_t)NG_ROLL * ROLL_B);
    }

    static cudaError_t prepare_warm() {
        static std::atomic<bool> d_wfold[64], d_wrefold[64];
        cudaError_t e;
        if ((e = prepare()) != cudaSuccess) return e;
        if ((e = chain_allow_smem(k_wfold<R, RT, N, M, NG_WARM>, d_wfold,
                                  (size_t)NG_WARM * WARM_B)) != cudaSuccess)
            return e;
        return chain_allow_smem(k_wrefold<R, RT, N, M, NG_WARM>, d_wrefold,
                                (size_t)NG_WARM * WARM_B);
    }

    static int blocks(long long items, int ng) { return (int)((items + ng - 1) / ng); }

    // The persistent launch (lqt_persist.cuh): groups per CTA from its group
    // block, as many CTAs as are co-resident (at most one group per chunk).
    static constexpr int PERSIST_B = persist_group_bytes<R, RT, N, M>();
    // an even number of groups per CTA (the up-sweep pairs them), at least two
    static constexpr int NG_PERSIST =
        (groups_for<N>(PERSIST_B) & ~1) > 2 ? (groups_for<N>(PERSIST_B) & ~1) : 2;
    // variants whose two groups do not fit one SM (FP64 at n = 32) always take
    // the per-level launches
    static constexpr bool kPersistFits = (long long)NG_PERSIST * PERSIST_B <= 227 * 1024;

    // only_if_small: launch nothing and return LQT_EUNSUPPORTED when the grid
    // would need more than half of the co-resident CTAs.  A cooperative launch
    // waits until its whole grid is resident, so a grid that covers the device
    // serialises it with the work of other streams (a server's concurrent
    // batches), where per-level kernels run beside them.
    static lqt_status run_persistent(const Args<R, RT>& a, const long long* active, int levels,
                                     GridBarrier* bar, cudaStream_t s, bool only_if_small) {
        if constexpr (!kPersistFits) {
            return LQT_EUNSUPPORTED;
        } else {
        if (levels > kMaxLevels) return LQT_EINVAL;
        auto kern = k_cpersist<R, RT, N, M, NG_PERSIST>;
        static std::atomic<bool> done[64];
        const size_t smem = (size_t)NG_PERSIST * PERSIST_B;
        if (chain_allow_smem(kern, done, smem) != cudaSuccess) return LQT_ECUDA;
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NG_PERSIST * N, smem) !=
                cudaSuccess)
            return LQT_ECUDA;
        if (per_sm < 1) return LQT_ECUDA;
        long long grid = (long long)per_sm * sms;
        const long long need = (a.C + NG_PERSIST - 1) / NG_PERSIST;
        if (only_if_small && 2 * need > grid) return LQT_EUNSUPPORTED;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        LevelPlan lp;
        memset(&lp, 0, sizeof(lp));
        lp.levels = levels;
        for (int l = 0; l < levels; ++l) lp.active[l] = active[l];
        if (cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s) != cudaSuccess) return LQT_ECUDA;
        Args<R, RT> aa = a;
        long long limit = 1LL << 22;  // polls of 64 ns sleeps: far above any phase's length
        void* args[] = {&aa, &lp, &bar, &limit};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3((unsigned)grid),
                                        dim3(NG_PERSIST * N), args, smem, s) != cudaSuccess)
            return LQT_ECUDA;
        return LQT_OK;
        }
    }
    static char* base_of(const ChainCall& call) { return static_cast<char*>(call.ws); }

    // Workspace layout of a call (bytes from the start of the workspace).
    struct Layout {
        size_t items1, items2, items3, consts, bar, E, V, FE, X, E2, Pref, refine0, total;
        long long C;
    };

    static size_t up(size_t x) { return (x + 255) / 256 * 256; }

    static Layout layout(const ChainProblem* probs, int count, bool refine, bool newton,
                         bool method2 = false) {
        Layout L;
        long long C = 0;
        for (int i = 0; i < count; ++i) C += probs[i].NC;
        L.C = C;
        size_t off = 256;  // status word
        L.items1 = off;
        off += up((size_t)count * sizeof(Item<R>));
        L.items2 = off;
        if (refine) off += up((size_t)count * sizeof(Item<R>));
        L.items3 = off;
        if (newton) off += up((size_t)count * sizeof(Item<R>));
        // the linear problem's constant matrices: L = 0 (N x M), U = I (M x M), H = I
        L.consts = off;
        if (newton) off += up((size_t)(N * M + M * M + N * N) * sizeof(R));
        L.bar = off;  // grid barrier of the persistent launch
        off += up(sizeof(GridBarrier));
        const size_t nc = (size_t)C;
        L.E = off;
        off += up(nc * LElem<N>::SIZE * sizeof(RT));
        L.V = off;
        off += up(nc * LValue<N>::SIZE * sizeof(RT));
        L.FE = off;
        off += up(nc * LAffine<N>::SIZE * sizeof(RT));
        L.X = off;
        off += up(nc * N * sizeof(RT));
        L.E2 = L.Pref = 0;
        if (method2) {  // Method 2: a copy of the chunk totals and the prefixes
            L.E2 = off;
            off += up(nc * LElem<N>::SIZE * sizeof(RT));
            L.Pref = off;
            off += up(nc * LElem<N>::SIZE * sizeof(RT));
        }
        L.refine0 = off;
        if (refine)
            for (int i = 0; i < count; ++i)
                off += kkt_bytes(probs[i].problem->T) +
                       (newton ? newton_bytes(probs[i].problem->T) : 0);
        L.total = off;
        return L;
    }

    // per problem, KKT correction: eta T x N, c~ T x N, U^{-1} h T x M,
    // feedforward T x M, eta_T N, x'_0 N; Newton correction: Phi T x N x N,
    // ct T x N, R (T + 1) x N x N, rho (T + 1) x N, dS (T + 1) x N x N, dv (T + 1) x N
    static size_t kkt_bytes(long long T) {
        const size_t t = (size_t)T;
        return 2 * up(t * N * sizeof(R)) + 2 * up(t * M * sizeof(R)) + 2 * up(N * sizeof(R)) +
               up((t + 1) * N * sizeof(R)) /* v' of the correction pass (Method 2) */;
    }
    static size_t newton_bytes(long long T) {
        const size_t t = (size_t)T;
        return up(t * N * N * sizeof(R)) + up(t * N * sizeof(R)) +
               2 * up((t + 1) * N * N * sizeof(R)) + 2 * up((t + 1) * N * sizeof(R));
    }
    // The correction problem of the KKT refinement: same matrices, linear state
    // terms eta, offsets c~, no references, dx_0 = 0; its feedforward goes to
    // dbuf and the rollout adds the correction into x and u.
    static void set_correction(Item<R>& b, const Item<R>& a, R* eta, R* ctil, R* etaT, R* qh,
                               R* dbuf, R* x0p) {
        b = a;
        b.D.r = nullptr;
        b.D.rT = nullptr;
        b.D.c = ctil;
        b.D.sc = N;
        b.D.eta = eta;
        b.D.seta = N;
        b.D.etaT = etaT;
        b.D.x0 = x0p;
        b.D.u = dbuf;
        b.u_out = a.D.u;
        b.qh = qh;
    }

    static size_t workspace(const ChainProblem* probs, int count, bool refine, bool newton,
                            bool method2) {
        return layout(probs, count, refine, newton, method2).total;
    }

    // Kernel names for the profile, by pass: the solve, the correction pass of
    // the KKT refinement, the Newton correction of S and v.
    static const char* pname(int kind, int phase) {
        static const char* names[3][6] = {
            {"chain_fold", "chain_up", "chain_down", "chain_refold", "chain_fwd", "chain_roll"},
            {"chain_fold.refine", "chain_up.refine", "chain_down.refine", "chain_refold.refine",
             "chain_fwd.refine", "chain_roll.refine"},
            {"chain_fold.newton", "chain_up.newton", "chain_down.newton", "chain_refold.newton",
             "chain_fwd.newton", "chain_roll.newton"}};
        return names[kind][phase];
    }

    // Method 2's forward element scan: up-sweep of the chunk totals E2, the
    // seed (0, x_0, 0, 0, 0) and the down-sweep into the prefixes Pref.  It
    // needs only the chunk totals, so it can run beside the backward scan.
    static void m2_scan(const Args<R, RT>& a, const long long* active, int levels, RT* E2,
                        RT* Pref, cudaStream_t s) {
        for (int l = 0; l < levels; ++l) {
            const int h = 1 << l;
            k_m2up<RT, N, NG_UP><<<blocks(active[l] / (2 * h), NG_UP), NG_UP * N,
                                   (size_t)NG_UP * UP_B, s>>>(E2, active[l], h, a.status);
        }
        k_m2seed<R, RT, N><<<a.count, N, 0, s>>>(a.items, Pref);
        for (int l = levels - 1; l >= 0; --l) {
            const int h = 1 << l;
            k_m2down<RT, N, NG_UP><<<blocks(active[l] / (2 * h), NG_UP), NG_UP * N,
                                     (size_t)NG_UP * UP_B, s>>>(E2, Pref, active[l], h,
                                                                a.status);
        }
    }

    // One pass: backward scan, re-fold, then (unless backward_only) the forward
    // scan and the rollout.  With Method 2 (E2 given) the forward element scan
    // runs on a second stream, forked after the chunk fold and joined before
    // the Method 2 rollout, so that it overlaps the backward scan (Lemma
    // LQT_trajectory_method2 needs no backward result for it); with kernel
    // timing on, it runs in line so that the events stay in launch order.
    static void pass(const Args<R, RT>& a, const long long* active, int levels, bool sequential,
                     int kind, bool backward_only, cudaStream_t s, Prof* prof, RT* E2 = nullptr,
                     RT* Pref = nullptr) {
        const long long C = a.C;
        const bool m2 = E2 != nullptr && !backward_only;
        ForkAux* fa = (m2 && !(prof && prof->enabled)) ? fork_aux() : nullptr;
        bool forked = false, scanned = false;
        if (!sequential) {
            prof_mark(prof, s, pname(kind, 0));
            k_cfold<R, RT, N, M, NG_FOLD>
                <<<blocks(C, NG_FOLD), NG_FOLD * N, (size_t)NG_FOLD * FOLD_B, s>>>(a);
            if (m2) {  // the chunk totals, before the backward up-sweep overwrites them
                cudaMemcpyAsync(E2, a.E, (size_t)C * LElem<N>::SIZE * sizeof(RT),
                                cudaMemcpyDeviceToDevice, s);
                if (fa && cudaEventRecord(fa->fork, s) == cudaSuccess &&
                    cudaStreamWaitEvent(fa->s, fa->fork, 0) == cudaSuccess) {
                    m2_scan(a, active, levels, E2, Pref, fa->s);
                    scanned = true;
                    if (cudaEventRecord(fa->join, fa->s) == cudaSuccess)
                        forked = true;
                    else
                        cudaStreamSynchronize(fa->s);  // join without the event
                }
            }
            if (levels > 0) prof_mark(prof, s, pname(kind, 1));
            for (int l = 0; l < levels; ++l) {
                const int h = 1 << l;
                k_cup<RT, N, NG_UP><<<blocks(active[l] / (2 * h), NG_UP), NG_UP * N,
                                      (size_t)NG_UP * UP_B, s>>>(a.E, active[l], h, a.status);
            }
        }
        prof_mark(prof, s, pname(kind, 2));
        k_cterm<R, RT, N><<<a.count, N, 0, s>>>(a);
        for (int l = levels - 1; l >= 0; --l) {
            const int h = 1 << l;
            k_cdown<RT, N, NG_DOWN><<<blocks(active[l] / (2 * h), NG_DOWN), NG_DOWN * N,
                                      (size_t)NG_DOWN * DOWN_B, s>>>(a.E, a.V, active[l], h,
                                                                     a.status);
        }
        prof_mark(prof, s, pname(kind, 3));
        k_crefold<R, RT, N, M, NG_REFOLD>
            <<<blocks(C, NG_REFOLD), NG_REFOLD * N, (size_t)NG_REFOLD * REFOLD_B, s>>>(a);
        if (backward_only) return;
        if (m2) {
            // Method 2: prefix scan of the elements from (0, x_0, 0, 0, 0)
            if (forked) {
                cudaStreamWaitEvent(s, fa->join, 0);
            } else if (!scanned) {
                prof_mark(prof, s, kind == 1 ? "chain_m2scan.refine" : "chain_m2scan");
                m2_scan(a, active, levels, E2, Pref, s);
            }
            prof_mark(prof, s, kind == 1 ? "chain_m2roll.refine" : "chain_m2roll");
            k_m2roll<R, RT, N, M, NG_M2>
                <<<blocks(C, NG_M2), NG_M2 * N, (size_t)NG_M2 * M2_B, s>>>(a, Pref);
            return;
        }
        if (levels > 0) {
            prof_mark(prof, s, pname(kind, 4));
            for (int l = 0; l < levels; ++l) {
                const int h = 1 << l;
                k_cfup<RT, N, NG_FUP><<<blocks(active[l] / (2 * h), NG_FUP), NG_FUP * N,
                                        (size_t)NG_FUP * FUP_B, s>>>(a.FE, active[l], h);
            }
            for (int l = levels - 1; l >= 0; --l) {
                const int h = 1 << l;
                k_cfdown<RT, N, NG_FDOWN><<<blocks(active[l] / (2 * h), NG_FDOWN),
                                            NG_FDOWN * N, (size_t)NG_FDOWN * FDOWN_B, s>>>(
                    a.FE, a.X, active[l], h);
            }
        }
        prof_mark(prof, s, pname(kind, 5));
        k_croll<R, RT, N, M, NG_ROLL>
            <<<blocks(C, NG_ROLL), NG_ROLL * N, (size_t)NG_ROLL * ROLL_B, s>>>(a);
    }

    // Forward affine scan of the maps FE from the seeds in each problem's top
    // slot of X: afterwards X[c] is the state at the start of chunk c.
    static void affine_scan(RT* FE, RT* X, const long long* active, int levels, cudaStream_t s) {
        for (int l = 0; l < levels; ++l) {
            const int h = 1 << l;
            k_cfup<RT, N, NG_FUP><<<blocks(active[l] / (2 * h), NG_FUP), NG_FUP * N,
                                    (size_t)NG_FUP * FUP_B, s>>>(FE, active[l], h);
        }
        for (int l = levels - 1; l >= 0; --l) {
            const int h = 1 << l;
            k_cfdown<RT, N, NG_FDOWN><<<blocks(active[l] / (2 * h), NG_FDOWN), NG_FDOWN * N,
                                        (size_t)NG_FDOWN * FDOWN_B, s>>>(FE, X, active[l], h);
        }
    }

    // Warm solve (lqt_warm.cuh): the value vector scanned from v_T over the
    // chunks' mirrored maps, the per-chunk v_k and d_k with the chunk maps of
    // the trajectory, the trajectory scanned from x_0, then the rollout.
    static lqt_status run_warm(const ChainCall& call, cudaStream_t s, Prof* prof) {
        if (prepare_warm() != cudaSuccess) return LQT_ECUDA;
        const int count = call.count;
        if (count <= 0) return LQT_OK;
        const Layout L = layout(call.probs, count, false, false, false);
        if (call.ws_bytes < L.total) return LQT_ENOMEM;
        char* base = static_cast<char*>(call.ws);
        std::vector<Item<R>> it1((size_t)count);
        long long c0 = 0;
        int maxNC = 1;
        for (int i = 0; i < count; ++i) {
            const ChainProblem& cp = call.probs[i];
            Item<R>& a = it1[(size_t)i];
            memset(&a, 0, sizeof(a));
            a.D = make_desc<R>(cp.problem, cp.solution);
            a.B = cp.B;
            a.c0 = c0;
            a.NC = cp.NC;
            c0 += cp.NC;
            if (cp.NC > maxNC) maxNC = cp.NC;
        }
        int levels = 0;
        while ((1 << levels) < maxNC) ++levels;
        std::vector<long long> active((size_t)levels + 1, 0);
        for (int l = 0; l < levels; ++l)
            for (int i = 0; i < count; ++i)
                if (call.probs[i].NC >= (2 << l)) active[(size_t)l] += call.probs[i].NC;
        Item<R>* d1 = reinterpret_cast<Item<R>*>(base + L.items1);
        if (count == 1) {
            k_set_items<R><<<1, 1, 0, s>>>(d1, it1[0], nullptr, it1[0]);
        } else if (param_upload(d1, it1.data(), it1.size() * sizeof(Item<R>), s) !=
                   cudaSuccess) {
            return LQT_ECUDA;
        }
        Args<R, RT> a;
        a.items = d1;
        a.count = count;
        a.C = L.C;
        a.E = reinterpret_cast<RT*>(base + L.E);
        a.V = reinterpret_cast<RT*>(base + L.V);
        a.FE = reinterpret_cast<RT*>(base + L.FE);
        a.X = reinterpret_cast<RT*>(base + L.X);
        a.status = call.status ? call.status : reinterpret_cast<int*>(base);
        a.out_mask = 0;
        a.refine_add = 0;
        // the chunk totals' region holds a copy of each chunk's Psi
        static_assert(LElem<N>::SIZE >= LAffine<N>::SIZE, "Psi copy fits the element slots");
        RT* psi = a.E;
        const long long C = a.C;
        prof_mark(prof, s, "warm_fold");
        k_wfold<R, RT, N, M, NG_WARM>
            <<<blocks(C, NG_WARM), NG_WARM * N, (size_t)NG_WARM * WARM_B, s>>>(a, psi);
        prof_mark(prof, s, "warm_vscan");
        k_wterm<R, RT, N><<<count, N, 0, s>>>(a);
        affine_scan(a.FE, a.X, active.data(), levels, s);
        prof_mark(prof, s, "warm_refold");
        k_wrefold<R, RT, N, M, NG_WARM>
            <<<blocks(C, NG_WARM), NG_WARM * N, (size_t)NG_WARM * WARM_B, s>>>(a, psi);
        prof_mark(prof, s, "warm_fwd");
        k_wseed<R, RT, N><<<count, N, 0, s>>>(a);
        affine_scan(a.FE, a.X, active.data(), levels, s);
        prof_mark(prof, s, "warm_roll");
        k_croll<R, RT, N, M, NG_ROLL>
            <<<blocks(C, NG_ROLL), NG_ROLL * N, (size_t)NG_ROLL * ROLL_B, s>>>(a);
        prof_end(prof, s);
        return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
    }

    static lqt_status run(const ChainCall& call, cudaStream_t s, Prof* prof) {
        if (call.warm) return run_warm(call, s, prof);
        if (prepare() != cudaSuccess) return LQT_ECUDA;
        const int count = call.count;
        if (count <= 0) return LQT_OK;
        const bool refine = call.refine;
        const bool newton = refine && call.newton;
        const bool method2 = call.method2;
        const Layout L = layout(call.probs, count, refine, newton, method2);
        RT* E2 = method2 ? reinterpret_cast<RT*>(base_of(call) + L.E2) : nullptr;
        RT* Pref = method2 ? reinterpret_cast<RT*>(base_of(call) + L.Pref) : nullptr;
        if (call.ws_bytes < L.total) return LQT_ENOMEM;
        char* base = static_cast<char*>(call.ws);
        // items of the first pass and of the correction pass
        std::vector<Item<R>> it1((size_t)count), it2(refine ? (size_t)count : 0),
            it3(newton ? (size_t)count : 0);
        R* cL = reinterpret_cast<R*>(base + L.consts);
        R* cU = cL + N * M;
        R* cH = cU + M * M;
        long long c0 = 0, r0 = 0;
        size_t roff = L.refine0;
        int maxNC = 1;
        for (int i = 0; i < count; ++i) {
            const ChainProblem& cp = call.probs[i];
            Item<R>& a = it1[(size_t)i];
            memset(&a, 0, sizeof(a));
            a.D = make_desc<R>(cp.problem, cp.solution);
            a.B = cp.B;
            a.c0 = c0;
            a.r0 = r0;
            a.NC = cp.NC;
            c0 += cp.NC;
            r0 += cp.problem->T + 1;
            if (cp.NC > maxNC) maxNC = cp.NC;
            if (refine) {
                const size_t t = (size_t)cp.problem->T;
                R* eta = reinterpret_cast<R*>(base + roff);
                R* ctil = reinterpret_cast<R*>(base + roff + up(t * N * sizeof(R)));
                R* qh = reinterpret_cast<R*>(base + roff + 2 * up(t * N * sizeof(R)));
                R* dbuf = reinterpret_cast<R*>(base + roff + 2 * up(t * N * sizeof(R)) +
                                               up(t * M * sizeof(R)));
                R* etaT = reinterpret_cast<R*>(base + roff + 2 * up(t * N * sizeof(R)) +
                                               2 * up(t * M * sizeof(R)));
                R* x0p = etaT + up(N * sizeof(R)) / sizeof(R);
                R* vcorr = x0p + up(N * sizeof(R)) / sizeof(R);
                char* nb = base + roff + kkt_bytes(cp.problem->T);
                roff += kkt_bytes(cp.problem->T) + (newton ? newton_bytes(cp.problem->T) : 0);
                set_correction(it2[(size_t)i], a, eta, ctil, etaT, qh, dbuf, x0p);
                if (method2) it2[(size_t)i].D.v = vcorr;
                if (!newton) continue;
                R* Phi = reinterpret_cast<R*>(nb);
                R* ct = reinterpret_cast<R*>(nb + up(t * N * N * sizeof(R)));
                R* Rk = reinterpret_cast<R*>(nb + up(t * N * N * sizeof(R)) +
                                             up(t * N * sizeof(R)));
                R* dS = Rk + up((t + 1) * N * N * sizeof(R)) / sizeof(R);
                R* rho = dS + up((t + 1) * N * N * sizeof(R)) / sizeof(R);
                R* dv = rho + up((t + 1) * N * sizeof(R)) / sizeof(R);
                // the Newton correction of (S, v) as an LQT problem (k_nresid)
                Item<R>& c3 = it3[(size_t)i];
                c3 = a;
                DescT<R>& D3 = c3.D;
                D3.p = N;
                D3.pT = N;
                D3.F = Phi;
                D3.sF = (long long)N * N;
                D3.c = ct;
                D3.sc = N;
                D3.L = cL;
                D3.sL = 0;
                D3.U = cU;
                D3.sU = 0;
                D3.H = cH;
                D3.sH = 0;
                D3.X = Rk;
                D3.sX = (long long)N * N;
                D3.r = nullptr;
                D3.sr = 0;
                D3.HT = cH;
                D3.XT = Rk + t * N * N;
                D3.rT = nullptr;
                D3.eta = rho;
                D3.seta = N;
                D3.etaT = rho + t * N;
                D3.S = dS;
                D3.v = dv;
                D3.K = nullptr;
                D3.x = nullptr;
                D3.u = dbuf;
            }
        }
        int levels = 0;
        while ((1 << levels) < maxNC) ++levels;
        std::vector<long long> active((size_t)levels + 1, 0);
        for (int l = 0; l < levels; ++l)
            for (int i = 0; i < count; ++i)
                if (call.probs[i].NC >= (2 << l)) active[(size_t)l] += call.probs[i].NC;
        Item<R>* d1 = reinterpret_cast<Item<R>*>(base + L.items1);
        Item<R>* d2 = reinterpret_cast<Item<R>*>(base + L.items2);
        Item<R>* d3 = reinterpret_cast<Item<R>*>(base + L.items3);
        if (count == 1) {
            // through kernel parameters (no pageable copy; capturable in a graph)
            k_set_items<R><<<1, 1, 0, s>>>(d1, it1[0], refine ? d2 : nullptr,
                                           refine ? it2[0] : it1[0]);
            if (newton) k_set_items<R><<<1, 1, 0, s>>>(d3, it3[0], nullptr, it3[0]);
        } else {
            // descriptors through kernel parameters (lqt_upload.cuh): no stream
            // synchronisation, capturable in a graph
            if (param_upload(d1, it1.data(), it1.size() * sizeof(Item<R>), s) != cudaSuccess)
                return LQT_ECUDA;
            if (refine && param_upload(d2, it2.data(), it2.size() * sizeof(Item<R>), s) !=
                              cudaSuccess)
                return LQT_ECUDA;
            if (newton && param_upload(d3, it3.data(), it3.size() * sizeof(Item<R>), s) !=
                              cudaSuccess)
                return LQT_ECUDA;
        }
        if (newton) k_consts<R, N, M><<<1, N, 0, s>>>(cL, cU, cH);
        Args<R, RT> a;
        a.items = d1;
        a.count = count;
        a.C = L.C;
        a.E = reinterpret_cast<RT*>(base + L.E);
        a.V = reinterpret_cast<RT*>(base + L.V);
        a.FE = reinterpret_cast<RT*>(base + L.FE);
        a.X = reinterpret_cast<RT*>(base + L.X);
        a.status = call.status ? call.status : reinterpret_cast<int*>(base);
        a.out_mask = 7;
        a.refine_add = 0;
        if (kPersistFits && call.persistent && !refine && !method2 && !call.sequential) {
            // one cooperative launch for the whole pass (batches)
            const lqt_status st =
                run_persistent(a, active.data(), levels,
                               reinterpret_cast<GridBarrier*>(base + L.bar), s,
                               call.persistent_if_small);
            if (st != LQT_EUNSUPPORTED || !call.persistent_if_small) {
                prof_end(prof, s);
                if (st != LQT_OK) return st;
                return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
            }
            // too large for the automatic choice: the per-level launches below
        }
        pass(a, active.data(), levels, call.sequential, 0, false, s, prof, E2, Pref);
        if (newton) {
            // Newton correction of S and v, then K from the corrected S and v
            prof_mark(prof, s, "chain_newton_resid");
            int gridn = blocks(r0, kCompNewton ? NG_NEWTON_C : NG_NEWTON);
            if (gridn > 4096) gridn = 4096;
            if constexpr (kCompNewton)
                k_nresid_c<N, M, NG_NEWTON_C>
                    <<<gridn, NG_NEWTON_C * N, (size_t)NG_NEWTON_C * NEWTON_C_B, s>>>(
                        d1, d3, count, r0, a.status);
            else
                k_nresid<R, N, M, NG_NEWTON>
                    <<<gridn, NG_NEWTON * N, (size_t)NG_NEWTON * NEWTON_B, s>>>(d1, d3, count, r0,
                                                                                a.status);
            Args<R, RT> c = a;
            c.items = d3;
            c.out_mask = 5;
            pass(c, active.data(), levels, call.sequential, 2, true, s, prof);
            prof_mark(prof, s, "chain_newton_gains");
            if constexpr (kCompNewton) {
                int gridg = blocks(r0, NG_NEWTON_G);
                if (gridg > 4096) gridg = 4096;
                k_ngains_c<N, M, NG_NEWTON_G>
                    <<<gridg, NG_NEWTON_G * N, (size_t)NG_NEWTON_G * NEWTON_G_B, s>>>(
                        d1, d3, count, r0, a.status);
            }
            else
                k_ngains<R, N, M, NG_NEWTON>
                    <<<gridn, NG_NEWTON * N, (size_t)NG_NEWTON * NEWTON_B, s>>>(d1, d3, count, r0,
                                                                                a.status);
            prof_mark(prof, s, "chain_newton_add");
            k_nadd<R, N><<<1024, 256, 0, s>>>(d1, d3, count, r0);
        }
        if (refine) {
            // one step of iterative refinement of the KKT system for x* and u*
            prof_mark(prof, s, "chain_resid");
            int grid = blocks(r0, NG_RESID);
            if (grid > 4096) grid = 4096;
            k_cresid<R, N, M, NG_RESID><<<grid, NG_RESID * N, (size_t)NG_RESID * RESID_B, s>>>(
                d1, d2, count, r0, a.status);
            Args<R, RT> b = a;
            b.items = d2;
            // the correction pass writes no S, v, K; with Method 2 its walk needs
            // the pass's own v', kept in a workspace buffer
            b.out_mask = method2 ? 4 : 0;
            b.refine_add = 1;
            pass(b, active.data(), levels, call.sequential, 1, false, s, prof, E2, Pref);
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
            &chain::Launcher<R, RT, N, M>::workspace, &chain::Launcher<R, RT, N, M>::run,       \
            &chain::Launcher<R, RT, N, M>::fold_kernel, &chain::Launcher<R, RT, N, M>::fold_smem, \
            &chain::Launcher<R, RT, N, M>::fold_groups_per_cta                                  \
    }

}  // namespace lqt
