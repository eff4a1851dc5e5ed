// The chunked pipeline of lqt_chain.cuh in one persistent launch.
//
// The level-by-level pipeline launches one kernel per tree level (a batch of
// 4096 problems took about 100 launches per state size).  Here one
// cooperative launch of as many CTAs as are co-resident runs every phase in
// turn: the chunk folds, the up-sweep levels of Alg. 1, the terminal values,
// the down-sweep levels of the value carries, the Riccati re-folds, the
// up- and down-sweep levels of the trajectory maps and the rollouts.  Within
// a phase the CTAs' lane groups take work items: the chunks of the fold,
// re-fold and rollout from a counter (whichever group is free takes the next
// one), the pairs of a tree level by a grid stride; between phases a grid
// barrier orders the global-memory results.  The per-item work is the same
// device code as the level kernels' (b_cfold, b_cup, ... in lqt_chain.cuh).
//
// Each group owns a block sized for the chunk phases (the largest of the
// fold, re-fold and rollout blocks, and of the level phases other than the
// up-sweep), so that as many groups share an SM as in the fold launch of the
// level-by-level pipeline; in the up-sweep levels, whose block is larger, the
// even groups work on two blocks and the odd ones wait.
//
// The barrier is a counter and a generation word in the workspace.  Every
// wait is bounded: a CTA that waits longer than the limit records
// LQT_ETIMEOUT in the status word and leaves the kernel, so a missing CTA can
// never hang the GPU.  The cooperative launch guarantees that all CTAs are
// resident at once, so the limit is never reached in a correct launch.
#pragma once

#include <cuda_runtime.h>

#include "lqt_chain.cuh"

namespace lqt {
namespace chain {

constexpr int kStatusTimeout = 6;  // LQT_ETIMEOUT
constexpr int kMaxLevels = 24;

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    unsigned long long next[3];  // work counters of the fold, re-fold and rollout phases
};

// The next chunk of a phase for the calling group (lane 0 draws, the group
// shares it): chunks go to whichever group is free, as the hardware would hand
// out the CTAs of a launch, so chunks of different lengths balance.
template <int N>
__device__ __forceinline__ long long next_chunk(unsigned long long* counter, const Group<N>& g) {
    unsigned long long c = 0;
    if (g.lr == 0) c = atomicAdd(counter, 1ull);
    return (long long)__shfl_sync(g.mask, c, (threadIdx.x & 31) - g.lr);
}

// Active chunk counts of the tree levels (as in the level-by-level launch).
struct LevelPlan {
    int levels;
    long long active[kMaxLevels];
};

// Grid-wide barrier; returns false (in every thread of the CTA) when the
// wait ran out.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned int nblocks,
                                          long long limit, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        volatile unsigned int* vgen = &b->gen;
        const unsigned int my = *vgen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            b->count = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long i = 0;
            while (*vgen == my) {
                if (++i > limit) {
                    s_ok = 0;
                    atomicCAS(status, 0, kStatusTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

// The terminal value of item q by one lane group (k_cterm's work): V[c0],
// S_T, v_T, the trajectory seed x_0 and, for T = 0, x_0 itself.  Y: group
// scratch of 2N x N + 2N elements of RT.
template <typename R, typename RT, int N>
__device__ __forceinline__ void b_cterm_group(const Args<R, RT>& a, int q, RT* Y,
                                              const Group<N>& g) {
    const Item<R>& it = a.items[q];
    const DescT<R>& D = it.D;
    const int r = g.lr;
    const int pT = D.pT;
    RT* xr = Y + 2 * N * N;
    for (int i = r; i < pT; i += N) {
        RT acc[N];
        RT t0 = RT(0);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = RT(0);
        for (int b = 0; b < pT; ++b) {
            const RT xib = static_cast<RT>(D.XT[i * pT + b]);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += xib * static_cast<RT>(D.HT[b * N + j]);
            if (D.rT) t0 += xib * static_cast<RT>(D.rT[b]);
        }
#pragma unroll
        for (int j = 0; j < N; ++j) Y[i * N + j] = acc[j];
        xr[i] = t0;
    }
    g.sync();
    RT acc[N];
    RT t = RT(0);
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = RT(0);
    for (int i = 0; i < pT; ++i) {
        const RT hi = static_cast<RT>(D.HT[i * N + r]);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] += hi * Y[i * N + j];
        t += hi * xr[i];
    }
    if (D.etaT) t = static_cast<RT>(D.etaT[r]);
    RT* val = a.V + it.c0 * LValue<N>::SIZE;
#pragma unroll
    for (int j = 0; j < N; ++j) val[LValue<N>::OS + r * LValue<N>::LD + j] = acc[j];
    val[LValue<N>::OV + r] = t;
    a.X[(it.c0 + it.NC - 1) * N + r] = static_cast<RT>(D.x0[r]);
    if (a.out_mask & 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) D.S[D.T * N * N + r * N + j] = static_cast<R>(acc[j]);
    }
    if (a.out_mask & 4) D.v[D.T * N + r] = static_cast<R>(t);
    if (D.T == 0) D.x[r] = D.x0[r];
    g.sync();
}

// Shared memory of one group of the persistent kernel (bytes, rounded to 16):
// the largest block of the chunk phases and of the level phases other than
// the up-sweep, which takes two blocks.
template <typename R, typename RT, int N, int M>
constexpr int persist_group_bytes() {
    constexpr int sizes[] = {gstride<N>(FoldSmem<N, M, R>::SIZE) * (int)sizeof(R),
                             gstride<N>(RefoldSmem<N, M>::SIZE) * (int)sizeof(R),
                             gstride<N>(RollSmem<N, M>::SIZE) * (int)sizeof(R),
                             gstride<N>(DownSmem<N>::SIZE) * (int)sizeof(RT),
                             gstride<N>(FupSmem<N>::SIZE) * (int)sizeof(RT),
                             gstride<N>(FdownSmem<N>::SIZE) * (int)sizeof(RT),
                             gstride<N>(2 * N * N + 2 * N) * (int)sizeof(RT)};
    int m = 0;
    for (int s : sizes) m = s > m ? s : m;
    return (m + 15) / 16 * 16;
}

template <typename R, typename RT, int N, int M>
constexpr bool persist_up_fits() {
    return gstride<N>(UpSmem<N>::SIZE) * (int)sizeof(RT) <= 2 * persist_group_bytes<R, RT, N, M>();
}

// The body of each phase addresses group gi's block at gi * gstride<N>(its own
// size); the persistent kernel gives each group a block of
// persist_group_bytes() instead, so it passes the group's own base with gi = 0.
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_cpersist(Args<R, RT> a, LevelPlan lp,
                                                    GridBarrier* bar, long long wait_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int GB = persist_group_bytes<R, RT, N, M>();
    const int gi = threadIdx.x / N;
    unsigned char* mine = smem_raw + gi * GB;
    const Group<N> g;
    const long long first = (long long)blockIdx.x * NG + gi;
    const long long stride = (long long)gridDim.x * NG;
    const unsigned int nb = gridDim.x;
    const long long C = a.C;
    // 1. chunk folds
    for (long long c = next_chunk(&bar->next[0], g); c < C; c = next_chunk(&bar->next[0], g))
        b_cfold<R, RT, N, M, NG>(a, c, mine, 0);
    if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    // 2. up-sweep levels
    static_assert(NG % 2 == 0, "the up-sweep pairs the groups of a CTA");
    static_assert(persist_up_fits<R, RT, N, M>(), "two blocks hold the up-sweep's");
    {
        // even groups only, each on its own block and the next group's
        const long long ufirst = (long long)blockIdx.x * (NG / 2) + gi / 2;
        const long long ustride = (long long)gridDim.x * (NG / 2);
        for (int l = 0; l < lp.levels; ++l) {
            const int h = 1 << l;
            const long long pairs = lp.active[l] / (2 * h);
            if ((gi & 1) == 0)
                for (long long q = ufirst; q < pairs; q += ustride)
                    b_cup<RT, N, NG>(a.E, lp.active[l], h, a.status, q * 2 * h, mine, 0);
            if (!grid_sync(bar, nb, wait_limit, a.status)) return;
        }
    }
    // 3. terminal values, then the down-sweep levels of the value carries
    for (long long q = first; q < a.count; q += stride)
        b_cterm_group<R, RT, N>(a, (int)q, reinterpret_cast<RT*>(mine), g);
    if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    for (int l = lp.levels - 1; l >= 0; --l) {
        const int h = 1 << l;
        const long long pairs = lp.active[l] / (2 * h);
        for (long long q = first; q < pairs; q += stride)
            b_cdown<RT, N, NG>(a.E, a.V, lp.active[l], h, a.status, q * 2 * h, mine, 0);
        if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    }
    // 4. Riccati re-folds with the outputs and the chunk maps
    for (long long c = next_chunk(&bar->next[1], g); c < C; c = next_chunk(&bar->next[1], g))
        b_crefold<R, RT, N, M, NG>(a, c, mine, 0);
    if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    // 5. trajectory maps: up-sweep, then down-sweep from x_0
    for (int l = 0; l < lp.levels; ++l) {
        const int h = 1 << l;
        const long long pairs = lp.active[l] / (2 * h);
        for (long long q = first; q < pairs; q += stride)
            b_cfup<RT, N, NG>(a.FE, lp.active[l], h, q * 2 * h + 2 * h - 1, mine, 0);
        if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    }
    for (int l = lp.levels - 1; l >= 0; --l) {
        const int h = 1 << l;
        const long long pairs = lp.active[l] / (2 * h);
        for (long long q = first; q < pairs; q += stride)
            b_cfdown<RT, N, NG>(a.FE, a.X, lp.active[l], h, q * 2 * h + 2 * h - 1, mine, 0);
        if (!grid_sync(bar, nb, wait_limit, a.status)) return;
    }
    // 6. rollouts
    for (long long c = next_chunk(&bar->next[2], g); c < C; c = next_chunk(&bar->next[2], g))
        b_croll<R, RT, N, M, NG>(a, c, mine, 0);
}

}  // namespace chain
}  // namespace lqt
