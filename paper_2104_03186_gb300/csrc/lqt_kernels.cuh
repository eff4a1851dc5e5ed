// Kernels of the blocked temporally parallel LQT solve.
//
// Time k = 0..T-1 is cut into chunks of B steps (one thread per chunk) and
// chunks into tiles of W chunks (one CTA per tile).  Block processing
// (Sec. V-C) folds each chunk sequentially; up/down sweeps (Sec. II-C,
// Alg. 1) scan the chunk totals inside a tile (shared memory) and the tile
// totals across the grid (one CTA).  Launch order on one stream:
//
//   bwd_up    a_k built on the fly (eq. lqt_init), chunk fold P <- a_k (x) P
//             (eq. lqt_comb), in-tile up-sweep; bulk-stores the tile tree.
//   bwd_top   suffix scan of tile totals; the carry into each tile is a value
//             (0, 0, 0, v, S) (Lemma LQT_assoc); writes S_T, v_T.
//   bwd_down  bulk-loads the tile tree, in-tile down-sweep of value carries;
//             per chunk a Riccati re-fold from its carry (S_k = J_{k,T+1},
//             v_k = eta_{k,T+1}) with the gains of eq. Control_LQT fused;
//             writes S, v, K and the feedforward (into u) through warp
//             staging; builds the chunk's closed-loop affine map (Sec. IV-C,
//             Method 1) and the in-tile forward up-sweep.
//   fwd_top   prefix scan of tile affine maps from x_0 (Lemma lqt_fwd_init).
//   fwd_down  in-tile down-sweep of states; per chunk the rollout
//             u*_k = -K_k x*_k + d_k, x*_{k+1} = F_k x*_k + c_k + L_k u*_k,
//             and, when refining, the shifted data of the second pass (first
//             pass) or x* = x^ + xi (second pass).
//
// Per-step records move between HBM and registers through per-warp shared
// memory rows (WarpRows), so that global accesses are coalesced although each
// thread walks its own chunk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lqt_dense.cuh"
#include "lqt_refine.cuh"
#include "lqt_tma.cuh"

namespace lqt {

enum : int {
    ST_OK = 0,
    ST_NOTSPD = 2,
    ST_NONFINITE = 3,
    ST_TIMEOUT = 6,
    ST_SINGULAR = 8,
};

enum : int { OUT_S = 1, OUT_V = 2, OUT_K = 4, OUT_ALL = 7 };

constexpr int kStageG = 2;  // steps per warp-staged group

template <typename R>
struct Params {
    int n, m, p, pT;
    long long T;
    const R *F, *c, *L, *U, *H, *r, *X;
    long long sF, sc, sL, sU, sH, sr, sX;
    const R *HT, *rT, *XT, *x0;
    R *S, *v, *K, *x, *u;
    // workspace
    int* status;
    R* tree;        // [tiles][ELEM][W]   in-tile backward up-sweep (left-anchored)
    R* tile_agg;    // [tiles][ELEM]      tile totals
    R* tile_carry;  // [tiles][VALUE]     value at the end of each tile
    R* ftree;       // [tiles][AFFINE][W] in-tile forward up-sweep (right-anchored)
    R* ftile_agg;   // [tiles][AFFINE]
    R* ftile_x;     // [tiles][N]         state at the start of each tile
    // refinement (see lqt_refine.cuh): shifted data written by the first pass
    R *rp, *cp, *rTp, *x0p;
    int B;          // steps per chunk
    int tiles;
    int has_c;
    int cost_invariant;  // H and X time-invariant: H^T X and H^T X H precomputed
    int dyn_invariant;   // F, L, U time-invariant: kept in shared memory
    int c_invariant;     // c time-invariant (or absent): kept in shared memory
    int out_mask;        // OUT_S | OUT_V | OUT_K: which of S, v, K this pass writes
    int refine_emit;     // first pass of a refined solve: write r', c', r'_T, x'_0
    int refine_add;      // second pass: x <- x + xi instead of x <- xi
    // top-level backward scan: 0 full operators; 1 full operators that also
    // record the maps of their vector parts in top_fac; 2 the vector parts
    // alone from top_fac (a pass whose matrices equal the recording pass's)
    int top_mode;
    R* top_fac;
    long long wait_limit;  // polls of each bounded mbarrier wait
    int wait_probe;        // > 0: k_bwd_down also waits this many polls on a barrier
                           // nothing completes (diagnostic of the timeout path)
};

__device__ __forceinline__ void set_status(int* status, int code) {
    if (code != ST_OK) atomicCAS(status, 0, code);
}

__host__ __device__ inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Shared-memory model area (floats of R), same layout in every kernel:
//   F[N*N] L[N*M] U[M*M] c[N] Q[SYM] HX[p*N] H[p*N]
// Each part starts on a multiple of 4 elements (16 bytes in FP32), and the
// area itself is 16-byte aligned in every kernel, so that load_step reads the
// parts with vector loads.
template <int N, int M>
struct ModelLayout {
    static constexpr int OF = 0, OL = round4(N * N), OU = round4(OL + N * M),
                         OC = round4(OU + M * M), OQ = round4(OC + N),
                         OHX = round4(OQ + Dims<N>::SYM);
    __host__ __device__ static constexpr int OH(int p) { return round4(OHX + p * N); }
    __host__ __device__ static constexpr int size(int p) { return round4(OH(p) + p * N); }
};

// Fill the model area from the time-invariant inputs (each part only when its
// stride is 0).  Ends with __syncthreads.
template <typename R, int N, int M>
__device__ __forceinline__ void model_prologue(const Params<R>& P, R* sm) {
    using ML = ModelLayout<N, M>;
    const int p = P.p;
    if (P.dyn_invariant) {
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) sm[ML::OF + e] = P.F[e];
        for (int e = threadIdx.x; e < N * M; e += blockDim.x) sm[ML::OL + e] = P.L[e];
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) sm[ML::OU + e] = P.U[e];
    }
    if (P.c_invariant)
        for (int e = threadIdx.x; e < N; e += blockDim.x) sm[ML::OC + e] = P.has_c ? P.c[e] : R(0);
    if (P.cost_invariant) {
        R* sHX = sm + ML::OHX;
        R* sH = sm + ML::OH(p);
        for (int e = threadIdx.x; e < p * N; e += blockDim.x) {
            const int a = e / N, i = e % N;
            R t = R(0);
            for (int b = 0; b < p; ++b) t += P.H[b * N + i] * P.X[b * p + a];
            sHX[e] = t;
            sH[e] = P.H[e];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            if (i > j) continue;
            R t = R(0);
            for (int a = 0; a < p; ++a) t += sHX[a * N + i] * P.H[a * N + j];
            sm[ML::OQ + sym<N>(i, j)] = t;
        }
    }
    __syncthreads();
}

// Vector stores of COUNT consecutive values when 16-byte aligned per item.
template <typename R, int COUNT>
__device__ __forceinline__ void store_row(R* dst, const R* vals) {
    constexpr int BYTES = COUNT * (int)sizeof(R);
    if constexpr (sizeof(R) == 4 && BYTES % 16 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 4)
            *reinterpret_cast<float4*>(dst + i) =
                make_float4(vals[i], vals[i + 1], vals[i + 2], vals[i + 3]);
    } else if constexpr (sizeof(R) == 8 && BYTES % 16 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 2)
            *reinterpret_cast<double2*>(dst + i) = make_double2(vals[i], vals[i + 1]);
    } else if constexpr (sizeof(R) == 4 && BYTES % 8 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 2)
            *reinterpret_cast<float2*>(dst + i) = make_float2(vals[i], vals[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < COUNT; ++i) dst[i] = vals[i];
    }
}

template <typename R, int COUNT>
__device__ __forceinline__ void load_row(const R* src, R* vals) {
    constexpr int BYTES = COUNT * (int)sizeof(R);
    if constexpr (sizeof(R) == 4 && BYTES % 16 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 4) {
            const float4 t = *reinterpret_cast<const float4*>(src + i);
            vals[i] = t.x; vals[i + 1] = t.y; vals[i + 2] = t.z; vals[i + 3] = t.w;
        }
    } else if constexpr (sizeof(R) == 8 && BYTES % 16 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 2) {
            const double2 t = *reinterpret_cast<const double2*>(src + i);
            vals[i] = t.x; vals[i + 1] = t.y;
        }
    } else if constexpr (sizeof(R) == 4 && BYTES % 8 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT; i += 2) {
            const float2 t = *reinterpret_cast<const float2*>(src + i);
            vals[i] = t.x; vals[i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < COUNT; ++i) vals[i] = src[i];
    }
}

// Step k of the model: F, c, L, U and the cost element Q = H^T X H, q = H^T X r,
// from the shared model area where the input is time-invariant.
template <typename R, int N, int M>
__device__ __forceinline__ void load_step(const Params<R>& P, long long k, const R* sm,
                                          const R* r_staged, Step<R, N, M>& st,
                                          int r_stride = 1) {
    using ML = ModelLayout<N, M>;
    if (P.dyn_invariant) {
        load_row<R, N * N>(sm + ML::OF, &st.F[0][0]);
        load_row<R, N * M>(sm + ML::OL, &st.L[0][0]);
        load_row<R, M * M>(sm + ML::OU, &st.U[0][0]);
    } else {
        const R* F = P.F + k * P.sF;
        const R* L = P.L + k * P.sL;
        const R* U = P.U + k * P.sU;
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) st.F[i][j] = __ldg(F + i * N + j);
#pragma unroll
            for (int a = 0; a < M; ++a) st.L[i][a] = __ldg(L + i * M + a);
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) st.U[a][b] = __ldg(U + a * M + b);
    }
    if (P.c_invariant) {
        load_row<R, N>(sm + ML::OC, st.c);
    } else {
        const R* c = P.c + k * P.sc;
#pragma unroll
        for (int i = 0; i < N; ++i) st.c[i] = __ldg(c + i);
    }
    const int p = P.p;
    const R* r = P.r ? P.r + k * P.sr : nullptr;
    if (P.cost_invariant) {
        const R* sHX = sm + ML::OHX;
        load_row<R, Dims<N>::SYM>(sm + ML::OQ, st.Q);
#pragma unroll
        for (int i = 0; i < N; ++i) st.q[i] = R(0);
        if (r) {
            for (int a = 0; a < p; ++a) {
                const R ra = r_staged ? r_staged[a * r_stride] : __ldg(r + a);
                R hx[N];
                load_row<R, N>(sHX + a * N, hx);
#pragma unroll
                for (int i = 0; i < N; ++i) st.q[i] += hx[i] * ra;
            }
        }
    } else {
        // Q = sum_a H_a^T y_a with y_a = (X H)_a ; q = sum_a H_a^T (X r)_a
        const R* H = P.H + k * P.sH;
        const R* X = P.X + k * P.sX;
#pragma unroll
        for (int k2 = 0; k2 < Dims<N>::SYM; ++k2) st.Q[k2] = R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) st.q[i] = R(0);
        for (int a = 0; a < p; ++a) {
            R y[N];
#pragma unroll
            for (int j = 0; j < N; ++j) y[j] = R(0);
            R xr = R(0);
            for (int b = 0; b < p; ++b) {
                const R xab = __ldg(X + a * p + b);
#pragma unroll
                for (int j = 0; j < N; ++j) y[j] += xab * __ldg(H + b * N + j);
                if (r) xr += xab * __ldg(r + b);
            }
            R h[N];
#pragma unroll
            for (int i = 0; i < N; ++i) h[i] = __ldg(H + a * N + i);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                st.q[i] += h[i] * xr;
#pragma unroll
                for (int j = i; j < N; ++j) st.Q[sym<N>(i, j)] += h[i] * y[j];
            }
        }
    }
}

// Chunk geometry of a tile.
struct TileGeo {
    long long T;
    long long chunk0;  // first chunk of the tile
    int B;
    __device__ void chunk(int c, long long& s, long long& e) const {
        s = (chunk0 + c) * (long long)B;
        e = s + B < T ? s + B : T;
        if (s > T) s = T;
    }
    // chunks of this tile that hold at least one step
    __device__ int live(int W) const {
        const long long first = chunk0 * (long long)B;
        if (first >= T) return 0;
        const long long n = (T - first + B - 1) / B;
        return n < W ? (int)n : W;
    }
};

// Backward group g of a chunk [s, e): steps [lo, hi), processed hi-1 .. lo.
__device__ __forceinline__ void bwd_group(long long s, long long e, int g, long long& lo,
                                          int& cnt) {
    const long long hi = e - (long long)g * kStageG;
    lo = hi - kStageG > s ? hi - kStageG : s;
    cnt = hi > lo ? (int)(hi - lo) : 0;
}

// Forward group g of a chunk [s, e): steps [lo, lo + cnt).
__device__ __forceinline__ void fwd_group(long long s, long long e, int g, long long& lo,
                                          int& cnt) {
    lo = s + (long long)g * kStageG;
    const long long hi = lo + kStageG < e ? lo + kStageG : e;
    cnt = hi > lo ? (int)(hi - lo) : 0;
}

// Per-thread prefetch of the references r_k of one staged group ahead
// (p <= kRStage; two buffers of kStageG steps each).  The buffers of a CTA are
// slot-major: value q of thread t at q * W + t, so that the lanes of a warp
// write and read consecutive words (a thread-major buffer of 16 values put
// every lane of a warp on the same two banks).
constexpr int kRStage = 4;
constexpr int kRBuf = 2 * kStageG * kRStage;  // values per thread

template <typename R>
__device__ __forceinline__ bool r_stageable(const Params<R>& P) {
    return P.r != nullptr && P.p <= kRStage;
}

// Issue the copies of r for steps [lo, lo + cnt) into buf (value a of slot jj
// at (jj * kRStage + a) * stride) and commit them as one group (an empty group
// when nothing is staged).
template <typename R>
__device__ __forceinline__ void r_prefetch(const Params<R>& P, R* buf, long long lo, int cnt,
                                           int stride) {
    if (r_stageable(P))
        for (int jj = 0; jj < cnt; ++jj)
            for (int a = 0; a < P.p; ++a)
                cp_async<sizeof(R)>(buf + (jj * kRStage + a) * stride,
                                    P.r + (lo + jj) * P.sr + a);
    cp_async_commit();
}

// Dynamic shared memory of the per-tile kernels: a 16-byte head holding the
// mbarrier, then the big area, then the per-thread r buffers, then the model
// area.
constexpr int kSmemHead = 16;

// The in-tile and top-level trees are stored field-major: field f of tree slot
// i sits at f * tstride(W, sizeof(R)) + tslot<R>(i).  One spare slot after
// every 32 slots (16 for FP64) puts the slots that one tree level touches
// (i = 2h t and 2h t + h, or 2h t + 2h - 1 and 2h t + h - 1) in distinct banks;
// unpadded, threads of a level 2h slots apart shared banks up to 16-fold.
__host__ __device__ constexpr int tree_shift(int es) { return es == 8 ? 4 : 5; }
__host__ __device__ constexpr int tstride(int w, int es) { return w + (w >> tree_shift(es)); }
template <typename R>
__host__ __device__ __forceinline__ constexpr int tslot(int i) {
    return i + (i >> tree_shift((int)sizeof(R)));
}

// Factor store of the top-level backward scan (k_bwd_top, modes 1 and 2):
// the 4 N^2 map entries of each of the up-sweep's combines (combine_view<REC>),
// then the 2 N^2 of each of the down-sweep's value applies (value_apply<REC>).
// Entry-major: entry e of node u at e * tp + u (fewer than tp nodes per
// sweep), so that the threads of a level, which handle consecutive nodes,
// touch consecutive words.
__host__ __device__ constexpr int top_fac_up(int n) { return 4 * n * n; }
__host__ __device__ constexpr int top_fac_dn(int n) { return 2 * n * n; }
__host__ __device__ constexpr long long top_fac_elems(int n, int tp) {
    return (long long)tp * (top_fac_up(n) + top_fac_dn(n));
}
// Dynamic shared memory of k_bwd_top: the tree and the carries, plus the
// staged factor store when it replays.
// Staging area of the tile totals (one per thread at most), whole 16-byte units.
__host__ __device__ constexpr long long top_stage_elems(int elem, int tp, int es) {
    return ((long long)tp * elem * es + 15) / 16 * 16 / es;
}
__host__ __device__ constexpr long long top_smem_bytes(int elem, int value, int n, int tp,
                                                       int es, bool replay) {
    return ((long long)(elem + value) * tstride(tp, es) + (replay ? top_fac_elems(n, tp) : 0) +
            top_stage_elems(elem, tp, es)) *
               es +
           16;  // the mbarrier of the bulk copies
}
constexpr long long kTopSmemMax = 227 * 1024;

template <typename R, int N, int M, int W>
struct Smem {
    static constexpr int NW = W / 32;
    // bwd_down staging row per lane: S, v, K, d of kStageG steps
    static constexpr int DS = 0, DV = DS + round4(kStageG * N * N),
                         DK = DV + round4(kStageG * N), DD = DK + round4(kStageG * M * N),
                         DROW = DD + round4(kStageG * M);
    // fwd_down staging row per lane: two input buffers (K, d, x^) and the
    // outputs (x, u, c', r' padded to 4 per step)
    static constexpr int FIK = 0, FID = FIK + round4(kStageG * M * N),
                         FIX = FID + round4(kStageG * M), FIN = FIX + round4(kStageG * N);
    static constexpr int FX = 2 * FIN, FU = FX + round4(kStageG * N),
                         FC = FU + round4(kStageG * M), FR = FC + round4(kStageG * N),
                         FROW = FR + kStageG * 4;
    static constexpr int WS = tstride(W, (int)sizeof(R));  // tree slots per field
    static constexpr int UP_BIG = Dims<N>::ELEM * WS;
    static constexpr int DOWN_BIG_A = (Dims<N>::ELEM + Dims<N>::VALUE) * WS;
    static constexpr int DOWN_BIG_B = NW * 32 * DROW;
    static constexpr int DOWN_BIG = DOWN_BIG_A > DOWN_BIG_B ? DOWN_BIG_A : DOWN_BIG_B;
    static constexpr int FDOWN_BIG_A = (Dims<N>::AFFINE + N) * WS;
    static constexpr int FDOWN_BIG_B = NW * 32 * FROW;
    static constexpr int FDOWN_BIG = FDOWN_BIG_A > FDOWN_BIG_B ? FDOWN_BIG_A : FDOWN_BIG_B;
    static constexpr int RBUF = W * kRBuf;
    static size_t bytes(int big, int p) {
        return kSmemHead + (size_t)(big + RBUF + ModelLayout<N, M>::size(p)) * sizeof(R);
    }
};

// Threads per tile (one CTA): 512 in FP32 (256 in FP64) unless the largest
// per-tile shared-memory layout would exceed the opt-in limit (227 KB), then
// half.  The in-tile trees hold W elements; W is a power of two.
template <typename R, int N, int M, int W>
constexpr size_t tile_smem_bytes_max() {
    using SM = Smem<R, N, M, W>;
    constexpr int big = SM::DOWN_BIG > SM::FDOWN_BIG ? SM::DOWN_BIG : SM::FDOWN_BIG;
    // model area with p up to 2N
    return kSmemHead + (size_t)(big + SM::RBUF + ModelLayout<N, M>::size(2 * N)) * sizeof(R);
}

template <typename R, int N, int M>
constexpr int tile_threads() {
    constexpr int w = sizeof(R) == 4 ? 512 : 256;
    return tile_smem_bytes_max<R, N, M, w>() <= 227 * 1024 ? w : w / 2;
}

// ===========================================================================
// bwd_up: chunk fold + in-tile up-sweep (left-anchored: after level d, slot
// i = j * 2^{d+1} holds the total of chunks [i, i + 2^{d+1}); slot i + 2^d
// keeps the total of [i + 2^d, i + 2^{d+1}) for the down-sweep).  Only the
// chunks that hold steps are swept (the rest are neutral).
// ===========================================================================
// The body of each per-tile kernel is a device function over one tile, so
// that the single-tile solve (k_solo) runs the same code back to back with
// its trees left in shared memory.  SOLO: the only tile of the problem; the
// tree is not stored for another kernel.  The model area `sm` is filled.
template <typename R, int N, int M, int W, bool SOLO>
__device__ __forceinline__ void bwd_up_body(const Params<R>& P, unsigned tile, R* tree,
                                            const R* sm) {
    using SM = Smem<R, N, M, W>;
    constexpr int WS = SM::WS;
    const int tid = threadIdx.x;
    const TileGeo geo{P.T, (long long)tile * W, P.B};
    const int Weff = next_pow2(geo.live(W));
    long long s, e;
    geo.chunk(tid, s, e);
    Elem<R, N> acc;
    set_neutral(acc);
    bool ok = true;
    for (long long k = e - 1; k >= s; --k) {
        Step<R, N, M> st;
        load_step<R, N, M>(P, k, sm, nullptr, st);
        ok &= fold_step<R, N, M>(st, P.has_c != 0, acc);
    }
    store_elem(acc, ElemView<R, N>{tree + tslot<R>(tid), WS});
    __syncthreads();
    bool ok2 = true;
#pragma unroll 1
    for (int h = 1; h < Weff; h <<= 1) {
        const int i = tid * 2 * h;
        if (i < Weff)
            ok2 &= combine_view<R, N>(ElemView<R, N>{tree + tslot<R>(i), WS},
                                      ElemView<R, N>{tree + tslot<R>(i + h), WS},
                                      ElemView<R, N>{tree + tslot<R>(i), WS});
        __syncthreads();
    }
    if (!SOLO) {
        if (tid < Dims<N>::ELEM) P.tile_agg[(size_t)tile * Dims<N>::ELEM + tid] = tree[tid * WS];
        cta_bulk_store(P.tree + (size_t)tile * Dims<N>::ELEM * WS, tree,
                       (uint32_t)(Dims<N>::ELEM * WS * sizeof(R)));
    }
    if (!ok) set_status(P.status, ST_NOTSPD);
    if (!ok2) set_status(P.status, ST_SINGULAR);
}

template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_bwd_up(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    using SM = Smem<R, N, M, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* tree = reinterpret_cast<R*>(smem_raw + kSmemHead);  // [ELEM][WS]
    R* sm = tree + SM::UP_BIG + SM::RBUF;
    model_prologue<R, N, M>(P, sm);
    bwd_up_body<R, N, M, W, false>(P, blockIdx.x, tree, sm);
}

// Terminal value S_T = H_T^T X_T H_T, v_T = H_T^T X_T r_T.
template <typename R, int N>
__device__ __forceinline__ void terminal_value(const Params<R>& P, Value<R, N>& z) {
    const int pT = P.pT;
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) z.S[k] = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) z.v[i] = R(0);
    for (int a = 0; a < pT; ++a) {
        R y[N];
        R xr = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) y[j] = R(0);
        for (int b = 0; b < pT; ++b) {
            const R xab = P.XT[a * pT + b];
#pragma unroll
            for (int j = 0; j < N; ++j) y[j] += xab * P.HT[b * N + j];
            if (P.rT) xr += xab * P.rT[b];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const R h = P.HT[a * N + i];
            z.v[i] += h * xr;
#pragma unroll
            for (int j = i; j < N; ++j) z.S[sym<N>(i, j)] += h * y[j];
        }
    }
}

// ===========================================================================
// bwd_top: one CTA of TP threads.  Thread t folds tiles [t g, (t+1) g)
// (g = ceil(tiles / TP); with g = 1 the tile totals come in by bulk copy), the
// CTA sweeps the partial totals, and the value carries flow back from the
// terminal value (S_T, v_T) of Lemma LQT_assoc.
// ===========================================================================
// MODE (the pass's Params::top_mode) selects the kernel: 0 full operators,
// 1 full operators recording their maps, 2 replay.  One kernel per mode keeps
// each one's code small: the single warp that works at the upper levels
// otherwise stalls on instruction fetch.  Modes 1 and 2 need one tile per
// thread (tiles <= TP), which the host checks.
template <typename R, int N, int TP, int MODE>
__global__ void __launch_bounds__(TP, 1) k_bwd_top(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TS = tstride(TP, (int)sizeof(R));      // tree slots per field
    constexpr int FU = top_fac_up(N), FD = top_fac_dn(N);
    R* tree = reinterpret_cast<R*>(smem_raw);            // [ELEM][TS]
    R* carry = tree + (size_t)Dims<N>::ELEM * TS;        // [VALUE][TS]
    R* sfac = carry + (size_t)Dims<N>::VALUE * TS;       // mode 2: staged factor store
    const int tid = threadIdx.x;
    const int tiles = P.tiles;
    const int g = tiles > 0 ? (tiles + TP - 1) / TP : 1;
    const int used = tiles > 0 ? (tiles + g - 1) / g : 1;
    const int Teff = next_pow2(used);
    const int t0 = min(tid * g, tiles), t1 = min(t0 + g, tiles);
    constexpr int mode = MODE;
    if (mode != 0 && g != 1) {
        // the factor store covers one tile per thread; the host rejects other
        // plans before launching, so this only guards against a bad caller
        if (tid == 0) set_status(P.status, ST_SINGULAR);
        return;
    }
    bool ok = true;

    // Shared memory after the carries: [mode 2: the recorded maps of both
    // sweeps] | the tile totals as stored ([tiles][ELEM], one tile per thread)
    // | the mbarrier of the bulk copies that bring both in.
    constexpr int E = Dims<N>::ELEM;
    constexpr long long kFacElems = mode == 2 ? top_fac_elems(N, TP) : 0;
    constexpr uint32_t kFacBytes = (uint32_t)(kFacElems * sizeof(R));
    static_assert(kFacBytes % 16 == 0, "bulk copy of 16-byte multiples");
    R* stg = sfac + kFacElems;
    uint64_t* bar = reinterpret_cast<uint64_t*>(stg + top_stage_elems(E, TP, (int)sizeof(R)));
    const bool bulk = g == 1 && tiles > 0;  // tile totals by bulk copy
    const bool stage = mode == 2 && Teff > 1;
    // the copy may round up past the last tile into the buffer's alignment padding
    const uint32_t agg_bytes = (uint32_t)(((size_t)tiles * E * sizeof(R) + 15) / 16 * 16);
    if ((bulk || stage) && tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (stage ? kFacBytes : 0u) + (bulk ? agg_bytes : 0u));
        if (stage) bulk_g2s(sfac, P.top_fac, kFacBytes, bar);
        if (bulk) bulk_g2s(stg, P.tile_agg, agg_bytes, bar);
    }
    // thread partial: tile totals t0..t1-1 folded right to left (neutral if empty)
    ElemView<R, N> mine{tree + tslot<R>(tid), TS};
    if (mode == 0 && !bulk && t1 > t0) {  // several tiles per thread (mode 0 only)
        const R* src = P.tile_agg + (size_t)(t1 - 1) * E;
        for (int k = 0; k < E; ++k) mine.p[k * TS] = src[k];
        for (int t = t1 - 2; t >= t0; --t)
            ok &= combine_view<R, N>(
                ElemView<R, N>{const_cast<R*>(P.tile_agg) + (size_t)t * E, 1}, mine, mine);
    }
    if (t1 <= t0) {
        Elem<R, N> e;
        set_neutral(e);
        store_elem(e, mine);
    }
    // The terminal value (S_T, v_T) seeds the down-sweep.  The last thread
    // never combines in the up-sweep (Teff <= TP), so it forms it meanwhile.
    if (tid == TP - 1) {
        Value<R, N> z;
        terminal_value<R, N>(P, z);
        store_value(z, ValueView<R, N>{carry, TS});
        R* ST = P.S + (size_t)P.T * N * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (P.out_mask & OUT_S) {
#pragma unroll
                for (int j = 0; j < N; ++j) ST[i * N + j] = z.S[sym<N>(i, j)];
            }
            if (P.out_mask & OUT_V) P.v[(size_t)P.T * N + i] = z.v[i];
        }
    }
    __syncthreads();  // the mbarrier is initialised before anyone waits on it
    if (bulk || stage) {
        const bool ok_load = mbar_wait(bar, 0, P.wait_limit);
        if (!ok_load) {
            mbar_wait(bar, 0, P.wait_limit);  // one more bounded wait for the copies in flight
            if (tid == 0) set_status(P.status, ST_TIMEOUT);
        }
    }
    if (bulk && t1 > t0) {
        // this thread's tile total into its tree slot (mode 2: the vectors alone)
        const R* row = stg + (size_t)tid * E;
        if (mode == 2) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                mine.b(k) = row[Dims<N>::OB + k];
                mine.eta(k) = row[Dims<N>::OE + k];
            }
        } else {
#pragma unroll 4
            for (int k = 0; k < E; ++k) mine.p[k * TS] = row[k];
        }
    }
    __syncthreads();
    // up-sweep; the combines of level h are numbered after those of the lower
    // levels (Teff / 2h of them), thread order within a level
    int node = 0;
#pragma unroll 1
    for (int h = 1; h < Teff; h <<= 1) {
        const int i = tid * 2 * h;
        if (i < Teff) {
            const ElemView<R, N> e1{tree + tslot<R>(i), TS}, e2{tree + tslot<R>(i + h), TS};
            if (mode == 2)
                combine_replay<R, N>(sfac + node + tid, TP, e1, e2, e1);
            else if (mode == 1)
                ok &= combine_view<R, N, true>(e1, e2, e1, P.top_fac + node + tid, TP);
            else
                ok &= combine_view<R, N>(e1, e2, e1);
        }
        node += Teff / (2 * h);
        __syncthreads();
    }
    // down-sweep, applies numbered the same way from the top level
    R* gdn = P.top_fac + (long long)TP * FU;
    const R* sdn = sfac + (long long)TP * FU;
    node = 0;
#pragma unroll 1
    for (int h = Teff / 2; h >= 1; h >>= 1) {
        const int i = tid * 2 * h;
        if (i < Teff) {
            const ValueView<R, N> ci{carry + tslot<R>(i), TS}, ch{carry + tslot<R>(i + h), TS};
            const ElemView<R, N> el{tree + tslot<R>(i + h), TS};
            if (mode == 2) {
                // the values' S equal the recording pass's: only v moves
                R v[N];
#pragma unroll
                for (int k = 0; k < N; ++k) v[k] = ci.v(k);
#pragma unroll
                for (int k = 0; k < N; ++k) ch.v(k) = v[k];
                value_replay<R, N>(sdn + node + tid, TP, el, v);
#pragma unroll
                for (int k = 0; k < N; ++k) ci.v(k) = v[k];
            } else {
                Value<R, N> c;
                load_value(c, ci);
                store_value(c, ch);
                if (mode == 1)
                    ok &= value_apply<R, N, true>(el, c, gdn + node + tid, TP);
                else
                    ok &= value_apply<R, N>(el, c);
                store_value(c, ci);
            }
        }
        node += Teff / (2 * h);
        __syncthreads();
    }
    // per-tile carries for this thread's tiles
    if (t1 > t0) {
        if (mode == 2) {
            // S of the carries stays as the recording pass wrote it
            R* dst = P.tile_carry + (size_t)t0 * Dims<N>::VALUE + Dims<N>::SYM;
#pragma unroll
            for (int k = 0; k < N; ++k) dst[k] = carry[(Dims<N>::SYM + k) * TS + tslot<R>(tid)];
        } else {
            Value<R, N> c;
            load_value(c, ValueView<R, N>{carry + tslot<R>(tid), TS});
            for (int t = t1 - 1; t >= t0; --t) {
                store_value(c, ValueView<R, N>{P.tile_carry + (size_t)t * Dims<N>::VALUE, 1});
                if (t > t0)
                    ok &= value_apply<R, N>(
                        ElemView<R, N>{const_cast<R*>(P.tile_agg) + (size_t)t * Dims<N>::ELEM, 1},
                        c);
            }
        }
    }
    if (!ok) set_status(P.status, ST_SINGULAR);
}

// ===========================================================================
// bwd_down: in-tile down-sweep of values, Riccati re-fold per chunk with the
// gains fused, and the forward affine up-sweep (right-anchored).
// ===========================================================================
// S_T and v_T of the terminal value z, as the pass's out_mask asks.
template <typename R, int N>
__device__ __forceinline__ void terminal_outputs(const Params<R>& P, const Value<R, N>& z) {
    R* ST = P.S + (size_t)P.T * N * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (P.out_mask & OUT_S) {
#pragma unroll
            for (int j = 0; j < N; ++j) ST[i * N + j] = z.S[sym<N>(i, j)];
        }
        if (P.out_mask & OUT_V) P.v[(size_t)P.T * N + i] = z.v[i];
    }
}

// bwd_down over one tile.  rbuf: this thread's r buffers (slot-major, stride
// W); sm: the model area, filled here unless SOLO (the caller filled it).
// SOLO: the up-sweep's tree is already in `big`, and the value carried into
// the tile is the terminal value (Lemma LQT_assoc), formed here.
template <typename R, int N, int M, int W, bool SOLO>
__device__ __forceinline__ void bwd_down_body(const Params<R>& P, unsigned tile,
                                              unsigned char* smem_raw, R* rbuf, R* sm) {
    using SM = Smem<R, N, M, W>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* probe_bar = bar + 1;  // second word of the head: the diagnostic wait
    R* big = reinterpret_cast<R*>(smem_raw + kSmemHead);
    constexpr int WS = SM::WS;
    R* tree = big;                                       // [ELEM][WS]
    R* carry = big + (size_t)Dims<N>::ELEM * WS;         // [VALUE][WS]
    const int tid = threadIdx.x;
    if (tid == 0) {
        if (!SOLO) mbar_init(bar, 1);
        if (P.wait_probe > 0) mbar_init(probe_bar, 1);
    }
    long long s, e;
    const TileGeo geo{P.T, (long long)tile * W, P.B};
    geo.chunk(tid, s, e);
    {
        long long lo;
        int cnt;
        bwd_group(s, e, 0, lo, cnt);
        r_prefetch(P, rbuf, lo, cnt, W);
    }
    if (SOLO)
        __syncthreads();  // the barrier is initialised before anyone waits on it
    else
        model_prologue<R, N, M>(P, sm);  // ends with __syncthreads

    bool ok_load = true;
    if (!SOLO) {
        uint32_t phase = 0;
        ok_load = cta_bulk_load(tree, P.tree + (size_t)tile * Dims<N>::ELEM * WS,
                                (uint32_t)(Dims<N>::ELEM * WS * sizeof(R)), bar, phase,
                                P.wait_limit);
    }
    // Diagnostic: a wait on a barrier that no copy and no thread completes runs
    // out after P.wait_probe polls, as a lost bulk copy would; the kernel then
    // flags the timeout and carries on like after any other timed-out wait.
    if (P.wait_probe > 0 && !mbar_wait(probe_bar, 0, P.wait_probe)) ok_load = false;
    const int Weff = next_pow2(geo.live(W));
    if (SOLO) {
        if (tid == W - 1) {
            Value<R, N> z;
            terminal_value<R, N>(P, z);
            store_value(z, ValueView<R, N>{carry, WS});
            terminal_outputs<R, N>(P, z);
        }
    } else if (tid < Dims<N>::VALUE) {
        carry[tid * WS] = P.tile_carry[(size_t)tile * Dims<N>::VALUE + tid];
    }
    __syncthreads();
    bool ok_sing = true;
#pragma unroll 1
    for (int h = Weff / 2; h >= 1; h >>= 1) {
        const int i = tid * 2 * h;
        if (i < Weff) {
            Value<R, N> c;
            load_value(c, ValueView<R, N>{carry + tslot<R>(i), WS});
            store_value(c, ValueView<R, N>{carry + tslot<R>(i + h), WS});
            ok_sing &= value_apply<R, N>(ElemView<R, N>{tree + tslot<R>(i + h), WS}, c);
            store_value(c, ValueView<R, N>{carry + tslot<R>(i), WS});
        }
        __syncthreads();
    }
    Value<R, N> val;
    load_value(val, ValueView<R, N>{carry + tslot<R>(tid), WS});
    __syncthreads();  // the big area becomes the warp staging rows

    const int lane = tid & 31, warp = tid >> 5;
    R* rows = big + (size_t)warp * 32 * SM::DROW;
    R* myrow = rows + lane * SM::DROW;
    const long long tbase = geo.chunk0 * P.B;  // first step of the tile
    const bool staged = r_stageable(P);
    R Phi[N][N], gam[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) Phi[i][j] = (i == j) ? R(1) : R(0);
        gam[i] = R(0);
    }
    bool ok = true, finite = true;
    const int groups = (P.B + kStageG - 1) / kStageG;
    for (int g = 0; g < groups; ++g) {
        if (g + 1 < groups) {
            long long lo1;
            int cnt1;
            bwd_group(s, e, g + 1, lo1, cnt1);
            r_prefetch(P, rbuf + ((g + 1) & 1) * kStageG * kRStage * W, lo1, cnt1, W);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        long long lo;
        int cnt;
        bwd_group(s, e, g, lo, cnt);
        const R* rg = rbuf + (g & 1) * kStageG * kRStage * W;
        for (int jj = cnt - 1; jj >= 0; --jj) {
            const long long k = lo + jj;
            Step<R, N, M> st;
            load_step<R, N, M>(P, k, sm, staged ? rg + jj * kRStage * W : nullptr, st, W);
            R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
            ok &= riccati_step<R, N, M>(st, P.has_c != 0, val.S, val.v, K, d, Ft, ct, Rc, Rinv);
            // records of step k into this lane's staging row
            R rec[N * N];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = 0; j < N; ++j) rec[i * N + j] = val.S[sym<N>(i, j)];
            store_row<R, N * N>(myrow + SM::DS + jj * N * N, rec);
            store_row<R, N>(myrow + SM::DV + jj * N, val.v);
            R Kk[M * N];
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int j = 0; j < N; ++j) Kk[a * N + j] = K[a][j];
            store_row<R, M * N>(myrow + SM::DK + jj * M * N, Kk);
            store_row<R, M>(myrow + SM::DD + jj * M, d);
#pragma unroll
            for (int i = 0; i < N; ++i) finite = finite && isfinite(val.v[i]) && isfinite(rec[i * N + i]);
            // chunk map: x_e = Phi x_k + gam after adding step k
#pragma unroll
            for (int i = 0; i < N; ++i) {
                R t = gam[i];
#pragma unroll
                for (int j = 0; j < N; ++j) t += Phi[i][j] * ct[j];
                gam[i] = t;
            }
            R Pn[N][N];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    R t = R(0);
#pragma unroll
                    for (int l = 0; l < N; ++l) t += Phi[i][l] * Ft[l][j];
                    Pn[i][j] = t;
                }
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = 0; j < N; ++j) Phi[i][j] = Pn[i][j];
        }
        __syncwarp();
        const int lrel = (int)(lo - tbase);
        if (P.out_mask & OUT_S)
            WarpRows<R, N * N, kStageG>::store(P.S, tbase, rows + SM::DS, SM::DROW, lrel, cnt);
        if (P.out_mask & OUT_V)
            WarpRows<R, N, kStageG>::store(P.v, tbase, rows + SM::DV, SM::DROW, lrel, cnt);
        if (P.out_mask & OUT_K)
            WarpRows<R, M * N, kStageG>::store(P.K, tbase, rows + SM::DK, SM::DROW, lrel, cnt);
        WarpRows<R, M, kStageG>::store(P.u, tbase, rows + SM::DD, SM::DROW, lrel, cnt);
        __syncwarp();
    }
    __syncthreads();  // the big area becomes the forward tree
    // forward up-sweep (right-anchored): after level d, slot j = i + 2^{d+1} - 1
    // holds the composite of chunks [i, i + 2^{d+1}); slot i + 2^d - 1 keeps [i, i + 2^d)
    R* ftree = big;  // [AFFINE][WS]
    {
        AffineView<R, N> mine{ftree + tslot<R>(tid), WS};
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) mine.F(i, j) = Phi[i][j];
            mine.c(i) = gam[i];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = 1; h < Weff; h <<= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < Weff)
            affine_compose_view<R, N>(AffineView<R, N>{ftree + tslot<R>(j - h), WS},
                                      AffineView<R, N>{ftree + tslot<R>(j), WS},
                                      AffineView<R, N>{ftree + tslot<R>(j), WS});
        __syncthreads();
    }
    if (!SOLO) {
        if (tid < Dims<N>::AFFINE)
            P.ftile_agg[(size_t)tile * Dims<N>::AFFINE + tid] =
                ftree[tid * WS + tslot<R>(Weff - 1)];
        cta_bulk_store(P.ftree + (size_t)tile * Dims<N>::AFFINE * WS, ftree,
                       (uint32_t)(Dims<N>::AFFINE * WS * sizeof(R)));
    }
    if (!ok) set_status(P.status, ST_NOTSPD);
    if (!finite) set_status(P.status, ST_NONFINITE);
    if (!ok_sing) set_status(P.status, ST_SINGULAR);
    if (!ok_load) set_status(P.status, ST_TIMEOUT);
}

template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_bwd_down(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    using SM = Smem<R, N, M, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* big = reinterpret_cast<R*>(smem_raw + kSmemHead);
    bwd_down_body<R, N, M, W, false>(P, blockIdx.x, smem_raw, big + SM::DOWN_BIG + threadIdx.x,
                                     big + SM::DOWN_BIG + SM::RBUF);
}

// ===========================================================================
// fwd_top: one CTA of TP threads; prefix scan of tile affine maps seeded with
// x_0 (Lemma lqt_fwd_init: the first element maps everything to the state).
// ===========================================================================
template <typename R, int N, int TP>
__global__ void __launch_bounds__(TP, 1) k_fwd_top(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TS = tstride(TP, (int)sizeof(R));  // tree slots per field
    R* tree = reinterpret_cast<R*>(smem_raw);      // [AFFINE][TS]
    R* xs = tree + (size_t)Dims<N>::AFFINE * TS;   // [N][TS]
    const int tid = threadIdx.x;
    const int tiles = P.tiles;
    const int g = tiles > 0 ? (tiles + TP - 1) / TP : 1;
    const int used = tiles > 0 ? (tiles + g - 1) / g : 1;
    const int Teff = next_pow2(used);
    const int t0 = min(tid * g, tiles), t1 = min(t0 + g, tiles);
    {
        AffineView<R, N> mine{tree + tslot<R>(tid), TS};
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) mine.F(i, j) = (i == j) ? R(1) : R(0);
            mine.c(i) = R(0);
        }
        for (int t = t0; t < t1; ++t)
            affine_compose_view<R, N>(
                mine, AffineView<R, N>{P.ftile_agg + (size_t)t * Dims<N>::AFFINE, 1}, mine);
    }
    __syncthreads();
#pragma unroll 1
    for (int h = 1; h < Teff; h <<= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < Teff)
            affine_compose_view<R, N>(AffineView<R, N>{tree + tslot<R>(j - h), TS},
                                      AffineView<R, N>{tree + tslot<R>(j), TS},
                                      AffineView<R, N>{tree + tslot<R>(j), TS});
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const R x0 = P.x0[i];
            xs[i * TS + tslot<R>(Teff - 1)] = x0;
            if (!P.refine_add) P.x[i] = x0;  // second pass: x*_0 = x^_0 + 0 stays
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = Teff / 2; h >= 1; h >>= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < Teff) {
            R xv[N];
#pragma unroll
            for (int i = 0; i < N; ++i) xv[i] = xs[i * TS + tslot<R>(j)];
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * TS + tslot<R>(j - h)] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{tree + tslot<R>(j - h), TS}, xv);
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * TS + tslot<R>(j)] = xv[i];
        }
        __syncthreads();
    }
    if (t1 > t0) {
        R xv[N];
#pragma unroll
        for (int i = 0; i < N; ++i) xv[i] = xs[i * TS + tslot<R>(tid)];
        for (int t = t0; t < t1; ++t) {
#pragma unroll
            for (int i = 0; i < N; ++i) P.ftile_x[(size_t)t * N + i] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{P.ftile_agg + (size_t)t * Dims<N>::AFFINE, 1}, xv);
        }
    }
}

// ===========================================================================
// fwd_down: in-tile down-sweep of states and the per-chunk rollout.
// First refined pass: also r'_k = r_k - H_k x^_k, c'_k = F_k x^_k + c_k - x^_{k+1}
// (compensated), r'_T and x'_0.  Second pass: x*_{k+1} = x^_{k+1} + xi_{k+1}.
// ===========================================================================
// fwd_down over one tile; sm: the model area, filled here unless SOLO.
// SOLO: the forward tree is already in `big` and the tile starts at x_0
// (Lemma lqt_fwd_init).
template <typename R, int N, int M, int W, bool SOLO>
__device__ __forceinline__ void fwd_down_body(const Params<R>& P, unsigned tile,
                                              unsigned char* smem_raw, R* sm) {
    using SM = Smem<R, N, M, W>;
    using ML = ModelLayout<N, M>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    R* big = reinterpret_cast<R*>(smem_raw + kSmemHead);
    constexpr int WS = SM::WS;
    R* ftree = big;                                      // [AFFINE][WS]
    R* xs = big + (size_t)Dims<N>::AFFINE * WS;          // [N][WS]
    const int tid = threadIdx.x;
    bool ok_load = true;
    if (!SOLO) {
        if (tid == 0) mbar_init(bar, 1);
        model_prologue<R, N, M>(P, sm);
        uint32_t phase = 0;
        ok_load = cta_bulk_load(ftree, P.ftree + (size_t)tile * Dims<N>::AFFINE * WS,
                                (uint32_t)(Dims<N>::AFFINE * WS * sizeof(R)), bar, phase,
                                P.wait_limit);
    }
    const TileGeo geo{P.T, (long long)tile * W, P.B};
    const int Weff = next_pow2(geo.live(W));
    if (tid < N) {
        if (SOLO) {
            const R x0 = P.x0[tid];
            xs[tid * WS + tslot<R>(Weff - 1)] = x0;
            if (!P.refine_add) P.x[tid] = x0;  // second pass: x*_0 = x^_0 + 0 stays
        } else {
            xs[tid * WS + tslot<R>(Weff - 1)] = P.ftile_x[(size_t)tile * N + tid];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = Weff / 2; h >= 1; h >>= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < Weff) {
            R xv[N];
#pragma unroll
            for (int i = 0; i < N; ++i) xv[i] = xs[i * WS + tslot<R>(j)];
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * WS + tslot<R>(j - h)] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{ftree + tslot<R>(j - h), WS}, xv);
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * WS + tslot<R>(j)] = xv[i];
        }
        __syncthreads();
    }
    // The chunk stores its own start state (the tree value) and the states of
    // its steps; the state after its last step is the next chunk's start (or,
    // for the last chunk, its own x_T).  Stored states and the shifted data of
    // the refinement are then consistent to the last bit.
    R x[N], xnext[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        x[i] = xs[i * WS + tslot<R>(tid)];
        xnext[i] = tid + 1 < W ? xs[i * WS + tslot<R>(tid + 1)] : R(0);
    }
    if (!SOLO && tid == W - 1 && tile + 1 < (unsigned)P.tiles) {
#pragma unroll
        for (int i = 0; i < N; ++i) xnext[i] = P.ftile_x[(size_t)(tile + 1) * N + i];
    }
    __syncthreads();  // the big area becomes the warp staging rows

    const int lane = tid & 31, warp = tid >> 5;
    R* rows = big + (size_t)warp * 32 * SM::FROW;
    R* myrow = rows + lane * SM::FROW;
    long long s, e;
    geo.chunk(tid, s, e);
    const long long tbase = geo.chunk0 * P.B;
    const int p = P.p;
    const R* sHm = sm + ML::OH(p);
    const int groups = (P.B + kStageG - 1) / kStageG;
    const bool stage_rp = P.refine_emit && p <= kRStage;  // r' kept with 4 floats per step
    // a time-invariant F, L stays in registers for the whole chunk
    R Fr[N][N], Lr[N][M];
    if (P.dyn_invariant) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) Fr[i][j] = sm[ML::OF + i * N + j];
#pragma unroll
            for (int a = 0; a < M; ++a) Lr[i][a] = sm[ML::OL + i * M + a];
        }
    }
    // inputs of group g into input buffer (g & 1); one cp.async group per call
    auto prefetch = [&](int g) {
        long long lo;
        int cnt;
        fwd_group(s, e, g, lo, cnt);
        const int lrel = (int)(lo - tbase);
        R* in = rows + (g & 1) * SM::FIN;
        WarpRows<R, M * N, kStageG>::load_async_stream(P.K, tbase, in + SM::FIK, SM::FROW, lrel, cnt);
        WarpRows<R, M, kStageG>::load_async(P.u, tbase, in + SM::FID, SM::FROW, lrel, cnt);
        if (P.refine_add)
            WarpRows<R, N, kStageG>::load_async_stream(P.x, tbase, in + SM::FIX, SM::FROW, lrel, cnt);
        cp_async_commit();
    };
    prefetch(0);
    for (int g = 0; g < groups; ++g) {
        if (g + 1 < groups) {
            prefetch(g + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        long long lo;
        int cnt;
        fwd_group(s, e, g, lo, cnt);
        const int lrel = (int)(lo - tbase);
        const R* in = myrow + (g & 1) * SM::FIN;
        for (int jj = 0; jj < cnt; ++jj) {
            const long long k = lo + jj;
            R Kk[M * N], d[M];
            load_row<R, M * N>(in + SM::FIK + jj * M * N, Kk);
            load_row<R, M>(in + SM::FID + jj * M, d);
            if (!P.dyn_invariant) {
                const R* Fg = P.F + k * P.sF;
                const R* Lg = P.L + k * P.sL;
#pragma unroll
                for (int i = 0; i < N; ++i) {
#pragma unroll
                    for (int j = 0; j < N; ++j) Fr[i][j] = __ldg(Fg + i * N + j);
#pragma unroll
                    for (int a = 0; a < M; ++a) Lr[i][a] = __ldg(Lg + i * M + a);
                }
            }
            const R* c = P.has_c ? (P.c_invariant ? sm + ML::OC : P.c + k * P.sc) : nullptr;
            R uk[M];
#pragma unroll
            for (int a = 0; a < M; ++a) {
                R t = d[a];
#pragma unroll
                for (int j = 0; j < N; ++j) t -= Kk[a * N + j] * x[j];
                uk[a] = t;
            }
            R xn[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                R t = c ? c[i] : R(0);
#pragma unroll
                for (int j = 0; j < N; ++j) t += Fr[i][j] * x[j];
#pragma unroll
                for (int a = 0; a < M; ++a) t += Lr[i][a] * uk[a];
                xn[i] = t;
            }
            const bool last_step = (k == e - 1);
            if (last_step && e < P.T) {
#pragma unroll
                for (int i = 0; i < N; ++i) xn[i] = xnext[i];
            }
            if (P.refine_emit) {
                // shifted data of the second pass, each a compensated dot product
                const R* rk = P.r ? P.r + k * P.sr : nullptr;
                const R* Hk = P.cost_invariant ? sHm : P.H + k * P.sH;
                R* rrow = myrow + SM::FR + jj * kRStage;
                for (int a = 0; a < p; ++a) {
                    Dot2<R> acc(rk ? rk[a] : R(0));
#pragma unroll
                    for (int j = 0; j < N; ++j) acc.add_prod(-Hk[a * N + j], x[j]);
                    if (stage_rp)
                        rrow[a] = acc.value();
                    else
                        P.rp[k * p + a] = acc.value();
                }
                if (stage_rp)
                    for (int a = p; a < kRStage; ++a) rrow[a] = R(0);
                R cpk[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    Dot2<R> acc(c ? c[i] : R(0));
#pragma unroll
                    for (int j = 0; j < N; ++j) acc.add_prod(Fr[i][j], x[j]);
                    acc.add(-xn[i]);
                    cpk[i] = acc.value();
                }
                store_row<R, N>(myrow + SM::FC + jj * N, cpk);
            }
            store_row<R, M>(myrow + SM::FU + jj * M, uk);
            // the state record of step k is x_k
            if (P.refine_add) {
                R xh[N], xo[N];
                load_row<R, N>(in + SM::FIX + jj * N, xh);
#pragma unroll
                for (int i = 0; i < N; ++i) xo[i] = add_rn(xh[i], x[i]);
                store_row<R, N>(myrow + SM::FX + jj * N, xo);
            } else {
                store_row<R, N>(myrow + SM::FX + jj * N, x);
            }
            if (k == P.T - 1) {
                // x_T, and the terminal reference of the shifted problem
                R* xT = P.x + (size_t)P.T * N;
                if (P.refine_add) {
#pragma unroll
                    for (int i = 0; i < N; ++i) xT[i] = add_rn(xT[i], xn[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < N; ++i) xT[i] = xn[i];
                }
                if (P.refine_emit)
                    for (int a = 0; a < P.pT; ++a) {
                        Dot2<R> acc(P.rT ? P.rT[a] : R(0));
#pragma unroll
                        for (int j = 0; j < N; ++j) acc.add_prod(-P.HT[a * N + j], xn[j]);
                        P.rTp[a] = acc.value();
                    }
            }
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = xn[i];
        }
        __syncwarp();
        WarpRows<R, N, kStageG>::store(P.x, tbase, rows + SM::FX, SM::FROW, lrel, cnt);
        WarpRows<R, M, kStageG>::store(P.u, tbase, rows + SM::FU, SM::FROW, lrel, cnt);
        if (P.refine_emit) {
            WarpRows<R, N, kStageG>::store(P.cp, tbase, rows + SM::FC, SM::FROW, lrel, cnt);
            if (stage_rp)
                WarpRows<R, kRStage, kStageG>::store(P.rp, tbase, rows + SM::FR, SM::FROW, lrel, cnt);
        }
        __syncwarp();
    }
    if (P.refine_emit && tile == 0 && tid < N) P.x0p[tid] = R(0);
    if (!ok_load) set_status(P.status, ST_TIMEOUT);
}

template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_fwd_down(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    using SM = Smem<R, N, M, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* big = reinterpret_cast<R*>(smem_raw + kSmemHead);
    fwd_down_body<R, N, M, W, false>(P, blockIdx.x, smem_raw, big + SM::FDOWN_BIG + SM::RBUF);
}

// ===========================================================================
// solo: a problem of one tile in one CTA -- the pass's up-sweep, value
// down-sweep with the Riccati re-folds, forward up-sweep and rollout back to
// back (the bodies above with SOLO), the trees kept in shared memory between
// them.  The top-level scans reduce to the terminal value and x_0, so a pass
// is one launch instead of five.
// ===========================================================================
template <typename R, int N, int M, int W>
struct SoloSmem {
    using SM = Smem<R, N, M, W>;
    static constexpr int BIG = SM::DOWN_BIG > SM::FDOWN_BIG ? SM::DOWN_BIG : SM::FDOWN_BIG;
    static_assert(SM::UP_BIG <= BIG, "the up-sweep's tree fits the common area");
    static size_t bytes(int p) { return SM::bytes(BIG, p); }
};

template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_solo(const Params<R> P) {
    griddep_launch_dependents();
    griddep_wait();
    using SM = Smem<R, N, M, W>;
    constexpr int BIG = SoloSmem<R, N, M, W>::BIG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* big = reinterpret_cast<R*>(smem_raw + kSmemHead);
    R* sm = big + BIG + SM::RBUF;
    model_prologue<R, N, M>(P, sm);  // ends with __syncthreads
    bwd_up_body<R, N, M, W, true>(P, 0, big, sm);
    __syncthreads();
    bwd_down_body<R, N, M, W, true>(P, 0, smem_raw, big + BIG + threadIdx.x, sm);
    __syncthreads();
    fwd_down_body<R, N, M, W, true>(P, 0, smem_raw, sm);
}

// ===========================================================================
// Sequential baseline (Sec. II-B): one thread runs the Riccati recursion
// backward and then the forward pass.  K is always written: the forward pass
// reads it back.
// ===========================================================================
template <typename R, int N, int M>
__global__ void __launch_bounds__(32, 1) k_riccati_seq(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    model_prologue<R, N, M>(P, sm);
    if (threadIdx.x != 0) return;
    Value<R, N> val;
    terminal_value<R, N>(P, val);
    bool ok = true;
    {
        R* ST = P.S + (size_t)P.T * N * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (P.out_mask & OUT_S) {
#pragma unroll
                for (int j = 0; j < N; ++j) ST[i * N + j] = val.S[sym<N>(i, j)];
            }
            if (P.out_mask & OUT_V) P.v[(size_t)P.T * N + i] = val.v[i];
        }
    }
    for (long long k = P.T - 1; k >= 0; --k) {
        Step<R, N, M> st;
        load_step<R, N, M>(P, k, sm, nullptr, st);
        R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
        ok &= riccati_step<R, N, M>(st, P.has_c != 0, val.S, val.v, K, d, Ft, ct, Rc, Rinv);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (P.out_mask & OUT_S) {
#pragma unroll
                for (int j = 0; j < N; ++j)
                    P.S[(size_t)k * N * N + i * N + j] = val.S[sym<N>(i, j)];
            }
            if (P.out_mask & OUT_V) P.v[(size_t)k * N + i] = val.v[i];
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
#pragma unroll
            for (int j = 0; j < N; ++j) P.K[(size_t)k * M * N + a * N + j] = K[a][j];
            P.u[(size_t)k * M + a] = d[a];
        }
    }
    R x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        x[i] = P.x0[i];
        if (!P.refine_add) P.x[i] = x[i];
    }
    using ML = ModelLayout<N, M>;
    const int p = P.p;
    const R* sHm = sm + ML::OH(p);
    for (long long k = 0; k < P.T; ++k) {
        const R* F = P.dyn_invariant ? sm + ML::OF : P.F + k * P.sF;
        const R* L = P.dyn_invariant ? sm + ML::OL : P.L + k * P.sL;
        const R* c = P.has_c ? (P.c_invariant ? sm + ML::OC : P.c + k * P.sc) : nullptr;
        R uk[M];
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R t = P.u[(size_t)k * M + a];
#pragma unroll
            for (int j = 0; j < N; ++j) t -= P.K[(size_t)k * M * N + a * N + j] * x[j];
            uk[a] = t;
        }
        R xn[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            R t = c ? c[i] : R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) t += F[i * N + j] * x[j];
#pragma unroll
            for (int a = 0; a < M; ++a) t += L[i * M + a] * uk[a];
            xn[i] = t;
        }
        if (P.refine_emit) {
            const R* rk = P.r ? P.r + k * P.sr : nullptr;
            const R* Hk = P.cost_invariant ? sHm : P.H + k * P.sH;
            const int rps = p <= kRStage ? kRStage : p;
            for (int a = 0; a < p; ++a) {
                Dot2<R> acc(rk ? rk[a] : R(0));
#pragma unroll
                for (int j = 0; j < N; ++j) acc.add_prod(-Hk[a * N + j], x[j]);
                P.rp[k * rps + a] = acc.value();
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                Dot2<R> acc(c ? c[i] : R(0));
#pragma unroll
                for (int j = 0; j < N; ++j) acc.add_prod(F[i * N + j], x[j]);
                acc.add(-xn[i]);
                P.cp[k * N + i] = acc.value();
            }
        }
#pragma unroll
        for (int a = 0; a < M; ++a) P.u[(size_t)k * M + a] = uk[a];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P.x[(size_t)(k + 1) * N + i] = P.refine_add ? add_rn(P.x[(size_t)(k + 1) * N + i], xn[i]) : xn[i];
            x[i] = xn[i];
        }
    }
    if (P.refine_emit) {
        for (int a = 0; a < P.pT; ++a) {
            Dot2<R> acc(P.rT ? P.rT[a] : R(0));
#pragma unroll
            for (int j = 0; j < N; ++j) acc.add_prod(-P.HT[a * N + j], x[j]);
            P.rTp[a] = acc.value();
        }
#pragma unroll
        for (int i = 0; i < N; ++i) P.x0p[i] = R(0);
    }
    if (!ok) set_status(P.status, ST_NOTSPD);
}

}  // namespace lqt
