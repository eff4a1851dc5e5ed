// Kernels of the blocked temporally parallel LQT solve.
//
// Time k = 0..T-1 is cut into chunks of B steps (one thread per chunk) and
// chunks into tiles of W chunks (one CTA per tile).  Block processing
// (Sec. V-C) folds each chunk sequentially; up/down sweeps (Sec. II-C,
// Alg. 1) scan the chunk totals inside a tile (shared memory) and the tile
// totals across the grid (one CTA).  Launch order on one stream:
//
//   bwd_up    a_k built on the fly (eq. lqt_init), chunk fold P <- a_k (x) P
//             (eq. lqt_comb), in-tile up-sweep; writes the tile tree and total.
//   bwd_top   suffix scan of tile totals; the carry into each tile is a value
//             (0, 0, 0, v, S) (Lemma LQT_assoc); writes S_T, v_T.
//   bwd_down  in-tile down-sweep of value carries; per chunk a Riccati re-fold
//             from its carry (S_k = J_{k,T+1}, v_k = eta_{k,T+1}) with the
//             gains of eq. Control_LQT fused; writes S, v, K and the
//             feedforward into u; builds the chunk's closed-loop affine map
//             (Sec. IV-C, Method 1) and the in-tile forward up-sweep.
//   fwd_top   prefix scan of tile affine maps from x_0 (Lemma lqt_fwd_init).
//   fwd_down  in-tile down-sweep of states; per chunk the rollout
//             u*_k = -K_k x*_k + d_k, x*_{k+1} = F_k x*_k + c_k + L_k u*_k.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lqt_dense.cuh"

namespace lqt {

enum : int {
    ST_OK = 0,
    ST_NOTSPD = 2,
    ST_NONFINITE = 3,
    ST_SINGULAR = 8,
};

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
    int B;          // steps per chunk
    int tiles;
    int has_c;
    int cost_invariant;  // H and X time-invariant: H^T X and H^T X H precomputed
    int out_mask;        // OUT_S | OUT_V | OUT_K: which of S, v, K this pass writes
};

enum : int { OUT_S = 1, OUT_V = 2, OUT_K = 4, OUT_ALL = 7 };

__device__ __forceinline__ void set_status(int* status, int code) {
    if (code != ST_OK) atomicCAS(status, 0, code);
}

// Shared-memory cost terms when H, X are time-invariant:
//   sHX[a * N + i] = (H^T X)[i][a]   (p x N)
//   sQ[sym(i, j)]  = (H^T X H)[i][j]
template <typename R, int N>
__device__ __forceinline__ void cost_prologue(const Params<R>& P, R* sQ, R* sHX) {
    if (!P.cost_invariant) return;
    const int p = P.p;
    for (int e = threadIdx.x; e < p * N; e += blockDim.x) {
        const int a = e / N, i = e % N;
        R t = R(0);
        for (int b = 0; b < p; ++b) t += P.H[b * N + i] * P.X[b * p + a];
        sHX[e] = t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e / N, j = e % N;
        if (i > j) continue;
        R t = R(0);
        for (int a = 0; a < p; ++a) t += sHX[a * N + i] * P.H[a * N + j];
        sQ[sym<N>(i, j)] = t;
    }
    __syncthreads();
}

// Step k of the model: F, c, L, U and the cost element Q = H^T X H, q = H^T X r.
template <typename R, int N, int M>
__device__ __forceinline__ void load_step(const Params<R>& P, long long k, const R* sQ,
                                          const R* sHX, Step<R, N, M>& st) {
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
    if (P.has_c) {
        const R* c = P.c + k * P.sc;
#pragma unroll
        for (int i = 0; i < N; ++i) st.c[i] = __ldg(c + i);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) st.c[i] = R(0);
    }
    const int p = P.p;
    const R* r = P.r ? P.r + k * P.sr : nullptr;
    if (P.cost_invariant) {
#pragma unroll
        for (int k2 = 0; k2 < Dims<N>::SYM; ++k2) st.Q[k2] = sQ[k2];
#pragma unroll
        for (int i = 0; i < N; ++i) st.q[i] = R(0);
        if (r) {
            for (int a = 0; a < p; ++a) {
                const R ra = __ldg(r + a);
#pragma unroll
                for (int i = 0; i < N; ++i) st.q[i] += sHX[a * N + i] * ra;
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

template <typename R, int N>
__host__ __device__ constexpr size_t cost_smem_elems(int p) {
    return (size_t)Dims<N>::SYM + (size_t)p * N;
}

// ===========================================================================
// bwd_up: chunk fold + in-tile up-sweep (left-anchored: after level d, slot
// i = j * 2^{d+1} holds the total of chunks [i, i + 2^{d+1}); slot i + 2^d
// keeps the total of [i + 2^d, i + 2^{d+1}) for the down-sweep).
// ===========================================================================
template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_bwd_up(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* tree = reinterpret_cast<R*>(smem_raw);           // [ELEM][W]
    R* sQ = tree + (size_t)Dims<N>::ELEM * W;
    R* sHX = sQ + Dims<N>::SYM;
    cost_prologue<R, N>(P, sQ, sHX);

    const int tid = threadIdx.x;
    const long long chunk = (long long)blockIdx.x * W + tid;
    const long long s = chunk * P.B;
    const long long e = min(s + (long long)P.B, P.T);
    Elem<R, N> acc;
    set_neutral(acc);
    bool ok = true;
    for (long long k = e - 1; k >= s; --k) {
        Step<R, N, M> st;
        load_step<R, N, M>(P, k, sQ, sHX, st);
        ok &= fold_step<R, N, M>(st, P.has_c != 0, acc);
    }
    store_elem(acc, ElemView<R, N>{tree + tid, W});
    __syncthreads();
    bool ok2 = true;
#pragma unroll 1
    for (int h = 1; h < W; h <<= 1) {
        const int i = tid * 2 * h;
        if (i < W)
            ok2 &= combine_view<R, N>(ElemView<R, N>{tree + i, W}, ElemView<R, N>{tree + i + h, W},
                                      ElemView<R, N>{tree + i, W});
        __syncthreads();
    }
    R* g = P.tree + (size_t)blockIdx.x * Dims<N>::ELEM * W;
    for (int k = tid; k < Dims<N>::ELEM * W; k += W) g[k] = tree[k];
    if (tid < Dims<N>::ELEM) P.tile_agg[(size_t)blockIdx.x * Dims<N>::ELEM + tid] = tree[tid * W];
    if (!ok) set_status(P.status, ST_NOTSPD);
    if (!ok2) set_status(P.status, ST_SINGULAR);
}

// ===========================================================================
// bwd_top: one CTA of TP threads.  Thread t folds tiles [t g, (t+1) g)
// (g = ceil(tiles / TP)), the CTA sweeps the TP partial totals, and the value
// carries flow back from the terminal value (S_T, v_T) of Lemma LQT_assoc.
// ===========================================================================
template <typename R, int N, int TP>
__global__ void __launch_bounds__(TP, 1) k_bwd_top(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* tree = reinterpret_cast<R*>(smem_raw);            // [ELEM][TP]
    R* carry = tree + (size_t)Dims<N>::ELEM * TP;        // [VALUE][TP]
    const int tid = threadIdx.x;
    const int tiles = P.tiles;
    const int g = (tiles + TP - 1) / TP;
    const int t0 = min(tid * g, tiles), t1 = min(t0 + g, tiles);
    bool ok = true;

    // thread partial: tile totals t0..t1-1 folded right to left, in shared
    // memory slot tid (neutral when the range is empty)
    {
        ElemView<R, N> mine{tree + tid, TP};
        if (t1 > t0) {
            const R* src = P.tile_agg + (size_t)(t1 - 1) * Dims<N>::ELEM;
            for (int k = 0; k < Dims<N>::ELEM; ++k) mine.p[k * TP] = src[k];
            // fold further tiles in from the left, through the carry area as scratch
            R* scratch = carry + tid;  // VALUE >= ... not enough room: use a second pass below
            (void)scratch;
        } else {
            Elem<R, N> e;
            set_neutral(e);
            store_elem(e, mine);
        }
    }
    __syncthreads();
    // g > 1: fold the remaining tiles of this thread into its slot, one at a
    // time, staging the left operand in global tile_agg (read-only) directly.
    if (g > 1) {
        for (int t = t1 - 2; t >= t0; --t) {
            ok &= combine_view<R, N>(
                ElemView<R, N>{const_cast<R*>(P.tile_agg) + (size_t)t * Dims<N>::ELEM, 1},
                ElemView<R, N>{tree + tid, TP}, ElemView<R, N>{tree + tid, TP});
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = 1; h < TP; h <<= 1) {
        const int i = tid * 2 * h;
        if (i < TP)
            ok &= combine_view<R, N>(ElemView<R, N>{tree + i, TP}, ElemView<R, N>{tree + i + h, TP},
                                     ElemView<R, N>{tree + i, TP});
        __syncthreads();
    }
    // terminal value: S_T = H_T^T X_T H_T, v_T = H_T^T X_T r_T
    if (tid == 0) {
        const int pT = P.pT;
        Value<R, N> z;
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
        store_value(z, ValueView<R, N>{carry, TP});
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
    __syncthreads();
#pragma unroll 1
    for (int h = TP / 2; h >= 1; h >>= 1) {
        const int i = tid * 2 * h;
        if (i < TP) {
            Value<R, N> c;
            load_value(c, ValueView<R, N>{carry + i, TP});
            store_value(c, ValueView<R, N>{carry + i + h, TP});
            ok &= value_apply<R, N>(ElemView<R, N>{tree + i + h, TP}, c);
            store_value(c, ValueView<R, N>{carry + i, TP});
        }
        __syncthreads();
    }
    // per-tile carries for this thread's tiles
    if (t1 > t0) {
        Value<R, N> c;
        load_value(c, ValueView<R, N>{carry + tid, TP});
        for (int t = t1 - 1; t >= t0; --t) {
            store_value(c, ValueView<R, N>{P.tile_carry + (size_t)t * Dims<N>::VALUE, 1});
            if (t > t0)
                ok &= value_apply<R, N>(
                    ElemView<R, N>{const_cast<R*>(P.tile_agg) + (size_t)t * Dims<N>::ELEM, 1}, c);
        }
    }
    if (!ok) set_status(P.status, ST_SINGULAR);
}

// ===========================================================================
// bwd_down: in-tile down-sweep of values, Riccati re-fold per chunk with the
// gains fused, and the forward affine up-sweep (right-anchored).
// ===========================================================================
template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_bwd_down(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* tree = reinterpret_cast<R*>(smem_raw);               // [ELEM][W]
    R* carry = tree + (size_t)Dims<N>::ELEM * W;            // [VALUE][W]
    R* sQ = carry + (size_t)Dims<N>::VALUE * W;
    R* sHX = sQ + Dims<N>::SYM;
    R* ftree = tree;  // [AFFINE][W], reuses the element tree once it is consumed
    cost_prologue<R, N>(P, sQ, sHX);

    const int tid = threadIdx.x;
    const R* g = P.tree + (size_t)blockIdx.x * Dims<N>::ELEM * W;
    for (int k = tid; k < Dims<N>::ELEM * W; k += W) tree[k] = g[k];
    if (tid < Dims<N>::VALUE)
        carry[tid * W] = P.tile_carry[(size_t)blockIdx.x * Dims<N>::VALUE + tid];
    __syncthreads();
    bool ok_sing = true;
#pragma unroll 1
    for (int h = W / 2; h >= 1; h >>= 1) {
        const int i = tid * 2 * h;
        if (i < W) {
            Value<R, N> c;
            load_value(c, ValueView<R, N>{carry + i, W});
            store_value(c, ValueView<R, N>{carry + i + h, W});
            ok_sing &= value_apply<R, N>(ElemView<R, N>{tree + i + h, W}, c);
            store_value(c, ValueView<R, N>{carry + i, W});
        }
        __syncthreads();
    }
    Value<R, N> val;
    load_value(val, ValueView<R, N>{carry + tid, W});
    __syncthreads();  // tree and carry slots are reused below

    const long long chunk = (long long)blockIdx.x * W + tid;
    const long long s = chunk * P.B;
    const long long e = min(s + (long long)P.B, P.T);
    R Phi[N][N], gam[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) Phi[i][j] = (i == j) ? R(1) : R(0);
        gam[i] = R(0);
    }
    bool ok = true, finite = true;
    for (long long k = e - 1; k >= s; --k) {
        Step<R, N, M> st;
        load_step<R, N, M>(P, k, sQ, sHX, st);
        R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
        ok &= riccati_step<R, N, M>(st, P.has_c != 0, val.S, val.v, K, d, Ft, ct, Rc, Rinv);
        // outputs at step k
        R Sk[N * N];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) Sk[i * N + j] = val.S[sym<N>(i, j)];
        if (P.out_mask & OUT_S) store_row<R, N * N>(P.S + (size_t)k * N * N, Sk);
        if (P.out_mask & OUT_V) store_row<R, N>(P.v + (size_t)k * N, val.v);
        if (P.out_mask & OUT_K) {
            R Kk[M * N];
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int j = 0; j < N; ++j) Kk[a * N + j] = K[a][j];
            store_row<R, M * N>(P.K + (size_t)k * M * N, Kk);
        }
        store_row<R, M>(P.u + (size_t)k * M, d);
#pragma unroll
        for (int i = 0; i < N; ++i) finite = finite && isfinite(val.v[i]) && isfinite(Sk[i * N + i]);
        // chunk map: x_e = Phi x_{k} + gam after adding step k
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
    // forward up-sweep (right-anchored): after level d, slot j = i + 2^{d+1} - 1
    // holds the composite of chunks [i, i + 2^{d+1}); slot i + 2^d - 1 keeps [i, i + 2^d)
    {
        AffineView<R, N> mine{ftree + tid, W};
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) mine.F(i, j) = Phi[i][j];
            mine.c(i) = gam[i];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = 1; h < W; h <<= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < W)
            affine_compose_view<R, N>(AffineView<R, N>{ftree + j - h, W}, AffineView<R, N>{ftree + j, W},
                                      AffineView<R, N>{ftree + j, W});
        __syncthreads();
    }
    R* fg = P.ftree + (size_t)blockIdx.x * Dims<N>::AFFINE * W;
    for (int k = tid; k < Dims<N>::AFFINE * W; k += W) fg[k] = ftree[k];
    if (tid < Dims<N>::AFFINE)
        P.ftile_agg[(size_t)blockIdx.x * Dims<N>::AFFINE + tid] = ftree[tid * W + W - 1];
    if (!ok) set_status(P.status, ST_NOTSPD);
    if (!finite) set_status(P.status, ST_NONFINITE);
    if (!ok_sing) set_status(P.status, ST_SINGULAR);
}

// ===========================================================================
// fwd_top: one CTA of TP threads; prefix scan of tile affine maps seeded with
// x_0 (Lemma lqt_fwd_init: the first element maps everything to the state).
// ===========================================================================
template <typename R, int N, int TP>
__global__ void __launch_bounds__(TP, 1) k_fwd_top(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* tree = reinterpret_cast<R*>(smem_raw);      // [AFFINE][TP]
    R* xs = tree + (size_t)Dims<N>::AFFINE * TP;   // [N][TP]
    const int tid = threadIdx.x;
    const int tiles = P.tiles;
    const int g = (tiles + TP - 1) / TP;
    const int t0 = min(tid * g, tiles), t1 = min(t0 + g, tiles);
    {
        AffineView<R, N> mine{tree + tid, TP};
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
    for (int h = 1; h < TP; h <<= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < TP)
            affine_compose_view<R, N>(AffineView<R, N>{tree + j - h, TP}, AffineView<R, N>{tree + j, TP},
                                      AffineView<R, N>{tree + j, TP});
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const R x0 = P.x0[i];
            xs[i * TP + TP - 1] = x0;
            P.x[i] = x0;
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = TP / 2; h >= 1; h >>= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < TP) {
            R xv[N];
#pragma unroll
            for (int i = 0; i < N; ++i) xv[i] = xs[i * TP + j];
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * TP + j - h] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{tree + j - h, TP}, xv);
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * TP + j] = xv[i];
        }
        __syncthreads();
    }
    if (t1 > t0) {
        R xv[N];
#pragma unroll
        for (int i = 0; i < N; ++i) xv[i] = xs[i * TP + tid];
        for (int t = t0; t < t1; ++t) {
#pragma unroll
            for (int i = 0; i < N; ++i) P.ftile_x[(size_t)t * N + i] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{P.ftile_agg + (size_t)t * Dims<N>::AFFINE, 1}, xv);
        }
    }
}

// ===========================================================================
// fwd_down: in-tile down-sweep of states and the per-chunk rollout.
// ===========================================================================
template <typename R, int N, int M, int W>
__global__ void __launch_bounds__(W, 1) k_fwd_down(const Params<R> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* ftree = reinterpret_cast<R*>(smem_raw);      // [AFFINE][W]
    R* xs = ftree + (size_t)Dims<N>::AFFINE * W;    // [N][W]
    const int tid = threadIdx.x;
    const R* fg = P.ftree + (size_t)blockIdx.x * Dims<N>::AFFINE * W;
    for (int k = tid; k < Dims<N>::AFFINE * W; k += W) ftree[k] = fg[k];
    if (tid < N) xs[tid * W + W - 1] = P.ftile_x[(size_t)blockIdx.x * N + tid];
    __syncthreads();
#pragma unroll 1
    for (int h = W / 2; h >= 1; h >>= 1) {
        const int j = tid * 2 * h + 2 * h - 1;
        if (j < W) {
            R xv[N];
#pragma unroll
            for (int i = 0; i < N; ++i) xv[i] = xs[i * W + j];
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * W + j - h] = xv[i];
            affine_apply_view<R, N>(AffineView<R, N>{ftree + j - h, W}, xv);
#pragma unroll
            for (int i = 0; i < N; ++i) xs[i * W + j] = xv[i];
        }
        __syncthreads();
    }
    R x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = xs[i * W + tid];
    const long long chunk = (long long)blockIdx.x * W + tid;
    const long long s = chunk * P.B;
    const long long e = min(s + (long long)P.B, P.T);
    for (long long k = s; k < e; ++k) {
        R Kk[M * N], d[M];
        load_row<R, M * N>(P.K + (size_t)k * M * N, Kk);
        load_row<R, M>(P.u + (size_t)k * M, d);
        const R* F = P.F + k * P.sF;
        const R* L = P.L + k * P.sL;
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
            R t = P.has_c ? __ldg(P.c + k * P.sc + i) : R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) t += __ldg(F + i * N + j) * x[j];
#pragma unroll
            for (int a = 0; a < M; ++a) t += __ldg(L + i * M + a) * uk[a];
            xn[i] = t;
        }
        store_row<R, M>(P.u + (size_t)k * M, uk);
        store_row<R, N>(P.x + (size_t)(k + 1) * N, xn);
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = xn[i];
    }
}

// ===========================================================================
// Sequential baseline (Sec. II-B): one thread runs the Riccati recursion
// backward and then the forward pass.  K is always written: the forward pass
// reads it back.
// ===========================================================================
template <typename R, int N, int M>
__global__ void __launch_bounds__(32, 1) k_riccati_seq(const Params<R> P) {
    __shared__ R sQ[Dims<N>::SYM];
    __shared__ R sHX[64 * N];
    if (threadIdx.x == 0 && P.cost_invariant) {
        // H^T X and H^T X H (p <= 64 here; the host checks)
        const int p = P.p;
        for (int a = 0; a < p; ++a)
            for (int i = 0; i < N; ++i) {
                R t = R(0);
                for (int b = 0; b < p; ++b) t += P.H[b * N + i] * P.X[b * p + a];
                sHX[a * N + i] = t;
            }
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                R t = R(0);
                for (int a = 0; a < p; ++a) t += sHX[a * N + i] * P.H[a * N + j];
                sQ[sym<N>(i, j)] = t;
            }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    Value<R, N> val;
    {
        const int pT = P.pT;
#pragma unroll
        for (int k = 0; k < Dims<N>::SYM; ++k) val.S[k] = R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) val.v[i] = R(0);
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
                val.v[i] += h * xr;
#pragma unroll
                for (int j = i; j < N; ++j) val.S[sym<N>(i, j)] += h * y[j];
            }
        }
    }
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
        load_step<R, N, M>(P, k, sQ, sHX, st);
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
        P.x[i] = x[i];
    }
    for (long long k = 0; k < P.T; ++k) {
        const R* F = P.F + k * P.sF;
        const R* L = P.L + k * P.sL;
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
            R t = P.has_c ? P.c[k * P.sc + i] : R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) t += F[i * N + j] * x[j];
#pragma unroll
            for (int a = 0; a < M; ++a) t += L[i * M + a] * uk[a];
            xn[i] = t;
        }
#pragma unroll
        for (int a = 0; a < M; ++a) P.u[(size_t)k * M + a] = uk[a];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P.x[(size_t)(k + 1) * N + i] = xn[i];
            x[i] = xn[i];
        }
    }
    if (!ok) set_status(P.status, ST_NOTSPD);
}

}  // namespace lqt
