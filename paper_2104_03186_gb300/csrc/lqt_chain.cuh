// Chunked single-problem pipeline for the lane-group sizes (n = 8, 16, 32).
//
// The T steps are cut into NC chunks (NC a power of two) of B steps; one lane
// group of N lanes (lane r owns row r) works on one chunk at a time, and the
// scans over the NC chunk results run level by level, one launch per level,
// with the chunk results in global memory.  Per pass:
//   k_cfold    chunk totals a_s (x) ... (x) a_{e-1} (eq. lqt_comb), folded one
//              step at a time from the end in the low-rank form of fold_step,
//   k_cup      up-sweep levels of the chunk totals (Alg. 1, left-anchored),
//   k_cterm    the terminal value (H_T^T X_T r_T, H_T^T X_T H_T),
//   k_cdown    down-sweep levels of the value carries (Lemma LQT_assoc: a
//              suffix applied to the value element (0, 0, 0, v, S)),
//   k_crefold  per chunk the Riccati recursion from its carry (Sec. II-B),
//              writing S_k, v_k, K_k and the feedforward d_k, and the chunk's
//              closed-loop affine map (Sec. IV-C),
//   k_cfup / k_cfdown  up- and down-sweeps of the affine maps from x_0
//              (right-anchored), giving every chunk's start state,
//   k_croll    per chunk the rollout of x*_k and u*_k (eq. Control_LQT).
// The chunk phases compute in R; the tree levels store and compute in RT
// (RT = double with R = float is the mixed-precision form: FP32 chunk work,
// FP64 tree levels and their (I + C J) solves).  k_cresid forms the shifted
// problem of the refinement pass (lqt_refine.cuh).
#pragma once

#include <cuda_runtime.h>

#include "lqt_lane_step.cuh"
#include "lqt_refine.cuh"

namespace lqt {
namespace chain {

using namespace lanes;

constexpr int kStatusSingular = 8;  // LQT_ESINGULAR

template <typename R, typename RT>
struct Args {
    DescT<R> D;
    long long B;  // steps per chunk
    int NC;       // chunks (a power of two)
    RT* E;        // NC chunk totals (LElem)
    RT* V;        // NC value carries (LValue): the value at each chunk's end
    RT* FE;       // NC chunk affine maps (LAffine)
    RT* X;        // NC chunk start states
    int* status;
    int out_mask;    // 1: write S, v, K (the refinement pass does not)
    int refine_add;  // 1: x <- x + xi (refinement pass)
};

// ---- shared-memory sizes per group (elements of the kernel's arithmetic type)
template <int N, int M>
struct FoldSmem {  // P | step (E, L, U) | scratch overlapping the step's Y
    static constexpr int P = 0;
    static constexpr int SB = LElem<N>::SIZE;
    static constexpr int SCR_OFF = SB + StepLayout<N, M>::Y;
    static constexpr int SCR = fold_scratch<N, M>() > StepLayout<N, M>::SIZE - StepLayout<N, M>::Y
                                   ? fold_scratch<N, M>()
                                   : StepLayout<N, M>::SIZE - StepLayout<N, M>::Y;
    static constexpr int SIZE = SCR_OFF + SCR;
};

template <int N, int M>
struct RefoldSmem {  // val | Phi | step | scratch (riccati + Kd + Ft) overlapping Y
    static constexpr int VAL = 0;
    static constexpr int PHI = LValue<N>::SIZE;
    static constexpr int SB = PHI + LAffine<N>::SIZE;
    static constexpr int SCR_OFF = SB + StepLayout<N, M>::Y;
    static constexpr int RIC = riccati_scratch<N, M>() + M * (N + 1) + LAffine<N>::SIZE;
    static constexpr int SCR = RIC > StepLayout<N, M>::SIZE - StepLayout<N, M>::Y
                                   ? RIC
                                   : StepLayout<N, M>::SIZE - StepLayout<N, M>::Y;
    static constexpr int SIZE = SCR_OFF + SCR;
};

template <int N>
struct UpSmem {
    static constexpr int SIZE = 2 * LElem<N>::SIZE + combine_scratch<N>();
};

template <int N>
struct DownSmem {
    static constexpr int SIZE = LElem<N>::SIZE + LValue<N>::SIZE + 4 * N * N + 2 * N;
};

template <int N>
struct FupSmem {
    static constexpr int SIZE = 2 * LAffine<N>::SIZE;
};

template <int N>
struct FdownSmem {
    static constexpr int SIZE = LAffine<N>::SIZE + N;
};

template <int N, int M>
struct RollSmem {
    static constexpr int SIZE = N + M;
};

// Groups per CTA: at most 256 threads and about 100 KB of shared memory.
template <int N>
constexpr int groups_for(int bytes_per_group) {
    int g = 256 / N;
    while (g > 1 && g * bytes_per_group > 100 * 1024) --g;
    return g;
}

template <typename A, typename B>
__device__ __forceinline__ void copy_in(A* dst, const B* src, int count, int lr, int lanes) {
    for (int i = lr; i < count; i += lanes) dst[i] = static_cast<A>(src[i]);
}

__device__ __forceinline__ void flag(int* status, bool ok) {
    if (!ok) atomicCAS(status, 0, kStatusSingular);
}

// ---- chunk totals ----------------------------------------------------------
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_cfold(Args<R, RT> a) {
    using S = FoldSmem<N, M>;
    using E = LElem<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sh = reinterpret_cast<R*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long c = (long long)blockIdx.x * NG + gi;
    if (c >= a.NC) return;
    R* gs = sh + gi * S::SIZE;
    R* P = gs + S::P;
    R* sb = gs + S::SB;
    R* scr = gs + S::SCR_OFF;
    const long long T = a.D.T;
    const long long s0 = c * a.B < T ? c * a.B : T;
    const long long e0 = s0 + a.B < T ? s0 + a.B : T;
    bool ok = true;
    set_neutral<N, N>(P, g);
    for (long long k = e0 - 1; k >= s0; --k) {
        load_step<R, N, M, false>(a.D, k, sb, scr, g, ok);
        ok &= fold_step<R, N, M>(P, sb, scr, g);
    }
    RT* out = a.E + c * E::SIZE;
    for (int i = g.lr; i < E::SIZE; i += N) out[i] = static_cast<RT>(P[i]);
    flag(a.status, ok);
}

// ---- up-sweep level h: E[i] <- E[i] (x) E[i + h], i a multiple of 2h -------
template <typename RT, int N, int NG>
__global__ void __launch_bounds__(NG* N) k_cup(RT* E_, int NC, int h, int* status) {
    using E = LElem<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RT* sh = reinterpret_cast<RT*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long i = ((long long)blockIdx.x * NG + gi) * 2 * h;
    if (i + h >= NC) return;
    RT* e1 = sh + gi * UpSmem<N>::SIZE;
    RT* e2 = e1 + E::SIZE;
    RT* scr = e2 + E::SIZE;
    copy_in(e1, E_ + i * E::SIZE, E::SIZE, g.lr, N);
    copy_in(e2, E_ + (i + h) * E::SIZE, E::SIZE, g.lr, N);
    g.sync();
    const bool ok = combine<N, N>(e1, e2, e1, scr, g);
    RT* out = E_ + i * E::SIZE;
    for (int t = g.lr; t < E::SIZE; t += N) out[t] = e1[t];
    flag(status, ok);
}

// ---- terminal value into V[0] (and S_T, v_T) -------------------------------
template <typename R, typename RT, int N>
__global__ void __launch_bounds__(N) k_cterm(Args<R, RT> a) {
    const DescT<R>& D = a.D;
    const int r = threadIdx.x;
    RT acc[N];
    RT t = RT(0);
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = RT(0);
    for (int i = 0; i < D.pT; ++i) {
        const RT hi = static_cast<RT>(D.HT[i * N + r]);
        for (int b = 0; b < D.pT; ++b) {
            const RT hx = hi * static_cast<RT>(D.XT[i * D.pT + b]);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += hx * static_cast<RT>(D.HT[b * N + j]);
            if (D.rT) t += hx * static_cast<RT>(D.rT[b]);
        }
    }
    RT* val = a.V;
#pragma unroll
    for (int j = 0; j < N; ++j) val[LValue<N>::OS + r * N + j] = acc[j];
    val[LValue<N>::OV + r] = t;
    if (a.out_mask) {
#pragma unroll
        for (int j = 0; j < N; ++j) D.S[D.T * N * N + r * N + j] = static_cast<R>(acc[j]);
        D.v[D.T * N + r] = static_cast<R>(t);
    }
}

// ---- down-sweep level h: V[i + h] <- V[i]; V[i] <- E[i + h] (x) V[i] --------
template <typename RT, int N, int NG>
__global__ void __launch_bounds__(NG* N) k_cdown(const RT* E_, RT* V_, int NC, int h,
                                                 int* status) {
    using E = LElem<N>;
    using V = LValue<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RT* sh = reinterpret_cast<RT*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long i = ((long long)blockIdx.x * NG + gi) * 2 * h;
    if (i + h >= NC) return;
    RT* e = sh + gi * DownSmem<N>::SIZE;
    RT* val = e + E::SIZE;
    RT* scr = val + V::SIZE;
    copy_in(e, E_ + (i + h) * E::SIZE, E::SIZE, g.lr, N);
    copy_in(val, V_ + i * V::SIZE, V::SIZE, g.lr, N);
    for (int t = g.lr; t < V::SIZE; t += N) V_[(i + h) * V::SIZE + t] = V_[i * V::SIZE + t];
    g.sync();
    const bool ok = value_apply<N, N>(e, val, scr, g);
    for (int t = g.lr; t < V::SIZE; t += N) V_[i * V::SIZE + t] = val[t];
    flag(status, ok);
}

// ---- per-chunk Riccati re-fold with outputs and the chunk affine map -------
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_crefold(Args<R, RT> a) {
    using S = RefoldSmem<N, M>;
    using V = LValue<N>;
    using A = LAffine<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sh = reinterpret_cast<R*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long c = (long long)blockIdx.x * NG + gi;
    if (c >= a.NC) return;
    const DescT<R>& D = a.D;
    R* gs = sh + gi * S::SIZE;
    R* val = gs + S::VAL;
    R* Phi = gs + S::PHI;
    R* sb = gs + S::SB;
    R* scr = gs + S::SCR_OFF;
    R* Kd = scr + riccati_scratch<N, M>();
    R* Ft = Kd + M * (N + 1);
    const int r = g.lr;
    const long long T = D.T;
    const long long s0 = c * a.B < T ? c * a.B : T;
    const long long e0 = s0 + a.B < T ? s0 + a.B : T;
    copy_in(val, a.V + c * V::SIZE, V::SIZE, r, N);
#pragma unroll
    for (int j = 0; j < N; ++j) Phi[A::OF + r * N + j] = r == j ? R(1) : R(0);
    Phi[A::OC + r] = R(0);
    g.sync();
    bool ok = true;
    for (long long k = e0 - 1; k >= s0; --k) {
        load_step<R, N, M, false>(D, k, sb, scr, g, ok);
        ok &= riccati<R, N, M>(val, sb, Kd, Ft, scr, g);
        if (a.out_mask) {
#pragma unroll
            for (int j = 0; j < N; ++j) D.S[k * N * N + r * N + j] = val[V::OS + r * N + j];
            D.v[k * N + r] = val[V::OV + r];
        }
        if (r < M) {
            if (a.out_mask) {
#pragma unroll
                for (int j = 0; j < N; ++j) D.K[k * M * N + r * N + j] = Kd[r * (N + 1) + j];
            }
            D.u[k * M + r] = Kd[r * (N + 1) + N];  // feedforward d_k, replaced in the rollout
        }
        // chunk map after adding step k: Phi <- Phi Ft, gamma <- gamma + Phi ct
        R pn[N];
        R gm = Phi[A::OC + r];
#pragma unroll
        for (int j = 0; j < N; ++j) pn[j] = R(0);
#pragma unroll 4
        for (int l = 0; l < N; ++l) {
            const R pl = Phi[A::OF + r * N + l];
#pragma unroll
            for (int j = 0; j < N; ++j) pn[j] += pl * Ft[A::OF + l * N + j];
            gm += pl * Ft[A::OC + l];
        }
        g.sync();
#pragma unroll
        for (int j = 0; j < N; ++j) Phi[A::OF + r * N + j] = pn[j];
        Phi[A::OC + r] = gm;
        g.sync();
    }
    RT* out = a.FE + c * A::SIZE;
    for (int t = r; t < A::SIZE; t += N) out[t] = static_cast<RT>(Phi[t]);
    flag(a.status, ok);
}

// ---- forward up-sweep level h: FE[j] <- FE[j] o FE[j - h], j = 2h q + 2h - 1
template <typename RT, int N, int NG>
__global__ void __launch_bounds__(NG* N) k_cfup(RT* FE, int NC, int h) {
    using A = LAffine<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RT* sh = reinterpret_cast<RT*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long j = ((long long)blockIdx.x * NG + gi) * 2 * h + 2 * h - 1;
    if (j >= NC) return;
    RT* f1 = sh + gi * FupSmem<N>::SIZE;
    RT* f2 = f1 + A::SIZE;
    copy_in(f1, FE + (j - h) * A::SIZE, A::SIZE, g.lr, N);
    copy_in(f2, FE + j * A::SIZE, A::SIZE, g.lr, N);
    g.sync();
    affine_compose<N, N>(f1, f2, f2, f1, g);
    for (int t = g.lr; t < A::SIZE; t += N) FE[j * A::SIZE + t] = f2[t];
}

// ---- forward down-sweep level h: X[j - h] <- X[j]; X[j] <- FE[j - h](X[j]) -
template <typename R, typename RT, int N, int NG>
__global__ void __launch_bounds__(NG* N) k_cfdown(const RT* FE, RT* X, const R* x0, int NC, int h,
                                                  int top) {
    using A = LAffine<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RT* sh = reinterpret_cast<RT*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long j = ((long long)blockIdx.x * NG + gi) * 2 * h + 2 * h - 1;
    if (j >= NC) return;
    RT* f = sh + gi * FdownSmem<N>::SIZE;
    RT* x = f + A::SIZE;
    const int r = g.lr;
    copy_in(f, FE + (j - h) * A::SIZE, A::SIZE, r, N);
    const RT xv = top ? static_cast<RT>(x0[r]) : X[j * N + r];
    x[r] = xv;
    X[(j - h) * N + r] = xv;
    g.sync();
    affine_apply<N, N>(f, x, g);
    X[j * N + r] = x[r];
}

// ---- per-chunk rollout of x*_k and u*_k ------------------------------------
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_croll(Args<R, RT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sh = reinterpret_cast<R*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long c = (long long)blockIdx.x * NG + gi;
    if (c >= a.NC) return;
    const DescT<R>& D = a.D;
    R* xc = sh + gi * RollSmem<N, M>::SIZE;
    R* us = xc + N;
    const int r = g.lr;
    const long long T = D.T;
    const long long s0 = c * a.B < T ? c * a.B : T;
    const long long e0 = s0 + a.B < T ? s0 + a.B : T;
    xc[r] = c == 0 ? D.x0[r] : static_cast<R>(a.X[c * N + r]);
    g.sync();
    for (long long k = s0; k < e0; ++k) {
        const R* F = D.F + k * D.sF;
        const R* Lk = D.L + k * D.sL;
        const R xr = xc[r];
        D.x[k * N + r] = a.refine_add ? D.x[k * N + r] + xr : xr;
        // u = d - K x (lanes a < M), published through shared memory
        if (r < M) {
            R t = D.u[k * M + r];
#pragma unroll
            for (int j = 0; j < N; ++j) t -= D.K[k * M * N + r * N + j] * xc[j];
            us[r] = t;
            D.u[k * M + r] = t;
        }
        g.sync();
        R t = D.c ? D.c[k * D.sc + r] : R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) t += __ldg(F + r * N + j) * xc[j];
#pragma unroll
        for (int b = 0; b < M; ++b) t += __ldg(Lk + r * M + b) * us[b];
        g.sync();
        xc[r] = t;
        g.sync();
        if (k == T - 1) D.x[T * N + r] = a.refine_add ? D.x[T * N + r] + t : t;
    }
    if (T == 0 && c == 0) D.x[r] = D.x0[r];
}

// ---- shifted problem of the refinement pass ---------------------------------
// Step k (one group per step, k = 0..T; k = T forms r'_T and x'_0):
//   r'_k = r_k - H_k x^_k,  c'_k = F_k x^_k + c_k - x^_{k+1}
// as compensated dot products (Dot2) of the first pass's trajectory x^.
template <typename R, int N, int NG>
__global__ void __launch_bounds__(NG* N) k_cresid(DescT<R> D, R* rp, R* cp, R* rTp, R* x0p) {
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const int r = g.lr;
    const long long T = D.T;
    const long long stride = (long long)gridDim.x * NG;
    for (long long k = (long long)blockIdx.x * NG + gi; k <= T; k += stride) {
        const R* xk = D.x + k * N;
        if (k == T) {
            for (int i = r; i < D.pT; i += N) {
                Dot2<R> d(D.rT ? D.rT[i] : R(0));
                for (int j = 0; j < N; ++j) d.add_prod(-D.HT[i * N + j], xk[j]);
                rTp[i] = d.value();
            }
            x0p[r] = R(0);
            continue;
        }
        const R* H = D.H + k * D.sH;
        for (int i = r; i < D.p; i += N) {
            Dot2<R> d(D.r ? D.r[k * D.sr + i] : R(0));
            for (int j = 0; j < N; ++j) d.add_prod(-H[i * N + j], xk[j]);
            rp[k * D.p + i] = d.value();
        }
        const R* F = D.F + k * D.sF;
        Dot2<R> d(D.c ? D.c[k * D.sc + r] : R(0));
        for (int j = 0; j < N; ++j) d.add_prod(F[r * N + j], xk[j]);
        d.add(-xk[N + r]);
        cp[k * N + r] = d.value();
    }
}

}  // namespace chain
}  // namespace lqt
