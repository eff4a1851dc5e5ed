// Warm solve: a problem whose matrices are those of an earlier solve shifted
// by s steps (a receding horizon over the same model and terminal weights).
// S_k and K_k depend only on F, L, U, H, X and the terminal weights, not on
// r, c or x_0 (Sec. II-B: the recursion for S_k never reads the vectors), so
// they are the earlier solve's S_{s+k} and K_{s+k}; only the vector parts of
// the value function, the feedforward and the trajectory are computed.  With
// the closed loop Ft_k = F_k - L_k K_k and G_k = L_k^T S_{k+1} L_k + U_k
// (Sec. II-B, eq. Control_LQT):
//   v_T = H_T^T X_T r_T,
//   w_k = v_{k+1} - S_{k+1} c_k,
//   v_k = Ft_k^T w_k + H_k^T X_k r_k,      d_k = G_k^{-1} L_k^T w_k,
//   x_{k+1} = F_k x_k + c_k + L_k u_k,     u_k = -K_k x_k + d_k.
// Both recursions are affine, so they are scanned like the trajectory of
// Sec. IV-C, on the chunks of the chunked pipeline (lqt_chain.cuh):
//   k_wfold    per chunk [s, e), walking back from v_e: the map
//              v_s = Psi v_e + beta with Psi = Ft_s^T ... Ft_{e-1}^T, stored at
//              the chunk's mirrored slot so that the forward scan kernels
//              (k_cfup, k_cfdown) compose the maps from the last chunk to the
//              first, seeded with v_T (k_wterm);
//   k_wrefold  per chunk, from its v_e: v_k and d_k step by step, then the
//              chunk's forward map x_e = Psi^T x_s + gamma (Psi^T = Ft_{e-1}
//              ... Ft_s is the closed-loop chunk map) by a rollout from 0;
//   k_wseed    x_0 into the top slot; the forward scan and k_croll follow.
// Per step this costs one n x n product (Psi) and the m x m solve for d_k,
// against the two folds and the Riccati step of a full solve.
#pragma once

#include <cuda_runtime.h>

#include "lqt_chain.cuh"

namespace lqt {
namespace chain {

using namespace lanes;

// Shared memory of one group of the warm kernels (elements of R).
template <int N, int M>
struct WarmSmem {
    static constexpr int LD = lds(N), LM = lds(M);
    static constexpr int PSI = 0;                 // Psi (N x LD)
    static constexpr int FT = PSI + N * LD;       // Ft (N x LD), row-major
    static constexpr int FS = FT + N * LD;        // F_k (N x LD)
    static constexpr int LS = FS + N * LD;        // L_k (N x LM)
    static constexpr int KS = LS + N * LM;        // K_k (M x LD)
    static constexpr int SS = KS + M * LD;        // S_{k+1} (N x LD)
    static constexpr int SLS = SS + N * LD;       // S_{k+1} L_k (N x LM)
    static constexpr int GS = SLS + N * LM;       // G_k (M x LM)
    static constexpr int US = GS + M * LM;        // U_k (M x LM)
    static constexpr int VEC = US + M * LM;       // vectors:
    static constexpr int OV = VEC, OW = OV + N, OC = OW + N, OY = OC + N, OQ = OY + 2 * N,
                         OD = OQ + N, OG = OD + M, OT = OG + N;
    static constexpr int SIZE = OT + M;
};

// y = X_k r_k (p <= 2N entries, lanes r and r + N), then q = H_k^T y into
// sh[OQ]; with H = I (hid) q = y.  Ends with a group sync.
template <typename R, int N, int M>
__device__ __forceinline__ void warm_q(const DescT<R>& D, long long k, R* gs, bool hid,
                                       const Group<N>& g) {
    using W = WarmSmem<N, M>;
    const int r = g.lr, p = D.p;
    R* y = gs + W::OY;
    if (D.r && p > 0) {
        const R* X = D.X + k * D.sX;
        const R* rk = D.r + k * D.sr;
        for (int a = r; a < p; a += N) {
            R t = R(0);
            for (int b = 0; b < p; ++b) t += X[a * p + b] * rk[b];
            y[a] = t;
        }
    }
    g.sync();
    R q = R(0);
    if (D.r && p > 0) {
        if (hid) {
            q = y[r];
        } else {
            const R* H = D.H + k * D.sH;
            for (int a = 0; a < p; ++a) q += H[a * N + r] * y[a];
        }
    }
    gs[W::OQ + r] = q;
    g.sync();
}

// F_k, L_k, K_k (and S_{k+1}, U_k when asked) into shared memory by
// coalesced asynchronous copies; waits for them and syncs the group.
template <typename R, int N, int M>
__device__ __forceinline__ void warm_stage(const DescT<R>& D, long long k, R* gs, bool want_s,
                                           bool want_u, const Group<N>& g) {
    using W = WarmSmem<N, M>;
    constexpr int LD = W::LD, LM = W::LM;
    const int r = g.lr;
    const R* F = D.F + k * D.sF;
    const R* Lk = D.L + k * D.sL;
    const R* K = D.K + k * M * N;
#pragma unroll 8
    for (int t = r; t < N * N; t += N) cp_async<sizeof(R)>(gs + W::FS + (t / N) * LD + t % N, F + t);
#pragma unroll 4
    for (int t = r; t < N * M; t += N) cp_async<sizeof(R)>(gs + W::LS + (t / M) * LM + t % M, Lk + t);
#pragma unroll 4
    for (int t = r; t < M * N; t += N) cp_async<sizeof(R)>(gs + W::KS + (t / N) * LD + t % N, K + t);
    if (want_s) {
        const R* S = D.S + (k + 1) * N * N;
#pragma unroll 8
        for (int t = r; t < N * N; t += N)
            cp_async<sizeof(R)>(gs + W::SS + (t / N) * LD + t % N, S + t);
    }
    if (want_u) {
        const R* U = D.U + k * D.sU;
        for (int t = r; t < M * M; t += N) cp_async<sizeof(R)>(gs + W::US + (t / M) * LM + t % M, U + t);
    }
    cp_async_commit();
    gs[W::OC + r] = D.c ? D.c[k * D.sc + r] : R(0);
    cp_async_wait<0>();
    g.sync();
}

// Column r of Ft_k = F_k - L_k K_k into sh[FT] (lane r writes column r).
template <typename R, int N, int M>
__device__ __forceinline__ void warm_ft_column(R* gs, int r) {
    using W = WarmSmem<N, M>;
    constexpr int LD = W::LD, LM = W::LM;
#pragma unroll 4
    for (int l = 0; l < N; ++l) {
        R t = gs[W::FS + l * LD + r];
#pragma unroll
        for (int a = 0; a < M; ++a) t -= gs[W::LS + l * LM + a] * gs[W::KS + a * LD + r];
        gs[W::FT + l * LD + r] = t;
    }
}

// ---- chunk maps of the value vector --------------------------------------
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_wfold(Args<R, RT> a, RT* psi_copy) {
    using W = WarmSmem<N, M>;
    using A = LAffine<N>;
    constexpr int LD = W::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sh = reinterpret_cast<R*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long c = (long long)blockIdx.x * NG + gi;
    if (c >= a.C) return;
    const Item<R>& it = a.items[find_chunk(a.items, a.count, c)];
    const DescT<R>& D = it.D;
    R* gs = sh + gi * gstride<N>(W::SIZE);
    const int r = g.lr;
    const long long T = D.T;
    const long long lc = c - it.c0;
    const long long s0 = lc * it.B < T ? lc * it.B : T;
    const long long e0 = s0 + it.B < T ? s0 + it.B : T;
#pragma unroll
    for (int j = 0; j < N; ++j) gs[W::PSI + r * LD + j] = r == j ? R(1) : R(0);
    R beta = R(0);
    const bool hid = h_is_identity(D, g);
    const bool has_c = D.c != nullptr;
    g.sync();
    for (long long k = e0 - 1; k >= s0; --k) {
        warm_stage<R, N, M>(D, k, gs, has_c, false, g);
        warm_q<R, N, M>(D, k, gs, hid, g);
        warm_ft_column<R, N, M>(gs, r);
        R w = beta;
        if (has_c) {
#pragma unroll 4
            for (int j = 0; j < N; ++j) w -= gs[W::SS + r * LD + j] * gs[W::OC + j];
        }
        gs[W::OW + r] = w;
        g.sync();
        // beta <- Ft^T w + q, Psi <- Ft^T Psi (row r of each)
        R bn = gs[W::OQ + r];
        R pn[N];
#pragma unroll
        for (int j = 0; j < N; ++j) pn[j] = R(0);
#pragma unroll 4
        for (int l = 0; l < N; ++l) {
            const R f = gs[W::FT + l * LD + r];
            bn += f * gs[W::OW + l];
#pragma unroll
            for (int j = 0; j < N; ++j) pn[j] += f * gs[W::PSI + l * LD + j];
        }
        g.sync();
#pragma unroll
        for (int j = 0; j < N; ++j) gs[W::PSI + r * LD + j] = pn[j];
        beta = bn;
        g.sync();
    }
    // the map at the mirrored slot (scan order: last chunk first) and a copy
    const long long cr = it.c0 + (it.NC - 1 - lc);
    RT* out = a.FE + cr * A::SIZE;
    RT* cp = psi_copy + c * A::SIZE;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const RT x = static_cast<RT>(gs[W::PSI + r * LD + j]);
        out[A::OF + r * A::LD + j] = x;
        cp[A::OF + r * A::LD + j] = x;
    }
    out[A::OC + r] = static_cast<RT>(beta);
}

// ---- v_T (one CTA of N threads per problem): the seed of the value scan ----
template <typename R, typename RT, int N>
__global__ void __launch_bounds__(N) k_wterm(Args<R, RT> a) {
    __shared__ RT y[2 * N];
    const Item<R>& it = a.items[blockIdx.x];
    const DescT<R>& D = it.D;
    const int r = threadIdx.x;
    const int pT = D.pT;
    for (int i = r; i < pT; i += N) {
        RT t = RT(0);
        if (D.rT)
            for (int b = 0; b < pT; ++b)
                t += static_cast<RT>(D.XT[i * pT + b]) * static_cast<RT>(D.rT[b]);
        y[i] = t;
    }
    __syncthreads();
    RT v = RT(0);
    for (int i = 0; i < pT; ++i) v += static_cast<RT>(D.HT[i * N + r]) * y[i];
    D.v[D.T * N + r] = static_cast<R>(v);
    a.X[(it.c0 + it.NC - 1) * N + r] = v;
    if (D.T == 0) D.x[r] = D.x0[r];
}

// ---- x_0 into each problem's top slot of the forward scan ---------------
template <typename R, typename RT, int N>
__global__ void __launch_bounds__(N) k_wseed(Args<R, RT> a) {
    const Item<R>& it = a.items[blockIdx.x];
    a.X[(it.c0 + it.NC - 1) * N + threadIdx.x] = static_cast<RT>(it.D.x0[threadIdx.x]);
}

// ---- per chunk: v_k, d_k, then the chunk's forward map --------------------
template <typename R, typename RT, int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_wrefold(Args<R, RT> a, const RT* psi_copy) {
    using W = WarmSmem<N, M>;
    using A = LAffine<N>;
    constexpr int LD = W::LD, LM = W::LM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sh = reinterpret_cast<R*>(smem_raw);
    const Group<N> g;
    const int gi = threadIdx.x / N;
    const long long c = (long long)blockIdx.x * NG + gi;
    if (c >= a.C) return;
    const Item<R>& it = a.items[find_chunk(a.items, a.count, c)];
    const DescT<R>& D = it.D;
    R* gs = sh + gi * gstride<N>(W::SIZE);
    const int r = g.lr;
    const long long T = D.T;
    const long long lc = c - it.c0;
    const long long s0 = lc * it.B < T ? lc * it.B : T;
    const long long e0 = s0 + it.B < T ? s0 + it.B : T;
    const long long cr = it.c0 + (it.NC - 1 - lc);
    R v = static_cast<R>(a.X[cr * N + r]);  // v at the chunk's end
    const bool hid = h_is_identity(D, g);
    const bool has_c = D.c != nullptr;
    bool ok = true;
    for (long long k = e0 - 1; k >= s0; --k) {
        warm_stage<R, N, M>(D, k, gs, true, true, g);
        warm_q<R, N, M>(D, k, gs, hid, g);
        warm_ft_column<R, N, M>(gs, r);
        R w = v;
        if (has_c) {
#pragma unroll 4
            for (int j = 0; j < N; ++j) w -= gs[W::SS + r * LD + j] * gs[W::OC + j];
        }
        gs[W::OW + r] = w;
        // S_{k+1} L_k, row r
        R sl[M];
#pragma unroll
        for (int b = 0; b < M; ++b) sl[b] = R(0);
#pragma unroll 4
        for (int j = 0; j < N; ++j) {
            const R s = gs[W::SS + r * LD + j];
#pragma unroll
            for (int b = 0; b < M; ++b) sl[b] += s * gs[W::LS + j * LM + b];
        }
#pragma unroll
        for (int b = 0; b < M; ++b) gs[W::SLS + r * LM + b] = sl[b];
        g.sync();
        // G = L^T (S L) + U and L^T w, rows a < M
        if (r < M) {
            R gr[M];
            R lw = R(0);
#pragma unroll
            for (int b = 0; b < M; ++b) gr[b] = gs[W::US + r * LM + b];
#pragma unroll 4
            for (int j = 0; j < N; ++j) {
                const R l = gs[W::LS + j * LM + r];
                lw += l * gs[W::OW + j];
#pragma unroll
                for (int b = 0; b < M; ++b) gr[b] += l * gs[W::SLS + j * LM + b];
            }
#pragma unroll
            for (int b = 0; b < M; ++b) gs[W::GS + r * LM + b] = gr[b];
            gs[W::OD + r] = lw;
        }
        g.sync();
        ok &= solve_spd<N, M, 1, R>(gs + W::GS, LM, gs + W::OD, 1, g);
        if (r < M) D.u[k * M + r] = gs[W::OD + r];  // d_k until the rollout
        // v_k = Ft^T w + q
        R vn = gs[W::OQ + r];
#pragma unroll 4
        for (int l = 0; l < N; ++l) vn += gs[W::FT + l * LD + r] * gs[W::OW + l];
        D.v[k * N + r] = vn;
        v = vn;
        g.sync();
    }
    // the chunk's forward offset: a rollout from x = 0 with u = d - K x
    R gm = R(0);
    gs[W::OG + r] = gm;
    g.sync();
    for (long long k = s0; k < e0; ++k) {
        warm_stage<R, N, M>(D, k, gs, false, false, g);
        if (r < M) {
            R t = D.u[k * M + r];
#pragma unroll
            for (int j = 0; j < N; ++j) t -= gs[W::KS + r * LD + j] * gs[W::OG + j];
            gs[W::OT + r] = t;
        }
        g.sync();
        R t = gs[W::OC + r];
#pragma unroll 4
        for (int j = 0; j < N; ++j) t += gs[W::FS + r * LD + j] * gs[W::OG + j];
#pragma unroll
        for (int b = 0; b < M; ++b) t += gs[W::LS + r * LM + b] * gs[W::OT + b];
        g.sync();
        gs[W::OG + r] = t;
        gm = t;
        g.sync();
    }
    // forward map (Psi^T, gamma) at the chunk's own slot
    RT* out = a.FE + c * A::SIZE;
    const RT* ps = psi_copy + c * A::SIZE;
#pragma unroll 4
    for (int j = 0; j < N; ++j) out[A::OF + r * A::LD + j] = ps[A::OF + j * A::LD + r];
    out[A::OC + r] = static_cast<RT>(gm);
    flag(a.status, ok);
}

}  // namespace chain
}  // namespace lqt
