// Partial condensing (Sec. V-C, "Block processing"): the problem is rewritten
// in blocks of B steps whose state is the block's first state x_{jB} and
// whose control is the stack u_bar_j = (u_{jB}, ..., u_{jB+B-1}).  Eliminating
// the states inside a block gives
//   x_{jB+i} = Phi_i x_{jB} + Gam_i u_bar_j + del_i      (Phi_0 = I, Gam_0 = 0, del_0 = 0,
//   Phi_{i+1} = F Phi_i, Gam_{i+1} = F Gam_i + L E_i, del_{i+1} = F del_i + c),
// so the block's dynamics are (F_bar, L_bar, c_bar) = (Phi_B, Gam_B, del_B) and its
// stage cost, with y_i = H (Phi_i x + Gam_i u_bar + del_i) - r stacked over i, is
//   1/2 (H_bar x - r_bar)^T X_bar (H_bar x - r_bar) + (H_bar x - r_bar)^T M u_bar
//   + 1/2 u_bar^T U_bar u_bar,
//   H_bar = [H Phi_i], r_bar = [r - H del_i], X_bar = blockdiag(X), G = [H Gam_i],
//   M = X_bar G, U_bar = blockdiag(U) + G^T X_bar G:
// the generalised stage cost of Sec. IV-D, which lqt_solve_cross solves with
// n states and B m controls (T / B steps, a shorter last block padded with
// steps that change nothing).  The block-start values and states are the
// original problem's; the expansion kernel re-runs each block's B Riccati
// steps backward from S, v at the block's end and its rollout forward from
// x_{jB} with the stacked controls, writing every step's S, v, K, x, u.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "lqt.h"
#include "lqt_dense.cuh"
#include "lqt_refine.cuh"

namespace lqt {
namespace {

constexpr size_t kAlignP = 256;
constexpr int kCondPMax = 8;  // rows of H_k the block kernels hold in registers
constexpr int kCondThreads = 128;

size_t up_p(size_t x) { return (x + kAlignP - 1) / kAlignP * kAlignP; }

template <typename R>
struct CondArgs {
    long long T, Tb;
    int p;
    int inv;  // time-invariant model and T a multiple of B: one copy of the block matrices
    const R *F, *c, *L, *U, *H, *r, *X;
    long long sF, sc, sL, sU, sH, sr, sX;
    // condensed problem (per block, dense)
    R *Fb, *Lb, *cb, *Ub, *Hb, *rb, *Xb, *Mb;
    // condensed solution
    const R *Sb, *vb, *xb, *ub;
    // original solution
    R *S, *v, *K, *x, *u;
    // second pass of the refinement: only the forward rollout, adding xi to x
    int shift_add;
    int* status;
    const int* pre_status;  // status of the kernels before the condensed solve
};

template <typename R>
__device__ __forceinline__ const R* at(const R* a, long long s, long long k) {
    return a ? a + s * k : nullptr;
}

// The vectors of block j of the condensed problem: del_0 = 0,
// del_{i+1} = F_k del_i + c_k, r_bar_i = r_k - H_k del_i (k = jB + i; zero
// rows past T) into rb (B p values), and c_bar_j = del_B into cb (N values).
template <typename R, int N>
__device__ __forceinline__ void block_vectors(const R* F0, long long sF, const R* c0, long long sc,
                                              const R* H0, long long sH, const R* r0,
                                              long long sr, int p, int B, long long T,
                                              long long j, R* rb, R* cb) {
    const long long k0 = j * B;
    R del[N];
#pragma unroll
    for (int s = 0; s < N; ++s) del[s] = R(0);
    for (int i = 0; i < B; ++i) {
        const long long k = k0 + i;
        if (k >= T) {
            for (int q = 0; q < p; ++q) rb[i * p + q] = R(0);
            continue;
        }
        const R* F = F0 + sF * k;
        const R* H = at(H0, sH, k);
        const R* r = at(r0, sr, k);
        const R* c = at(c0, sc, k);
        for (int q = 0; q < p; ++q) {
            R t = r ? r[q] : R(0);
#pragma unroll
            for (int s = 0; s < N; ++s) t -= H[q * N + s] * del[s];
            rb[i * p + q] = t;
        }
        R dn[N];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            R t = c ? c[s] : R(0);
#pragma unroll
            for (int l = 0; l < N; ++l) t += F[s * N + l] * del[l];
            dn[s] = t;
        }
#pragma unroll
        for (int s = 0; s < N; ++s) del[s] = dn[s];
    }
#pragma unroll
    for (int s = 0; s < N; ++s) cb[s] = del[s];
}

template <typename R, int N, int M, int B>
__global__ void __launch_bounds__(kCondThreads) k_condense(CondArgs<R> a) {
    constexpr int MB = M * B;
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const int p = a.p, pb = p * B;
    const long long k0 = j * B;
    const int b = (int)(a.T - k0 < B ? a.T - k0 : B);
    R Phi[N][N], Gam[N][MB], del[N], UG[MB][MB];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int l = 0; l < N; ++l) Phi[i][l] = i == l ? R(1) : R(0);
#pragma unroll
        for (int l = 0; l < MB; ++l) Gam[i][l] = R(0);
        del[i] = R(0);
    }
#pragma unroll
    for (int i = 0; i < MB; ++i)
#pragma unroll
        for (int l = 0; l < MB; ++l) UG[i][l] = R(0);
    // with a time-invariant model every block's matrices are block 0's: the
    // other threads compute them (cheaply) but only write r_bar
    const bool mats = !a.inv || j == 0;
    const long long jm = a.inv ? 0 : j;
    R* Hb = a.Hb + jm * (long long)pb * N;
    R* rb = a.rb + j * (long long)pb;
    R* Xb = a.Xb + jm * (long long)pb * pb;
    R* Mb = a.Mb + jm * (long long)pb * MB;
    if (mats)
        for (int e = 0; e < pb * pb; ++e) Xb[e] = R(0);
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (i < b) {
            const long long k = k0 + i;
            const R* F = a.F + a.sF * k;
            const R* L = a.L + a.sL * k;
            const R* U = a.U + a.sU * k;
            const R* c = at(a.c, a.sc, k);
            const R* H = at(a.H, a.sH, k);
            const R* r = at(a.r, a.sr, k);
            const R* X = at(a.X, a.sX, k);
            // rows of stage i: H Phi_i, G_i = H Gam_i, r - H del_i
            R g[kCondPMax][MB];
            for (int q = 0; q < p; ++q) {
                R hr[N];
#pragma unroll
                for (int l = 0; l < N; ++l) hr[l] = H[q * N + l];
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    R t = R(0);
#pragma unroll
                    for (int s = 0; s < N; ++s) t += hr[s] * Phi[s][l];
                    if (mats) Hb[(i * p + q) * N + l] = t;
                }
#pragma unroll
                for (int l = 0; l < MB; ++l) {
                    R t = R(0);
#pragma unroll
                    for (int s = 0; s < N; ++s) t += hr[s] * Gam[s][l];
                    g[q][l] = t;
                }
                R t = r ? r[q] : R(0);
#pragma unroll
                for (int s = 0; s < N; ++s) t -= hr[s] * del[s];
                rb[i * p + q] = t;
            }
            // X_bar block, M rows X G_i, and G_i^T X G_i into U_bar
            for (int q = 0; q < p; ++q) {
                R mrow[MB];
#pragma unroll
                for (int l = 0; l < MB; ++l) mrow[l] = R(0);
                for (int s = 0; s < p; ++s) {
                    const R xqs = X[q * p + s];
                    if (mats) Xb[(i * p + q) * pb + i * p + s] = xqs;
#pragma unroll
                    for (int l = 0; l < MB; ++l) mrow[l] += xqs * g[s][l];
                }
                if (mats)
#pragma unroll
                    for (int l = 0; l < MB; ++l) Mb[(i * p + q) * MB + l] = mrow[l];
#pragma unroll
                for (int c1 = 0; c1 < MB; ++c1)
#pragma unroll
                    for (int c2 = 0; c2 < MB; ++c2) UG[c1][c2] += g[q][c1] * mrow[c2];
            }
#pragma unroll
            for (int c1 = 0; c1 < M; ++c1)
#pragma unroll
                for (int c2 = 0; c2 < M; ++c2) UG[i * M + c1][i * M + c2] += U[c1 * M + c2];
            // advance the block's maps by step k
            R Pn[N][N], Gn[N][MB], dn[N];
#pragma unroll
            for (int s = 0; s < N; ++s) {
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    R t = R(0);
#pragma unroll
                    for (int q = 0; q < N; ++q) t += F[s * N + q] * Phi[q][l];
                    Pn[s][l] = t;
                }
#pragma unroll
                for (int l = 0; l < MB; ++l) {
                    R t = R(0);
#pragma unroll
                    for (int q = 0; q < N; ++q) t += F[s * N + q] * Gam[q][l];
                    Gn[s][l] = t;
                }
                R t = c ? c[s] : R(0);
#pragma unroll
                for (int q = 0; q < N; ++q) t += F[s * N + q] * del[q];
                dn[s] = t;
            }
#pragma unroll
            for (int s = 0; s < N; ++s) {
#pragma unroll
                for (int l = 0; l < N; ++l) Phi[s][l] = Pn[s][l];
#pragma unroll
                for (int l = 0; l < MB; ++l) Gam[s][l] = Gn[s][l];
#pragma unroll
                for (int l = 0; l < M; ++l) Gam[s][i * M + l] += L[s * M + l];
                del[s] = dn[s];
            }
        } else {
            // padding step past T: no cost rows, an identity weight on its
            // controls (which then stay zero), no effect on the state
            for (int q = 0; q < p; ++q) {
#pragma unroll
                for (int l = 0; l < N; ++l) Hb[(i * p + q) * N + l] = R(0);
#pragma unroll
                for (int l = 0; l < MB; ++l) Mb[(i * p + q) * MB + l] = R(0);
                rb[i * p + q] = R(0);
            }
#pragma unroll
            for (int c1 = 0; c1 < M; ++c1) UG[i * M + c1][i * M + c1] += R(1);
        }
    }
    // c_bar: one per block unless the model and its offsets are time-invariant
    const bool cvar = !a.inv || (a.c && a.sc != 0);
    if (cvar || j == 0) {
        R* cb = a.cb + (cvar ? j : 0) * N;
#pragma unroll
        for (int s = 0; s < N; ++s) cb[s] = del[s];
    }
    if (!mats) return;
    R* Fb = a.Fb + jm * N * N;
    R* Lb = a.Lb + jm * N * MB;
    R* Ub = a.Ub + jm * MB * MB;
#pragma unroll
    for (int s = 0; s < N; ++s) {
#pragma unroll
        for (int l = 0; l < N; ++l) Fb[s * N + l] = Phi[s][l];
#pragma unroll
        for (int l = 0; l < MB; ++l) Lb[s * MB + l] = Gam[s][l];
    }
#pragma unroll
    for (int c1 = 0; c1 < MB; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < MB; ++c2) Ub[c1 * MB + c2] = UG[c1][c2];
}

// Step k of the original problem for riccati_step: F, c, L, U, Q = H^T X H,
// q = H^T X r.
template <typename R, int N, int M>
__device__ __forceinline__ void cond_step(const CondArgs<R>& a, long long k, Step<R, N, M>& st) {
    const R* F = a.F + a.sF * k;
    const R* L = a.L + a.sL * k;
    const R* U = a.U + a.sU * k;
    const R* c = at(a.c, a.sc, k);
    const R* H = at(a.H, a.sH, k);
    const R* r = at(a.r, a.sr, k);
    const R* X = at(a.X, a.sX, k);
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int l = 0; l < N; ++l) st.F[i][l] = F[i * N + l];
#pragma unroll
        for (int l = 0; l < M; ++l) st.L[i][l] = L[i * M + l];
        st.c[i] = c ? c[i] : R(0);
        st.q[i] = R(0);
    }
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int l = 0; l < M; ++l) st.U[i][l] = U[i * M + l];
#pragma unroll
    for (int s = 0; s < Dims<N>::SYM; ++s) st.Q[s] = R(0);
    const int p = a.p;
    for (int q = 0; q < p; ++q) {
        R y[N];
        R xr = R(0);
#pragma unroll
        for (int l = 0; l < N; ++l) y[l] = R(0);
        for (int s = 0; s < p; ++s) {
            const R xqs = X[q * p + s];
#pragma unroll
            for (int l = 0; l < N; ++l) y[l] += xqs * H[s * N + l];
            if (r) xr += xqs * r[s];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const R h = H[q * N + i];
            st.q[i] += h * xr;
#pragma unroll
            for (int l = i; l < N; ++l) st.Q[sym<N>(i, l)] += h * y[l];
        }
    }
}

// Status of an expansion: a failure recorded before the condensed solve (whose
// start clears the status word) is the root cause and wins.
template <typename R>
__device__ __forceinline__ void expand_status(const CondArgs<R>& a, long long j, bool ok,
                                              bool finite) {
    if (j == 0 && a.pre_status && *a.pre_status != 0) atomicExch(a.status, *a.pre_status);
    if (!ok) atomicCAS(a.status, 0, (int)LQT_ENOTSPD);
    if (!finite) atomicCAS(a.status, 0, (int)LQT_ENONFINITE);
}

template <typename R, int N, int M, int B>
__global__ void __launch_bounds__(kCondThreads) k_expand(CondArgs<R> a) {
    constexpr int MB = M * B;
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const long long k0 = j * B;
    const int b = (int)(a.T - k0 < B ? a.T - k0 : B);
    bool ok = true, finite = true;
    if (!a.shift_add) {
        // backward: the block's Riccati steps from the value at its end
        R S[Dims<N>::SYM], v[N];
        const R* Se = a.Sb + (j + 1) * N * N;
        const R* ve = a.vb + (j + 1) * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int l = i; l < N; ++l) S[sym<N>(i, l)] = Se[i * N + l];
            v[i] = ve[i];
        }
        if (j == a.Tb - 1) {
            // terminal value S_T, v_T
#pragma unroll
            for (int i = 0; i < N; ++i) {
#pragma unroll
                for (int l = 0; l < N; ++l) a.S[a.T * N * N + i * N + l] = Se[i * N + l];
                a.v[a.T * N + i] = ve[i];
            }
        }
#pragma unroll
        for (int i = B - 1; i >= 0; --i) {
            if (i < b) {
                const long long k = k0 + i;
                Step<R, N, M> st;
                cond_step<R, N, M>(a, k, st);
                R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
                ok &= riccati_step<R, N, M>(st, a.c != nullptr, S, v, K, d, Ft, ct, Rc, Rinv);
#pragma unroll
                for (int s = 0; s < N; ++s) {
#pragma unroll
                    for (int l = 0; l < N; ++l) a.S[k * N * N + s * N + l] = S[sym<N>(s, l)];
                    a.v[k * N + s] = v[s];
                    finite = finite && isfinite(v[s]);
                }
#pragma unroll
                for (int s = 0; s < M; ++s)
#pragma unroll
                    for (int l = 0; l < N; ++l) a.K[(k * M + s) * N + l] = K[s][l];
            }
        }
    }
    // forward: the rollout from x_{jB} with the block's stacked controls
    R x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = a.xb[j * N + i];
    const R* ub = a.ub + j * MB;
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (i < b) {
            const long long k = k0 + i;
            const R* F = a.F + a.sF * k;
            const R* L = a.L + a.sL * k;
            const R* c = at(a.c, a.sc, k);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                const R xo = a.shift_add ? a.x[k * N + s] + x[s] : x[s];
                a.x[k * N + s] = xo;
                finite = finite && isfinite(xo);
            }
#pragma unroll
            for (int s = 0; s < M; ++s) a.u[k * M + s] = ub[i * M + s];
            R xn[N];
#pragma unroll
            for (int s = 0; s < N; ++s) {
                R t = c ? c[s] : R(0);
#pragma unroll
                for (int l = 0; l < N; ++l) t += F[s * N + l] * x[l];
#pragma unroll
                for (int l = 0; l < M; ++l) t += L[s * M + l] * ub[i * M + l];
                xn[s] = t;
            }
#pragma unroll
            for (int s = 0; s < N; ++s) x[s] = xn[s];
        }
    }
    if (j == a.Tb - 1) {
        // x_T: the condensed solve's last state (the block rollout agrees to rounding)
#pragma unroll
        for (int s = 0; s < N; ++s)
            a.x[a.T * N + s] = a.shift_add ? a.x[a.T * N + s] + a.xb[a.Tb * N + s]
                                           : a.xb[a.Tb * N + s];
    }
    expand_status(a, j, ok, finite);
}

// ---- rank-reduced condensing (any block size with B m <= 32 and B p <= 32) --
// The condensed block problem of the kernels above has B m stacked controls,
// more than the compiled solvers take at larger B.  Its state dimension stays
// n, and the controls reach the next block only through w = L_bar u_bar (n
// values).  For given block start x (output error y = H_bar x - r_bar) and w,
// the best u_bar minimises 1/2 u^T U_bar u + y^T M u subject to L_bar u = w;
// with A = U_bar^{-1} L_bar^T, Z = U_bar^{-1} M^T and the eigenbasis
// W = L_bar A = V diag(lam) V^T, writing w = V z:
//   u_bar = P z - Q y,   P = A V diag(1/lam),   Q = Z - P V^T L_bar Z,
// and the block's cost becomes 1/2 z^T diag(1/lam) z + y^T M_r z
// + 1/2 y^T X_r y with M_r = M A V diag(1/lam), X_r = X_bar - M Z +
// M_r (M A V)^T.  So each block is exactly one step of a problem with n
// controls z: dynamics (F_bar, c_bar, L_r = V), U_r = diag(1/lam), and the
// generalised cost of Sec. IV-D with H_bar, r_bar, X_r, M_r, which
// lqt_solve_cross solves at (n, n).  A direction with lam = 0 (a block that
// cannot move the state that way, such as a last block of fewer than n / m
// steps) gets a zero column of L_r and a unit weight, so its control stays 0.
// The stacked controls are then rebuilt per block from (x, z) and expanded as
// before.  The reduction runs in FP64.
constexpr int kRedMax = 32;      // largest B m and B p
constexpr int kRedThreads = 128;

template <typename R>
struct RedArgs {
    long long T, Tb;
    int m, p, B;
    int inv;  // time-invariant model and T a multiple of B: one copy of the block matrices
    const R *F, *c, *L, *U, *H, *r, *X;
    long long sF, sc, sL, sU, sH, sr, sX;
    // reduced problem: per block (inv: one copy), except r_bar (per block)
    R *Fb, *cb, *Lb, *Ub, *Hb, *rb, *Xb, *Mb;
    // rebuilding the stacked controls: P (B m x n), Q (B m x B p)
    R *Pb, *Qb;
    double* HD;  // inv: H del_i, i < B (B x p), for r_bar of every block
    // reduced solution, stacked controls
    const R *xb, *wb;
    R* ub;
    int* status;  // the reduction's failures, merged by the expansion
};

template <int N>
struct RedSmem {  // doubles; MB = B m, PB = B p, both <= kRedMax
    static constexpr int X = kRedMax;
    static constexpr int PHI = 0, DEL = PHI + N * N, GAM = DEL + N, TP = GAM + N * X,
                         TD = TP + N * N, TG = TD + N, HBAR = TG + N * X, G = HBAR + X * N,
                         UB = G + X * X, MM = UB + X * X, XBAR = MM + X * X, RBAR = XBAR + X * X,
                         RHS = RBAR + X, W = RHS + X * (N + X), WI = W + N * N, MA = WI + N * N,
                         MR = MA + X * N, XR = MR + X * N, PP = XR + X * X, LZ = PP + X * N,
                         SIZE = LZ + N * X;
};

template <typename R, int N, int M>
__global__ void __launch_bounds__(kRedThreads) k_cond_reduce(RedArgs<R> a) {
    using S = RedSmem<N>;
    extern __shared__ __align__(16) double rs[];
    double* Phi = rs + S::PHI;
    double* del = rs + S::DEL;
    double* Gam = rs + S::GAM;   // N x MB
    double* tP = rs + S::TP;
    double* td = rs + S::TD;
    double* tG = rs + S::TG;
    double* Hbar = rs + S::HBAR;  // PB x N
    double* G = rs + S::G;        // PB x MB
    double* Ub = rs + S::UB;      // MB x MB
    double* Mm = rs + S::MM;      // PB x MB
    double* Xbar = rs + S::XBAR;  // PB x PB
    double* rbar = rs + S::RBAR;  // PB
    double* RHS = rs + S::RHS;    // MB x (N + PB)
    double* W = rs + S::W;
    double* Wi = rs + S::WI;
    double* MA = rs + S::MA;      // PB x N
    double* Mr = rs + S::MR;      // PB x N
    double* Xr = rs + S::XR;      // PB x PB
    double* Pm = rs + S::PP;      // MB x N
    double* LZ = rs + S::LZ;      // N x PB
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = a.m, p = a.p, B = a.B, MB = B * m, PB = B * p, NR = N + PB;
    const long long j = blockIdx.x;
    const long long k0 = j * B;
    const int b = (int)(a.T - k0 < B ? a.T - k0 : B);
    for (int e = tid; e < S::SIZE; e += nt) rs[e] = 0.0;
    __syncthreads();
    for (int e = tid; e < N; e += nt) Phi[e * N + e] = 1.0;
    __syncthreads();
    // 1. the block's stages: rows H Phi_i, H Gam_i, r - H del_i, X_bar, U_bar
    for (int i = 0; i < B; ++i) {
        const bool live = i < b;
        const long long k = k0 + i;
        const R* F = a.F + a.sF * k;
        const R* L = a.L + a.sL * k;
        const R* U = a.U + a.sU * k;
        const R* c = at(a.c, a.sc, k);
        const R* H = at(a.H, a.sH, k);
        const R* r = at(a.r, a.sr, k);
        const R* X = at(a.X, a.sX, k);
        if (live) {
            for (int e = tid; e < p * N; e += nt) {
                const int q = e / N, l = e % N;
                double t = 0.0;
                for (int s = 0; s < N; ++s) t += (double)H[q * N + s] * Phi[s * N + l];
                Hbar[(i * p + q) * N + l] = t;
            }
            for (int e = tid; e < p * MB; e += nt) {
                const int q = e / MB, l = e % MB;
                double t = 0.0;
                for (int s = 0; s < N; ++s) t += (double)H[q * N + s] * Gam[s * MB + l];
                G[(i * p + q) * MB + l] = t;
            }
            for (int q = tid; q < p; q += nt) {
                double hd = 0.0;
                for (int s = 0; s < N; ++s) hd += (double)H[q * N + s] * del[s];
                rbar[i * p + q] = (r ? (double)r[q] : 0.0) - hd;
                if (a.inv && a.HD) a.HD[i * p + q] = hd;
            }
            for (int e = tid; e < p * p; e += nt)
                Xbar[(i * p + e / p) * PB + i * p + e % p] = (double)X[e];
            for (int e = tid; e < m * m; e += nt)
                Ub[(i * m + e / m) * MB + i * m + e % m] += (double)U[e];
        } else {
            // padding past T: no cost rows, identity weight on its (zero) controls
            for (int e = tid; e < m; e += nt) Ub[(i * m + e) * MB + i * m + e] += 1.0;
            if (a.inv && a.HD)
                for (int q = tid; q < p; q += nt) a.HD[i * p + q] = 0.0;
        }
        __syncthreads();
        if (live) {
            for (int e = tid; e < N * N; e += nt) {
                const int s = e / N, l = e % N;
                double t = 0.0;
                for (int q = 0; q < N; ++q) t += (double)F[s * N + q] * Phi[q * N + l];
                tP[e] = t;
            }
            for (int e = tid; e < N * MB; e += nt) {
                const int s = e / MB, l = e % MB;
                double t = 0.0;
                for (int q = 0; q < N; ++q) t += (double)F[s * N + q] * Gam[q * MB + l];
                if (l >= i * m && l < i * m + m) t += (double)L[s * m + (l - i * m)];
                tG[e] = t;
            }
            for (int s = tid; s < N; s += nt) {
                double t = c ? (double)c[s] : 0.0;
                for (int q = 0; q < N; ++q) t += (double)F[s * N + q] * del[q];
                td[s] = t;
            }
            __syncthreads();
            for (int e = tid; e < N * N; e += nt) Phi[e] = tP[e];
            for (int e = tid; e < N * MB; e += nt) Gam[e] = tG[e];
            for (int s = tid; s < N; s += nt) del[s] = td[s];
            __syncthreads();
        }
    }
    // 2. M = X_bar G, U_bar += G^T M.  X_bar is block diagonal (stage i's X),
    // and the rows of stage i of G (and of M) vanish in the columns of stages
    // i and later (a control acts on the outputs of the following stages), so
    // both products run over the stages that contribute only.
    for (int e = tid; e < PB * MB; e += nt) {
        const int q = e / MB, l = e % MB, i0 = q / p;
        double t = 0.0;
        if (l < i0 * m)
            for (int s = i0 * p; s < i0 * p + p; ++s) t += Xbar[q * PB + s] * G[s * MB + l];
        Mm[e] = t;
    }
    __syncthreads();
    for (int e = tid; e < MB * MB; e += nt) {
        const int c1 = e / MB, c2 = e % MB;
        const int s1 = c1 / m, s2 = c2 / m;
        double t = 0.0;
        for (int q = ((s1 > s2 ? s1 : s2) + 1) * p; q < PB; ++q) t += G[q * MB + c1] * Mm[q * MB + c2];
        Ub[e] += t;
    }
    __syncthreads();
    // 3. Cholesky U_bar = R R^T (lower, in place), then [A | Z] = U_bar^{-1} [L_bar^T | M^T]
    __shared__ int s_ok;
    if (tid == 0) s_ok = 1;
    __syncthreads();
    for (int kk = 0; kk < MB; ++kk) {
        if (tid == 0) {
            const double d = Ub[kk * MB + kk];
            if (!(d > 0.0) || !isfinite(d)) s_ok = 0;
            Ub[kk * MB + kk] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double piv = Ub[kk * MB + kk];
        for (int i = kk + 1 + tid; i < MB; i += nt) Ub[i * MB + kk] /= piv;
        __syncthreads();
        const int rest = MB - kk - 1;
        for (int e = tid; e < rest * rest; e += nt) {
            const int i = kk + 1 + e / rest, jj = kk + 1 + e % rest;
            if (jj <= i) Ub[i * MB + jj] -= Ub[i * MB + kk] * Ub[jj * MB + kk];
        }
        __syncthreads();
    }
    for (int e = tid; e < MB * NR; e += nt) {
        const int i = e / NR, cc = e % NR;
        RHS[e] = cc < N ? Gam[cc * MB + i] : Mm[(cc - N) * MB + i];
    }
    __syncthreads();
    for (int cc = tid; cc < NR; cc += nt) {
        for (int i = 0; i < MB; ++i) {  // R y = rhs
            double t = RHS[i * NR + cc];
            for (int l = 0; l < i; ++l) t -= Ub[i * MB + l] * RHS[l * NR + cc];
            RHS[i * NR + cc] = t / Ub[i * MB + i];
        }
        for (int i = MB - 1; i >= 0; --i) {  // R^T x = y
            double t = RHS[i * NR + cc];
            for (int l = i + 1; l < MB; ++l) t -= Ub[l * MB + i] * RHS[l * NR + cc];
            RHS[i * NR + cc] = t / Ub[i * MB + i];
        }
    }
    __syncthreads();
    // 4. W = L_bar A = V diag(lam) V^T; M A; M_r = M A V / lam; P = A V / lam;
    //    X_r = X_bar - M Z + sum_i (M A v_i)(M A v_i)^T / lam_i (live directions)
    for (int e = tid; e < N * N; e += nt) {
        const int r0 = e / N, cc = e % N;
        double t = 0.0;
        for (int i = 0; i < MB; ++i) t += Gam[r0 * MB + i] * RHS[i * NR + cc];
        W[e] = t;
    }
    __syncthreads();
    if (tid == 0) {
        // cyclic Jacobi rotations on the symmetric W; V (in Wi) collects them
        double Aw[N][N], V[N][N];
        for (int i = 0; i < N; ++i)
            for (int l = 0; l < N; ++l) {
                Aw[i][l] = 0.5 * (W[i * N + l] + W[l * N + i]);
                V[i][l] = i == l ? 1.0 : 0.0;
            }
        for (int sweep = 0; sweep < 32; ++sweep) {
            double off = 0.0;
            for (int i = 0; i < N; ++i)
                for (int l = i + 1; l < N; ++l) off += Aw[i][l] * Aw[i][l];
            if (!(off > 1e-60)) break;
            for (int pp = 0; pp < N; ++pp)
                for (int qq = pp + 1; qq < N; ++qq) {
                    if (Aw[pp][qq] == 0.0) continue;
                    const double th = 0.5 * (Aw[qq][qq] - Aw[pp][pp]) / Aw[pp][qq];
                    const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                    for (int l = 0; l < N; ++l) {  // columns p, q
                        const double ap = Aw[l][pp], aq = Aw[l][qq];
                        Aw[l][pp] = cs * ap - sn * aq;
                        Aw[l][qq] = sn * ap + cs * aq;
                    }
                    for (int l = 0; l < N; ++l) {  // rows p, q
                        const double ap = Aw[pp][l], aq = Aw[qq][l];
                        Aw[pp][l] = cs * ap - sn * aq;
                        Aw[qq][l] = sn * ap + cs * aq;
                    }
                    for (int l = 0; l < N; ++l) {
                        const double vp = V[l][pp], vq = V[l][qq];
                        V[l][pp] = cs * vp - sn * vq;
                        V[l][qq] = sn * vp + cs * vq;
                    }
                }
        }
        double lmax = 0.0;
        for (int i = 0; i < N; ++i) lmax = fmax(lmax, Aw[i][i]);
        if (!(lmax > 0.0) || !isfinite(lmax)) s_ok = 0;
        for (int i = 0; i < N; ++i) {
            const double lam = Aw[i][i];
            // W[i] now holds 1 / lam_i for a live direction, 0 for a null one
            W[i] = lam > 1e-12 * lmax ? 1.0 / lam : 0.0;
            for (int l = 0; l < N; ++l) Wi[l * N + i] = V[l][i];
        }
    }
    __syncthreads();
    const double* ilam = W;  // N entries
    const double* Vm = Wi;   // N x N, column i = eigenvector i
    for (int e = tid; e < PB * N; e += nt) {  // (M A) V
        const int q = e / N, cc = e % N;
        double t = 0.0;
        for (int l = 0; l < MB; ++l) {
            double av = 0.0;
            for (int d = 0; d < N; ++d) av += RHS[l * NR + d] * Vm[d * N + cc];
            t += Mm[q * MB + l] * av;
        }
        MA[e] = t;
    }
    for (int e = tid; e < MB * N; e += nt) {  // P = A V / lam
        const int l = e / N, cc = e % N;
        double av = 0.0;
        for (int d = 0; d < N; ++d) av += RHS[l * NR + d] * Vm[d * N + cc];
        Pm[e] = av * ilam[cc];
    }
    for (int e = tid; e < N * PB; e += nt) {  // V^T L_bar Z
        const int cc = e / PB, s = e % PB;
        double t = 0.0;
        for (int d = 0; d < N; ++d) {
            double lz = 0.0;
            for (int l = 0; l < MB; ++l) lz += Gam[d * MB + l] * RHS[l * NR + N + s];
            t += Vm[d * N + cc] * lz;
        }
        LZ[e] = t;
    }
    __syncthreads();
    for (int e = tid; e < PB * N; e += nt) Mr[e] = MA[e] * ilam[e % N];
    __syncthreads();
    for (int e = tid; e < PB * PB; e += nt) {
        const int q = e / PB, s = e % PB;
        double t = Xbar[e];
        for (int l = 0, le = (q / p) * m; l < le; ++l) t -= Mm[q * MB + l] * RHS[l * NR + N + s];
        for (int cc = 0; cc < N; ++cc) t += Mr[q * N + cc] * MA[s * N + cc];
        Xr[e] = t;
    }
    __syncthreads();
    // 5. outputs (one copy of the matrices when the model is time-invariant)
    const bool mats = !a.inv || j == 0;
    const long long jm = a.inv ? 0 : j;
    if (mats) {
        R* Fb = a.Fb + jm * N * N;
        R* cb = a.cb + jm * N;
        R* Lrb = a.Lb + jm * N * N;
        R* Urb = a.Ub + jm * N * N;
        R* Hb = a.Hb + jm * (long long)PB * N;
        R* Xb = a.Xb + jm * (long long)PB * PB;
        R* Mb = a.Mb + jm * (long long)PB * N;
        R* Pb = a.Pb + jm * (long long)MB * N;
        R* Qb = a.Qb + jm * (long long)MB * PB;
        for (int e = tid; e < N * N; e += nt) {
            const int r0 = e / N, cc = e % N;
            const bool live = W[cc] > 0.0;  // 1 / lam of direction cc, 0 when null
            Fb[e] = static_cast<R>(Phi[e]);
            // L_r = V (null directions: zero column), U_r = diag(1 / lam) (null: 1)
            Lrb[e] = static_cast<R>(live ? Wi[r0 * N + cc] : 0.0);
            Urb[e] = static_cast<R>(r0 == cc ? (live ? W[cc] : 1.0) : 0.0);
        }
        if (!a.inv || !a.c || a.sc == 0)  // else k_cond_rbar writes every block's
            for (int s = tid; s < N; s += nt) cb[s] = static_cast<R>(del[s]);
        for (int e = tid; e < PB * N; e += nt) {
            Hb[e] = static_cast<R>(Hbar[e]);
            Mb[e] = static_cast<R>(Mr[e]);
        }
        for (int e = tid; e < PB * PB; e += nt) {
            const int q = e / PB, s = e % PB;
            Xb[e] = static_cast<R>(0.5 * (Xr[e] + Xr[s * PB + q]));
        }
        for (int e = tid; e < MB * N; e += nt) Pb[e] = static_cast<R>(Pm[e]);
        for (int e = tid; e < MB * PB; e += nt) {  // Q = Z - P V^T L_bar Z
            const int l = e / PB, s = e % PB;
            double t = RHS[l * NR + N + s];
            for (int cc = 0; cc < N; ++cc) t -= Pm[l * N + cc] * LZ[cc * PB + s];
            Qb[e] = static_cast<R>(t);
        }
    }
    if (!a.inv)
        for (int q = tid; q < PB; q += nt) a.rb[j * PB + q] = static_cast<R>(rbar[q]);
    if (tid == 0 && !s_ok) atomicCAS(a.status, 0, (int)LQT_ENOTSPD);
}

// r_bar of every block of a time-invariant model (one thread per block).
// Offsets c fixed (or none): r_{jB+i} - H del_i with del_i from the reduction
// of block 0.  Offsets c_k that vary (matrices still time-invariant): each
// block's own del_i (del_0 = 0, del_{i+1} = F del_i + c_{jB+i}) and
// c_bar_j = del_B.
template <typename R, int N>
__global__ void __launch_bounds__(kCondThreads) k_cond_rbar(RedArgs<R> a) {
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const int p = a.p, B = a.B;
    const long long k0 = j * B;
    R* rb = a.rb + j * (long long)B * p;
    if (!a.c || a.sc == 0) {
        for (int i = 0; i < B; ++i) {
            const long long k = k0 + i;
            const R* r = at(a.r, a.sr, k);
            for (int q = 0; q < p; ++q)
                rb[i * p + q] =
                    k < a.T ? static_cast<R>((r ? (double)r[q] : 0.0) - a.HD[i * p + q]) : R(0);
        }
        return;
    }
    block_vectors<R, N>(a.F, a.sF, a.c, a.sc, a.H, a.sH, a.r, a.sr, p, B, a.T, j, rb,
                        a.cb + j * N);
}

// The stacked controls of every block from the reduced solution (one thread
// per block): u_bar_j = P w_j - Q (H_bar x_j - r_bar_j).
template <typename R, int N>
__global__ void __launch_bounds__(kCondThreads) k_cond_unreduce(RedArgs<R> a) {
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const int MB = a.B * a.m, PB = a.B * a.p;
    const long long jm = a.inv ? 0 : j;
    const R* Hb = a.Hb + jm * (long long)PB * N;
    const R* Pb = a.Pb + jm * (long long)MB * N;
    const R* Qb = a.Qb + jm * (long long)MB * PB;
    const R* rb = a.rb + j * PB;
    R x[N], w[N];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        x[s] = a.xb[j * N + s];
        w[s] = a.wb[j * N + s];
    }
    R y[kRedMax];
    for (int q = 0; q < PB; ++q) {
        R t = -rb[q];
#pragma unroll
        for (int s = 0; s < N; ++s) t += Hb[q * N + s] * x[s];
        y[q] = t;
    }
    for (int l = 0; l < MB; ++l) {
        R t = R(0);
#pragma unroll
        for (int s = 0; s < N; ++s) t += Pb[l * N + s] * w[s];
        for (int q = 0; q < PB; ++q) t -= Qb[l * PB + q] * y[q];
        a.ub[j * MB + l] = t;
    }
}

// Expansion with a run-time block size (the block loop of k_expand).
template <typename R, int N, int M>
__global__ void __launch_bounds__(kCondThreads) k_expand_rt(CondArgs<R> a, int B) {
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const long long k0 = j * B;
    const int b = (int)(a.T - k0 < B ? a.T - k0 : B);
    bool ok = true, finite = true;
    if (!a.shift_add) {
        R S[Dims<N>::SYM], v[N];
        const R* Se = a.Sb + (j + 1) * N * N;
        const R* ve = a.vb + (j + 1) * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int l = i; l < N; ++l) S[sym<N>(i, l)] = Se[i * N + l];
            v[i] = ve[i];
        }
        if (j == a.Tb - 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
#pragma unroll
                for (int l = 0; l < N; ++l) a.S[a.T * N * N + i * N + l] = Se[i * N + l];
                a.v[a.T * N + i] = ve[i];
            }
        }
        for (int i = b - 1; i >= 0; --i) {
            const long long k = k0 + i;
            Step<R, N, M> st;
            cond_step<R, N, M>(a, k, st);
            R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
            ok &= riccati_step<R, N, M>(st, a.c != nullptr, S, v, K, d, Ft, ct, Rc, Rinv);
#pragma unroll
            for (int s = 0; s < N; ++s) {
#pragma unroll
                for (int l = 0; l < N; ++l) a.S[k * N * N + s * N + l] = S[sym<N>(s, l)];
                a.v[k * N + s] = v[s];
                finite = finite && isfinite(v[s]);
            }
#pragma unroll
            for (int s = 0; s < M; ++s)
#pragma unroll
                for (int l = 0; l < N; ++l) a.K[(k * M + s) * N + l] = K[s][l];
        }
    }
    R x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = a.xb[j * N + i];
    const R* ub = a.ub + j * (long long)B * M;
    for (int i = 0; i < b; ++i) {
        const long long k = k0 + i;
        const R* F = a.F + a.sF * k;
        const R* L = a.L + a.sL * k;
        const R* c = at(a.c, a.sc, k);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const R xo = a.shift_add ? a.x[k * N + s] + x[s] : x[s];
            a.x[k * N + s] = xo;
            finite = finite && isfinite(xo);
        }
#pragma unroll
        for (int s = 0; s < M; ++s) a.u[k * M + s] = ub[i * M + s];
        R xn[N];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            R t = c ? c[s] : R(0);
#pragma unroll
            for (int l = 0; l < N; ++l) t += F[s * N + l] * x[l];
#pragma unroll
            for (int l = 0; l < M; ++l) t += L[s * M + l] * ub[i * M + l];
            xn[s] = t;
        }
#pragma unroll
        for (int s = 0; s < N; ++s) x[s] = xn[s];
    }
    if (j == a.Tb - 1) {
#pragma unroll
        for (int s = 0; s < N; ++s)
            a.x[a.T * N + s] = a.shift_add ? a.x[a.T * N + s] + a.xb[a.Tb * N + s]
                                           : a.xb[a.Tb * N + s];
    }
    expand_status(a, j, ok, finite);
}

// The vectors of the condensed problem alone (block_vectors, one thread per
// block), for a second solve whose matrices (F, L, U, H, X) are those of the
// first.
template <typename R>
struct VecArgs {
    long long T, Tb;
    int p, B;
    const R *F, *c, *H, *r;
    long long sF, sc, sH, sr;
    R *rb, *cb;
};

template <typename R, int N>
__global__ void __launch_bounds__(kCondThreads) k_cond_vec(VecArgs<R> a) {
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    block_vectors<R, N>(a.F, a.sF, a.c, a.sc, a.H, a.sH, a.r, a.sr, a.p, a.B, a.T, j,
                        a.rb + j * (long long)a.B * a.p, a.cb + j * N);
}

template <typename R>
lqt_status launch_vec(const lqt_problem* P, int B, long long Tb, char* rb, char* cb,
                      cudaStream_t s) {
    VecArgs<R> a;
    a.T = P->T;
    a.Tb = Tb;
    a.p = P->p;
    a.B = B;
    auto in = [](const lqt_in& i, const R** ptr, long long* st) {
        *ptr = static_cast<const R*>(i.ptr);
        *st = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    a.rb = reinterpret_cast<R*>(rb);
    a.cb = reinterpret_cast<R*>(cb);
    const long long blocks = (Tb + kCondThreads - 1) / kCondThreads;
    if (blocks > INT32_MAX) return LQT_EINVAL;
    switch (P->n) {
        case 1: k_cond_vec<R, 1><<<(unsigned)blocks, kCondThreads, 0, s>>>(a); break;
        case 2: k_cond_vec<R, 2><<<(unsigned)blocks, kCondThreads, 0, s>>>(a); break;
        case 3: k_cond_vec<R, 3><<<(unsigned)blocks, kCondThreads, 0, s>>>(a); break;
        case 4: k_cond_vec<R, 4><<<(unsigned)blocks, kCondThreads, 0, s>>>(a); break;
        default: return LQT_EUNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

// Compiled (dtype, n, m, B): the condensed size (n, B m) has a solver.
struct CondVariant {
    int dtype, n, m, B;
    void (*condense)(const void* args, long long blocks, cudaStream_t s);
    void (*expand)(const void* args, long long blocks, cudaStream_t s);
};

template <typename R, int N, int M, int B>
void run_condense(const void* args, long long blocks, cudaStream_t s) {
    k_condense<R, N, M, B><<<(unsigned)blocks, kCondThreads, 0, s>>>(
        *static_cast<const CondArgs<R>*>(args));
}
template <typename R, int N, int M, int B>
void run_expand(const void* args, long long blocks, cudaStream_t s) {
    k_expand<R, N, M, B><<<(unsigned)blocks, kCondThreads, 0, s>>>(
        *static_cast<const CondArgs<R>*>(args));
}

#define LQT_COND(R, N, M, B)                                                        \
    CondVariant{sizeof(R) == 8 ? LQT_F64 : LQT_F32, N, M, B, &run_condense<R, N, M, B>, \
                &run_expand<R, N, M, B>}

const CondVariant kCondVariants[] = {
    LQT_COND(float, 2, 1, 2), LQT_COND(float, 3, 1, 2), LQT_COND(float, 4, 1, 2),
    LQT_COND(float, 4, 1, 4), LQT_COND(float, 4, 2, 2), LQT_COND(double, 4, 1, 2),
};

const CondVariant* find_cond(int dtype, int n, int m, int B) {
    for (const CondVariant& v : kCondVariants)
        if (v.dtype == dtype && v.n == n && v.m == m && v.B == B) return &v;
    return nullptr;
}

struct CondPlan {
    lqt_problem Pc;       // condensed problem (pointers into the workspace)
    lqt_cross cross;      // its cross weights
    lqt_solution sc;      // its solution (in the workspace)
    size_t cross_ws, Fb, Lb, cb, Ub, Hb, rb, Xb, Mb, Sb, vb, Kb, xb, ub, total;
    long long Tb;
    bool inv;
};

bool ok_in(const lqt_in& in, int64_t size, size_t es, bool required, int64_t T) {
    if (!in.ptr) return !(required && T > 0);
    if (reinterpret_cast<uintptr_t>(in.ptr) % es) return false;
    return in.step_stride == 0 || in.step_stride >= size;
}

// cross_min: the condensed solve's workspace is at least this large, so that
// the two solves of a refinement share one layout.
lqt_status plan_cond(const lqt_problem* P, int B, const lqt_options* o, char* base,
                     CondPlan* cp, size_t cross_min = 0) {
    if (!P || B < 1) return LQT_EINVAL;
    if (P->dtype != LQT_F32 && P->dtype != LQT_F64) return LQT_EINVAL;
    if (P->n < 1 || P->m < 1 || P->p < 0 || P->pT < 0 || P->T < 0 || !P->x0) return LQT_EINVAL;
    if (P->p > kCondPMax) return LQT_EUNSUPPORTED;
    if (!find_cond(P->dtype, P->n, P->m, B)) return LQT_EUNSUPPORTED;
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    const int64_t n = P->n, m = P->m, p = P->p;
    if (!ok_in(P->F, n * n, es, true, P->T) || !ok_in(P->L, n * m, es, true, P->T) ||
        !ok_in(P->U, m * m, es, true, P->T) || !ok_in(P->c, n, es, false, P->T) ||
        !ok_in(P->H, p * n, es, p > 0, P->T) || !ok_in(P->r, p, es, false, P->T) ||
        !ok_in(P->X, p * p, es, p > 0, P->T))
        return LQT_EINVAL;
    const long long Tb = (P->T + B - 1) / B;
    const int64_t mb = m * B, pb = p * B;
    cp->Tb = Tb;
    auto fixed = [](const lqt_in& in) { return !in.ptr || in.step_stride == 0; };
    // offsets c_k may vary: they enter only c_bar and r_bar, which are per block
    cp->inv = P->T % B == 0 && fixed(P->F) && fixed(P->L) && fixed(P->U) && fixed(P->H) &&
              fixed(P->X);
    const long long Tm = cp->inv ? 1 : Tb;  // rows of the block matrices
    const long long Tc = cp->inv && fixed(P->c) ? 1 : Tb;  // rows of c_bar
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up_p(bytes > 0 ? bytes : 1);
        return at;
    };
    const size_t Fb = take(Tm * n * n * es), Lb = take(Tm * n * mb * es), cb = take(Tb * n * es),
                 Ub = take(Tm * mb * mb * es), Hb = take(Tm * pb * n * es),
                 rb = take(Tb * pb * es), Xb = take(Tm * pb * pb * es),
                 Mb = take(Tm * pb * mb * es), Sb = take((Tb + 1) * n * n * es),
                 vb = take((Tb + 1) * n * es), Kb = take(Tb * mb * n * es),
                 xb = take((Tb + 1) * n * es), ub = take(Tb * mb * es);
    const size_t tail = off;
    char* bb = base ? base : reinterpret_cast<char*>(size_t(1) << 20);
    auto point = [&](size_t at0) {
        lqt_problem& Q = cp->Pc;
        Q = *P;
        Q.m = (int32_t)mb;
        Q.p = (int32_t)pb;
        Q.T = Tb;
        const int64_t v = cp->inv ? 0 : 1;  // step strides of the block matrices
        Q.F = lqt_in{bb + at0 + Fb, v * n * n};
        Q.L = lqt_in{bb + at0 + Lb, v * n * mb};
        Q.c = lqt_in{bb + at0 + cb, Tc > 1 ? n : 0};
        Q.U = lqt_in{bb + at0 + Ub, v * mb * mb};
        Q.H = lqt_in{pb > 0 ? bb + at0 + Hb : nullptr, v * pb * n};
        Q.r = lqt_in{pb > 0 ? bb + at0 + rb : nullptr, pb};
        Q.X = lqt_in{pb > 0 ? bb + at0 + Xb : nullptr, v * pb * pb};
        cp->cross.M = lqt_in{pb > 0 ? bb + at0 + Mb : nullptr, v * pb * mb};
        cp->cross.s = lqt_in{nullptr, 0};
        cp->sc.S = bb + at0 + Sb;
        cp->sc.v = bb + at0 + vb;
        cp->sc.K = bb + at0 + Kb;
        cp->sc.x = bb + at0 + xb;
        cp->sc.u = bb + at0 + ub;
    };
    point(kAlignP);
    const size_t cross_ws = lqt_cross_workspace_bytes(&cp->Pc, &cp->cross, o);
    if (cross_ws == 0) return LQT_EUNSUPPORTED;
    cp->cross_ws = up_p(cross_ws > cross_min ? cross_ws : cross_min);
    point(cp->cross_ws);
    cp->Fb = cp->cross_ws + Fb;
    cp->Lb = cp->cross_ws + Lb;
    cp->cb = cp->cross_ws + cb;
    cp->Ub = cp->cross_ws + Ub;
    cp->Hb = cp->cross_ws + Hb;
    cp->rb = cp->cross_ws + rb;
    cp->Xb = cp->cross_ws + Xb;
    cp->Mb = cp->cross_ws + Mb;
    cp->Sb = cp->cross_ws + Sb;
    cp->vb = cp->cross_ws + vb;
    cp->Kb = cp->cross_ws + Kb;
    cp->xb = cp->cross_ws + xb;
    cp->ub = cp->cross_ws + ub;
    cp->total = cp->cross_ws + tail;
    return LQT_OK;
}

template <typename R>
CondArgs<R> cond_args(const lqt_problem* P, const lqt_solution* sol, const CondPlan& cp,
                      char* base, const int* pre, bool shift_add) {
    CondArgs<R> a;
    a.T = P->T;
    a.Tb = cp.Tb;
    a.p = P->p;
    a.inv = cp.inv ? 1 : 0;
    auto in = [](const lqt_in& i, const R** ptr, long long* s) {
        *ptr = static_cast<const R*>(i.ptr);
        *s = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->L, &a.L, &a.sL);
    in(P->U, &a.U, &a.sU);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    in(P->X, &a.X, &a.sX);
    a.Fb = reinterpret_cast<R*>(base + cp.Fb);
    a.Lb = reinterpret_cast<R*>(base + cp.Lb);
    a.cb = reinterpret_cast<R*>(base + cp.cb);
    a.Ub = reinterpret_cast<R*>(base + cp.Ub);
    a.Hb = reinterpret_cast<R*>(base + cp.Hb);
    a.rb = reinterpret_cast<R*>(base + cp.rb);
    a.Xb = reinterpret_cast<R*>(base + cp.Xb);
    a.Mb = reinterpret_cast<R*>(base + cp.Mb);
    a.Sb = reinterpret_cast<const R*>(base + cp.Sb);
    a.vb = reinterpret_cast<const R*>(base + cp.vb);
    a.xb = reinterpret_cast<const R*>(base + cp.xb);
    a.ub = reinterpret_cast<const R*>(base + cp.ub);
    a.S = static_cast<R*>(sol->S);
    a.v = static_cast<R*>(sol->v);
    a.K = static_cast<R*>(sol->K);
    a.x = static_cast<R*>(sol->x);
    a.u = static_cast<R*>(sol->u);
    a.status = reinterpret_cast<int*>(base);
    a.pre_status = pre;
    a.shift_add = shift_add ? 1 : 0;
    return a;
}

// Rank-reduced variants: the original (n, m) of the expansion; the reduced
// problem is solved at (n, n).
struct RedVariant {
    int n, m;
    void (*reduce)(const void* args, unsigned grid, size_t smem, cudaStream_t s);
    void (*unreduce)(const void* args, long long blocks, cudaStream_t s);
    void (*expand)(const void* args, int B, long long blocks, cudaStream_t s);
};

template <typename R, int N, int M>
void run_reduce(const void* args, unsigned grid, size_t smem, cudaStream_t s) {
    static bool attr = false;  // a benign race: every caller sets the same value
    if (!attr) {
        cudaFuncSetAttribute(k_cond_reduce<R, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = true;
    }
    const RedArgs<R>& a = *static_cast<const RedArgs<R>*>(args);
    k_cond_reduce<R, N, M><<<grid, kRedThreads, smem, s>>>(a);
    if (a.inv) {
        const long long blocks = (a.Tb + kCondThreads - 1) / kCondThreads;
        k_cond_rbar<R, N><<<(unsigned)blocks, kCondThreads, 0, s>>>(a);
    }
}
template <typename R, int N>
void run_unreduce(const void* args, long long blocks, cudaStream_t s) {
    k_cond_unreduce<R, N><<<(unsigned)blocks, kCondThreads, 0, s>>>(
        *static_cast<const RedArgs<R>*>(args));
}
template <typename R, int N, int M>
void run_expand_rt(const void* args, int B, long long blocks, cudaStream_t s) {
    k_expand_rt<R, N, M><<<(unsigned)blocks, kCondThreads, 0, s>>>(
        *static_cast<const CondArgs<R>*>(args), B);
}

#define LQT_RED(N, M) \
    RedVariant { N, M, &run_reduce<float, N, M>, &run_unreduce<float, N>, &run_expand_rt<float, N, M> }
const RedVariant kRedVariants[] = {LQT_RED(4, 2), LQT_RED(4, 1), LQT_RED(2, 1), LQT_RED(2, 2),
                                   LQT_RED(1, 1)};

const RedVariant* find_red(int dtype, int n, int m) {
    if (dtype != LQT_F32) return nullptr;
    for (const RedVariant& v : kRedVariants)
        if (v.n == n && v.m == m) return &v;
    return nullptr;
}

struct RedPlan {
    lqt_problem Pc;   // reduced problem: n states, n controls, B p outputs, T/B steps
    lqt_cross cross;  // its cross weights M_r
    lqt_solution sc;  // its solution (w in sc.u)
    size_t cross_ws, Fb, cb, Lb, Ub, Hb, rb, Xb, Mb, Pb, Qb, HD, Sb, vb, Kb, xb, wb, ub, total;
    long long Tb;
    bool inv;
};

lqt_status plan_red(const lqt_problem* P, int B, const lqt_options* o, char* base, RedPlan* rp,
                    size_t cross_min = 0) {
    if (!P || B < 2) return LQT_EINVAL;
    if (P->n < 1 || P->m < 1 || P->p < 0 || P->pT < 0 || P->T < 0 || !P->x0) return LQT_EINVAL;
    if (!find_red(P->dtype, P->n, P->m)) return LQT_EUNSUPPORTED;
    const int64_t n = P->n, m = P->m, p = P->p;
    if (m * B > kRedMax || p * B > kRedMax) return LQT_EUNSUPPORTED;
    const size_t es = 4;
    if (!ok_in(P->F, n * n, es, true, P->T) || !ok_in(P->L, n * m, es, true, P->T) ||
        !ok_in(P->U, m * m, es, true, P->T) || !ok_in(P->c, n, es, false, P->T) ||
        !ok_in(P->H, p * n, es, p > 0, P->T) || !ok_in(P->r, p, es, false, P->T) ||
        !ok_in(P->X, p * p, es, p > 0, P->T))
        return LQT_EINVAL;
    const long long Tb = (P->T + B - 1) / B;
    const int64_t mb = m * B, pb = p * B;
    rp->Tb = Tb;
    auto fixed = [](const lqt_in& in) { return !in.ptr || in.step_stride == 0; };
    rp->inv = P->T % B == 0 && fixed(P->F) && fixed(P->L) && fixed(P->U) && fixed(P->H) &&
              fixed(P->X);
    const long long Tm = rp->inv ? 1 : Tb;
    const long long Tc = rp->inv && fixed(P->c) ? 1 : Tb;  // rows of c_bar
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at0 = off;
        off += up_p(bytes > 0 ? bytes : 1);
        return at0;
    };
    const size_t Fb = take(Tm * n * n * es), cb = take(Tb * n * es), Lb = take(Tm * n * n * es),
                 Ub = take(Tm * n * n * es), Hb = take(Tm * pb * n * es), rb = take(Tb * pb * es),
                 Xb = take(Tm * pb * pb * es), Mb = take(Tm * pb * n * es),
                 Pb = take(Tm * mb * n * es), Qb = take(Tm * mb * pb * es),
                 HD = take((size_t)B * p * sizeof(double)), Sb = take((Tb + 1) * n * n * es),
                 vb = take((Tb + 1) * n * es), Kb = take(Tb * n * n * es),
                 xb = take((Tb + 1) * n * es), wb = take(Tb * n * es), ub = take(Tb * mb * es);
    const size_t tail = off;
    char* bb = base ? base : reinterpret_cast<char*>(size_t(1) << 20);
    auto point = [&](size_t at0) {
        lqt_problem& Q = rp->Pc;
        Q = *P;
        Q.m = (int32_t)n;
        Q.p = (int32_t)pb;
        Q.T = Tb;
        const int64_t v = rp->inv ? 0 : 1;
        Q.F = lqt_in{bb + at0 + Fb, v * n * n};
        Q.c = lqt_in{bb + at0 + cb, Tc > 1 ? n : 0};
        Q.L = lqt_in{bb + at0 + Lb, v * n * n};
        Q.U = lqt_in{bb + at0 + Ub, v * n * n};
        Q.H = lqt_in{pb > 0 ? bb + at0 + Hb : nullptr, v * pb * n};
        Q.r = lqt_in{pb > 0 ? bb + at0 + rb : nullptr, pb};
        Q.X = lqt_in{pb > 0 ? bb + at0 + Xb : nullptr, v * pb * pb};
        rp->cross.M = lqt_in{pb > 0 ? bb + at0 + Mb : nullptr, v * pb * n};
        rp->cross.s = lqt_in{nullptr, 0};
        rp->sc.S = bb + at0 + Sb;
        rp->sc.v = bb + at0 + vb;
        rp->sc.K = bb + at0 + Kb;
        rp->sc.x = bb + at0 + xb;
        rp->sc.u = bb + at0 + wb;
    };
    point(kAlignP);
    const size_t cross_ws = lqt_cross_workspace_bytes(&rp->Pc, &rp->cross, o);
    if (cross_ws == 0) return LQT_EUNSUPPORTED;
    rp->cross_ws = up_p(cross_ws > cross_min ? cross_ws : cross_min);
    point(rp->cross_ws);
    const size_t o0 = rp->cross_ws;
    rp->Fb = o0 + Fb;
    rp->cb = o0 + cb;
    rp->Lb = o0 + Lb;
    rp->Ub = o0 + Ub;
    rp->Hb = o0 + Hb;
    rp->rb = o0 + rb;
    rp->Xb = o0 + Xb;
    rp->Mb = o0 + Mb;
    rp->Pb = o0 + Pb;
    rp->Qb = o0 + Qb;
    rp->HD = o0 + HD;
    rp->Sb = o0 + Sb;
    rp->vb = o0 + vb;
    rp->Kb = o0 + Kb;
    rp->xb = o0 + xb;
    rp->wb = o0 + wb;
    rp->ub = o0 + ub;
    rp->total = o0 + tail;
    return LQT_OK;
}

RedArgs<float> red_args(const lqt_problem* P, int B, const RedPlan& rp, char* base, int* pre) {
    RedArgs<float> a;
    a.T = P->T;
    a.Tb = rp.Tb;
    a.m = P->m;
    a.p = P->p;
    a.B = B;
    a.inv = rp.inv ? 1 : 0;
    auto in = [](const lqt_in& i, const float** ptr, long long* s) {
        *ptr = static_cast<const float*>(i.ptr);
        *s = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->L, &a.L, &a.sL);
    in(P->U, &a.U, &a.sU);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    in(P->X, &a.X, &a.sX);
    a.Fb = reinterpret_cast<float*>(base + rp.Fb);
    a.cb = reinterpret_cast<float*>(base + rp.cb);
    a.Lb = reinterpret_cast<float*>(base + rp.Lb);
    a.Ub = reinterpret_cast<float*>(base + rp.Ub);
    a.Hb = reinterpret_cast<float*>(base + rp.Hb);
    a.rb = reinterpret_cast<float*>(base + rp.rb);
    a.Xb = reinterpret_cast<float*>(base + rp.Xb);
    a.Mb = reinterpret_cast<float*>(base + rp.Mb);
    a.Pb = reinterpret_cast<float*>(base + rp.Pb);
    a.Qb = reinterpret_cast<float*>(base + rp.Qb);
    a.HD = reinterpret_cast<double*>(base + rp.HD);
    a.xb = reinterpret_cast<const float*>(base + rp.xb);
    a.wb = reinterpret_cast<const float*>(base + rp.wb);
    a.ub = reinterpret_cast<float*>(base + rp.ub);
    a.status = pre;
    return a;
}

// The expansion's arguments from the reduced plan (the CondArgs of the small path).
CondArgs<float> red_expand_args(const lqt_problem* P, const lqt_solution* sol, const RedPlan& rp,
                                char* base, const int* pre, bool shift_add) {
    CondArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.T = P->T;
    a.Tb = rp.Tb;
    a.p = P->p;
    a.inv = rp.inv ? 1 : 0;
    auto in = [](const lqt_in& i, const float** ptr, long long* s) {
        *ptr = static_cast<const float*>(i.ptr);
        *s = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->L, &a.L, &a.sL);
    in(P->U, &a.U, &a.sU);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    in(P->X, &a.X, &a.sX);
    a.Sb = reinterpret_cast<const float*>(base + rp.Sb);
    a.vb = reinterpret_cast<const float*>(base + rp.vb);
    a.xb = reinterpret_cast<const float*>(base + rp.xb);
    a.ub = reinterpret_cast<const float*>(base + rp.ub);
    a.S = static_cast<float*>(sol->S);
    a.v = static_cast<float*>(sol->v);
    a.K = static_cast<float*>(sol->K);
    a.x = static_cast<float*>(sol->x);
    a.u = static_cast<float*>(sol->u);
    a.status = reinterpret_cast<int*>(base);
    a.pre_status = pre;
    a.shift_add = shift_add ? 1 : 0;
    return a;
}

// ---- refinement of the condensed solve --------------------------------------
// The expansion rebuilds u_bar = P z - Q (H_bar x - r_bar) (or the condensed
// solver's u_bar) from block starts and references of order one, a small
// difference of large terms when the tracking error is small; the error of
// u grows with B.  As lqt_solve does for n <= 4, the whole condensed solve
// runs twice: on the problem, giving x^, then on the problem shifted by x^
// (x = x^ + xi: r'_k = r_k - H_k x^_k, c'_k = F_k x^_k + c_k - x^_{k+1},
// r'_T = r_T - H_T x^_T, x'_0 = 0; the same matrices, so S, K are those of
// the first solve), whose controls are u* and whose states are xi.  The
// shifted data are compensated dot products; every term of the second
// solve is of the size of u.  S, v, K are the first solve's.

template <typename R>
struct ShiftArgs {
    long long T;
    int n, p, pT;
    const R *F, *c, *H, *r, *HT, *rT;
    long long sF, sc, sH, sr;
    const R* x;  // x^ (T + 1 states)
    R *rp, *cp, *rTp, *x0p;
    const int* status;  // the first solve's status
    int* pre_status;    // carried into the second solve's
};

// One thread per step k < T (r'_k, c'_k); thread T writes r'_T and x'_0 and
// carries the first solve's status.
template <typename R>
__global__ void __launch_bounds__(kCondThreads) k_cond_shift(ShiftArgs<R> a) {
    const long long k = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (k > a.T) return;
    const int n = a.n;
    const R* x = a.x + k * n;
    if (k == a.T) {
        for (int q = 0; q < a.pT; ++q) {
            Dot2<R> acc(a.rT ? a.rT[q] : R(0));
            for (int s = 0; s < n; ++s) acc.add_prod(-a.HT[q * n + s], x[s]);
            a.rTp[q] = acc.value();
        }
        for (int s = 0; s < n; ++s) a.x0p[s] = R(0);
        if (*a.status != 0) atomicCAS(a.pre_status, 0, *a.status);
        return;
    }
    const R* F = a.F + a.sF * k;
    const R* c = at(a.c, a.sc, k);
    const R* H = at(a.H, a.sH, k);
    const R* r = at(a.r, a.sr, k);
    for (int q = 0; q < a.p; ++q) {
        Dot2<R> acc(r ? r[q] : R(0));
        for (int s = 0; s < n; ++s) acc.add_prod(-H[q * n + s], x[s]);
        a.rp[k * a.p + q] = acc.value();
    }
    for (int i = 0; i < n; ++i) {
        Dot2<R> acc(c ? c[i] : R(0));
        for (int s = 0; s < n; ++s) acc.add_prod(F[i * n + s], x[s]);
        acc.add(-x[n + i]);
        a.cp[k * n + i] = acc.value();
    }
}

// Workspace after the condensed solve's own: the status word of the kernels
// before the condensed solve, then (refined) the shifted data.
struct Tail {
    size_t cross;  // workspace of the condensed solve (the same for both solves)
    size_t pre, rp, cp, rTp, x0p, total;
};

Tail tail_layout(const lqt_problem* P, size_t core, bool refine) {
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    Tail t;
    size_t off = core;
    auto take = [&](size_t bytes) {
        const size_t at0 = off;
        off += up_p(bytes > 0 ? bytes : 1);
        return at0;
    };
    t.pre = take(sizeof(int));
    t.rp = t.cp = t.rTp = t.x0p = 0;
    if (refine) {
        t.rp = take((size_t)P->T * P->p * es);
        t.cp = take((size_t)P->T * P->n * es);
        t.rTp = take((size_t)P->pT * es);
        t.x0p = take((size_t)P->n * es);
    }
    t.total = off;
    return t;
}

// The shifted problem: the same matrices, r', c', r'_T, x'_0 at `base` + the
// tail's offsets (any base with the workspace's alignment, for sizing).
lqt_problem shifted(const lqt_problem* P, char* base, const Tail& t) {
    lqt_problem Q = *P;
    Q.r = lqt_in{P->p > 0 ? base + t.rp : nullptr, P->p};
    Q.c = lqt_in{base + t.cp, P->n};
    Q.rT = P->pT > 0 ? base + t.rTp : nullptr;
    Q.x0 = base + t.x0p;
    return Q;
}

// Workspace of one condensed solve of P (either path) and of its condensed
// solve within it, or the error.
lqt_status core_bytes(const lqt_problem* P, int B, const lqt_options* o, size_t cross_min,
                      size_t* bytes, size_t* cross) {
    CondPlan cp;
    lqt_status st = plan_cond(P, B, o, nullptr, &cp, cross_min);
    if (st == LQT_OK) {
        *bytes = cp.total;
        *cross = cp.cross_ws;
        return st;
    }
    if (st != LQT_EUNSUPPORTED) return st;
    RedPlan rp;
    if ((st = plan_red(P, B, o, nullptr, &rp, cross_min)) == LQT_OK) {
        *bytes = rp.total;
        *cross = rp.cross_ws;
    }
    return st;
}

// Refinement of a condensed solve: two solves (see above) for LQT_REFINE_ON
// and LQT_REFINE_FULL (and AUTO on FP32); the condensed problem itself is
// solved without refinement either way.
lqt_status condensed_options(const lqt_problem* P, const lqt_options* o, bool* twice,
                             lqt_options* inner) {
    lqt_options d;
    memset(&d, 0, sizeof(d));
    d.refine = LQT_REFINE_AUTO;
    if (o) d = *o;
    const int r = d.refine;
    if (r != LQT_REFINE_OFF && r != LQT_REFINE_ON && r != LQT_REFINE_AUTO && r != LQT_REFINE_FULL)
        return LQT_EINVAL;
    *twice = r == LQT_REFINE_ON || r == LQT_REFINE_FULL || (r == LQT_REFINE_AUTO && P->dtype == LQT_F32);
    *inner = d;
    inner->refine = LQT_REFINE_OFF;
    return LQT_OK;
}

lqt_status sizes(const lqt_problem* P, int B, const lqt_options* o, bool* twice,
                 lqt_options* inner, Tail* t) {
    lqt_status st = condensed_options(P, o, twice, inner);
    if (st != LQT_OK) return st;
    size_t core = 0, cross = 0;
    if ((st = core_bytes(P, B, inner, 0, &core, &cross)) != LQT_OK) return st;
    if (*twice) {
        // the second solve keeps the first's block matrices: one layout for both
        const Tail t0 = tail_layout(P, 0, true);
        const lqt_problem P2 = shifted(P, reinterpret_cast<char*>(size_t(1) << 20), t0);
        size_t core2 = 0, cross2 = 0;
        if ((st = core_bytes(&P2, B, inner, cross, &core2, &cross2)) != LQT_OK) return st;
        if (cross2 > cross &&
            (st = core_bytes(P, B, inner, cross2, &core, &cross)) != LQT_OK)
            return st;
        if (core2 > core) core = core2;
    }
    *t = tail_layout(P, up_p(core), *twice);
    t->cross = cross;
    return LQT_OK;
}

lqt_status solve_reduced(const lqt_problem* prob, int32_t B, const lqt_solution* sol,
                         const lqt_options* opts, char* base, int* pre, bool shift_add,
                         size_t cross, cudaStream_t s) {
    RedPlan rp;
    lqt_status st = plan_red(prob, B, opts, base, &rp, cross);
    if (st != LQT_OK) return st;
    st = lqt_solve_cross(&rp.Pc, &rp.cross, &rp.sc, opts, base, 0, s);
    if (st != LQT_ENOMEM) return st == LQT_OK ? LQT_EINVAL : st;
    const RedVariant* var = find_red(prob->dtype, prob->n, prob->m);
    const long long blocks = (rp.Tb + kCondThreads - 1) / kCondThreads;
    if (blocks > INT32_MAX || rp.Tb > INT32_MAX) return LQT_EINVAL;
    const size_t smem = (size_t)RedSmem<4>::SIZE * sizeof(double);
    const RedArgs<float> a = red_args(prob, B, rp, base, pre);
    if (shift_add) {
        // the second solve of the refinement: the first's reduction stands
        if ((st = launch_vec<float>(prob, B, rp.Tb, base + rp.rb, base + rp.cb, s)) != LQT_OK)
            return st;
    } else {
        var->reduce(&a, rp.inv ? 1u : (unsigned)rp.Tb, smem, s);
        if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
    }
    if ((st = lqt_solve_cross(&rp.Pc, &rp.cross, &rp.sc, opts, base, rp.cross_ws, s)) != LQT_OK)
        return st;
    var->unreduce(&a, blocks, s);
    const CondArgs<float> e = red_expand_args(prob, sol, rp, base, pre, shift_add);
    var->expand(&e, B, blocks, s);
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

// One condensed solve of prob into sol (shift_add: the second solve of the
// refinement, which adds its states to sol->x and writes sol->u only).
lqt_status solve_once(const lqt_problem* prob, int32_t B, const lqt_solution* sol,
                      const lqt_options* opts, char* base, int* pre, bool shift_add,
                      size_t cross, cudaStream_t s) {
    CondPlan cp;
    lqt_status st = plan_cond(prob, B, opts, base, &cp, cross);
    if (st == LQT_EUNSUPPORTED)
        return solve_reduced(prob, B, sol, opts, base, pre, shift_add, cross, s);
    if (st != LQT_OK) return st;
    // argument check of the condensed solve before anything is launched
    st = lqt_solve_cross(&cp.Pc, &cp.cross, &cp.sc, opts, base, 0, s);
    if (st != LQT_ENOMEM) return st == LQT_OK ? LQT_EINVAL : st;
    const CondVariant* var = find_cond(prob->dtype, prob->n, prob->m, B);
    const long long blocks = (cp.Tb + kCondThreads - 1) / kCondThreads;
    if (blocks > INT32_MAX) return LQT_EINVAL;
    if (shift_add) {
        // the second solve of the refinement: the first's block matrices stand
        st = prob->dtype == LQT_F64
                 ? launch_vec<double>(prob, B, cp.Tb, base + cp.rb, base + cp.cb, s)
                 : launch_vec<float>(prob, B, cp.Tb, base + cp.rb, base + cp.cb, s);
        if (st != LQT_OK) return st;
    } else if (prob->dtype == LQT_F64) {
        const CondArgs<double> a = cond_args<double>(prob, sol, cp, base, pre, shift_add);
        var->condense(&a, blocks, s);
    } else {
        const CondArgs<float> a = cond_args<float>(prob, sol, cp, base, pre, shift_add);
        var->condense(&a, blocks, s);
    }
    if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
    if ((st = lqt_solve_cross(&cp.Pc, &cp.cross, &cp.sc, opts, base, cp.cross_ws, s)) != LQT_OK)
        return st;
    if (prob->dtype == LQT_F64) {
        const CondArgs<double> a = cond_args<double>(prob, sol, cp, base, pre, shift_add);
        var->expand(&a, blocks, s);
    } else {
        const CondArgs<float> a = cond_args<float>(prob, sol, cp, base, pre, shift_add);
        var->expand(&a, blocks, s);
    }
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

template <typename R>
lqt_status launch_shift(const lqt_problem* P, const lqt_solution* sol, char* base,
                        const Tail& t, cudaStream_t s) {
    ShiftArgs<R> a;
    a.T = P->T;
    a.n = P->n;
    a.p = P->p;
    a.pT = P->pT;
    auto in = [](const lqt_in& i, const R** ptr, long long* st) {
        *ptr = static_cast<const R*>(i.ptr);
        *st = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    a.HT = static_cast<const R*>(P->HT);
    a.rT = static_cast<const R*>(P->rT);
    a.x = static_cast<const R*>(sol->x);
    a.rp = reinterpret_cast<R*>(base + t.rp);
    a.cp = reinterpret_cast<R*>(base + t.cp);
    a.rTp = reinterpret_cast<R*>(base + t.rTp);
    a.x0p = reinterpret_cast<R*>(base + t.x0p);
    a.status = reinterpret_cast<const int*>(base);
    a.pre_status = reinterpret_cast<int*>(base + t.pre);
    const long long blocks = (P->T + 1 + kCondThreads - 1) / kCondThreads;
    if (blocks > INT32_MAX) return LQT_EINVAL;
    k_cond_shift<R><<<(unsigned)blocks, kCondThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_condensed_workspace_bytes(const lqt_problem* prob, int32_t B,
                                     const lqt_options* opts) {
    if (prob && B == 1) return lqt_workspace_bytes(prob, opts);
    if (!prob) return 0;
    bool twice = false;
    lqt_options inner;
    Tail t;
    return sizes(prob, B, opts, &twice, &inner, &t) == LQT_OK ? t.total : 0;
}

lqt_status lqt_solve_condensed(const lqt_problem* prob, int32_t B, const lqt_solution* sol,
                               const lqt_options* opts, void* workspace, size_t workspace_bytes,
                               void* stream) {
    if (!prob || !sol) return LQT_EINVAL;
    if (B == 1) return lqt_solve(prob, sol, opts, workspace, workspace_bytes, stream);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlignP) return LQT_EINVAL;
    char* base = static_cast<char*>(workspace);
    bool twice = false;
    lqt_options inner;
    Tail t;
    lqt_status st = sizes(prob, B, opts, &twice, &inner, &t);
    if (st != LQT_OK) return st;
    if (workspace_bytes < t.total) return LQT_ENOMEM;
    if (prob->T == 0) return LQT_EUNSUPPORTED;  // nothing to condense: use lqt_solve
    const void* outs[] = {sol->S, sol->v, sol->K, sol->x, sol->u};
    for (const void* q : outs)
        if (!q || reinterpret_cast<uintptr_t>(q) % 16) return LQT_EINVAL;
    if (prob->pT > 0 && !prob->HT) return LQT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* pre = reinterpret_cast<int*>(base + t.pre);
    if (cudaMemsetAsync(pre, 0, sizeof(int), s) != cudaSuccess) return LQT_ECUDA;
    if ((st = solve_once(prob, B, sol, &inner, base, pre, false, t.cross, s)) != LQT_OK || !twice)
        return st;
    st = prob->dtype == LQT_F64 ? launch_shift<double>(prob, sol, base, t, s)
                                : launch_shift<float>(prob, sol, base, t, s);
    if (st != LQT_OK) return st;
    const lqt_problem P2 = shifted(prob, base, t);
    return solve_once(&P2, B, sol, &inner, base, pre, true, t.cross, s);
}

}  // extern "C"
