// Generalised stage cost with a cross weight and a control offset (Sec. IV-D,
// eq. generalised_cost):
//
//   l_k(x, u) = 1/2 e^T X_k e + e^T M_k (u - s_k) + 1/2 (u - s_k)^T U_k (u - s_k),
//   e = H_k x - r_k.
//
// The paper reduces it to eq. LQT_problem by the substitution
// u~_k = W_k (H_k x_k - r_k) + u_k - s_k with W_k = U_k^{-1} M_k^T:
//
//   F~_k = F_k - L_k W_k H_k,   c~_k = c_k + L_k (W_k r_k + s_k),
//   X~_k = X_k - M_k W_k,       U~_k = U_k,
//
// and recovers u_k = u~_k - W_k (H_k x_k - r_k) + s_k.  The gain of the original
// control law is K_k = K~_k + W_k H_k; S_k, v_k and x*_k are unchanged.
//
// Three steps on the caller's stream: k_cross_pre writes F~, c~, X~ and the
// post-transform terms (W_k H_k, g_k = W_k r_k + s_k) into the workspace, lqt_solve
// solves the transformed problem, and k_cross_post turns K~, u~ into K, u:
//   K_k = K~_k + (W H)_k,   u_k = u~_k - (W H)_k x*_k + g_k.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lqt.h"
#include "lqt_lanes.cuh"
#include "lqt_variants.h"

namespace lqt {
namespace {

constexpr size_t kAlign = 256;
constexpr int kPreThreads = 128;
constexpr int kVecMaxM = 32;  // largest m of k_cross_vec

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

template <typename R>
struct CrossPre {
    int n, m, p;
    long long rows;  // steps with work (T, or 1 when every output is time-invariant)
    int group_elems;
    const R *F, *c, *L, *U, *H, *r, *X, *M, *s;
    long long sF, sc, sL, sU, sH, sr, sX, sM, ss;
    R *Ft, *ct, *Xt, *WH, *g;           // outputs (null: not needed)
    R* Wm;                              // W of step 0 (m x p), for k_cross_vec (null: none)
    long long oF, oc, oX, oW, og;       // output step strides (0: time-invariant)
    int* status;                        // transform status word
};

// Lane groups of G lanes, one group per step.  Per group in shared memory:
// U (m x m, overwritten by its Cholesky factor), W (m x p, starts as M^T),
// W H (m x n) and g (m); odd row strides.
template <typename R, int G>
__global__ void __launch_bounds__(kPreThreads) k_cross_pre(CrossPre<R> a) {
    extern __shared__ __align__(16) unsigned char cross_smem[];
    const int gi = threadIdx.x / G;
    const long long k = (long long)blockIdx.x * (kPreThreads / G) + gi;
    if (k >= a.rows) return;  // whole groups leave together
    const lanes::Group<G> grp;
    const int lane = grp.lr;
    const int n = a.n, m = a.m, p = a.p;
    const int ldu = m | 1, ldw = p | 1, ldh = n | 1;
    R* Us = reinterpret_cast<R*>(cross_smem) + (size_t)gi * a.group_elems;
    R* Ws = Us + m * ldu;
    R* WHs = Ws + m * ldw;
    R* gs = WHs + m * ldh;

    const R* U = a.U + a.sU * k;
    const R* M = a.M ? a.M + a.sM * k : nullptr;
    const R* H = a.H ? a.H + a.sH * k : nullptr;
    const R* r = a.r ? a.r + a.sr * k : nullptr;
    const R* s = a.s ? a.s + a.ss * k : nullptr;
    const R* L = a.L + a.sL * k;

    if (M) {
        for (int e = lane; e < m * m; e += G) Us[(e / m) * ldu + e % m] = U[e];
        for (int e = lane; e < p * m; e += G) Ws[(e % m) * ldw + e / m] = M[e];  // M^T
        grp.sync();
        // Cholesky U = R R^T (lower factor in place), column by column
        bool ok = true;
        for (int j = 0; j < m; ++j) {
            const R d = Us[j * ldu + j];
            ok = ok && d > R(0) && isfinite(d);
            const R ljj = sqrt(d);
            const R inv = R(1) / ljj;
            grp.sync();
            for (int i = j + 1 + lane; i < m; i += G) Us[i * ldu + j] *= inv;
            if (lane == 0) Us[j * ldu + j] = ljj;
            grp.sync();
            const int t = m - j - 1;
            for (int e = lane; e < t * t; e += G) {
                const int i = j + 1 + e / t, l = j + 1 + e % t;
                if (l <= i) Us[i * ldu + l] -= Us[i * ldu + j] * Us[l * ldu + j];
            }
            grp.sync();
        }
        if (!ok) {
            if (lane == 0) atomicCAS(a.status, 0, (int)LQT_ENOTSPD);
            return;
        }
        // W = U^{-1} M^T: one column per lane, R y = M^T col, then R^T w = y
        for (int j = lane; j < p; j += G) {
            for (int i = 0; i < m; ++i) {
                R acc = Ws[i * ldw + j];
                for (int l = 0; l < i; ++l) acc -= Us[i * ldu + l] * Ws[l * ldw + j];
                Ws[i * ldw + j] = acc / Us[i * ldu + i];
            }
            for (int i = m - 1; i >= 0; --i) {
                R acc = Ws[i * ldw + j];
                for (int l = i + 1; l < m; ++l) acc -= Us[l * ldu + i] * Ws[l * ldw + j];
                Ws[i * ldw + j] = acc / Us[i * ldu + i];
            }
        }
        grp.sync();
    }

    // (W H)_k and g_k = W_k r_k + s_k
    const bool first = k == 0;
    if (M && a.Wm && first)
        for (int e = lane; e < m * p; e += G) a.Wm[e] = Ws[(e / p) * ldw + e % p];
    for (int e = lane; e < m * n; e += G) {
        const int i = e / n, l = e % n;
        R acc = R(0);
        if (M)
            for (int j = 0; j < p; ++j) acc += Ws[i * ldw + j] * H[j * n + l];
        WHs[i * ldh + l] = acc;
        if (a.WH && (a.oW || first)) a.WH[a.oW * k + e] = acc;
    }
    for (int i = lane; i < m; i += G) {
        R acc = s ? s[i] : R(0);
        if (M && r)
            for (int j = 0; j < p; ++j) acc += Ws[i * ldw + j] * r[j];
        gs[i] = acc;
        if (a.g && (a.og || first)) a.g[a.og * k + i] = acc;
    }
    grp.sync();

    // F~ = F - L (W H),  c~ = c + L g
    if (a.Ft && (a.oF || first)) {
        const R* F = a.F + a.sF * k;
        for (int e = lane; e < n * n; e += G) {
            const int i = e / n, l = e % n;
            R acc = F[e];
            for (int q = 0; q < m; ++q) acc -= L[i * m + q] * WHs[q * ldh + l];
            a.Ft[a.oF * k + e] = acc;
        }
    }
    if (a.ct && (a.oc || first)) {
        const R* c = a.c ? a.c + a.sc * k : nullptr;
        for (int i = lane; i < n; i += G) {
            R acc = c ? c[i] : R(0);
            for (int q = 0; q < m; ++q) acc += L[i * m + q] * gs[q];
            a.ct[a.oc * k + i] = acc;
        }
    }
    // X~ = X - M W, each entry (i, j) computed as its upper-triangle twin so
    // that X~ is exactly symmetric
    if (M && a.Xt && (a.oX || first)) {
        const R* X = a.X + a.sX * k;
        for (int e = lane; e < p * p; e += G) {
            const int i0 = e / p, j0 = e % p;
            const int i = i0 < j0 ? i0 : j0, j = i0 < j0 ? j0 : i0;
            R acc = X[i * p + j];
            for (int q = 0; q < m; ++q) acc -= M[i * m + q] * Ws[q * ldw + j];
            a.Xt[a.oX * k + e] = acc;
        }
    }
}

// One thread per step for the compiled small sizes (n = NX, m = MX, p <= PX):
// the same arithmetic as k_cross_pre with every matrix in registers (the p
// loops run to the compile-time bound with run-time guards, so indexing stays
// static).
// Time-varying outputs leave through a shared-memory stage so that each block
// writes one contiguous run per array (a thread's own rows are 16 to 256
// bytes apart from its neighbours').
constexpr int kSmallThreads = 64;

// Copies the rows the block's threads left in the stage to out[k0 * E ...]
// (one contiguous run), or, for a time-invariant output, step 0's row alone.
template <typename R>
__device__ __forceinline__ void stage_flush(const R* stage, int lds, int E, R* out,
                                            long long stride, long long k0, int nvalid,
                                            bool first) {
    __syncthreads();
    if (stride) {
        const int count = nvalid * E;
        R* dst = out + k0 * E;
        for (int i = threadIdx.x; i < count; i += kSmallThreads)
            dst[i] = stage[(i / E) * lds + i % E];
    } else if (first) {
        for (int e = 0; e < E; ++e) out[e] = stage[threadIdx.x * lds + e];
    }
    __syncthreads();
}

template <typename R, int NX, int MX, int PX>
__global__ void __launch_bounds__(kSmallThreads) k_cross_pre_small(CrossPre<R> a) {
    constexpr int LDS = (NX * NX > PX * PX ? NX * NX : PX * PX) | 1;
    __shared__ R stage[kSmallThreads * LDS];
    const long long k0 = (long long)blockIdx.x * kSmallThreads;
    const long long k = k0 + threadIdx.x;
    const bool valid = k < a.rows;
    const int nvalid = (int)(a.rows - k0 < kSmallThreads ? a.rows - k0 : kSmallThreads);
    const long long kk = valid ? k : k0;  // in-range index for the loads of idle threads
    constexpr int n = NX, m = MX;
    const int p = a.p;
    const R* U = a.U + a.sU * kk;
    const R* M = a.M ? a.M + a.sM * kk : nullptr;
    const R* H = a.H ? a.H + a.sH * kk : nullptr;
    const R* r = a.r ? a.r + a.sr * kk : nullptr;
    const R* s = a.s ? a.s + a.ss * kk : nullptr;
    const R* L = a.L + a.sL * kk;
    const bool first = k == 0;
    R W[MX][PX];  // U^{-1} M^T
#pragma unroll
    for (int i = 0; i < MX; ++i)
#pragma unroll
        for (int j = 0; j < PX; ++j) W[i][j] = (M && i < m && j < p) ? M[j * m + i] : R(0);
    if (M) {
        // Cholesky U = R R^T in registers
        R C[MX][MX];
#pragma unroll
        for (int i = 0; i < MX; ++i)
#pragma unroll
            for (int j = 0; j < MX; ++j) C[i][j] = (i < m && j < m) ? U[i * m + j] : R(1);
        bool ok = true;
#pragma unroll
        for (int j = 0; j < MX; ++j) {
            if (j < m) {
                R d = C[j][j];
#pragma unroll
                for (int l = 0; l < MX; ++l)
                    if (l < j) d -= C[j][l] * C[j][l];
                ok = ok && d > R(0) && isfinite(d);
                const R ljj = sqrt(d);
                const R inv = R(1) / ljj;
                C[j][j] = inv;  // the factor's diagonal is kept as its reciprocal
#pragma unroll
                for (int i = 0; i < MX; ++i)
                    if (i > j && i < m) {
                        R acc = C[i][j];
#pragma unroll
                        for (int l = 0; l < MX; ++l)
                            if (l < j) acc -= C[i][l] * C[j][l];
                        C[i][j] = acc * inv;
                    }
            }
        }
        if (!ok && valid) atomicCAS(a.status, 0, (int)LQT_ENOTSPD);
        // R y = M^T, then R^T w = y, for the p columns
#pragma unroll
        for (int j = 0; j < PX; ++j)
            if (j < p) {
#pragma unroll
                for (int i = 0; i < MX; ++i)
                    if (i < m) {
                        R acc = W[i][j];
#pragma unroll
                        for (int l = 0; l < MX; ++l)
                            if (l < i) acc -= C[i][l] * W[l][j];
                        W[i][j] = acc * C[i][i];
                    }
#pragma unroll
                for (int i = MX - 1; i >= 0; --i)
                    if (i < m) {
                        R acc = W[i][j];
#pragma unroll
                        for (int l = 0; l < MX; ++l)
                            if (l > i && l < m) acc -= C[l][i] * W[l][j];
                        W[i][j] = acc * C[i][i];
                    }
            }
    }
    R WH[MX * NX], g[MX];
#pragma unroll
    for (int i = 0; i < MX; ++i) {
        R acc = (s && i < m) ? s[i] : R(0);
#pragma unroll
        for (int j = 0; j < PX; ++j)
            if (M && r && i < m && j < p) acc += W[i][j] * r[j];
        g[i] = acc;
#pragma unroll
        for (int l = 0; l < NX; ++l) {
            R h = R(0);
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if (M && i < m && j < p && l < n) h += W[i][j] * H[j * n + l];
            WH[i * NX + l] = h;
        }
    }
    // outputs, each packed to its run-time size in this thread's stage row
    if (M && a.Wm && first)
#pragma unroll
        for (int i = 0; i < MX; ++i)
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if (i < m && j < p) a.Wm[i * p + j] = W[i][j];
    R* row = stage + threadIdx.x * LDS;
    if (a.WH) {
#pragma unroll
        for (int i = 0; i < MX; ++i)
#pragma unroll
            for (int l = 0; l < NX; ++l)
                if (i < m && l < n) row[i * n + l] = WH[i * NX + l];
        stage_flush(stage, LDS, m * n, a.WH, a.oW, k0, nvalid, first);
    }
    if (a.g) {
#pragma unroll
        for (int i = 0; i < MX; ++i)
            if (i < m) row[i] = g[i];
        stage_flush(stage, LDS, m, a.g, a.og, k0, nvalid, first);
    }
    if (a.Ft) {
        const R* F = a.F + a.sF * kk;
#pragma unroll
        for (int i = 0; i < NX; ++i)
#pragma unroll
            for (int l = 0; l < NX; ++l)
                if (i < n && l < n) {
                    R acc = F[i * n + l];
#pragma unroll
                    for (int q = 0; q < MX; ++q)
                        if (q < m) acc -= L[i * m + q] * WH[q * NX + l];
                    row[i * n + l] = acc;
                }
        stage_flush(stage, LDS, n * n, a.Ft, a.oF, k0, nvalid, first);
    }
    if (a.ct) {
        const R* c = a.c ? a.c + a.sc * kk : nullptr;
#pragma unroll
        for (int i = 0; i < NX; ++i)
            if (i < n) {
                R acc = c ? c[i] : R(0);
#pragma unroll
                for (int q = 0; q < MX; ++q)
                    if (q < m) acc += L[i * m + q] * g[q];
                row[i] = acc;
            }
        stage_flush(stage, LDS, n, a.ct, a.oc, k0, nvalid, first);
    }
    if (a.M && a.Xt) {
        const R* X = a.X + a.sX * kk;
        // upper triangle computed once, mirrored: X~ exactly symmetric
#pragma unroll
        for (int i = 0; i < PX; ++i)
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if (i <= j && j < p) {
                    R acc = X[i * p + j];
#pragma unroll
                    for (int q = 0; q < MX; ++q)
                        if (q < m) acc -= M[i * m + q] * W[q][j];
                    row[i * p + j] = acc;
                    row[j * p + i] = acc;
                }
        stage_flush(stage, LDS, p * p, a.Xt, a.oX, k0, nvalid, first);
    }
}

// The vectors of the transform where its matrices do not vary with k (U, M,
// H, F, L, X time-invariant) but r_k, s_k or c_k do: W, W H, F~ and X~ come
// from the pre-transform of step 0 alone, and one thread per step forms
// g_k = W r_k + s_k and c~_k = c_k + L g_k.
template <typename R, int MX>
__global__ void __launch_bounds__(kPreThreads) k_cross_vec(CrossPre<R> a, long long T) {
    const long long k = (long long)blockIdx.x * kPreThreads + threadIdx.x;
    if (k >= T) return;
    const int n = a.n, m = a.m, p = a.p;
    const R* r = a.r ? a.r + a.sr * k : nullptr;
    const R* s = a.s ? a.s + a.ss * k : nullptr;
    const R* c = a.c ? a.c + a.sc * k : nullptr;
    const R* L = a.L + a.sL * k;
    R g[MX];
#pragma unroll
    for (int i = 0; i < MX; ++i) {
        if (i >= m) continue;
        R acc = s ? s[i] : R(0);
        if (r)
            for (int j = 0; j < p; ++j) acc += a.Wm[i * p + j] * r[j];
        g[i] = acc;
        if (a.og) a.g[a.og * k + i] = acc;
    }
    if (a.oc)
        for (int l = 0; l < n; ++l) {
            R acc = c ? c[l] : R(0);
#pragma unroll
            for (int i = 0; i < MX; ++i)
                if (i < m) acc += L[l * m + i] * g[i];
            a.ct[a.oc * k + l] = acc;
        }
}

// Small sizes: a block per 256 steps.  K += W H as one contiguous run of the
// block's steps (coalesced), then one thread per step for u, whose W H rows
// the first phase has just brought into L1.
constexpr int kPostThreads = 256;

template <typename R, int NX, int MX>
__global__ void __launch_bounds__(kPostThreads)
    k_cross_post_small(long long T, R* K, R* u, const R* x, const R* WH, long long oW, const R* g,
                       long long og, const int* pre_status, int* status) {
    constexpr int n = NX, m = MX, MN = MX * NX;
    const long long k0 = (long long)blockIdx.x * kPostThreads;
    const int nb = (int)(T - k0 < kPostThreads ? T - k0 : kPostThreads);
    for (int i = threadIdx.x; i < nb * MN; i += kPostThreads) {
        const long long k = k0 + i / MN;
        K[k0 * MN + i] += WH[oW * k + i % MN];
    }
    if ((int)threadIdx.x < nb) {
        const long long k = k0 + threadIdx.x;
        const R* wh = WH + oW * k;
        R xk[NX];
#pragma unroll
        for (int l = 0; l < n; ++l) xk[l] = x[k * n + l];
#pragma unroll
        for (int i = 0; i < m; ++i) {
            R acc = u[k * m + i] + g[og * k + i];
#pragma unroll
            for (int l = 0; l < n; ++l) acc -= wh[i * n + l] * xk[l];
            u[k * m + i] = acc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *pre_status != 0)
        *status = *pre_status;  // the root cause wins
}

// K_k += (W H)_k, u_k += g_k - (W H)_k x*_k; then the transform status is
// written into the solve's status word (a failed transform is the root cause).
template <typename R>
__global__ void k_cross_post(long long T, int n, int m, R* K, R* u, const R* x, const R* WH,
                             long long oW, const R* g, long long og, const int* pre_status,
                             int* status) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long mn = (long long)m * n;
    for (long long e = tid; e < T * mn; e += nth) {
        const long long k = e / mn;
        K[e] += WH[oW * k + (e - k * mn)];
    }
    for (long long q = tid; q < T * m; q += nth) {
        const long long k = q / m;
        const int i = (int)(q - k * m);
        const R* wh = WH + oW * k + (long long)i * n;
        const R* xk = x + k * n;
        R acc = u[q] + g[og * k + i];
        for (int l = 0; l < n; ++l) acc -= wh[l] * xk[l];
        u[q] = acc;
    }
    if (tid == 0 && *pre_status != 0) *status = *pre_status;  // the root cause wins
}

bool tv(const lqt_in& in) { return in.ptr && in.step_stride != 0; }

// Workspace layout and the transformed problem.
struct CrossPlan {
    lqt_problem P2;  // pointers into the workspace are offsets from `base`
    size_t solver, pre_status, Ft, ct, Xt, WH, g, Wm, total;
    bool split;  // matrices from step 0 alone, vectors by k_cross_vec
    long long oF, oc, oX, oW, og;
    bool hasF, hasX;
    long long rows;
};

lqt_status validate_cross(const lqt_problem* P, const lqt_cross* X) {
    if (!P) return LQT_EINVAL;
    if (!X) return LQT_OK;
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    const struct {
        const lqt_in* in;
        int64_t size;
    } ins[] = {{&X->M, (int64_t)P->p * P->m}, {&X->s, P->m}};
    for (const auto& i : ins) {
        if (!i.in->ptr) continue;
        if (reinterpret_cast<uintptr_t>(i.in->ptr) % es) return LQT_EINVAL;
        if (i.in->step_stride < 0 || (i.in->step_stride != 0 && i.in->step_stride < i.size))
            return LQT_EINVAL;
    }
    return LQT_OK;
}

// Plans the transformed problem P2 with its workspace pointers at `base`.
lqt_status plan_cross(const lqt_problem* P, const lqt_cross* X, const lqt_options* o,
                      char* base, CrossPlan* cp) {
    lqt_status st = validate_cross(P, X);
    if (st != LQT_OK) return st;
    const bool hasM = X && X->M.ptr && P->p > 0;
    const bool hasS = X && X->s.ptr;
    const int n = P->n, m = P->m, p = P->p;
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    const long long T = P->T;
    const lqt_in M = hasM ? X->M : lqt_in{nullptr, 0};
    const lqt_in S = hasS ? X->s : lqt_in{nullptr, 0};
    // time variation of each transformed quantity
    const bool tvW = tv(P->U) || tv(M);
    const bool tvWH = hasM && (tvW || tv(P->H));
    const bool tvg = (hasM && (tvW || tv(P->r))) || tv(S);
    const bool tvF = tvWH || (hasM && (tv(P->F) || tv(P->L)));
    const bool tvc = tvg || tv(P->c) || ((hasM || hasS) && tv(P->L));
    const bool tvX = hasM && (tvW || tv(P->X));
    cp->hasF = hasM;
    cp->hasX = hasM;
    cp->oW = tvWH ? (long long)m * n : 0;
    cp->og = tvg ? m : 0;
    cp->oF = tvF ? (long long)n * n : 0;
    cp->oc = tvc ? n : 0;
    cp->oX = tvX ? (long long)p * p : 0;
    const bool any_tv = tvWH || tvg || tvF || tvc || tvX;
    cp->split = hasM && !tvW && !tvWH && !tvF && !tvX && (tvg || tvc) && m <= kVecMaxM;
    cp->rows = T == 0 ? 0 : (any_tv && !cp->split ? T : 1);
    const long long rW = cp->oW ? T : 1, rg = cp->og ? T : 1, rF = cp->oF ? T : 1,
                    rc = cp->oc ? T : 1, rX = cp->oX ? T : 1;

    lqt_problem& P2 = cp->P2;
    P2 = *P;
    // placeholder addresses for the size query; the layout does not depend on them
    char* b = base ? base : reinterpret_cast<char*>(size_t(1) << 20);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += align_up(bytes);
        return at;
    };
    // offsets after the solver's workspace, filled in below
    const size_t pre_status = take(sizeof(int));
    const size_t Ft = cp->hasF ? take(rF * n * n * es) : 0;
    const size_t ct = take(rc * n * es);
    const size_t Xt = cp->hasX ? take(rX * p * p * es) : 0;
    const size_t WH = take(rW * m * n * es);
    const size_t g = take(rg * m * es);
    const size_t Wm = cp->split ? take((size_t)m * p * es) : 0;
    const size_t tail = off;
    // the solver's workspace comes first (its status word at offset 0); its
    // size depends on the problem's sizes and options only
    auto point = [&](size_t solver) {
        if (cp->hasF) P2.F = lqt_in{b + solver + Ft, cp->oF};
        P2.c = lqt_in{b + solver + ct, cp->oc};
        if (cp->hasX) P2.X = lqt_in{b + solver + Xt, cp->oX};
    };
    point(kAlign);
    const size_t solver = T == 0 ? lqt_workspace_bytes(P, o) : lqt_workspace_bytes(&P2, o);
    if (solver == 0) return LQT_EUNSUPPORTED;  // the caller re-diagnoses through lqt_solve
    cp->solver = align_up(solver);
    point(cp->solver);
    cp->pre_status = cp->solver + pre_status;
    cp->Ft = cp->solver + Ft;
    cp->ct = cp->solver + ct;
    cp->Xt = cp->solver + Xt;
    cp->WH = cp->solver + WH;
    cp->g = cp->solver + g;
    cp->Wm = cp->solver + Wm;
    cp->total = cp->solver + tail;
    if (T == 0) P2 = *P;
    return LQT_OK;
}

// The compiled small (n, m) variants get the register kernels: p <= 2 and
// p <= 8 instantiations.  False: no small kernel for this size.
template <typename R>
bool launch_pre_small(const CrossPre<R>& a, unsigned blocks, cudaStream_t s) {
    bool done = false;
#define LQT_CROSS_PRE_SMALL(RR, N, M)                                                         \
    if constexpr (std::is_same<R, RR>::value) {                                              \
        if (!done && a.n == N && a.m == M) {                                                 \
            if (a.p <= 2)                                                                    \
                k_cross_pre_small<R, N, M, 2><<<blocks, kSmallThreads, 0, s>>>(a);           \
            else                                                                             \
                k_cross_pre_small<R, N, M, 8><<<blocks, kSmallThreads, 0, s>>>(a);           \
            done = true;                                                                     \
        }                                                                                    \
    }
    LQT_VARIANTS(LQT_CROSS_PRE_SMALL)
#undef LQT_CROSS_PRE_SMALL
    return done;
}

template <typename R>
bool launch_post_small(long long T, int n, int m, R* K, R* u, const R* x, const R* WH,
                       long long oW, const R* g, long long og, const int* pre_status,
                       int* status, unsigned blocks, cudaStream_t s) {
    bool done = false;
#define LQT_CROSS_POST_SMALL(RR, N, M)                                                        \
    if constexpr (std::is_same<R, RR>::value) {                                              \
        if (!done && n == N && m == M) {                                                     \
            k_cross_post_small<R, N, M><<<(unsigned)((T + kPostThreads - 1) / kPostThreads), \
                                          kPostThreads, 0, s>>>(T, K, u, x, WH, oW, g, og,   \
                                                                pre_status, status);         \
            done = true;                                                                     \
        }                                                                                    \
    }
    LQT_VARIANTS(LQT_CROSS_POST_SMALL)
#undef LQT_CROSS_POST_SMALL
    return done;
}

template <typename R, int G>
lqt_status launch_pre(const lqt_problem* P, const lqt_cross* X, const CrossPlan& cp, char* base,
                      cudaStream_t s) {
    CrossPre<R> a;
    a.n = P->n;
    a.m = P->m;
    a.p = P->p;
    a.rows = cp.rows;
    a.group_elems = a.m * (a.m | 1) + a.m * (a.p | 1) + a.m * (a.n | 1) + a.m;
    auto in = [](const lqt_in& i, const R** ptr, long long* stride) {
        *ptr = static_cast<const R*>(i.ptr);
        *stride = i.step_stride;
    };
    in(P->F, &a.F, &a.sF);
    in(P->c, &a.c, &a.sc);
    in(P->L, &a.L, &a.sL);
    in(P->U, &a.U, &a.sU);
    in(P->H, &a.H, &a.sH);
    in(P->r, &a.r, &a.sr);
    in(P->X, &a.X, &a.sX);
    const bool hasM = X && X->M.ptr && P->p > 0;
    in(hasM ? X->M : lqt_in{nullptr, 0}, &a.M, &a.sM);
    in(X && X->s.ptr ? X->s : lqt_in{nullptr, 0}, &a.s, &a.ss);
    a.Ft = cp.hasF ? reinterpret_cast<R*>(base + cp.Ft) : nullptr;
    a.ct = reinterpret_cast<R*>(base + cp.ct);
    a.Xt = cp.hasX ? reinterpret_cast<R*>(base + cp.Xt) : nullptr;
    a.WH = reinterpret_cast<R*>(base + cp.WH);
    a.g = reinterpret_cast<R*>(base + cp.g);
    a.oF = cp.oF;
    a.oc = cp.oc;
    a.oX = cp.oX;
    a.oW = cp.oW;
    a.og = cp.og;
    a.Wm = cp.split ? reinterpret_cast<R*>(base + cp.Wm) : nullptr;
    a.status = reinterpret_cast<int*>(base + cp.pre_status);
    auto vectors = [&]() -> lqt_status {
        if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
        if (!cp.split) return LQT_OK;
        const long long vb = (P->T + kPreThreads - 1) / kPreThreads;
        if (vb > INT32_MAX) return LQT_EINVAL;
        if (a.m <= 8)
            k_cross_vec<R, 8><<<(unsigned)vb, kPreThreads, 0, s>>>(a, P->T);
        else
            k_cross_vec<R, kVecMaxM><<<(unsigned)vb, kPreThreads, 0, s>>>(a, P->T);
        return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
    };
    if (a.p <= 8) {
        const long long blocks = (cp.rows + kSmallThreads - 1) / kSmallThreads;
        if (blocks > INT32_MAX) return LQT_EINVAL;
        if (launch_pre_small(a, (unsigned)blocks, s)) return vectors();
    }
    constexpr int groups = kPreThreads / G;
    const size_t smem = (size_t)groups * a.group_elems * sizeof(R);
    if (smem > 227 * 1024) return LQT_EUNSUPPORTED;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_cross_pre<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return LQT_ECUDA;
    const long long blocks = (cp.rows + groups - 1) / groups;
    if (blocks > INT32_MAX) return LQT_EINVAL;
    k_cross_pre<R, G><<<(unsigned)blocks, kPreThreads, smem, s>>>(a);
    return vectors();
}

template <typename R>
lqt_status launch_post(const lqt_problem* P, const lqt_solution* sol, const CrossPlan& cp,
                       char* base, cudaStream_t s) {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LQT_ECUDA;
    const bool small = P->n <= 4 && P->m <= 4;
    const long long work = P->T * (long long)P->m * P->n;
    long long blocks = (work + 255) / 256;
    if (blocks > 16LL * sms) blocks = 16LL * sms;
    if (blocks < 1) blocks = 1;
    if (small &&
        launch_post_small<R>(P->T, P->n, P->m, static_cast<R*>(sol->K), static_cast<R*>(sol->u),
                             static_cast<const R*>(sol->x),
                             reinterpret_cast<const R*>(base + cp.WH), cp.oW,
                             reinterpret_cast<const R*>(base + cp.g), cp.og,
                             reinterpret_cast<const int*>(base + cp.pre_status),
                             reinterpret_cast<int*>(base), (unsigned)blocks, s))
        return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
    k_cross_post<R><<<(unsigned)blocks, 256, 0, s>>>(
        P->T, P->n, P->m, static_cast<R*>(sol->K), static_cast<R*>(sol->u),
        static_cast<const R*>(sol->x), reinterpret_cast<const R*>(base + cp.WH), cp.oW,
        reinterpret_cast<const R*>(base + cp.g), cp.og,
        reinterpret_cast<const int*>(base + cp.pre_status), reinterpret_cast<int*>(base));
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_cross_workspace_bytes(const lqt_problem* prob, const lqt_cross* cross,
                                 const lqt_options* opts) {
    CrossPlan cp;
    if (plan_cross(prob, cross, opts, nullptr, &cp) != LQT_OK) return 0;
    return cp.total;
}

lqt_status lqt_solve_cross(const lqt_problem* prob, const lqt_cross* cross,
                           const lqt_solution* sol, const lqt_options* opts, void* workspace,
                           size_t workspace_bytes, void* stream) {
    if (!prob) return LQT_EINVAL;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign) return LQT_EINVAL;
    char* base = static_cast<char*>(workspace);
    CrossPlan cp;
    lqt_status st = plan_cross(prob, cross, opts, base, &cp);
    if (st == LQT_EUNSUPPORTED) {
        // the size query failed: let lqt_solve name the reason (it launches
        // nothing when its own workspace query fails)
        st = lqt_solve(prob, sol, opts, workspace, 0, stream);
        return st == LQT_OK || st == LQT_ENOMEM ? LQT_EUNSUPPORTED : st;
    }
    if (st != LQT_OK) return st;
    if (workspace_bytes < cp.total) return LQT_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prob->T == 0) return lqt_solve(prob, sol, opts, workspace, cp.solver, stream);
    // one post-transform block per kPostThreads steps
    if ((prob->T + kPostThreads - 1) / kPostThreads > INT32_MAX) return LQT_EINVAL;
    // argument check of the transformed solve before anything is launched:
    // lqt_solve validates everything, then reports LQT_ENOMEM for a zero-byte
    // workspace without launching
    st = lqt_solve(&cp.P2, sol, opts, workspace, 0, stream);
    if (st != LQT_ENOMEM) return st == LQT_OK ? LQT_EINVAL : st;
    if (cudaMemsetAsync(base + cp.pre_status, 0, sizeof(int), s) != cudaSuccess) return LQT_ECUDA;
    const bool wide = prob->n > 4 || prob->m > 4 || prob->p > 8;
    if (prob->dtype == LQT_F64)
        st = wide ? launch_pre<double, 32>(prob, cross, cp, base, s)
                  : launch_pre<double, 4>(prob, cross, cp, base, s);
    else
        st = wide ? launch_pre<float, 32>(prob, cross, cp, base, s)
                  : launch_pre<float, 4>(prob, cross, cp, base, s);
    if (st != LQT_OK) return st;
    if ((st = lqt_solve(&cp.P2, sol, opts, workspace, cp.solver, stream)) != LQT_OK) return st;
    return prob->dtype == LQT_F64 ? launch_post<double>(prob, sol, cp, base, s)
                                  : launch_post<float>(prob, sol, cp, base, s);
}

}  // extern "C"
