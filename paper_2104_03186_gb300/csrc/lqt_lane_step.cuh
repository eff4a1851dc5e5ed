// Per-step lane-group routines shared by the batched kernel (lqt_batch.cuh)
// and the chunked single-problem pipeline (lqt_chain.cuh), in the arithmetic
// type R:
//   * load_step: the model of step k in shared memory, with the element terms
//     of eq. lqt_init (A = F_k, b = c_k, eta = H^T X r, J = H^T X H and, when
//     asked for, C = L U^{-1} L^T),
//   * riccati:   one step of the Riccati recursion of Sec. II-B with the gains
//     of eq. Control_LQT,
//   * fold_step: P <- a_k (x) P, eq. lqt_comb with a step element as the left
//     operand, in its low-rank form (C_k = L U^{-1} L^T has rank m, so the
//     n x n solve with I + C_k J_P reduces to one m x m solve with
//     G = U + L^T J_P L by the Woodbury identity).
// Lane r of the group (N lanes) owns row r of every N-row matrix.
#pragma once

#include <cuda_runtime.h>

#include "lqt_lanes.cuh"
#include "lqt_mma.cuh"
#include "lqt_tma.cuh"

namespace lqt {

// One problem as the lane kernels see it (device pointers of type R).
template <typename R>
struct DescT {
    int n, m, p, pT;
    long long T;
    const R *F, *c, *L, *U, *H, *r, *X;
    long long sF, sc, sL, sU, sH, sr, sX;
    const R *HT, *rT, *XT, *x0;
    R *S, *v, *K, *x, *u;
    // optional linear state terms replacing H^T X r (the correction problem of
    // the refinement pass): eta_k = eta[k * seta .. + n), eta_T = etaT[0 .. n)
    const R* eta;
    long long seta;
    const R* etaT;
};
using BatchDesc = DescT<float>;

namespace lanes {

// Group buffer of one step's model: an element-shaped block E (A = F_k,
// b = c_k, C, eta, J), then L_k (N x M), U_k (M x M) and the scratch Y = X H
// (p x N), X r.  Row strides are odd (lds).
template <int N, int M>
struct StepLayout {
    static constexpr int PMAX = 2 * N;  // largest p (rows of H) the lane path takes
    static constexpr int LD = lds(N), LM = lds(M);
    static constexpr int E = 0;
    static constexpr int L = LElem<N>::SIZE;
    static constexpr int U = L + N * LM;
    static constexpr int Y = U + M * LM;
    static constexpr int SIZE = Y + PMAX * LD + PMAX;
};

// Scratch of load_step with the C term (M x M copy of U and M x N right sides).
template <int N, int M>
constexpr int load_scratch() {
    return M * lds(M) + M * lds(N);
}

// Step k of D (inputs of type RI) into the step buffer sb (type R).  WITH_C
// also forms C = L U^{-1} L^T (the general combine needs it; fold_step and
// riccati do not); COST = false loads the dynamics only.  With a staging area
// (stage, stage_cap elements) large enough, X_k, H_k and r_k are first copied
// to shared memory by coalesced loads; h_identity (H_k = I, p = N, checked by
// the caller) then skips the products: J = X_k, eta = X_k r_k.
template <typename R, int N, int M, bool WITH_C, typename RI = R, bool COST = true>
__device__ void load_step(const DescT<RI>& D, long long k, R* sb, R* scr, const Group<N>& g,
                          bool& ok, R* stage = nullptr, int stage_cap = 0,
                          bool h_identity = false) {
    using SL = StepLayout<N, M>;
    using E = LElem<N>;
    constexpr int LD = SL::LD, LM = SL::LM;
    R* e = sb + SL::E;
    R* L = sb + SL::L;
    R* U = sb + SL::U;
    R* Y = sb + SL::Y;          // p x N: X H
    R* xr = Y + SL::PMAX * LD;  // p: X r
    const int r = g.lr;
    const int p = D.p;
    const RI* F = D.F + k * D.sF;
    const RI* Lk = D.L + k * D.sL;
    const RI* Uk = D.U + k * D.sU;
    const RI* H = D.H + k * D.sH;
    const RI* X = D.X + k * D.sX;
    const RI* rk = D.r ? D.r + k * D.sr : nullptr;
    const int lp = p | 1;
    // staged X_k, H_k (none when H_k = I) and r_k
    const int hs = h_identity ? 0 : p * LD;
    const bool staged = COST && stage && p * lp + hs + p <= stage_cap;
    if constexpr (sizeof(R) == sizeof(RI)) {
        // every copy of the step in flight at once (cp.async, consecutive lanes
        // on consecutive elements), one wait
#pragma unroll 8
        for (int t = r; t < N * N; t += N) cp_async<sizeof(R)>(e + E::OA + (t / N) * LD + t % N, F + t);
#pragma unroll 4
        for (int t = r; t < N * M; t += N) cp_async<sizeof(R)>(L + (t / M) * LM + t % M, Lk + t);
#pragma unroll 4
        for (int t = r; t < M * M; t += N) cp_async<sizeof(R)>(U + (t / M) * LM + t % M, Uk + t);
        if (D.c) cp_async<sizeof(R)>(e + E::OB + r, D.c + k * D.sc + r);
        else e[E::OB + r] = R(0);
        if (staged) {
            R* Xs = stage;
            R* Hs = Xs + p * lp;
            R* rs = Hs + hs;
            for (int a = 0; a < p; ++a)
                for (int b = r; b < p; b += N) cp_async<sizeof(R)>(Xs + a * lp + b, X + a * p + b);
            if (!h_identity)
                for (int b = 0; b < p; ++b) cp_async<sizeof(R)>(Hs + b * LD + r, H + b * N + r);
            for (int b = r; b < p; b += N) {
                if (rk) cp_async<sizeof(R)>(rs + b, rk + b);
                else rs[b] = R(0);
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
    } else {
#pragma unroll 8
        for (int t = r; t < N * N; t += N) e[E::OA + (t / N) * LD + t % N] = R(__ldg(F + t));
#pragma unroll 4
        for (int t = r; t < N * M; t += N) L[(t / M) * LM + t % M] = R(__ldg(Lk + t));
#pragma unroll 4
        for (int t = r; t < M * M; t += N) U[(t / M) * LM + t % M] = R(__ldg(Uk + t));
        e[E::OB + r] = D.c ? R(__ldg(D.c + k * D.sc + r)) : R(0);
        if (staged) {
            R* Xs = stage;
            R* Hs = Xs + p * lp;
            R* rs = Hs + hs;
            for (int a = 0; a < p; ++a)
                for (int b = r; b < p; b += N) Xs[a * lp + b] = R(__ldg(X + a * p + b));
            if (!h_identity)
                for (int b = 0; b < p; ++b) Hs[b * LD + r] = R(__ldg(H + b * N + r));
            for (int b = r; b < p; b += N) rs[b] = rk ? R(__ldg(rk + b)) : R(0);
        }
    }
    if (!COST) {  // dynamics only (F, c, L, U)
        g.sync();
        return;
    }
    if (staged && h_identity) {
        // H = I (p = N): J = X, eta = X r
        g.sync();
        const R* Xs = stage;
        const R* rs = stage + p * lp;  // no staged H
        R t = R(0);
#pragma unroll 8
        for (int j = 0; j < N; ++j) {
            const R xj = Xs[r * lp + j];
            e[E::OJ + r * LD + j] = xj;
            t += xj * rs[j];
        }
        e[E::OE + r] = D.eta ? R(D.eta[k * D.seta + r]) : t;
    } else if (staged) {
        // X_k, H_k and r_k staged in shared memory
        R* Xs = stage;         // p x p, row stride lp
        R* Hs = Xs + p * lp;   // p x N, row stride LD
        R* rs = Hs + p * LD;   // p
        g.sync();
        // Y = X H and X r, rows spread over the lanes
        for (int a = r; a < p; a += N) {
            R acc[N];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] = R(0);
            R t = R(0);
#pragma unroll 4
            for (int b = 0; b < p; ++b) {
                const R xab = Xs[a * lp + b];
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] += xab * Hs[b * LD + j];
                t += xab * rs[b];
            }
#pragma unroll
            for (int j = 0; j < N; ++j) Y[a * LD + j] = acc[j];
            xr[a] = t;
        }
        g.sync();
        // J = H^T Y, eta = H^T (X r)
        R acc[N];
        R t = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = R(0);
#pragma unroll 4
        for (int a = 0; a < p; ++a) {
            const R h = Hs[a * LD + r];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += h * Y[a * LD + j];
            t += h * xr[a];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) e[E::OJ + r * LD + j] = acc[j];
        e[E::OE + r] = D.eta ? R(D.eta[k * D.seta + r]) : t;
    } else {
        // Y = X H and X r, rows spread over the lanes, operands from global memory
        for (int a = r; a < p; a += N) {
            R acc[N];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] = R(0);
            R t = R(0);
            for (int b = 0; b < p; ++b) {
                const R xab = R(__ldg(X + a * p + b));
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] += xab * R(__ldg(H + b * N + j));
                if (rk) t += xab * R(__ldg(rk + b));
            }
#pragma unroll
            for (int j = 0; j < N; ++j) Y[a * LD + j] = acc[j];
            xr[a] = t;
        }
        g.sync();
        // J = H^T Y, eta = H^T (X r)
        R acc[N];
        R t = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = R(0);
        for (int a = 0; a < p; ++a) {
            const R h = R(__ldg(H + a * N + r));
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += h * Y[a * LD + j];
            t += h * xr[a];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) e[E::OJ + r * LD + j] = acc[j];
        e[E::OE + r] = D.eta ? R(D.eta[k * D.seta + r]) : t;
    }
    if (WITH_C) {
        // C = L U^{-1} L^T: solve U Z = L^T (M x M SPD, N right-hand sides)
        R* Z = scr + M * LM;
        if (r < M) {
#pragma unroll
            for (int j = 0; j < N; ++j) Z[r * LD + j] = L[j * LM + r];
        }
        g.sync();
        ok &= solve_spd<N, M, N>(U, LM, Z, LD, g);
        row_mul_pair<N, M, N>(e + E::OC, LD, L, LM, Z, LD, r);
    }
    g.sync();
}

// Scratch of gains / riccati (elements of R), excluding the caller's Kd and Ft:
// S L, S F, G, v - S c, and for 32-lane groups (the tensor-core form in FP32)
// a block O that stages the new S and v; the lane form symmetrises S in place.
template <int N, int M>
constexpr int riccati_scratch() {
    return N * lds(M) + N * lds(N) + M * lds(M) + N + (N == 32 ? N * lds(N) + N : 0);
}

// Row stride of Kd = [K | d] (M x (N + 1)).
template <int N>
constexpr int kd_ld() {
    return lds(N + 1);
}

// Groups of 32 lanes in FP32 (n = 32) run their dense products on the tensor
// cores (lqt_mma.cuh, 3xTF32 with FP32 accumulation); the solves and the
// vector terms stay on the CUDA cores.
template <typename R, int N>
constexpr bool use_tensor_cores() {
    return N == 32 && sizeof(R) == 4;
}

// riccati (below) for a 32-lane FP32 group: the same formulas and shared-memory
// layout, with S L, S F, U + L^T S L, L^T S F, F - L K, S F - S L K and
// Q + F^T (S Ft) as warp-wide tensor-core products.
template <int N, int M>
__device__ bool riccati_tc(float* val, const float* sb, float* Kd, float* Ft, float* scr,
                           const Group<N>& g) {
    using SLay = StepLayout<N, M>;
    using E = LElem<N>;
    using V = LValue<N>;
    using A = LAffine<N>;
    constexpr int LD = SLay::LD, LM = SLay::LM, LK = kd_ld<N>();
    const float* e = sb + SLay::E;
    const float* F = e + E::OA;
    const float* c = e + E::OB;
    const float* Q = e + E::OJ;
    const float* q = e + E::OE;
    const float* L = sb + SLay::L;
    const float* U = sb + SLay::U;
    const float* S = val + V::OS;
    const float* v = val + V::OV;
    float* SL = scr;            // N x M
    float* SF = SL + N * LM;    // N x N  (later S Ft)
    float* G = SF + N * LD;     // M x M
    float* ev = G + M * LM;     // N
    float* O = ev + N;          // N x N + N
    const int r = g.lr;
    mma_mul<N, N, M, false>(SL, LM, S, LD, L, LM, nullptr, 0, 1.f);
    mma_mul<N, N, N, false>(SF, LD, S, LD, F, LD, nullptr, 0, 1.f);
    {
        float t = v[r];
#pragma unroll
        for (int k = 0; k < N; ++k) t -= S[r * LD + k] * c[k];
        ev[r] = t;
    }
    g.sync();
    // G = U + L^T S L ; [L^T S F | L^T (v - S c)]
    mma_mul<M, N, M, true>(G, LM, L, LM, SL, LM, U, LM, 1.f);
    mma_mul<M, N, N, true>(Kd, LK, SL, LM, F, LD, nullptr, 0, 1.f);
    if (r < M) {
        float w = 0.f;
#pragma unroll 4
        for (int k = 0; k < N; ++k) w += L[k * LM + r] * ev[k];
        Kd[r * LK + N] = w;
    }
    g.sync();
    const bool ok = solve_spd<N, M, N + 1>(G, LM, Kd, LK, g);
    // Ft = F - L K ; ct = c + L d ; S Ft = SF - SL K
    mma_mul<N, M, N, false>(Ft + A::OF, LD, L, LM, Kd, LK, F, LD, -1.f);
    mma_mul<N, M, N, false>(SF, LD, SL, LM, Kd, LK, SF, LD, -1.f);
    {
        float ct = c[r];
#pragma unroll
        for (int a = 0; a < M; ++a) ct += L[r * LM + a] * Kd[a * LK + N];
        Ft[A::OC + r] = ct;
    }
    g.sync();
    // S <- F^T (S Ft) + Q ; v <- Ft^T (v - S c) + q
    mma_mul<N, N, N, true>(O, LD, F, LD, SF, LD, Q, LD, 1.f);
    {
        float t = q[r];
#pragma unroll 4
        for (int k = 0; k < N; ++k) t += Ft[A::OF + k * LD + r] * ev[k];
        O[N * LD + r] = t;
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < N; ++j) val[V::OS + r * LD + j] = 0.5f * (O[r * LD + j] + O[j * LD + r]);
    val[V::OV + r] = O[N * LD + r];
    g.sync();
    return ok;
}

// The gains of one Riccati step (Sec. II-B, eq. Control_LQT) at the value
// (S, v) in val: Kd = [K | d] (M x (N + 1), row stride kd_ld, u = d - K x)
// from G = U + L^T S L,  G [K | d] = [L^T S F | L^T (v - S c)].  Leaves
// SL = S L, SF = S F and ev = v - S c in the scratch for the caller.
template <typename R, int N, int M>
__device__ bool gains(const R* val, const R* sb, R* Kd, R* scr, const Group<N>& g) {
    using SLay = StepLayout<N, M>;
    using E = LElem<N>;
    using V = LValue<N>;
    constexpr int LD = SLay::LD, LM = SLay::LM, LK = kd_ld<N>();
    const R* e = sb + SLay::E;
    const R* F = e + E::OA;
    const R* c = e + E::OB;
    const R* L = sb + SLay::L;
    const R* U = sb + SLay::U;
    const R* S = val + V::OS;
    const R* v = val + V::OV;
    R* SL = scr;             // N x M
    R* SF = SL + N * LM;     // N x N
    R* G = SF + N * LD;      // M x M
    R* ev = G + M * LM;      // N
    const int r = g.lr;
    row_mul_pair<N, N, M>(SL, LM, S, LD, L, LM, r);
    row_mul_pair<N, N, N>(SF, LD, S, LD, F, LD, r);
    {
        R t = v[r];
#pragma unroll
        for (int k = 0; k < N; ++k) t -= S[r * LD + k] * c[k];
        ev[r] = t;
    }
    g.sync();
    if (r < M) {
        // G = U + L^T S L ; [L^T S F | L^T (v - S c)]
        R gg[M], pp[N];
        R w = R(0);
#pragma unroll
        for (int b = 0; b < M; ++b) gg[b] = U[r * LM + b];
#pragma unroll
        for (int j = 0; j < N; ++j) pp[j] = R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R lk = L[k * LM + r];
            const R sk = SL[k * LM + r];
#pragma unroll
            for (int b = 0; b < M; ++b) gg[b] += lk * SL[k * LM + b];
#pragma unroll
            for (int j = 0; j < N; ++j) pp[j] += sk * F[k * LD + j];
            w += lk * ev[k];
        }
#pragma unroll
        for (int b = 0; b < M; ++b) G[r * LM + b] = gg[b];
#pragma unroll
        for (int j = 0; j < N; ++j) Kd[r * LK + j] = pp[j];
        Kd[r * LK + N] = w;
    }
    g.sync();
    return solve_spd<N, M, N + 1>(G, LM, Kd, LK, g);
}

// One Riccati step on the value (S, v) in val (Sec. II-B): writes the gains
// into Kd ([K | d], M x (N + 1), with u = d - K x) and the closed loop into Ft
// (LAffine: F - L K, c + L d), and replaces val by (S_k, v_k).
template <typename R, int N, int M>
__device__ bool riccati(R* val, const R* sb, R* Kd, R* Ft, R* scr, const Group<N>& g) {
    if constexpr (use_tensor_cores<R, N>())
        return riccati_tc<N, M>(val, sb, Kd, Ft, scr, g);
    using SLay = StepLayout<N, M>;
    using E = LElem<N>;
    using V = LValue<N>;
    using A = LAffine<N>;
    constexpr int LD = SLay::LD, LM = SLay::LM, LK = kd_ld<N>();
    const R* e = sb + SLay::E;
    const R* F = e + E::OA;
    const R* c = e + E::OB;
    const R* Q = e + E::OJ;
    const R* q = e + E::OE;
    const R* L = sb + SLay::L;
    R* SL = scr;             // N x M
    R* SF = SL + N * LM;     // N x N  (later S Ft)
    R* G = SF + N * LD;      // M x M
    R* ev = G + M * LM;      // N
    const int r = g.lr;
    const bool ok = gains<R, N, M>(val, sb, Kd, scr, g);
    // Ft = F - L K ; ct = c + L d ; S Ft = SF - SL K
    {
        R ft[N], sft[N];
        R ct = c[r];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            ft[j] = F[r * LD + j];
            sft[j] = SF[r * LD + j];
        }
#pragma unroll 4
        for (int a = 0; a < M; ++a) {
            const R la = L[r * LM + a];
            const R sa = SL[r * LM + a];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                ft[j] -= la * Kd[a * LK + j];
                sft[j] -= sa * Kd[a * LK + j];
            }
            ct += la * Kd[a * LK + N];
        }
        g.sync();
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Ft[A::OF + r * LD + j] = ft[j];
            SF[r * LD + j] = sft[j];
        }
        Ft[A::OC + r] = ct;
    }
    g.sync();
    // S <- F^T (S Ft) + Q, two rows per lane pair over half the columns each
    // (as in row_mul_pair); v <- Ft^T (v - S c) + q, row r per lane
    {
        constexpr int H = N / 2;
        const int r0 = r & ~1, c0 = (r & 1) * H;
        R a0[H], a1[H];
#pragma unroll
        for (int c = 0; c < H; ++c) {
            a0[c] = Q[r0 * LD + c0 + c];
            a1[c] = Q[(r0 + 1) * LD + c0 + c];
        }
        R t = q[r];
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R f0 = F[k * LD + r0], f1 = F[k * LD + r0 + 1];
#pragma unroll
            for (int c = 0; c < H; ++c) {
                const R y = SF[k * LD + c0 + c];
                a0[c] += f0 * y;
                a1[c] += f1 * y;
            }
            t += Ft[A::OF + k * LD + r] * ev[k];
        }
        // nothing in this phase reads val: the new rows go there directly (the
        // odd lane in reverse order, as in row_mul_pair)
        const bool odd = r & 1;
#pragma unroll
        for (int c = 0; c < H; ++c) {
            const int cc = odd ? H - 1 - c : c;
            val[V::OS + r0 * LD + c0 + cc] = odd ? a0[H - 1 - c] : a0[c];
            val[V::OS + (r0 + 1) * LD + c0 + cc] = odd ? a1[H - 1 - c] : a1[c];
        }
        val[V::OV + r] = t;
    }
    g.sync();
    // symmetrise S: row r becomes the mean of row r and column r
    {
        R ss[N];
#pragma unroll
        for (int j = 0; j < N; ++j)
            ss[j] = R(0.5) * (val[V::OS + r * LD + j] + val[V::OS + j * LD + r]);
        g.sync();
#pragma unroll
        for (int j = 0; j < N; ++j) val[V::OS + r * LD + j] = ss[j];
    }
    g.sync();
    return ok;
}

// Scratch of fold_step (elements of R).  The tensor-core form (32-lane FP32
// groups) keeps every product in shared memory; the lane form keeps in
// registers the rows that only their own lane reads again (A2 F, A2 L,
// F^T J2 F), and symmetrises C and J in place, which keeps a lane group's
// shared memory, and so the groups per SM, in check.
template <int N, int M, typename R = float>
constexpr int fold_scratch() {
    if (use_tensor_cores<R, N>())
        return 2 * N * lds(N) /*JF | A2F, later the staged C and J*/ + N * lds(N) /*F^T J2 F*/ +
               2 * N * lds(M) /*P2, JL*/ + M * lds(N) /*Z*/ + 2 * N /*w, A2 c*/ +
               M * lds(M) /*G*/ + M * lds(2 * N + 1) /*rhs*/;
    return N * lds(N) /*JF*/ + N * lds(M) /*JL*/ + M * lds(N) /*Z*/ + 2 * N /*w, A2 c*/ +
           M * lds(M) /*G*/ + M * lds(2 * N + 1) /*rhs*/;
}

// fold_step (below) for a 32-lane FP32 group: the same formulas and scratch
// layout, with J2 F, J2 L, A2 F, A2 L, U + L^T J2 L, L^T J2 F, F^T J2 F,
// A2 F - P2 Zt, C2 + P2 Pt and J1 + F^T J2 F - Z^T Zt as warp-wide
// tensor-core products.
template <int N, int M>
__device__ bool fold_step_tc(float* P, const float* sb, float* scr, const Group<N>& g) {
    using SLay = StepLayout<N, M>;
    using E = LElem<N>;
    constexpr int NR = 2 * N + 1;
    constexpr int LD = SLay::LD, LM = SLay::LM, LR = lds(NR);
    const float* e1 = sb + SLay::E;
    const float* F = e1 + E::OA;
    const float* c = e1 + E::OB;
    const float* L = sb + SLay::L;
    const float* U = sb + SLay::U;
    float* JF = scr;              // N x N
    float* A2F = JF + N * LD;     // N x N
    float* FJF = A2F + N * LD;    // N x N
    float* P2 = FJF + N * LD;     // N x M
    float* JL = P2 + N * LM;      // N x M
    float* Z = JL + N * LM;       // M x N
    float* w = Z + M * LD;        // N
    float* A2c = w + N;           // N
    float* G = A2c + N;           // M x M
    float* rhs = G + M * LM;      // M x NR
    float* O = JF;                // staged C and J (2 N x N), after JF and A2F are consumed
    const int r = g.lr;
    // 1. J2 F, J2 L, A2 F, A2 L; w = eta2 - J2 c, A2 c
    mma_mul<N, N, N, false>(JF, LD, P + E::OJ, LD, F, LD, nullptr, 0, 1.f);
    mma_mul<N, N, M, false>(JL, LM, P + E::OJ, LD, L, LM, nullptr, 0, 1.f);
    mma_mul<N, N, N, false>(A2F, LD, P + E::OA, LD, F, LD, nullptr, 0, 1.f);
    mma_mul<N, N, M, false>(P2, LM, P + E::OA, LD, L, LM, nullptr, 0, 1.f);
    {
        float t = P[E::OE + r], ac = 0.f;
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            t -= P[E::OJ + r * LD + k] * c[k];
            ac += P[E::OA + r * LD + k] * c[k];
        }
        w[r] = t;
        A2c[r] = ac;
    }
    g.sync();
    // P2^T into the right sides
#pragma unroll 4
    for (int a = 0; a < M; ++a) rhs[a * LR + N + 1 + r] = P2[r * LM + a];
    // 2. G = U + L^T JL, Z = L^T JF, L^T w; F^T JF
    mma_mul<M, N, M, true>(G, LM, L, LM, JL, LM, U, LM, 1.f);
    mma_mul<M, N, N, true>(Z, LD, L, LM, JF, LD, nullptr, 0, 1.f);
    mma_mul<N, N, N, true>(FJF, LD, F, LD, JF, LD, nullptr, 0, 1.f);
    if (r < M) {
        float t = 0.f;
#pragma unroll 4
        for (int k = 0; k < N; ++k) t += L[k * LM + r] * w[k];
        rhs[r * LR + N] = t;
    }
    g.sync();
    if (r < M) {
#pragma unroll
        for (int j = 0; j < N; ++j) rhs[r * LR + j] = Z[r * LD + j];
    }
    g.sync();
    // 3. [Zt | om | Pt] = G^{-1} [Z | L^T w | P2^T]
    const bool ok = solve_spd<N, M, NR>(G, LM, rhs, LR, g);
    // 4. A = A2F - P2 Zt, b = A2 c + P2 om + b2 (A2 is not read again)
    mma_mul<N, M, N, false>(P + E::OA, LD, P2, LM, rhs, LR, A2F, LD, -1.f);
    {
        float t = A2c[r] + P[E::OB + r];
#pragma unroll
        for (int a = 0; a < M; ++a) t += P2[r * LM + a] * rhs[a * LR + N];
        P[E::OB + r] = t;
        // J1 + F^T J2 F, in place (row r)
#pragma unroll
        for (int j = 0; j < N; ++j) FJF[r * LD + j] += e1[E::OJ + r * LD + j];
    }
    g.sync();  // A2F and JF consumed: O (over JF, A2F) may be written
    //    C = C2 + P2 Pt and J = J1 + F^T J2 F - Z^T Zt staged in O
    mma_mul<N, M, N, false>(O, LD, P2, LM, rhs + N + 1, LR, P + E::OC, LD, 1.f);
    mma_mul<N, M, N, true>(O + N * LD, LD, Z, LD, rhs, LR, FJF, LD, -1.f);
    //    eta = eta1 + F^T w - Z^T om
    {
        float t = e1[E::OE + r];
#pragma unroll
        for (int a = 0; a < M; ++a) t -= Z[a * LD + r] * rhs[a * LR + N];
#pragma unroll 4
        for (int k = 0; k < N; ++k) t += F[k * LD + r] * w[k];
        P[E::OE + r] = t;
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < N; ++j) {
        P[E::OC + r * LD + j] = 0.5f * (O[r * LD + j] + O[j * LD + r]);
        P[E::OJ + r * LD + j] = 0.5f * (O[N * LD + r * LD + j] + O[N * LD + j * LD + r]);
    }
    g.sync();
    return ok;
}

// P <- a_k (x) P (eq. lqt_comb, a_k = (F, c, L U^{-1} L^T, H^T X r, H^T X H)
// from the step buffer).  With C_k = L W L^T, W = U^{-1}, and
// G = U + L^T J2 L:  (I + C_k J2)^{-1} = I - L G^{-1} L^T J2, and
// (I + C_k J2)^{-1} C_k = L G^{-1} L^T.  Writing Z = L^T J2 F, w = eta2 - J2 c,
// P2 = A2 L and [Zt | om | Pt] = G^{-1} [Z | L^T w | P2^T]:
//   A   = A2 F - P2 Zt              b   = A2 c + P2 om + b2
//   C   = C2 + P2 Pt                J   = J1 + F^T J2 F - Z^T Zt
//   eta = eta1 + F^T w - Z^T om
// Returns false if G is numerically singular.
template <typename R, int N, int M>
__device__ bool fold_step(R* P, const R* sb, R* scr, const Group<N>& g) {
    if constexpr (use_tensor_cores<R, N>()) return fold_step_tc<N, M>(P, sb, scr, g);
    using SLay = StepLayout<N, M>;
    using E = LElem<N>;
    constexpr int NR = 2 * N + 1;
    constexpr int LD = SLay::LD, LM = SLay::LM, LR = lds(NR);
    const R* e1 = sb + SLay::E;
    const R* F = e1 + E::OA;
    const R* c = e1 + E::OB;
    const R* L = sb + SLay::L;
    const R* U = sb + SLay::U;
    R* JF = scr;              // N x N
    R* JL = JF + N * LD;      // N x M
    R* Z = JL + N * LM;       // M x N
    R* w = Z + M * LD;        // N
    R* A2c = w + N;           // N
    R* G = A2c + N;           // M x M
    R* rhs = G + M * LM;      // M x NR
    const int r = g.lr;
    // 1. JF = J2 F and JL = J2 L (lane pairs, into shared memory);
    //    w = eta2 - J2 c (row r of J2)
    row_mul_pair<N, N, N>(JF, LD, P + E::OJ, LD, F, LD, r);
    row_mul_pair<N, N, M>(JL, LM, P + E::OJ, LD, L, LM, r);
    {
        R t = P[E::OE + r];
#pragma unroll 4
        for (int k = 0; k < N; ++k) t -= P[E::OJ + r * LD + k] * c[k];
        w[r] = t;
    }
    //    row r of A2 F and P2 = A2 L kept in registers (P2 also into the right
    //    sides, transposed), A2 c
    R af[N], pl[M];
    {
        R t = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) af[j] = R(0);
#pragma unroll
        for (int a = 0; a < M; ++a) pl[a] = R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R ak = P[E::OA + r * LD + k];
#pragma unroll
            for (int j = 0; j < N; ++j) af[j] += ak * F[k * LD + j];
#pragma unroll
            for (int a = 0; a < M; ++a) pl[a] += ak * L[k * LM + a];
            t += ak * c[k];
        }
#pragma unroll 4
        for (int a = 0; a < M; ++a) rhs[a * LR + N + 1 + r] = pl[a];
        A2c[r] = t;
    }
    g.sync();
    // 2. G = U + L^T JL, Z = L^T JF, L^T w (lanes a < M); row r of F^T JF in
    //    registers (all lanes)
    if (r < M) {
        R gg[M], zz[N];
        R t = R(0);
#pragma unroll
        for (int b = 0; b < M; ++b) gg[b] = U[r * LM + b];
#pragma unroll
        for (int j = 0; j < N; ++j) zz[j] = R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R lk = L[k * LM + r];
#pragma unroll
            for (int b = 0; b < M; ++b) gg[b] += lk * JL[k * LM + b];
#pragma unroll
            for (int j = 0; j < N; ++j) zz[j] += lk * JF[k * LD + j];
            t += lk * w[k];
        }
#pragma unroll
        for (int b = 0; b < M; ++b) G[r * LM + b] = gg[b];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Z[r * LD + j] = zz[j];
            rhs[r * LR + j] = zz[j];
        }
        rhs[r * LR + N] = t;
    }
    R fjf[N];
    {
#pragma unroll
        for (int j = 0; j < N; ++j) fjf[j] = R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R fk = F[k * LD + r];
#pragma unroll
            for (int j = 0; j < N; ++j) fjf[j] += fk * JF[k * LD + j];
        }
    }
    g.sync();
    // 3. [Zt | om | Pt] = G^{-1} [Z | L^T w | P2^T]
    const bool ok = solve_spd<N, M, NR>(G, LM, rhs, LR, g);
    // 4. A = A2F - P2 Zt, b = A2 c + P2 om + b2 (in place: row r of A2 is read
    //    by lane r alone)
    {
        R t = A2c[r] + P[E::OB + r];
#pragma unroll 4
        for (int a = 0; a < M; ++a) {
            const R pa = pl[a];
#pragma unroll
            for (int j = 0; j < N; ++j) af[j] -= pa * rhs[a * LR + j];
            t += pa * rhs[a * LR + N];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) P[E::OA + r * LD + j] = af[j];
        P[E::OB + r] = t;
    }
    //    C = C2 + P2 Pt and J = J1 + F^T J2 F - Z^T Zt, row r of each in place
    //    (row r of C2 is read by lane r alone); eta = eta1 + F^T w - Z^T om
    {
        R cc[N], jj[N];
#pragma unroll
        for (int j = 0; j < N; ++j) cc[j] = P[E::OC + r * LD + j];
#pragma unroll 4
        for (int a = 0; a < M; ++a) {
            const R pa = pl[a];
#pragma unroll
            for (int j = 0; j < N; ++j) cc[j] += pa * rhs[a * LR + N + 1 + j];
        }
        R t = e1[E::OE + r];
#pragma unroll
        for (int j = 0; j < N; ++j) jj[j] = e1[E::OJ + r * LD + j] + fjf[j];
#pragma unroll 4
        for (int a = 0; a < M; ++a) {
            const R za = Z[a * LD + r];
#pragma unroll
            for (int j = 0; j < N; ++j) jj[j] -= za * rhs[a * LR + j];
            t -= za * rhs[a * LR + N];
        }
#pragma unroll 4
        for (int k = 0; k < N; ++k) t += F[k * LD + r] * w[k];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            P[E::OC + r * LD + j] = cc[j];
            P[E::OJ + r * LD + j] = jj[j];
        }
        P[E::OE + r] = t;
    }
    g.sync();
    // symmetrise C and J: row r becomes the mean of row r and column r
    {
        R cs[N], js[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            cs[j] = R(0.5) * (P[E::OC + r * LD + j] + P[E::OC + j * LD + r]);
            js[j] = R(0.5) * (P[E::OJ + r * LD + j] + P[E::OJ + j * LD + r]);
        }
        g.sync();
#pragma unroll
        for (int j = 0; j < N; ++j) {
            P[E::OC + r * LD + j] = cs[j];
            P[E::OJ + r * LD + j] = js[j];
        }
    }
    g.sync();
    return ok;
}

}  // namespace lanes
}  // namespace lqt
