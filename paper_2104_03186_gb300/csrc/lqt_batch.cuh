// Batched (ragged) LQT solves: one persistent launch per (n, m) variant.
//
// Each CTA takes problems from a work queue (an atomic ticket) and runs the
// whole temporally parallel solve of one problem on chip: the problem's steps
// are cut into NG chunks, one lane group of N lanes per chunk (lane r owns
// row r; lanes.cuh).  Per problem:
//   1. chunk folds P <- a_k (x) P with the elements of eq. lqt_init and the
//      operator of eq. lqt_comb in its low-rank single-step form (fold_step),
//   2. an up-sweep of the NG chunk totals (Alg. 1) in shared memory,
//   3. the terminal value (Lemma LQT_assoc) and a down-sweep of value
//      carries,
//   4. per chunk the Riccati re-fold from its carry (Sec. II-B) writing S_k,
//      v_k, K_k and the feedforward, and the chunk's closed-loop affine map,
//   5. up- and down-sweeps of the affine maps from x_0 (Lemma lqt_fwd_init),
//   6. per chunk the rollout of x*_k and u*_k (eq. Control_LQT).
// No grid-wide dependency exists, so one launch serves the whole batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lqt_lane_step.cuh"

namespace lqt {

namespace batch {

using namespace lanes;

template <int N, int M, int NG>
struct Layout {
    using SL = StepLayout<N, M>;
    static constexpr int LG = N;
    static constexpr int THREADS = NG * LG;
    // per-group buffer: the step (element-shaped, with L, U and X H), then the
    // operator scratch
    static constexpr int G_STEP = 0;
    static constexpr int G_SCR = SL::SIZE;
    static constexpr int SCR = combine_scratch<N>() > riccati_scratch<N, M>() + M * kd_ld<N>() +
                                                           LAffine<N>::SIZE
                                   ? combine_scratch<N>()
                                   : riccati_scratch<N, M>() + M * kd_ld<N>() + LAffine<N>::SIZE;
    static constexpr int G_SIZE = gstride<N>(G_SCR + SCR);
    // CTA: tree of chunk totals, value carries, affine maps, chunk start states
    static constexpr int TREE = 0;
    static constexpr int CARRY = TREE + NG * LElem<N>::SIZE;
    static constexpr int FTREE = CARRY + NG * LValue<N>::SIZE;
    static constexpr int XS = FTREE + NG * LAffine<N>::SIZE;
    static constexpr int GROUPS = XS + NG * N;
    static constexpr int TICKET = GROUPS + NG * G_SIZE;  // 1 int
    static constexpr int TOTAL = TICKET + 4;
    static size_t bytes() { return (size_t)TOTAL * sizeof(float); }
    static_assert(fold_scratch<N, M>() <= SCR, "fold scratch");
};

template <int N, int M, int NG>
__global__ void __launch_bounds__(NG* N) k_batch(const BatchDesc* __restrict__ items, int count,
                                                 int* ticket, int* status) {
    using Lay = Layout<N, M, NG>;
    using E = LElem<N>;
    using V = LValue<N>;
    using A = LAffine<N>;
    extern __shared__ __align__(16) float sh[];
    float* tree = sh + Lay::TREE;
    float* carry = sh + Lay::CARRY;
    float* ftree = sh + Lay::FTREE;
    float* xs = sh + Lay::XS;
    int* s_ticket = reinterpret_cast<int*>(sh + Lay::TICKET);
    const Group<N> g;
    const int gi = threadIdx.x / N;  // chunk group
    const int r = g.lr;
    float* gs = sh + Lay::GROUPS + gi * Lay::G_SIZE;
    float* scr = gs + Lay::G_SCR;
    bool ok = true;

    for (;;) {
        if (threadIdx.x == 0) *s_ticket = atomicAdd(ticket, 1);
        __syncthreads();
        const int item = *s_ticket;
        __syncthreads();
        if (item >= count) break;
        const BatchDesc D = items[item];
        const long long T = D.T;
        const long long B = T > 0 ? (T + NG - 1) / NG : 1;
        const long long s = gi * B < T ? gi * B : T;
        const long long e = s + B < T ? s + B : T;
        const int live = T > 0 ? (int)((T + B - 1) / B) : 0;
        int Geff = 1;
        while (Geff < live) Geff <<= 1;

        // 1. chunk fold
        float* P = tree + gi * E::SIZE;
        set_neutral<N, N>(P, g);
        for (long long k = e - 1; k >= s; --k) {
            load_step<float, N, M, false>(D, k, gs, scr, g, ok);
            ok &= fold_step<float, N, M>(P, gs + Lay::G_STEP, scr, g);
        }
        __syncthreads();
        // 2. up-sweep (left-anchored)
        for (int h = 1; h < Geff; h <<= 1) {
            const int i = gi * 2 * h;
            if (i < Geff) ok &= combine<N, N>(tree + i * E::SIZE, tree + (i + h) * E::SIZE,
                                              tree + i * E::SIZE, scr, g);
            __syncthreads();
        }
        // 3. terminal value, down-sweep of value carries
        if (gi == 0) {
            float acc[N];
            float t = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] = 0.f;
            for (int a = 0; a < D.pT; ++a) {
                const float h = D.HT[a * N + r];
                for (int b = 0; b < D.pT; ++b) {
                    const float hx = h * D.XT[a * D.pT + b];
#pragma unroll
                    for (int j = 0; j < N; ++j) acc[j] += hx * D.HT[b * N + j];
                    if (D.rT) t += hx * D.rT[b];
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                carry[V::OS + r * V::LD + j] = acc[j];
                D.S[T * N * N + r * N + j] = acc[j];
            }
            carry[V::OV + r] = t;
            D.v[T * N + r] = t;
        }
        __syncthreads();
        for (int h = Geff / 2; h >= 1; h >>= 1) {
            const int i = gi * 2 * h;
            if (i < Geff) {
                float* ci = carry + i * V::SIZE;
                float* ch = carry + (i + h) * V::SIZE;
#pragma unroll
                for (int j = 0; j < N; ++j) ch[V::OS + r * V::LD + j] = ci[V::OS + r * V::LD + j];
                ch[V::OV + r] = ci[V::OV + r];
                g.sync();
                ok &= value_apply<N, N>(tree + (i + h) * E::SIZE, ci, scr, g);
            }
            __syncthreads();
        }
        // 4. Riccati re-fold per chunk with outputs and the chunk affine map
        float* val = carry + gi * V::SIZE;
        float* Phi = ftree + gi * A::SIZE;
#pragma unroll
        for (int j = 0; j < N; ++j) Phi[A::OF + r * A::LD + j] = r == j ? 1.f : 0.f;
        Phi[A::OC + r] = 0.f;
        g.sync();
        float* Kd = scr + riccati_scratch<N, M>();
        float* Ft = Kd + M * kd_ld<N>();
        for (long long k = e - 1; k >= s; --k) {
            load_step<float, N, M, false>(D, k, gs, scr, g, ok);
            ok &= riccati<float, N, M>(val, gs, Kd, Ft, scr, g);
#pragma unroll
            for (int j = 0; j < N; ++j) D.S[k * N * N + r * N + j] = val[V::OS + r * V::LD + j];
            D.v[k * N + r] = val[V::OV + r];
            if (r < M) {
#pragma unroll
                for (int j = 0; j < N; ++j) D.K[k * M * N + r * N + j] = Kd[r * kd_ld<N>() + j];
                D.u[k * M + r] = Kd[r * kd_ld<N>() + N];
            }
            // chunk map after adding step k: Phi <- Phi Ft, gamma <- gamma + Phi ct
            float pn[N];
            float gm = Phi[A::OC + r];
#pragma unroll
            for (int j = 0; j < N; ++j) pn[j] = 0.f;
#pragma unroll
            for (int l = 0; l < N; ++l) {
                const float pl = Phi[A::OF + r * A::LD + l];
#pragma unroll
                for (int j = 0; j < N; ++j) pn[j] += pl * Ft[A::OF + l * A::LD + j];
                gm += pl * Ft[A::OC + l];
            }
            g.sync();
#pragma unroll
            for (int j = 0; j < N; ++j) Phi[A::OF + r * A::LD + j] = pn[j];
            Phi[A::OC + r] = gm;
            g.sync();
        }
        __syncthreads();
        // 5. forward sweeps (right-anchored) from x_0
        for (int h = 1; h < Geff; h <<= 1) {
            const int j = gi * 2 * h + 2 * h - 1;
            if (j < Geff)
                affine_compose<N, N>(ftree + (j - h) * A::SIZE, ftree + j * A::SIZE,
                                     ftree + j * A::SIZE, scr, g);
            __syncthreads();
        }
        if (gi == 0) xs[(Geff - 1) * N + r] = D.x0[r];
        __syncthreads();
        for (int h = Geff / 2; h >= 1; h >>= 1) {
            const int j = gi * 2 * h + 2 * h - 1;
            if (j < Geff) {
                const float xv = xs[j * N + r];
                xs[(j - h) * N + r] = xv;
                g.sync();
                affine_apply<N, N>(ftree + (j - h) * A::SIZE, xs + j * N, g);
            }
            __syncthreads();
        }
        // 6. rollout
        float* xc = xs + gi * N;  // this chunk's state, updated in place
        for (long long k = s; k < e; ++k) {
            const float* F = D.F + k * D.sF;
            const float* Lk = D.L + k * D.sL;
            const float xr_ = xc[r];
            D.x[k * N + r] = xr_;
            g.sync();
            // u = d - K x (lanes a < M), published through the scratch
            if (r < M) {
                float t = D.u[k * M + r];
#pragma unroll
                for (int j = 0; j < N; ++j) t -= D.K[k * M * N + r * N + j] * xc[j];
                scr[r] = t;
                D.u[k * M + r] = t;
            }
            g.sync();
            float t = D.c ? D.c[k * D.sc + r] : 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) t += __ldg(F + r * N + j) * xc[j];
#pragma unroll
            for (int a = 0; a < M; ++a) t += __ldg(Lk + r * M + a) * scr[a];
            g.sync();
            xc[r] = t;
            g.sync();
            if (k == T - 1) D.x[T * N + r] = t;
        }
        if (T == 0 && gi == 0) D.x[r] = D.x0[r];
        __syncthreads();
    }
    if (!ok) atomicCAS(status, 0, 8);
}

}  // namespace batch
}  // namespace lqt
