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

#include "lqt.h"
#include "lqt_dense.cuh"

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
    int* status;
};

template <typename R>
__device__ __forceinline__ const R* at(const R* a, long long s, long long k) {
    return a ? a + s * k : nullptr;
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
    if (!mats) return;
    R* Fb = a.Fb + jm * N * N;
    R* Lb = a.Lb + jm * N * MB;
    R* cb = a.cb + jm * N;
    R* Ub = a.Ub + jm * MB * MB;
#pragma unroll
    for (int s = 0; s < N; ++s) {
#pragma unroll
        for (int l = 0; l < N; ++l) Fb[s * N + l] = Phi[s][l];
#pragma unroll
        for (int l = 0; l < MB; ++l) Lb[s * MB + l] = Gam[s][l];
        cb[s] = del[s];
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

template <typename R, int N, int M, int B>
__global__ void __launch_bounds__(kCondThreads) k_expand(CondArgs<R> a) {
    constexpr int MB = M * B;
    const long long j = (long long)blockIdx.x * kCondThreads + threadIdx.x;
    if (j >= a.Tb) return;
    const long long k0 = j * B;
    const int b = (int)(a.T - k0 < B ? a.T - k0 : B);
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
    bool ok = true, finite = true;
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
            for (int s = 0; s < N; ++s) a.x[k * N + s] = x[s];
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
        for (int s = 0; s < N; ++s) a.x[a.T * N + s] = a.xb[a.Tb * N + s];
    }
    if (!ok) atomicCAS(a.status, 0, (int)LQT_ENOTSPD);
    if (!finite) atomicCAS(a.status, 0, (int)LQT_ENONFINITE);
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

lqt_status plan_cond(const lqt_problem* P, int B, const lqt_options* o, char* base,
                     CondPlan* cp) {
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
    cp->inv = P->T % B == 0 && fixed(P->F) && fixed(P->L) && fixed(P->U) && fixed(P->c) &&
              fixed(P->H) && fixed(P->X);
    const long long Tm = cp->inv ? 1 : Tb;  // rows of the block matrices
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up_p(bytes > 0 ? bytes : 1);
        return at;
    };
    const size_t Fb = take(Tm * n * n * es), Lb = take(Tm * n * mb * es), cb = take(Tm * n * es),
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
        Q.c = lqt_in{bb + at0 + cb, v * n};
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
    cp->cross_ws = up_p(cross_ws);
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
                      char* base) {
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
    return a;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_condensed_workspace_bytes(const lqt_problem* prob, int32_t B,
                                     const lqt_options* opts) {
    if (prob && B == 1) return lqt_workspace_bytes(prob, opts);
    CondPlan cp;
    if (plan_cond(prob, B, opts, nullptr, &cp) != LQT_OK) return 0;
    return cp.total;
}

lqt_status lqt_solve_condensed(const lqt_problem* prob, int32_t B, const lqt_solution* sol,
                               const lqt_options* opts, void* workspace, size_t workspace_bytes,
                               void* stream) {
    if (!prob || !sol) return LQT_EINVAL;
    if (B == 1) return lqt_solve(prob, sol, opts, workspace, workspace_bytes, stream);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlignP) return LQT_EINVAL;
    char* base = static_cast<char*>(workspace);
    CondPlan cp;
    lqt_status st = plan_cond(prob, B, opts, base, &cp);
    if (st != LQT_OK) return st;
    if (workspace_bytes < cp.total) return LQT_ENOMEM;
    if (prob->T == 0) return LQT_EUNSUPPORTED;  // nothing to condense: use lqt_solve
    const void* outs[] = {sol->S, sol->v, sol->K, sol->x, sol->u};
    for (const void* q : outs)
        if (!q || reinterpret_cast<uintptr_t>(q) % 16) return LQT_EINVAL;
    // argument check of the condensed solve before anything is launched
    st = lqt_solve_cross(&cp.Pc, &cp.cross, &cp.sc, opts, workspace, 0, stream);
    if (st != LQT_ENOMEM) return st == LQT_OK ? LQT_EINVAL : st;
    const CondVariant* var = find_cond(prob->dtype, prob->n, prob->m, B);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long blocks = (cp.Tb + kCondThreads - 1) / kCondThreads;
    if (blocks > INT32_MAX) return LQT_EINVAL;
    if (prob->dtype == LQT_F64) {
        const CondArgs<double> a = cond_args<double>(prob, sol, cp, base);
        var->condense(&a, blocks, s);
    } else {
        const CondArgs<float> a = cond_args<float>(prob, sol, cp, base);
        var->condense(&a, blocks, s);
    }
    if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
    if ((st = lqt_solve_cross(&cp.Pc, &cp.cross, &cp.sc, opts, workspace, cp.cross_ws, stream)) !=
        LQT_OK)
        return st;
    if (prob->dtype == LQT_F64) {
        const CondArgs<double> a = cond_args<double>(prob, sol, cp, base);
        var->expand(&a, blocks, s);
    } else {
        const CondArgs<float> a = cond_args<float>(prob, sol, cp, base);
        var->expand(&a, blocks, s);
    }
    return cudaGetLastError() == cudaSuccess ? LQT_OK : LQT_ECUDA;
}

}  // extern "C"
