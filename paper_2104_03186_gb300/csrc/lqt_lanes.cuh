// Lane-group dense algebra for the LQT operators at larger state sizes, in
// the arithmetic type R (float or double).
//
// A group of LG = N lanes (N a power of two, N <= 32) owns one element; lane r
// of the group owns row r of every N-row matrix, and the matrices live in
// shared memory, row-major with an odd row stride (lds: the lanes reading one
// column of their own rows then hit distinct banks).  Products are row
// products: lane r reads its row of the left factor and the whole right
// factor (broadcast reads).  Phases that read what other lanes wrote are
// separated by a group sync.  The formulas are those of lqt_dense.cuh:
// eq. lqt_comb for the operator, the Riccati step of Sec. II-B with the gains
// of eq. Control_LQT, and the affine maps of Sec. IV-C.
#pragma once

#include <cuda_runtime.h>

namespace lqt {
namespace lanes {

template <int LG>
struct Group {
    int lr;         // lane within the group = owned row
    unsigned mask;  // lanes of the group within the warp
    __device__ Group() {
        const int lane = threadIdx.x & 31;
        lr = lane % LG;
        const int g = lane / LG;
        mask = LG == 32 ? 0xffffffffu : (((1u << LG) - 1u) << (g * LG));
    }
    __device__ void sync() const { __syncwarp(mask); }
};

// Row stride of a shared-memory matrix with `cols` columns: the next odd number.
constexpr int lds(int cols) { return cols | 1; }

// Distance, in elements, between the shared-memory blocks of neighbouring
// groups: the block rounded up to 32 elements, plus N when several groups share
// a warp.  The 32 / N groups of a warp then start N banks apart; with the odd
// row strides of lds() the column sweeps of all lanes of the warp fall in
// distinct banks (FP32; for FP64 within each half-warp wavefront), where an
// unpadded block of a multiple of 32 elements put every group's lane r on one
// bank.
template <int N>
constexpr int gstride(int size) {
    return (size + 31) / 32 * 32 + (N < 32 ? N : 0);
}

// IEEE round-to-nearest reciprocal in the arithmetic type
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// out = X Y for rows 0..ROWS of X (ROWS x K) and Y (K x C), with two output
// rows per lane pair: lanes 2i and 2i + 1 both compute rows 2i and 2i + 1,
// lane 2i the first C/2 columns and lane 2i + 1 the rest.  Each step of k
// reads two left entries and C/2 right entries per lane, where a lane that
// owned one whole row would read one and C: the right factor's broadcast
// reads per FMA halve.  Each output element is one accumulator summed over k
// in order.  ROWS and C even; lanes lr < ROWS take part.
template <int ROWS, int K, int C, typename R>
__device__ __forceinline__ void row_mul_pair(R* out, int ldo, const R* X, int ldx, const R* Y,
                                             int ldy, int lr) {
    static_assert(ROWS % 2 == 0 && C % 2 == 0, "pairs of rows, halves of columns");
    constexpr int H = C / 2;
    if (lr >= ROWS) return;
    const int r0 = lr & ~1, c0 = (lr & 1) * H;
    R a0[H], a1[H];
#pragma unroll
    for (int c = 0; c < H; ++c) {
        a0[c] = R(0);
        a1[c] = R(0);
    }
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const R x0 = X[r0 * ldx + k], x1 = X[(r0 + 1) * ldx + k];
#pragma unroll
        for (int c = 0; c < H; ++c) {
            const R y = Y[k * ldy + c0 + c];
            a0[c] += x0 * y;
            a1[c] += x1 * y;
        }
    }
    // the odd lane of a pair stores its half in reverse order: with odd row
    // strides the two halves then fall on banks of opposite parity, so no two
    // lanes of a warp store to one bank
    const bool odd = lr & 1;
#pragma unroll
    for (int c = 0; c < H; ++c) {
        const int cc = odd ? H - 1 - c : c;
        out[r0 * ldo + c0 + cc] = odd ? a0[H - 1 - c] : a0[c];
        out[(r0 + 1) * ldo + c0 + cc] = odd ? a1[H - 1 - c] : a1[c];
    }
}

// out[lr][0..C) = X[0..K)[lr]^T-row, i.e. (X^T Y)[lr], X stored K x ROWS
template <int ROWS, int K, int C, typename R>
__device__ __forceinline__ void row_mul_tn(R* out, int ldo, const R* X, int ldx, const R* Y,
                                           int ldy, int lr) {
    if (lr >= ROWS) return;
    R acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = R(0);
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const R xk = X[k * ldx + lr];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] += xk * Y[k * ldy + c];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) out[lr * ldo + c] = acc[c];
}

// Gauss-Jordan elimination with partial pivoting on [Mx | Bx] (R x R, R x NR),
// rows owned by lanes lr < R.  On return Bx holds Mx^{-1} Bx.  Returns false
// for a zero or non-finite pivot (every lane returns the same value).
template <int LG, int R, int NR, typename T>
__device__ bool solve_gj(T* Mx, int ldm, T* Bx, int ldb, const Group<LG>& g) {
    bool ok = true;
    const int lr = g.lr;
    for (int k = 0; k < R; ++k) {
        // every lane finds the pivot row redundantly
        int piv = k;
        T best = fabs(Mx[k * ldm + k]);
        for (int i = k + 1; i < R; ++i) {
            const T a = fabs(Mx[i * ldm + k]);
            if (a > best) { best = a; piv = i; }
        }
        ok = ok && (best > T(0)) && isfinite(best);
        g.sync();
        if (piv != k) {
            // swap rows k and piv, columns spread over the lanes
            for (int j = lr; j < R + NR; j += LG) {
                T* a = j < R ? &Mx[k * ldm + j] : &Bx[k * ldb + (j - R)];
                T* b = j < R ? &Mx[piv * ldm + j] : &Bx[piv * ldb + (j - R)];
                const T t = *a;
                *a = *b;
                *b = t;
            }
        }
        g.sync();
        const T inv = rcp(Mx[k * ldm + k]);
        T f = T(0);
        if (lr < R && lr != k) f = Mx[lr * ldm + k] * inv;
        g.sync();
        if (lr < R && lr != k) {
#pragma unroll 4
            for (int j = k + 1; j < R; ++j) Mx[lr * ldm + j] -= f * Mx[k * ldm + j];
#pragma unroll 4
            for (int j = 0; j < NR; ++j) Bx[lr * ldb + j] -= f * Bx[k * ldb + j];
        }
        g.sync();
    }
    if (lr < R) {
        const T inv = rcp(Mx[lr * ldm + lr]);
#pragma unroll 4
        for (int j = 0; j < NR; ++j) Bx[lr * ldb + j] *= inv;
    }
    g.sync();
    return ok;
}

// Solves G Z = B for a symmetric positive definite G (R x R, row stride ldg)
// and B (R x NR, row stride ldb) by Gauss-Jordan elimination without
// pivoting (stable for SPD G).  The R + NR columns of [G | B] are spread over
// the group's lanes (column j in lane j % LG, register slot j / LG) and stay
// in registers; the factors of each pivot column are broadcast from its lane
// by warp shuffles, so the elimination needs no group sync.  Z overwrites B.
// Returns false for a non-positive or non-finite pivot.
template <int LG, int R, int NR, typename T>
__device__ bool solve_spd(const T* G, int ldg, T* B, int ldb, const Group<LG>& g) {
    constexpr int COLS = R + NR;
    constexpr int SL = (COLS + LG - 1) / LG;
    const int lane = g.lr;
    T col[SL][R];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int j = s * LG + lane;
#pragma unroll
        for (int i = 0; i < R; ++i)
            col[s][i] = j < R ? G[i * ldg + j] : (j < COLS ? B[i * ldb + (j - R)] : T(0));
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int ks = k / LG, kl = k % LG;
        const T piv = __shfl_sync(g.mask, col[ks][k], kl, LG);
        ok = ok && piv > T(0) && isfinite(piv);
        const T inv = rcp(piv);
        T f[R];
#pragma unroll
        for (int i = 0; i < R; ++i) f[i] = __shfl_sync(g.mask, col[ks][i], kl, LG) * inv;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const T pk = col[s][k];
#pragma unroll
            for (int i = 0; i < R; ++i) col[s][i] = i == k ? pk * inv : col[s][i] - f[i] * pk;
        }
    }
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int j = s * LG + lane;
        if (j >= R && j < COLS) {
#pragma unroll
            for (int i = 0; i < R; ++i) B[i * ldb + (j - R)] = col[s][i];
        }
    }
    g.sync();
    return ok;
}

// Full element in shared memory: A[N][N], b[N], C[N][N], eta[N], J[N][N]
// (matrices with row stride LD).
template <int N>
struct LElem {
    static constexpr int LD = lds(N);
    static constexpr int OA = 0, OB = N * LD, OC = OB + N, OE = OC + N * LD, OJ = OE + N,
                         SIZE = OJ + N * LD;
};

template <int N>
struct LValue {  // S[N][N], v[N]
    static constexpr int LD = lds(N);
    static constexpr int OS = 0, OV = N * LD, SIZE = N * LD + N;
};

template <int N>
struct LAffine {  // F[N][N], c[N]
    static constexpr int LD = lds(N);
    static constexpr int OF = 0, OC = N * LD, SIZE = N * LD + N;
};

// Scratch a group needs for combine (elements of the arithmetic type).
template <int N>
constexpr int combine_scratch() {
    return N * lds(N) /*Mx*/ + N * lds(2 * N + 1) /*Bx*/ + N /*w*/ + N * lds(N) /*JX or T3*/ +
           LElem<N>::SIZE;
}

// Scratch of value_apply.
template <int N>
constexpr int value_scratch() {
    return 4 * N * lds(N) + 2 * N;
}

template <int LG, int N, typename R>
__device__ void set_neutral(R* e, const Group<LG>& g) {
    constexpr int LD = LElem<N>::LD;
    const int r = g.lr;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        e[LElem<N>::OA + r * LD + j] = r == j ? R(1) : R(0);
        e[LElem<N>::OC + r * LD + j] = R(0);
        e[LElem<N>::OJ + r * LD + j] = R(0);
    }
    e[LElem<N>::OB + r] = R(0);
    e[LElem<N>::OE + r] = R(0);
    g.sync();
}

// out = e1 (x) e2 (eq. lqt_comb).  out may alias e1 or e2.
template <int LG, int N, typename R>
__device__ bool combine(const R* e1, const R* e2, R* out, R* scr, const Group<LG>& g) {
    using E = LElem<N>;
    constexpr int LD = E::LD;
    constexpr int NR = 2 * N + 1;
    constexpr int LB = lds(NR);
    R* Mx = scr;
    R* Bx = Mx + N * LD;
    R* w = Bx + N * LB;
    R* T = w + N;
    R* O = T + N * LD;  // result staged here, copied to out at the end
    const int r = g.lr;
    // Mx = I + C1 J2 ; Bx = [A1 | b1 + C1 eta2 | C1]
    {
        R acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = r == j ? R(1) : R(0);
        R be = e1[E::OB + r];
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R ck = e1[E::OC + r * LD + k];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += ck * e2[E::OJ + k * LD + j];
            be += ck * e2[E::OE + k];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Mx[r * LD + j] = acc[j];
            Bx[r * LB + j] = e1[E::OA + r * LD + j];
            Bx[r * LB + N + 1 + j] = e1[E::OC + r * LD + j];
        }
        Bx[r * LB + N] = be;
        // w = eta2 - J2 b1
        R t = e2[E::OE + r];
#pragma unroll
        for (int k = 0; k < N; ++k) t -= e2[E::OJ + r * LD + k] * e1[E::OB + k];
        w[r] = t;
    }
    g.sync();
    const bool ok = solve_gj<LG, N, NR>(Mx, LD, Bx, LB, g);
    // eta = X1^T w + eta1 ; JX = J2 X1 (into T)
    {
        R t = e1[E::OE + r];
#pragma unroll
        for (int k = 0; k < N; ++k) t += Bx[k * LB + r] * w[k];
        O[E::OE + r] = t;
    }
    row_mul_pair<N, N, N>(T, LD, e2 + E::OJ, LD, Bx, LB, r);
    g.sync();
    // J = A1^T JX + J1
    {
        R acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = e1[E::OJ + r * LD + j];
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R a = e1[E::OA + k * LD + r];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += a * T[k * LD + j];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) O[E::OJ + r * LD + j] = acc[j];
    }
    g.sync();
    // A = A2 X1 ; b = A2 x2 + b2 ; T = A2 X3
    {
        R aa[N], tt[N];
        R bb = e2[E::OB + r];
#pragma unroll
        for (int j = 0; j < N; ++j) aa[j] = tt[j] = R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R a2 = e2[E::OA + r * LD + k];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                aa[j] += a2 * Bx[k * LB + j];
                tt[j] += a2 * Bx[k * LB + N + 1 + j];
            }
            bb += a2 * Bx[k * LB + N];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            O[E::OA + r * LD + j] = aa[j];
            T[r * LD + j] = tt[j];
        }
        O[E::OB + r] = bb;
    }
    g.sync();
    // C = T A2^T + C2
    {
        R acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = e2[E::OC + r * LD + j];
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R t = T[r * LD + k];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += t * e2[E::OA + j * LD + k];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) O[E::OC + r * LD + j] = acc[j];
    }
    g.sync();
    // symmetrise C and J while copying out
#pragma unroll
    for (int j = 0; j < N; ++j) {
        out[E::OA + r * LD + j] = O[E::OA + r * LD + j];
        out[E::OC + r * LD + j] = R(0.5) * (O[E::OC + r * LD + j] + O[E::OC + j * LD + r]);
        out[E::OJ + r * LD + j] = R(0.5) * (O[E::OJ + r * LD + j] + O[E::OJ + j * LD + r]);
    }
    out[E::OB + r] = O[E::OB + r];
    out[E::OE + r] = O[E::OE + r];
    g.sync();
    return ok;
}

// value (S, v) <- P (x) (0, 0, 0, v, S)
template <int LG, int N, typename R>
__device__ bool value_apply(const R* P, R* val, R* scr, const Group<LG>& g) {
    using E = LElem<N>;
    using V = LValue<N>;
    constexpr int LD = E::LD;
    R* Mx = scr;
    R* X = Mx + N * LD;
    R* T = X + N * LD;
    R* e = T + N * LD;
    R* O = e + N;
    const int r = g.lr;
    {
        R acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = r == j ? R(1) : R(0);
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R ck = P[E::OC + r * LD + k];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += ck * val[V::OS + k * LD + j];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Mx[r * LD + j] = acc[j];
            X[r * LD + j] = P[E::OA + r * LD + j];
        }
        R t = val[V::OV + r];
#pragma unroll
        for (int k = 0; k < N; ++k) t -= val[V::OS + r * LD + k] * P[E::OB + k];
        e[r] = t;
    }
    g.sync();
    const bool ok = solve_gj<LG, N, N>(Mx, LD, X, LD, g);
    // T = S X1 ; v' = X1^T e + eta
    row_mul_pair<N, N, N>(T, LD, val + V::OS, LD, X, LD, r);
    {
        R t = P[E::OE + r];
#pragma unroll
        for (int k = 0; k < N; ++k) t += X[k * LD + r] * e[k];
        O[V::OV + r] = t;
    }
    g.sync();
    // S' = A^T T + J
    {
        R acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = P[E::OJ + r * LD + j];
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
            const R a = P[E::OA + k * LD + r];
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += a * T[k * LD + j];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) O[V::OS + r * LD + j] = acc[j];
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < N; ++j)
        val[V::OS + r * LD + j] = R(0.5) * (O[V::OS + r * LD + j] + O[V::OS + j * LD + r]);
    val[V::OV + r] = O[V::OV + r];
    g.sync();
    return ok;
}

// f2 after f1: (F2 F1, F2 c1 + c2) into out (may alias f1 or f2)
template <int LG, int N, typename R>
__device__ void affine_compose(const R* f1, const R* f2, R* out, R* scr, const Group<LG>& g) {
    using A = LAffine<N>;
    constexpr int LD = A::LD;
    const int r = g.lr;
    R acc[N];
    R c = f2[A::OC + r];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = R(0);
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
        const R a = f2[A::OF + r * LD + k];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] += a * f1[A::OF + k * LD + j];
        c += a * f1[A::OC + k];
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < N; ++j) out[A::OF + r * LD + j] = acc[j];
    out[A::OC + r] = c;
    g.sync();
    (void)scr;
}

// x <- F x + c for x in shared memory
template <int LG, int N, typename R>
__device__ void affine_apply(const R* f, R* x, const Group<LG>& g) {
    using A = LAffine<N>;
    constexpr int LD = A::LD;
    const int r = g.lr;
    R t = f[A::OC + r];
#pragma unroll
    for (int k = 0; k < N; ++k) t += f[A::OF + r * LD + k] * x[k];
    g.sync();
    x[r] = t;
    g.sync();
}

}  // namespace lanes
}  // namespace lqt
