// Register-resident small dense algebra for the parallel LQT scans.
//
// Every routine is fully unrolled for a compile-time state size N and control
// size M, so matrices live in registers; operands that already sit in shared
// memory are read from there through SoA "views" (component k of item i at
// base[k * stride + i]) to keep register pressure low in the tree levels.
//
// Element (A, b, C, eta, J): the dual-form conditional value function of
// eq. g_ki (Sec. IV-A).  C and J are symmetric and stored packed (upper
// triangle, row by row).  Value (S, v): V(x) = z + 1/2 x^T S x - v^T x
// (eq. V_k_LQT).  Affine (F, c): x -> F x + c (eq. trajectory_element).
#pragma once

#include <cuda_runtime.h>

namespace lqt {

template <int N>
struct Dims {
    static constexpr int SYM = N * (N + 1) / 2;
    static constexpr int ELEM = N * N + N + SYM + N + SYM;  // A, b, C, eta, J
    static constexpr int VALUE = SYM + N;                    // S, v
    static constexpr int AFFINE = N * N + N;                 // F, c
    // component offsets inside an element
    static constexpr int OA = 0, OB = N * N, OC = N * N + N, OE = N * N + N + SYM,
                         OJ = N * N + N + SYM + N;
};

// packed index of the symmetric entry (i, j), any order
template <int N>
__host__ __device__ constexpr int sym(int i, int j) {
    return i <= j ? i * N - i * (i - 1) / 2 + (j - i) : j * N - j * (j - 1) / 2 + (i - j);
}

template <typename R, int N>
struct Elem {
    R A[N][N];
    R b[N];
    R C[Dims<N>::SYM];
    R eta[N];
    R J[Dims<N>::SYM];
};

template <typename R, int N>
struct Value {
    R S[Dims<N>::SYM];
    R v[N];
};

// One time step of the model, in registers.
template <typename R, int N, int M>
struct Step {
    R F[N][N];
    R c[N];
    R L[N][M];
    R U[M][M];
    R Q[Dims<N>::SYM];  // H^T X H
    R q[N];             // H^T X r
};

// Correctly rounded reciprocal (the same value as R(1) / x, without the
// general division code).
template <typename R>
__device__ __forceinline__ R rcp_(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float rcp_(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double rcp_(double x) { return __drcp_rn(x); }

template <typename R>
__device__ __forceinline__ R abs_(R x) { return fabs(x); }

// ---------------------------------------------------------------------------
// neutral element (I, 0, 0, 0, 0): e (x) a = a (x) e = a
// ---------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void set_neutral(Elem<R, N>& e) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) e.A[i][j] = (i == j) ? R(1) : R(0);
        e.b[i] = R(0);
        e.eta[i] = R(0);
    }
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) {
        e.C[k] = R(0);
        e.J[k] = R(0);
    }
}

// ---------------------------------------------------------------------------
// One Riccati step (Sec. II-B) on a value (S, v) given at step k+1:
//   G  = L^T S L + U = Rc Rc^T (Cholesky, M x M)
//   K  = G^{-1} L^T S F,   d = G^{-1} L^T (v - S c)
//   Ft = F - L K,          ct = c + L d
//   S <- F^T S F - (L^T S F)^T G^{-1} (L^T S F) + Q      (= F^T S Ft + Q)
//   v <- Ft^T (v - S c) + q
// d is the feedforward of the control law: u = -K x + d, i.e. K^v v - K^c c.
// Rc holds the Cholesky factor (lower), Rinv the reciprocals of its diagonal.
// Returns false when G is not numerically positive definite.
// ---------------------------------------------------------------------------
template <typename R, int N, int M>
__device__ __forceinline__ bool riccati_step(const Step<R, N, M>& st, bool has_c,
                                             R (&S)[Dims<N>::SYM], R (&v)[N], R (&K)[M][N],
                                             R (&d)[M], R (&Ft)[N][N], R (&ct)[N],
                                             R (&Rc)[M][M], R (&Rinv)[M]) {
    // SL = S L
    R SL[N][M];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R t = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) t += S[sym<N>(i, j)] * st.L[j][a];
            SL[i][a] = t;
        }
    // G = L^T S L + U (upper half) and its Cholesky factor
    bool ok = true;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        R g = st.U[a][a];
#pragma unroll
        for (int i = 0; i < N; ++i) g += st.L[i][a] * SL[i][a];
#pragma unroll
        for (int k = 0; k < a; ++k) g -= Rc[a][k] * Rc[a][k];
        ok = ok && (g > R(0));
        const R r = sqrt(g);
        Rc[a][a] = r;
        Rinv[a] = rcp_(r);
#pragma unroll
        for (int b = a + 1; b < M; ++b) {
            R t = st.U[a][b];
#pragma unroll
            for (int i = 0; i < N; ++i) t += st.L[i][a] * SL[i][b];
#pragma unroll
            for (int k = 0; k < a; ++k) t -= Rc[b][k] * Rc[a][k];
            Rc[b][a] = t * Rinv[a];
        }
    }
    // SF = S F ; P1 = (S L)^T F = L^T S F
    R SF[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += S[sym<N>(i, k)] * st.F[k][j];
            SF[i][j] = t;
        }
    R W[M][N];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int i = 0; i < N; ++i) t += SL[i][a] * st.F[i][j];
            W[a][j] = t;
        }
    // e = v - S c ; g = L^T e
    R e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) e[i] = v[i];
    if (has_c) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            R t = e[i];
#pragma unroll
            for (int j = 0; j < N; ++j) t -= S[sym<N>(i, j)] * st.c[j];
            e[i] = t;
        }
    }
    R w[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        R t = R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) t += st.L[i][a] * e[i];
        w[a] = t;
    }
    // forward substitution: W <- Rc^{-1} W, w <- Rc^{-1} w
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = W[a][j];
#pragma unroll
            for (int k = 0; k < a; ++k) t -= Rc[a][k] * W[k][j];
            W[a][j] = t * Rinv[a];
        }
        R t = w[a];
#pragma unroll
        for (int k = 0; k < a; ++k) t -= Rc[a][k] * w[k];
        w[a] = t * Rinv[a];
    }
    // back substitution: K = Rc^{-T} W, d = Rc^{-T} w
#pragma unroll
    for (int a = M - 1; a >= 0; --a) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = W[a][j];
#pragma unroll
            for (int k = a + 1; k < M; ++k) t -= Rc[k][a] * K[k][j];
            K[a][j] = t * Rinv[a];
        }
        R t = w[a];
#pragma unroll
        for (int k = a + 1; k < M; ++k) t -= Rc[k][a] * d[k];
        d[a] = t * Rinv[a];
    }
    // closed loop: Ft = F - L K, ct = c + L d
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = st.F[i][j];
#pragma unroll
            for (int a = 0; a < M; ++a) t -= st.L[i][a] * K[a][j];
            Ft[i][j] = t;
        }
        R t = has_c ? st.c[i] : R(0);
#pragma unroll
        for (int a = 0; a < M; ++a) t += st.L[i][a] * d[a];
        ct[i] = t;
    }
    // S <- F^T S F - W^T W + Q (upper half; W = Rc^{-1} L^T S F)
    R Sn[Dims<N>::SYM];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            R t = st.Q[sym<N>(i, j)];
#pragma unroll
            for (int k = 0; k < N; ++k) t += st.F[k][i] * SF[k][j];
#pragma unroll
            for (int a = 0; a < M; ++a) t -= W[a][i] * W[a][j];
            Sn[sym<N>(i, j)] = t;
        }
    // v <- Ft^T e + q
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = st.q[i];
#pragma unroll
        for (int k = 0; k < N; ++k) t += Ft[k][i] * e[k];
        v[i] = t;
    }
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) S[k] = Sn[k];
    return ok;
}

// ---------------------------------------------------------------------------
// P <- a_k (x) P for a single-step element a_k = (F, c, L U^{-1} L^T, q, Q)
// of eq. lqt_init and an accumulated element P (eq. lqt_comb).  With
// C_1 = L U^{-1} L^T the Woodbury identity (the one used in the proof of
// Lemma LQT_assoc) gives (I + C_1 J_P)^{-1} = I - L G^{-1} L^T J_P with
// G = U + L^T J_P L, so the operator becomes a Riccati step on (J_P, eta_P)
// plus
//   A <- A_P Ft,  b <- A_P ct + b_P,  C <- C_P + (A_P L) G^{-1} (A_P L)^T.
// Only an M x M Cholesky is needed.  Returns false when G is not SPD.
// ---------------------------------------------------------------------------
template <typename R, int N, int M>
__device__ __forceinline__ bool fold_step(const Step<R, N, M>& st, bool has_c, Elem<R, N>& P) {
    // Y = A_P L (before A_P changes)
    R Y[N][M];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R t = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) t += P.A[i][j] * st.L[j][a];
            Y[i][a] = t;
        }
    R K[M][N], d[M], Ft[N][N], ct[N], Rc[M][M], Rinv[M];
    const bool ok = riccati_step<R, N, M>(st, has_c, P.J, P.eta, K, d, Ft, ct, Rc, Rinv);
    // Z = Y Rc^{-T}: row i solves Rc z = Y[i]^T ; C += Z Z^T
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R t = Y[i][a];
#pragma unroll
            for (int k = 0; k < a; ++k) t -= Rc[a][k] * Y[i][k];
            Y[i][a] = t * Rinv[a];
        }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            R t = P.C[sym<N>(i, j)];
#pragma unroll
            for (int a = 0; a < M; ++a) t += Y[i][a] * Y[j][a];
            P.C[sym<N>(i, j)] = t;
        }
    // b <- A_P ct + b ; A <- A_P Ft
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = P.b[i];
#pragma unroll
        for (int j = 0; j < N; ++j) t += P.A[i][j] * ct[j];
        P.b[i] = t;
    }
    R An[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += P.A[i][k] * Ft[k][j];
            An[i][j] = t;
        }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) P.A[i][j] = An[i][j];
    return ok;
}

// ---------------------------------------------------------------------------
// SoA views: component k of item i at base[k * stride] (base already offset by i)
// ---------------------------------------------------------------------------
template <typename R, int N>
struct ElemView {
    R* p;
    int s;
    __device__ R& A(int i, int j) const { return p[(Dims<N>::OA + i * N + j) * s]; }
    __device__ R& b(int i) const { return p[(Dims<N>::OB + i) * s]; }
    __device__ R& C(int i, int j) const { return p[(Dims<N>::OC + sym<N>(i, j)) * s]; }
    __device__ R& eta(int i) const { return p[(Dims<N>::OE + i) * s]; }
    __device__ R& J(int i, int j) const { return p[(Dims<N>::OJ + sym<N>(i, j)) * s]; }
};

template <typename R, int N>
struct ValueView {
    R* p;
    int s;
    __device__ R& S(int i, int j) const { return p[sym<N>(i, j) * s]; }
    __device__ R& v(int i) const { return p[(Dims<N>::SYM + i) * s]; }
};

template <typename R, int N>
struct AffineView {
    R* p;
    int s;
    __device__ R& F(int i, int j) const { return p[(i * N + j) * s]; }
    __device__ R& c(int i) const { return p[(N * N + i) * s]; }
};

template <typename R, int N>
__device__ __forceinline__ void store_elem(const Elem<R, N>& e, ElemView<R, N> o) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) o.A(i, j) = e.A[i][j];
        o.b(i) = e.b[i];
        o.eta(i) = e.eta[i];
    }
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) {
        o.p[(Dims<N>::OC + k) * o.s] = e.C[k];
        o.p[(Dims<N>::OJ + k) * o.s] = e.J[k];
    }
}

// Gaussian elimination with partial pivoting on [Mx | B] (N x N, N x NR),
// rows swapped by predicated selects so every index stays compile-time.
// On return B holds Mx^{-1} B.  Returns false for a zero or non-finite pivot.
template <typename R, int N, int NR>
__device__ __forceinline__ bool solve_pivoted(R (&Mx)[N][N], R (&B)[N][NR]) {
    bool ok = true;
    R invd[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int piv = k;
        R best = abs_(Mx[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const R a = abs_(Mx[i][k]);
            if (a > best) { best = a; piv = i; }
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool sw = (piv == i);
#pragma unroll
            for (int j = k; j < N; ++j) {
                const R x = Mx[k][j], y = Mx[i][j];
                Mx[k][j] = sw ? y : x;
                Mx[i][j] = sw ? x : y;
            }
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const R x = B[k][j], y = B[i][j];
                B[k][j] = sw ? y : x;
                B[i][j] = sw ? x : y;
            }
        }
        ok = ok && (best > R(0)) && isfinite(best);
        invd[k] = rcp_(Mx[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const R f = Mx[i][k] * invd[k];
#pragma unroll
            for (int j = k + 1; j < N; ++j) Mx[i][j] -= f * Mx[k][j];
#pragma unroll
            for (int j = 0; j < NR; ++j) B[i][j] -= f * B[k][j];
        }
    }
#pragma unroll
    for (int k = N - 1; k >= 0; --k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            R t = B[k][j];
#pragma unroll
            for (int l = k + 1; l < N; ++l) t -= Mx[k][l] * B[l][j];
            B[k][j] = t * invd[k];
        }
    return ok;
}

// ---------------------------------------------------------------------------
// The operator of eq. lqt_comb on two elements in shared memory:
//   out = e1 (x) e2, e1 covering k -> j (earlier), e2 covering j -> i.
// With M = I + C1 J2 and one pivoted elimination for [A1 | b1 + C1 eta2 | C1]:
//   X1 = M^{-1} A1, x2 = M^{-1}(b1 + C1 eta2), X3 = M^{-1} C1
//   A = A2 X1, b = A2 x2 + b2, C = A2 X3 A2^T + C2,
//   eta = X1^T (eta2 - J2 b1) + eta1,  J = A1^T J2 X1 + J1
// using (I + J2 C1)^{-1} = M^{-T} and M^{-T} J2 = J2 M^{-1} (C, J symmetric).
// `out` may alias e1 (in-place up-sweep); it must not alias e2.
//
// The vector parts are linear in the operands' vectors,
//   b = b2 + G1 b1 + G2 eta2,   eta = eta1 + H1 eta2 + H2 b1,
// with G1 = A2 M^{-1}, G2 = A2 M^{-1} C1, H1 = X1^T, H2 = -(J2 X1)^T.  With REC
// the elimination also carries I (for M^{-1}) and the four maps are written
// to fac (4 N^2 values, row-major G1 | G2 | H1 | H2), so that a problem with
// the same matrices and other vectors can be combined by combine_replay.
// Entry e of the maps is stored at fac[e * fs].
// ---------------------------------------------------------------------------
template <typename R, int N, bool REC = false>
__device__ __forceinline__ bool combine_view(ElemView<R, N> e1, ElemView<R, N> e2,
                                             ElemView<R, N> out, R* fac = nullptr, int fs = 1) {
    constexpr int NI = 2 * N + 1;  // first column of I when recording
    constexpr int NR = NI + (REC ? N : 0);
    R Mx[N][N];
    R B[N][NR];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = (i == j) ? R(1) : R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += e1.C(i, k) * e2.J(k, j);
            Mx[i][j] = t;
            B[i][j] = e1.A(i, j);
            B[i][N + 1 + j] = e1.C(i, j);
            if constexpr (REC) B[i][NI + j] = (i == j) ? R(1) : R(0);
        }
        R t = e1.b(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += e1.C(i, k) * e2.eta(k);
        B[i][N] = t;
    }
    const bool ok = solve_pivoted<R, N, NR>(Mx, B);

    // eta and J first: they still need e1's A, b, eta, J
    R w[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = e2.eta(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t -= e2.J(i, k) * e1.b(k);
        w[i] = t;
    }
    R etan[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = e1.eta(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += B[k][i] * w[k];
        etan[i] = t;
    }
    R JX[N][N];  // J2 X1
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += e2.J(i, k) * B[k][j];
            JX[i][j] = t;
        }
    R Jn[Dims<N>::SYM];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            R t = e1.J(i, j);
#pragma unroll
            for (int k = 0; k < N; ++k) t += e1.A(k, i) * JX[k][j];
            Jn[sym<N>(i, j)] = t;
        }
    // A, b, C from e2 and the solves
    R An[N][N], bn[N], T3[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R a = R(0), c = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                a += e2.A(i, k) * B[k][j];
                c += e2.A(i, k) * B[k][N + 1 + j];
            }
            An[i][j] = a;
            T3[i][j] = c;
        }
        R t = e2.b(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += e2.A(i, k) * B[k][N];
        bn[i] = t;
    }
    R Cn[Dims<N>::SYM];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            R t = e2.C(i, j);
#pragma unroll
            for (int k = 0; k < N; ++k) t += T3[i][k] * e2.A(j, k);
            Cn[sym<N>(i, j)] = t;
        }
    if constexpr (REC) {
        // T3 = A2 M^{-1} C1 is G2; e2 is not aliased by out
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                R g = R(0);
#pragma unroll
                for (int k = 0; k < N; ++k) g += e2.A(i, k) * B[k][NI + j];
                fac[(i * N + j) * fs] = g;
                fac[(N * N + i * N + j) * fs] = T3[i][j];
                fac[(2 * N * N + i * N + j) * fs] = B[j][i];
                fac[(3 * N * N + i * N + j) * fs] = -JX[j][i];
            }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) out.A(i, j) = An[i][j];
        out.b(i) = bn[i];
        out.eta(i) = etan[i];
    }
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) {
        out.p[(Dims<N>::OC + k) * out.s] = Cn[k];
        out.p[(Dims<N>::OJ + k) * out.s] = Jn[k];
    }
    return ok;
}

// The vector parts of e1 (x) e2 from the maps combine_view<REC> recorded for
// operands with the same matrices: out.b, out.eta (out may alias e1).
template <typename R, int N>
__device__ __forceinline__ void combine_replay(const R* fac, int fs, ElemView<R, N> e1,
                                               ElemView<R, N> e2, ElemView<R, N> out) {
    R b1[N], h1[N], b2[N], h2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        b1[i] = e1.b(i);
        h1[i] = e1.eta(i);
        b2[i] = e2.b(i);
        h2[i] = e2.eta(i);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R b = b2[i], h = h1[i];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            b += fac[(i * N + k) * fs] * b1[k] + fac[(N * N + i * N + k) * fs] * h2[k];
            h += fac[(2 * N * N + i * N + k) * fs] * h2[k] +
                 fac[(3 * N * N + i * N + k) * fs] * b1[k];
        }
        out.b(i) = b;
        out.eta(i) = h;
    }
}

// ---------------------------------------------------------------------------
// Value carry through an element: (S, v) <- value part of P (x) (0, 0, 0, v, S)
// (eq. lqt_comb with A2 = b2 = C2 = 0, as in the proof of Lemma LQT_assoc):
//   X1 = (I + C_P S)^{-1} A_P
//   S <- A_P^T S X1 + J_P,   v <- X1^T (v - S b_P) + eta_P
// With REC the maps of the vector part, v <- eta_P + V1 v + V2 b_P with
// V1 = X1^T and V2 = -(S X1)^T, are written to fac (2 N^2 values, V1 | V2)
// for value_replay (entry e at fac[e * fs]).
// ---------------------------------------------------------------------------
template <typename R, int N, bool REC = false>
__device__ __forceinline__ bool value_apply(ElemView<R, N> P, Value<R, N>& val,
                                            R* fac = nullptr, int fs = 1) {
    R Mx[N][N];
    R X[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = (i == j) ? R(1) : R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += P.C(i, k) * val.S[sym<N>(k, j)];
            Mx[i][j] = t;
            X[i][j] = P.A(i, j);
        }
    const bool ok = solve_pivoted<R, N, N>(Mx, X);
    R e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = val.v[i];
#pragma unroll
        for (int k = 0; k < N; ++k) t -= val.S[sym<N>(i, k)] * P.b(k);
        e[i] = t;
    }
    R SX[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += val.S[sym<N>(i, k)] * X[k][j];
            SX[i][j] = t;
        }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = P.eta(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += X[k][i] * e[k];
        val.v[i] = t;
    }
    if constexpr (REC) {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                fac[(i * N + j) * fs] = X[j][i];
                fac[(N * N + i * N + j) * fs] = -SX[j][i];
            }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) {
            R t = P.J(i, j);
#pragma unroll
            for (int k = 0; k < N; ++k) t += P.A(k, i) * SX[k][j];
            val.S[sym<N>(i, j)] = t;
        }
    return ok;
}

// The vector part of value_apply from the maps value_apply<REC> recorded
// for an element and a value with the same matrices: v <- eta_P + V1 v + V2 b_P.
template <typename R, int N>
__device__ __forceinline__ void value_replay(const R* fac, int fs, ElemView<R, N> P,
                                             R (&v)[N]) {
    R vn[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = P.eta(i);
#pragma unroll
        for (int k = 0; k < N; ++k)
            t += fac[(i * N + k) * fs] * v[k] + fac[(N * N + i * N + k) * fs] * P.b(k);
        vn[i] = t;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = vn[i];
}

template <typename R, int N>
__device__ __forceinline__ void load_value(Value<R, N>& val, ValueView<R, N> in) {
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) val.S[k] = in.p[k * in.s];
#pragma unroll
    for (int i = 0; i < N; ++i) val.v[i] = in.v(i);
}

template <typename R, int N>
__device__ __forceinline__ void store_value(const Value<R, N>& val, ValueView<R, N> out) {
#pragma unroll
    for (int k = 0; k < Dims<N>::SYM; ++k) out.p[k * out.s] = val.S[k];
#pragma unroll
    for (int i = 0; i < N; ++i) out.v(i) = val.v[i];
}

// ---------------------------------------------------------------------------
// Affine maps (Lemma LQT_trajectory_combination): f1 then f2 is
// (F2 F1, F2 c1 + c2).  `out` may alias f2 (right-anchored in-place sweep).
// ---------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void affine_compose_view(AffineView<R, N> f1, AffineView<R, N> f2,
                                                    AffineView<R, N> out) {
    R Fn[N][N], cn[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R t = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) t += f2.F(i, k) * f1.F(k, j);
            Fn[i][j] = t;
        }
        R t = f2.c(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += f2.F(i, k) * f1.c(k);
        cn[i] = t;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) out.F(i, j) = Fn[i][j];
        out.c(i) = cn[i];
    }
}

// x <- F x + c
template <typename R, int N>
__device__ __forceinline__ void affine_apply_view(AffineView<R, N> f, R (&x)[N]) {
    R y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R t = f.c(i);
#pragma unroll
        for (int k = 0; k < N; ++k) t += f.F(i, k) * x[k];
        y[i] = t;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = y[i];
}

}  // namespace lqt
