/*
 * FP64 CPU oracle for the linear quadratic tracker (LQT).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no source,
 * header or helper with the CUDA path.
 *
 * Source: Särkkä & García-Fernández, "Temporal Parallelisation of Dynamic
 * Programming and Linear Quadratic Control" (arXiv 2104.03186).
 *
 *   oracle_riccati      Sec. II-B: the sequential LQT solution.  Eq. LQT_problem
 *                       defines the problem; eqs. v_k_recursion / S_k_recursion
 *                       and the gain formulas give S_k, v_k, K_k, K^v_k, K^c_k;
 *                       eq. Control_LQT with eq. optimal_trajectory gives the
 *                       forward pass u*_k, x*_k.
 *   oracle_element      Lemma LQT_assoc, eq. lqt_init: the element a_k, and the
 *                       terminal element a_T.
 *   oracle_combine      Lemma LQT_combination, eq. lqt_comb: the associative
 *                       operator, with both inverses formed as written.
 *   oracle_affine_combine  Lemma LQT_trajectory_combination.
 *   oracle_method2_state   Lemma LQT_trajectory_method2, eq. lqt_method_2.
 *
 * Readings of the paper that this file takes:
 *   - The terminal eta is H_T^T X_T r_T (Lemma LQT_assoc prints H_T^T r_T);
 *     this matches the terminal cost of eq. LQT_problem and v_T of Sec. II-B.
 *   - v_T uses r_T (Sec. II-B prints r_N).
 *   - The controls of the forward pass are the control law eq. Control_LQT
 *     evaluated on the optimal states.
 *
 * Matrices are row-major.  Per-step inputs are given with a step stride in
 * elements; a stride of 0 means the same matrix at every step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n, m, p, pT;
    long T;
    const double *F, *c, *L, *U; /* k = 0..T-1: n x n, n, n x m, m x m (c may be NULL) */
    const double *H, *r, *X;     /* k = 0..T-1: p x n, p, p x p     (r may be NULL) */
    long sF, sc, sL, sU, sH, sr, sX;
    const double *HT, *rT, *XT;  /* terminal: pT x n, pT, pT x pT   (rT may be NULL) */
    const double *x0;            /* n */
} oracle_problem;

/* ---- plain dense linear algebra (row-major) ---------------------------- */

/* C (r x c) = A (r x k) * B (k x c) */
static void mm(const double *A, const double *B, double *C, int r, int k, int c)
{
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * c + j];
            C[i * c + j] = s;
        }
}

/* C (r x c) = A^T * B with A stored k x r, B k x c */
static void mtm(const double *A, const double *B, double *C, int r, int k, int c)
{
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[l * r + i] * B[l * c + j];
            C[i * c + j] = s;
        }
}

/* B (c x r) = A^T, A stored r x c */
static void tr(const double *A, double *B, int r, int c)
{
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) B[j * r + i] = A[i * c + j];
}

/* y (r) = A (r x k) x (k) ; x may be NULL (treated as zero) */
static void mv(const double *A, const double *x, double *y, int r, int k)
{
    for (int i = 0; i < r; ++i) {
        double s = 0.0;
        if (x)
            for (int l = 0; l < k; ++l) s += A[i * k + l] * x[l];
        y[i] = s;
    }
}

/* Solve A X = B for X (n x q) by Gaussian elimination with partial pivoting.
 * A and B are not modified.  Returns 0, or -1 when a pivot is exactly zero. */
static int solve(const double *A, const double *B, double *Xout, int n, int q)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n * q);
    memcpy(a, A, sizeof(double) * (size_t)n * n);
    memcpy(b, B, sizeof(double) * (size_t)n * q);
    int rc = 0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > fabs(a[piv * n + k])) piv = i;
        if (a[piv * n + k] == 0.0) { rc = -1; break; }
        if (piv != k) {
            for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[piv * n + j]; a[piv * n + j] = t; }
            for (int j = 0; j < q; ++j) { double t = b[k * q + j]; b[k * q + j] = b[piv * q + j]; b[piv * q + j] = t; }
        }
        for (int i = k + 1; i < n; ++i) {
            double f = a[i * n + k] / a[k * n + k];
            for (int j = k; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
            for (int j = 0; j < q; ++j) b[i * q + j] -= f * b[k * q + j];
        }
    }
    if (rc == 0)
        for (int k = n - 1; k >= 0; --k)
            for (int j = 0; j < q; ++j) {
                double s = b[k * q + j];
                for (int l = k + 1; l < n; ++l) s -= a[k * n + l] * Xout[l * q + j];
                Xout[k * q + j] = s / a[k * n + k];
            }
    free(a);
    free(b);
    return rc;
}

/* Ainv = A^{-1} (n x n) */
static int inverse(const double *A, double *Ainv, int n)
{
    double *I = (double *)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    int rc = solve(A, I, Ainv, n, n);
    free(I);
    return rc;
}

static const double *at(const double *base, long stride, long k)
{
    return base ? base + stride * k : NULL;
}

/* Q = H^T X H (n x n) and q = H^T X r (n) for a p x n H. */
static void cost_terms(const double *H, const double *X, const double *r, int p, int n,
                       double *Q, double *q)
{
    double *HtX = (double *)malloc(sizeof(double) * (size_t)n * p);
    mtm(H, X, HtX, n, p, p);            /* H^T X : n x p */
    mm(HtX, H, Q, n, p, n);             /* H^T X H */
    mv(HtX, r, q, n, p);                /* H^T X r */
    free(HtX);
}

/* ---- Sec. II-B: sequential Riccati recursion and forward pass ----------- */

/*
 * S: (T+1) n x n, v: (T+1) n, K: T m x n, Kv: T m x n (may be NULL),
 * Kc: T m x n (may be NULL), x: (T+1) n, u: T m.
 * Returns 0, or -1 when L^T S L + U is singular at some step.
 */
int oracle_riccati(const oracle_problem *P, double *S, double *v, double *K, double *Kv,
                   double *Kc, double *x, double *u)
{
    const int n = P->n, m = P->m, p = P->p;
    const long T = P->T;
    int rc = 0;
    double *Q = malloc(sizeof(double) * n * n), *q = malloc(sizeof(double) * n);
    double *LtS = malloc(sizeof(double) * m * n), *G = malloc(sizeof(double) * m * m);
    double *rhs = malloc(sizeof(double) * m * (3 * n)), *sol = malloc(sizeof(double) * m * (3 * n));
    double *LtSF = malloc(sizeof(double) * m * n), *Lt = malloc(sizeof(double) * m * n);
    double *LK = malloc(sizeof(double) * n * n), *Fcl = malloc(sizeof(double) * n * n);
    double *Sc = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double *SFcl = malloc(sizeof(double) * n * n), *Kx = malloc(sizeof(double) * m);
    double *Kvv = malloc(sizeof(double) * m), *Kcc = malloc(sizeof(double) * m);
    double *Kloc = malloc(sizeof(double) * m * n), *Kvloc = malloc(sizeof(double) * m * n);
    double *Kcloc = malloc(sizeof(double) * m * n), *Lu = malloc(sizeof(double) * n);
    double *Fx = malloc(sizeof(double) * n);

    /* S_T = H_T^T X_T H_T, v_T = H_T^T X_T r_T */
    cost_terms(P->HT, P->XT, P->rT, P->pT, n, S + (size_t)T * n * n, v + (size_t)T * n);

    for (long k = T - 1; k >= 0; --k) {
        const double *F = at(P->F, P->sF, k), *c = at(P->c, P->sc, k);
        const double *L = at(P->L, P->sL, k), *U = at(P->U, P->sU, k);
        const double *Sn = S + (size_t)(k + 1) * n * n, *vn = v + (size_t)(k + 1) * n;

        /* G = L^T S_{k+1} L + U */
        mtm(L, Sn, LtS, m, n, n);
        mm(LtS, L, G, m, n, m);
        for (int i = 0; i < m * m; ++i) G[i] += U[i];

        /* K = G^{-1} L^T S F,  K^v = G^{-1} L^T,  K^c = G^{-1} L^T S */
        mm(LtS, F, LtSF, m, n, n);
        tr(L, Lt, n, m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                rhs[i * 3 * n + j] = LtSF[i * n + j];
                rhs[i * 3 * n + n + j] = Lt[i * n + j];
                rhs[i * 3 * n + 2 * n + j] = LtS[i * n + j];
            }
        if (solve(G, rhs, sol, m, 3 * n)) { rc = -1; goto done; }
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                Kloc[i * n + j] = sol[i * 3 * n + j];
                Kvloc[i * n + j] = sol[i * 3 * n + n + j];
                Kcloc[i * n + j] = sol[i * 3 * n + 2 * n + j];
            }
        memcpy(K + (size_t)k * m * n, Kloc, sizeof(double) * m * n);
        if (Kv) memcpy(Kv + (size_t)k * m * n, Kvloc, sizeof(double) * m * n);
        if (Kc) memcpy(Kc + (size_t)k * m * n, Kcloc, sizeof(double) * m * n);

        /* F - L K */
        mm(L, Kloc, LK, n, m, n);
        for (int i = 0; i < n * n; ++i) Fcl[i] = F[i] - LK[i];

        cost_terms(at(P->H, P->sH, k), at(P->X, P->sX, k), at(P->r, P->sr, k), p, n, Q, q);

        /* v_k = (F - L K)^T (v_{k+1} - S_{k+1} c_k) + H^T X r */
        mv(Sn, c, Sc, n, n);
        for (int i = 0; i < n; ++i) w[i] = vn[i] - Sc[i];
        double *vk = v + (size_t)k * n;
        mtm(Fcl, w, vk, n, n, 1);
        for (int i = 0; i < n; ++i) vk[i] += q[i];

        /* S_k = F^T S_{k+1} (F - L K) + H^T X H */
        double *Sk = S + (size_t)k * n * n;
        mm(Sn, Fcl, SFcl, n, n, n);
        mtm(F, SFcl, Sk, n, n, n);
        for (int i = 0; i < n * n; ++i) Sk[i] += Q[i];
    }

    /* forward pass: x*_0 = x_0, u_k = -K x + K^v v_{k+1} - K^c c, x_{k+1} = F x + c + L u */
    memcpy(x, P->x0, sizeof(double) * n);
    for (long k = 0; k < T; ++k) {
        const double *F = at(P->F, P->sF, k), *c = at(P->c, P->sc, k);
        const double *L = at(P->L, P->sL, k);
        const double *xk = x + (size_t)k * n, *vn = v + (size_t)(k + 1) * n;
        const double *Kk = K + (size_t)k * m * n;
        /* K^v and K^c are recomputed when the caller did not keep them */
        const double *Kvk, *Kck;
        if (Kv && Kc) {
            Kvk = Kv + (size_t)k * m * n;
            Kck = Kc + (size_t)k * m * n;
        } else {
            const double *Sn = S + (size_t)(k + 1) * n * n;
            const double *U = at(P->U, P->sU, k);
            mtm(L, Sn, LtS, m, n, n);
            mm(LtS, L, G, m, n, m);
            for (int i = 0; i < m * m; ++i) G[i] += U[i];
            tr(L, Lt, n, m);
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) {
                    rhs[i * 2 * n + j] = Lt[i * n + j];
                    rhs[i * 2 * n + n + j] = LtS[i * n + j];
                }
            if (solve(G, rhs, sol, m, 2 * n)) { rc = -1; goto done; }
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) {
                    Kvloc[i * n + j] = sol[i * 2 * n + j];
                    Kcloc[i * n + j] = sol[i * 2 * n + n + j];
                }
            Kvk = Kvloc;
            Kck = Kcloc;
        }
        double *uk = u + (size_t)k * m;
        mv(Kk, xk, Kx, m, n);
        mv(Kvk, vn, Kvv, m, n);
        mv(Kck, c, Kcc, m, n);
        for (int i = 0; i < m; ++i) uk[i] = -Kx[i] + Kvv[i] - Kcc[i];
        mv(F, xk, Fx, n, n);
        mv(L, uk, Lu, n, m);
        double *xn = x + (size_t)(k + 1) * n;
        for (int i = 0; i < n; ++i) xn[i] = Fx[i] + (c ? c[i] : 0.0) + Lu[i];
    }

done:
    free(Q); free(q); free(LtS); free(G); free(rhs); free(sol); free(LtSF); free(Lt);
    free(LK); free(Fcl); free(Sc); free(w); free(SFcl); free(Kx); free(Kvv); free(Kcc);
    free(Kloc); free(Kvloc); free(Kcloc); free(Lu); free(Fx);
    return rc;
}

/* ---- Lemma LQT_assoc, eq. lqt_init: elements --------------------------- */

/*
 * Element a_k = (A, b, C, eta, J) for k < T:
 *   A = F_k, b = c_k, C = L_k U_k^{-1} L_k^T, eta = H_k^T X_k r_k, J = H_k^T X_k H_k;
 * terminal element k == T:
 *   A = 0, b = 0, C = 0, eta = H_T^T X_T r_T, J = H_T^T X_T H_T.
 */
int oracle_element(const oracle_problem *P, long k, double *A, double *b, double *C,
                   double *eta, double *J)
{
    const int n = P->n, m = P->m;
    if (k == P->T) {
        memset(A, 0, sizeof(double) * n * n);
        memset(b, 0, sizeof(double) * n);
        memset(C, 0, sizeof(double) * n * n);
        cost_terms(P->HT, P->XT, P->rT, P->pT, n, J, eta);
        return 0;
    }
    const double *F = at(P->F, P->sF, k), *c = at(P->c, P->sc, k);
    const double *L = at(P->L, P->sL, k), *U = at(P->U, P->sU, k);
    memcpy(A, F, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) b[i] = c ? c[i] : 0.0;
    double *Uinv = malloc(sizeof(double) * m * m), *LUi = malloc(sizeof(double) * n * m);
    double *Lt = malloc(sizeof(double) * m * n);
    int rc = inverse(U, Uinv, m);
    if (rc == 0) {
        mm(L, Uinv, LUi, n, m, m);
        tr(L, Lt, n, m);
        mm(LUi, Lt, C, n, m, n);
    }
    free(Uinv); free(LUi); free(Lt);
    cost_terms(at(P->H, P->sH, k), at(P->X, P->sX, k), at(P->r, P->sr, k), P->p, n, J, eta);
    return rc;
}

/* ---- Lemma LQT_combination, eq. lqt_comb: the associative operator ----- */

/*
 * (A, b, C, eta, J) = (A1, b1, C1, eta1, J1) (x) (A2, b2, C2, eta2, J2), where
 * element 1 covers k -> j and element 2 covers j -> i:
 *   A   = A2 (I + C1 J2)^{-1} A1
 *   b   = A2 (I + C1 J2)^{-1} (b1 + C1 eta2) + b2
 *   C   = A2 (I + C1 J2)^{-1} C1 A2^T + C2
 *   eta = A1^T (I + J2 C1)^{-1} (eta2 - J2 b1) + eta1
 *   J   = A1^T (I + J2 C1)^{-1} J2 A1 + J1
 * Both inverses are formed explicitly, as the formula is written.
 * Outputs may not alias inputs.  Returns -1 when either matrix is singular.
 */
int oracle_combine(int n, const double *A1, const double *b1, const double *C1,
                   const double *eta1, const double *J1, const double *A2, const double *b2,
                   const double *C2, const double *eta2, const double *J2, double *A,
                   double *b, double *C, double *eta, double *J)
{
    size_t nn = (size_t)n * n;
    double *M1 = malloc(sizeof(double) * nn), *M2 = malloc(sizeof(double) * nn);
    double *M1i = malloc(sizeof(double) * nn), *M2i = malloc(sizeof(double) * nn);
    double *T1 = malloc(sizeof(double) * nn), *T2 = malloc(sizeof(double) * nn);
    double *T3 = malloc(sizeof(double) * nn), *A2t = malloc(sizeof(double) * nn);
    double *w1 = malloc(sizeof(double) * n), *w2 = malloc(sizeof(double) * n);
    int rc = 0;

    /* M1 = I + C1 J2, M2 = I + J2 C1 */
    mm(C1, J2, M1, n, n, n);
    mm(J2, C1, M2, n, n, n);
    for (int i = 0; i < n; ++i) { M1[i * n + i] += 1.0; M2[i * n + i] += 1.0; }
    if (inverse(M1, M1i, n) || inverse(M2, M2i, n)) { rc = -1; goto done; }

    /* A = A2 M1^{-1} A1 */
    mm(A2, M1i, T1, n, n, n);            /* T1 = A2 M1^{-1} */
    mm(T1, A1, A, n, n, n);

    /* b = A2 M1^{-1} (b1 + C1 eta2) + b2 */
    mv(C1, eta2, w1, n, n);
    for (int i = 0; i < n; ++i) w1[i] += b1[i];
    mv(T1, w1, b, n, n);
    for (int i = 0; i < n; ++i) b[i] += b2[i];

    /* C = A2 M1^{-1} C1 A2^T + C2 */
    mm(T1, C1, T2, n, n, n);
    tr(A2, A2t, n, n);
    mm(T2, A2t, C, n, n, n);
    for (size_t i = 0; i < nn; ++i) C[i] += C2[i];

    /* eta = A1^T M2^{-1} (eta2 - J2 b1) + eta1 */
    mtm(A1, M2i, T3, n, n, n);           /* T3 = A1^T M2^{-1} */
    mv(J2, b1, w2, n, n);
    for (int i = 0; i < n; ++i) w2[i] = eta2[i] - w2[i];
    mv(T3, w2, eta, n, n);
    for (int i = 0; i < n; ++i) eta[i] += eta1[i];

    /* J = A1^T M2^{-1} J2 A1 + J1 */
    mm(T3, J2, T2, n, n, n);
    mm(T2, A1, J, n, n, n);
    for (size_t i = 0; i < nn; ++i) J[i] += J1[i];

done:
    free(M1); free(M2); free(M1i); free(M2i); free(T1); free(T2); free(T3); free(A2t);
    free(w1); free(w2);
    return rc;
}

/* ---- Lemma LQT_trajectory_combination: affine maps --------------------- */

/* (F, c) = (F1, c1) (x) (F2, c2) with map 1 applied first:
 *   F = F2 F1,  c = F2 c1 + c2. */
void oracle_affine_combine(int n, const double *F1, const double *c1, const double *F2,
                           const double *c2, double *F, double *c)
{
    mm(F2, F1, F, n, n, n);
    mv(F2, c1, c, n, n);
    for (int i = 0; i < n; ++i) c[i] += c2[i];
}

/* ---- Lemma LQT_trajectory_method2, eq. lqt_method_2 -------------------- */

/* x*_k = (I + C_{S,k} S_k)^{-1} (A_{S,k} x_S + b_{S,k} + C_{S,k} v_k) */
int oracle_method2_state(int n, const double *A, const double *b, const double *C,
                         const double *S, const double *v, const double *xS, double *x)
{
    size_t nn = (size_t)n * n;
    double *M = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    mm(C, S, M, n, n, n);
    for (int i = 0; i < n; ++i) M[i * n + i] += 1.0;
    mv(A, xS, w, n, n);
    mv(C, v, t, n, n);
    for (int i = 0; i < n; ++i) w[i] += b[i] + t[i];
    int rc = solve(M, w, x, n, 1);
    free(M); free(w); free(t);
    return rc;
}
