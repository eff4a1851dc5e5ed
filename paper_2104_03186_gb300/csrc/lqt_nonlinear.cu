// Iterated nonlinear LQT (Sec. IV-D, "Extension to nonlinear control";
// the unicycle of Sec. VI-E).
//
// Each pass linearises the dynamics around the nominal trajectory (x̄, ū) by
// the first-order Taylor series of eq. nonlinear_linarisation, solves the
// resulting LQT problem with lqt_solve (or the sequential recursion), and
// takes its optimal trajectory as the next nominal.
//
// The linearised problem is posed in state deviations from the nominal,
// x = x̄ + dx, with the control kept absolute:
//   dx_{k+1} = F_k dx_k + L_k u_k + (f(x̄_k, ū_k) - L_k ū_k - x̄_{k+1}),
//   stage cost 1/2 (H_k dx_k - (r_k - H_k x̄_k))^T X_k (...) + 1/2 u_k^T U_k u_k,
//   dx_0 = x_0 - x̄_0.
// It has the same minimiser as the affine model F_k x + c_k + L_k u with
// c_k = f(x̄_k, ū_k) - F_k x̄_k - L_k ū_k.  In absolute coordinates the unicycle's
// F_k x̄_k and c_k both grow with the unwrapped heading (hundreds of radians
// after many laps) and cancel; in deviations every offset stays at the size of
// the nominal's dynamics defect and tracking error.
//
// The nominal trajectory is kept in FP64 whatever the problem's dtype: after
// many laps the unwrapped heading is near 10^3 rad, where an FP32 heading is
// only good to 1e-4 rad, and the Jacobians (sin and cos of the heading) and
// the offsets are formed from it.  Each pass's solve runs in the problem's
// dtype on the small deviation data and its correction dx is added to the
// FP64 nominal.
//
// Outputs: S_k, K_k of the last linearisation; v_k in absolute coordinates
// (v = v' + S_k x̄_k for the deviation problem's v'); x*, u* of the last pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lqt.h"

namespace lqt {
namespace {

constexpr size_t kAlignN = 256;
size_t up_n(size_t x) { return (x + kAlignN - 1) / kAlignN * kAlignN; }

template <typename R>
struct NlBufs {
    double *xb, *ub;   // nominal trajectory, FP64: (T+1) x n, T x m
    R *F, *L, *c;      // linearised dynamics: T x n x n, n x m (time-invariant), T x n
    R *r, *rT, *x0;    // shifted references (T x p, pT) and initial deviation (n)
};

// First nominal: x̄_k = x_init_k or x_0, ū_k = u_init_k or 0; and the
// unicycle's constant control Jacobian L = d f / d (a, omega).
template <typename R>
__global__ void k_nl_init(long long T, const R* x_init, const R* u_init, const R* x0, R dt,
                          NlBufs<R> b) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long e = tid; e < (T + 1) * 4; e += nth)
        b.xb[e] = static_cast<double>(x_init ? x_init[e] : x0[e % 4]);
    for (long long e = tid; e < T * 2; e += nth)
        b.ub[e] = u_init ? static_cast<double>(u_init[e]) : 0.0;
    if (tid < 8) {
        // rows (p_x, p_y, theta, s), columns (a, omega)
        const int i = (int)tid / 2, j = (int)tid % 2;
        b.L[tid] = (i == 2 && j == 1) || (i == 3 && j == 0) ? dt : R(0);
    }
}

// Linearisation at the nominal (eq. nonlinear_linarisation) for the unicycle
// f(x, u) = (p_x + s cos(theta) dt, p_y + s sin(theta) dt, theta + omega dt, s + a dt):
// F_k = d f / d x at (x̄_k, ū_k), the offset f(x̄_k, ū_k) - L ū_k - x̄_{k+1}, and
// the shifted references r_k - H_k x̄_k (k = T: the terminal ones and the
// initial deviation).
template <typename R>
__global__ void k_nl_linearise(long long T, int p, int pT, R dt, const R* H, long long sH,
                               const R* r, long long sr, const R* HT, const R* rT, const R* x0,
                               NlBufs<R> b) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > T) return;
    const double* x = b.xb + k * 4;
    if (k == T) {
        for (int i = 0; i < pT; ++i) {
            double acc = rT ? static_cast<double>(rT[i]) : 0.0;
            for (int j = 0; j < 4; ++j) acc -= static_cast<double>(HT[i * 4 + j]) * x[j];
            b.rT[i] = static_cast<R>(acc);
        }
        // initial deviation x_0 - x̄_0 (x points at x̄_T here)
        for (int j = 0; j < 4; ++j) b.x0[j] = static_cast<R>(static_cast<double>(x0[j]) - b.xb[j]);
        return;
    }
    const double* xn = b.xb + (k + 1) * 4;
    const double th = x[2], s = x[3], h = static_cast<double>(dt);
    double sn, cs;
    sincos(th, &sn, &cs);
    R* F = b.F + k * 16;
    F[0] = R(1), F[1] = R(0), F[2] = static_cast<R>(-s * sn * h), F[3] = static_cast<R>(cs * h);
    F[4] = R(0), F[5] = R(1), F[6] = static_cast<R>(s * cs * h), F[7] = static_cast<R>(sn * h);
    F[8] = R(0), F[9] = R(0), F[10] = R(1), F[11] = R(0);
    F[12] = R(0), F[13] = R(0), F[14] = R(0), F[15] = R(1);
    // f(x̄_k, ū_k) - L ū_k - x̄_{k+1}: the control terms of f are L u, so they
    // cancel exactly and ū_k drops out
    R* c = b.c + k * 4;
    c[0] = static_cast<R>((x[0] - xn[0]) + s * cs * h);
    c[1] = static_cast<R>((x[1] - xn[1]) + s * sn * h);
    c[2] = static_cast<R>(x[2] - xn[2]);
    c[3] = static_cast<R>(x[3] - xn[3]);
    const R* Hk = H + sH * k;
    for (int i = 0; i < p; ++i) {
        double acc = r ? static_cast<double>(r[sr * k + i]) : 0.0;
        for (int j = 0; j < 4; ++j) acc -= static_cast<double>(Hk[i * 4 + j]) * x[j];
        b.r[k * p + i] = static_cast<R>(acc);
    }
}

// x̄ += dx, ū = u (the control is absolute); on the last pass also the outputs in absolute
// coordinates: v_k += S_k x̄_k (old nominal), x_k = x̄_k + dx_k.
template <typename R>
__global__ void k_nl_update(long long T, NlBufs<R> b, R* S, R* v, R* x, R* u, int last) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long k = tid; k <= T; k += nth) {
        double* xb = b.xb + k * 4;
        const R* Sk = S + k * 16;
        double xo[4];
        for (int j = 0; j < 4; ++j) xo[j] = xb[j];
        for (int j = 0; j < 4; ++j) {
            const double nx = xo[j] + static_cast<double>(x[k * 4 + j]);
            xb[j] = nx;
            if (last) x[k * 4 + j] = static_cast<R>(nx);
        }
        if (last)
            for (int i = 0; i < 4; ++i) {
                double acc = static_cast<double>(v[k * 4 + i]);
                for (int j = 0; j < 4; ++j) acc += static_cast<double>(Sk[i * 4 + j]) * xo[j];
                v[k * 4 + i] = static_cast<R>(acc);
            }
        if (k < T)
            for (int j = 0; j < 2; ++j) b.ub[k * 2 + j] = static_cast<double>(u[k * 2 + j]);
    }
}

struct NlPlan {
    lqt_problem P2;
    size_t solver, xb, ub, F, L, c, r, rT, x0, total;
};

lqt_status validate_nl(const lqt_problem* P, const lqt_nonlinear* nl) {
    if (!P || !nl) return LQT_EINVAL;
    if (nl->model != LQT_MODEL_UNICYCLE) return LQT_EINVAL;
    if (P->n != 4 || P->m != 2) return LQT_EINVAL;
    if (nl->iterations < 1 || nl->reserved != 0 || !(nl->dt == nl->dt)) return LQT_EINVAL;
    if (P->T < 0 || P->p < 0 || P->pT < 0 || !P->x0) return LQT_EINVAL;
    if (P->p > 0 && P->T > 0 && !P->H.ptr) return LQT_EINVAL;
    if (P->pT > 0 && !P->HT) return LQT_EINVAL;
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    if (P->dtype != LQT_F32 && P->dtype != LQT_F64) return LQT_EINVAL;
    const void* ptrs[] = {nl->x_init, nl->u_init};
    for (const void* q : ptrs)
        if (q && reinterpret_cast<uintptr_t>(q) % es) return LQT_EINVAL;
    return LQT_OK;
}

lqt_status plan_nl(const lqt_problem* P, const lqt_nonlinear* nl, const lqt_options* o,
                   char* base, NlPlan* np) {
    lqt_status st = validate_nl(P, nl);
    if (st != LQT_OK) return st;
    const size_t es = P->dtype == LQT_F64 ? 8 : 4;
    const long long T = P->T;
    const int n = 4, m = 2, p = P->p, pT = P->pT;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up_n(bytes > 0 ? bytes : 1);
        return at;
    };
    const size_t xb = take((T + 1) * n * 8), ub = take(T * m * 8), F = take(T * n * n * es),
                 L = take(n * m * es), c = take(T * n * es), r = take(T * p * es),
                 rT = take(pT * es), x0 = take(n * es);
    const size_t tail = off;
    char* b = base ? base : reinterpret_cast<char*>(size_t(1) << 20);
    auto point = [&](size_t solver) {
        lqt_problem& Q = np->P2;
        Q = *P;
        Q.F = lqt_in{b + solver + F, n * n};
        Q.L = lqt_in{b + solver + L, 0};
        Q.c = lqt_in{b + solver + c, n};
        Q.r = lqt_in{p > 0 ? b + solver + r : nullptr, p};
        Q.rT = pT > 0 ? b + solver + rT : nullptr;
        Q.x0 = b + solver + x0;
    };
    point(kAlignN);
    const size_t solver = lqt_workspace_bytes(&np->P2, o);
    if (solver == 0) return LQT_EUNSUPPORTED;
    np->solver = up_n(solver);
    point(np->solver);
    np->xb = np->solver + xb;
    np->ub = np->solver + ub;
    np->F = np->solver + F;
    np->L = np->solver + L;
    np->c = np->solver + c;
    np->r = np->solver + r;
    np->rT = np->solver + rT;
    np->x0 = np->solver + x0;
    np->total = np->solver + tail;
    return LQT_OK;
}

template <typename R>
lqt_status run_nl(const lqt_problem* P, const lqt_nonlinear* nl, const lqt_solution* sol,
                  const lqt_options* o, const NlPlan& np, char* base, size_t ws_bytes,
                  cudaStream_t s) {
    NlBufs<R> b;
    b.xb = reinterpret_cast<double*>(base + np.xb);
    b.ub = reinterpret_cast<double*>(base + np.ub);
    b.F = reinterpret_cast<R*>(base + np.F);
    b.L = reinterpret_cast<R*>(base + np.L);
    b.c = reinterpret_cast<R*>(base + np.c);
    b.r = reinterpret_cast<R*>(base + np.r);
    b.rT = reinterpret_cast<R*>(base + np.rT);
    b.x0 = reinterpret_cast<R*>(base + np.x0);
    const long long T = P->T;
    const R dt = static_cast<R>(nl->dt);
    const long long rows = T + 1;
    if ((rows + 127) / 128 > INT32_MAX) return LQT_EINVAL;
    const unsigned grid_init = (unsigned)((rows * 4 + 255) / 256 < 4096 ? (rows * 4 + 255) / 256 : 4096);
    k_nl_init<R><<<grid_init, 256, 0, s>>>(T, static_cast<const R*>(nl->x_init),
                                            static_cast<const R*>(nl->u_init),
                                            static_cast<const R*>(P->x0), dt, b);
    if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
    const unsigned grid_lin = (unsigned)((rows + 127) / 128);
    const unsigned grid_upd = (unsigned)((rows + 255) / 256 < 4096 ? (rows + 255) / 256 : 4096);
    for (int it = 0; it < nl->iterations; ++it) {
        k_nl_linearise<R><<<grid_lin, 128, 0, s>>>(
            T, P->p, P->pT, dt, static_cast<const R*>(P->H.ptr), P->H.step_stride,
            static_cast<const R*>(P->r.ptr), P->r.step_stride, static_cast<const R*>(P->HT),
            static_cast<const R*>(P->rT), static_cast<const R*>(P->x0), b);
        if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
        const lqt_status st = nl->sequential
                                  ? lqt_riccati_sequential(&np.P2, sol, o, base, np.solver, s)
                                  : lqt_solve(&np.P2, sol, o, base, np.solver, s);
        if (st != LQT_OK) return st;
        k_nl_update<R><<<grid_upd, 256, 0, s>>>(
            T, b, static_cast<R*>(sol->S), static_cast<R*>(sol->v), static_cast<R*>(sol->x),
            static_cast<R*>(sol->u), it == nl->iterations - 1);
        if (cudaGetLastError() != cudaSuccess) return LQT_ECUDA;
    }
    (void)ws_bytes;
    return LQT_OK;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" {

size_t lqt_nonlinear_workspace_bytes(const lqt_problem* prob, const lqt_nonlinear* nl,
                                     const lqt_options* opts) {
    NlPlan np;
    if (plan_nl(prob, nl, opts, nullptr, &np) != LQT_OK) return 0;
    return np.total;
}

lqt_status lqt_solve_nonlinear(const lqt_problem* prob, const lqt_nonlinear* nl,
                               const lqt_solution* sol, const lqt_options* opts, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlignN) return LQT_EINVAL;
    char* base = static_cast<char*>(workspace);
    NlPlan np;
    lqt_status st = plan_nl(prob, nl, opts, base, &np);
    if (st == LQT_EUNSUPPORTED) {
        // the size query failed: lqt_solve names the reason without launching
        st = lqt_solve(&np.P2, sol, opts, workspace, 0, stream);
        return st == LQT_OK || st == LQT_ENOMEM ? LQT_EUNSUPPORTED : st;
    }
    if (st != LQT_OK) return st;
    if (workspace_bytes < np.total) return LQT_ENOMEM;
    // argument check of the pass's solve before anything is launched
    st = nl->sequential ? lqt_riccati_sequential(&np.P2, sol, opts, workspace, 0, stream)
                        : lqt_solve(&np.P2, sol, opts, workspace, 0, stream);
    if (st != LQT_ENOMEM) return st == LQT_OK ? LQT_EINVAL : st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return prob->dtype == LQT_F64
               ? run_nl<double>(prob, nl, sol, opts, np, base, workspace_bytes, s)
               : run_nl<float>(prob, nl, sol, opts, np, base, workspace_bytes, s);
}

}  // extern "C"
