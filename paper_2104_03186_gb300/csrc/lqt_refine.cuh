// Kernels of the mixed-precision refinement pass (lqt_options.refine).
//
// After a first solve with trajectory x^, the problem is shifted to
// x = x^ + xi (Sec. II-B problem with the same F, L, U, H, X):
//   r'_k = r_k - H_k x^_k,   c'_k = F_k x^_k + c_k - x^_{k+1},
//   r'_T = r_T - H_T x^_T,   x'_0 = 0,
// whose controls are the optimal controls of the original problem and whose
// states give x* = x^ + xi.  The residual terms are small differences of O(1)
// numbers, so they are formed with error-free transformations -- Knuth's
// TwoSum and the FMA form of Dekker's TwoProduct -- accumulated as in the
// compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26(6), 2005), i.e. as if in twice the working precision.
#pragma once

#include <cuda_runtime.h>

namespace lqt {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// s + e = a + b exactly (TwoSum)
template <typename R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
    s = add_rn(a, b);
    const R z = sub_rn(s, a);
    e = add_rn(sub_rn(a, sub_rn(s, z)), sub_rn(b, z));
}

// Running compensated sum: value = s + c with c collecting the exact errors.
template <typename R>
struct Dot2 {
    R s, c;
    __device__ explicit Dot2(R init) : s(init), c(R(0)) {}
    __device__ void add(R a) {
        R t, e;
        two_sum(s, a, t, e);
        s = t;
        c = add_rn(c, e);
    }
    __device__ void add_prod(R a, R b) {
        const R p = mul_rn(a, b);
        const R ep = fma_rn(a, b, -p);  // a*b - p exactly
        R t, e;
        two_sum(s, p, t, e);
        s = t;
        c = add_rn(c, add_rn(e, ep));
    }
    __device__ R value() const { return add_rn(s, c); }
};

// One thread per step k in [0, T]; thread T forms the terminal reference.
// Writes r' (T x p), rT' (pT), c' (T x n) and x'_0 = 0 (n).
template <typename R>
__global__ void k_refine_prep(int n, int p, int pT, long long T, const R* __restrict__ F,
                              long long sF, const R* __restrict__ c, long long sc,
                              const R* __restrict__ H, long long sH, const R* __restrict__ r,
                              long long sr, const R* __restrict__ HT, const R* __restrict__ rT,
                              const R* __restrict__ xh, R* __restrict__ rp, R* __restrict__ rTp,
                              R* __restrict__ cp, R* __restrict__ x0p) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > T) return;
    const R* x = xh + k * n;
    if (k == T) {
        for (int a = 0; a < pT; ++a) {
            Dot2<R> acc(rT ? rT[a] : R(0));
            for (int j = 0; j < n; ++j) acc.add_prod(-HT[a * n + j], x[j]);
            rTp[a] = acc.value();
        }
        for (int i = 0; i < n; ++i) x0p[i] = R(0);
        return;
    }
    const R* Hk = H + k * sH;
    const R* rk = r ? r + k * sr : nullptr;
    for (int a = 0; a < p; ++a) {
        Dot2<R> acc(rk ? rk[a] : R(0));
        for (int j = 0; j < n; ++j) acc.add_prod(-Hk[a * n + j], x[j]);
        rp[k * p + a] = acc.value();
    }
    const R* Fk = F + k * sF;
    const R* ck = c ? c + k * sc : nullptr;
    const R* xn = x + n;
    for (int i = 0; i < n; ++i) {
        Dot2<R> acc(ck ? ck[i] : R(0));
        for (int j = 0; j < n; ++j) acc.add_prod(Fk[i * n + j], x[j]);
        acc.add(-xn[i]);
        cp[k * n + i] = acc.value();
    }
}

// x <- x^ + xi over all (T+1) n entries.
template <typename R>
__global__ void k_refine_finish(long long count, R* __restrict__ x, const R* __restrict__ xi) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = add_rn(x[i], xi[i]);
}

}  // namespace lqt
