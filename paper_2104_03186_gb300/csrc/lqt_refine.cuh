// Compensated arithmetic of the mixed-precision refinement (lqt_options.refine).
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
// Comput. 26(6), 2005), i.e. as if in twice the working precision.  The
// first pass's rollout (k_fwd_down) forms the shifted data; the second pass's
// rollout adds xi to x^.
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

}  // namespace lqt
