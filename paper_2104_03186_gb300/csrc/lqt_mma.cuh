// Warp-level tensor-core products for the 32-lane groups (n = 32, FP32).
//
// A 32-lane group is one warp, so the dense products of a step (32 x 32 x 32
// and 32 x 16 x 32) can run on the tensor cores with mma.sync m16n8k8 TF32
// and FP32 accumulation, on operands that stay in the group's shared-memory
// matrices.  TF32 keeps 10 mantissa bits; each FP32 operand x is split into
// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), and a product takes
// the three terms hi*hi + hi*lo + lo*hi ("3xTF32"): the dropped lo*lo term
// and the rounding of lo are below FP32 rounding of the result, so the
// products keep FP32 accuracy (the solves stay in FP32 on the CUDA cores).
//
// Fragment layout of m16n8k8 (PTX ISA, TF32): with groupID g = lane / 4 and
// t = lane % 4, the A registers hold (g, t), (g + 8, t), (g, t + 4),
// (g + 8, t + 4) of the 16 x 8 tile, the B registers (t, g) and (t + 4, g)
// of the 8 x 8 tile, and the accumulators (g, 2t), (g, 2t + 1), (g + 8, 2t),
// (g + 8, 2t + 1) of the 16 x 8 result.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lqt {
namespace lanes {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo, both TF32
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_m16n8k8_tf32(float (&d)[4], const uint32_t (&a)[4],
                                                  const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// out = init + alpha * op(X) Y over one warp (all 32 lanes call it together):
//   op(X) = X (ROWS x K, row stride ldx) or, with TX, X^T for X stored K x ROWS;
//   Y is K x C (row stride ldy); init (ROWS x C, stride ldi) may be null (0)
//   and may alias out; alpha is +1 or -1.
// ROWS in {16, 32}; K and C multiples of 8.  The inputs must be visible to
// the whole warp on entry; the caller syncs the warp before reading out.
template <int ROWS, int K, int C, bool TX>
__device__ __forceinline__ void mma_mul(float* out, int ldo, const float* X, int ldx,
                                        const float* Y, int ldy, const float* init, int ldi,
                                        float alpha) {
    static_assert(ROWS % 16 == 0 && K % 8 == 0 && C % 8 == 0, "tile sizes");
    constexpr int MT = ROWS / 16, NT = C / 8, KT = K / 8;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int i0 = mt * 16 + g, j0 = nt * 8 + 2 * t;
            if (init) {
                acc[mt][nt][0] = init[i0 * ldi + j0];
                acc[mt][nt][1] = init[i0 * ldi + j0 + 1];
                acc[mt][nt][2] = init[(i0 + 8) * ldi + j0];
                acc[mt][nt][3] = init[(i0 + 8) * ldi + j0 + 1];
            } else {
                acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
            }
        }
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
        uint32_t ah[MT][4], al[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int rr[4] = {mt * 16 + g, mt * 16 + g + 8, mt * 16 + g, mt * 16 + g + 8};
            const int cc[4] = {kt * 8 + t, kt * 8 + t, kt * 8 + t + 4, kt * 8 + t + 4};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float x = TX ? X[cc[q] * ldx + rr[q]] : X[rr[q] * ldx + cc[q]];
                tf32_split(alpha * x, ah[mt][q], al[mt][q]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            uint32_t bh[2], bl[2];
            tf32_split(Y[(kt * 8 + t) * ldy + nt * 8 + g], bh[0], bl[0]);
            tf32_split(Y[(kt * 8 + t + 4) * ldy + nt * 8 + g], bh[1], bl[1]);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                // small terms first, then the leading one
                mma_m16n8k8_tf32(acc[mt][nt], al[mt], bh);
                mma_m16n8k8_tf32(acc[mt][nt], ah[mt], bl);
                mma_m16n8k8_tf32(acc[mt][nt], ah[mt], bh);
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int i0 = mt * 16 + g, j0 = nt * 8 + 2 * t;
            out[i0 * ldo + j0] = acc[mt][nt][0];
            out[i0 * ldo + j0 + 1] = acc[mt][nt][1];
            out[(i0 + 8) * ldo + j0] = acc[mt][nt][2];
            out[(i0 + 8) * ldo + j0 + 1] = acc[mt][nt][3];
        }
}

}  // namespace lanes
}  // namespace lqt
