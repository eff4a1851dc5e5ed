// Internal interface between the C ABI (lqt_api.cu, lqt_batch.cu, lqt_chain.cu)
// and the compiled variants of the chunked pipeline (lqt_chain.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lqt.h"
#include "lqt_lane_step.cuh"
#include "lqt_launch.cuh"

namespace lqt {

// One problem of a chain call with its chunk geometry.
struct ChainProblem {
    const lqt_problem* problem;
    const lqt_solution* solution;
    int NC;       // chunks (power of two)
    long long B;  // steps per chunk
};

// A call: problems of one variant, by decreasing NC; the workspace starts
// with the status word.
struct ChainCall {
    const ChainProblem* probs;
    int count;
    bool refine, newton, sequential;
    bool method2;  // trajectory by Method 2 (Lemma LQT_trajectory_method2)
    void* ws;
    size_t ws_bytes;
    int* status;  // device status word (nullptr: the first word of ws)
    // warm solve (lqt_warm.cuh): S and K of every problem are given in its
    // solution; only v, the feedforward, x* and u* are computed
    bool warm = false;
    // one persistent cooperative launch instead of one launch per tree level
    // (no refinement, Method 1 only)
    bool persistent = false;
    // ... but only when its grid needs at most half of the CTAs the device
    // holds at once; larger launches take the per-level path
    bool persistent_if_small = false;
};

struct ChainVariant {
    int dtype, n, m;
    int mixed;         // FP32 chunk work with FP64 tree levels
    size_t (*workspace)(const ChainProblem* probs, int count, bool refine, bool newton,
                        bool method2);
    lqt_status (*run)(const ChainCall& call, cudaStream_t s, Prof* prof);
    const void* (*fold_kernel)();
    size_t (*fold_smem)();
    int (*fold_groups)();
};

// Variants compiled in lqt_chain_n4.cu, lqt_chain_n8.cu, lqt_chain_n16.cu and
// lqt_chain_n32.cu.
const ChainVariant* chain_variants_n4(int* count);
const ChainVariant* chain_variants_n8(int* count);
const ChainVariant* chain_variants_n16(int* count);
const ChainVariant* chain_variants_n32(int* count);

template <typename R>
DescT<R> make_desc(const lqt_problem* P, const lqt_solution* S) {
    DescT<R> d;
    d.n = P->n;
    d.m = P->m;
    d.p = P->p;
    d.pT = P->pT;
    d.T = P->T;
    d.F = static_cast<const R*>(P->F.ptr);
    d.sF = P->F.step_stride;
    d.c = static_cast<const R*>(P->c.ptr);
    d.sc = P->c.step_stride;
    d.L = static_cast<const R*>(P->L.ptr);
    d.sL = P->L.step_stride;
    d.U = static_cast<const R*>(P->U.ptr);
    d.sU = P->U.step_stride;
    d.H = static_cast<const R*>(P->H.ptr);
    d.sH = P->H.step_stride;
    d.r = static_cast<const R*>(P->r.ptr);
    d.sr = P->r.step_stride;
    d.X = static_cast<const R*>(P->X.ptr);
    d.sX = P->X.step_stride;
    d.HT = static_cast<const R*>(P->HT);
    d.rT = static_cast<const R*>(P->rT);
    d.XT = static_cast<const R*>(P->XT);
    d.x0 = static_cast<const R*>(P->x0);
    d.S = static_cast<R*>(S->S);
    d.v = static_cast<R*>(S->v);
    d.K = static_cast<R*>(S->K);
    d.x = static_cast<R*>(S->x);
    d.u = static_cast<R*>(S->u);
    d.eta = nullptr;
    d.seta = 0;
    d.etaT = nullptr;
    return d;
}

// Chain path entry points used by the C ABI (lqt_chain.cu).
// Lane-group sizes (n >= 8): the chunked pipeline is the solver.
bool chain_supported(int dtype, int n, int m);
// n <= 4 sizes with a compiled chain variant: used for Method 2 and the FULL
// refinement, which the thread-per-step kernels do not provide.
bool chain_small_supported(int dtype, int n, int m);
// Single problem: workspace bytes, chunk geometry and kernel launches.
lqt_status chain_workspace(const lqt_problem* P, bool refine, bool newton, bool sequential,
                           bool method2, size_t* bytes, int* NC, long long* B, int* kernels);
lqt_status chain_solve(const lqt_problem* P, const lqt_solution* sol, bool refine, bool newton,
                       bool sequential, bool method2, void* ws, size_t ws_bytes, cudaStream_t s,
                       Prof* prof);
// Batch of problems of one FP32 (n, m), no refinement: items[idx[0..count)].
lqt_status chain_batch_workspace(const lqt_batch_item* items, const int* idx, int count,
                                 size_t* bytes);
lqt_status chain_batch_solve(const lqt_batch_item* items, const int* idx, int count, void* ws,
                             size_t ws_bytes, int* status, cudaStream_t s);
// Warm solves (S and K known): the sizes with a chain variant, FP32 or FP64.
bool chain_warm_supported(int dtype, int n, int m);
lqt_status chain_warm_workspace(const lqt_batch_item* items, const int* idx, int count,
                                size_t* bytes);
lqt_status chain_warm_solve(const lqt_batch_item* items, const int* idx, int count, void* ws,
                            size_t ws_bytes, int* status, cudaStream_t s);

}  // namespace lqt
