// Chunked single-problem pipeline behind the C ABI (lqt_solve and
// lqt_riccati_sequential for the lane-group sizes): variant lookup, chunk
// geometry, workspace layout.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "lqt_chain_api.h"

namespace lqt {
namespace {

// smallest chunk the planner makes, in steps
constexpr long long kMinChunk = 4;

// Batches of the lane sizes: one launch per tree level, one persistent
// launch, or (the default) the persistent launch where its grid needs at most
// half of the CTAs the device holds at once, per-level launches otherwise
// (lqt_batch_set_tuning).  Measured on one GB300 (time-varying random
// problems, p = n, chunk lengths as planned): the persistent launch took
// 5-20% off single problems and batches of 16 at n = 8, 16, 32 and
// T = 128..2048, and lost where its chunks were many waves of the device's
// groups (n = 32, 16 problems of T = 2048 in 4-step chunks: 7.5 against
// 6.1 ms; the 4096-problem benchmark batch: 47.3 against 45.8 ms).  A server
// running batches on several streams at once lost twice its latency at
// 20 000 requests/s when every batch took a cooperative launch: a launch whose
// grid covers the device waits for the other streams' kernels to leave.
std::atomic<int> g_batch_mode{LQT_BATCH_AUTO};

// Tuned chunk lengths of batches (lqt_batch_set_tuning): entry e applies to
// problems of state size n = e.n with T <= e.t_max (the first such entry).
constexpr int kMaxTune = 64;
std::mutex g_tune_mu;
lqt_batch_tune_entry g_tune[kMaxTune];
int g_tune_count = 0;

// The tuned chunk length for a problem, or 0 (none).
long long tuned_chunk(int n, long long T) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int i = 0; i < g_tune_count; ++i)
        if (g_tune[i].n == n && T <= g_tune[i].t_max) return g_tune[i].chunk_steps;
    return 0;
}

const ChainVariant* find_chain(int dtype, int n, int m, bool mixed) {
    const ChainVariant* (*tables[])(int*) = {&chain_variants_n4, &chain_variants_n8,
                                             &chain_variants_n16, &chain_variants_n32};
    for (auto t : tables) {
        int cnt = 0;
        const ChainVariant* v = t(&cnt);
        for (int i = 0; i < cnt; ++i)
            if (v[i].dtype == dtype && v[i].n == n && v[i].m == m &&
                (dtype == LQT_F64 || (v[i].mixed != 0) == mixed))
                return &v[i];
    }
    return nullptr;
}

// Resident lane groups of the fold kernel on the whole device.
lqt_status fold_slots(const ChainVariant& v, long long* slots) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LQT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LQT_ECUDA;
    const size_t smem = v.fold_smem();
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(v.fold_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return LQT_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fold_kernel(),
                                                      v.fold_groups() * v.n, smem) != cudaSuccess)
        return LQT_ECUDA;
    *slots = (long long)sms * (per_sm > 0 ? per_sm : 1) * v.fold_groups();
    return LQT_OK;
}

lqt_status geometry(const ChainVariant& v, const lqt_problem* P, bool sequential, int* NC,
                    long long* B) {
    const long long T = P->T;
    if (sequential) {
        *NC = 1;
        *B = T > 0 ? T : 1;
        return LQT_OK;
    }
    long long slots = 0;
    const lqt_status st = fold_slots(v, &slots);
    if (st != LQT_OK) return st;
    long long cap = T / kMinChunk;
    if (cap > slots) cap = slots;
    if (cap > (1LL << 24)) cap = 1LL << 24;
    long long nc = 1;
    while (nc * 2 <= cap) nc *= 2;
    *NC = (int)nc;
    *B = T > 0 ? (T + nc - 1) / nc : 1;
    return LQT_OK;
}

int levels(int NC) {
    int l = 0;
    while ((1 << l) < NC) ++l;
    return l;
}

// Chunk geometry of a batch of one variant: a chunk length B* from the
// total work over the resident fold groups, clamped to [kMinChunk,
// kMaxBatchChunk] so that no problem's latency grows with the batch, or the
// tuned length of the problem's (n, T) where it is shorter than the unclamped
// fill length; each problem takes the largest power-of-two chunk count with
// chunks of at least that many steps.  Problems sorted by decreasing chunk
// count.
constexpr long long kMaxBatchChunk = 64;

lqt_status batch_geometry(const ChainVariant& v, const lqt_batch_item* items, const int* idx,
                          int count, std::vector<ChainProblem>* out) {
    long long slots = 0;
    const lqt_status st = fold_slots(v, &slots);
    if (st != LQT_OK) return st;
    long long total = 0;
    for (int i = 0; i < count; ++i) total += items[idx[i]].problem.T;
    long long fill = (total + slots - 1) / (slots > 0 ? slots : 1);
    if (fill < kMinChunk) fill = kMinChunk;
    const long long Bt = fill < kMaxBatchChunk ? fill : kMaxBatchChunk;
    out->resize((size_t)count);
    for (int i = 0; i < count; ++i) {
        const lqt_batch_item& it = items[idx[i]];
        const long long T = it.problem.T;
        // a tuned length applies up to the one that fills the device: a batch
        // with less work than that keeps every resident group busy instead
        const long long tuned = tuned_chunk(it.problem.n, T);
        const long long Bi = tuned > 0 ? (tuned < fill ? tuned : fill) : Bt;
        long long nc = 1;
        while (nc * 2 * Bi <= T && nc < (1LL << 20)) nc *= 2;
        ChainProblem& cp = (*out)[(size_t)i];
        cp.problem = &it.problem;
        cp.solution = &it.solution;
        cp.NC = (int)nc;
        cp.B = T > 0 ? (T + nc - 1) / nc : 1;
    }
    std::stable_sort(out->begin(), out->end(),
                     [](const ChainProblem& a, const ChainProblem& b) { return a.NC > b.NC; });
    return LQT_OK;
}

}  // namespace

bool chain_supported(int dtype, int n, int m) {
    return n >= 8 && find_chain(dtype, n, m, false) != nullptr;
}

bool chain_small_supported(int dtype, int n, int m) {
    return n < 8 && find_chain(dtype, n, m, false) != nullptr;
}

lqt_status chain_workspace(const lqt_problem* P, bool refine, bool newton, bool sequential,
                           bool method2, size_t* bytes, int* NC, long long* B, int* kernels) {
    if (P->p > 2 * P->n || P->pT > 2 * P->n) return LQT_EUNSUPPORTED;
    // FP64 tree levels with the FULL refinement (the Newton step); FP32 otherwise
    const bool mixed = refine && newton && P->dtype == LQT_F32;
    const ChainVariant* v = find_chain(P->dtype, P->n, P->m, mixed);
    if (!v) return LQT_EUNSUPPORTED;
    int nc = 1;
    long long b = 1;
    const lqt_status st = geometry(*v, P, sequential, &nc, &b);
    if (st != LQT_OK) return st;
    ChainProblem cp{P, nullptr, nc, b};
    const bool rf = refine && P->T > 0;
    if (bytes) *bytes = v->workspace(&cp, 1, rf, rf && newton, method2);
    if (NC) *NC = nc;
    if (B) *B = b;
    if (kernels) {
        const int l = levels(nc);
        // Method 2: the element copy, 2 l sweep levels, the seeds, the walk
        const int fwd = method2 ? 2 * l + 2 : (sequential ? 0 : 2 * l);
        const int per_pass = (sequential ? 2 : 3 + 2 * l) + fwd + (method2 ? 0 : 1);
        const int bwd = sequential ? 2 : 3 + 2 * l;
        int k = 1 + per_pass;  // the item upload, the solve
        if (rf) k += 1 + 1 + per_pass;  // item upload, KKT residuals, correction solve
        if (rf && newton) k += 2 + bwd + 2;  // constants, residuals, dS/dv scan, gains, add
        *kernels = k;
    }
    return LQT_OK;
}

lqt_status chain_solve(const lqt_problem* P, const lqt_solution* sol, bool refine, bool newton,
                       bool sequential, bool method2, void* ws, size_t ws_bytes, cudaStream_t s,
                       Prof* prof) {
    if (P->p > 2 * P->n || P->pT > 2 * P->n) return LQT_EUNSUPPORTED;
    const bool mixed = refine && newton && P->dtype == LQT_F32;
    const ChainVariant* v = find_chain(P->dtype, P->n, P->m, mixed);
    if (!v) return LQT_EUNSUPPORTED;
    int NC = 1;
    long long B = 1;
    const lqt_status st = geometry(*v, P, sequential, &NC, &B);
    if (st != LQT_OK) return st;
    ChainProblem cp{P, sol, NC, B};
    const bool rf = refine && P->T > 0;
    ChainCall call{&cp, 1, rf, rf && newton, sequential, method2, ws, ws_bytes, nullptr};
    return v->run(call, s, prof);
}

lqt_status chain_batch_workspace(const lqt_batch_item* items, const int* idx, int count,
                                 size_t* bytes) {
    *bytes = 0;
    if (count <= 0) return LQT_OK;
    const lqt_problem& P0 = items[idx[0]].problem;
    const ChainVariant* v = find_chain(LQT_F32, P0.n, P0.m, false);
    if (!v) return LQT_EUNSUPPORTED;
    std::vector<ChainProblem> probs;
    const lqt_status st = batch_geometry(*v, items, idx, count, &probs);
    if (st != LQT_OK) return st;
    *bytes = v->workspace(probs.data(), count, false, false, false);
    return LQT_OK;
}

lqt_status chain_batch_solve(const lqt_batch_item* items, const int* idx, int count, void* ws,
                             size_t ws_bytes, int* status, cudaStream_t s) {
    if (count <= 0) return LQT_OK;
    const lqt_problem& P0 = items[idx[0]].problem;
    const ChainVariant* v = find_chain(LQT_F32, P0.n, P0.m, false);
    if (!v) return LQT_EUNSUPPORTED;
    std::vector<ChainProblem> probs;
    const lqt_status st = batch_geometry(*v, items, idx, count, &probs);
    if (st != LQT_OK) return st;
    ChainCall call{probs.data(), count, false, false, false, false, ws, ws_bytes, status};
    const int mode = g_batch_mode.load();
    call.persistent = mode != LQT_BATCH_PER_LEVEL;
    call.persistent_if_small = mode == LQT_BATCH_AUTO;
    return v->run(call, s, nullptr);
}

bool chain_warm_supported(int dtype, int n, int m) {
    return find_chain(dtype, n, m, false) != nullptr;
}

namespace {

// Chunk geometry of a warm call: one problem as lqt_solve cuts it, a batch as
// lqt_solve_batched does.
lqt_status warm_geometry(const ChainVariant& v, const lqt_batch_item* items, const int* idx,
                         int count, std::vector<ChainProblem>* probs) {
    if (count == 1) {
        const lqt_batch_item& it = items[idx[0]];
        int nc = 1;
        long long b = 1;
        const lqt_status st = geometry(v, &it.problem, false, &nc, &b);
        if (st != LQT_OK) return st;
        probs->assign(1, ChainProblem{&it.problem, &it.solution, nc, b});
        return LQT_OK;
    }
    return batch_geometry(v, items, idx, count, probs);
}

}  // namespace

lqt_status chain_warm_workspace(const lqt_batch_item* items, const int* idx, int count,
                                size_t* bytes) {
    *bytes = 0;
    if (count <= 0) return LQT_OK;
    const lqt_problem& P0 = items[idx[0]].problem;
    const ChainVariant* v = find_chain(P0.dtype, P0.n, P0.m, false);
    if (!v) return LQT_EUNSUPPORTED;
    std::vector<ChainProblem> probs;
    const lqt_status st = warm_geometry(*v, items, idx, count, &probs);
    if (st != LQT_OK) return st;
    *bytes = v->workspace(probs.data(), count, false, false, false);
    return LQT_OK;
}

lqt_status chain_warm_solve(const lqt_batch_item* items, const int* idx, int count, void* ws,
                            size_t ws_bytes, int* status, cudaStream_t s) {
    if (count <= 0) return LQT_OK;
    const lqt_problem& P0 = items[idx[0]].problem;
    const ChainVariant* v = find_chain(P0.dtype, P0.n, P0.m, false);
    if (!v) return LQT_EUNSUPPORTED;
    std::vector<ChainProblem> probs;
    const lqt_status st = warm_geometry(*v, items, idx, count, &probs);
    if (st != LQT_OK) return st;
    ChainCall call{probs.data(), count, false, false, false, false, ws, ws_bytes, status};
    call.warm = true;
    return v->run(call, s, nullptr);
}

}  // namespace lqt

extern "C" lqt_status lqt_batch_set_tuning(const lqt_batch_tune_entry* entries, int32_t count,
                                           int32_t persistent) {
    using namespace lqt;
    if (count < 0 || count > kMaxTune || (count > 0 && !entries)) return LQT_EINVAL;
    if (persistent < LQT_BATCH_PER_LEVEL || persistent > LQT_BATCH_AUTO) return LQT_EINVAL;
    for (int i = 0; i < count; ++i)
        if (entries[i].n < 1 || entries[i].t_max < 0 || entries[i].chunk_steps < 1)
            return LQT_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int i = 0; i < count; ++i) g_tune[i] = entries[i];
    g_tune_count = count;
    g_batch_mode.store(persistent);
    return LQT_OK;
}
