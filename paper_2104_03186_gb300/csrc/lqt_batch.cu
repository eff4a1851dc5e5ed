// C ABI of the ragged batch (include/lqt.h: lqt_solve_batched): grouping by
// (n, m); n = 4 problems go to one persistent launch of the one-CTA-per-problem
// kernel (lqt_batch.cuh), the lane-group sizes to the chunked pipeline
// (lqt_chain.cuh) with all problems of a size in each of its launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lqt.h"
#include "lqt_batch_launch.cuh"
#include "lqt_chain_api.h"
#include "lqt_upload.cuh"

namespace lqt {
namespace {

constexpr size_t kAlignB = 256;
size_t up(size_t x) { return (x + kAlignB - 1) / kAlignB * kAlignB; }

struct BatchVariant {
    int n, m;
    void (*launch)(const BatchDesc* d, int count, int* ticket, int* status, cudaStream_t s,
                   cudaError_t* err);
};

const BatchVariant kBatchVariants[] = {
    {4, 2, &launch_batch<4, 2, 64>},
};
constexpr int kNumBatchVariants = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);

int batch_variant(int n, int m) {
    for (int i = 0; i < kNumBatchVariants; ++i)
        if (kBatchVariants[i].n == n && kBatchVariants[i].m == m) return i;
    return -1;
}

bool is_aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

lqt_status check_item(const lqt_batch_item& it) {
    const lqt_problem& P = it.problem;
    const lqt_solution& S = it.solution;
    if (P.dtype != LQT_F32) return LQT_EUNSUPPORTED;
    if (P.T < 0 || P.p < 1 || P.pT < 0 || P.p > 2 * P.n) return LQT_EINVAL;
    const bool lanes = chain_supported(LQT_F32, P.n, P.m);
    if (batch_variant(P.n, P.m) < 0 && !lanes) return LQT_EUNSUPPORTED;
    if (lanes && P.pT > 2 * P.n) return LQT_EUNSUPPORTED;
    if (P.T > 0 && (!P.F.ptr || !P.L.ptr || !P.U.ptr || !P.H.ptr || !P.X.ptr)) return LQT_EINVAL;
    if (!P.x0 || (P.pT > 0 && (!P.HT || !P.XT))) return LQT_EINVAL;
    if (!S.S || !S.v || !S.x || (P.T > 0 && (!S.K || !S.u))) return LQT_EINVAL;
    const int64_t n = P.n, m = P.m, p = P.p;
    const struct {
        const lqt_in* in;
        int64_t size;
    } ins[] = {{&P.F, n * n}, {&P.c, n},     {&P.L, n * m}, {&P.U, m * m},
               {&P.H, p * n}, {&P.r, p},     {&P.X, p * p}};
    for (const auto& i : ins) {
        if (!i.in->ptr) continue;
        if (!is_aligned(i.in->ptr, 4)) return LQT_EINVAL;
        if (i.in->step_stride < 0 || (i.in->step_stride != 0 && i.in->step_stride < i.size))
            return LQT_EINVAL;
    }
    return LQT_OK;
}

BatchDesc to_desc(const lqt_batch_item& it) {
    const lqt_problem& P = it.problem;
    const lqt_solution& S = it.solution;
    BatchDesc d;
    memset(&d, 0, sizeof(d));
    d.n = P.n;
    d.m = P.m;
    d.p = P.p;
    d.pT = P.pT;
    d.T = P.T;
    d.F = static_cast<const float*>(P.F.ptr);
    d.sF = P.F.step_stride;
    d.c = static_cast<const float*>(P.c.ptr);
    d.sc = P.c.step_stride;
    d.L = static_cast<const float*>(P.L.ptr);
    d.sL = P.L.step_stride;
    d.U = static_cast<const float*>(P.U.ptr);
    d.sU = P.U.step_stride;
    d.H = static_cast<const float*>(P.H.ptr);
    d.sH = P.H.step_stride;
    d.r = static_cast<const float*>(P.r.ptr);
    d.sr = P.r.step_stride;
    d.X = static_cast<const float*>(P.X.ptr);
    d.sX = P.X.step_stride;
    d.HT = static_cast<const float*>(P.HT);
    d.rT = static_cast<const float*>(P.rT);
    d.XT = static_cast<const float*>(P.XT);
    d.x0 = static_cast<const float*>(P.x0);
    d.S = static_cast<float*>(S.S);
    d.v = static_cast<float*>(S.v);
    d.K = static_cast<float*>(S.K);
    d.x = static_cast<float*>(S.x);
    d.u = static_cast<float*>(S.u);
    return d;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

// Problems of the chunked pipeline, grouped by (n, m): indices into items.
static std::vector<std::vector<int>> lane_groups(const lqt_batch_item* items, int32_t count) {
    std::vector<std::vector<int>> groups;
    std::vector<std::pair<int, int>> keys;
    for (int i = 0; i < count; ++i) {
        const lqt_problem& P = items[i].problem;
        if (batch_variant(P.n, P.m) >= 0) continue;
        size_t g = 0;
        while (g < keys.size() && keys[g] != std::make_pair(P.n, P.m)) ++g;
        if (g == keys.size()) {
            keys.emplace_back(P.n, P.m);
            groups.emplace_back();
        }
        groups[g].push_back(i);
    }
    return groups;
}

static size_t head_bytes(int32_t count) {
    return up(256) + up(64 * sizeof(int)) + up((size_t)count * sizeof(BatchDesc));
}

// The lane sizes of a batch with at least kForkSteps steps run side by side,
// each on an auxiliary stream forked from the caller's stream after the
// workspace head is cleared and joined back to it (events; a CUDA graph
// captures them as parallel branches), beside the n = 4 launch on the caller's
// stream: the sizes are independent, and one size's tree levels and last wave
// leave most SMs idle.  Smaller batches (a server's) keep the caller's stream:
// the auxiliary streams belong to the host thread, so a thread's small batches
// on several streams would otherwise queue on them.
constexpr long long kForkSteps = 1LL << 20;
constexpr int kMaxAux = 4;

struct BatchAux {
    cudaStream_t s[kMaxAux] = {};
    cudaEvent_t fork = nullptr, join[kMaxAux] = {};
    bool ready = false;
};

// This host thread's auxiliary streams and events on the current device,
// created on its first large batch there and kept until the process exits;
// nullptr if they cannot be created (the batch then runs on one stream).
static BatchAux* batch_aux() {
    thread_local BatchAux aux[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    BatchAux& a = aux[dev];
    if (!a.ready) {
        // handles made by an earlier, failed attempt are kept and not made again
        if (!a.fork && cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
        for (int i = 0; i < kMaxAux; ++i)
            if ((!a.s[i] && cudaStreamCreateWithFlags(&a.s[i], cudaStreamNonBlocking) !=
                                cudaSuccess) ||
                (!a.join[i] &&
                 cudaEventCreateWithFlags(&a.join[i], cudaEventDisableTiming) != cudaSuccess))
                return nullptr;
        a.ready = true;
    }
    return &a;
}

// Workspace bytes of each lane group (its own region, so that the groups may
// run at once); false if a group is invalid.
static bool lane_bytes_of(const lqt_batch_item* items, const std::vector<std::vector<int>>& groups,
                          std::vector<size_t>* bytes) {
    bytes->clear();
    for (const std::vector<int>& g : groups) {
        size_t b = 0;
        if (chain_batch_workspace(items, g.data(), (int)g.size(), &b) != LQT_OK) return false;
        bytes->push_back(up(b));
    }
    return true;
}

extern "C" size_t lqt_batch_workspace_bytes(const lqt_batch_item* items, int32_t count) {
    if (count < 0 || (count > 0 && !items)) return 0;
    for (int i = 0; i < count; ++i)
        if (check_item(items[i]) != LQT_OK) return 0;
    std::vector<size_t> bytes;
    if (!lane_bytes_of(items, lane_groups(items, count), &bytes)) return 0;
    size_t lane = 0;
    for (size_t b : bytes) lane += b;
    return head_bytes(count) + lane;
}

extern "C" lqt_status lqt_solve_batched(const lqt_batch_item* items, int32_t count,
                                        void* workspace, size_t workspace_bytes, void* stream) {
    if (count < 0 || (count > 0 && !items)) return LQT_EINVAL;
    if (!workspace || !is_aligned(workspace, kAlignB)) return LQT_EINVAL;
    for (int i = 0; i < count; ++i) {
        const lqt_status st = check_item(items[i]);
        if (st != LQT_OK) return st;
    }
    const size_t need = lqt_batch_workspace_bytes(items, count);
    if (need == 0 || workspace_bytes < need) return LQT_ENOMEM;
    // descriptors of the one-CTA-per-problem kernel, grouped by (n, m)
    std::vector<BatchDesc> descs;
    descs.reserve(count);
    int offset[kNumBatchVariants + 1] = {0};
    for (int v = 0; v < kNumBatchVariants; ++v) {
        offset[v] = (int)descs.size();
        for (int i = 0; i < count; ++i)
            if (batch_variant(items[i].problem.n, items[i].problem.m) == v)
                descs.push_back(to_desc(items[i]));
    }
    offset[kNumBatchVariants] = (int)descs.size();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    int* status = reinterpret_cast<int*>(base);
    int* tickets = reinterpret_cast<int*>(base + up(256));
    BatchDesc* d_desc = reinterpret_cast<BatchDesc*>(base + up(256) + up(64 * sizeof(int)));
    if (cudaMemsetAsync(base, 0, up(256) + up(64 * sizeof(int)), s) != cudaSuccess)
        return LQT_ECUDA;
    if (count == 0) return LQT_OK;
    const std::vector<std::vector<int>> groups = lane_groups(items, count);
    std::vector<size_t> group_bytes;
    if (!lane_bytes_of(items, groups, &group_bytes)) return LQT_EINVAL;
    long long total_steps = 0;
    for (int i = 0; i < count; ++i) total_steps += items[i].problem.T;
    const int lanes_running = (int)groups.size();
    BatchAux* aux = nullptr;
    if (lanes_running >= 1 && lanes_running <= kMaxAux &&
        lanes_running + (descs.empty() ? 0 : 1) >= 2 && total_steps >= kForkSteps)
        aux = batch_aux();
    if (aux && cudaEventRecord(aux->fork, s) != cudaSuccess) return LQT_ECUDA;
    if (!descs.empty()) {
        // through kernel parameters (lqt_upload.cuh): a pageable copy would
        // first wait for the stream, and could not be captured in a graph
        if (param_upload(d_desc, descs.data(), descs.size() * sizeof(BatchDesc), s) !=
            cudaSuccess)
            return LQT_ECUDA;
        for (int v = 0; v < kNumBatchVariants; ++v) {
            const int c = offset[v + 1] - offset[v];
            if (c == 0) continue;
            cudaError_t err = cudaSuccess;
            kBatchVariants[v].launch(d_desc + offset[v], c, tickets + v, status, s, &err);
            if (err != cudaSuccess) return LQT_ECUDA;
        }
    }
    char* lane_ws = base + head_bytes(count);
    // The auxiliary streams that already hold part of the batch rejoin the
    // caller's stream on every return, an error included: the work they hold
    // still uses the workspace, and a capture on `stream` must end joined.
    int forked = 0;
    auto rejoin = [&](lqt_status st) {
        for (int i = 0; i < forked; ++i)
            if (cudaEventRecord(aux->join[i], aux->s[i]) != cudaSuccess ||
                cudaStreamWaitEvent(s, aux->join[i], 0) != cudaSuccess)
                st = st == LQT_OK ? LQT_ECUDA : st;
        return st;
    };
    for (size_t i = 0; i < groups.size(); ++i) {
        const std::vector<int>& g = groups[i];
        cudaStream_t gs = s;
        if (aux) {
            gs = aux->s[i];
            if (cudaStreamWaitEvent(gs, aux->fork, 0) != cudaSuccess) return rejoin(LQT_ECUDA);
            forked = (int)i + 1;
        }
        const lqt_status st = chain_batch_solve(items, g.data(), (int)g.size(), lane_ws,
                                                group_bytes[i], status, gs);
        if (st != LQT_OK) return rejoin(st);
        lane_ws += group_bytes[i];
    }
    return rejoin(LQT_OK);
}
