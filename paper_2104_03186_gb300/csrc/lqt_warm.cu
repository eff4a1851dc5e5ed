// C ABI of the warm solve (include/lqt.h: lqt_solve_warm): problems whose S_k
// and K_k are known (a receding horizon over an earlier solve's model), solved
// for v, x* and u* by the vector scans of lqt_warm.cuh.  Problems are grouped
// by (dtype, n, m); each group is one chain call, the groups run one after
// another on the stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "lqt.h"
#include "lqt_chain_api.h"

namespace lqt {
namespace {

constexpr size_t kAlignW = 256;
size_t up(size_t x) { return (x + kAlignW - 1) / kAlignW * kAlignW; }

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

lqt_status check_warm_item(const lqt_batch_item& it) {
    const lqt_problem& P = it.problem;
    const lqt_solution& S = it.solution;
    if (P.dtype != LQT_F32 && P.dtype != LQT_F64) return LQT_EINVAL;
    if (P.n < 1 || P.m < 1 || P.T < 0 || P.p < 0 || P.pT < 0) return LQT_EINVAL;
    if (!chain_warm_supported(P.dtype, P.n, P.m)) return LQT_EUNSUPPORTED;
    if (P.p > 2 * P.n || P.pT > 2 * P.n) return LQT_EUNSUPPORTED;
    if (P.T > 0 && (!P.F.ptr || !P.L.ptr || !P.U.ptr)) return LQT_EINVAL;
    if (P.T > 0 && P.p > 0 && (!P.H.ptr || !P.X.ptr)) return LQT_EINVAL;
    if (!P.x0 || (P.pT > 0 && (!P.HT || !P.XT))) return LQT_EINVAL;
    if (!S.S || !S.v || !S.x || (P.T > 0 && (!S.K || !S.u))) return LQT_EINVAL;
    const size_t es = P.dtype == LQT_F64 ? 8 : 4;
    const int64_t n = P.n, m = P.m, p = P.p;
    const struct {
        const lqt_in* in;
        int64_t size;
    } ins[] = {{&P.F, n * n}, {&P.c, n}, {&P.L, n * m}, {&P.U, m * m},
               {&P.H, p * n}, {&P.r, p}, {&P.X, p * p}};
    for (const auto& i : ins) {
        if (!i.in->ptr) continue;
        if (!aligned_to(i.in->ptr, es)) return LQT_EINVAL;
        if (i.in->step_stride < 0 || (i.in->step_stride != 0 && i.in->step_stride < i.size))
            return LQT_EINVAL;
    }
    const void* outs[] = {S.S, S.v, S.K, S.x, S.u};
    for (const void* o : outs)
        if (o && !aligned_to(o, es)) return LQT_EINVAL;
    return LQT_OK;
}

// Indices of the items, grouped by (dtype, n, m).
std::vector<std::vector<int>> warm_groups(const lqt_batch_item* items, int32_t count) {
    std::vector<std::vector<int>> groups;
    std::vector<std::pair<int, std::pair<int, int>>> keys;
    for (int i = 0; i < count; ++i) {
        const lqt_problem& P = items[i].problem;
        const auto key = std::make_pair((int)P.dtype, std::make_pair(P.n, P.m));
        size_t g = 0;
        while (g < keys.size() && keys[g] != key) ++g;
        if (g == keys.size()) {
            keys.push_back(key);
            groups.emplace_back();
        }
        groups[g].push_back(i);
    }
    return groups;
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" size_t lqt_warm_workspace_bytes(const lqt_batch_item* items, int32_t count) {
    if (count < 0 || (count > 0 && !items)) return 0;
    for (int i = 0; i < count; ++i)
        if (check_warm_item(items[i]) != LQT_OK) return 0;
    size_t most = 0;
    for (const std::vector<int>& g : warm_groups(items, count)) {
        size_t b = 0;
        if (chain_warm_workspace(items, g.data(), (int)g.size(), &b) != LQT_OK) return 0;
        most = std::max(most, b);
    }
    return up(256) + up(most);
}

extern "C" lqt_status lqt_solve_warm(const lqt_batch_item* items, int32_t count, void* workspace,
                                     size_t workspace_bytes, void* stream) {
    if (count < 0 || (count > 0 && !items)) return LQT_EINVAL;
    if (!workspace || !aligned_to(workspace, kAlignW)) return LQT_EINVAL;
    for (int i = 0; i < count; ++i) {
        const lqt_status st = check_warm_item(items[i]);
        if (st != LQT_OK) return st;
    }
    const size_t need = lqt_warm_workspace_bytes(items, count);
    if (need == 0 || workspace_bytes < need) return LQT_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    int* status = reinterpret_cast<int*>(base);
    if (cudaMemsetAsync(base, 0, sizeof(int), s) != cudaSuccess) return LQT_ECUDA;
    char* ws = base + up(256);
    const size_t ws_bytes = workspace_bytes - up(256);
    for (const std::vector<int>& g : warm_groups(items, count)) {
        const lqt_status st = chain_warm_solve(items, g.data(), (int)g.size(), ws, ws_bytes,
                                               status, s);
        if (st != LQT_OK) return st;
    }
    return LQT_OK;
}
