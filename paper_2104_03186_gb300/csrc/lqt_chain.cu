// Chunked single-problem pipeline behind the C ABI (lqt_solve and
// lqt_riccati_sequential for the lane-group sizes): variant lookup, chunk
// geometry, workspace layout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lqt_chain_api.h"

namespace lqt {
namespace {

constexpr size_t kAlignC = 256;
constexpr size_t kStatusC = 256;
size_t up_c(size_t x) { return (x + kAlignC - 1) / kAlignC * kAlignC; }

// smallest chunk the planner makes, in steps
constexpr long long kMinChunk = 4;

const ChainVariant* find_chain(int dtype, int n, int m, bool mixed) {
    const ChainVariant* (*tables[])(int*) = {&chain_variants_n8, &chain_variants_n16,
                                             &chain_variants_n32};
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

struct ChainLayout {
    size_t E, V, FE, X, rp, cp, rTp, x0p, total;
};

ChainLayout chain_layout(const ChainVariant& v, const lqt_problem* P, int NC, bool refine) {
    const size_t n = (size_t)P->n, rt = (size_t)v.rtsize, r = (size_t)v.rsize;
    const size_t nc = (size_t)NC;
    ChainLayout L;
    size_t off = kStatusC;
    L.E = off;
    off += up_c(nc * (3 * n * n + 2 * n) * rt);
    L.V = off;
    off += up_c(nc * (n * n + n) * rt);
    L.FE = off;
    off += up_c(nc * (n * n + n) * rt);
    L.X = off;
    off += up_c(nc * n * rt);
    L.rp = L.cp = L.rTp = L.x0p = 0;
    if (refine) {
        const size_t T = (size_t)P->T;
        L.rp = off;
        off += up_c(T * (size_t)P->p * r);
        L.cp = off;
        off += up_c(T * n * r);
        L.rTp = off;
        off += up_c((size_t)P->pT * r);
        L.x0p = off;
        off += up_c(n * r);
    }
    L.total = off;
    return L;
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

}  // namespace

bool chain_supported(int dtype, int n, int m) { return find_chain(dtype, n, m, false) != nullptr; }

lqt_status chain_workspace(const lqt_problem* P, bool refine, bool sequential, size_t* bytes,
                           int* NC, long long* B, int* kernels) {
    if (P->p > 2 * P->n) return LQT_EUNSUPPORTED;
    const bool mixed = refine && P->dtype == LQT_F32;
    const ChainVariant* v = find_chain(P->dtype, P->n, P->m, mixed);
    if (!v) return LQT_EUNSUPPORTED;
    int nc = 1;
    long long b = 1;
    const lqt_status st = geometry(*v, P, sequential, &nc, &b);
    if (st != LQT_OK) return st;
    if (bytes) *bytes = chain_layout(*v, P, nc, refine).total;
    if (NC) *NC = nc;
    if (B) *B = b;
    if (kernels) {
        const int l = levels(nc);
        const int per_pass = sequential ? 3 : 4 + 4 * l;
        *kernels = (refine && P->T > 0) ? 2 * per_pass + 1 : per_pass;
    }
    return LQT_OK;
}

lqt_status chain_solve(const lqt_problem* P, const lqt_solution* sol, bool refine,
                       bool sequential, void* ws, size_t ws_bytes, cudaStream_t s, Prof* prof) {
    if (P->p > 2 * P->n) return LQT_EUNSUPPORTED;
    const bool mixed = refine && P->dtype == LQT_F32;
    const ChainVariant* v = find_chain(P->dtype, P->n, P->m, mixed);
    if (!v) return LQT_EUNSUPPORTED;
    int NC = 1;
    long long B = 1;
    lqt_status st = geometry(*v, P, sequential, &NC, &B);
    if (st != LQT_OK) return st;
    const ChainLayout L = chain_layout(*v, P, NC, refine);
    if (ws_bytes < L.total) return LQT_ENOMEM;
    char* base = static_cast<char*>(ws);
    ChainCall call;
    call.problem = P;
    call.solution = sol;
    call.NC = NC;
    call.B = B;
    call.refine = refine;
    call.sequential = sequential;
    call.status = reinterpret_cast<int*>(base);
    call.E = base + L.E;
    call.V = base + L.V;
    call.FE = base + L.FE;
    call.X = base + L.X;
    call.rp = refine ? base + L.rp : nullptr;
    call.cp = refine ? base + L.cp : nullptr;
    call.rTp = refine ? base + L.rTp : nullptr;
    call.x0p = refine ? base + L.x0p : nullptr;
    return v->run(call, s, prof);
}

}  // namespace lqt
