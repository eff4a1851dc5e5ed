// C ABI of the LQT solver (include/lqt.h): argument validation, launch
// planning, workspace layout, dispatch to the compiled (dtype, n, m) variants,
// kernel timing and the host-buffer solve.
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "lqt.h"
#include "lqt_chain_api.h"
#include "lqt_kernels.cuh"
#include "lqt_launch.cuh"
#include "lqt_refine.cuh"
#include "lqt_variants.h"

namespace lqt {

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStatusBytes = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int sm_count_current() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev].load(std::memory_order_relaxed) == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        cache[dev].store(sms, std::memory_order_relaxed);
        return sms;
    }
    return cache[dev].load(std::memory_order_relaxed);
}

size_t elem_bytes(int dtype) { return dtype == LQT_F64 ? 8 : 4; }

// Per-instantiation sizes the planner needs.
struct Variant {
    int dtype, n, m;
    int W, TP;
    int elem, value, affine;  // components of an element, a value, an affine map
    lqt_status (*solve)(const void* params, const Plan& plan, cudaStream_t s, Prof* prof,
                        cudaEvent_t bwd_done);
    lqt_status (*seq)(const void* params, cudaStream_t s);
};

template <typename R, int N, int M>
lqt_status solve_thunk(const void* params, const Plan& plan, cudaStream_t s, Prof* prof,
                       cudaEvent_t bwd_done) {
    return launch_solve<R, N, M>(*static_cast<const Params<R>*>(params), plan, s, prof, bwd_done);
}

template <typename R, int N, int M>
lqt_status seq_thunk(const void* params, cudaStream_t s) {
    return launch_seq<R, N, M>(*static_cast<const Params<R>*>(params), s);
}

#define LQT_VARIANT_ROW(R, N, M)                                                                \
    Variant{sizeof(R) == 8 ? LQT_F64 : LQT_F32, N, M, tile_threads<R, N, M>(), top_threads(),        \
            Dims<N>::ELEM, Dims<N>::VALUE, Dims<N>::AFFINE, &solve_thunk<R, N, M>,                \
            &seq_thunk<R, N, M>},

const Variant kVariants[] = {LQT_VARIANTS(LQT_VARIANT_ROW)};

const Variant* find_variant(int dtype, int n, int m) {
    for (const Variant& v : kVariants)
        if (v.dtype == dtype && v.n == n && v.m == m) return &v;
    return nullptr;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The chunked pipeline solves the lane-group sizes, and the n <= 4 problems
// that ask for Method 2 or the FULL refinement where a small chain variant is
// compiled.  False with *unsupported set: no kernel serves these options.
bool use_chain(const lqt_problem* P, const Variant* var, bool newton, bool method2,
               bool* unsupported) {
    *unsupported = false;
    if (!var) {
        *unsupported = !chain_supported(P->dtype, P->n, P->m);
        return !*unsupported;
    }
    const bool small_chain = chain_small_supported(P->dtype, P->n, P->m) &&
                             P->p <= 2 * P->n && P->pT <= 2 * P->n;
    if (method2 && !small_chain) *unsupported = true;
    return (method2 || newton) && small_chain;
}

// Validates everything that does not depend on a compiled variant.
lqt_status validate(const lqt_problem* P, const lqt_solution* sol) {
    if (!P) return LQT_EINVAL;
    if (P->dtype != LQT_F32 && P->dtype != LQT_F64) return LQT_EINVAL;
    if (P->n < 1 || P->m < 1 || P->p < 0 || P->pT < 0 || P->T < 0) return LQT_EINVAL;
    if (P->T > (int64_t(1) << 40)) return LQT_EINVAL;
    const size_t es = elem_bytes(P->dtype);
    const int64_t n = P->n, m = P->m, p = P->p, pT = P->pT;
    struct In {
        const lqt_in* in;
        int64_t size;
        bool optional;
    } ins[] = {{&P->F, n * n, false}, {&P->c, n, true},     {&P->L, n * m, false},
               {&P->U, m * m, false}, {&P->H, p * n, p == 0}, {&P->r, p, true},
               {&P->X, p * p, p == 0}};
    for (const In& i : ins) {
        if (!i.in->ptr) {
            if (!i.optional && P->T > 0) return LQT_EINVAL;
            continue;
        }
        if (!aligned(i.in->ptr, es)) return LQT_EINVAL;
        if (i.in->step_stride != 0 && i.in->step_stride < i.size) return LQT_EINVAL;
        if (i.in->step_stride < 0) return LQT_EINVAL;
    }
    if (pT > 0 && (!P->HT || !P->XT)) return LQT_EINVAL;
    if (!P->x0) return LQT_EINVAL;
    const void* terms[] = {P->HT, P->rT, P->XT, P->x0};
    for (const void* t : terms)
        if (t && !aligned(t, es)) return LQT_EINVAL;
    if (sol) {
        if (!sol->S || !sol->v || !sol->x) return LQT_EINVAL;
        if (P->T > 0 && (!sol->K || !sol->u)) return LQT_EINVAL;
        const void* outs[] = {sol->S, sol->v, sol->K, sol->x, sol->u};
        for (const void* o : outs)
            if (o && !aligned(o, 16)) return LQT_EINVAL;
    }
    return LQT_OK;
}

lqt_status resolve_refine(const lqt_problem* P, const lqt_options* o, bool* refine,
                          bool* newton = nullptr, bool* method2 = nullptr) {
    int mode = LQT_REFINE_AUTO;
    if (o) {
        for (int r : o->reserved)
            if (r != 0) return LQT_EINVAL;
        if (o->wait_probe_polls < 0) return LQT_EINVAL;
        if (o->method != LQT_METHOD_DEFAULT && o->method != LQT_METHOD_1 &&
            o->method != LQT_METHOD_2)
            return LQT_EINVAL;
        mode = o->refine;
    }
    const bool m2 = o && o->method == LQT_METHOD_2;
    if (method2) *method2 = m2;
    if (newton) *newton = mode == LQT_REFINE_FULL;
    if (mode == LQT_REFINE_AUTO)
        *refine = P->dtype == LQT_F32;
    else if (mode == LQT_REFINE_ON || mode == LQT_REFINE_OFF || mode == LQT_REFINE_FULL)
        *refine = mode != LQT_REFINE_OFF;
    else
        return LQT_EINVAL;
    if (*refine && P->T > 0 && P->p > 0 && !P->H.ptr) return LQT_EINVAL;
    return LQT_OK;
}

// A problem whose steps fit one tile with chunks of at most this many steps
// (0 < T <= W x this) runs in one CTA, each pass one launch of k_solo; 0
// turns that off.  lqt_set_single_tile_chunk sets it.
constexpr int kSingleTileChunkDefault = 2;
std::atomic<int> g_single_tile_chunk{kSingleTileChunkDefault};

lqt_status make_plan(const lqt_problem* P, const Variant& var, Plan* plan) {
    const int sms = sm_count_current();
    if (sms <= 0) return LQT_ECUDA;
    const int64_t W = var.W;
    plan->solo = 0;
    if (P->T > 0 && P->T <= W * (int64_t)g_single_tile_chunk.load()) {
        // one tile: chunks of ceil(T / W) steps, every pass one launch
        const int64_t B = (P->T + W - 1) / W;
        if (B <= INT32_MAX) {
            plan->B = (int)B;
            plan->W = (int)W;
            plan->tiles = 1;
            plan->TP = var.TP;
            plan->solo = 1;
            return LQT_OK;
        }
    }
    const int64_t target = (int64_t)sms * W;
    int64_t B = (P->T + target - 1) / target;
    if (B < 1) B = 1;
    const int64_t tiles = (P->T + W * B - 1) / (W * B);
    if (B > INT32_MAX || tiles > INT32_MAX) return LQT_EINVAL;
    plan->B = (int)B;
    plan->W = (int)W;
    plan->tiles = (int)tiles;
    plan->TP = var.TP;
    return LQT_OK;
}

// Step stride of the shifted references r' (padded to 4 when p <= 4 so that the
// rollout can store them through its warp staging rows).
int refine_r_stride(int p) { return p <= kRStage ? kRStage : p; }

struct Layout {
    size_t tree, tile_agg, tile_carry, ftree, ftile_agg, ftile_x;
    // refinement: maps recorded by the first pass's top-level scan (0: none)
    size_t top_fac;
    // refinement: shifted references and offsets, zero initial state
    size_t rp, rTp, cp, x0p;
    size_t total;
};

// The second pass of a refined solve replays the first pass's top-level
// backward scan from recorded maps when every top-scan thread holds one tile
// and the staged maps fit the CTA's shared memory.
bool top_replay(const Variant& var, const Plan& plan, size_t es) {
    return plan.tiles > 0 && plan.tiles <= var.TP &&
           top_smem_bytes(var.elem, var.value, var.n, var.TP, (int)es, true) <= kTopSmemMax;
}

Layout layout(const Variant& var, const Plan& plan, size_t es, const lqt_problem* P,
              bool refine) {
    Layout L;
    size_t off = kStatusBytes;
    const size_t t = (size_t)plan.tiles;
    L.tree = off;
    off += align_up(t * var.elem * tstride(plan.W, (int)es) * es);
    L.tile_agg = off;
    off += align_up(t * var.elem * es);
    L.tile_carry = off;
    off += align_up(t * var.value * es);
    L.ftree = off;
    off += align_up(t * var.affine * tstride(plan.W, (int)es) * es);
    L.ftile_agg = off;
    off += align_up(t * var.affine * es);
    L.ftile_x = off;
    off += align_up(t * var.n * es);
    L.rp = L.rTp = L.cp = L.x0p = 0;
    L.top_fac = 0;
    if (refine && top_replay(var, plan, es)) {
        L.top_fac = off;
        off += align_up((size_t)top_fac_elems(var.n, var.TP) * es);
    }
    if (refine) {
        const size_t T = (size_t)P->T, n = (size_t)P->n;
        L.rp = off;
        off += align_up(T * (size_t)refine_r_stride(P->p) * es);
        L.rTp = off;
        off += align_up((size_t)P->pT * es);
        L.cp = off;
        off += align_up(T * n * es);
        L.x0p = off;
        off += align_up(n * es);
    }
    L.total = off;
    return L;
}

template <typename R>
void fill_params(Params<R>& K, const lqt_problem* P, const lqt_solution* sol, void* ws,
                 const Layout* L, const Plan* plan) {
    memset(&K, 0, sizeof(K));
    K.n = P->n;
    K.m = P->m;
    K.p = P->p;
    K.pT = P->pT;
    K.T = P->T;
    K.F = static_cast<const R*>(P->F.ptr);
    K.c = static_cast<const R*>(P->c.ptr);
    K.L = static_cast<const R*>(P->L.ptr);
    K.U = static_cast<const R*>(P->U.ptr);
    K.H = static_cast<const R*>(P->H.ptr);
    K.r = static_cast<const R*>(P->r.ptr);
    K.X = static_cast<const R*>(P->X.ptr);
    K.sF = P->F.step_stride;
    K.sc = P->c.step_stride;
    K.sL = P->L.step_stride;
    K.sU = P->U.step_stride;
    K.sH = P->H.step_stride;
    K.sr = P->r.step_stride;
    K.sX = P->X.step_stride;
    K.HT = static_cast<const R*>(P->HT);
    K.rT = static_cast<const R*>(P->rT);
    K.XT = static_cast<const R*>(P->XT);
    K.x0 = static_cast<const R*>(P->x0);
    K.S = static_cast<R*>(sol->S);
    K.v = static_cast<R*>(sol->v);
    K.K = static_cast<R*>(sol->K);
    K.x = static_cast<R*>(sol->x);
    K.u = static_cast<R*>(sol->u);
    char* base = static_cast<char*>(ws);
    K.status = reinterpret_cast<int*>(base);
    if (L) {
        K.tree = reinterpret_cast<R*>(base + L->tree);
        K.tile_agg = reinterpret_cast<R*>(base + L->tile_agg);
        K.tile_carry = reinterpret_cast<R*>(base + L->tile_carry);
        K.ftree = reinterpret_cast<R*>(base + L->ftree);
        K.ftile_agg = reinterpret_cast<R*>(base + L->ftile_agg);
        K.ftile_x = reinterpret_cast<R*>(base + L->ftile_x);
        if (L->top_fac) K.top_fac = reinterpret_cast<R*>(base + L->top_fac);
        if (L->rp | L->rTp | L->cp | L->x0p) {
            K.rp = reinterpret_cast<R*>(base + L->rp);
            K.rTp = reinterpret_cast<R*>(base + L->rTp);
            K.cp = reinterpret_cast<R*>(base + L->cp);
            K.x0p = reinterpret_cast<R*>(base + L->x0p);
        }
    }
    if (plan) {
        K.B = plan->B;
        K.tiles = plan->tiles;
    }
    K.has_c = P->c.ptr != nullptr;
    // p == 0 (no stage tracking cost) also takes the precomputed path
    K.cost_invariant = (P->p == 0) || (P->H.step_stride == 0 && P->X.step_stride == 0);
    K.dyn_invariant =
        P->F.step_stride == 0 && P->L.step_stride == 0 && P->U.step_stride == 0 ? 1 : 0;
    K.c_invariant = (P->c.ptr == nullptr || P->c.step_stride == 0) ? 1 : 0;
    K.out_mask = OUT_ALL;
    K.wait_limit = kWaitLimit;
    K.wait_probe = 0;
}

std::mutex g_prof_mu;
Prof g_prof;

lqt_status prof_begin(Prof** out) {
    *out = nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof.enabled) return LQT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LQT_ECUDA;
    if (g_prof.device != dev) {
        if (g_prof.device >= 0)
            for (cudaEvent_t& e : g_prof.ev)
                if (e) cudaEventDestroy(e), e = nullptr;
        for (cudaEvent_t& e : g_prof.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return LQT_ECUDA;
        g_prof.device = dev;
    }
    g_prof.count = 0;
    *out = &g_prof;
    return LQT_OK;
}

size_t input_elems(const lqt_in& in, int64_t per_step, int64_t T) {
    if (!in.ptr || T <= 0) return 0;
    if (in.step_stride == 0) return (size_t)per_step;
    return (size_t)((T - 1) * in.step_stride + per_step);
}

}  // namespace
}  // namespace lqt

using namespace lqt;

extern "C" {

const char* lqt_strerror(lqt_status s) {
    switch (s) {
        case LQT_OK: return "ok";
        case LQT_EINVAL: return "invalid argument";
        case LQT_ENOTSPD: return "L^T S L + U (or U) not positive definite";
        case LQT_ENONFINITE: return "non-finite value in the solution";
        case LQT_ENOMEM: return "workspace too small";
        case LQT_ECUDA: return "CUDA runtime error";
        case LQT_ETIMEOUT: return "bounded device wait ran out";
        case LQT_EUNSUPPORTED: return "no kernel compiled for this (n, m, dtype)";
        case LQT_ESINGULAR: return "I + C J numerically singular in a combine";
    }
    return "unknown status";
}

lqt_status lqt_plan(const lqt_problem* prob, const lqt_options* opts, int32_t* chunk_steps,
                    int32_t* tile_threads_out, int32_t* tiles, int32_t* kernels) {
    lqt_status st = validate(prob, nullptr);
    if (st != LQT_OK) return st;
    bool refine = false, newton = false, method2 = false;
    if ((st = resolve_refine(prob, opts, &refine, &newton, &method2)) != LQT_OK) return st;
    const Variant* var = find_variant(prob->dtype, prob->n, prob->m);
    bool unsupported = false;
    const bool chain = use_chain(prob, var, refine && newton, method2, &unsupported);
    if (unsupported) return LQT_EUNSUPPORTED;
    if (chain) {
        int NC = 0, nk = 0;
        long long B = 0;
        if ((st = chain_workspace(prob, refine, newton, false, method2, nullptr, &NC, &B, &nk)) !=
            LQT_OK)
            return st;
        if (B > INT32_MAX) return LQT_EINVAL;
        if (chunk_steps) *chunk_steps = (int32_t)B;
        if (tile_threads_out) *tile_threads_out = prob->n;
        if (tiles) *tiles = NC;
        if (kernels) *kernels = nk;
        return LQT_OK;
    }
    Plan plan;
    if ((st = make_plan(prob, *var, &plan)) != LQT_OK) return st;
    if (chunk_steps) *chunk_steps = plan.B;
    if (tile_threads_out) *tile_threads_out = plan.W;
    if (tiles) *tiles = plan.tiles;
    const int per_pass = plan.solo ? 1 : (plan.tiles > 0 ? 5 : 2);
    if (kernels) *kernels = (refine && prob->T > 0) ? 2 * per_pass : per_pass;
    return LQT_OK;
}

size_t lqt_workspace_bytes(const lqt_problem* prob, const lqt_options* opts) {
    if (validate(prob, nullptr) != LQT_OK) return 0;
    bool refine = false, newton = false, method2 = false;
    if (resolve_refine(prob, opts, &refine, &newton, &method2) != LQT_OK) return 0;
    const Variant* var = find_variant(prob->dtype, prob->n, prob->m);
    bool unsupported = false;
    const bool chain = use_chain(prob, var, refine && newton, method2, &unsupported);
    if (unsupported) return 0;
    if (chain) {
        size_t bytes = 0;
        if (chain_workspace(prob, refine, newton, false, method2, &bytes, nullptr, nullptr,
                            nullptr) != LQT_OK)
            return 0;
        return bytes;
    }
    Plan plan;
    if (make_plan(prob, *var, &plan) != LQT_OK) return 0;
    return layout(*var, plan, elem_bytes(prob->dtype), prob, refine).total;
}

}  // extern "C"

namespace lqt {
namespace {

// One pass of the parallel solve or of the sequential baseline.
template <typename R>
lqt_status run_pass(const Variant& var, const lqt_problem* P, const lqt_solution* sol,
                    void* ws, const Layout& L, const Plan& plan, int out_mask, int refine_emit,
                    int refine_add, bool sequential, int wait_probe, cudaStream_t s, Prof* prof,
                    cudaEvent_t bwd_done = nullptr) {
    Params<R> K;
    fill_params(K, P, sol, ws, &L, &plan);
    K.wait_probe = wait_probe;
    K.out_mask = out_mask;
    K.refine_emit = refine_emit;
    K.refine_add = refine_add;
    // the first pass of a refined solve records the top scan's maps, the
    // second (same matrices) replays them
    K.top_mode = K.top_fac ? (refine_add ? 2 : (refine_emit ? 1 : 0)) : 0;
    if (sequential) {
        if (prof) prof_mark(prof, s, refine_add ? "riccati_seq.refine" : "riccati_seq");
        return var.seq(&K, s);
    }
    return var.solve(&K, plan, s, prof, bwd_done);
}

template <typename R>
lqt_status run_solve(const Variant& var, const lqt_problem* P, const lqt_solution* sol,
                     void* ws, const Layout& L, const Plan& plan, bool refine, bool sequential,
                     int wait_probe, cudaStream_t s, Prof* prof, cudaEvent_t bwd_done) {
    refine = refine && P->T > 0;
    // pass 1: the problem; when refining it also writes the shifted data
    lqt_status st = run_pass<R>(var, P, sol, ws, L, plan, OUT_ALL, refine ? 1 : 0, 0, sequential,
                                wait_probe, s, prof, sequential ? nullptr : bwd_done);
    if (st != LQT_OK || !refine) {
        if (prof) prof_end(prof, s);
        return st;
    }
    // pass 2: the problem shifted by the first trajectory, x = x^ + xi, with
    // the same matrices, small references and offsets, and x'_0 = 0.  Its S
    // and K equal those of pass 1 bit for bit (they do not depend on r or c):
    // the pass does not write S, v, K again, reads K back, writes u* and adds
    // xi into x.
    char* base = static_cast<char*>(ws);
    lqt_problem P2 = *P;
    P2.r.ptr = P->p > 0 ? base + L.rp : nullptr;
    P2.r.step_stride = refine_r_stride(P->p);
    P2.c.ptr = base + L.cp;
    P2.c.step_stride = P->n;
    P2.rT = P->pT > 0 ? base + L.rTp : nullptr;
    P2.x0 = base + L.x0p;
    st = run_pass<R>(var, &P2, sol, ws, L, plan, 0, 0, 1, sequential, wait_probe, s, prof);
    if (prof) prof_end(prof, s);
    return st;
}

// bwd_done (may be null): recorded on the stream once S, v and K are final,
// where the path can tell (the thread-per-chunk kernels); *recorded says so.
lqt_status solve_common(const lqt_problem* prob, const lqt_solution* sol, const lqt_options* opts,
                        void* workspace, size_t workspace_bytes, void* stream, bool sequential,
                        cudaEvent_t bwd_done = nullptr, bool* recorded = nullptr) {
    if (recorded) *recorded = false;
    lqt_status st = validate(prob, sol);
    if (st != LQT_OK) return st;
    if (!workspace || !aligned(workspace, kAlign)) return LQT_EINVAL;
    bool refine = false, newton = false, method2 = false;
    if ((st = resolve_refine(prob, opts, &refine, &newton, &method2)) != LQT_OK) return st;
    if (sequential && prob->p > 64) return LQT_EUNSUPPORTED;
    const Variant* var = find_variant(prob->dtype, prob->n, prob->m);
    bool unsupported = false;
    const bool chain = use_chain(prob, var, refine && newton, method2, &unsupported);
    if (unsupported) return LQT_EUNSUPPORTED;
    // the diagnostic wait lives in the thread-per-chunk scan kernels
    const int wait_probe = opts ? opts->wait_probe_polls : 0;
    if (wait_probe > 0 && (chain || sequential)) return LQT_EUNSUPPORTED;
    if (chain) {
        // the chunked pipeline (one chunk when sequential)
        size_t need = 0;
        if ((st = chain_workspace(prob, refine, newton, sequential, method2, &need, nullptr,
                                  nullptr, nullptr)) != LQT_OK)
            return st;
        if (workspace_bytes < need) return LQT_ENOMEM;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (cudaMemsetAsync(workspace, 0, sizeof(int), s) != cudaSuccess) return LQT_ECUDA;
        Prof* prof = nullptr;
        if ((st = prof_begin(&prof)) != LQT_OK) return st;
        return chain_solve(prob, sol, refine, newton, sequential, method2, workspace,
                           workspace_bytes, s, prof);
    }
    Plan plan;
    if ((st = make_plan(prob, *var, &plan)) != LQT_OK) return st;
    const Layout L = layout(*var, plan, elem_bytes(prob->dtype), prob, refine);
    if (workspace_bytes < L.total) return LQT_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(workspace, 0, sizeof(int), s) != cudaSuccess) return LQT_ECUDA;
    Prof* prof = nullptr;
    if ((st = prof_begin(&prof)) != LQT_OK) return st;
    if (recorded) *recorded = bwd_done != nullptr && !sequential;
    if (prob->dtype == LQT_F64)
        return run_solve<double>(*var, prob, sol, workspace, L, plan, refine, sequential,
                                 wait_probe, s, prof, bwd_done);
    return run_solve<float>(*var, prob, sol, workspace, L, plan, refine, sequential, wait_probe, s,
                            prof, bwd_done);
}

}  // namespace
}  // namespace lqt

extern "C" {

lqt_status lqt_solve(const lqt_problem* prob, const lqt_solution* sol, const lqt_options* opts,
                     void* workspace, size_t workspace_bytes, void* stream) {
    return solve_common(prob, sol, opts, workspace, workspace_bytes, stream, false);
}

lqt_status lqt_set_single_tile_chunk(int32_t max_chunk_steps, int32_t* previous) {
    if (max_chunk_steps < 0) return LQT_EINVAL;
    const int old = lqt::g_single_tile_chunk.exchange(max_chunk_steps);
    if (previous) *previous = old;
    return LQT_OK;
}

lqt_status lqt_riccati_sequential(const lqt_problem* prob, const lqt_solution* sol,
                                  const lqt_options* opts, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    return solve_common(prob, sol, opts, workspace, workspace_bytes, stream, true);
}

lqt_status lqt_workspace_status(const void* workspace, void* stream) {
    if (!workspace) return LQT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    if (cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LQT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LQT_ECUDA;
    return static_cast<lqt_status>(h);
}

lqt_status lqt_profile_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.enabled = enable != 0;
    g_prof.count = 0;
    return LQT_OK;
}

int lqt_profile_read(float* ms, const char** names, int max_entries) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof.enabled || g_prof.count == 0) return 0;
    if (cudaEventSynchronize(g_prof.ev[g_prof.count]) != cudaSuccess) return -1;
    for (int i = 0; i < g_prof.count && i < max_entries; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_prof.ev[i], g_prof.ev[i + 1]) != cudaSuccess) return -1;
        if (ms) ms[i] = t;
        if (names) names[i] = g_prof.names[i];
    }
    return g_prof.count;
}

}  // extern "C"

namespace lqt {
namespace {

// Per host thread and device: a non-blocking stream and two events with which
// lqt_solve_host copies S, v and K back while the rest of the solve runs.
// Per host thread and device: the stream that copies S, v, K back early and
// its two events.  Created on first use and deliberately never destroyed: a
// thread_local destructor can run after the CUDA runtime has shut down at
// process exit.
struct HostAux {
    cudaStream_t s = nullptr;
    cudaEvent_t bwd = nullptr, done = nullptr;
};

HostAux* host_aux() {
    thread_local HostAux aux[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    HostAux& a = aux[dev];
    if (!a.s) {
        cudaStream_t s = nullptr;
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) {
            if (e1) cudaEventDestroy(e1);
            cudaStreamDestroy(s);
            return nullptr;
        }
        a.s = s;
        a.bwd = e1;
        a.done = e2;
    }
    return &a;
}

}  // namespace
}  // namespace lqt

extern "C" {

size_t lqt_host_solve_bytes(const lqt_problem* prob, const lqt_options* opts) {
    if (validate(prob, nullptr) != LQT_OK) return 0;
    const size_t es = elem_bytes(prob->dtype);
    const int64_t n = prob->n, m = prob->m, p = prob->p, pT = prob->pT, T = prob->T;
    size_t total = lqt_workspace_bytes(prob, opts);
    if (total == 0) return 0;
    const size_t in_elems[] = {input_elems(prob->F, n * n, T), input_elems(prob->c, n, T),
                               input_elems(prob->L, n * m, T), input_elems(prob->U, m * m, T),
                               input_elems(prob->H, p * n, T), input_elems(prob->r, p, T),
                               input_elems(prob->X, p * p, T)};
    for (size_t e : in_elems) total += align_up(e * es);
    total += align_up((size_t)pT * n * es) + align_up((size_t)pT * es) +
             align_up((size_t)pT * pT * es) + align_up((size_t)n * es);
    total += align_up((size_t)(T + 1) * n * n * es) + align_up((size_t)(T + 1) * n * es) +
             align_up((size_t)T * m * n * es) + align_up((size_t)(T + 1) * n * es) +
             align_up((size_t)T * m * es);
    return total;
}

lqt_status lqt_solve_host(const lqt_problem* hp, const lqt_solution* hs, const lqt_options* opts,
                          void* device_buffer, size_t device_bytes, void* stream) {
    lqt_status st = validate(hp, hs);
    if (st != LQT_OK) return st;
    if (!device_buffer || !aligned(device_buffer, kAlign)) return LQT_EINVAL;
    const size_t need = lqt_host_solve_bytes(hp, opts);
    if (need == 0)
        return find_variant(hp->dtype, hp->n, hp->m) || chain_supported(hp->dtype, hp->n, hp->m)
                   ? LQT_EINVAL
                   : LQT_EUNSUPPORTED;
    if (device_bytes < need) return LQT_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = elem_bytes(hp->dtype);
    const int64_t n = hp->n, m = hp->m, p = hp->p, pT = hp->pT, T = hp->T;
    char* base = static_cast<char*>(device_buffer);
    const size_t ws_bytes = lqt_workspace_bytes(hp, opts);
    void* ws = base;
    size_t off = ws_bytes;
    auto put = [&](const void* src, size_t elems) -> const void* {
        if (!src) return nullptr;
        char* dst = base + off;
        off += align_up(elems * es);
        if (elems && cudaMemcpyAsync(dst, src, elems * es, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return reinterpret_cast<const void*>(-1);
        return dst;
    };
    lqt_problem dp = *hp;
    const void* bad = reinterpret_cast<const void*>(-1);
    struct Cp {
        const lqt_in* src;
        lqt_in* dst;
        int64_t size;
    } cps[] = {{&hp->F, &dp.F, n * n}, {&hp->c, &dp.c, n},     {&hp->L, &dp.L, n * m},
               {&hp->U, &dp.U, m * m}, {&hp->H, &dp.H, p * n}, {&hp->r, &dp.r, p},
               {&hp->X, &dp.X, p * p}};
    for (const Cp& c : cps) {
        c.dst->ptr = put(c.src->ptr, input_elems(*c.src, c.size, T));
        if (c.dst->ptr == bad) return LQT_ECUDA;
    }
    if ((dp.HT = put(hp->HT, (size_t)pT * n)) == bad) return LQT_ECUDA;
    if ((dp.rT = put(hp->rT, (size_t)pT)) == bad) return LQT_ECUDA;
    if ((dp.XT = put(hp->XT, (size_t)pT * pT)) == bad) return LQT_ECUDA;
    if ((dp.x0 = put(hp->x0, (size_t)n)) == bad) return LQT_ECUDA;
    lqt_solution ds;
    const size_t sizes[] = {(size_t)(T + 1) * n * n, (size_t)(T + 1) * n, (size_t)T * m * n,
                            (size_t)(T + 1) * n, (size_t)T * m};
    void** douts[] = {&ds.S, &ds.v, &ds.K, &ds.x, &ds.u};
    void* houts[] = {hs->S, hs->v, hs->K, hs->x, hs->u};
    for (int i = 0; i < 5; ++i) {
        *douts[i] = base + off;
        off += align_up(sizes[i] * es);
    }
    // S, v, K are final once the first pass's backward kernels end: where the
    // path records that point, they go back on the auxiliary stream while the
    // forward scan and the refinement pass run (the host link, not the copy
    // engines, is the limit, so one stream carries them)
    HostAux* aux = host_aux();
    bool recorded = false;
    st = solve_common(&dp, &ds, opts, ws, ws_bytes, stream, false, aux ? aux->bwd : nullptr,
                      &recorded);
    if (st != LQT_OK) return st;
    int first = 0;
    if (aux && recorded) {
        if (cudaStreamWaitEvent(aux->s, aux->bwd, 0) != cudaSuccess) return LQT_ECUDA;
        for (int i = 0; i < 3; ++i)
            if (sizes[i] && houts[i] &&
                cudaMemcpyAsync(houts[i], *douts[i], sizes[i] * es, cudaMemcpyDeviceToHost,
                                aux->s) != cudaSuccess)
                return LQT_ECUDA;
        if (cudaEventRecord(aux->done, aux->s) != cudaSuccess ||
            cudaStreamWaitEvent(s, aux->done, 0) != cudaSuccess)
            return LQT_ECUDA;
        first = 3;
    }
    for (int i = first; i < 5; ++i)
        if (sizes[i] && houts[i] &&
            cudaMemcpyAsync(houts[i], *douts[i], sizes[i] * es, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
            return LQT_ECUDA;
    return lqt_workspace_status(ws, stream);
}

}  // extern "C"
