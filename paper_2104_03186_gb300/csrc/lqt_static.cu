// lqt_solve_static: the parallel solve with its scratch space in one array
// compiled into the library, for callers that cannot allocate device memory
// (see include/lqt.h).  It reuses lqt_solve unchanged and only supplies the
// array as the workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "lqt.h"

namespace {

// The scratch array.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_static_scratch[LQT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];  // device address of g_static_scratch, per device

// Host code cannot use g_static_scratch as a pointer (on the host the name is
// only a stand-in for the symbol): ask the runtime for its address on the
// current device, once per device.  The kept address is that of the device's
// current context; a device reset reloads the module, after which it may be
// stale (the header tells callers not to use this entry point after one).
lqt_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LQT_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return LQT_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LQT_OK;
}

}  // namespace

extern "C" lqt_status lqt_solve_static(const lqt_problem* prob, const lqt_solution* sol,
                                       const lqt_options* opts, void* stream) {
    const size_t need = lqt_workspace_bytes(prob, opts);
    if (need == 0) {
        // same diagnosis as lqt_solve for invalid or unsupported problems
        return lqt_solve(prob, sol, opts, nullptr, 0, stream);
    }
    if (need > LQT_STATIC_SCRATCH_BYTES) return LQT_ENOMEM;
    void* ws = nullptr;
    lqt_status st = scratch_address(&ws);
    if (st != LQT_OK) return st;
    // lqt_solve clears the status word at the start of the array; every other
    // region it uses is written before it is read within the same solve.
    st = lqt_solve(prob, sol, opts, ws, LQT_STATIC_SCRATCH_BYTES, stream);
    if (st != LQT_OK) return st;
    return lqt_workspace_status(ws, stream);
}
