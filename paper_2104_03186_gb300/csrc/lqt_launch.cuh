// Launch plan and per-instantiation launchers shared by the C ABI and the
// translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>

#include "lqt.h"

namespace lqt {

template <typename R>
struct Params;

// Threads of the single-CTA top-level scans.
constexpr int top_threads() { return 256; }

struct Plan {
    int B;      // steps per chunk (one thread)
    int W;      // chunks per tile (one CTA)
    int tiles;  // CTAs of the per-tile kernels
    int TP;     // threads of the top-level scans
    int solo;   // 1: a single tile, each pass one launch of k_solo
};

// Kernel timing (lqt_profile_enable); owned by the C ABI.
struct Prof {
    static constexpr int MAXK = 32;
    bool enabled = false;
    int device = -1;
    int count = 0;
    cudaEvent_t ev[MAXK + 1] = {};
    const char* names[MAXK] = {};
};

// Record the start event of the next kernel / the end event of the last one.
inline void prof_mark(Prof* prof, cudaStream_t stream, const char* name) {
    if (!prof || !prof->enabled || prof->count >= Prof::MAXK) return;
    cudaEventRecord(prof->ev[prof->count], stream);
    prof->names[prof->count] = name;
    prof->count += 1;
}

inline void prof_end(Prof* prof, cudaStream_t stream) {
    if (!prof || !prof->enabled) return;
    cudaEventRecord(prof->ev[prof->count], stream);
}

template <typename R, int N, int M>
// bwd_done (may be null) is recorded on the stream once the first pass has
// written S, v and K.
lqt_status launch_solve(const Params<R>& P, const Plan& plan, cudaStream_t stream, Prof* prof,
                        cudaEvent_t bwd_done = nullptr);

template <typename R, int N, int M>
lqt_status launch_seq(const Params<R>& P, cudaStream_t stream);

}  // namespace lqt
