// Bulk (TMA) copies between global and shared memory with an mbarrier, and
// warp-cooperative transposed copies of per-step records.
//
// Every wait is bounded: when a copy does not complete within the limit the
// kernel records LQT_ETIMEOUT in the status word, waits once more (bounded)
// and carries on; its results are then flagged as invalid by the status.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lqt {

constexpr long long kWaitLimit = 1LL << 24;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// true when the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait of at most `limit` polls; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitLimit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// global -> shared bulk copy completing on `bar` (bytes: multiple of 16,
// both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// shared -> global bulk copy in the calling thread's bulk group
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// wait until the committed bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// wait until the committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// make generic-proxy shared-memory writes visible to the async proxy
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Load `bytes` (multiple of 16) from global into shared memory with one bulk
// copy issued by thread 0; every thread of the CTA waits.  Returns false on a
// wait timeout.  `bar` must be initialised with count 1; `phase` is its
// current parity and is flipped.
__device__ __forceinline__ bool cta_bulk_load(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint32_t& phase,
                                              long long limit = kWaitLimit) {
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, src, bytes, bar);
    }
    bool ok = mbar_wait(bar, phase, limit);
    if (!ok) mbar_wait(bar, phase, limit);  // give the copy in flight one more bounded wait
    phase ^= 1u;
    return ok;
}

// Store `bytes` (multiple of 16) from shared memory to global with one bulk
// copy issued by thread 0 after a CTA barrier.  Thread 0 waits until the copy
// has completed; callers must not overwrite the source before the next
// __syncthreads that follows this call.
__device__ __forceinline__ void cta_bulk_store(void* dst, const void* src, uint32_t bytes) {
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_s2g(dst, src, bytes);
        bulk_commit();
        bulk_wait_all();
    }
}

// Ampere-style asynchronous copies (global -> shared, 4/8/16 bytes per thread)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src_gmem) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst_smem)),
                 "l"(src_gmem), "n"(BYTES)
                 : "memory");
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may be scheduled while its predecessor in
// the stream still runs; griddep_wait() returns once the predecessor grid has
// completed and its memory operations are visible (at once when there is no
// such predecessor).  griddep_launch_dependents() lets the next kernel be
// scheduled; the kernels call it on entry and wait before any global access.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// 16-byte asynchronous copy that bypasses L1 (cached in L2 only): for
// streaming records that no thread reads twice, so that they do not evict the
// lines of other loads.
__device__ __forceinline__ void cp_async_cg16(void* dst_smem, const void* src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)),
                 "l"(src_gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// wait until at most PENDING of this thread's committed groups are in flight
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// ---------------------------------------------------------------------------
// Warp-cooperative transposed copies of per-step records.
//
// Lane r of a warp owns `cnt_r` consecutive steps starting at `base + lo_r` of
// an array whose record for step k is X[k * WX .. k * WX + WX) (dense; array
// base 16-byte aligned).  In shared memory the warp keeps one row per lane;
// lane r's records sit at row_r[(k - base - lo_r) * WX + c].  A copy moves all
// 32 rows with vector accesses spread over the lanes, so that consecutive lanes
// touch consecutive global addresses.  Every lane passes its own (lo, cnt); the
// others' are fetched with shuffles.
// ---------------------------------------------------------------------------
template <typename R, int WX, int G>
struct WarpRows {
    static constexpr int SPAN = G * WX;  // elements per lane row
    static constexpr int VEC =
        sizeof(R) == 4 ? (WX % 4 == 0 ? 4 : (WX % 2 == 0 ? 2 : 1)) : (WX % 2 == 0 ? 2 : 1);
    static constexpr int NV = SPAN / VEC;  // vectors per row

    __device__ static void copy_vec(R* dst, const R* src) {
        if constexpr (VEC == 4 && sizeof(R) == 4) {
            *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
        } else if constexpr (VEC == 2 && sizeof(R) == 4) {
            *reinterpret_cast<float2*>(dst) = *reinterpret_cast<const float2*>(src);
        } else if constexpr (VEC == 2 && sizeof(R) == 8) {
            *reinterpret_cast<double2*>(dst) = *reinterpret_cast<const double2*>(src);
        } else {
            *dst = *src;
        }
    }

    // shared rows -> global
    __device__ static void store(R* gX, long long base, const R* rows, int rowstride, int lo,
                                 int cnt) {
        const int lane = threadIdx.x & 31;
        R* g = gX + base * WX;
#pragma unroll
        for (int it = 0; it < NV; ++it) {
            const int f = it * 32 + lane;
            const int r = f / NV, v = f % NV;
            const int lo_r = __shfl_sync(0xffffffffu, lo, r);
            const int cnt_r = __shfl_sync(0xffffffffu, cnt, r);
            if (v * VEC < cnt_r * WX)
                copy_vec(g + (long long)lo_r * WX + v * VEC, rows + r * rowstride + v * VEC);
        }
    }

    // global -> shared rows, asynchronously (complete with cp_async_wait + __syncwarp)
    __device__ static void load_async(const R* gX, long long base, R* rows, int rowstride, int lo,
                                      int cnt) {
        const int lane = threadIdx.x & 31;
        const R* g = gX + base * WX;
#pragma unroll
        for (int it = 0; it < NV; ++it) {
            const int f = it * 32 + lane;
            const int r = f / NV, v = f % NV;
            const int lo_r = __shfl_sync(0xffffffffu, lo, r);
            const int cnt_r = __shfl_sync(0xffffffffu, cnt, r);
            if (v * VEC < cnt_r * WX)
                cp_async<VEC * (int)sizeof(R)>(rows + r * rowstride + v * VEC,
                                               g + (long long)lo_r * WX + v * VEC);
        }
    }

    // global -> shared rows, asynchronously and bypassing L1 where the vectors
    // are 16 bytes (streaming records)
    __device__ static void load_async_stream(const R* gX, long long base, R* rows, int rowstride,
                                             int lo, int cnt) {
        const int lane = threadIdx.x & 31;
        const R* g = gX + base * WX;
#pragma unroll
        for (int it = 0; it < NV; ++it) {
            const int f = it * 32 + lane;
            const int r = f / NV, v = f % NV;
            const int lo_r = __shfl_sync(0xffffffffu, lo, r);
            const int cnt_r = __shfl_sync(0xffffffffu, cnt, r);
            if (v * VEC < cnt_r * WX) {
                if constexpr (VEC * sizeof(R) == 16)
                    cp_async_cg16(rows + r * rowstride + v * VEC, g + (long long)lo_r * WX + v * VEC);
                else
                    cp_async<VEC * (int)sizeof(R)>(rows + r * rowstride + v * VEC,
                                                   g + (long long)lo_r * WX + v * VEC);
            }
        }
    }

    // global -> shared rows
    __device__ static void load(const R* gX, long long base, R* rows, int rowstride, int lo,
                                int cnt) {
        const int lane = threadIdx.x & 31;
        const R* g = gX + base * WX;
#pragma unroll
        for (int it = 0; it < NV; ++it) {
            const int f = it * 32 + lane;
            const int r = f / NV, v = f % NV;
            const int lo_r = __shfl_sync(0xffffffffu, lo, r);
            const int cnt_r = __shfl_sync(0xffffffffu, cnt, r);
            if (v * VEC < cnt_r * WX)
                copy_vec(rows + r * rowstride + v * VEC, g + (long long)lo_r * WX + v * VEC);
        }
    }
};

__host__ __device__ constexpr int round4(int x) { return (x + 3) / 4 * 4; }

}  // namespace lqt
