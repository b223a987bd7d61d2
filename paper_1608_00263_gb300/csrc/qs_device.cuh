// qs_device.cuh -- device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace qs {

template <typename R> struct V2T;
template <> struct V2T<float> { using T = float2; };
template <> struct V2T<double> { using T = double2; };

template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Inserts a zero bit at position q of j.
__device__ __forceinline__ uint64_t insert_zero(uint64_t j, int q)
{
    uint64_t lo = j & ((1ULL << q) - 1);
    return ((j >> q) << (q + 1)) | lo;
}

// Waits for the phase `parity` of the shared-memory mbarrier at `mbar`
// (shared address) to complete, for at most `limit_ns` nanoseconds of the
// global timer (and at most `max_iter` polls, should the timer not advance).
// Returns whether the phase completed; never blocks longer.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, uint64_t limit_ns,
                                                  uint32_t max_iter = 1u << 26)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= limit_ns) return false;
    }
    return false;
}

// Acquire load of a global counter at GPU scope: writes released before the
// increments it observes are visible to this thread's later loads.
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits until the counter *count reaches `target` (acquire), for at most
// `limit_ns` nanoseconds of the global timer and `max_iter` polls.  Gives
// up early when *abort becomes nonzero (another CTA's wait ran out).
// Returns 0 when the target was reached, 1 when the limit ran out, 2 on
// abort; never blocks longer.
__device__ __forceinline__ int flag_wait_bounded(const unsigned int *count, unsigned int target,
                                                 const unsigned int *abort, uint64_t limit_ns,
                                                 uint32_t max_iter = 1u << 24)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t it = 0; it < max_iter; ++it) {
        if (ld_acquire_gpu(count) >= target) return 0;
        if (*(volatile const unsigned int *)abort) return 2;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= limit_ns) return 1;
        __nanosleep(128);
    }
    return 1;
}

// ---------------------------------------------------------------------------
// Checked build (QS_CHECKED): device-side index checks.  A failed check
// records its site code in this translation unit's check word (the first
// failure wins) and evaluates to false, so the guarded access is skipped --
// no out-of-range access, no trap.  The host turns a nonzero word into
// QS_ERR_INVALID_ARG (check_poll_all, after every public call that
// launches work).  In the normal build every check is `true` and compiles
// away.
// ---------------------------------------------------------------------------
#ifdef QS_CHECKED
static __device__ unsigned int g_qs_check_word;
__device__ __forceinline__ bool qs_dcheck_fail(unsigned int site)
{
    atomicCAS(&g_qs_check_word, 0u, site);
    return false;
}
#define QS_DCHECK(cond, site) ((cond) ? true : qs_dcheck_fail(site))
// Host reader of this translation unit's check word: returns
// QS_ERR_INVALID_ARG naming the site and clears the word if it is set.
#define QS_CHECK_READER(fn)                                                                 \
    qs_status fn()                                                                          \
    {                                                                                       \
        unsigned int w = 0;                                                                 \
        cudaError_t e = cudaMemcpyFromSymbol(&w, g_qs_check_word, sizeof w);               \
        if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "check word: %s", cudaGetErrorString(e)); \
        if (!w) return QS_OK;                                                               \
        const unsigned int z = 0;                                                           \
        cudaMemcpyToSymbol(g_qs_check_word, &z, sizeof z);                                  \
        return set_error(QS_ERR_INVALID_ARG, "device index check failed at site %u", w);   \
    }
#else
#define QS_DCHECK(cond, site) true
#define QS_CHECK_READER(fn) \
    qs_status fn() { return QS_OK; }
#endif

#define QS_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess)                                                   \
            return set_error(QS_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,       \
                             cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

#define QS_LAUNCH_CHECK()                                                        \
    do {                                                                         \
        cudaError_t e_ = cudaGetLastError();                                     \
        if (e_ != cudaSuccess)                                                   \
            return set_error(QS_ERR_CUDA, "kernel launch failed: %s (%s:%d)",   \
                             cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

inline int grid_for(uint64_t work, int threads, int num_sms, int per_sm = 8)
{
    uint64_t b = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace qs
