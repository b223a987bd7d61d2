// qs_stats_device.cuh -- device helpers of the output statistics: the
// per-element terms of the Porter-Thomas statistics and the fixed-order
// block reduction, shared by the single-state read-out, the batched
// statistics kernels and the persistent ensemble kernel.
#pragma once

#include "qs_device.cuh"

namespace qs {

constexpr int kStatThreads = 256;
constexpr int kStatAcc = 12;   // sum y, sum y ln y, sum ln y, sum y^k (k=2..10)

// ---------------------------------------------------------------------------
// block reduction helpers (fixed order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums acc over the block's kStatThreads threads (warp shuffles, then the
// warps' sums in warp order) and stores the K sums at dst (threads < K).
template <int K>
__device__ __forceinline__ void block_sum_store(double (&acc)[K], double *dst)
{
    __shared__ double red[kStatThreads / 32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0;
        for (int w = 0; w < kStatThreads / 32; ++w) s += red[w][threadIdx.x];
        dst[threadIdx.x] = s;
    }
}

// Accumulates one element's contributions.  y = N p.
template <typename T>
__device__ __forceinline__ void stat_terms(T y, T (&c)[kStatAcc])
{
    T ly = (sizeof(T) == 4) ? (T)__logf((float)y) : (T)log((double)y);
    c[0] += y;
    c[1] += (y > (T)0) ? y * ly : (T)0;
    c[2] += ly;
    T yk = y;
#pragma unroll
    for (int k = 2; k <= 10; ++k) {
        yk *= y;
        c[k + 1] += yk;
    }
}

// Statistics partials of one chunk of a complex64 state (cnt amplitudes at
// a, cnt even, a 16-byte aligned; scaleN = N of the instance): each thread
// takes 16-byte pairs of amplitudes blockDim.x apart, eight loads in flight
// at a time, and sums the terms of 64 amplitudes in FP32 before adding them
// into FP64 accumulators (terms of y = N p > 4096 formed in FP64); then the
// block's fixed-order sum goes to dst[0 .. kStatAcc).  The whole block
// (kStatThreads threads) calls it.  Amplitudes are read through L2
// (ld.global.cg), so the chunk may have been written earlier in the same
// launch by another CTA (after an acquire of that CTA's release).
__device__ __forceinline__ void batch_stats_chunk(const float2 *a, uint64_t cnt, float scaleN, double *dst)
{
    constexpr int kLoads = 8;                      // 16-byte loads in flight per thread
    constexpr int kGroup = 32;                     // pairs per FP32 partial (64 amplitudes)
    const float4 *a4 = reinterpret_cast<const float4 *>(a);
    const uint64_t units = cnt / 2, bd = blockDim.x;
    double acc[kStatAcc];
#pragma unroll
    for (int k = 0; k < kStatAcc; ++k) acc[k] = 0;
    for (uint64_t u0 = threadIdx.x; u0 < units; u0 += bd * kGroup) {
        float c[kStatAcc];
#pragma unroll
        for (int k = 0; k < kStatAcc; ++k) c[k] = 0.f;
        double big[kStatAcc];
        bool any_big = false;
        for (int j0 = 0; j0 < kGroup; j0 += kLoads) {
            float4 v[kLoads];
#pragma unroll
            for (int k = 0; k < kLoads; ++k) {
                const uint64_t u = u0 + (uint64_t)(j0 + k) * bd;
                v[k] = u < units ? __ldcg(a4 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kLoads; ++k) {
                if (u0 + (uint64_t)(j0 + k) * bd >= units) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float re = h ? v[k].z : v[k].x, im = h ? v[k].w : v[k].y;
                    const float y = (re * re + im * im) * scaleN;
                    if (y > 4096.f) {
                        if (!any_big) {
#pragma unroll
                            for (int q = 0; q < kStatAcc; ++q) big[q] = 0;
                            any_big = true;
                        }
                        stat_terms<double>(((double)re * re + (double)im * im) * (double)scaleN, big);
                    } else {
                        stat_terms<float>(y, c);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kStatAcc; ++k) acc[k] += (double)c[k];
        if (any_big) {
#pragma unroll
            for (int k = 0; k < kStatAcc; ++k) acc[k] += big[k];
        }
    }
    block_sum_store<kStatAcc>(acc, dst);
}

}  // namespace qs
