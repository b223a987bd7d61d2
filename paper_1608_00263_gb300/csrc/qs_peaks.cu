// qs_peaks.cu -- arithmetic-rate probe (measurement support, no part of the
// paper's method).
//
// The state-vector passes move 16 bytes per amplitude, but the fused pass
// also does tens of floating-point operations per amplitude, so its bound
// can be the arithmetic pipes rather than HBM.  This probe measures the rate
// of fused multiply-adds this GPU sustains on long independent chains:
// scalar FP32, packed FP32x2 (the sm_100+ instructions the fused pass uses
// for its butterflies) and FP64 (the complex128 path).  The rate is a
// denominator for the roofline of ALU-bound kernels.
#include <cuda_runtime.h>

#include "qs_device.cuh"

namespace qs {
namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_rate(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_ffma2_rate(float *out, int iters, float a, float b)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_alu_rate(int kind, void *cuda_stream, double *fma_per_s)
{
    clear_error();
    if (!fma_per_s) return set_error(QS_ERR_INVALID_ARG, "fma_per_s is NULL");
    if (kind < 0 || kind > 2) return set_error(QS_ERR_INVALID_ARG, "kind %d not in 0..2", kind);
    int dev = 0, sms = 1;
    QS_CUDA_TRY(cudaGetDevice(&dev));
    QS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * 8;         // 64 warps per SM
    const int iters = kind == 2 ? 64 : 4096;
    void *buf = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&buf, (size_t)blocks * kPeakThreads * sizeof(double), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qs_status rc = QS_OK;
    float ms = 0;
    auto launch = [&]() {
        if (kind == 0)
            k_fma_rate<float><<<blocks, kPeakThreads, 0, st>>>((float *)buf, iters, 0.999f, 1e-3f);
        else if (kind == 1)
            k_ffma2_rate<<<blocks, kPeakThreads, 0, st>>>((float *)buf, iters, 0.999f, 1e-3f);
        else
            k_fma_rate<double><<<blocks, kPeakThreads, 0, st>>>((double *)buf, iters, 0.999, 1e-3);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = set_error(QS_ERR_CUDA, "event creation failed");
    } else {
        launch();                        // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) launch();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = set_error(QS_ERR_CUDA, "rate probe failed");
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    if (rc) return rc;
    // lanes x chains x unroll x iterations x launches; FP32x2 counts two
    // FMAs per instruction lane
    const double fmas = (double)blocks * kPeakThreads * kChains * 4.0 * iters * 5.0 * (kind == 1 ? 2.0 : 1.0);
    *fma_per_s = fmas / (ms * 1e-3);
    return QS_OK;
}
