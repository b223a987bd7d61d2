// qs_stats.cu -- output probabilities, Porter-Thomas statistics, inverse-CDF
// sampler and sample cross entropy.
//
//   probabilities  p_U(x) = |<x|psi>|^2                     (Sec. cqs)
//   statistics     S = sum p, and for p/S: -sum p ln p (Eq. lps, eu),
//                  -(1/N) sum ln p (Eq. eue), N^{k-1} sum p^k (normalised
//                  IPR, Sec. "Convergence to Porter-Thomas")
//   sampler        x_j = min{x : C_x > u_j C_{N-1}}, C = cumulative p
//   cross entropy  (1/m) sum_j ln(1/p(x_j)) and Delta H (Eq. ae)
//
// Reductions read the state once.  Per element the complex64 path works in
// FP32 on y = N p (O(1) for Porter-Thomas states), accumulates FP32 partial
// sums over 128 elements and adds those into FP64 accumulators; the
// complex128 path is FP64 throughout.  Block partials are combined in a
// fixed order, so results are deterministic.
//
// The sampler never materialises a 2^n array: it keeps one FP64 sum per
// 256-amplitude chunk (N/32 bytes), scans those, and for each sample
// rescans one chunk with exactly the arithmetic that produced the chunk's
// sum.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_device.cuh"
#include "qs_stats_device.cuh"

namespace qs {

constexpr int kChunk = 256;    // sampler chunk (amplitudes)

// ---------------------------------------------------------------------------
// probabilities
// ---------------------------------------------------------------------------
// FP32 -> FP64 by integer operations (exact): this GPU's FP64 pipe is
// narrow, and one conversion per amplitude would bound the pass.  Zero and
// normal values take the integer path; subnormals (and inf / nan) the
// hardware conversion.
__device__ __forceinline__ double widen_f32(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if ((b & 0x7FFFFFFFu) == 0) return 0.0;
    if (e == 0 || e == 0xFFu) return (double)f;
    const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                       ((uint64_t)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// |psi|^2 of a complex64 amplitude: formed in FP32 (one FMA), the state's
// own precision, then widened exactly when the output is FP64.
__device__ __forceinline__ float prob32(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

template <typename R, typename O>
__global__ void k_probs(const typename V2T<R>::T *__restrict__ a, O *__restrict__ out,
                        uint64_t first, uint64_t count)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        auto v = a[first + i];
        if constexpr (sizeof(R) == 4) {
            const float p = prob32(v);
            if constexpr (sizeof(O) == 8) out[i] = widen_f32(p);
            else out[i] = p;
        } else {
            out[i] = (O)(v.x * v.x + v.y * v.y);
        }
    }
}

// complex64, two amplitudes per thread and step (16-byte loads, 8- or
// 16-byte stores); the same values as k_probs.
template <typename O>
__global__ void k_probs_c64x2(const float4 *__restrict__ a2, O *__restrict__ out, uint64_t first2,
                              uint64_t count2)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count2; i += stride) {
        const float4 v = a2[first2 + i];
        const float p0 = prob32(make_float2(v.x, v.y)), p1 = prob32(make_float2(v.z, v.w));
        if constexpr (sizeof(O) == 8)
            reinterpret_cast<double2 *>(out)[i] = make_double2(widen_f32(p0), widen_f32(p1));
        else
            reinterpret_cast<float2 *>(out)[i] = make_float2(p0, p1);
    }
}

qs_status launch_probabilities(const qs_state *s, void *out, int fp64, uint64_t first,
                               uint64_t count)
{
    const int th = 256;
    if (s->dt == QS_C64 && first == 0 && count == (1ULL << s->n) && !((uintptr_t)out & 15))
        return readout_c64(s, out, fp64 ? 2 : 1);
    if (s->dt == QS_C64) {
        const bool pairs = !(first & 1) && !(count & 1) && !((uintptr_t)out & (fp64 ? 15 : 7));
        if (pairs) {
            const int grid = grid_for(count / 2, th, s->num_sms, 32);
            if (fp64)
                k_probs_c64x2<double><<<grid, th, 0, s->stream>>>((const float4 *)s->amps, (double *)out, first / 2,
                                                                  count / 2);
            else
                k_probs_c64x2<float><<<grid, th, 0, s->stream>>>((const float4 *)s->amps, (float *)out, first / 2,
                                                                 count / 2);
        } else {
            const int grid = grid_for(count, th, s->num_sms, 32);
            if (fp64) k_probs<float, double><<<grid, th, 0, s->stream>>>((const float2 *)s->amps, (double *)out, first, count);
            else k_probs<float, float><<<grid, th, 0, s->stream>>>((const float2 *)s->amps, (float *)out, first, count);
        }
    } else {
        const int grid = grid_for(count, th, s->num_sms, 16);
        if (fp64) k_probs<double, double><<<grid, th, 0, s->stream>>>((const double2 *)s->amps, (double *)out, first, count);
        else k_probs<double, float><<<grid, th, 0, s->stream>>>((const double2 *)s->amps, (float *)out, first, count);
    }
    QS_LAUNCH_CHECK();
    return QS_OK;
}

// The same for two probabilities already formed in FP32 (the second one
// only if `two`).  Beyond the FP32 range of y^10 the terms are formed from
// the FP32 probability in FP64.
__device__ __forceinline__ void stat_pair_p(float p0, float p1, bool two, float scaleN, float (&c)[kStatAcc],
                                            double (&acc)[kStatAcc])
{
    const float y0 = p0 * scaleN, y1 = two ? p1 * scaleN : 0.f;
    if (y0 > 4096.f || y1 > 4096.f) {
        stat_terms<double>((double)p0 * (double)scaleN, acc);
        if (two) stat_terms<double>((double)p1 * (double)scaleN, acc);
    } else {
        stat_terms<float>(y0, c);
        if (two) stat_terms<float>(y1, c);
    }
}

__global__ void __launch_bounds__(kStatThreads)
k_stats_c128(const double2 *__restrict__ a, uint64_t N, double scaleN, double *__restrict__ part)
{
    double acc[kStatAcc];
#pragma unroll
    for (int k = 0; k < kStatAcc; ++k) acc[k] = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double2 v = a[i];
        stat_terms<double>((v.x * v.x + v.y * v.y) * scaleN, acc);
    }
    block_sum_store<kStatAcc>(acc, part + (size_t)blockIdx.x * kStatAcc);
}

// Final fixed-order sum of block partials.
__global__ void k_sum_partials(const double *__restrict__ part, int nblocks, int K, double *__restrict__ out)
{
    if (threadIdx.x < K) {
        double s = 0;
        for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * K + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

__global__ void k_read_back(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

qs_status read_back(const qs_state *s, void *host, const void *dev, size_t bytes)
{
    if (bytes % 8 || bytes > kHostBoxBytes)
        return set_error(QS_ERR_INVALID_ARG, "read-back of %zu bytes", bytes);
    k_read_back<<<1, 64, 0, s->stream>>>((const unsigned long long *)dev, (unsigned long long *)s->hbox_dev,
                                         (int)(bytes / 8));
    QS_LAUNCH_CHECK();
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    std::memcpy(host, s->hbox, bytes);
    return QS_OK;
}

qs_status stage_view(const qs_state *s, size_t bytes, void **host, void **dev)
{
    if (s->stage_bytes < bytes) {
        if (s->stage) cudaFreeHost(s->stage);
        s->stage = s->stage_dev = nullptr;
        s->stage_bytes = 0;
        const size_t cap = std::max(bytes, (size_t)1 << 20);
        void *h = nullptr, *d = nullptr;
        cudaError_t e = cudaHostAlloc(&h, cap, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (h) cudaFreeHost(h);
            return set_error(QS_ERR_OOM, "host staging of %zu bytes: %s", cap, cudaGetErrorString(e));
        }
        s->stage = h;
        s->stage_dev = d;
        s->stage_bytes = cap;
    }
    *host = s->stage;
    *dev = s->stage_dev;
    return QS_OK;
}

qs_status stats_moments(const qs_state *s, int kmax, double *moments, double *entropy,
                        double *uniform_ce, double *norm)
{
    const uint64_t N = 1ULL << s->n;
    int grid;
    double *part = s->ws_f64;
    if (s->dt == QS_C64) {
        // the read-out cache holds the partials of the current state, or a
        // fused read-out pass forms them (with the sampler's chunk sums)
        if (!readout_cached(s, kReadoutStats))
            if (qs_status st = readout_c64(s, nullptr, 0)) return st;
        part = readout_part(s);
        grid = readout_grid(s);
    } else {
        grid = grid_for(N, kStatThreads, s->num_sms, 4);
        k_stats_c128<<<grid, kStatThreads, 0, s->stream>>>((const double2 *)s->amps, N,
                                                            std::ldexp(1.0, s->n), part);
        QS_LAUNCH_CHECK();
    }
    double *fin = part + (size_t)grid * kStatAcc;
    k_sum_partials<<<1, 32, 0, s->stream>>>(part, grid, kStatAcc, fin);
    QS_LAUNCH_CHECK();
    double h[kStatAcc];
    if (qs_status st = read_back(s, h, fin, sizeof h)) return st;
    // Statistics of the normalised distribution p / S, S = sum p: the
    // arithmetic of the evolution leaves |S - 1| at the rounding level
    // (systematic for FP32: rounded phase constants have modulus below 1),
    // and dividing it out keeps that drift out of the entropy, moments and
    // uniform cross entropy.  With y = N p and Y = sum y = N S:
    //   H      = -sum (p/S) ln(p/S) = ln S + ln N - (sum y ln y) / Y
    //   CE_u   = -(1/N) sum ln(p/S) = ln S + ln N - (sum ln y) / N
    //   M_k    = N^{k-1} sum (p/S)^k = (sum y^k) / (N S^k)
    const double Nd = (double)N, lnN = s->n * std::log(2.0);
    const double S = h[0] / Nd;
    if (norm) *norm = S;
    const double lnS = S > 0 ? std::log(S) : -INFINITY;
    if (entropy) *entropy = S > 0 ? lnS + lnN - h[1] / h[0] : 0.0;
    if (uniform_ce) *uniform_ce = S > 0 ? lnS + lnN - h[2] / Nd : INFINITY;
    for (int k = 1; k <= kmax; ++k)
        moments[k - 1] = S > 0 ? (k == 1 ? 1.0 : h[k + 1] / (Nd * std::pow(S, k))) : 0.0;
    return QS_OK;
}

// ---------------------------------------------------------------------------
// batched statistics: item = (element offset, count) of one instance's state;
// per-item partials are summed per instance in item order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kStatThreads)
k_batch_stats(const float2 *__restrict__ amps, const uint64_t *__restrict__ item_off,
              const uint64_t *__restrict__ item_cnt, const float *__restrict__ item_scale, int nitems,
              double *__restrict__ part)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        batch_stats_chunk(amps + item_off[it], item_cnt[it], item_scale[it], part + (size_t)it * kStatAcc);
        __syncthreads();
    }
}

__global__ void k_batch_stats_sum(const double *__restrict__ part, const int *__restrict__ first_item,
                                  int count, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int k = 0; k < kStatAcc; ++k) {
        double s = 0;
        for (int it = first_item[i]; it < first_item[i + 1]; ++it) s += part[(size_t)it * kStatAcc + k];
        out[(size_t)i * kStatAcc + k] = s;
    }
}

qs_status launch_batch_stats(cudaStream_t st, int num_sms, const void *amps, const uint64_t *item_off,
                             const uint64_t *item_cnt, const float *item_scale, int nitems,
                             const int *first_item, int count, double *part, double *out)
{
    const int grid = nitems < num_sms * 8 ? nitems : num_sms * 8;
    k_batch_stats<<<grid, kStatThreads, 0, st>>>((const float2 *)amps, item_off, item_cnt, item_scale, nitems,
                                                 part);
    QS_LAUNCH_CHECK();
    k_batch_stats_sum<<<(count + 127) / 128, 128, 0, st>>>(part, first_item, count, out);
    QS_LAUNCH_CHECK();
    return QS_OK;
}

void stats_from_sums(const double *h, int n, int kmax, double *norm, double *entropy, double *uniform_ce,
                     double *moments)
{
    const double Nd = std::ldexp(1.0, n), lnN = n * std::log(2.0);
    const double S = h[0] / Nd;
    const double lnS = S > 0 ? std::log(S) : -INFINITY;
    if (norm) *norm = S;
    if (entropy) *entropy = S > 0 ? lnS + lnN - h[1] / h[0] : 0.0;
    if (uniform_ce) *uniform_ce = S > 0 ? lnS + lnN - h[2] / Nd : INFINITY;
    for (int k = 1; k <= kmax; ++k)
        moments[k - 1] = S > 0 ? (k == 1 ? 1.0 : h[k + 1] / (Nd * std::pow(S, k))) : 0.0;
}

// ---------------------------------------------------------------------------
// sampler
// ---------------------------------------------------------------------------
// Lane l of a warp covers elements [8l, 8l+8) of a 256-amplitude chunk.  The
// lane totals and their inclusive warp scan are formed in the element type's
// precision (FP32 for complex64, FP64 for complex128) and widened exactly to
// FP64; the chunk sum is the scan's last lane.  The search kernels repeat
// exactly this arithmetic, so chunk sums and in-chunk prefixes agree (the
// chunk offsets themselves are FP64 scans of the chunk sums).
template <typename R>
__device__ __forceinline__ void lane_probs(const typename V2T<R>::T *a, uint64_t chunk, int lane,
                                           uint64_t N, R (&p)[8])
{
    const uint64_t base = chunk * kChunk + (uint64_t)lane * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint64_t idx = base + i;
        if (idx < N) {
            auto v = a[idx];
            if constexpr (sizeof(R) == 4) p[i] = prob32(v);
            else p[i] = v.x * v.x + v.y * v.y;
        } else {
            p[i] = (R)0;
        }
    }
}

template <typename R>
__device__ __forceinline__ R lane_total(const R (&p)[8])
{
    R s = (R)0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += p[i];
    return s;
}

__device__ __forceinline__ double warp_incl_scan(double v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ float warp_incl_scan_f(float v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// In-chunk prefix of a lane: inclusive and exclusive scan of the lane totals.
__device__ __forceinline__ void chunk_scan(double lt, double &incl, double &excl)
{
    incl = warp_incl_scan(lt);
    excl = incl - lt;
}
__device__ __forceinline__ void chunk_scan(float lt, double &incl, double &excl)
{
    const float fi = warp_incl_scan_f(lt);
    const float fe = __shfl_up_sync(0xffffffffu, fi, 1);
    incl = widen_f32(fi);
    excl = (threadIdx.x & 31) ? widen_f32(fe) : 0.0;
}

// One warp per chunk.
template <typename R>
__global__ void k_chunk_sums(const typename V2T<R>::T *__restrict__ a, uint64_t N, uint64_t nchunks,
                             double *__restrict__ csum)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        R p[8];
        lane_probs<R>(a, c, lane, N, p);
        double incl, excl;
        chunk_scan(lane_total<R>(p), incl, excl);
        if (lane == 31) csum[c] = incl;
    }
}

// In-place inclusive FP64 scan of x[0..n): three kernels with a fixed
// association order.  Segment of one block: kScanSeg elements, kScanPer per
// thread, sequential inside a thread, warp shuffle scan across threads,
// shared-memory scan across warps.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanSeg = kScanThreads * kScanPer;

__device__ __forceinline__ double block_excl_scan(double v, double *total)
{
    __shared__ double wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double incl = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double w = lane < kScanThreads / 32 ? wsum[lane] : 0.0;
        double wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) wsum[lane] = wi - w;   // exclusive
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    double r = wsum[warp] + (incl - v);
    __syncthreads();
    return r;
}

__global__ void k_scan_block_totals(const double *__restrict__ x, uint64_t n, double *__restrict__ btot)
{
    __shared__ double tot;
    const uint64_t base = (uint64_t)blockIdx.x * kScanSeg + (uint64_t)threadIdx.x * kScanPer;
    double s = 0;
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += x[base + i];
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block totals (sequential per thread).
__global__ void k_scan_totals(double *__restrict__ btot, int nb)
{
    __shared__ double tot;
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per;
    double s = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) s += btot[b0 + i];
    double off = block_excl_scan(s, &tot);
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) {
            double v = btot[b0 + i];
            btot[b0 + i] = off;
            off += v;
        }
}

__global__ void k_scan_apply(double *__restrict__ x, uint64_t n, const double *__restrict__ boff)
{
    __shared__ double tot;
    const uint64_t base = (uint64_t)blockIdx.x * kScanSeg + (uint64_t)threadIdx.x * kScanPer;
    double s = 0;
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += x[base + i];
    double off = block_excl_scan(s, &tot) + boff[blockIdx.x];
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) {
            off += x[base + i];
            x[base + i] = off;
        }
}

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// One warp handles 32 samples: each lane binary-searches the chunk of its
// own sample, then the warp rescans each of the 32 chunks in turn.
template <typename R>
__global__ void k_sample_search(const typename V2T<R>::T *__restrict__ a, uint64_t N, uint64_t nchunks,
                                const double *__restrict__ cincl, uint64_t k, uint64_t seed,
                                uint64_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const double total = cincl[nchunks - 1];
    for (uint64_t j0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; j0 < k;
         j0 += warps * 32) {
        const uint64_t j = j0 + lane;
        double tloc = 0;
        uint64_t chunk = 0;
        if (j < k) {
            const double u = (double)(splitmix_out(seed, j) >> 11) * (1.0 / 9007199254740992.0);
            const double target = u * total;
            uint64_t lo = 0, hi = nchunks - 1;   // cincl[hi] = total > target
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (cincl[mid] > target) hi = mid; else lo = mid + 1;
            }
            chunk = lo;
            tloc = target - (lo ? cincl[lo - 1] : 0.0);
        }
        const int cnt = (int)((k - j0) < 32 ? (k - j0) : 32);
        for (int q = 0; q < cnt; ++q) {
            const uint64_t c = __shfl_sync(0xffffffffu, chunk, q);
            const double tq = __shfl_sync(0xffffffffu, tloc, q);
            R p[8];
            lane_probs<R>(a, c, lane, N, p);
            const R lt = lane_total<R>(p);
            double incl, excl;
            chunk_scan(lt, incl, excl);
            unsigned hit = __ballot_sync(0xffffffffu, incl > tq);
            unsigned nz = __ballot_sync(0xffffffffu, lt > (R)0);
            int L = hit ? __ffs(hit) - 1 : 31 - __clz(nz);   // rounding edge: last non-empty lane
            uint64_t res = 0;
            if (lane == L) {
                R acc = (R)0;
                int pick = -1, last_nz = -1;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc += p[i];
                    if (p[i] > (R)0) last_nz = i;
                    if (pick < 0 && p[i] > (R)0 && excl + (double)acc > tq) pick = i;
                }
                if (pick < 0) pick = last_nz;
                res = c * kChunk + (uint64_t)L * 8 + (uint64_t)pick;
            }
            res = __shfl_sync(0xffffffffu, res, L);
            // the sample lies inside the state (checked build)
            if (lane == q && QS_DCHECK(res < N && c < nchunks, 301)) out[j0 + q] = res;
        }
    }
}

// ---------------------------------------------------------------------------
// fused read-out of a complex64 state
//
// One warp per 256-amplitude chunk (lane l: amplitudes 8l .. 8l+7, four
// 16-byte loads), one read of the state for three results: p = |psi|^2 (FP32,
// or widened exactly to FP64; optional), the chunk sums of the sampler (the
// lane totals and FP32 warp scan of lane_probs / chunk_scan, so the search
// kernel's in-chunk prefixes agree with them) and the statistics partials of
// each block (per-lane FP32 over eight chunks, then FP64, fixed order).  The
// statistics and chunk sums are the same whether or not p is written.
// ---------------------------------------------------------------------------
template <int OUT>   // 0: no p, 1: FP32 p, 2: FP64 p
__global__ void __launch_bounds__(kStatThreads, 3)
k_readout_c64(const float2 *__restrict__ a, uint64_t N, uint64_t nchunks, float scaleN, void *__restrict__ out,
              void *__restrict__ out_hi, uint64_t csplit, double *__restrict__ csum, double *__restrict__ part)
{
    __shared__ __align__(16) float stage_all[kStatThreads / 32][kChunk];
    float *stage = stage_all[threadIdx.x >> 5];
    double acc[kStatAcc];
#pragma unroll
    for (int k = 0; k < kStatAcc; ++k) acc[k] = 0;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    while (c < nchunks) {
        float cf[kStatAcc];
#pragma unroll
        for (int k = 0; k < kStatAcc; ++k) cf[k] = 0.f;
        for (int it = 0; it < 8 && c < nchunks; ++it, c += warps) {
            const uint64_t base = c * kChunk + (uint64_t)lane * 8;
            float p[8];
            if ((c + 1) * kChunk <= N) {   // a whole chunk: the same branch for all lanes of the warp
                const float4 *src = reinterpret_cast<const float4 *>(a + base);
                float4 v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = src[i];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    p[2 * i] = prob32(make_float2(v[i].x, v[i].y));
                    p[2 * i + 1] = prob32(make_float2(v[i].z, v[i].w));
                }
                if constexpr (OUT != 0) {
                    // through shared memory, so that each store instruction
                    // writes 32 consecutive 16-byte units (whole lines, also
                    // when `out` is page-locked host memory)
#pragma unroll
                    for (int i = 0; i < 8; ++i) stage[lane * 8 + i] = p[i];
                    __syncwarp();
                    const float4 *st4 = reinterpret_cast<const float4 *>(stage);
                    // chunks from csplit on go to the second output
                    void *dst = c < csplit ? out : out_hi;
                    const uint64_t cd = c < csplit ? c : c - csplit;
                    if constexpr (OUT == 2) {
                        double2 *o = reinterpret_cast<double2 *>(static_cast<double *>(dst) + cd * kChunk);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float2 q = reinterpret_cast<const float2 *>(stage)[k * 32 + lane];
                            o[k * 32 + lane] = make_double2(widen_f32(q.x), widen_f32(q.y));
                        }
                    } else {
                        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(dst) + cd * kChunk);
#pragma unroll
                        for (int k = 0; k < 2; ++k) o[k * 32 + lane] = st4[k * 32 + lane];
                    }
                    __syncwarp();
                }
            } else {
                // a state of fewer than 256 amplitudes (n < 8): one partial chunk
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    p[i] = base + i < N ? prob32(a[base + i]) : 0.f;
                    if (base + i < N) {
                        if constexpr (OUT == 2) static_cast<double *>(out)[base + i] = widen_f32(p[i]);
                        else if constexpr (OUT == 1) static_cast<float *>(out)[base + i] = p[i];
                    }
                }
            }
            double incl, excl;
            chunk_scan(lane_total<float>(p), incl, excl);
            if (lane == 31) csum[c] = incl;
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                if (base + i < N)
                    stat_pair_p(p[i], p[i + 1], base + i + 1 < N, scaleN, cf, acc);
            }
        }
#pragma unroll
        for (int k = 0; k < kStatAcc; ++k) acc[k] += (double)cf[k];
    }
    block_sum_store<kStatAcc>(acc, part + (size_t)blockIdx.x * kStatAcc);
}

int readout_grid(const qs_state *s)
{
    const uint64_t nchunks = ((1ULL << s->n) + kChunk - 1) / kChunk;
    return grid_for(nchunks * 32, kStatThreads, s->num_sms, 3);
}

// Device buffers of the read-out cache: statistics partials (+ their sum)
// and chunk sums (+ the scan's block totals).
static qs_status readout_buffers(const qs_state *s)
{
    const uint64_t nchunks = ((1ULL << s->n) + kChunk - 1) / kChunk;
    const uint64_t nblk = (nchunks + kScanSeg - 1) / kScanSeg;
    const size_t want = ((size_t)readout_grid(s) + 1) * kStatAcc + nchunks + nblk + 1;
    if (s->rc_buf && s->rc_doubles >= want) return QS_OK;
    if (s->rc_buf) cudaFree(s->rc_buf);
    s->rc_buf = nullptr;
    s->rc_doubles = 0;
    cudaError_t e = cudaMalloc((void **)&s->rc_buf, want * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->rc_buf = nullptr;
        return set_error(QS_ERR_OOM, "read-out cache of %zu doubles: %s", want, cudaGetErrorString(e));
    }
    s->rc_doubles = want;
    return QS_OK;
}

double *readout_part(const qs_state *s) { return s->rc_buf; }
double *readout_csum(const qs_state *s) { return s->rc_buf + ((size_t)readout_grid(s) + 1) * kStatAcc; }

uint64_t readout_chunks(const qs_state *s) { return ((1ULL << s->n) + kChunk - 1) / kChunk; }

qs_status readout_c64(const qs_state *s, void *out, int out_kind, void *out_hi, uint64_t csplit)
{
    if (qs_status st = readout_buffers(s)) return st;
    const uint64_t N = 1ULL << s->n;
    const uint64_t nchunks = (N + kChunk - 1) / kChunk;
    // a state of one partial chunk (n < 8) is never split
    if (!out_hi || csplit >= nchunks || N < kChunk) {
        out_hi = nullptr;
        csplit = nchunks;
    }
    const int grid = readout_grid(s);
    const float scaleN = (float)std::ldexp(1.0, s->n);
    const float2 *a = (const float2 *)s->amps;
    if (out_kind == 2)
        k_readout_c64<2><<<grid, kStatThreads, 0, s->stream>>>(a, N, nchunks, scaleN, out, out_hi, csplit,
                                                                readout_csum(s), readout_part(s));
    else if (out_kind == 1)
        k_readout_c64<1><<<grid, kStatThreads, 0, s->stream>>>(a, N, nchunks, scaleN, out, out_hi, csplit,
                                                                readout_csum(s), readout_part(s));
    else
        k_readout_c64<0><<<grid, kStatThreads, 0, s->stream>>>(a, N, nchunks, scaleN, nullptr, nullptr, nchunks,
                                                                readout_csum(s), readout_part(s));
    QS_LAUNCH_CHECK();
    s->rc_version = s->version;
    s->rc_flags = kReadoutStats | kReadoutChunks;
    return QS_OK;
}

bool readout_cached(const qs_state *s, int flag)
{
    return !s->escaped && s->rc_buf && s->rc_version == s->version && (s->rc_flags & flag);
}

// complex64: the chunk sums come from the read-out cache (a fused read-out
// pass when it holds none for the current state) and are scanned in place
// once; later samples of the same state reuse the scanned offsets.
static qs_status sampler_run_c64(const qs_state *s, uint64_t k, uint64_t seed, uint64_t *dev_out)
{
    const uint64_t N = 1ULL << s->n;
    const uint64_t nchunks = (N + kChunk - 1) / kChunk;
    const uint64_t nblk = (nchunks + kScanSeg - 1) / kScanSeg;
    if (!readout_cached(s, kReadoutChunks))
        if (qs_status st = readout_c64(s, nullptr, 0)) return st;
    double *csum = readout_csum(s), *btot = csum + nchunks;
    if (!(s->rc_flags & kReadoutScanned)) {
        k_scan_block_totals<<<(unsigned)nblk, kScanThreads, 0, s->stream>>>(csum, nchunks, btot);
        k_scan_totals<<<1, kScanThreads, 0, s->stream>>>(btot, (int)nblk);
        k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, s->stream>>>(csum, nchunks, btot);
        QS_LAUNCH_CHECK();
        s->rc_flags |= kReadoutScanned;
    }
    double total = 0;
    if (qs_status rb = read_back(s, &total, csum + nchunks - 1, sizeof(double))) return rb;
    if (!(total > 0) || !std::isfinite(total))
        return set_error(QS_ERR_INVALID_ARG, "state has zero or non-finite norm (%g)", total);
    if (k > 0) {
        const int th = 256;
        const int g2 = grid_for((k + 31) / 32 * 32, th, s->num_sms, 16);
        k_sample_search<float><<<g2, th, 0, s->stream>>>((const float2 *)s->amps, N, nchunks, csum, k, seed, dev_out);
        QS_LAUNCH_CHECK();
    }
    return QS_OK;
}

qs_status sampler_run(const qs_state *s, uint64_t k, uint64_t seed, uint64_t *dev_out)
{
    if (s->dt == QS_C64) return sampler_run_c64(s, k, seed, dev_out);
    const uint64_t N = 1ULL << s->n;
    const uint64_t nchunks = (N + kChunk - 1) / kChunk;
    const uint64_t nblk = (nchunks + kScanSeg - 1) / kScanSeg;
    const size_t bytes = (nchunks + nblk + 1) * sizeof(double);
    double *csum = nullptr;
    QS_CUDA_TRY(cudaMallocAsync((void **)&csum, bytes, s->stream));
    double *btot = csum + nchunks;
    qs_status st = QS_OK;
    const int th = 256;
    const int g1 = grid_for(nchunks * 32, th, s->num_sms, 16);
    if (s->dt == QS_C64)
        k_chunk_sums<float><<<g1, th, 0, s->stream>>>((const float2 *)s->amps, N, nchunks, csum);
    else
        k_chunk_sums<double><<<g1, th, 0, s->stream>>>((const double2 *)s->amps, N, nchunks, csum);
    k_scan_block_totals<<<(unsigned)nblk, kScanThreads, 0, s->stream>>>(csum, nchunks, btot);
    k_scan_totals<<<1, kScanThreads, 0, s->stream>>>(btot, (int)nblk);
    k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, s->stream>>>(csum, nchunks, btot);
    double total = 0;
    cudaError_t e = cudaSuccess;
    if (qs_status rb = read_back(s, &total, csum + nchunks - 1, sizeof(double))) {
        st = rb;
    } else if (!(total > 0) || !std::isfinite(total)) {
        st = set_error(QS_ERR_INVALID_ARG, "state has zero or non-finite norm (%g)", total);
    } else if (k > 0) {
        const int g2 = grid_for((k + 31) / 32 * 32, th, s->num_sms, 16);
        if (s->dt == QS_C64)
            k_sample_search<float><<<g2, th, 0, s->stream>>>((const float2 *)s->amps, N, nchunks, csum, k, seed, dev_out);
        else
            k_sample_search<double><<<g2, th, 0, s->stream>>>((const double2 *)s->amps, N, nchunks, csum, k, seed, dev_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = set_error(QS_ERR_CUDA, "sampler launch failed: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(csum, s->stream);
    return st;
}

// ---------------------------------------------------------------------------
// batched sampler: every instance of a batch, k samples each
//
// Chunks of 256 amplitudes never straddle instances: instance i owns global
// chunks [cbase[i], cbase[i+1]) (its last chunk may be short).  One
// inclusive FP64 scan runs over all chunk sums; instance i's CDF is the scan
// minus the value before its first chunk.  Sample (i, j) draws u from the
// counter-based stream at index i k + j and applies the measurement bit
// flips of the error model (bit b flips if the draw at index (i k + j) 64 + b
// of the stream seeded with seed ^ 0xD1B54A32D192ED03 is below r_mes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_instance_of(const uint64_t *cbase, int count, uint64_t c)
{
    int lo = 0, hi = count - 1;   // largest i with cbase[i] <= c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cbase[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_chunk_sums(const float2 *__restrict__ amps, const uint64_t *__restrict__ off,
                                   const int *__restrict__ nq, const uint64_t *__restrict__ cbase, int count,
                                   double *__restrict__ csum)
{
    const int lane = threadIdx.x & 31;
    const uint64_t nchunks = cbase[count];
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        const int i = batch_instance_of(cbase, count, c);
        float p[8];
        lane_probs<float>(amps + off[i], c - cbase[i], lane, 1ULL << nq[i], p);
        double incl, excl;
        chunk_scan(lane_total<float>(p), incl, excl);
        if (lane == 31) csum[c] = incl;
    }
}

__global__ void k_batch_sample_search(const float2 *__restrict__ amps, const uint64_t *__restrict__ off,
                                      const int *__restrict__ nq, const uint64_t *__restrict__ cbase, int count,
                                      const double *__restrict__ cincl, uint64_t k, uint64_t seed, double r_mes,
                                      uint64_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t m = (uint64_t)count * k;
    const uint64_t flip_seed = seed ^ 0xD1B54A32D192ED03ULL;
    for (uint64_t j0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; j0 < m;
         j0 += warps * 32) {
        const uint64_t j = j0 + lane;
        int inst = 0;
        double tloc = 0;
        uint64_t chunk = 0;
        bool ok = false;
        if (j < m) {
            inst = (int)(j / k);
            const uint64_t c0 = cbase[inst], c1 = cbase[inst + 1];
            const double before = c0 ? cincl[c0 - 1] : 0.0;
            const double total = cincl[c1 - 1] - before;
            ok = total > 0;
            const double u = (double)(splitmix_out(seed, j) >> 11) * (1.0 / 9007199254740992.0);
            const double target = before + u * total;
            uint64_t lo = c0, hi = c1 - 1;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                if (cincl[mid] > target) hi = mid; else lo = mid + 1;
            }
            chunk = lo;
            tloc = target - (lo ? cincl[lo - 1] : 0.0);
        }
        const int cnt = (int)((m - j0) < 32 ? (m - j0) : 32);
        for (int q = 0; q < cnt; ++q) {
            const uint64_t c = __shfl_sync(0xffffffffu, chunk, q);
            const double tq = __shfl_sync(0xffffffffu, tloc, q);
            const int iq = __shfl_sync(0xffffffffu, inst, q);
            const uint64_t lc = c - cbase[iq];
            float p[8];
            lane_probs<float>(amps + off[iq], lc, lane, 1ULL << nq[iq], p);
            const float lt = lane_total<float>(p);
            double incl, excl;
            chunk_scan(lt, incl, excl);
            const unsigned hit = __ballot_sync(0xffffffffu, incl > tq);
            const unsigned nz = __ballot_sync(0xffffffffu, lt > 0.f);
            const int L = hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : 0);
            uint64_t res = 0;
            if (lane == L) {
                float acc = 0.f;
                int pick = -1, last_nz = -1;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    acc += p[t];
                    if (p[t] > 0.f) last_nz = t;
                    if (pick < 0 && p[t] > 0.f && excl + (double)acc > tq) pick = t;
                }
                if (pick < 0) pick = last_nz < 0 ? 0 : last_nz;
                res = lc * kChunk + (uint64_t)L * 8 + (uint64_t)pick;
            }
            res = __shfl_sync(0xffffffffu, res, L);
            if (lane == q) {
                if (ok) {
                    for (int b = 0; b < nq[iq]; ++b) {
                        const double v = (double)(splitmix_out(flip_seed, j * 64 + (uint64_t)b) >> 11) *
                                         (1.0 / 9007199254740992.0);
                        if (v < r_mes) res ^= 1ULL << b;
                    }
                } else {
                    res = ~0ULL;      // instance with zero norm: no sample
                }
                out[j0 + q] = res;
            }
        }
    }
}

qs_status batch_sampler_run(cudaStream_t st, int num_sms, const void *amps_v, const uint64_t *off_h,
                            const int *n_h, int count, uint64_t k, uint64_t seed, double r_mes, uint64_t *host_out)
{
    const float2 *amps = static_cast<const float2 *>(amps_v);
    std::vector<uint64_t> cb(count + 1, 0);
    for (int i = 0; i < count; ++i) cb[i + 1] = cb[i] + (((1ULL << n_h[i]) + kChunk - 1) / kChunk);
    const uint64_t nchunks = cb[count];
    const uint64_t nblk = (nchunks + kScanSeg - 1) / kScanSeg;
    const uint64_t m = (uint64_t)count * k;
    // one scratch buffer: instance tables, chunk sums, block totals, samples
    const size_t b_off = (size_t)count * 8, b_cb = (size_t)(count + 1) * 8, b_n = (size_t)count * 4;
    const size_t o_cb = b_off, o_n = o_cb + b_cb, o_cs = (o_n + b_n + 15) / 16 * 16;
    const size_t o_bt = o_cs + nchunks * 8, o_out = o_bt + (nblk + 1) * 8;
    const size_t bytes = o_out + m * 8;
    char *buf = nullptr;
    QS_CUDA_TRY(cudaMallocAsync((void **)&buf, bytes, st));
    std::vector<char> host(o_cs);
    std::memcpy(host.data(), off_h, b_off);
    std::memcpy(host.data() + o_cb, cb.data(), b_cb);
    std::memcpy(host.data() + o_n, n_h, b_n);
    qs_status status = QS_OK;
    cudaError_t e = cudaMemcpyAsync(buf, host.data(), o_cs, cudaMemcpyHostToDevice, st);
    const uint64_t *d_off = (const uint64_t *)buf, *d_cb = (const uint64_t *)(buf + o_cb);
    const int *d_n = (const int *)(buf + o_n);
    double *csum = (double *)(buf + o_cs), *btot = (double *)(buf + o_bt);
    uint64_t *d_out = (uint64_t *)(buf + o_out);
    if (e == cudaSuccess) {
        const int th = 256;
        k_batch_chunk_sums<<<grid_for(nchunks * 32, th, num_sms, 16), th, 0, st>>>(amps, d_off, d_n, d_cb, count,
                                                                                csum);
        k_scan_block_totals<<<(unsigned)nblk, kScanThreads, 0, st>>>(csum, nchunks, btot);
        k_scan_totals<<<1, kScanThreads, 0, st>>>(btot, (int)nblk);
        k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, st>>>(csum, nchunks, btot);
        if (m)
            k_batch_sample_search<<<grid_for((m + 31) / 32 * 32, th, num_sms, 16), th, 0, st>>>(
                amps, d_off, d_n, d_cb, count, csum, k, seed, r_mes, d_out);
        e = cudaGetLastError();
        if (e == cudaSuccess && m) e = cudaMemcpyAsync(host_out, d_out, m * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) status = set_error(QS_ERR_CUDA, "batch sampler: %s", cudaGetErrorString(e));
    cudaFreeAsync(buf, st);
    return status;
}

// ---------------------------------------------------------------------------
// batch against a reference state (appendix "Residual correlations after
// discrete errors"): per instance i the sums S_ab = sum_x p_i(x) p_ref(x),
// S_aa = sum p_i^2, S_a = sum p_i, S_bb, S_b, in items of one instance chunk
// (FP32 products over strips of 64 elements per thread, FP64 across strips,
// fixed-order block and item reductions); and the mean distribution
// (1/count) sum_i p_i(x) (Fig. 1error), summed over instances in index order.
// ---------------------------------------------------------------------------
constexpr int kOvlAcc = 5;

__global__ void __launch_bounds__(kStatThreads)
k_batch_overlap(const float2 *__restrict__ amps, const float2 *__restrict__ ref,
                const uint64_t *__restrict__ item_off, const uint64_t *__restrict__ item_ref,
                const uint64_t *__restrict__ item_cnt, int nitems, double *__restrict__ part)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const float2 *a = amps + item_off[it];
        const float2 *r = ref + item_ref[it];
        const uint64_t cnt = item_cnt[it];
        double acc[kOvlAcc] = {0, 0, 0, 0, 0};
        for (uint64_t i0 = threadIdx.x; i0 < cnt; i0 += (uint64_t)blockDim.x * 64) {
            float c[kOvlAcc] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (uint64_t i = i0, j = 0; j < 64 && i < cnt; ++j, i += blockDim.x) {
                const float2 u = a[i], v = r[i];
                const float pa = u.x * u.x + u.y * u.y, pb = v.x * v.x + v.y * v.y;
                c[0] = fmaf(pa, pb, c[0]);
                c[1] = fmaf(pa, pa, c[1]);
                c[2] += pa;
                c[3] = fmaf(pb, pb, c[3]);
                c[4] += pb;
            }
#pragma unroll
            for (int k = 0; k < kOvlAcc; ++k) acc[k] += (double)c[k];
        }
        block_sum_store<kOvlAcc>(acc, part + (size_t)it * kOvlAcc);
        __syncthreads();
    }
}

__global__ void k_batch_overlap_sum(const double *__restrict__ part, const int *__restrict__ first_item,
                                    int count, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int k = 0; k < kOvlAcc; ++k) {
        double s = 0;
        for (int it = first_item[i]; it < first_item[i + 1]; ++it) s += part[(size_t)it * kOvlAcc + k];
        out[(size_t)i * kOvlAcc + k] = s;
    }
}

__global__ void k_batch_mean_probs(const float2 *__restrict__ amps, uint64_t N, int count,
                                   double *__restrict__ out)
{
    const double inv = 1.0 / count;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (uint64_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int i = 0; i < count; ++i) {
            const float2 u = amps[(uint64_t)i * N + x];
            s += (double)(u.x * u.x + u.y * u.y);
        }
        out[x] = s * inv;
    }
}

// Sums per instance into host_sums[i * 5 + {S_ab, S_aa, S_a, S_bb, S_b}].
qs_status batch_overlap_run(cudaStream_t st, int num_sms, const void *amps_v, const void *ref_v,
                            const uint64_t *off_h, int count, int n, double *host_sums)
{
    const float2 *amps = static_cast<const float2 *>(amps_v);
    const float2 *ref = static_cast<const float2 *>(ref_v);
    const uint64_t N = 1ULL << n, chunk = std::min<uint64_t>(N, 1ULL << 16), per = N / chunk;
    const int nitems = (int)(per * (uint64_t)count);
    std::vector<uint64_t> tab(3 * (size_t)nitems);
    std::vector<int> first(count + 1);
    for (int i = 0; i < count; ++i) {
        first[i] = (int)(i * per);
        for (uint64_t c = 0; c < per; ++c) {
            const size_t it = (size_t)(i * per + c);
            tab[it] = off_h[i] + c * chunk;
            tab[nitems + it] = c * chunk;
            tab[2 * (size_t)nitems + it] = chunk;
        }
    }
    first[count] = nitems;
    const size_t b_tab = tab.size() * 8, b_first = (size_t)(count + 1) * 4;
    const size_t o_first = b_tab, o_part = (o_first + b_first + 15) / 16 * 16;
    const size_t o_out = o_part + (size_t)nitems * kOvlAcc * 8;
    const size_t bytes = o_out + (size_t)count * kOvlAcc * 8;
    char *buf = nullptr;
    QS_CUDA_TRY(cudaMallocAsync((void **)&buf, bytes, st));
    cudaError_t e = cudaMemcpyAsync(buf, tab.data(), b_tab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_first, first.data(), b_first, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const uint64_t *d_tab = (const uint64_t *)buf;
        double *part = (double *)(buf + o_part), *out = (double *)(buf + o_out);
        const int grid = nitems < num_sms * 8 ? nitems : num_sms * 8;
        k_batch_overlap<<<grid, kStatThreads, 0, st>>>(amps, ref, d_tab, d_tab + nitems, d_tab + 2 * (size_t)nitems,
                                                       nitems, part);
        k_batch_overlap_sum<<<(count + 127) / 128, 128, 0, st>>>(part, (const int *)(buf + o_first), count, out);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_sums, out, (size_t)count * kOvlAcc * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "batch overlap: %s", cudaGetErrorString(e));
    return QS_OK;
}

qs_status batch_mean_probs_run(cudaStream_t st, int num_sms, const void *amps_v, int count, int n,
                               double *device_out)
{
    const uint64_t N = 1ULL << n;
    k_batch_mean_probs<<<grid_for(N, 256, num_sms, 8), 256, 0, st>>>(static_cast<const float2 *>(amps_v), N,
                                                                     count, device_out);
    QS_LAUNCH_CHECK();
    return QS_OK;
}

// ---------------------------------------------------------------------------
// sample cross entropy (Eq. ae)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kStatThreads)
k_cross_entropy(const typename V2T<R>::T *__restrict__ a, uint64_t N, const uint64_t *__restrict__ x,
                uint64_t m, double *__restrict__ part, unsigned long long *__restrict__ bad)
{
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        uint64_t i = x[j];
        if (i >= N) {
            atomicAdd(bad, 1ULL);
            continue;
        }
        auto v = a[i];
        double re = (double)v.x, im = (double)v.y;
        acc[0] -= log(re * re + im * im);
    }
    block_sum_store<1>(acc, part + blockIdx.x);
}

qs_status cross_entropy_run(const qs_state *s, const uint64_t *dev_samples, uint64_t m, double *ce)
{
    const uint64_t N = 1ULL << s->n;
    const int grid = grid_for(m, kStatThreads, s->num_sms, 4);
    double *part = s->ws_f64;
    unsigned long long *bad = (unsigned long long *)s->ws_u64;
    QS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s->stream));
    if (s->dt == QS_C64)
        k_cross_entropy<float><<<grid, kStatThreads, 0, s->stream>>>((const float2 *)s->amps, N, dev_samples, m, part, bad);
    else
        k_cross_entropy<double><<<grid, kStatThreads, 0, s->stream>>>((const double2 *)s->amps, N, dev_samples, m, part, bad);
    QS_LAUNCH_CHECK();
    k_sum_partials<<<1, 32, 0, s->stream>>>(part, grid, 1, part + grid);
    QS_LAUNCH_CHECK();
    double sum = 0;
    unsigned long long nbad = 0;
    if (qs_status st = read_back(s, &sum, part + grid, sizeof sum)) return st;
    if (qs_status st = read_back(s, &nbad, bad, sizeof nbad)) return st;
    if (nbad) return set_error(QS_ERR_INVALID_ARG, "%llu sample indices >= 2^n", nbad);
    *ce = sum / (double)m;
    return QS_OK;
}

QS_CHECK_READER(check_poll_stats)

}  // namespace qs

// ---------------------------------------------------------------------------
// Allocation-free sampler: qs_sample_noalloc
//
// The same chunk-sum / scan / search kernels as qs_sample, but their scratch
// is a fixed file-scope device array instead of memory obtained at run time.
// It holds one FP64 sum per 256-amplitude chunk plus the scan's block totals
// for up to 2^28 amplitudes (8 MiB, resident on every device that loads the
// library until the process exits).
// ---------------------------------------------------------------------------
namespace qs {

constexpr uint64_t kNoAllocMaxChunks = 1ULL << 20;   // 2^28 amplitudes / 256
constexpr uint64_t kNoAllocMaxBlocks = (kNoAllocMaxChunks + kScanSeg - 1) / kScanSeg;
constexpr int kNoAllocMaxQubits = 28;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxChunks + kNoAllocMaxBlocks];

// Device address of g_noalloc_scratch on the current device (host code only
// sees a host-side stand-in under the array's name).  Looked up on every
// call rather than cached: the address belongs to the module loaded in the
// current context, which a device reset replaces.
static qs_status noalloc_scratch(double **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return set_error(QS_ERR_CUDA, "cudaGetSymbolAddress for the sampler scratch failed: %s",
                         cudaGetErrorString(e));
    *out = (double *)p;
    return QS_OK;
}

static bool noalloc_is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace qs

using namespace qs;

extern "C" qs_status qs_sample_noalloc(int n, qs_dtype dt, const void *device_amps, void *cuda_stream,
                                       uint64_t k, uint64_t seed, uint64_t *device_out)
{
    clear_error();
    if (n < 1 || n > kNoAllocMaxQubits)
        return set_error(QS_ERR_INVALID_ARG,
                         "qs_sample_noalloc supports 1..%d qubits (its fixed scratch holds %llu chunk "
                         "sums); got n = %d", kNoAllocMaxQubits, (unsigned long long)kNoAllocMaxChunks, n);
    if (dt != QS_C64 && dt != QS_C128) return set_error(QS_ERR_INVALID_ARG, "bad dtype %d", (int)dt);
    if (!device_amps || ((uintptr_t)device_amps & 15))
        return set_error(QS_ERR_INVALID_ARG, "device_amps is NULL or not 16-byte aligned");
    if (k && !device_out) return set_error(QS_ERR_INVALID_ARG, "device_out is NULL");
    if (!noalloc_is_device(device_amps)) return set_error(QS_ERR_INVALID_ARG, "device_amps is not device memory");
    if (k && !noalloc_is_device(device_out)) return set_error(QS_ERR_INVALID_ARG, "device_out is not device memory");
    double *scratch = nullptr;
    if (qs_status st = noalloc_scratch(&scratch)) return st;
    int dev = 0, sms = 1;
    QS_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    const uint64_t N = 1ULL << n;
    const uint64_t nchunks = (N + kChunk - 1) / kChunk;
    const uint64_t nblk = (nchunks + kScanSeg - 1) / kScanSeg;
    double *csum = scratch;                 // every entry used is written below
    double *btot = scratch + kNoAllocMaxChunks;
    const int th = 256;
    const int g1 = grid_for(nchunks * 32, th, sms, 16);
    if (dt == QS_C64)
        k_chunk_sums<float><<<g1, th, 0, stream>>>((const float2 *)device_amps, N, nchunks, csum);
    else
        k_chunk_sums<double><<<g1, th, 0, stream>>>((const double2 *)device_amps, N, nchunks, csum);
    k_scan_block_totals<<<(unsigned)nblk, kScanThreads, 0, stream>>>(csum, nchunks, btot);
    k_scan_totals<<<1, kScanThreads, 0, stream>>>(btot, (int)nblk);
    k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, stream>>>(csum, nchunks, btot);
    QS_LAUNCH_CHECK();
    double total = 0;
    QS_CUDA_TRY(cudaMemcpyAsync(&total, csum + nchunks - 1, sizeof(double), cudaMemcpyDeviceToHost, stream));
    QS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (!(total > 0) || !std::isfinite(total))
        return set_error(QS_ERR_INVALID_ARG, "state has zero or non-finite norm (%g)", total);
    if (k == 0) return QS_OK;
    const int g2 = grid_for((k + 31) / 32 * 32, th, sms, 16);
    if (dt == QS_C64)
        k_sample_search<float><<<g2, th, 0, stream>>>((const float2 *)device_amps, N, nchunks, csum, k, seed, device_out);
    else
        k_sample_search<double><<<g2, th, 0, stream>>>((const double2 *)device_amps, N, nchunks, csum, k, seed, device_out);
    QS_LAUNCH_CHECK();
    return QS_OK;
}
