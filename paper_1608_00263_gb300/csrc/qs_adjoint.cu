// qs_adjoint.cu -- gradient of the sample cross entropy with respect to the
// angles of parameterised gates, by the adjoint (reverse) method.
//
// Loss (Eq. ae without the constant H_0): L(theta) = -(1/m) sum_j ln p(x_j),
// p(x) = |psi(x)|^2, psi = G_{K-1} ... G_0 |0>.  For a real parameter of gate
// k, dL/dtheta = 2 Re <lambda_k | (dG_k/dtheta) G_k^dagger | psi_k>, where
// psi_k is the state after gate k and lambda_k the adjoint state there:
//   lambda_{K-1} = -sum_j psi(x_j) / (m p(x_j)) |x_j>    (duplicates add)
//   psi_{k-1} = G_k^dagger psi_k,  lambda_{k-1} = G_k^dagger lambda_k.
// For R_P(theta) = exp(-i theta/2 P): (dG/dtheta) G^dagger = -(i/2) P, so
// dL/dtheta = Im <lambda_k| P |psi_k>.  For CPHASE(phi) = diag(1,1,1,e^{i phi}):
// (dG/dphi) G^dagger = i Pi_11, so dL/dphi = -2 Im <lambda_k| Pi_11 |psi_k>.
// Two state vectors in total (psi in place, lambda); gates are un-applied in
// tile groups (one pass over both states per group, see k_adj_group);
// per-gate reductions go to per-CTA partials summed in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_device.cuh"

namespace qs {

constexpr int kAdjThreads = 256;

template <typename R> struct AdjMat {
    R m[8];   // G^dagger, u00 u01 u10 u11 as (re, im)
};

// derivative kinds
enum { D_NONE = 0, D_X = 1, D_Y = 2, D_Z = 3, D_P11 = 4 };

// lambda = -sum_j psi(x_j) / (m p(x_j)) |x_j>; lambda is zero on entry.
template <typename R>
__global__ void k_adj_seed(const typename V2T<R>::T *__restrict__ psi, typename V2T<R>::T *__restrict__ lam,
                           const uint64_t *__restrict__ x, uint64_t m)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint64_t i = x[j];
        const auto v = psi[i];
        const double p = (double)v.x * v.x + (double)v.y * v.y;
        const double f = -1.0 / ((double)m * p);
        atomicAdd(&lam[i].x, (R)(f * v.x));
        atomicAdd(&lam[i].y, (R)(f * v.y));
    }
}

static bool is_param(int kind)
{
    return kind == QS_RX || kind == QS_RY || kind == QS_RZ || kind == QS_CPHASE;
}

// ---------------------------------------------------------------------------
// Tile-grouped reverse sweep.  Consecutive gates (taken from the end of the
// list backwards) whose qubits, with the lowest `kAdjLow` qubits for
// coalesced runs, fit in a tile of `t` qubits form a group; one launch per
// group loads the tile of psi and of lambda into shared memory (CTA tau owns
// the amplitudes whose out-of-tile qubits spell tau, as in the fused pass),
// un-applies the group's gates in reverse order on both, reducing each
// parameterised gate's derivative term before it is un-applied, and stores
// both tiles: two state passes per group instead of per gate.  Each CTA
// accumulates its derivative terms over its tiles in a fixed order and
// writes one partial per (parameter, CTA); the partials are summed in a
// fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kAdjGroupMax = 96;          // gates per group (descriptor table)
constexpr int kAdjUnits = 16;             // 16-byte units per thread per state: tiles of <= 2^12 complex64

struct AdjGate {        // one gate of a group, in reverse (un-apply) order
    int32_t two;        // 0: single-qubit on tile bit b0; 1: diagonal on tile bits b0 < b1
    int32_t b0, b1;
    int32_t deriv;      // D_* kind
    int32_t slot;       // parameter index (deriv != D_NONE)
    int32_t diag;       // single-qubit gate with G^dagger diagonal (m[2..5] zero)
    double m[8];        // G^dagger (u00 u01 u10 u11 as re, im), or conj(d) in m[0], m[1]
};

struct AdjGroup {
    int32_t t;                   // tile qubits
    int32_t ngates;
    int32_t gate_begin;          // index into the descriptor array
    int32_t nparam;              // parameterised gates of the group
    uint8_t L[16];               // qubit of each tile bit (ascending)
    uint8_t G[64];               // qubits outside the tile (ascending)
};

// The derivative terms are formed in the state's precision (R): each
// thread's partial covers a few pairs of one tile; partials are widened to
// FP64 for the reductions across threads, tiles and CTAs.  (GB300's FP64
// rate is ~1/60 of its FP32 rate, so FP64 products here would bound the
// complex64 sweep.)
template <typename R>
__device__ __forceinline__ void adj_pair(typename V2T<R>::T *ps, typename V2T<R>::T *lm, uint32_t i0, uint32_t i1,
                                         const AdjGate &g, R &acc)
{
    using V = typename V2T<R>::T;
    const V x0 = ps[i0], x1 = ps[i1], l0 = lm[i0], l1 = lm[i1];
    if (g.deriv) {
        const R l0r = l0.x, l0i = l0.y, l1r = l1.x, l1i = l1.y;
        const R a0r = x0.x, a0i = x0.y, a1r = x1.x, a1i = x1.y;
        if (g.deriv == D_X)
            acc += (l0r * a1i - l0i * a1r) + (l1r * a0i - l1i * a0r);
        else if (g.deriv == D_Y)
            acc += -(l0r * a1r + l0i * a1i) + (l1r * a0r + l1i * a0i);
        else
            acc += (l0r * a0i - l0i * a0r) - (l1r * a1i - l1i * a1r);
    }
    const R m0 = (R)g.m[0], m1 = (R)g.m[1], m6 = (R)g.m[6], m7 = (R)g.m[7];
    V y0, y1, k0, k1;
    // diagonal G^dagger (T, RZ): one complex product per amplitude -- taken
    // for complex128, whose sweep is FP64-bound; the complex64 sweep is
    // bound elsewhere and measured faster without the extra branch
    if (sizeof(R) == 8 && g.diag) {
        y0.x = m0 * x0.x - m1 * x0.y; y0.y = m0 * x0.y + m1 * x0.x;
        y1.x = m6 * x1.x - m7 * x1.y; y1.y = m6 * x1.y + m7 * x1.x;
        k0.x = m0 * l0.x - m1 * l0.y; k0.y = m0 * l0.y + m1 * l0.x;
        k1.x = m6 * l1.x - m7 * l1.y; k1.y = m6 * l1.y + m7 * l1.x;
        ps[i0] = y0; ps[i1] = y1; lm[i0] = k0; lm[i1] = k1;
        return;
    }
    const R m2 = (R)g.m[2], m3 = (R)g.m[3], m4 = (R)g.m[4], m5 = (R)g.m[5];
    y0.x = m0 * x0.x - m1 * x0.y + m2 * x1.x - m3 * x1.y;
    y0.y = m0 * x0.y + m1 * x0.x + m2 * x1.y + m3 * x1.x;
    y1.x = m4 * x0.x - m5 * x0.y + m6 * x1.x - m7 * x1.y;
    y1.y = m4 * x0.y + m5 * x0.x + m6 * x1.y + m7 * x1.x;
    k0.x = m0 * l0.x - m1 * l0.y + m2 * l1.x - m3 * l1.y;
    k0.y = m0 * l0.y + m1 * l0.x + m2 * l1.y + m3 * l1.x;
    k1.x = m4 * l0.x - m5 * l0.y + m6 * l1.x - m7 * l1.y;
    k1.y = m4 * l0.y + m5 * l0.x + m6 * l1.y + m7 * l1.x;
    ps[i0] = y0; ps[i1] = y1; lm[i0] = k0; lm[i1] = k1;
}

template <typename R>
__global__ void __launch_bounds__(kAdjThreads, 3)
k_adj_group(typename V2T<R>::T *__restrict__ psi, typename V2T<R>::T *__restrict__ lam,
            const AdjGroup *__restrict__ grp_g, const AdjGate *__restrict__ gates_g, uint64_t ntiles,
            double *__restrict__ part, int nparts)
{
    using V = typename V2T<R>::T;
    extern __shared__ __align__(16) unsigned char smem_adj[];
    __shared__ AdjGroup P;
    __shared__ AdjGate G[kAdjGroupMax];
    __shared__ double red[kAdjThreads / 32];
    __shared__ double acc_sh[kAdjGroupMax];
    __shared__ uint64_t it_off[kAdjUnits];
    const int tid = threadIdx.x;
    if (tid < (int)(sizeof(AdjGroup) / 4))
        reinterpret_cast<uint32_t *>(&P)[tid] = reinterpret_cast<const uint32_t *>(grp_g)[tid];
    __syncthreads();
    for (int i = tid; i < P.ngates * (int)(sizeof(AdjGate) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(G)[i] = reinterpret_cast<const uint32_t *>(gates_g + P.gate_begin)[i];
    for (int i = tid; i < kAdjGroupMax; i += blockDim.x) acc_sh[i] = 0.0;
    __syncthreads();
    const int t = P.t;
    const uint32_t T = 1u << t;
    V *ps = reinterpret_cast<V *>(smem_adj), *lm = ps + T;
    // 16-byte units: unit u holds tile elements 2u, 2u + 1 (tile bit 0 is
    // qubit 0, so they are neighbours in memory); unit tid + kAdjThreads i
    // sits at base | tid_off | it_off[i] (the deposit over the tile qubits is
    // linear and the bits are disjoint)
    constexpr int kEl = 16 / (int)sizeof(V);          // elements per unit
    const uint32_t units = T / kEl;
    auto deposit = [&](uint32_t e) {
        uint64_t a = 0;
        for (int b = 0; b < t; ++b) a |= (uint64_t)((e >> b) & 1u) << P.L[b];
        return a;
    };
    for (uint32_t i = tid; i * kAdjThreads < units && i < (uint32_t)kAdjUnits; i += blockDim.x)
        it_off[i] = deposit(kEl * kAdjThreads * i);
    const uint64_t tid_off = deposit(kEl * (uint32_t)tid);
    __syncthreads();
    // contiguous range of tiles per CTA; tile base = deposit of the tile
    // index over the out-of-tile qubits
    const uint64_t per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
    const uint64_t t0 = blockIdx.x * per + (blockIdx.x < extra ? blockIdx.x : extra);
    const uint64_t t1 = t0 + per + (blockIdx.x < extra ? 1 : 0);
    int nglob = 0;
    uint64_t gmask = 0;
    for (int i = 0; i < 64 && P.G[i] != 0xFF; ++i) {
        gmask |= 1ULL << P.G[i];
        ++nglob;
    }
    uint64_t base = 0;
    for (int i = 0; i < nglob; ++i) base |= ((t0 >> i) & 1ULL) << P.G[i];
    for (uint64_t tau = t0; tau < t1; ++tau, base = ((base | ~gmask) + 1) & gmask) {
        // load: unit tid + kAdjThreads i of the tile, 16 bytes of each state
#pragma unroll 4
        for (uint32_t i = 0; i * kAdjThreads < units; ++i) {
            if (i * kAdjThreads + tid >= units) break;
            const uint64_t a = base | tid_off | it_off[i];
            // the amplitudes lie inside the state (checked build)
            if (QS_DCHECK((a >> (t + nglob)) == 0, 401)) {
                const uint32_t e = kEl * (tid + kAdjThreads * i);
                *reinterpret_cast<float4 *>(ps + e) = *reinterpret_cast<const float4 *>(psi + a);
                *reinterpret_cast<float4 *>(lm + e) = *reinterpret_cast<const float4 *>(lam + a);
            }
        }
        __syncthreads();
        int slot = 0;
        for (int k = 0; k < P.ngates; ++k) {
            const AdjGate &g = G[k];
            R acc = (R)0;
            if (!g.two) {
                const uint32_t bit = 1u << g.b0, lo_mask = bit - 1;
                for (uint32_t p = tid; p < T / 2; p += blockDim.x) {
                    const uint32_t i0 = ((p & ~lo_mask) << 1) | (p & lo_mask);
                    adj_pair<R>(ps, lm, i0, i0 | bit, g, acc);
                }
            } else {
                const uint32_t set = (1u << g.b0) | (1u << g.b1);
                for (uint32_t j = tid; j < T / 4; j += blockDim.x) {
                    uint32_t i = ((j >> g.b0) << (g.b0 + 1)) | (j & ((1u << g.b0) - 1));
                    i = ((i >> g.b1) << (g.b1 + 1)) | (i & ((1u << g.b1) - 1));
                    i |= set;
                    V x = ps[i], l = lm[i];
                    if (g.deriv) acc += l.x * x.y - l.y * x.x;
                    const R dr = (R)g.m[0], di = (R)g.m[1];
                    V y, kk;
                    y.x = dr * x.x - di * x.y; y.y = dr * x.y + di * x.x;
                    kk.x = dr * l.x - di * l.y; kk.y = dr * l.y + di * l.x;
                    ps[i] = y; lm[i] = kk;
                }
            }
            if (g.deriv) {
                // fixed-order block reduction of this gate's term on this tile
                double accd = (double)acc;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) accd += __shfl_xor_sync(0xffffffffu, accd, o);
                if ((tid & 31) == 0) red[tid >> 5] = accd;
                __syncthreads();
                if (tid == 0) {
                    double sum = 0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
                    acc_sh[slot] += sum;
                }
                ++slot;
            }
            __syncthreads();
        }
#pragma unroll 4
        for (uint32_t i = 0; i * kAdjThreads < units; ++i) {
            if (i * kAdjThreads + tid >= units) break;
            const uint64_t a = base | tid_off | it_off[i];
            if (QS_DCHECK((a >> (t + nglob)) == 0, 402)) {
                const uint32_t e = kEl * (tid + kAdjThreads * i);
                *reinterpret_cast<float4 *>(psi + a) = *reinterpret_cast<const float4 *>(ps + e);
                *reinterpret_cast<float4 *>(lam + a) = *reinterpret_cast<const float4 *>(lm + e);
            }
        }
        __syncthreads();
    }
    // this CTA's partial of every parameter of the group
    for (int k = tid; k < P.nparam; k += blockDim.x) part[(size_t)k * nparts + blockIdx.x] = acc_sh[k];
}

__global__ void k_adj_sums(const double *__restrict__ part, int nparts, int nparam, const double *__restrict__ scale,
                           double *__restrict__ out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nparam; k += gridDim.x * blockDim.x) {
        double s = 0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)k * nparts + b];
        out[k] = s * scale[k];
    }
}

// Groups of the reverse sweep (see above), their gate descriptors and the
// scale of every parameter's derivative term (1 for R_P, -2 for CPHASE).
template <typename R>
static void adjoint_groups(int n, const qs_gate *g, size_t ng, int t, int low, std::vector<AdjGroup> *groups,
                           std::vector<AdjGate> *gates, std::vector<int> *param_of_slot, std::vector<double> *scale)
{
    const uint64_t lowm = (1ULL << low) - 1;
    size_t pidx = 0;
    for (size_t k = 0; k < ng; ++k) pidx += is_param(g[k].kind);
    long k = (long)ng - 1;
    while (k >= 0) {
        uint64_t tq = lowm;
        long b = k;
        int cnt = 0;
        while (b >= 0 && cnt < kAdjGroupMax) {
            uint64_t q = 1ULL << g[b].q0;
            if (gate_is_two_qubit(g[b].kind)) q |= 1ULL << g[b].q1;
            if (__builtin_popcountll(tq | q) > t) break;
            tq |= q;
            --b;
            ++cnt;
        }
        // pad the tile with the lowest unused qubits up to t
        for (int q = 0; q < n && __builtin_popcountll(tq) < t; ++q) tq |= 1ULL << q;
        AdjGroup G;
        std::memset(&G, 0, sizeof G);
        std::memset(G.G, 0xFF, sizeof G.G);
        G.t = __builtin_popcountll(tq);
        G.gate_begin = (int)gates->size();
        int tb = 0, gb = 0, bit_of[64];
        for (int q = 0; q < n; ++q) {
            if ((tq >> q) & 1) { bit_of[q] = tb; G.L[tb++] = (uint8_t)q; }
            else { bit_of[q] = -1; G.G[gb++] = (uint8_t)q; }
        }
        int slot = 0;
        for (long i = k; i > b; --i) {             // reverse order
            const qs_gate &x = g[i];
            AdjGate d;
            std::memset(&d, 0, sizeof d);
            Cplx u[4];
            gate_matrix(x.kind, x.theta, u);
            const bool param = is_param(x.kind);
            if (gate_is_two_qubit(x.kind)) {
                const int b0 = bit_of[x.q0], b1 = bit_of[x.q1];
                d.two = 1;
                d.b0 = b0 < b1 ? b0 : b1;
                d.b1 = b0 < b1 ? b1 : b0;
                d.m[0] = u[3].re;
                d.m[1] = -u[3].im;
                d.deriv = param ? D_P11 : D_NONE;
            } else {
                d.b0 = bit_of[x.q0];
                const int perm[4] = {0, 2, 1, 3};       // (G^dagger)_{rc} = conj(G_{cr})
                for (int e = 0; e < 4; ++e) {
                    d.m[2 * e] = u[perm[e]].re;
                    d.m[2 * e + 1] = -u[perm[e]].im;
                }
                d.deriv = x.kind == QS_RX ? D_X : x.kind == QS_RY ? D_Y : x.kind == QS_RZ ? D_Z : D_NONE;
                d.diag = d.m[2] == 0 && d.m[3] == 0 && d.m[4] == 0 && d.m[5] == 0;
            }
            if (param) {
                --pidx;
                d.slot = slot++;
                param_of_slot->push_back((int)pidx);
                scale->push_back(d.two ? -2.0 : 1.0);
            }
            gates->push_back(d);
        }
        G.ngates = (int)(gates->size() - (size_t)G.gate_begin);
        G.nparam = slot;
        groups->push_back(G);
        k = b;
    }
}

template <typename R>
static qs_status adjoint_t(qs_state *s, const qs_gate *g, size_t ng, const uint64_t *dev_x, uint64_t m,
                           double *grad)
{
    using V = typename V2T<R>::T;
    const int n = s->n;
    const uint64_t N = 1ULL << n;
    // tiles of psi and lambda in shared memory: 2 x 2^t amplitudes (64 KB)
    const int t = std::min(n, sizeof(R) == 4 ? 12 : 11);
    const int low = std::min(t, sizeof(R) == 4 ? 4 : 3);
    std::vector<AdjGroup> groups;
    std::vector<AdjGate> gates;
    std::vector<int> pslot;       // parameter index of each group slot, in sweep order
    std::vector<double> scale;
    adjoint_groups<R>(n, g, ng, t, low, &groups, &gates, &pslot, &scale);
    const size_t nparam = pslot.size();
    V *psi = (V *)s->amps, *lam = nullptr;
    const int ctas = 3 * s->num_sms;          // three CTAs per SM (64 KB of tiles each)
    const size_t smem = 2 * ((size_t)1 << t) * sizeof(V);
    QS_CUDA_TRY(cudaFuncSetAttribute(k_adj_group<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // device tables: groups | gates | scale (in sweep-slot order) | partials | sums
    const size_t b_grp = groups.size() * sizeof(AdjGroup), b_gate = gates.size() * sizeof(AdjGate);
    const size_t b_scale = (nparam ? nparam : 1) * sizeof(double);
    const size_t b_part = (nparam ? nparam : 1) * (size_t)ctas * sizeof(double);
    const size_t b_out = (nparam ? nparam : 1) * sizeof(double);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_gate = al(b_grp), o_scale = o_gate + al(b_gate), o_part = o_scale + al(b_scale),
                 o_out = o_part + al(b_part), total = o_out + al(b_out);
    std::vector<unsigned char> host(o_part, 0);
    std::memcpy(host.data(), groups.data(), b_grp);
    if (b_gate) std::memcpy(host.data() + o_gate, gates.data(), b_gate);
    if (nparam) std::memcpy(host.data() + o_scale, scale.data(), nparam * sizeof(double));
    unsigned char *dev = nullptr;
    QS_CUDA_TRY(cudaMallocAsync((void **)&lam, N * sizeof(V), s->stream));
    cudaError_t e = cudaMallocAsync((void **)&dev, total, s->stream);
    qs_status st = QS_OK;
    if (e != cudaSuccess) {
        st = set_error(QS_ERR_OOM, "adjoint workspace: %s", cudaGetErrorString(e));
    } else {
        e = cudaMemcpyAsync(dev, host.data(), o_part, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(lam, 0, N * sizeof(V), s->stream);
        // partials of CTAs beyond a small group's grid stay zero
        if (e == cudaSuccess) e = cudaMemsetAsync(dev + o_part, 0, b_part, s->stream);
        if (e == cudaSuccess) {
            k_adj_seed<R><<<grid_for(m, 256, s->num_sms, 4), 256, 0, s->stream>>>(psi, lam, dev_x, m);
            size_t slot0 = 0;
            for (size_t gi = 0; gi < groups.size(); ++gi) {
                const uint64_t ntiles = N >> groups[gi].t;
                const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctas);
                // partial of (group slot j, CTA b) at part[(slot0 + j) * ctas + b]
                k_adj_group<R><<<grid, kAdjThreads, smem, s->stream>>>(
                    psi, lam, (const AdjGroup *)dev + gi, (const AdjGate *)(dev + o_gate),
                    ntiles, (double *)(dev + o_part) + slot0 * (size_t)ctas, ctas);
                slot0 += groups[gi].nparam;
            }
            if (nparam)
                k_adj_sums<<<grid_for(nparam, 128, s->num_sms, 1), 128, 0, s->stream>>>(
                    (const double *)(dev + o_part), ctas, (int)nparam, (const double *)(dev + o_scale),
                    (double *)(dev + o_out));
            if (e == cudaSuccess) e = cudaGetLastError();
            std::vector<double> h(nparam);
            if (e == cudaSuccess && nparam)
                e = cudaMemcpyAsync(h.data(), dev + o_out, nparam * sizeof(double), cudaMemcpyDeviceToHost,
                                    s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e == cudaSuccess) {
                for (size_t k = 0; k < ng; ++k) grad[k] = 0.0;
                // slot order is the sweep order; map back to gate positions
                std::vector<size_t> gate_of_param;
                for (size_t k = 0; k < ng; ++k)
                    if (is_param(g[k].kind)) gate_of_param.push_back(k);
                for (size_t j = 0; j < nparam; ++j) grad[gate_of_param[(size_t)pslot[j]]] = h[j];
            }
        }
        if (e != cudaSuccess) st = set_error(QS_ERR_CUDA, "adjoint sweep: %s", cudaGetErrorString(e));
    }
    if (lam) cudaFreeAsync(lam, s->stream);
    if (dev) cudaFreeAsync(dev, s->stream);
    cudaStreamSynchronize(s->stream);
    return st;
}

qs_status adjoint_run(qs_state *s, const qs_gate *g, size_t ng, const uint64_t *dev_x, uint64_t m, double *grad)
{
    return s->dt == QS_C64 ? adjoint_t<float>(s, g, ng, dev_x, m, grad)
                           : adjoint_t<double>(s, g, ng, dev_x, m, grad);
}

QS_CHECK_READER(check_poll_adjoint)

}  // namespace qs
