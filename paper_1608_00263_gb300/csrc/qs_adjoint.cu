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
// Two state vectors in total (psi in place, lambda); one pass over both per
// gate; per-gate reductions go to block partials summed in a fixed order.
#include <cmath>
#include <vector>

#include "qs_device.cuh"

namespace qs {

constexpr int kAdjThreads = 256;

template <typename R> struct AdjMat {
    R m[8];   // G^dagger, u00 u01 u10 u11 as (re, im)
};

// derivative kinds
enum { D_NONE = 0, D_X = 1, D_Y = 2, D_Z = 3, D_P11 = 4 };

__device__ __forceinline__ double block_sum1(double v)
{
    __shared__ double red[kAdjThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kAdjThreads / 32; ++w) s += red[w];
    return s;
}

// Single-qubit gate step: accumulate the gradient term (if any) on
// (lambda, psi) before uncomputing, then apply G^dagger to both.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_1q(typename V2T<R>::T *__restrict__ psi, typename V2T<R>::T *__restrict__ lam, int q, uint64_t npairs,
         AdjMat<R> g, int deriv, double *__restrict__ part)
{
    using V = typename V2T<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t bit = 1ULL << q;
    double acc = 0.0;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
        const uint64_t i0 = insert_zero(p, q), i1 = i0 | bit;
        const V x0 = psi[i0], x1 = psi[i1], l0 = lam[i0], l1 = lam[i1];
        if (deriv) {
            // Im( conj(l0) (P psi)_0 + conj(l1) (P psi)_1 )
            double im;
            const double l0r = l0.x, l0i = l0.y, l1r = l1.x, l1i = l1.y;
            const double a0r = x0.x, a0i = x0.y, a1r = x1.x, a1i = x1.y;
            if (deriv == D_X)        // (P psi) = (psi1, psi0)
                im = (l0r * a1i - l0i * a1r) + (l1r * a0i - l1i * a0r);
            else if (deriv == D_Y)   // (P psi) = (-i psi1, i psi0)
                im = -(l0r * a1r + l0i * a1i) + (l1r * a0r + l1i * a0i);
            else                     // (P psi) = (psi0, -psi1)
                im = (l0r * a0i - l0i * a0r) - (l1r * a1i - l1i * a1r);
            acc += im;
        }
        V y0, y1, k0, k1;
        y0.x = g.m[0] * x0.x - g.m[1] * x0.y + g.m[2] * x1.x - g.m[3] * x1.y;
        y0.y = g.m[0] * x0.y + g.m[1] * x0.x + g.m[2] * x1.y + g.m[3] * x1.x;
        y1.x = g.m[4] * x0.x - g.m[5] * x0.y + g.m[6] * x1.x - g.m[7] * x1.y;
        y1.y = g.m[4] * x0.y + g.m[5] * x0.x + g.m[6] * x1.y + g.m[7] * x1.x;
        k0.x = g.m[0] * l0.x - g.m[1] * l0.y + g.m[2] * l1.x - g.m[3] * l1.y;
        k0.y = g.m[0] * l0.y + g.m[1] * l0.x + g.m[2] * l1.y + g.m[3] * l1.x;
        k1.x = g.m[4] * l0.x - g.m[5] * l0.y + g.m[6] * l1.x - g.m[7] * l1.y;
        k1.y = g.m[4] * l0.y + g.m[5] * l0.x + g.m[6] * l1.y + g.m[7] * l1.x;
        psi[i0] = y0; psi[i1] = y1; lam[i0] = k0; lam[i1] = k1;
    }
    if (deriv) {
        const double s = block_sum1(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// Two-qubit diagonal step (CZ, CPHASE): only amplitudes with both bits set
// change (factor conj(d)); the CPHASE term is Im <lambda| Pi_11 |psi>.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_2q(typename V2T<R>::T *__restrict__ psi, typename V2T<R>::T *__restrict__ lam, int lo, int hi,
         uint64_t count, R dr, R di, int deriv, double *__restrict__ part)
{
    using V = typename V2T<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t set = (1ULL << lo) | (1ULL << hi);
    double acc = 0.0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
        const uint64_t i = insert_zero(insert_zero(j, lo), hi) | set;
        V x = psi[i], l = lam[i];
        if (deriv) acc += (double)l.x * x.y - (double)l.y * x.x;
        V y, k;
        y.x = dr * x.x - di * x.y; y.y = dr * x.y + di * x.x;
        k.x = dr * l.x - di * l.y; k.y = dr * l.y + di * l.x;
        psi[i] = y; lam[i] = k;
    }
    if (deriv) {
        const double s = block_sum1(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

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

__global__ void k_adj_sum(const double *__restrict__ part, int nblocks, double scale, double *__restrict__ out)
{
    if (threadIdx.x == 0) {
        double s = 0;
        for (int b = 0; b < nblocks; ++b) s += part[b];
        *out = s * scale;
    }
}

static bool is_param(int kind)
{
    return kind == QS_RX || kind == QS_RY || kind == QS_RZ || kind == QS_CPHASE;
}

template <typename R>
static qs_status adjoint_t(qs_state *s, const qs_gate *g, size_t ng, const uint64_t *dev_x, uint64_t m,
                           double *grad)
{
    using V = typename V2T<R>::T;
    const int n = s->n;
    const uint64_t N = 1ULL << n;
    V *psi = (V *)s->amps, *lam = nullptr;
    size_t nparam = 0;
    for (size_t k = 0; k < ng; ++k) nparam += is_param(g[k].kind);
    const int grid1 = grid_for(N / 2, kAdjThreads, s->num_sms, 4);
    const int grid2 = grid_for(N / 4 ? N / 4 : 1, kAdjThreads, s->num_sms, 4);
    const int gmax = grid1 > grid2 ? grid1 : grid2;
    double *part = nullptr, *dgrad = nullptr;
    const size_t bytes_state = N * sizeof(V);
    const size_t bytes_part = (nparam ? nparam : 1) * (size_t)gmax * sizeof(double);
    QS_CUDA_TRY(cudaMallocAsync((void **)&lam, bytes_state, s->stream));
    cudaError_t e = cudaMallocAsync((void **)&part, bytes_part, s->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dgrad, (nparam ? nparam : 1) * sizeof(double), s->stream);
    qs_status st = QS_OK;
    if (e != cudaSuccess) {
        st = set_error(QS_ERR_OOM, "adjoint workspace: %s", cudaGetErrorString(e));
    } else {
        e = cudaMemsetAsync(lam, 0, bytes_state, s->stream);
        if (e == cudaSuccess) {
            k_adj_seed<R><<<grid_for(m, 256, s->num_sms, 4), 256, 0, s->stream>>>(psi, lam, dev_x, m);
            size_t pi = nparam;
            for (size_t kk = ng; kk-- > 0;) {
                const qs_gate &x = g[kk];
                Cplx u[4];
                gate_matrix(x.kind, x.theta, u);
                const bool param = is_param(x.kind);
                if (param) --pi;
                double *pp = part + pi * (size_t)gmax;
                if (gate_is_two_qubit(x.kind)) {
                    const int lo = x.q0 < x.q1 ? x.q0 : x.q1, hi = x.q0 < x.q1 ? x.q1 : x.q0;
                    k_adj_2q<R><<<grid2, kAdjThreads, 0, s->stream>>>(
                        psi, lam, lo, hi, N / 4, (R)u[3].re, (R)-u[3].im, param ? D_P11 : D_NONE, pp);
                    if (param)
                        k_adj_sum<<<1, 32, 0, s->stream>>>(pp, grid2, -2.0, dgrad + pi);
                } else {
                    AdjMat<R> a;   // G^dagger: (G^dagger)_{rc} = conj(G_{cr})
                    const int perm[4] = {0, 2, 1, 3};
                    for (int k = 0; k < 4; ++k) {
                        a.m[2 * k] = (R)u[perm[k]].re;
                        a.m[2 * k + 1] = (R)-u[perm[k]].im;
                    }
                    const int d = x.kind == QS_RX ? D_X : x.kind == QS_RY ? D_Y : x.kind == QS_RZ ? D_Z : D_NONE;
                    k_adj_1q<R><<<grid1, kAdjThreads, 0, s->stream>>>(psi, lam, x.q0, N / 2, a, d, pp);
                    if (param) k_adj_sum<<<1, 32, 0, s->stream>>>(pp, grid1, 1.0, dgrad + pi);
                }
            }
            e = cudaGetLastError();
            if (e == cudaSuccess && nparam) {
                std::vector<double> h(nparam);
                e = cudaMemcpyAsync(h.data(), dgrad, nparam * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
                if (e == cudaSuccess) {
                    size_t j = 0;
                    for (size_t k = 0; k < ng; ++k) grad[k] = is_param(g[k].kind) ? h[j++] : 0.0;
                }
            } else if (e == cudaSuccess) {
                for (size_t k = 0; k < ng; ++k) grad[k] = 0.0;
                e = cudaStreamSynchronize(s->stream);
            }
        }
        if (e != cudaSuccess) st = set_error(QS_ERR_CUDA, "adjoint sweep: %s", cudaGetErrorString(e));
    }
    if (lam) cudaFreeAsync(lam, s->stream);
    if (part) cudaFreeAsync(part, s->stream);
    if (dgrad) cudaFreeAsync(dgrad, s->stream);
    cudaStreamSynchronize(s->stream);
    return st;
}

qs_status adjoint_run(qs_state *s, const qs_gate *g, size_t ng, const uint64_t *dev_x, uint64_t m, double *grad)
{
    return s->dt == QS_C64 ? adjoint_t<float>(s, g, ng, dev_x, m, grad)
                           : adjoint_t<double>(s, g, ng, dev_x, m, grad);
}

}  // namespace qs
