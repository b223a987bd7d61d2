// qs_plain.cu -- state initialisation and the plain per-gate kernels: one
// pass over (the affected part of) the state per gate.
//
// Single-qubit gates follow Eq. sqgunitaryoperation: every pair of
// amplitudes whose indices differ only in bit q is multiplied by the 2x2
// matrix.  Gate specialisation as in the appendix "Quantum Simulation
// Details": a diagonal gate with a 1 on the diagonal touches only the
// amplitudes it changes (T: the half with bit q set, 8N bytes for complex64;
// CZ / CPHASE: the quarter with both bits set, 4N bytes).
#include <cmath>

#include "qs_device.cuh"

namespace qs {

template <typename R> struct Mat2 {
    R m[8];   // u00 u01 u10 u11 as (re, im)
};

// ----- dense single-qubit gate, generic (one pair per iteration) -----------
template <typename R>
__global__ void k_dense1(typename V2T<R>::T *__restrict__ a, int q, uint64_t npairs, Mat2<R> u)
{
    using V = typename V2T<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t bit = 1ULL << q;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
        uint64_t i0 = insert_zero(p, q), i1 = i0 | bit;
        if (!QS_DCHECK(i1 < 2 * npairs, 101)) continue;
        V x = a[i0], y = a[i1];
        V o0, o1;
        o0.x = u.m[0] * x.x - u.m[1] * x.y + u.m[2] * y.x - u.m[3] * y.y;
        o0.y = u.m[0] * x.y + u.m[1] * x.x + u.m[2] * y.y + u.m[3] * y.x;
        o1.x = u.m[4] * x.x - u.m[5] * x.y + u.m[6] * y.x - u.m[7] * y.y;
        o1.y = u.m[4] * x.y + u.m[5] * x.x + u.m[6] * y.y + u.m[7] * y.x;
        a[i0] = o0;
        a[i1] = o1;
    }
}

// complex64, q >= 1: two neighbouring pairs per iteration with 16-byte
// accesses (their bit-0 neighbours share the same q-bit).
__global__ void k_dense1_c64v(float4 *__restrict__ a4, int q, uint64_t nquads, Mat2<float> u)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t half = 1ULL << (q - 1);      // offset of i1 in float4 units
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nquads; w += stride) {
        // pairs p = 2w, 2w+1 -> i0 = insert_zero(2w, q) (even), i0 + 1
        uint64_t i0 = insert_zero(2 * w, q) >> 1;    // float4 index
        if (!QS_DCHECK(i0 + half < 2 * nquads, 102)) continue;
        float4 x = a4[i0], y = a4[i0 + half];
        float4 o0, o1;
        o0.x = u.m[0] * x.x - u.m[1] * x.y + u.m[2] * y.x - u.m[3] * y.y;
        o0.y = u.m[0] * x.y + u.m[1] * x.x + u.m[2] * y.y + u.m[3] * y.x;
        o1.x = u.m[4] * x.x - u.m[5] * x.y + u.m[6] * y.x - u.m[7] * y.y;
        o1.y = u.m[4] * x.y + u.m[5] * x.x + u.m[6] * y.y + u.m[7] * y.x;
        o0.z = u.m[0] * x.z - u.m[1] * x.w + u.m[2] * y.z - u.m[3] * y.w;
        o0.w = u.m[0] * x.w + u.m[1] * x.z + u.m[2] * y.w + u.m[3] * y.z;
        o1.z = u.m[4] * x.z - u.m[5] * x.w + u.m[6] * y.z - u.m[7] * y.w;
        o1.w = u.m[4] * x.w + u.m[5] * x.z + u.m[6] * y.w + u.m[7] * y.z;
        a4[i0] = o0;
        a4[i0 + half] = o1;
    }
}

// complex64, q == 0: one float4 holds a whole pair.
__global__ void k_dense1_c64q0(float4 *__restrict__ a4, uint64_t npairs, Mat2<float> u)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
        float4 v = a4[p];
        float4 o;
        o.x = u.m[0] * v.x - u.m[1] * v.y + u.m[2] * v.z - u.m[3] * v.w;
        o.y = u.m[0] * v.y + u.m[1] * v.x + u.m[2] * v.w + u.m[3] * v.z;
        o.z = u.m[4] * v.x - u.m[5] * v.y + u.m[6] * v.z - u.m[7] * v.w;
        o.w = u.m[4] * v.y + u.m[5] * v.x + u.m[6] * v.w + u.m[7] * v.z;
        a4[p] = o;
    }
}

// ----- phase on the amplitudes whose bits in `mask` are all set ------------
// (T: mask = {q}; CZ, CPHASE: mask = {a, b}).  Iterates over exactly those
// amplitudes: index = j with zero bits inserted at the mask positions, then
// the mask ORed in.
template <typename R>
__global__ void k_phase_sel(typename V2T<R>::T *__restrict__ a, int qa, int qb, uint64_t count,
                            R pre, R pim, int negate_only)
{
    using V = typename V2T<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t set = (1ULL << qa);
    if (qb >= 0) set |= 1ULL << qb;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
        uint64_t i = insert_zero(j, qa);
        if (qb >= 0) i = insert_zero(i, qb);
        i |= set;
        if (!QS_DCHECK(i < (count << (qb >= 0 ? 2 : 1)), 103)) continue;
        V v = a[i];
        if (negate_only) {
            v.x = -v.x; v.y = -v.y;
        } else {
            R x = v.x * pre - v.y * pim;
            v.y = v.x * pim + v.y * pre;
            v.x = x;
        }
        a[i] = v;
    }
}

// ----- full diagonal on one qubit: d0 on bit 0, d1 on bit 1 (RZ) -----------
template <typename R>
__global__ void k_diag1(typename V2T<R>::T *__restrict__ a, int q, uint64_t N, R d0r, R d0i, R d1r, R d1i)
{
    using V = typename V2T<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        bool one = (i >> q) & 1;
        R dr = one ? d1r : d0r, di = one ? d1i : d0i;
        V v = a[i];
        R x = v.x * dr - v.y * di;
        v.y = v.x * di + v.y * dr;
        v.x = x;
        a[i] = v;
    }
}

// ----- |0...0> ---------------------------------------------------------------
template <typename R>
__global__ void k_set_basis0(typename V2T<R>::T *a)
{
    a[0].x = (R)1;
    a[0].y = (R)0;
}

qs_status launch_init_zero(qs_state *s)
{
    ++s->version;
    const size_t bytes = (size_t(1) << s->n) * dtype_bytes(s->dt);
    QS_CUDA_TRY(cudaMemsetAsync(s->amps, 0, bytes, s->stream));
    if (s->dt == QS_C64)
        k_set_basis0<float><<<1, 1, 0, s->stream>>>((float2 *)s->amps);
    else
        k_set_basis0<double><<<1, 1, 0, s->stream>>>((double2 *)s->amps);
    QS_LAUNCH_CHECK();
    return QS_OK;
}

// H on every qubit of |0...0>: the uniform superposition, two complex64 (or
// one complex128) amplitudes per 16-byte store.
template <typename R>
__global__ void k_fill_uniform(float4 *a, uint64_t units, R v)
{
    float4 u;
    if constexpr (sizeof(R) == 4) {
        u = make_float4(v, 0.f, v, 0.f);
    } else {
        const double2 d = make_double2(v, 0.0);
        u = *reinterpret_cast<const float4 *>(&d);
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < units; i += stride) a[i] = u;
}

qs_status launch_init_uniform(qs_state *s)
{
    ++s->version;
    const uint64_t N = 1ULL << s->n;
    const double v = std::pow(2.0, -0.5 * s->n);
    const int th = 256;
    if (s->dt == QS_C64 && N >= 2) {
        const uint64_t units = N / 2;
        k_fill_uniform<float><<<grid_for(units, th, s->num_sms, 16), th, 0, s->stream>>>((float4 *)s->amps, units,
                                                                                      (float)v);
    } else if (s->dt == QS_C64) {
        const float2 one = make_float2((float)v, 0.f);
        QS_CUDA_TRY(cudaMemcpyAsync(s->amps, &one, sizeof one, cudaMemcpyHostToDevice, s->stream));
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    } else {
        k_fill_uniform<double><<<grid_for(N, th, s->num_sms, 16), th, 0, s->stream>>>((float4 *)s->amps, N, v);
    }
    QS_LAUNCH_CHECK();
    return QS_OK;
}

template <typename R>
static qs_status plain_gate_t(qs_state *s, const qs_gate &g)
{
    using V = typename V2T<R>::T;
    V *a = (V *)s->amps;
    const int n = s->n;
    const uint64_t N = 1ULL << n;
    const int th = 256;
    Cplx u[4];
    gate_matrix(g.kind, g.theta, u);
    switch (g.kind) {
    case QS_H: case QS_X_HALF: case QS_Y_HALF: case QS_RX: case QS_RY: {
        const int q = g.q0;
        Mat2<R> m;
        for (int e = 0; e < 4; ++e) { m.m[2 * e] = (R)u[e].re; m.m[2 * e + 1] = (R)u[e].im; }
        if (sizeof(R) == 4 && n >= 2) {
            Mat2<float> mf;
            for (int e = 0; e < 8; ++e) mf.m[e] = (float)m.m[e];
            if (q == 0)
                k_dense1_c64q0<<<grid_for(N / 2, th, s->num_sms), th, 0, s->stream>>>(
                    (float4 *)s->amps, N / 2, mf);
            else
                k_dense1_c64v<<<grid_for(N / 4, th, s->num_sms), th, 0, s->stream>>>(
                    (float4 *)s->amps, q, N / 4, mf);
        } else {
            k_dense1<R><<<grid_for(N / 2, th, s->num_sms), th, 0, s->stream>>>(a, q, N / 2, m);
        }
        break;
    }
    case QS_T:
        k_phase_sel<R><<<grid_for(N / 2, th, s->num_sms), th, 0, s->stream>>>(
            a, g.q0, -1, N / 2, (R)u[3].re, (R)u[3].im, 0);
        break;
    case QS_CZ: case QS_CPHASE: {
        int lo = g.q0 < g.q1 ? g.q0 : g.q1, hi = g.q0 < g.q1 ? g.q1 : g.q0;
        k_phase_sel<R><<<grid_for(N / 4, th, s->num_sms), th, 0, s->stream>>>(
            a, lo, hi, N / 4, (R)u[3].re, (R)u[3].im, g.kind == QS_CZ);
        break;
    }
    case QS_RZ:
        k_diag1<R><<<grid_for(N, th, s->num_sms), th, 0, s->stream>>>(
            a, g.q0, N, (R)u[0].re, (R)u[0].im, (R)u[3].re, (R)u[3].im);
        break;
    default:
        return set_error(QS_ERR_INVALID_ARG, "unknown gate kind %d", g.kind);
    }
    QS_LAUNCH_CHECK();
    return QS_OK;
}

qs_status launch_plain_gate(qs_state *s, const qs_gate &g)
{
    return s->dt == QS_C64 ? plain_gate_t<float>(s, g) : plain_gate_t<double>(s, g);
}

QS_CHECK_READER(check_poll_plain)

}  // namespace qs
