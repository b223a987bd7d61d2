// qs_fused.cu -- fused tile pass on CUDA cores.
//
// GB300 analogue of the appendix's cache blocking ("Quantum Simulation
// Details": operate on groups of consecutive gates that update a small part
// of the state held in a fast memory), moved from the CPU's last-level cache
// to each SM's shared memory and registers:
//
//   * A pass keeps t qubits local (the planner's tile set L; the c lowest
//     qubits are always in it so that global accesses are contiguous runs).
//     CTA tau owns the 2^t amplitudes whose out-of-tile qubits spell tau, so
//     tiles are disjoint and the pass runs in place.  Because each tile may
//     gather any qubits, a high qubit becomes local without moving data: the
//     qubit-to-tile-bit map of the pass is the remapping step.
//   * The tile is copied to shared memory with 16-byte cp.async transfers.
//   * A phase holds 2^RB amplitudes per thread in registers, spanning RB
//     chosen tile bits; the phase's gates run on them: non-diagonal gates on
//     register bits, diagonal gates (T, CZ, RZ, CPHASE) on any qubit, since a
//     qubit outside the register set has a value fixed per thread (tile bits)
//     or per tile (global bits).  The appendix's gate specialisation is kept:
//     H, X^1/2 and Y^1/2 are applied as additions with the common 1/sqrt2
//     factors deferred to one multiply at the end of the pass; CZ is a sign
//     flip; T a phase on half of the amplitudes.
//   * Shared memory uses a 16-byte-granular XOR swizzle (linear over GF(2),
//     so slot addresses are XORs of per-bit offsets) to spread the strided
//     phase accesses over the banks.
#include "qs_device.cuh"

namespace qs {

namespace {

constexpr int kThreadsMax = 256;

// Swizzled shared-memory index of tile element e: elements are grouped in
// 16-byte units u = e / CE; bits 0..2 of u are XORed with a fold of its
// higher bits.  Linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).
template <int CE>
__host__ __device__ __forceinline__ uint32_t swz(uint32_t e)
{
    uint32_t u = e / CE;
    uint32_t f = ((u >> 3) ^ (u >> 6) ^ (u >> 9) ^ (u >> 12)) & 7u;
    return e ^ (f * CE);
}

// ---- register-bit operations (J = register bit, compile time) -------------
template <int NS, int J, typename V>
__device__ __forceinline__ void reg_h(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) {
            V x = a[s], y = a[s | (1 << J)];
            a[s].x = x.x + y.x; a[s].y = x.y + y.y;
            a[s | (1 << J)].x = x.x - y.x; a[s | (1 << J)].y = x.y - y.y;
        }
}

// [[1, -i], [-i, 1]]
template <int NS, int J, typename V>
__device__ __forceinline__ void reg_xh(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) {
            V x = a[s], y = a[s | (1 << J)];
            a[s].x = x.x + y.y; a[s].y = x.y - y.x;
            a[s | (1 << J)].x = y.x + x.y; a[s | (1 << J)].y = y.y - x.x;
        }
}

// [[1, -1], [1, 1]]
template <int NS, int J, typename V>
__device__ __forceinline__ void reg_yh(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) {
            V x = a[s], y = a[s | (1 << J)];
            a[s].x = x.x - y.x; a[s].y = x.y - y.y;
            a[s | (1 << J)].x = x.x + y.x; a[s | (1 << J)].y = x.y + y.y;
        }
}

template <int NS, int J, typename V, typename R>
__device__ __forceinline__ void reg_dense(V *a, const R *m)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) {
            V x = a[s], y = a[s | (1 << J)];
            V o0, o1;
            o0.x = m[0] * x.x - m[1] * x.y + m[2] * y.x - m[3] * y.y;
            o0.y = m[0] * x.y + m[1] * x.x + m[2] * y.y + m[3] * y.x;
            o1.x = m[4] * x.x - m[5] * x.y + m[6] * y.x - m[7] * y.y;
            o1.y = m[4] * x.y + m[5] * x.x + m[6] * y.y + m[7] * y.x;
            a[s] = o0;
            a[s | (1 << J)] = o1;
        }
}

// Phase / sign on the slots whose register bits include all of M.
template <int NS, int M, typename V, typename R>
__device__ __forceinline__ void reg_phase(V *a, R pr, R pi)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if ((s & M) == M) {
            R x = a[s].x * pr - a[s].y * pi;
            a[s].y = a[s].x * pi + a[s].y * pr;
            a[s].x = x;
        }
}

template <int NS, int M, typename V>
__device__ __forceinline__ void reg_neg(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if ((s & M) == M) { a[s].x = -a[s].x; a[s].y = -a[s].y; }
}

#define QS_CASE_BIT(J, CALL) case J: CALL(J); break;

template <int RB, typename V, typename R>
__device__ __forceinline__ void dispatch_bit_op(int type, int j, V *a, const R *m)
{
    constexpr int NS = 1 << RB;
#define QS_H_(J) reg_h<NS, (J < RB ? J : 0)>(a)
#define QS_X_(J) reg_xh<NS, (J < RB ? J : 0)>(a)
#define QS_Y_(J) reg_yh<NS, (J < RB ? J : 0)>(a)
#define QS_D_(J) reg_dense<NS, (J < RB ? J : 0)>(a, m)
    switch (type) {
    case OP_H: switch (j) { QS_CASE_BIT(0, QS_H_) QS_CASE_BIT(1, QS_H_) QS_CASE_BIT(2, QS_H_)
                            QS_CASE_BIT(3, QS_H_) QS_CASE_BIT(4, QS_H_) QS_CASE_BIT(5, QS_H_) } break;
    case OP_XH: switch (j) { QS_CASE_BIT(0, QS_X_) QS_CASE_BIT(1, QS_X_) QS_CASE_BIT(2, QS_X_)
                             QS_CASE_BIT(3, QS_X_) QS_CASE_BIT(4, QS_X_) QS_CASE_BIT(5, QS_X_) } break;
    case OP_YH: switch (j) { QS_CASE_BIT(0, QS_Y_) QS_CASE_BIT(1, QS_Y_) QS_CASE_BIT(2, QS_Y_)
                             QS_CASE_BIT(3, QS_Y_) QS_CASE_BIT(4, QS_Y_) QS_CASE_BIT(5, QS_Y_) } break;
    case OP_DENSE: switch (j) { QS_CASE_BIT(0, QS_D_) QS_CASE_BIT(1, QS_D_) QS_CASE_BIT(2, QS_D_)
                                QS_CASE_BIT(3, QS_D_) QS_CASE_BIT(4, QS_D_) QS_CASE_BIT(5, QS_D_) } break;
    default: break;
    }
#undef QS_H_
#undef QS_X_
#undef QS_Y_
#undef QS_D_
}

#define QS_M4(B, F) F(B + 0) F(B + 1) F(B + 2) F(B + 3)
#define QS_M16(B, F) QS_M4(B, F) QS_M4(B + 4, F) QS_M4(B + 8, F) QS_M4(B + 12, F)
#define QS_M32(F) QS_M16(0, F) QS_M16(16, F)

template <int RB, typename V, typename R>
__device__ __forceinline__ void dispatch_mask_phase(int mask, V *a, R pr, R pi)
{
    constexpr int NS = 1 << RB;
#define QS_PC(M) case M: reg_phase<NS, (M) & (NS - 1)>(a, pr, pi); break;
    switch (mask) { QS_M32(QS_PC) default: break; }
#undef QS_PC
}

template <int RB, typename V>
__device__ __forceinline__ void dispatch_mask_neg(int mask, V *a)
{
    constexpr int NS = 1 << RB;
#define QS_NC(M) case M: reg_neg<NS, (M) & (NS - 1)>(a); break;
    switch (mask) { QS_M32(QS_NC) default: break; }
#undef QS_NC
}

// Deposits the low bits of x into the positions listed in pos[0..cnt).
__device__ __forceinline__ uint64_t deposit(uint64_t x, const uint8_t *pos, int cnt)
{
    uint64_t r = 0;
    for (int i = 0; i < cnt; ++i) r |= ((x >> i) & 1ULL) << pos[i];
    return r;
}

}  // namespace

// One launch = one pass over the state.  blockDim.x = 2^(t - RB).
template <typename R, int RB>
__global__ void __launch_bounds__(kThreadsMax, 2)
k_fused_pass(typename V2T<R>::T *__restrict__ amps, const DevPass *__restrict__ pass_g,
             const DevPhase *__restrict__ phases_g, const DevOp *__restrict__ ops_g,
             uint64_t ntiles)
{
    using V = typename V2T<R>::T;
    constexpr int NS = 1 << RB;                 // register slots per thread
    constexpr int CE = 16 / (int)sizeof(V);     // elements per 16-byte unit
    constexpr int CPT = NS / CE;                // 16-byte units per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);
    __shared__ DevPass P;
    __shared__ uint64_t it_off[CPT];

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    for (int i = tid; i < (int)(sizeof(DevPass) / 4); i += nthr)
        reinterpret_cast<uint32_t *>(&P)[i] = reinterpret_cast<const uint32_t *>(pass_g)[i];
    __syncthreads();
    const int t = P.t;
    const int ng = P.n - t;                     // out-of-tile qubits
    // qubit offset of the 16-byte units handled by this thread
    for (int i = tid; i < CPT; i += nthr) it_off[i] = deposit((uint64_t)(CE * nthr) * i, P.L, t);
    const uint64_t tid_off = deposit((uint64_t)CE * tid, P.L, t);
    __syncthreads();

    const R gsr = (R)P.gscale_re, gsi = (R)P.gscale_im;
    const bool gscale_one = (P.gscale_re == 1.0 && P.gscale_im == 0.0);
    const bool gscale_real = (P.gscale_im == 0.0);

    for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
        const uint64_t base = deposit(tau, P.G, ng);
        // ---- load the tile (16-byte cp.async, coalesced runs) ----
#pragma unroll
        for (int it = 0; it < CPT; ++it) {
            uint32_t e = (uint32_t)(CE * (it * nthr + tid));
            const V *src = amps + (base | tid_off | it_off[it]);
            uint32_t saddr = (uint32_t)__cvta_generic_to_shared(tile + swz<CE>(e));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(src)
                         : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();

        for (int ph = 0; ph < P.nphases; ++ph) {
            const DevPhase PH = phases_g[P.phase_begin + ph];
            // thread bits: tile bits outside the register set, ascending
            uint32_t e_th = 0;
            uint64_t q_th = 0;
            {
                uint32_t regmask = 0;
#pragma unroll
                for (int j = 0; j < RB; ++j) regmask |= 1u << PH.R[j];
                int k = 0;
                for (int b = 0; b < t; ++b) {
                    if ((regmask >> b) & 1u) continue;
                    uint32_t bitv = (tid >> k) & 1u;
                    e_th |= bitv << b;
                    q_th |= (uint64_t)bitv << P.L[b];
                    ++k;
                }
            }
            const uint64_t idx_th = base | q_th;
            const uint32_t p_th = swz<CE>(e_th);
            uint32_t pb[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) pb[j] = swz<CE>(1u << PH.R[j]);
            V a[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uint32_t off = 0;
#pragma unroll
                for (int j = 0; j < RB; ++j)
                    if ((s >> j) & 1) off ^= pb[j];
                a[s] = tile[p_th ^ off];
            }
            for (int o = PH.op_begin; o < PH.op_end; ++o) {
                const DevOp *op = ops_g + o;
                const int type = __ldg(&op->type);
                if (type == OP_PHASE || type == OP_NEG) {
                    const uint64_t qm = __ldg(&op->qmask);
                    if ((idx_th & qm) != qm) continue;
                    const int rm = __ldg(&op->rmask);
                    if (type == OP_NEG)
                        dispatch_mask_neg<RB>(rm, a);
                    else
                        dispatch_mask_phase<RB>(rm, a, (R)__ldg(&op->m[0]), (R)__ldg(&op->m[1]));
                } else {
                    R m[8];
                    if (type == OP_DENSE) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) m[e] = (R)__ldg(&op->m[e]);
                    }
                    dispatch_bit_op<RB>(type, __ldg(&op->a), a, m);
                }
            }
            if (ph == P.nphases - 1 && !gscale_one) {
                if (gscale_real) {
#pragma unroll
                    for (int s = 0; s < NS; ++s) { a[s].x *= gsr; a[s].y *= gsr; }
                } else {
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        R x = a[s].x * gsr - a[s].y * gsi;
                        a[s].y = a[s].x * gsi + a[s].y * gsr;
                        a[s].x = x;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uint32_t off = 0;
#pragma unroll
                for (int j = 0; j < RB; ++j)
                    if ((s >> j) & 1) off ^= pb[j];
                tile[p_th ^ off] = a[s];
            }
            __syncthreads();
        }
        // ---- store the tile ----
#pragma unroll
        for (int it = 0; it < CPT; ++it) {
            uint32_t e = (uint32_t)(CE * (it * nthr + tid));
            const float4 v = *reinterpret_cast<const float4 *>(tile + swz<CE>(e));
            *reinterpret_cast<float4 *>(amps + (base | tid_off | it_off[it])) = v;
        }
        __syncthreads();
    }
}

template <typename R, int RB>
static qs_status run_fused_t(qs_state *s, const Plan &plan, const void *dev_plan)
{
    using V = typename V2T<R>::T;
    const DevPass *dpass = reinterpret_cast<const DevPass *>(dev_plan);
    const DevPhase *dphase = reinterpret_cast<const DevPhase *>(dpass + plan.passes.size());
    const DevOp *dops = reinterpret_cast<const DevOp *>(dphase + plan.phases.size());
    auto kern = k_fused_pass<R, RB>;
    for (size_t p = 0; p < plan.passes.size(); ++p) {
        const DevPass &hp = plan.passes[p];
        if (hp.r != RB || hp.t < RB || hp.t - RB > 8)
            return set_error(QS_ERR_INVALID_ARG, "pass %zu: tile %d / register bits %d unsupported",
                             p, hp.t, hp.r);
        const int threads = 1 << (hp.t - RB);
        const size_t smem = (size_t(1) << hp.t) * sizeof(V);
        QS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const uint64_t ntiles = 1ULL << (plan.n - hp.t);
        const uint64_t cap = (uint64_t)s->num_sms * 2;
        const int grid = (int)(ntiles < cap ? ntiles : cap);
        kern<<<grid, threads, smem, s->stream>>>((V *)s->amps, dpass + p, dphase, dops, ntiles);
        QS_LAUNCH_CHECK();
    }
    return QS_OK;
}

qs_status run_fused_plan(qs_state *s, const Plan &plan, const void *dev_plan)
{
    if (s->dt == QS_C64) return run_fused_t<float, 5>(s, plan, dev_plan);
    return run_fused_t<double, 4>(s, plan, dev_plan);
}

}  // namespace qs
