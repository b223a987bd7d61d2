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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "qs_device.cuh"
#include "qs_stats_device.cuh"

namespace qs {

namespace {

constexpr int kThreadsMax = 256;

// Compact op record staged in shared memory once per CTA; one flat code per
// op so the interpreter takes a single indirect branch per op.
enum : uint32_t {
    K_H = 0, K_XH = 8, K_YH = 16, K_SHX = 24,     // + register bit
    K_SHY = 160,                                   // + register bit
    K_T = 32,                                      // + register mask (1..31): T phase
    K_NEG = 64,                                    // + register mask: sign flip
    K_PH = 96,                                     // + register mask: general phase
    K_UT = 128, K_UNEG = 129, K_UPH = 130,         // thread-uniform selection
    K_COND = 256                                   // flag: selection has qubits
                                                   // outside the register set
};


// Swizzled shared-memory index of tile element e: elements are grouped in
// 16-byte units u = e / CE; bits 0..2 of u are XORed with a fold of its
// higher bits.  Linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).
template <int CE>
__host__ __device__ __forceinline__ uint32_t swz(uint32_t e)
{
    return tile_swizzle(e, CE);
}

// ---- register-bit operations (J = register bit, compile time) -------------
// Every update is written in place (each output overwrites one input and no
// temporary is live across it), so the op interpreter keeps the slots in
// fixed registers.  For the deferred-scale butterflies the second output is
// formed from the first: H: x' = x + y, y' = x' - 2y (= x - y); Y^1/2:
// x' = x - y, y' = x' + 2y (= x + y); X^1/2: x' = x - i y, y' = y - i x with
// the same trick per component.  complex64 uses the packed FP32x2
// instructions of sm_100+ where both components see the same operation.
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ void bf_h(float2 &x, float2 &y)
{
    x = __fadd2_rn(x, y);
    y = __ffma2_rn(y, make_float2(-2.f, -2.f), x);
}
__device__ __forceinline__ void bf_h(double2 &x, double2 &y)
{
    x.x += y.x; x.y += y.y;
    y.x = fma(y.x, -2.0, x.x); y.y = fma(y.y, -2.0, x.y);
}
__device__ __forceinline__ void bf_yh(float2 &x, float2 &y)
{
    x = __ffma2_rn(y, make_float2(-1.f, -1.f), x);
    y = __ffma2_rn(y, make_float2(2.f, 2.f), x);
}
__device__ __forceinline__ void bf_yh(double2 &x, double2 &y)
{
    x.x -= y.x; x.y -= y.y;
    y.x = fma(y.x, 2.0, x.x); y.y = fma(y.y, 2.0, x.y);
}
template <typename V>
__device__ __forceinline__ void bf_xh(V &x, V &y)
{
    x.x = x.x + y.y;               // x'r = xr + yi
    y.y = fmaR(y.y, (decltype(y.y))2, -x.x);   // y'i = yi - xr
    x.y = x.y - y.x;               // x'i = xi - yr
    y.x = fmaR(y.x, (decltype(y.x))2, x.y);    // y'r = yr + xi
}
// multiply by c (1 + i), c = 1/sqrt2 (the T phase), in place
template <typename V, typename R>
__device__ __forceinline__ void ph_t(V &v, R c)
{
    v.x = v.x * c;
    v.x = fmaR(v.y, -c, v.x);      // c re - c im
    v.y = fmaR(v.y, 2 * c, v.x);   // c re + c im
}
template <typename V, typename R>
__device__ __forceinline__ void ph_gen(V &v, R pr, R pi)
{
    const R x = v.x;
    v.x = fmaR(v.x, pr, -v.y * pi);
    v.y = fmaR(x, pi, v.y * pr);
}

template <int NS, int J, typename V>
__device__ __forceinline__ void reg_h(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) bf_h(a[s], a[s | (1 << J)]);
}

template <int NS, int J, typename V>
__device__ __forceinline__ void reg_xh(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) bf_xh(a[s], a[s | (1 << J)]);
}

template <int NS, int J, typename V>
__device__ __forceinline__ void reg_yh(V *a)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) bf_yh(a[s], a[s | (1 << J)]);
}

__device__ __forceinline__ void axpy(float2 &x, const float2 &y, float k)
{
    x = __ffma2_rn(y, make_float2(k, k), x);
}
__device__ __forceinline__ void axpy(double2 &x, const double2 &y, double k)
{
    x.x = fma(y.x, k, x.x); x.y = fma(y.y, k, x.y);
}
// Shear on register bit J: x += k y (WHICH = 0) or y += k x (WHICH = 1),
// x the slot with the bit clear, y its partner.
template <int NS, int J, int WHICH, typename V, typename R>
__device__ __forceinline__ void reg_shear(V *a, R k)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & (1 << J))) {
            if (WHICH == 0) axpy(a[s], a[s | (1 << J)], k);
            else axpy(a[s | (1 << J)], a[s], k);
        }
}

// Phase on the slots whose register bits include all of M.  `tgate` selects
// the in-place T form (pr = pi = 1/sqrt2).
template <int NS, int M, typename V, typename R>
__device__ __forceinline__ void reg_phase(V *a, R pr, R pi, bool tgate)
{
    if (tgate) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if ((s & M) == M) ph_t(a[s], pr);
    } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if ((s & M) == M) ph_gen(a[s], pr, pi);
    }
}

__device__ __forceinline__ void mul_sign(float2 &v, float sg) { v = __fmul2_rn(v, make_float2(sg, sg)); }
__device__ __forceinline__ void mul_sign(double2 &v, double sg) { v.x *= sg; v.y *= sg; }

template <int NS, int M, typename V, typename R>
__device__ __forceinline__ void reg_sign(V *a, R sg)
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if ((s & M) == M) mul_sign(a[s], sg);
}


// Trailing zeros of a positive integer known at compile time (the callers
// use it on unrolled loop indices, so it folds to a constant).
template <int X> struct CtzT { static constexpr int value = (X & 1) ? 0 : 1 + CtzT<(X >> 1)>::value; };
template <> struct CtzT<0> { static constexpr int value = 0; };

// Loads / stores the register slots of a phase from / to the shared tile,
// visiting slots in Gray-code order so that each address differs from the
// previous one by one register bit (one XOR with that bit's offset); the two
// halves of the slots run as two interleaved chains.
// COUNT slots (or slot pairs when SHIFT = 1: register bit 0 is tile bit 0,
// so slots s and s+1 are one 16-byte unit).
template <int COUNT, int SHIFT>
struct SlotIO {
    // offsets are in bytes from the start of the tile
    // two Gray-code chains, one per half of the slots (top register bit
    // clear / set): half the dependent address XORs per load sequence
    static constexpr int kTop = CtzT<COUNT>::value - 1;
    template <int I, typename V>
    struct Step2 {
        static __device__ __forceinline__ void ld(V *a, const char *tile, uint32_t o0, uint32_t o1, const uint32_t *pb)
        {
            if (I) { o0 ^= pb[SHIFT + CtzT<I>::value]; o1 ^= pb[SHIFT + CtzT<I>::value]; }
            constexpr int s0 = (I ^ (I >> 1)) << SHIFT;
            constexpr int s1 = s0 + ((COUNT / 2) << SHIFT);
            if (SHIFT) {
                const float4 v = *reinterpret_cast<const float4 *>(tile + o0);
                const float4 w = *reinterpret_cast<const float4 *>(tile + o1);
                a[s0].x = v.x; a[s0].y = v.y; a[s0 + 1].x = v.z; a[s0 + 1].y = v.w;
                a[s1].x = w.x; a[s1].y = w.y; a[s1 + 1].x = w.z; a[s1 + 1].y = w.w;
            } else {
                a[s0] = *reinterpret_cast<const V *>(tile + o0);
                a[s1] = *reinterpret_cast<const V *>(tile + o1);
            }
            Step2<I + 1, V>::ld(a, tile, o0, o1, pb);
        }
        static __device__ __forceinline__ void st(const V *a, char *tile, uint32_t o0, uint32_t o1, const uint32_t *pb)
        {
            if (I) { o0 ^= pb[SHIFT + CtzT<I>::value]; o1 ^= pb[SHIFT + CtzT<I>::value]; }
            constexpr int s0 = (I ^ (I >> 1)) << SHIFT;
            constexpr int s1 = s0 + ((COUNT / 2) << SHIFT);
            if (SHIFT) {
                *reinterpret_cast<float4 *>(tile + o0) = make_float4(a[s0].x, a[s0].y, a[s0 + 1].x, a[s0 + 1].y);
                *reinterpret_cast<float4 *>(tile + o1) = make_float4(a[s1].x, a[s1].y, a[s1 + 1].x, a[s1 + 1].y);
            } else {
                *reinterpret_cast<V *>(tile + o0) = a[s0];
                *reinterpret_cast<V *>(tile + o1) = a[s1];
            }
            Step2<I + 1, V>::st(a, tile, o0, o1, pb);
        }
    };
    template <typename V>
    struct Step2<COUNT / 2, V> {
        static __device__ __forceinline__ void ld(V *, const char *, uint32_t, uint32_t, const uint32_t *) {}
        static __device__ __forceinline__ void st(const V *, char *, uint32_t, uint32_t, const uint32_t *) {}
    };
    template <typename V>
    static __device__ __forceinline__ void load(V *a, const char *tile, uint32_t off, const uint32_t *pb)
    { Step2<0, V>::ld(a, tile, off, off ^ pb[SHIFT + kTop], pb); }
    template <typename V>
    static __device__ __forceinline__ void store(const V *a, char *tile, uint32_t off, const uint32_t *pb)
    { Step2<0, V>::st(a, tile, off, off ^ pb[SHIFT + kTop], pb); }
};

// Executes one staged op on the register slots.  `sel` is the part of a
// diagonal op's selection outside the register set (true when the op has
// none); diagonal ops apply branch-free with sign / identity when unmet.
// FULL = false leaves out the cases of the parameterised gates (shears,
// general phases and T-valued phases on two register bits), which the
// Clifford+T circuits never stage; the smaller interpreter costs less
// instruction fetch per op.
template <int RB, bool FULL, typename V, typename R>
__device__ __forceinline__ void exec_op(uint32_t code, V *a, uint64_t idx_th, uint64_t qmask, R &fr,
                                        R &fi, const R *phase)
{
    constexpr int NS = 1 << RB;
    const R c = (R)0.70710678118654752440;
    // selection bits outside the register set (thread / tile constant); only
    // the diagonal cases read it
#define sel ((idx_th & qmask) == qmask)
#define QS_SGN (sel ? (R)-1 : (R)1)
#define QS_PR (sel ? phase[0] : (R)1)
#define QS_PI (sel ? phase[1] : (R)0)
    switch (code & ~K_COND) {
#define QS_B(J)                                                                  \
    case K_H + J: reg_h<NS, J>(a); break;                                        \
    case K_XH + J: reg_xh<NS, J>(a); break;                                      \
    case K_YH + J: reg_yh<NS, J>(a); break;                                      \
    case K_SHX + J: if (FULL) reg_shear<NS, J, 0>(a, phase[0]); break;                     \
    case K_SHY + J: if (FULL) reg_shear<NS, J, 1>(a, phase[0]); break;
    QS_B(0) QS_B(1) QS_B(2) QS_B(3)
#undef QS_B
#define QS_M(M)                                                                  \
    case K_T + M: if (FULL || !((M) & ((M) - 1))) reg_phase<NS, M>(a, c, c, true); break; \
    case K_NEG + M: reg_sign<NS, M>(a, QS_SGN); break;                           \
    case K_PH + M: if (FULL) reg_phase<NS, M>(a, QS_PR, QS_PI, false); break;
    // one- and two-qubit gates select at most two register bits
    QS_M(1) QS_M(2) QS_M(4) QS_M(8) QS_M(3) QS_M(5) QS_M(6) QS_M(9) QS_M(10) QS_M(12)
#undef QS_M
#define QS_B4(J)                                                                 \
    case K_H + J: reg_h<NS, (J < RB ? J : 0)>(a); break;                         \
    case K_XH + J: reg_xh<NS, (J < RB ? J : 0)>(a); break;                       \
    case K_YH + J: reg_yh<NS, (J < RB ? J : 0)>(a); break;                       \
    case K_SHX + J: if (FULL) reg_shear<NS, (J < RB ? J : 0), 0>(a, phase[0]); break;      \
    case K_SHY + J: if (FULL) reg_shear<NS, (J < RB ? J : 0), 1>(a, phase[0]); break;
#define QS_M4(M)                                                                 \
    case K_T + M: if (FULL || !((M) & ((M) - 1))) reg_phase<NS, ((M) & (NS - 1))>(a, c, c, true); break; \
    case K_NEG + M: reg_sign<NS, ((M) & (NS - 1))>(a, QS_SGN); break;            \
    case K_PH + M: if (FULL) reg_phase<NS, ((M) & (NS - 1))>(a, QS_PR, QS_PI, false); break;
    QS_B4(4) QS_M4(16) QS_M4(17) QS_M4(18) QS_M4(20) QS_M4(24)
#undef QS_B4
#undef QS_M4
    case K_UT: {
        // T on a selection outside the register set: f *= e^{i pi/4} if sel
        const R tr = sel ? c : (R)1, ti = sel ? c : (R)0;
        const R x = fr * tr - fi * ti;
        fi = fr * ti + fi * tr;
        fr = x;
        break;
    }
    case K_UNEG: fr *= QS_SGN; fi *= QS_SGN; break;
    case K_UPH: {
        const R pr = QS_PR, pi = QS_PI;
        const R x = fr * pr - fi * pi;
        fi = fr * pi + fi * pr;
        fr = x;
        break;
    }
    default: break;
    }
#undef QS_SGN
#undef QS_PR
#undef QS_PI
#undef sel
}

// ---- Clifford+T interpreter: one dense byte code per op ----
// The passes of the paper's circuits (H, X^1/2, Y^1/2, T, CZ) stage each op
// as one byte from a dense range, so the interpreter's dispatch is one byte
// load and one indexed branch; the one-op-per-case layout keeps the slots
// in fixed registers as in exec_op.
enum : uint32_t {
    C_H = 0, C_XH = 5, C_YH = 10,     // + register bit
    C_T = 15,                         // + register bit: T phase on the slots with the bit set
    C_CZ = 20,                        // + index of the register-bit pair (cz_pair_index)
    C_CZO = 30,                       // + register bit: sign on the slots with the bit set where
                                      //   the op's selection outside the register set holds
    C_Z = 35,                         // + register bit: unconditional sign
    C_COUNT = 40
};

// Pairs (j, k), j < k < 5, numbered (0,1) (0,2) (0,3) (0,4) (1,2) (1,3) ...
__host__ __device__ __forceinline__ int cz_pair_index(int j, int k)
{
    return j * 4 - (j * (j + 1)) / 2 + (k - 1);
}

template <int RB, typename V, typename R, typename OpT>
__device__ __forceinline__ void exec_ct(uint32_t code, V *a, uint64_t idx_th, const OpT *op)
{
    constexpr int NS = 1 << RB;
    const R c = (R)0.70710678118654752440;
    switch (code) {
#define QS_J(J)                                                                          \
    case C_H + J: reg_h<NS, (J < RB ? J : 0)>(a); break;                                 \
    case C_XH + J: reg_xh<NS, (J < RB ? J : 0)>(a); break;                               \
    case C_YH + J: reg_yh<NS, (J < RB ? J : 0)>(a); break;                               \
    case C_T + J: reg_phase<NS, (1 << (J < RB ? J : 0))>(a, c, c, true); break;          \
    case C_CZO + J: {                                                                    \
        const uint64_t qm = op->qmask;                                                   \
        reg_sign<NS, (1 << (J < RB ? J : 0))>(a, ((idx_th & qm) == qm) ? (R)-1 : (R)1);  \
        break;                                                                           \
    }                                                                                    \
    case C_Z + J: reg_sign<NS, (1 << (J < RB ? J : 0))>(a, (R)-1); break;
    QS_J(0) QS_J(1) QS_J(2) QS_J(3) QS_J(4)
#undef QS_J
#define QS_P(J, K) \
    case C_CZ + (J * 4 - (J * (J + 1)) / 2 + (K - 1)): reg_sign<NS, ((1 << J) | (1 << K)) & (NS - 1)>(a, (R)-1); break;
    QS_P(0, 1) QS_P(0, 2) QS_P(0, 3) QS_P(0, 4) QS_P(1, 2) QS_P(1, 3) QS_P(1, 4) QS_P(2, 3) QS_P(2, 4) QS_P(3, 4)
#undef QS_P
    default: break;
    }
}

// Byte code of a staged op in the Clifford+T interpreter, or -1 when the op
// needs the full interpreter (parameterised gates, general phases, a T
// phase selected outside the register set).  Thread-uniform diagonal ops
// (no register bits) run in the phase tail and get no code.
__host__ __device__ inline int ct_code(const DevOp &d)
{
    // lowest / highest set bit and count of the 8-bit register mask
    int lo = -1, hi = -1, bits = 0;
    for (int b = 0; b < 8; ++b)
        if ((d.rmask >> b) & 1) {
            if (lo < 0) lo = b;
            hi = b;
            ++bits;
        }
    switch (d.type) {
    case OP_H: return C_H + d.a;
    case OP_XH: return C_XH + d.a;
    case OP_YH: return C_YH + d.a;
    case OP_PHASE: {
        if (d.rmask == 0) return C_COUNT;          // tail
        const bool tphase = d.m[0] == d.m[1] && d.m[0] > 0.7071 && d.m[0] < 0.7072;
        if (!tphase || bits != 1 || d.qmask) return -1;
        return C_T + hi;
    }
    case OP_NEG: {
        if (d.rmask == 0) return C_COUNT;          // tail
        if (bits == 1) return (d.qmask ? C_CZO : C_Z) + hi;
        if (bits == 2 && !d.qmask) return C_CZ + cz_pair_index(lo, hi);
        return -1;
    }
    default: return -1;
    }
}

// Deposits the low bits of x into the positions listed in pos[0..cnt).
__device__ __forceinline__ uint64_t deposit(uint64_t x, const uint8_t *pos, int cnt)
{
    uint64_t r = 0;
    for (int i = 0; i < cnt; ++i) r |= ((x >> i) & 1ULL) << pos[i];
    return r;
}

}  // namespace

template <typename R>
struct SOp {
    uint32_t code;
    uint32_t aux;       // index into the staged phase / shear-factor table
    uint64_t qmask;     // qubit selection outside the register set
};

struct SPhase {
    uint32_t pb[kMaxRegBits];   // swizzled tile byte offset of each register bit
    int32_t op_begin, op_end;
    int32_t paired;             // register bit 0 is tile bit 0 (16-byte slots)
    int32_t uniform_begin;      // first op of the thread-uniform diagonal tail
    int32_t kind;               // 0 register phase, 1 tensor-core block phase
    int32_t slot;               // kind 1: slot of the block in tensor memory
    int32_t scale_exp;          // kind 1: FP16 operand scale 2^scale_exp
    int32_t pad;
};

// Tensor-core phase tables: swizzled tile offset of every block index and
// of every column index (the XOR swizzle is linear, so an element's offset
// is blk_off ^ col_off).
struct TcSmem {
    uint32_t blk_off[kMaxTcPerPass][64];
    uint32_t col_off[kMaxTcPerPass][128];
    uint64_t mbar;
    uint32_t tmem_base;
    int32_t abort;
};

struct SThread {
    uint32_t phys;              // swizzled tile byte offset of the thread's slot 0
    uint32_t pad;
    uint64_t qoff;              // qubit-index bits of the thread's tile bits
};

template <typename R, int RB>
struct FusedSmem {
    DevPass P;
    SPhase ph[kMaxPhasesPerPass];
    SOp<R> ops[kMaxOpsPerPass];
    R phase[kMaxOpsPerPass][2];
    uint8_t code8[kMaxOpsPerPass + 4];      // Clifford+T interpreter (FULL = false)
    SThread th[kMaxPhasesPerPass][kThreadsMax];
    uint64_t it_off[(1 << RB)];
    // diagonal prefix folded into the first pass's generated state
    // (FoldArgs): CZ partners of each qubit as a qubit mask and as a mask of
    // the tile bits holding them, T counts, the unit table and the eight
    // values uniform * e^{i pi k / 4}
    uint64_t fnb[kMaxQubits];
    uint64_t fm[3];
    uint16_t fg[kMaxQubits];
    uint8_t fu[(1 << RB)];
    typename V2T<R>::T fw[8];
};

// ---------------------------------------------------------------------------
// tensor-core block phase (tcgen05, complex64 tiles of 2^13 amplitudes)
//
// The 64 x 64 block unitary acts on the 6 block qubits of the tile for each
// of the 128 columns (values of the other 7 tile qubits).  Realified:
// D (128 x 128) = A (128 x 128) * B (128 x 128) with B[k][col] = re (k < 64)
// or im (k >= 64) of the tile amplitude (block index k mod 64, col).  Rows
// of A and D interleave the real and imaginary parts of the 64 output block
// rows, so neighbouring lanes of the epilogue store the two halves of one
// amplitude.  A and B are split into the terms of the operand precision
// (tc_prec: FP16 / BF16 / TF32, one to three terms) and the products of the
// terms whose combined order is below the term count are accumulated in
// FP32 in tensor memory: hi hi, hi lo, lo hi for two terms; all six pairs of
// order <= 2 for three.  FP16 values are first scaled by 2^14 / 2^ceil(d/2),
// d = deferred 1/sqrt2 factors pending in the tile: |value| <= 2^(d/2)
// ||psi||, so scaled values stay below the FP16 maximum (a power of two:
// exact); BF16 and TF32 carry FP32's exponent range and need no scale.
// A lives in tensor memory (loaded once per CTA), B in shared memory
// (canonical K-major layout without swizzle: 8 rows x 16-byte core
// matrices, 128 bytes apart along K, 16 cores apart along the 128 columns),
// D in tensor memory.  When A's terms fit 128 columns (FP16x3, BF16x3,
// TF32) a CTA holds 256 columns and B takes the tile's own shared buffer,
// so two CTAs share an SM and one CTA's tile traffic and MMA wait overlap
// the other's work; BF16x6 and TF32x3 hold 512 columns and B continues past
// the tile, one CTA per SM.
// ---------------------------------------------------------------------------
constexpr uint64_t kTcWaitNs = 1000000000ull;   // 1 s: far beyond 96 products of 128 x 128 x 16

// Compile-time layout of a precision (TCP = qs_precision value, 1..5).
template <int TCP>
struct TcCfg {
    static constexpr TcPrec P = tc_prec(TCP);
    static constexpr int kTerms = P.terms;
    static constexpr int kElem = P.elem_bytes;
    static constexpr int kAColsPerTerm = 128 * kElem / 4;         // tensor-memory columns
    static constexpr uint32_t kTmemCols = (128 + kTerms * kAColsPerTerm) <= 256 ? 256u : 512u;
    static constexpr int kCtasPerSm = kTmemCols == 256 ? 2 : 1;
    static constexpr int kBTermBytes = 128 * 128 * kElem;          // one term of B
    // B's terms start in the tile's own buffer (its amplitudes are in
    // registers while the terms are written) and continue into the dynamic
    // shared memory that follows the tile when they exceed its 64 KB
    static constexpr int kBExtraBytes = kTerms * kBTermBytes > 65536 ? kTerms * kBTermBytes - 65536 : 0;
    static constexpr int kKSteps = 128 / (32 / kElem);             // MMAs along K per product
    static constexpr uint32_t kSbo = 128u * (128 * kElem / 16);     // bytes between 8-column groups
    static constexpr int kProducts = kTerms == 3 ? 6 : (kTerms == 2 ? 3 : 1);
    // instruction descriptor: D FP32, A and B of the same format, K-major,
    // N = 128, M = 128
    static constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)P.fmt << 7) | ((uint32_t)P.fmt << 10) |
                                       ((128u >> 3) << 17) | ((128u >> 4) << 24);
};

// Dynamic shared memory of the tensor-core form: the tile, the part of B's
// terms beyond the tile's 64 KB, and the slack that aligns the tile to 1024
// bytes.
__host__ __device__ constexpr size_t tc_dyn_smem(int tcp)
{
    return 65536 +
           (tc_prec(tcp).terms * 128 * 128 * tc_prec(tcp).elem_bytes > 65536
                ? (size_t)tc_prec(tcp).terms * 128 * 128 * tc_prec(tcp).elem_bytes - 65536
                : 0) +
           1024;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;     // leading (K) byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;      // stride (column) byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    return d;
}

__device__ __forceinline__ void tmem_st32(uint32_t addr, const uint32_t *r)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(addr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr)
        : "memory");
}

// Allocates tensor memory, loads this pass's block matrices (warps 0-3: one
// row per thread, every term) and initialises the completion barrier.
template <int TCP>
__device__ __forceinline__ void tc_setup(TcSmem &TS, const DevPhase *phases, int nph,
                                         const uint32_t *tc_words)
{
    using C = TcCfg<TCP>;
    constexpr int kRowWords = C::kTerms * C::kAColsPerTerm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&TS.tmem_base)),
                     "r"(C::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&TS.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = TS.tmem_base;
    if (warp < 4) {
        const int m = warp * 32 + lane;
        int slot = 0;
        for (int ph = 0; ph < nph; ++ph) {
            if (phases[ph].kind != 1) continue;
            const uint32_t *w = tc_words + (size_t)phases[ph].tc_block * tc_words_per_block(TCP) +
                                (size_t)m * kRowWords;
            for (int c = 0; c < kRowWords / 32; ++c) {
                uint32_t r[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = __ldg(w + c * 32 + j);
                tmem_st32(tbase + ((uint32_t)(warp * 32) << 16) + 128 + kRowWords * slot + 32 * c, r);
            }
            ++slot;
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

template <int TCP>
__device__ __forceinline__ void tc_teardown(TcSmem &TS)
{
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(TS.tmem_base),
                     "r"(TcCfg<TCP>::kTmemCols));
    }
}

// Term t of a split: the operand type's rounding of what terms 0..t-1 leave.
// 16-bit formats work on pairs of values (one 32-bit word, lower value in
// the low half); TF32 on single values (the low 13 bits of the word zero).
template <int FMT>
__device__ __forceinline__ uint32_t split_pair(float &r0, float &r1)
{
    uint32_t w;
    float2 v;
    if (FMT == 0) {
        const __half2 h = __floats2half2_rn(r0, r1);
        w = *reinterpret_cast<const uint32_t *>(&h);
        v = __half22float2(h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
        w = *reinterpret_cast<const uint32_t *>(&h);
        v = __bfloat1622float2(h);
    }
    r0 -= v.x;
    r1 -= v.y;
    return w;
}

__device__ __forceinline__ uint32_t split_tf32(float &r)
{
    uint32_t w;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w) : "f"(r));
    r -= __uint_as_float(w);
    return w;
}

template <int TCP>
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc)
{
    if constexpr (TcCfg<TCP>::P.fmt == 2)
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
                     "r"(a), "l"(bdesc), "r"(TcCfg<TCP>::kIdesc), "r"(acc));
    else
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
                     "r"(a), "l"(bdesc), "r"(TcCfg<TCP>::kIdesc), "r"(acc));
}

// One block phase on the shared tile (all 256 threads).  Every thread first
// moves its 32 amplitudes (4 units of 8 block rows of one column) to
// registers, then writes their terms in the MMA layout (into the tile's own
// buffer and, past its 64 KB, the shared memory after it); after the
// products complete, the accumulator is scattered back into the tile.
template <int TCP>
__device__ __forceinline__ void tc_phase(TcSmem &TS, int slot, int scale_exp, float2 *tile,
                                         unsigned char *bbuf, uint32_t parity, int *err_flag)
{
    using C = TcCfg<TCP>;
    const float sc = C::P.scaled ? ldexpf(1.f, scale_exp) : 1.f;
    const float inv_sc = C::P.scaled ? ldexpf(1.f, -scale_exp) : 1.f;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t *blk = TS.blk_off[slot], *col = TS.col_off[slot];
    float2 xv[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int u = tid + 256 * i;
        const uint32_t base = col[u & 127] ^ blk[(u >> 7) * 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) xv[i][j] = tile[base ^ blk[j]];
    }
    __syncthreads();
    // ---- registers (FP32) -> B terms (canonical K-major layout) ----
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int u = tid + 256 * i;
        const int nu = u & 127, bg = u >> 7;
        float rr[8], ri[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { rr[j] = xv[i][j].x * sc; ri[j] = xv[i][j].y * sc; }
        if constexpr (C::kElem == 2) {
            // 8 block rows = one 16-byte core row of K; imaginary K + 64
            const uint32_t off_re = (uint32_t)(((nu >> 3) * 16 + bg) * 128 + (nu & 7) * 16);
            const uint32_t off_im = off_re + 8 * 128;
#pragma unroll
            for (int t = 0; t < C::kTerms; ++t) {
                uint32_t wr[4], wi[4];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    wr[j / 2] = split_pair<C::P.fmt>(rr[j], rr[j + 1]);
                    wi[j / 2] = split_pair<C::P.fmt>(ri[j], ri[j + 1]);
                }
                unsigned char *bt = bbuf + t * C::kBTermBytes;
                *reinterpret_cast<uint4 *>(bt + off_re) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
                *reinterpret_cast<uint4 *>(bt + off_im) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
            }
        } else {
            // TF32: 8 block rows = two 16-byte core rows of K (4 values each)
            const uint32_t off_re = (uint32_t)((nu >> 3) * C::kSbo + (2 * bg) * 128 + (nu & 7) * 16);
            const uint32_t off_im = off_re + 16 * 128;
#pragma unroll
            for (int t = 0; t < C::kTerms; ++t) {
                uint32_t wr[8], wi[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    wr[j] = split_tf32(rr[j]);
                    wi[j] = split_tf32(ri[j]);
                }
                unsigned char *bt = bbuf + t * C::kBTermBytes;
                *reinterpret_cast<uint4 *>(bt + off_re) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
                *reinterpret_cast<uint4 *>(bt + off_re + 128) = make_uint4(wr[4], wr[5], wr[6], wr[7]);
                *reinterpret_cast<uint4 *>(bt + off_im) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
                *reinterpret_cast<uint4 *>(bt + off_im + 128) = make_uint4(wi[4], wi[5], wi[6], wi[7]);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    const uint32_t tbase = TS.tmem_base;
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // products (A term, B term), smallest first within each K step
        constexpr int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
        constexpr int pa3[3] = {1, 0, 0}, pb3[3] = {0, 1, 0};
        const uint32_t a0 = tbase + 128 + (uint32_t)(C::kTerms * C::kAColsPerTerm * slot);
        const uint32_t sb = smem_addr(bbuf);
#pragma unroll
        for (int k = 0; k < C::kKSteps; ++k) {
#pragma unroll
            for (int q = 0; q < C::kProducts; ++q) {
                const int ta = C::kProducts == 6 ? pa[q] : (C::kProducts == 3 ? pa3[q] : 0);
                const int tb = C::kProducts == 6 ? pb[q] : (C::kProducts == 3 ? pb3[q] : 0);
                const uint64_t bd = tc_desc(sb + tb * C::kBTermBytes + 256 * k, C::kSbo);
                tc_mma<TCP>(tbase, a0 + ta * C::kAColsPerTerm + 8 * k, bd, (k > 0 || q > 0) ? 1u : 0u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&TS.mbar)));
    }
    // ---- bounded wait for the products ----
    {
        const uint32_t mb = smem_addr(&TS.mbar);
        if (!mbar_wait_bounded(mb, parity, kTcWaitNs)) {
            // give up on this launch: the products may still be in flight,
            // so wait once more (bounded) before the caller releases the
            // tensor memory, and skip the epilogue
            TS.abort = 1;
            atomicExch(err_flag, 1);
            mbar_wait_bounded(mb, parity, kTcWaitNs);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (TS.abort) return;
    // ---- D (TMEM) -> tile: warp w reads lanes 32 (w & 3) .., columns 64 (w >> 2) .. ----
    {
        const int m = 32 * (warp & 3) + lane;
        const uint32_t rowoff = blk[m >> 1];     // rows interleave re / im
        const int comp = m & 1;
        float *tf = reinterpret_cast<float *>(tile);
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const int c0 = 64 * (warp >> 2) + 32 * c;
            uint32_t r[32];
            tmem_ld32(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + c0, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j)
                tf[2 * (rowoff ^ col[c0 + j]) + comp] = C::P.scaled ? __uint_as_float(r[j]) * inv_sc
                                                                    : __uint_as_float(r[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
}

// complex64 slot <-> 64-bit word (re in the low half) for the PTX op loop
__device__ __forceinline__ unsigned long long f2_bits(float2 v)
{
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long b)
{
    return make_float2(__uint_as_float((uint32_t)b), __uint_as_float((uint32_t)(b >> 32)));
}

#include "qs_ct_asm.inc"

// Barrier of the threads that work on one tile: the whole CTA, or in the
// grouped form the tile's thread group (named barrier 1 + group for groups
// of whole warps, a warp-lane barrier for smaller groups).
template <bool GROUPED>
__device__ __forceinline__ void tile_sync(int nthr, int gi)
{
    if constexpr (!GROUPED) {
        __syncthreads();
    } else if (nthr >= 32) {
        asm volatile("bar.sync %0, %1;" ::"r"(gi + 1), "r"(nthr) : "memory");
    } else {
        const unsigned lane0 = (threadIdx.x & 31u) & ~(unsigned)(nthr - 1);
        __syncwarp((nthr == 32 ? 0xffffffffu : ((1u << nthr) - 1u)) << lane0);
    }
}

// One launch = one pass over the state.  blockDim.x = 2^(t - RB).
// TCP > 0: tensor-core variant of operand precision TCP (complex64, t = 13);
// its dynamic shared memory holds the tile (and a separate B buffer when
// the precision's B terms exceed the tile's 64 KB).
// Runs tiles [t_begin, t_end) of one pass on `amps`: stages the pass's
// phases and ops into shared memory, then loads, transforms and stores each
// tile.  Shared by the single-state kernel and the batched kernels.
// GROUPED: the CTA has kThreadsMax threads whatever the tile size; it splits
// into blockDim.x / 2^(t - RB) groups of 2^(t - RB) threads, each with its
// own tile buffer (2^t amplitudes at 2^t * group in the dynamic shared
// memory), and group g runs tiles t_begin + g, t_begin + g + groups, ...
// with its own barriers (the staged pass is shared).
template <typename R, int RB, int TCP, bool FULL, bool GROUPED = false>
__device__ __forceinline__ void fused_pass_body(typename V2T<R>::T *__restrict__ amps,
                                                const DevPass *__restrict__ pass_g,
                                                const DevPhase *__restrict__ phases_g,
                                                const DevOp *__restrict__ ops_g, uint64_t t_begin,
                                                uint64_t t_end, const uint32_t *__restrict__ tc_words,
                                                int *__restrict__ err_flag, FusedSmem<R, RB> &S, TcSmem &TS,
                                                unsigned char *smem_raw, R uniform = (R)0, bool folded = false)
{
    using V = typename V2T<R>::T;
    constexpr int NS = 1 << RB;                 // register slots per thread
    constexpr int CE = 16 / (int)sizeof(V);     // elements per 16-byte unit
    constexpr int CPT = NS / CE;                // 16-byte units per thread
    static_assert(!(GROUPED && TCP), "the grouped form has no tensor-core phases");
    V *tile = reinterpret_cast<V *>(smem_raw);

    for (int i = threadIdx.x; i < (int)(sizeof(DevPass) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&S.P)[i] = reinterpret_cast<const uint32_t *>(pass_g)[i];
    __syncthreads();
    const int t = S.P.t;
    const int ng = S.P.n - t;                   // out-of-tile qubits
    const int nph = S.P.nphases;
    // tile threads: the CTA, or one group of the grouped form
    const int nthr = GROUPED ? (1 << (t - RB)) : (int)blockDim.x;
    const int tid = GROUPED ? (int)(threadIdx.x & (unsigned)(nthr - 1)) : (int)threadIdx.x;
    const int gi = GROUPED ? (int)(threadIdx.x >> (t - RB)) : 0;
    const int ngr = GROUPED ? (int)(blockDim.x >> (t - RB)) : 1;
    // ---- stage phases, ops and per-thread phase tables (once per CTA) ----
    for (int ph = 0; ph < nph; ++ph) {
        const DevPhase &D = phases_g[S.P.phase_begin + ph];
        if (threadIdx.x == 0) {
            for (int j = 0; j < RB; ++j) S.ph[ph].pb[j] = swz<CE>(1u << D.R[j]) * (uint32_t)sizeof(V);
            S.ph[ph].op_begin = D.op_begin - phases_g[S.P.phase_begin].op_begin;
            S.ph[ph].op_end = D.op_end - phases_g[S.P.phase_begin].op_begin;
            S.ph[ph].paired = (CE == 2 && D.R[0] == 0) ? 1 : 0;
            S.ph[ph].kind = D.kind;
            // keep scaled values below 2^14 whatever the deferred factors
            S.ph[ph].scale_exp = 14 - (D.defer_before + 1) / 2;
            // the planner puts the thread-uniform diagonal ops last
            int ub = D.op_end;
            while (ub > D.op_begin && (ops_g[ub - 1].type == OP_PHASE || ops_g[ub - 1].type == OP_NEG) &&
                   ops_g[ub - 1].rmask == 0)
                --ub;
            S.ph[ph].uniform_begin = ub - phases_g[S.P.phase_begin].op_begin;
        }
        // thread-index bit k sits on tile bit T[k] (the planner picks the
        // lane bits that spread the phase's accesses over the banks)
        uint32_t e = 0;
        uint64_t q = 0;
        if (D.kind == 0) {
            for (int k = 0; k < t - RB; ++k) {
                const int b = D.T[k];
                const uint32_t bit = (tid >> k) & 1u;
                e |= bit << b;
                q |= (uint64_t)bit << S.P.L[b];
            }
        }
        if (gi == 0) {
            S.th[ph][tid].phys = swz<CE>(e) * (uint32_t)sizeof(V);
            S.th[ph][tid].qoff = q;
        }
    }
    int ntc = 0;
    if (TCP) {
        for (int ph = 0; ph < nph; ++ph) {
            const DevPhase &D = phases_g[S.P.phase_begin + ph];
            if (D.kind != 1) continue;
            if (tid == 0) S.ph[ph].slot = ntc;
            uint32_t bmask = 0;
            for (int j = 0; j < kTcBits; ++j) bmask |= 1u << D.R[j];
            if (tid < 64) {
                uint32_t e = 0;
                for (int j = 0; j < kTcBits; ++j) e |= (uint32_t)((tid >> j) & 1) << D.R[j];
                TS.blk_off[ntc][tid] = swz<CE>(e);
            }
            if (tid < 128) {
                uint32_t e = 0;
                for (int b = 0, k = 0; b < t; ++b) {
                    if ((bmask >> b) & 1u) continue;
                    e |= (uint32_t)((tid >> k) & 1) << b;
                    ++k;
                }
                TS.col_off[ntc][tid] = swz<CE>(e);
            }
            ++ntc;
        }
        if (tid == 0) TS.abort = 0;
        if constexpr (TCP > 0)
            if (ntc) tc_setup<TCP>(TS, phases_g + S.P.phase_begin, nph, tc_words);
    }
    {
        const int o0 = phases_g[S.P.phase_begin].op_begin;
        const int o1 = phases_g[S.P.phase_begin + nph - 1].op_end;
        for (int o = o0 + (int)threadIdx.x; o < o1; o += (int)blockDim.x) {
            const DevOp &d = ops_g[o];
            SOp<R> so;
            const bool tphase = d.type == OP_PHASE && d.m[0] == d.m[1] && d.m[0] > 0.7071 && d.m[0] < 0.7072;
            switch (d.type) {
            case OP_H: so.code = K_H + d.a; break;
            case OP_XH: so.code = K_XH + d.a; break;
            case OP_YH: so.code = K_YH + d.a; break;
            case OP_SHX: so.code = K_SHX + d.a; break;
            case OP_SHY: so.code = K_SHY + d.a; break;
            case OP_PHASE:
                so.code = d.rmask ? ((tphase ? K_T : K_PH) + d.rmask) : (tphase ? K_UT : K_UPH);
                break;
            default: so.code = d.rmask ? K_NEG + d.rmask : K_UNEG; break;
            }
            if (d.type == OP_PHASE || d.type == OP_NEG) {
                if (d.qmask) so.code |= K_COND;
            }
            so.aux = (uint32_t)(o - o0);
            so.qmask = d.qmask;
            if (!FULL) S.code8[o - o0] = (uint8_t)ct_code(d);
            S.phase[o - o0][0] = (R)d.m[0];
            S.phase[o - o0][1] = (R)d.m[1];
            S.ops[o - o0] = so;
        }
    }
    for (int i = threadIdx.x; i < CPT; i += blockDim.x) S.it_off[i] = deposit((uint64_t)(CE * nthr) * i, S.P.L, t);
    const uint64_t tid_off = deposit((uint64_t)CE * tid, S.P.L, t);
    // T count of qubit q (mod 8), for the folded diagonal prefix
    auto fcount = [&](int q) -> uint32_t {
        return (uint32_t)((S.fm[0] >> q) & 1) + 2u * (uint32_t)((S.fm[1] >> q) & 1) +
               4u * (uint32_t)((S.fm[2] >> q) & 1);
    };
    if (folded) {
        // each qubit's CZ partners as tile bits
        for (int q = threadIdx.x; q < S.P.n; q += blockDim.x) {
            uint32_t m = 0;
            for (int b = 0; b < t; ++b) m |= (uint32_t)((S.fnb[q] >> S.P.L[b]) & 1) << b;
            S.fg[q] = (uint16_t)m;
        }
        // unit u = (it, q) of every thread: tile element CE nthr it + q;
        // 4 (CZ pairs among its tile bits) + (its T counts), mod 8
        for (int u = threadIdx.x; u < CPT * CE; u += blockDim.x) {
            const uint32_t eu = (uint32_t)(CE * nthr) * (uint32_t)(u / CE) + (uint32_t)(u % CE);
            uint32_t pairs = 0, tcnt = 0;
            for (uint32_t w = eu; w; w &= w - 1) {
                const int qb = S.P.L[__ffs(w) - 1];
                for (uint32_t v = w & (w - 1); v; v &= v - 1) pairs += (uint32_t)(S.fnb[qb] >> S.P.L[__ffs(v) - 1]) & 1u;
                tcnt += fcount(qb);
            }
            S.fu[u] = (uint8_t)((4u * (pairs & 1u) + tcnt) & 7u);
        }
        // uniform * e^{i pi k / 4}: 2^(-n/2) and 2^(-n/2) / sqrt2 formed in
        // FP64 from n (the latter a power of two for odd n)
        if (threadIdx.x < 8) {
            const int k = (int)threadIdx.x;
            const double a = std::exp2(-0.5 * S.P.n), c = a * 0.70710678118654752440;
            const double re[8] = {a, c, 0.0, -c, -a, -c, 0.0, c};
            const double im[8] = {0.0, c, a, c, 0.0, -c, -a, -c};
            S.fw[k].x = (R)re[k];
            S.fw[k].y = (R)im[k];
        }
    }
    const R gsr = (R)S.P.gscale_re, gsi = (R)S.P.gscale_im;
    const bool gscale_one = (S.P.gscale_re == 1.0 && S.P.gscale_im == 0.0);
    __syncthreads();
    // the pass-wide factor rides on the last phase's registers when that is a
    // register phase; otherwise it is applied at the tile store
    const bool gs_in_phase = !gscale_one && S.ph[nph - 1].kind == 0;
    const bool gs_at_store = !gscale_one && !gs_in_phase;
    // this thread's tile buffer (the group's in the grouped form)
    unsigned char *gsm = GROUPED ? smem_raw + ((size_t)gi << t) * sizeof(V) : smem_raw;
    // tile element CE (it nthr + tid) sits at swizzled byte offset
    // sw_tid ^ swz(CE it nthr) (the swizzle is linear, the bits are disjoint)
    const uint32_t tile_sa = smem_addr(gsm);
    const uint32_t sw_tid = swz<CE>((uint32_t)(CE * tid)) * (uint32_t)sizeof(V);

    // the tile base (bits of the out-of-tile qubits) advances by a masked
    // increment over the contiguous tile range (grouped: deposited afresh,
    // the group's tiles being `ngr` apart)
    uint64_t gmask = 0;
    for (int i = 0; i < ng; ++i) gmask |= 1ULL << S.P.G[i];
    uint64_t lmask = 0;             // every tile bit's qubit (checked build)
    for (int b = 0; b < t; ++b) lmask |= 1ULL << S.P.L[b];
    (void)lmask;
    uint64_t base = deposit(t_begin + (uint64_t)gi, S.P.G, ng);
    uint32_t tc_parity = 0;
    // grouped form: every group runs the same number of iterations, so the
    // warps that hold several small groups stay converged up to the CTA's
    // closing barrier; a group past the end of the range (inactive) only
    // takes part in its barriers
    for (uint64_t tau0 = t_begin; tau0 < t_end;
         tau0 += (uint64_t)ngr, base = (GROUPED && ngr > 1) ? deposit(tau0 + (uint64_t)gi, S.P.G, ng)
                                                            : (((base | ~gmask) + 1) & gmask)) {
        const uint64_t tau = tau0 + (uint64_t)gi;
        bool active = !GROUPED || tau < t_end;
        if (TCP && TS.abort) break;
        // the tile's highest element index must lie inside the state
        if (active && !QS_DCHECK(((base | lmask) >> S.P.n) == 0, 201)) {
            if constexpr (!GROUPED) break;
            active = false;
        }
        // out-of-tile and thread bits are disjoint from it_off: OR = add
        const V *tsrc = amps + (base | tid_off);
        // ---- load the tile (16-byte cp.async, coalesced runs) ----
        if (active && uniform != (R)0 && folded) {
            // the pass starts from the uniform state times the folded
            // diagonal prefix: element x gets e^{i pi k(x) / 4} 2^(-n/2) with
            // k = 4 (CZ pairs within x) + (T counts of x), mod 8, summed over
            // the out-of-tile bits (the tile base), the thread's tile bits
            // (element CE tid) and the unit's (CE nthr it + q), plus the
            // pairs across those parts
            uint32_t pb = 0, nbm = 0;
            for (uint64_t w = base; w; w &= w - 1) {
                const int i = __ffsll((long long)w) - 1;
                pb ^= (uint32_t)__popcll(base & S.fnb[i] & (~0ULL << i << 1));
                nbm ^= S.fg[i];
            }
            const uint32_t lb = (uint32_t)(__popcll(base & S.fm[0]) + 2 * __popcll(base & S.fm[1]) +
                                           4 * __popcll(base & S.fm[2]));
            const uint32_t et = (uint32_t)(CE * tid);
            uint32_t pt = 0, nt = 0, lt = 0;
            for (uint32_t w = et; w; w &= w - 1) {
                const int b = __ffs(w) - 1;
                const int q = S.P.L[b];
                pt ^= (uint32_t)__popc(et & (uint32_t)S.fg[q] & (~0u << b << 1));
                nt ^= S.fg[q];
                lt += fcount(q);
            }
            const uint32_t k0 = 4u * ((pb ^ pt ^ (uint32_t)__popc(et & nbm)) & 1u) + lb + lt;
            const uint32_t nu = nbm ^ nt;
#pragma unroll
            for (int it = 0; it < CPT; ++it) {
                V fill[CE];
#pragma unroll
                for (int q = 0; q < CE; ++q) {
                    const uint32_t eu = (uint32_t)(CE * nthr) * (uint32_t)it + (uint32_t)q;
                    const uint32_t k = (k0 + S.fu[it * CE + q] + 4u * ((uint32_t)__popc(eu & nu) & 1u)) & 7u;
                    fill[q] = S.fw[k];
                }
                const uint32_t sw = sw_tid ^ (swz<CE>((uint32_t)(CE * it * nthr)) * (uint32_t)sizeof(V));
                *reinterpret_cast<float4 *>(gsm + sw) = *reinterpret_cast<const float4 *>(fill);
            }
        } else if (active && uniform != (R)0) {
            // the pass starts from the uniform state (the leading Hadamard
            // layer on |0...0>): the tile is written, not loaded
            V fill[CE];
#pragma unroll
            for (int q = 0; q < CE; ++q) {
                fill[q].x = uniform;
                fill[q].y = (R)0;
            }
#pragma unroll
            for (int it = 0; it < CPT; ++it) {
                const uint32_t sw = sw_tid ^ (swz<CE>((uint32_t)(CE * it * nthr)) * (uint32_t)sizeof(V));
                *reinterpret_cast<float4 *>(gsm + sw) = *reinterpret_cast<const float4 *>(fill);
            }
        } else if (active) {
#pragma unroll
            for (int it = 0; it < CPT; ++it) {
                const uint32_t sw = sw_tid ^ (swz<CE>((uint32_t)(CE * it * nthr)) * (uint32_t)sizeof(V));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tile_sa + sw),
                             "l"(tsrc + S.it_off[it])
                             : "memory");
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        tile_sync<GROUPED>(nthr, gi);

        for (int ph = 0; ph < nph; ++ph) {
            if constexpr (TCP > 0) {
                if (S.ph[ph].kind == 1) {
                    unsigned char *bbuf = reinterpret_cast<unsigned char *>(tile);
                    tc_phase<TCP>(TS, S.ph[ph].slot, S.ph[ph].scale_exp, reinterpret_cast<float2 *>(tile), bbuf,
                                  tc_parity, err_flag);
                    tc_parity ^= 1u;
                    if (TS.abort) break;
                    continue;
                }
            }
            if (active) {
            const SThread T = S.th[ph][tid];
            const uint64_t idx_th = base | T.qoff;
            uint32_t pb[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) pb[j] = S.ph[ph].pb[j];
            const bool paired = S.ph[ph].paired;
            V a[NS];
            // slots in Gray-code order: one XOR per slot address
            if (CE == 2 && paired)
                SlotIO<NS / 2, 1>::template load<V>(a, reinterpret_cast<const char *>(gsm), T.phys, pb);
            else
                SlotIO<NS, 0>::template load<V>(a, reinterpret_cast<const char *>(gsm), T.phys, pb);
            R fr = (R)1, fi = (R)0;             // thread-uniform pending factor
            const int ob = S.ph[ph].op_begin, oe = S.ph[ph].op_end, ub = S.ph[ph].uniform_begin;
            const bool fpend = ub < oe;
            if constexpr (FULL) {
                for (int o = ob; o < ub; ++o) {
                    const SOp<R> op = S.ops[o];
                    exec_op<RB, FULL>(op.code, a, idx_th, op.qmask, fr, fi, S.phase[op.aux]);
                }
            } else if constexpr (sizeof(R) == 4 && RB == 5) {
                // complex64: the op loop in PTX with an indexed branch per op
                // (the same arithmetic as exec_ct, see qs_ct_asm.inc)
                if (ob < ub) {
                    unsigned long long u[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s) u[s] = f2_bits(a[s]);
                    CtAsm<GROUPED ? 1 : 0>::run(u, smem_addr(S.code8), smem_addr(S.ops) + 8u, ob, ub, idx_th);
#pragma unroll
                    for (int s = 0; s < NS; ++s) a[s] = bits_f2(u[s]);
                }
            } else {
                // the next op's code is loaded while the current op runs
                uint32_t cn = S.code8[ob];
                for (int o = ob; o < ub; ++o) {
                    const uint32_t cc = cn;
                    cn = S.code8[o + 1];
                    exec_ct<RB, V, R>(cc, a, idx_th, &S.ops[o]);
                }
            }
            // tail: diagonal ops selected outside the register set multiply
            // the thread's pending factor (no interpreter dispatch)
            for (int o = ub; o < oe; ++o) {
                const SOp<R> op = S.ops[o];
                if ((idx_th & op.qmask) == op.qmask) {
                    const bool neg = (op.code & ~K_COND) == K_UNEG;
                    const R pr = neg ? (R)-1 : S.phase[op.aux][0], pi = neg ? (R)0 : S.phase[op.aux][1];
                    const R x = fr * pr - fi * pi;
                    fi = fr * pi + fi * pr;
                    fr = x;
                }
            }
            bool fmul = fpend;
            if (gs_in_phase && ph == nph - 1) {
                const R x = fr * gsr - fi * gsi;
                fi = fr * gsi + fi * gsr;
                fr = x;
                fmul = true;
            }
            if (fmul) {
                if (fi == (R)0) {
#pragma unroll
                    for (int s = 0; s < NS; ++s) mul_sign(a[s], fr);
                } else {
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const R x = a[s].x * fr - a[s].y * fi;
                        a[s].y = a[s].x * fi + a[s].y * fr;
                        a[s].x = x;
                    }
                }
            }
            {
                // reload the addressing state from shared memory rather than
                // keeping it live across the op loop
                uint32_t pb2[RB];
#pragma unroll
                for (int j = 0; j < RB; ++j) pb2[j] = S.ph[ph].pb[j];
                const uint32_t phys = S.th[ph][tid].phys;
                if (CE == 2 && S.ph[ph].paired)
                    SlotIO<NS / 2, 1>::template store<V>(a, reinterpret_cast<char *>(gsm), phys, pb2);
                else
                    SlotIO<NS, 0>::template store<V>(a, reinterpret_cast<char *>(gsm), phys, pb2);
            }
            }  // active
            tile_sync<GROUPED>(nthr, gi);
        }
        // ---- store the tile ----
        V *tdst = amps + (base | tid_off);
        if (active)
#pragma unroll
        for (int it = 0; it < CPT; ++it) {
            const uint32_t sw = sw_tid ^ (swz<CE>((uint32_t)(CE * it * nthr)) * (uint32_t)sizeof(V));
            V v[CE];
            *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(gsm + sw);
            if (gs_at_store) {
#pragma unroll
                for (int q = 0; q < CE; ++q) {
                    const R x = v[q].x * gsr - v[q].y * gsi;
                    v[q].y = v[q].x * gsi + v[q].y * gsr;
                    v[q].x = x;
                }
            }
            *reinterpret_cast<float4 *>(tdst + S.it_off[it]) = *reinterpret_cast<const float4 *>(v);
        }
        tile_sync<GROUPED>(nthr, gi);
    }
    if constexpr (TCP > 0)
        if (ntc) tc_teardown<TCP>(TS);
    __syncthreads();
}

// CTAs per SM of a pass: two, or one for tensor-core precisions whose
// block terms need 512 tensor-memory columns.
__host__ __device__ constexpr int pass_ctas_per_sm(int tcp)
{
    return tcp == 0 ? 2
                    : (128 + tc_prec(tcp).terms * (128 * tc_prec(tcp).elem_bytes / 4) <= 256 ? 2 : 1);
}

// FOLD: the instance that may start from the folded diagonal prefix (the
// first pass of a circuit); the others compile without that code.
template <typename R, int RB, int TCP, bool FULL, bool FOLD = false>
__global__ void __launch_bounds__(kThreadsMax, pass_ctas_per_sm(TCP))
k_fused_pass(typename V2T<R>::T *__restrict__ amps, const DevPass *__restrict__ pass_g,
             const DevPhase *__restrict__ phases_g, const DevOp *__restrict__ ops_g,
             uint64_t ntiles, const uint32_t *__restrict__ tc_words, int *__restrict__ err_flag, R uniform,
             FoldArgs fold)
{
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    __shared__ FusedSmem<R, RB> S;
    __shared__ TcSmem TS;
    // the folded diagonal prefix (first pass of a circuit only); the pass
    // body's first barrier publishes it
    const bool folded = FOLD && fold.nfold > 0 && uniform != (R)0;
    if (folded && threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < kMaxQubits; ++i) S.fnb[i] = fold.nb[i];
        S.fm[0] = fold.m1;
        S.fm[1] = fold.m2;
        S.fm[2] = fold.m4;
    }
    // the tensor-core form starts the tile (its MMA operand buffer) on a
    // 1024-byte boundary of the shared window; the launch adds the slack
    unsigned char *smem_raw = smem_dyn;
    if (TCP) smem_raw += (1024u - (smem_addr(smem_dyn) & 1023u)) & 1023u;
    // contiguous range of tiles per CTA
    const uint64_t per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
    const uint64_t t_begin = blockIdx.x * per + (blockIdx.x < extra ? blockIdx.x : extra);
    const uint64_t t_end = t_begin + per + (blockIdx.x < extra ? 1 : 0);
    fused_pass_body<R, RB, TCP, FULL>(amps, pass_g, phases_g, ops_g, t_begin, t_end, tc_words, err_flag, S, TS,
                                      smem_raw, uniform, folded);
}

// True when pass `hp` stages an op that the Clifford+T interpreter has no
// byte code for (shears, general phases, T phases selected outside the
// register set): such passes run the full interpreter.  Mirrors the device
// staging (ct_code on the same ops).
static bool pass_needs_full(const Plan &plan, const DevPass &hp)
{
    for (int ph = 0; ph < hp.nphases; ++ph) {
        const DevPhase &D = plan.phases[hp.phase_begin + ph];
        bool tail = false;     // thread-uniform diagonal ops must close the phase
        for (int o = D.op_begin; o < D.op_end; ++o) {
            const int c = ct_code(plan.ops[o]);
            if (c < 0 || (tail && c != (int)C_COUNT)) return true;
            tail = c == (int)C_COUNT;
        }
    }
    return false;
}

// Batched form: work item = (instance amplitudes, pass, tile range); the
// CTA restages the pass for every item.  All items of a launch share one
// tile size (blockDim.x = 2^(t - RB)).
struct BatchItem {
    uint64_t amp_off;       // element offset of the instance's state
    uint32_t pass;          // index into the batch's pass array
    uint32_t tile_begin, tile_end;
    uint32_t pad;
};

template <typename R, int RB, bool FULL>
__global__ void __launch_bounds__(kThreadsMax, 2)
k_batch_pass(typename V2T<R>::T *__restrict__ amps, const BatchItem *__restrict__ items, int nitems,
             const DevPass *__restrict__ passes, const DevPhase *__restrict__ phases_g,
             const DevOp *__restrict__ ops_g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FusedSmem<R, RB> S;
    __shared__ TcSmem TS;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        fused_pass_body<R, RB, 0, FULL>(amps + w.amp_off, passes + w.pass, phases_g, ops_g, w.tile_begin,
                                      w.tile_end, nullptr, nullptr, S, TS, smem_raw);
    }
}

// Persistent ensemble kernel (see PersistItem): kThreadsMax threads per CTA
// whatever the instances' tile sizes (13-qubit tiles take the whole CTA,
// smaller ones run in the grouped form), two CTAs per SM.  Thread 0 takes the next item from the queue head, waits for
// the item's dependencies (acquire, bounded by kPersistWaitNs), the CTA
// runs it, and thread 0 publishes its completion (release).  A wait that
// runs out sets ctl->err and ctl->abort; from then on items are taken and
// counted without work, so every CTA finishes and the host reports the
// timeout.  The last statistics item of an instance to finish sums the
// instance's partials in slot order (deterministic).
template <int RB, bool ANY_FULL>
__global__ void __launch_bounds__(kThreadsMax, 2)
k_batch_persistent(float2 *amps, const PersistItem *__restrict__ items, int nitems,
                   const DevPass *__restrict__ passes, const DevPhase *__restrict__ phases_g,
                   const DevOp *__restrict__ ops_g, uint32_t *done, PersistCtl *ctl, double *part,
                   double *sums, uint64_t wait_ns)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FusedSmem<float, RB> S;
    __shared__ TcSmem TS;
    __shared__ int s_item, s_go, s_last;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&ctl->next, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const PersistItem w = items[it];
        if (threadIdx.x == 0) {
            int go = *(volatile const uint32_t *)&ctl->abort == 0;
            if (go && w.need) {
                const int r = flag_wait_bounded(done + w.inst, w.need, &ctl->abort, wait_ns);
                if (r == 1) {
                    atomicExch(&ctl->err, 1u);
                    atomicExch(&ctl->abort, 1u);
                }
                go = r == 0;
            }
            s_go = go;
        }
        __syncthreads();
        if (s_go) {
            if (w.kind == kPersistInit) {
                float4 *a = reinterpret_cast<float4 *>(amps + w.amp_off);
                const float4 u = make_float4(w.f0, 0.f, w.f0, 0.f);
                for (uint32_t e = threadIdx.x; e < w.lo / 2; e += blockDim.x) a[e] = u;
                if (threadIdx.x == 0) a[0] = make_float4(w.f1, 0.f, w.f0, 0.f);
            } else if (w.kind == kPersistPass) {
                // a tile of 2^(RB + 8) amplitudes takes the whole CTA: the
                // plain body (CTA barriers); smaller tiles run grouped
                if (passes[w.pass].t == RB + 8)
                    fused_pass_body<float, RB, 0, false, false>(amps + w.amp_off, passes + w.pass, phases_g, ops_g,
                                                                w.lo, w.hi, nullptr, nullptr, S, TS, smem_raw);
                else
                    fused_pass_body<float, RB, 0, false, true>(amps + w.amp_off, passes + w.pass, phases_g, ops_g,
                                                               w.lo, w.hi, nullptr, nullptr, S, TS, smem_raw);
            } else if (w.kind == kPersistPassFull) {
                // (the launch compiles the full interpreter in only when
                // some item needs it)
                if constexpr (ANY_FULL)
                    fused_pass_body<float, RB, 0, true, true>(amps + w.amp_off, passes + w.pass, phases_g, ops_g,
                                                              w.lo, w.hi, nullptr, nullptr, S, TS, smem_raw);
            } else {
                batch_stats_chunk(amps + w.amp_off, w.lo, w.f0, part + (size_t)w.pass * kStatAcc);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t prev = atomicAdd(done + w.inst, 1u);
            if (w.kind == kPersistStats) {
                s_last = prev + 1 == w.total;
                __threadfence();
            }
        }
        if (w.kind == kPersistStats) {
            __syncthreads();
            if (s_last && threadIdx.x < kStatAcc) {
                double acc = 0;
                for (uint32_t j = 0; j < w.nslots; ++j) acc += __ldcg(part + (size_t)(w.hi + j) * kStatAcc + threadIdx.x);
                sums[(size_t)w.inst * kStatAcc + threadIdx.x] = acc;
            }
        }
    }
}

template <typename R, int RB>
static qs_status run_fused_t(qs_state *s, const Plan &plan, const void *dev_plan, double uniform,
                             const FoldArgs *fold)
{
    const FoldArgs none{};
    using V = typename V2T<R>::T;
    const DevPass *dpass = reinterpret_cast<const DevPass *>(dev_plan);
    const DevPhase *dphase = reinterpret_cast<const DevPhase *>(dpass + plan.passes.size());
    const DevOp *dops = reinterpret_cast<const DevOp *>(dphase + plan.phases.size());
    const uint32_t *dwords = reinterpret_cast<const uint32_t *>(dops + plan.ops.size());
    int *err = reinterpret_cast<int *>(s->ws_u64);
    bool any_tc = false;
    for (size_t p = 0; p < plan.passes.size(); ++p) {
        const DevPass &hp = plan.passes[p];
        if (hp.r != RB || hp.t < RB || hp.t - RB > 8)
            return set_error(QS_ERR_INVALID_ARG, "pass %zu: tile %d / register bits %d unsupported",
                             p, hp.t, hp.r);
        bool tc = false;
        for (int ph = 0; ph < hp.nphases; ++ph) tc |= plan.phases[hp.phase_begin + ph].kind == 1;
        const int threads = 1 << (hp.t - RB);
        const uint64_t ntiles = 1ULL << (plan.n - hp.t);
        if (tc) {
            if constexpr (sizeof(R) == 4) {
                if (hp.t != 13)
                    return set_error(QS_ERR_INVALID_ARG, "tensor-core phases need 13-bit tiles");
                if (!any_tc) QS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s->stream));
                any_tc = true;
                // register phases of a Clifford+T pass run the byte-code op loop
                const bool full = pass_needs_full(plan, hp);
                decltype(&k_fused_pass<R, RB, 1, true>) kern;
                switch (plan.precision) {
#define QS_TC_KERN(P) (full ? k_fused_pass<R, RB, P, true> : k_fused_pass<R, RB, P, false>)
                case QS_PREC_BF16X3: kern = QS_TC_KERN(QS_PREC_BF16X3); break;
                case QS_PREC_BF16X6: kern = QS_TC_KERN(QS_PREC_BF16X6); break;
                case QS_PREC_TF32X3: kern = QS_TC_KERN(QS_PREC_TF32X3); break;
                case QS_PREC_TF32: kern = QS_TC_KERN(QS_PREC_TF32); break;
                case QS_PREC_FP16X3: kern = QS_TC_KERN(QS_PREC_FP16X3); break;
#undef QS_TC_KERN
                default: return set_error(QS_ERR_INVALID_ARG, "tensor-core precision %d", plan.precision);
                }
                const size_t smem = tc_dyn_smem(plan.precision);
                QS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                const uint64_t cap = (uint64_t)s->num_sms * pass_ctas_per_sm(plan.precision);
                const int grid = (int)(ntiles < cap ? ntiles : cap);
                kern<<<grid, threads, smem, s->stream>>>((V *)s->amps, dpass + p, dphase, dops, ntiles, dwords,
                                                         err, p == 0 ? (R)uniform : (R)0, none);
            } else {
                return set_error(QS_ERR_INVALID_ARG, "tensor-core phases need complex64");
            }
        } else {
            // the circuit's first pass forms the folded prefix's phases
            const bool fold_here = p == 0 && fold && fold->nfold > 0 && uniform != 0.0;
            auto kern = pass_needs_full(plan, hp)
                            ? (fold_here ? k_fused_pass<R, RB, 0, true, true> : k_fused_pass<R, RB, 0, true>)
                            : (fold_here ? k_fused_pass<R, RB, 0, false, true> : k_fused_pass<R, RB, 0, false>);
            const size_t smem = (size_t(1) << hp.t) * sizeof(V);
            QS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const uint64_t cap = (uint64_t)s->num_sms * 2;
            const int grid = (int)(ntiles < cap ? ntiles : cap);
            kern<<<grid, threads, smem, s->stream>>>((V *)s->amps, dpass + p, dphase, dops, ntiles, nullptr, nullptr,
                                                     p == 0 ? (R)uniform : (R)0, fold_here ? *fold : none);
        }
        QS_LAUNCH_CHECK();
    }
    if (any_tc) {
        int h = 0;
        QS_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (h) return set_error(QS_ERR_TIMEOUT, "tensor-core pass: completion wait ran out");
    }
    return QS_OK;
}

bool plan_pass_needs_full(const Plan &plan, int pass)
{
    return pass_needs_full(plan, plan.passes[pass]);
}

qs_status launch_batch_round(cudaStream_t st, int num_sms, void *amps, const void *items, int nitems,
                             int tile_bits, const DevPass *passes, const DevPhase *phases, const DevOp *ops,
                             bool full)
{
    if (tile_bits < 5 || tile_bits > 13) return set_error(QS_ERR_INVALID_ARG, "batch tile bits %d", tile_bits);
    auto kern = full ? k_batch_pass<float, 5, true> : k_batch_pass<float, 5, false>;
    const size_t smem = (size_t(1) << tile_bits) * sizeof(float2);
    const int cap = num_sms * 2;
    const int grid = nitems < cap ? nitems : cap;
    kern<<<grid, 1 << (tile_bits - 5), smem, st>>>((float2 *)amps, (const BatchItem *)items, nitems, passes,
                                                   phases, ops);
    QS_LAUNCH_CHECK();
    return QS_OK;
}

// Resident CTAs per SM of the two persistent-kernel variants (occupancy
// API, set by batch_kernel_setup before any launch or capture).
static int g_persist_per_sm[2] = {2, 2};

qs_status launch_batch_persistent(cudaStream_t st, int num_sms, void *amps, const PersistItem *items, int nitems,
                                  const DevPass *passes, const DevPhase *phases, const DevOp *ops,
                                  uint32_t *done, PersistCtl *ctl, double *part, double *sums, bool any_full)
{
    if (nitems <= 0) return QS_OK;
    const int cap = num_sms * g_persist_per_sm[any_full ? 1 : 0];
    const int grid = nitems < cap ? nitems : cap;
    auto kern = any_full ? k_batch_persistent<5, true> : k_batch_persistent<5, false>;
    kern<<<grid, kThreadsMax, 65536, st>>>((float2 *)amps, items, nitems, passes, phases, ops, done, ctl, part, sums,
                                           kPersistWaitNs);
    QS_LAUNCH_CHECK();
    return QS_OK;
}

int batch_persistent_ctas_per_sm(bool any_full) { return g_persist_per_sm[any_full ? 1 : 0]; }

qs_status batch_kernel_setup()
{
    QS_CUDA_TRY(cudaFuncSetAttribute(k_batch_persistent<5, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    QS_CUDA_TRY(cudaFuncSetAttribute(k_batch_persistent<5, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    QS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_persist_per_sm[0], k_batch_persistent<5, false>,
                                                              kThreadsMax, 65536));
    QS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_persist_per_sm[1], k_batch_persistent<5, true>,
                                                              kThreadsMax, 65536));
    for (int &v : g_persist_per_sm) v = v < 1 ? 1 : v;
    QS_CUDA_TRY(cudaFuncSetAttribute(k_batch_pass<float, 5, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    QS_CUDA_TRY(cudaFuncSetAttribute(k_batch_pass<float, 5, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    return QS_OK;
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

void batch_item_fill(void *dst, uint64_t amp_off, uint32_t pass, uint32_t tb, uint32_t te)
{
    BatchItem w{amp_off, pass, tb, te, 0};
    std::memcpy(dst, &w, sizeof w);
}

QS_CHECK_READER(check_poll_fused)

qs_status run_fused_plan(qs_state *s, const Plan &plan, const void *dev_plan, double uniform,
                         const FoldArgs *fold)
{
    if (s->dt == QS_C64) return run_fused_t<float, 5>(s, plan, dev_plan, uniform, fold);
    return run_fused_t<double, 4>(s, plan, dev_plan, uniform, fold);
}

}  // namespace qs
