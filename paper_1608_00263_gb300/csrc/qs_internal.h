// qs_internal.h -- private declarations shared by the library's translation
// units: the state handle, the planner's device plan format, and the kernel
// launchers.  Not part of the public ABI (include/qs.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qs.h"

#ifdef __CUDACC__
#include <cuda_runtime.h>
#else
struct CUstream_st;
typedef CUstream_st *cudaStream_t;
struct CUevent_st;
typedef CUevent_st *cudaEvent_t;
#endif

#ifdef __CUDACC__
#define QS_TC_HD __host__ __device__
#else
#define QS_TC_HD
#endif

namespace qs {

constexpr int kMaxQubits = 34;
constexpr int kMaxMoments = 10;

// ---------------------------------------------------------------------------
// Error reporting (thread-local message, returned status)
// ---------------------------------------------------------------------------
qs_status set_error(qs_status st, const char *fmt, ...);
void clear_error();
const char *last_error_cstr();

// ---------------------------------------------------------------------------
// Gate helpers (host)
// ---------------------------------------------------------------------------
struct Cplx {
    double re, im;
};

bool gate_is_two_qubit(int kind);
bool gate_is_diagonal(int kind);
// 2x2 matrix (row-major u00 u01 u10 u11) of a gate; for two-qubit kinds the
// matrix applied to the target when the control bit is set.
void gate_matrix(int kind, double theta, Cplx u[4]);
qs_status validate_gates(int n, const qs_gate *g, size_t ng);
// n when the gate list opens with H on every qubit (n gates, each qubit
// once), else 0: on |0...0> that layer is the uniform superposition
// (Sec. pt, cycle 0), generated by the first fused pass (or written as one
// fill before plain per-gate kernels) instead of run as gates.
size_t leading_h_layer(const qs_gate *g, size_t ng, int n);

// Diagonal prefix folded into the initial state.  After a leading Hadamard
// layer on |0...0>, a T or CZ gate none of whose qubits has yet met a
// non-diagonal gate commutes with every gate before it, so it acts on the
// uniform superposition: psi_0(x) = 2^(-n/2) exp(i pi k(x) / 4) with
// k(x) = 4 sum_{CZ (i,j)} x_i x_j + sum_i c_i x_i (mod 8), c_i the number of
// such T gates on qubit i (Sec. pt, cycle 0; Eq. sqgunitaryoperation).
struct FoldArgs {
    uint64_t nb[kMaxQubits];    // CZ partners of each qubit (a repeated pair cancels)
    uint64_t m1, m2, m4;        // bits 0, 1, 2 of each qubit's T count
    int nfold;                  // gates folded (0: the plain uniform state)
    int pad;
};
// Splits the gates after a leading Hadamard layer into the foldable
// diagonal prefix (into *f) and the rest, in order (into *rest).  Returns
// the number of gates folded.
size_t fold_diagonal_prefix(const qs_gate *g, size_t ng, std::vector<qs_gate> *rest, FoldArgs *f);

// ---------------------------------------------------------------------------
// Fused-pass plan (built on the host, executed by the fused kernels)
// ---------------------------------------------------------------------------
enum OpType : uint8_t {
    OP_DENSE = 0,   // general 2x2 complex matrix on register bit `a`
    OP_H = 1,       // [[1, 1], [1, -1]]      (1/sqrt2 deferred to pass end)
    OP_XH = 2,      // [[1, -i], [-i, 1]]     (1/sqrt2 deferred)
    OP_YH = 3,      // [[1, -1], [1, 1]]      (1/sqrt2 deferred)
    OP_PHASE = 4,   // multiply by m[0] + i m[1] where all bits of the op's
                    // qubit set are 1 (register part rmask, rest qmask)
    OP_NEG = 5,     // multiply by -1, same selection as OP_PHASE
    OP_MATRIX = 6,  // tensor-core dense block (TC mode only): index of the
                    // block matrix in `a`
    OP_SHX = 7,     // shear x += m[0] * y on register bit `a` (x: bit 0, y: bit 1)
    OP_SHY = 8,     // shear y += m[0] * x on register bit `a`
};

struct DevOp {          // 80 bytes
    uint8_t type;
    uint8_t a;          // register bit (dense ops) / block index (OP_MATRIX)
    uint8_t rmask;      // register-slot bits of the selection (phase ops)
    uint8_t pad0;
    uint32_t pad1;
    uint64_t qmask;     // qubit-index bits of the selection outside the
                        // register set (phase ops)
    double m[8];        // matrix u00 u01 u10 u11 as (re, im) pairs, or phase
};

constexpr int kMaxTileBits = 16;
constexpr int kMaxRegBits = 8;
constexpr int kMaxPhasesPerPass = 8;    // per-thread phase tables live in shared memory
constexpr int kMaxOpsPerPass = 256;     // op descriptors live in shared memory

struct DevPhase {       // 40 bytes
    uint8_t R[kMaxRegBits];  // tile bit of each register (or block) bit
    uint8_t T[8];            // register phases: tile bit of thread-index bit k
                             // (bits 0..4 are the lane bits of a warp)
    int32_t op_begin, op_end;
    int32_t kind;            // 0: register phase, 1: tensor-core block phase
    int32_t tc_block;        // kind 1: index of the block matrix
    int32_t defer_before;    // kind 1: deferred 1/sqrt2 factors pending in the
                             // tile when the phase runs (values are up to
                             // 2^(defer_before/2) times their true size)
    int32_t pad;
};

// Tensor-core block phase: a k = 6 qubit block unitary U (64 x 64 complex)
// realified to A (128 x 128): row 2i is (Re U_i, -Im U_i) and row 2i+1 is
// (Im U_i, Re U_i) over the K columns (re block, then im block), i.e. the
// rows of [[Re U, -Im U], [Im U, Re U]] with real and imaginary output rows
// interleaved; split into the terms of the operand precision and stored
// row-major as 32-bit words: per row, the words of term 0, then term 1, ...
// (16-bit formats: two consecutive K elements per word, lower K in the low
// half; TF32: one element per word).
constexpr int kTcBits = 6;
constexpr int kMaxTcPerPass = 1;        // TMEM per CTA: accumulator + 1 block's terms

// Operand format of a tensor-core precision (qs_precision): element type
// (0 FP16, 1 BF16, 2 TF32, the instruction descriptor's encoding), number
// of terms of each operand, and whether tiles are scaled into FP16's range.
struct TcPrec {
    int fmt;
    int terms;
    int elem_bytes;
    bool scaled;
};
QS_TC_HD constexpr TcPrec tc_prec(int precision)
{
    return precision == QS_PREC_BF16X3   ? TcPrec{1, 2, 2, false}
           : precision == QS_PREC_BF16X6 ? TcPrec{1, 3, 2, false}
           : precision == QS_PREC_TF32X3 ? TcPrec{2, 2, 4, false}
           : precision == QS_PREC_TF32   ? TcPrec{2, 1, 4, false}
                                         : TcPrec{0, 2, 2, true};
}
// 32-bit words of one block matrix: 128 rows x terms x 128 K elements.
QS_TC_HD constexpr int tc_words_per_block(int precision)
{
    return 128 * tc_prec(precision).terms * (128 * tc_prec(precision).elem_bytes / 4);
}
constexpr int kTcWordsPerBlock = 128 * 128;   // FP16x3 (the default precision)

struct DevPass {
    int32_t t;              // tile bits
    int32_t r;              // register bits per phase (or block bits, TC)
    int32_t nphases;
    int32_t phase_begin;    // index into the plan's phase array
    int32_t ngates;         // gates this pass applies
    int32_t deferred;       // number of deferred 1/sqrt2 factors
    int32_t n;              // qubits of the state
    int32_t pad;
    double gscale_re, gscale_im;  // pass-wide factor applied at the end
    uint8_t L[kMaxTileBits];      // qubit of each tile bit (ascending)
    uint8_t G[64];                // qubits outside the tile (ascending)
};

struct Plan {
    int n = 0;
    int t = 0, r = 0, c = 0;
    int mode = 0;
    std::vector<DevPass> passes;
    std::vector<DevPhase> phases;
    std::vector<DevOp> ops;
    std::vector<uint32_t> tc_words;  // TC mode: packed block matrices (see tc_prec)
    int precision = QS_PREC_FP16X3;  // TC mode: operand precision of tc_words
    int gates = 0;
};

struct PlanParams {
    int n;
    int t;           // tile bits (<= n)
    int r;           // register bits per phase
    int c;           // low qubits always inside the tile (coalescing)
    int mode;        // QS_MODE_FUSED or QS_MODE_FUSED_TC
    int k;           // TC block bits
    int tc_ok;       // tensor-core phases allowed (complex64, 13-bit tiles)
    int esz = 8;     // bytes per amplitude (8 complex64, 16 complex128)
    int precision = QS_PREC_FP16X3;   // TC operand precision (qs_precision, not DEFAULT)
    int look_steps = 2;   // tile choice: additions scored by greedy completion
    int look_top = 6;     // ... among this many best-scoring candidates
    int hoist_diagonals = 1;   // move late diagonal ops to the last phase's uniform tail
};

// XOR swizzle of the shared-memory tile (element e -> element index): the
// element's 16-byte unit u = e / CE (CE elements per unit) has bits 0..2
// XORed with a fold of its higher bits.  Linear over GF(2).  Shared by the
// kernels and the planner's bank-conflict model.
#ifdef __CUDACC__
#define QS_HD __host__ __device__
#else
#define QS_HD
#endif
QS_HD inline uint32_t tile_swizzle(uint32_t e, uint32_t CE)
{
    const uint32_t u = e / CE;
    const uint32_t f = ((u >> 3) ^ (u >> 6) ^ (u >> 9) ^ (u >> 12)) & 7u;
    return e ^ (f * CE);
}

qs_status build_plan(const PlanParams &pp, const qs_gate *g, size_t ng, Plan *out);
uint16_t f64_to_f16_bits(double x);
double f16_bits_to_f64(uint16_t h);
// bfloat16 (8 exponent bits, 7 fraction bits) and TF32 (8 exponent bits, 10
// fraction bits, kept in a 32-bit word with the low 13 bits zero) from a
// double, round to nearest even.
uint16_t f64_to_bf16_bits(double x);
double bf16_bits_to_f64(uint16_t h);
uint32_t f64_to_tf32_bits(double x);
double tf32_bits_to_f64(uint32_t w);
PlanParams default_plan_params(int n, qs_dtype dt, const qs_opts *o);
double plan_bytes(const Plan &p, qs_dtype dt);

// Persistent ensemble kernel: one launch runs a batch's whole work list
// from a device queue.  Items are taken in list order by an atomic head;
// item j of instance i waits (bounded) until done[i] >= need, runs, then
// increments done[i] (release).  Every item's dependencies precede it in
// the list, so the earliest unfinished item can always run.
enum PersistKind : uint32_t {
    kPersistInit = 0,      // write the initial amplitudes of one chunk
    kPersistPass = 1,      // fused tile pass, Clifford+T interpreter
    kPersistPassFull = 2,  // fused tile pass, full interpreter
    kPersistStats = 3      // statistics partials of one chunk
};
struct PersistItem {
    uint64_t amp_off;      // pass: the instance's state; init / stats: the chunk
    uint32_t kind;         // PersistKind
    uint32_t inst;         // instance (its completion counter)
    uint32_t need;         // completed items of the instance this one waits for
    uint32_t total;        // items of the instance (the last statistics item sums)
    uint32_t pass;         // pass: index into the pass array; stats: partial slot
    uint32_t lo, hi;       // pass: tile range [lo, hi); init / stats: lo = amplitudes
                           // of the chunk; stats: hi = the instance's first slot
    uint32_t nslots;       // stats: the instance's partial slots
    float f0, f1;          // init: fill value, first amplitude; stats: f0 = N
};
struct PersistCtl {
    uint32_t next;         // queue head
    uint32_t abort;        // a wait ran out: the remaining items drain without work
    uint32_t err;          // 1 when a wait ran out
    uint32_t pad;
};

// Work list of the persistent ensemble engine for the instances `idx` of a
// batch (instance i: n[i] qubits at element offset off[i]; plans[i] its
// plan, empty when its list is only the Hadamard layer; full[i][r] whether
// pass r needs the full interpreter; hl[i] nonzero when the circuit opens
// with a Hadamard layer, so the initial state is uniform).  Order: every
// instance's initial-state chunks (kWorkChunk amplitudes), then the passes
// round-major (pass r of every instance, larger instances first, before
// pass r + 1 of any; items of 2^kPassItemBits amplitudes = 2^(18 - t)
// tiles, so a CTA restages a pass once per 32 tiles of 2^13), then, with
// `stats`, the statistics chunks (kWorkChunk amplitudes, as the lockstep
// engine's; slot order = list order).  Item need = the number of the instance's items in
// all earlier levels (initial chunks; pass 0; pass 1; ...; statistics), so
// done[i] >= need holds exactly when those levels are complete, and every
// one of them precedes the item in the list.
constexpr uint64_t kWorkChunk = 1ULL << 16;
constexpr int kPassItemBits = 18;
struct Work {
    std::vector<DevPass> passes;
    std::vector<DevPhase> phases;
    std::vector<DevOp> ops;
    std::vector<PersistItem> items;
    double bytes = 0;                // algorithmic bytes of the passes
    int nslots = 0;                  // statistics partial slots
};
void build_work(const std::vector<int> &n, const std::vector<uint64_t> &off, const std::vector<Plan> &plans,
                const std::vector<std::vector<char>> &full, const std::vector<int> &idx,
                const std::vector<size_t> &hl, bool stats, Work *W);

// ---------------------------------------------------------------------------
// State handle
// ---------------------------------------------------------------------------
// Two plan slots per state: a plan can be built and uploaded (stream-ordered,
// from pinned memory) while the device still runs the other slot's plan, so
// host planning of the next circuit overlaps the current evolution.
struct DevicePlanSlot {
    bool valid = false;
    uint64_t key = 0;          // hash of (gates, options)
    size_t ngates = 0;
    void *dev = nullptr;       // passes | phases | ops | blocks on device
    void *staging = nullptr;   // pinned host source of the upload
    size_t bytes = 0;          // capacity of dev and staging
    cudaEvent_t done = nullptr;   // after the slot's last upload or apply
    uint64_t last_use = 0;
    Plan plan;
};

struct DevicePlanCache {
    DevicePlanSlot slot[2];
    uint64_t clock = 0;
};

}  // namespace qs

struct qs_state {
    int n;
    qs_dtype dt;
    void *amps;              // device, 2^n amplitudes
    bool owns;
    cudaStream_t stream;
    int device;
    int num_sms;
    // statistics / sampler workspace (device)
    double *ws_f64;          // reduction partials
    size_t ws_f64_count;
    uint64_t *ws_u64;        // small integer scratch (flags, counters)
    qs::DevicePlanCache plan_cache;
    // |0...0> bookkeeping, for applying a leading layer of Hadamards as one
    // uniform write: is_zero -- the state is |0...0> (written, or pending:
    // zero_pending defers the reset's write to the next use); escaped -- the
    // caller can reach the memory (attached, or after qs_state_amplitudes),
    // so resets are written at once and nothing is assumed about it.
    bool is_zero = false;
    mutable bool zero_pending = false;
    mutable bool escaped = false;
    // asynchronous host read-out (qs_probabilities_async): the read-out
    // kernel writes the first share of the probabilities (ro_frac of the
    // 256-probability chunks, set by qs_readout_share) into the page-locked
    // host memory itself and the rest into ro_buf, which the copy engine
    // moves on ro_stream while later work runs; ro_done marks the end of the
    // last copy (the buffer is free)
    mutable void *ro_buf = nullptr;
    mutable size_t ro_bytes = 0;
    mutable cudaStream_t ro_stream = nullptr;
    mutable cudaEvent_t ro_ready = nullptr, ro_done = nullptr;
    double ro_frac = 0.0;
    // page-locked host memory mapped into the device: kernels write small
    // results (hbox) and host-side sample arrays (stage) there directly, so
    // no copy-engine transfer is needed and nothing queues behind an
    // asynchronous read-out still copying
    void *hbox = nullptr, *hbox_dev = nullptr;
    mutable void *stage = nullptr, *stage_dev = nullptr;
    mutable size_t stage_bytes = 0;
    // read-out cache (complex64): statistics partials and sampler chunk sums
    // formed by the fused read-out pass, valid while `version` (bumped by
    // every change of the amplitudes) equals rc_version and the caller cannot
    // reach the memory
    mutable uint64_t version = 0;
    mutable double *rc_buf = nullptr;
    mutable size_t rc_doubles = 0;
    mutable uint64_t rc_version = ~0ULL;
    mutable int rc_flags = 0;
};

namespace qs {

// Launchers (defined in the .cu files).  All are asynchronous on `st` and
// return QS_ERR_CUDA (with message) on a launch failure.
qs_status launch_init_zero(qs_state *s);
// Every amplitude = 2^(-n/2): H^{(x)n} |0...0>.
qs_status launch_init_uniform(qs_state *s);
qs_status launch_plain_gate(qs_state *s, const qs_gate &g);
// Runs a fused plan on the state.  uniform != 0: the state is taken to be
// the uniform superposition with that amplitude (the leading Hadamard layer
// on |0...0>, not written): the first pass writes its tiles in shared memory
// instead of loading them, so the state's memory is not read.  With `fold`
// (nfold > 0) those tiles also carry the folded diagonal prefix's phases.
qs_status run_fused_plan(qs_state *s, const Plan &plan, const void *dev_plan, double uniform = 0.0,
                         const FoldArgs *fold = nullptr);
qs_status run_tc_plan(qs_state *s, const Plan &plan, const void *dev_plan,
                      int precision);
qs_status launch_probabilities(const qs_state *s, void *out, int fp64,
                               uint64_t first, uint64_t count);
qs_status stats_moments(const qs_state *s, int kmax, double *moments,
                        double *entropy, double *uniform_ce, double *norm);
qs_status sampler_run(const qs_state *s, uint64_t k, uint64_t seed,
                      uint64_t *dev_out);
qs_status cross_entropy_run(const qs_state *s, const uint64_t *dev_samples,
                            uint64_t m, double *ce);
qs_status adjoint_run(qs_state *s, const qs_gate *g, size_t ng, const uint64_t *dev_x,
                      uint64_t m, double *grad);

size_t dtype_bytes(qs_dtype dt);

// Checked build: synchronises the device and reads every translation unit's
// device check word (QS_ERR_INVALID_ARG if one is set); QS_OK at once in
// the normal build.  Site codes: 1xx plain kernels, 2xx fused pass, 3xx
// statistics and sampler, 4xx batch, 9xx the check probe.
qs_status check_poll_all();
qs_status check_poll_plain();
qs_status check_poll_fused();
qs_status check_poll_stats();
qs_status check_poll_api();
qs_status check_poll_batch();
qs_status check_poll_adjoint();

constexpr size_t kHostBoxBytes = 4096;
// Copies `bytes` (a multiple of 8, at most kHostBoxBytes) of device memory
// to `host` through the state's mapped host box: a one-block kernel on the
// state's stream, then a stream synchronisation.
qs_status read_back(const qs_state *s, void *host, const void *dev, size_t bytes);

// Fused read-out of a complex64 state (one read): p = |psi|^2 into `out`
// (out_kind 1: FP32, 2: FP64, 0: none; device-accessible, 16-byte aligned),
// the statistics partials and the sampler's chunk sums into the read-out
// cache, which it marks valid for the current state.
constexpr int kReadoutStats = 1, kReadoutChunks = 2, kReadoutScanned = 4;
// Fused complex64 read-out (probabilities, statistics partials, sampler
// chunk sums); with out_hi, chunks [csplit, nchunks) of the probabilities go
// to out_hi (chunk csplit at its start) instead of out.  Chunks are
// readout_chunks(s) groups of 256 probabilities.
qs_status readout_c64(const qs_state *s, void *out, int out_kind, void *out_hi = nullptr, uint64_t csplit = 0);
uint64_t readout_chunks(const qs_state *s);
bool readout_cached(const qs_state *s, int flag);
int readout_grid(const qs_state *s);
double *readout_part(const qs_state *s);
double *readout_csum(const qs_state *s);
// Page-locked, device-mapped staging of at least `bytes` (grown on demand):
// host and device addresses of the same memory.
qs_status stage_view(const qs_state *s, size_t bytes, void **host, void **dev);

// batched ensemble helpers
constexpr int kStatSums = 12;
// One lockstep round of the batched pass; `full` selects the interpreter
// with the parameterised-gate cases (else the Clifford+T one, valid when
// plan_pass_needs_full is false for every pass of the round's items).
qs_status launch_batch_round(cudaStream_t st, int num_sms, void *amps, const void *items, int nitems,
                             int tile_bits, const DevPass *passes, const DevPhase *phases, const DevOp *ops,
                             bool full);
bool plan_pass_needs_full(const Plan &plan, int pass);
size_t batch_item_bytes();
qs_status batch_kernel_setup();

constexpr uint64_t kPersistWaitNs = 2000000000ull;   // per dependency wait
// Launches the persistent kernel over nitems items (device array) with
// counters done[count instances] and ctl zeroed beforehand; statistics
// partials go to part[slot * kStatSums], per-instance sums to
// sums[inst * kStatSums].  any_full: some item is kPersistPassFull (the
// variant with the full interpreter); grid = resident CTAs (occupancy API).
qs_status launch_batch_persistent(cudaStream_t st, int num_sms, void *amps, const PersistItem *items, int nitems,
                                  const DevPass *passes, const DevPhase *phases, const DevOp *ops,
                                  uint32_t *done, PersistCtl *ctl, double *part, double *sums, bool any_full);
// Resident CTAs per SM of the persistent kernel (after batch_kernel_setup).
int batch_persistent_ctas_per_sm(bool any_full);
void batch_item_fill(void *dst, uint64_t amp_off, uint32_t pass, uint32_t tb, uint32_t te);
// Batched sampler over instances laid out at element offsets off_h[i]
// (2^n_h[i] complex64 each): k samples per instance into host_out[i k + j].
qs_status batch_sampler_run(cudaStream_t st, int num_sms, const void *amps_v, const uint64_t *off_h,
                            const int *n_h, int count, uint64_t k, uint64_t seed, double r_mes,
                            uint64_t *host_out);
// Per-instance overlap sums with a reference complex64 state of the same n
// (instances at element offsets off_h, all of n qubits): host_sums[i*5 ..] =
// sum p_i p_ref, sum p_i^2, sum p_i, sum p_ref^2, sum p_ref.
qs_status batch_overlap_run(cudaStream_t st, int num_sms, const void *amps, const void *ref,
                            const uint64_t *off_h, int count, int n, double *host_sums);
// Mean distribution over `count` consecutive instances of n qubits.
qs_status batch_mean_probs_run(cudaStream_t st, int num_sms, const void *amps, int count, int n,
                               double *device_out);
qs_status launch_batch_stats(cudaStream_t st, int num_sms, const void *amps, const uint64_t *item_off,
                             const uint64_t *item_cnt, const float *item_scale, int nitems,
                             const int *first_item, int count, double *part, double *out);
void stats_from_sums(const double *h, int n, int kmax, double *norm, double *entropy, double *uniform_ce,
                     double *moments);

}  // namespace qs
