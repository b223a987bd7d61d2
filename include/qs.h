/*
 * qs.h -- C ABI of the GB300 (sm_103a) state-vector library for the random
 * circuit sampling method of Boixo et al., "Characterizing Quantum Supremacy
 * in Near-Term Devices" (arXiv:1608.00263).
 *
 * The calls follow the paper's statement of the problem (Sec.
 * "Characterizing quantum supremacy", the four-step estimation procedure):
 * choose a circuit U, evolve |psi> = U|0...0>, take m samples x_j from
 * p_U(x) = |<x|psi>|^2, compute log 1/p_U(x_j) and estimate the cross-entropy
 * difference (Eq. ae); plus the Porter-Thomas statistics of Sec.
 * "Convergence to Porter-Thomas" (entropy, Eq. eu; uniform cross entropy,
 * Eq. eue; moments / inverse participation ratios).
 *
 * Conventions (all calls)
 *   - Bit j of a basis-state index is qubit j.  Results are always in this
 *     canonical order, whatever tiling the library uses internally.
 *   - Every call returns a qs_status; on failure qs_last_error() gives a
 *     thread-local message.  Arguments are validated on the host before any
 *     kernel launch; no call aborts, traps or exits the process.
 *   - Work is ordered on the state's CUDA stream.  Calls that return host
 *     scalars (qs_cross_entropy, qs_pt_moments) synchronise that stream.
 *   - Device memory of a state created by qs_state_create is owned by the
 *     library; qs_state_attach wraps caller-owned device memory (for example
 *     a torch tensor), which must outlive the handle.
 *   - Output buffers are caller-owned.  Pointer arguments documented as
 *     "host or device" are classified with cudaPointerGetAttributes.
 *   - Gate arrays are read during the call only.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef QS_PUBLIC_API_H_
#define QS_PUBLIC_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_state qs_state;

typedef enum {
    QS_OK = 0,
    QS_ERR_INVALID_ARG = 1,   /* bad size, qubit, pointer or option */
    QS_ERR_OOM = 2,           /* device or host allocation failed */
    QS_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    QS_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
    QS_ERR_UNSUPPORTED = 5    /* valid request this build does not handle */
} qs_status;

/* Amplitude storage: complex64 (interleaved float re, im; 8 B) or complex128
 * (interleaved double re, im; 16 B).  The paper's simulator used double
 * complex (appendix "Quantum Simulation Details"). */
typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Gate kinds.  Fixed gates of Sec. "Convergence to Porter-Thomas":
 *   H; X^1/2 = exp(-i pi/4 X) and Y^1/2 = exp(-i pi/4 Y) (pi/2 rotations);
 *   T = diag(1, e^{i pi/4}); CZ = diag(1, 1, 1, -1).
 * Parameterised forms (theta in radians):
 *   RX/RY/RZ(theta) = exp(-i theta/2 P);  CPHASE(theta) = diag(1,1,1,e^{i theta}).
 * Two-qubit kinds (CZ, CPHASE) use q0 and q1 (q0 != q1, either order; both
 * are diagonal and symmetric); single-qubit kinds use q0 and ignore q1. */
typedef enum {
    QS_H = 0, QS_X_HALF = 1, QS_Y_HALF = 2, QS_T = 3, QS_CZ = 4,
    QS_RX = 5, QS_RY = 6, QS_RZ = 7, QS_CPHASE = 8
} qs_kind;

/* One gate, 16 bytes.  `cycle` is informational (clock cycle of the gate in
 * the generated circuit); gates are applied in array order. */
typedef struct {
    uint8_t kind, q0, q1, pad;
    uint32_t cycle;
    double theta;
} qs_gate;

/* Execution forms of qs_apply_circuit. */
typedef enum {
    QS_MODE_PLAIN = 0,     /* one kernel, one state pass per gate; gate
                              specialisation as in the appendix: diagonal
                              gates touch only the amplitudes they change */
    QS_MODE_FUSED = 1,     /* planner groups gates into tile passes; each
                              pass stages 2^t-amplitude tiles through shared
                              memory and applies many gates in registers
                              (exact FP32 / FP64 CUDA-core arithmetic) */
    QS_MODE_FUSED_TC = 2   /* as FUSED, but gates are merged into dense
                              k-qubit blocks applied as complex matrix
                              products on the tcgen05 tensor cores */
} qs_mode;

/* Operand precision of QS_MODE_FUSED_TC (ignored by the other modes).  The
 * block matrix (host-multiplied in FP64) and the state tile are split into
 * terms of the operand type; the products listed are accumulated in FP32
 * by the tensor cores.  The paper itself works in double precision
 * throughout (appendix "Quantum Simulation Details"); these forms trade
 * operand width for tensor-core rate. */
typedef enum {
    QS_PREC_DEFAULT = 0,   /* QS_PREC_FP16X3 */
    QS_PREC_FP16X3 = 1,    /* hi + lo FP16 terms of both operands, three
                              products (hi hi, hi lo, lo hi), per-tile
                              power-of-two scaling into FP16's range: ~22
                              significant bits */
    QS_PREC_BF16X3 = 2,    /* hi + lo BF16 terms, three products: ~16
                              significant bits; lossy against the 1e-5
                              state bound (its error is reported) */
    QS_PREC_BF16X6 = 3,    /* hi + mid + lo BF16 terms, six products (all
                              pairs of combined order <= 2): ~24 bits */
    QS_PREC_TF32X3 = 4,    /* hi + lo TF32 terms, three products: ~22 bits */
    QS_PREC_TF32 = 5       /* one TF32 term, one product: ~11 bits; lossy,
                              for comparison (its error is reported) */
} qs_precision;

/* Options for qs_apply_circuit; NULL means defaults
 * {QS_MODE_FUSED, QS_PREC_DEFAULT, k = 0 (library choice), tile_log2 = 0
 * (library choice), autotune = 0}. */
typedef struct {
    int mode;        /* qs_mode */
    int precision;   /* qs_precision */
    int k;           /* TC block size in qubits (6 is the only built value) */
    int tile_log2;   /* fused tile size in amplitudes, log2 (0 = default) */
    int autotune;    /* 1: the library times candidate tile sizes (and, for
                        QS_MODE_FUSED_TC, the register form) and keeps the
                        fastest (see qs_apply_circuit, qs_batch_set_options);
                        0: use the other fields as given */
} qs_opts;

/* Planner summary (host-only, see qs_plan_circuit). */
typedef struct {
    int passes;          /* state passes (kernel launches over the state) */
    int phases;          /* register / tensor-core phases over all passes */
    int ops;             /* device ops over all phases */
    int tile_log2;       /* tile size used, log2 amplitudes */
    int reg_log2;        /* register (or block) bits per phase */
    int gates;           /* gates planned */
    double bytes;        /* algorithmic HBM bytes of the plan (read+write) */
} qs_plan_stats;

/* Library version string, e.g. "qs 1.0 sm_103a". */
const char *qs_version(void);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *qs_last_error(void);

/* Creates an n-qubit state (1 <= n <= 34) of type dt in device memory owned
 * by the library, initialised to |0...0>, with all work ordered on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * Returns QS_ERR_OOM if 2^n amplitudes do not fit.  *out is set only on
 * success. */
qs_status qs_state_create(int n, qs_dtype dt, void *cuda_stream, qs_state **out);

/* Wraps caller-owned device memory `device_amps` (2^n amplitudes of type dt,
 * 16-byte aligned) as a state.  The contents are left untouched.  The
 * library still allocates its small statistics workspace. */
qs_status qs_state_attach(int n, qs_dtype dt, void *device_amps,
                          void *cuda_stream, qs_state **out);

/* Releases the handle (and the amplitudes if the library owns them).
 * NULL is accepted.  Synchronises the state's stream first. */
qs_status qs_state_destroy(qs_state *s);

/* Device pointer of the amplitudes (interleaved re, im).  Once the caller
 * holds the pointer, resets are written at once and the library assumes
 * nothing about the contents (see qs_state_reset): read-out results are
 * formed afresh by every call. */
qs_status qs_state_amplitudes(const qs_state *s, void **device_amps);

/* Sets the state to |0...0>.  For a state whose memory the caller cannot
 * reach (created by qs_state_create, pointer never taken) the write is
 * deferred to the next call that uses the state, and a following
 * qs_apply_circuit whose gates open with H on every qubit takes the uniform
 * superposition 2^(-n/2) in their place (Sec. "Convergence to
 * Porter-Thomas": cycle 0 is that layer): the first fused pass generates it
 * in its tiles instead of reading the state (plain mode: one fill), and in
 * QS_MODE_FUSED also forms the phases of the T and CZ gates that follow the
 * layer before any non-diagonal gate on their qubits.  Attached states,
 * and states whose pointer was taken, are written at once. */
qs_status qs_state_reset(qs_state *s);

/* Applies `ngates` gates (host array, read during the call) in order:
 * |psi> <- G_{ngates-1} ... G_0 |psi>  (Eq. sqgunitaryoperation for each
 * single-qubit gate; controlled form for CZ / CPHASE).  Every gate is
 * validated first (kind < 9, qubits < n, q0 != q1 for two-qubit kinds); on
 * error nothing is launched.  `opts` may be NULL.
 * opts->autotune = 1 (fused modes, tile_log2 = 0): the first call for a
 * given (device, n, dtype, mode, precision) times this gate list on a
 * scratch copy of the state (allocated stream-ordered for the duration of
 * the call) with every candidate tile size (9..13 qubits, 12 for
 * complex128, at most n) and, when QS_MODE_FUSED_TC was asked for, the
 * tensor-core form; the fastest is cached for the rest of the process and
 * used by this and later calls.  States of more than 26 qubits use the
 * defaults (13-qubit tiles, the fastest measured from 20 qubits on). */
qs_status qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t ngates,
                           const qs_opts *opts);

/* Plans `gates` for this state on the host and enqueues the plan upload on
 * the state's stream without launching any kernel.  A following
 * qs_apply_circuit with the same gate list and options reuses the plan, so
 * its call only launches kernels.  The state keeps two plans: preparing the
 * next circuit while the device still evolves the state with the other plan
 * does not wait for the device (the host blocks only when the slot it
 * replaces is still in use by earlier enqueued work).  `gates` may be
 * released on return.  Validation as for qs_apply_circuit; QS_MODE_PLAIN
 * needs no plan and returns QS_OK. */
qs_status qs_prepare_circuit(qs_state *s, const qs_gate *gates, size_t ngates,
                             const qs_opts *opts);

/* Runs the planner only (no device work): fills *stats for the given gate
 * list, qubit count, dtype and options. */
qs_status qs_plan_circuit(int n, qs_dtype dt, const qs_gate *gates,
                          size_t ngates, const qs_opts *opts,
                          qs_plan_stats *stats);

/* Writes p_U(x) = |<x|psi>|^2 for all 2^n x in canonical order into `out`
 * (host or device, caller-owned): doubles if out_is_fp64, else floats.
 * Asynchronous for device `out`; synchronous for host `out`.  For complex64
 * states the same read of the state also forms the partial sums of
 * qs_pt_moments and the chunk sums of qs_sample; those calls reuse them
 * while the amplitudes are unchanged (never for a state whose pointer the
 * caller holds), with the same results as a fresh pass. */
qs_status qs_probabilities(const qs_state *s, void *out, int out_is_fp64);

/* As qs_probabilities, but stream-ordered for every kind of `out` except
 * pageable host memory (which is served synchronously, as by
 * qs_probabilities).  For page-locked host `out` (cudaHostAlloc /
 * cudaHostRegister) the read-out kernel runs on the state's stream and, for
 * complex64 states with 16-byte aligned `out`, writes a share of the
 * probabilities (whole groups of 256, from index 0) into `out` itself; the
 * rest (all of them for complex128 states or unaligned `out`) goes to a
 * library-owned device buffer (2^n floats or doubles, allocated on first use
 * and kept with the state) and is copied to `out` by the copy engine on a
 * second stream, so the copy overlaps the work the caller enqueues next
 * (e.g. the next circuit).  The share is 0 unless set by
 * qs_readout_share: writing part of the output directly pays on hosts where
 * the copy engine cannot move the whole read-out in the time of the work
 * between read-outs (the kernel's own host writes hold up the state's
 * stream, the copy engine's do not).  `out` holds the probabilities of the
 * state as it was at the call once qs_state_sync(s) has returned; until
 * then the caller must neither read nor free it.  Successive asynchronous read-outs
 * of one state are copied in call order; the values are those of
 * qs_probabilities whatever the share.  QS_ERR_OOM if the device buffer
 * cannot be allocated. */
qs_status qs_probabilities_async(const qs_state *s, void *out, int out_is_fp64);

/* Share of qs_probabilities_async's output that the read-out kernel writes
 * into page-locked host memory itself (complex64 states; rounded to whole
 * groups of 256 probabilities).  `share` in [0, 1] sets it for the
 * following calls; a negative value restores the default, 0 (everything
 * through the copy engine); NaN changes nothing.  `current` (may be NULL)
 * receives the share in force.  QS_ERR_INVALID_ARG for a share above 1. */
qs_status qs_readout_share(qs_state *s, double share, double *current);

/* Waits for all work of the state: its stream and any asynchronous
 * read-out copies (qs_probabilities_async).  QS_ERR_CUDA on a device error. */
qs_status qs_state_sync(const qs_state *s);

/* Draws k bitstrings from p_U (inverse-CDF sampling, Sec. "Characterizing
 * quantum supremacy", step 2 of the procedure).  Sample j uses the uniform
 * u_j = (SplitMix64 output j of a stream seeded with `seed`) >> 11, times
 * 2^-53, and returns the smallest x with C_x > u_j * C_{N-1}, where C is the
 * cumulative sum of p in index order.  The total C_{N-1} normalises away any
 * norm drift; x with p(x) = 0 is never returned.  `out` (host or device,
 * caller-owned) receives k uint64 indices in sample order.  Synchronous for
 * host `out`.  Returns QS_ERR_INVALID_ARG if the state has zero norm. */
qs_status qs_sample(const qs_state *s, uint64_t k, uint64_t seed, uint64_t *out);

/* Allocation-free variant of qs_sample, for callers that must not allocate
 * device memory while they run: applications and host frameworks that hand
 * all device memory to their own pool or fix their memory budget up front,
 * so that a library call that allocates would fail or break that budget.
 * The paper has no counterpart; it is a deployment convenience.
 *   n, dt, device_amps: the state (2^n amplitudes of type dt in device
 *     memory, 16-byte aligned, canonical order), read only;
 *   k, seed: as for qs_sample; device_out: k uint64 slots in device memory.
 * Results are identical to qs_sample's for the same state, k and seed.  The
 * scratch (one FP64 sum per 256 amplitudes plus scan totals) is a fixed
 * array of 8 MiB compiled into the library, held by every GPU that loads it
 * until the process exits, so n is limited to 1..28 (larger n returns
 * QS_ERR_INVALID_ARG before any device work).  No call allocates memory.
 * Every call looks up the current device's address of the array; the first
 * call on a device also loads the library's device code there.  All calls
 * share the one array: calls whose work overlaps on the GPU (different
 * streams, or host threads) race and must be serialised by the caller; the
 * array keeps the previous call's contents, and every entry a call reads is
 * written by that same call first.  Work is ordered on cuda_stream (NULL =
 * legacy default stream); the call synchronises that stream once to check
 * the norm (QS_ERR_INVALID_ARG for a zero or non-finite norm) and returns
 * with the search kernel queued. */
qs_status qs_sample_noalloc(int n, qs_dtype dt, const void *device_amps, void *cuda_stream,
                            uint64_t k, uint64_t seed, uint64_t *device_out);

/* Cross entropy of a sample against the ideal distribution, Eq. ae:
 *   *ce = (1/m) sum_j ln(1/p_U(x_j)),  *delta_h = ln N + gamma - *ce
 * (gamma = Euler's constant; ln N + gamma = H_0 of Eq. au).  `samples`
 * (host or device) holds m indices < 2^n; an index out of range returns
 * QS_ERR_INVALID_ARG.  ce or delta_h may be NULL.  Synchronous. */
qs_status qs_cross_entropy(const qs_state *s, const uint64_t *samples,
                           uint64_t m, double *ce, double *delta_h);

/* Gradient of the sample cross entropy L(theta) = -(1/m) sum_j ln p_theta(x_j)
 * (the CE of Eq. ae) with respect to the angle of every parameterised gate
 * (RX, RY, RZ, CPHASE) of `gates`, by the adjoint method: the call resets the
 * state to |0...0>, evolves it with `gates` (form chosen by `opts`, NULL =
 * fused), computes *loss = L on the m sample indices `samples` (host or
 * device), seeds lambda = -sum_j psi(x_j) / (m p(x_j)) |x_j>, and sweeps the
 * gates in reverse, uncomputing psi and lambda with G^dagger and reading
 *   dL/dtheta = Im <lambda|P|psi>            for R_P(theta) = exp(-i theta/2 P),
 *   dL/dphi   = -2 Im <lambda|Pi_11|psi>     for CPHASE(phi).
 * grad[k] receives the derivative for gate k (0 for fixed gates).  Uses one
 * extra state vector (lambda), allocated stream-ordered for the call.  On
 * return the state holds the uncomputed vector (|0...0> up to rounding).
 * The paper has no gradients; this serves circuit-parameter studies around
 * the paper's cross-entropy benchmark.  Synchronous. */
qs_status qs_adjoint_gradient(qs_state *s, const qs_gate *gates, size_t ngates,
                              const uint64_t *samples, uint64_t m, const qs_opts *opts,
                              double *loss, double *grad);

/* Statistics after every cycle (Sec. "Convergence to Porter-Thomas":
 * statistics of measurements after each cycle; Figs. evd and mvd follow
 * entropy and inverse participation ratios with depth).  Resets the state
 * to |0...0>, then for each run of gates with equal `cycle` field (cycle
 * numbers must not decrease) applies that cycle (form chosen by `opts`) and
 * records the statistics of qs_pt_moments: stats[c*(4+kmax) ..] = cycle,
 * norm, entropy, uniform cross entropy, moments 1..kmax.  *ncycles receives
 * the number of cycles; if stats is NULL or capacity (rows) is smaller,
 * nothing is run (count query).  The planner fuses gates only within a cycle
 * here, since the state must exist after each one.  Synchronous. */
qs_status qs_cycle_statistics(qs_state *s, const qs_gate *gates, size_t ngates, const qs_opts *opts,
                              int kmax, double *stats, size_t capacity, size_t *ncycles);

/* Denser random circuits with periodic boundaries (appendix "Depth to
 * reach Porter-Thomas for denser 2D circuits"), on a rows x cols torus (both
 * even, rows * cols <= 64; qubit r*cols+c):
 *   cycle 0: H on every qubit;
 *   layer l = 1..layers: cycle 2l-1 single-qubit gates, cycle 2l CZ gates.
 * The CZ cycle of layer l puts every qubit in exactly one CZ, pattern
 * (l-1) mod 4 of H_even, V_even, H_odd, V_odd (horizontal / vertical
 * nearest-neighbour pairs starting at an even / odd column / row, wrapping
 * around the torus).  Single-qubit gates follow the rules of
 * qs_circuit_generate (only after a CZ in the previous cycle, T first after
 * H, then a SplitMix64 pick from {X^1/2, Y^1/2, T} without the previous
 * gate), so layer 1 has CZs only.  Output, count query and errors as
 * qs_circuit_generate. */
qs_status qs_circuit_generate_dense(int rows, int cols, int layers, uint64_t seed,
                                    qs_gate *out, size_t *ngates);

/* Convergence to Porter-Thomas (Sec. "Convergence to Porter-Thomas", Fig.
 * pt_depth): *first = the smallest i such that entropy[j] is within 4 sigma
 * of ln N - 1 + gamma for every j >= i, sigma = 0.75 * 2^(-n/2) (the
 * spread of the entropy of Porter-Thomas states), N = 2^n; count if the last
 * entry is outside.  Host only, entropy[count] read during the call. */
qs_status qs_pt_convergence(const double *entropy, size_t count, int n, size_t *first);

/* Porter-Thomas statistics of p_U in one read of the state, FP64
 * accumulation (Sec. "Convergence to Porter-Thomas").  They are computed
 * for the normalised distribution p / S, S = sum p, so that the rounding
 * drift of the state's norm does not enter them (the paper's quantities are
 * defined for a normalised distribution):
 *   moments[k-1] = N^{k-1} sum_x (p_x/S)^k for k = 1..kmax (kmax <= 10), the
 *                  normalised inverse participation ratios (-> k! for
 *                  Porter-Thomas);
 *   *entropy     = -sum (p/S) ln(p/S) (Eq. lps; Porter-Thomas value
 *                  ln N - 1 + gamma, Eq. eu);
 *   *uniform_ce  = -(1/N) sum ln(p/S) (Eq. eue; ln N + gamma), +inf if some
 *                  p is exactly zero;
 *   *norm        = S = sum p.
 * For a zero state: norm 0, entropy 0, uniform_ce +inf, moments 0.
 * Any output pointer may be NULL (kmax = 0 skips moments).  Synchronous. */
qs_status qs_pt_moments(const qs_state *s, int kmax, double *moments,
                        double *entropy, double *uniform_ce, double *norm);

/* Batched ensemble of independent circuits (the paper's statistics are
 * ensemble averages over circuit instances, Secs. "Characterizing quantum
 * supremacy" and "Convergence to Porter-Thomas").  All `count` complex64
 * states (nqubits[i] in 5..30) stay resident in one device allocation made
 * by qs_batch_create; work is ordered on cuda_stream (NULL = legacy default
 * stream). */
typedef struct qs_batch qs_batch;
qs_status qs_batch_create(int count, const int *nqubits, void *cuda_stream, qs_batch **out);

/* Resets every state to |0...0>, applies instance i's gates
 * gates[offsets[i] .. offsets[i+1]) (host arrays, offsets has count+1
 * entries, offsets[0] = 0), and writes per-instance statistics of the
 * normalised output distribution (as qs_pt_moments) to stats[i*(3+kmax) ..]:
 * norm, entropy, uniform cross entropy, moments 1..kmax (kmax <= 10; stats
 * may be NULL when kmax = 0).  The engine (qs_batch_set_engine) decides how
 * the device work is issued: by default one persistent launch runs the reset,
 * every instance's fused tile passes and the statistics from a device work
 * queue (each work item waits, bounded, only for its own instance's earlier
 * items; QS_ERR_TIMEOUT if such a wait runs out, which a correct run never
 * meets); the lockstep engine runs round r (pass r of every instance) as
 * one launch per tile size.  The device work is captured once into a CUDA
 * graph and replayed while the gate lists are unchanged (a new gate list
 * replans and recaptures).  Synchronous. */
qs_status qs_batch_run(qs_batch *b, const qs_gate *gates, const uint64_t *offsets, int kmax,
                       double *stats);

/* Samples every instance of the batch (its current states): out[i*k + j],
 * j < k, is sample j of instance i, drawn by the inverse-CDF rule of
 * qs_sample from u = the counter-based draw number i*k + j of the stream
 * seeded with `seed` (see qs_sample), then each bit b < n_i flipped when the
 * draw number (i*k + j)*64 + b of the stream seeded with
 * seed ^ 0xD1B54A32D192ED03 is below r_mes (the measurement bit-flip errors
 * of the digital error model, Sec. "Characterizing quantum supremacy";
 * r_mes = 0: plain samples).  An instance with zero norm gives
 * UINT64_MAX samples.  out is a host array of count*k entries.
 * Synchronous. */
qs_status qs_batch_sample(qs_batch *b, uint64_t k, uint64_t seed, double r_mes, uint64_t *out);

/* One discrete error at a chosen location (appendix "Residual correlations
 * after discrete errors", Fig. 1error): copies the gate list (cycle numbers
 * must not decrease) and inserts the Pauli `pauli` (1 = X, 2 = Y, 3 = Z,
 * emitted as R_X / R_Y / R_Z(pi)) on `qubit` after the last gate whose cycle
 * is <= `cycle` (cycle 0 = right after the H layer).  Output and count
 * query as qs_circuit_generate (ngates + 1 gates).  Host only. */
qs_status qs_single_error_circuit(const qs_gate *gates, size_t ngates, int n, uint32_t cycle,
                                  int qubit, int pauli, qs_gate *out, size_t *nout);

/* Residual correlations after discrete errors (appendix "Residual
 * correlations after discrete errors", Figs. zcorr / xcorr): corr[i] =
 * Pearson correlation over the 2^n basis states between instance i's output
 * distribution and the reference state's, both complex64 of the same n
 * (e.g. the circuit with one Pauli inserted vs the ideal circuit).  Sums of
 * p_i p_ref, p_i^2, p_i, p_ref^2, p_ref are accumulated in FP64 over FP32
 * products; corr = cov / sqrt(var_i var_ref) (0 if a variance is zero).
 * Synchronous. */
qs_status qs_batch_correlation(qs_batch *b, const qs_state *ref, double *corr);

/* Mean output distribution over all instances (same n), out[x] =
 * (1/count) sum_i |<x|psi_i>|^2 in FP64, host array of 2^n doubles: the
 * error-averaged distribution of Fig. 1error when the instances carry one
 * Pauli error each.  Synchronous. */
qs_status qs_batch_mean_probabilities(qs_batch *b, double *out);

/* One trajectory of the digital error model (Sec. "Characterizing quantum
 * supremacy": a depolarising channel after every gate, Eq. 6): copies the
 * gate list, inserting after each one-qubit gate, with probability r1, one
 * of X, Y, Z (each r1/3), and after each two-qubit gate, with probability
 * r2, one of the 15 non-identity two-qubit Paulis (each r2/15), and before
 * the circuit an X on each qubit with probability r_init (initialisation
 * bit flip).  Paulis are emitted as QS_RX / QS_RY / QS_RZ with theta = pi
 * (the Pauli times the global phase -i), in the cycle of the gate they
 * follow.  Draws: one SplitMix64 stream seeded with `seed`, u = (z >> 11)
 * 2^-53; first one per qubit (initialisation, X if u < r_init), then one per
 * gate in list order (one-qubit: Pauli floor(3u/r1) of X, Y, Z if u < r1;
 * two-qubit: if u < r2, e = floor(15u/r2) + 1 read as base-4 digits
 * (e / 4 on q0, e % 4 on q1; 0 = I, 1..3 = X, Y, Z)).  Output and count
 * query as qs_circuit_generate (*nout in: capacity, out: count).  Host only. */
qs_status qs_noisy_circuit(const qs_gate *gates, size_t ngates, int n, double r1, double r2,
                           double r_init, uint64_t seed, qs_gate *out, size_t *nout);

/* qs_batch_run without statistics: resets every state and applies instance
 * i's gates (same arguments and rules, kmax = 0). */
qs_status qs_batch_apply(qs_batch *b, const qs_gate *gates, const uint64_t *offsets);

/* Device pointer of instance i's amplitudes (canonical order). */
qs_status qs_batch_state(const qs_batch *b, int i, void **device_amps);

/* Options of later runs of the batch (the paper has no counterpart; a
 * throughput knob of the ensemble engine): opts->mode must be
 * QS_MODE_FUSED (the batched pass has no tensor-core form:
 * QS_ERR_UNSUPPORTED for QS_MODE_FUSED_TC); opts->tile_log2 in 5..13 fixes
 * the tile size of every instance (0 = the planner's default, 13 qubits or
 * n if smaller); opts->autotune = 1 lets the library choose the tile size
 * per instance size n instead: on the next run it times the evolution of
 * the batch's own instances of each size n on the batch's engine with every
 * candidate tile size (9..13 qubits, at most n) on their own state memory
 * (CUDA events; one untimed and one timed run per candidate), keeps the
 * fastest, and caches the choice per (device, n, engine) for the rest of
 * the process, so later batches with instances of a size already seen skip
 * the timing.  NULL
 * restores the defaults.  The next run replans.  Host only. */
qs_status qs_batch_set_options(qs_batch *b, const qs_opts *opts);

/* Engines of the batched ensemble (qs_batch_set_engine). */
enum {
    QS_BATCH_PERSISTENT = 0,   /* one launch per run: a persistent kernel
                                  (two CTAs of 256 threads per SM) takes
                                  work items from a device queue: every
                                  instance's initial-state chunks (2^16
                                  amplitudes), then its fused passes in
                                  items of 2^18 amplitudes, round-major
                                  (pass r of every instance before pass
                                  r + 1 of any; larger instances first),
                                  then its statistics chunks; an item waits
                                  for its own instance's earlier items
                                  only, so instances overlap freely */
    QS_BATCH_ROUNDS = 1        /* lockstep rounds: round r (pass r of every
                                  instance) is one launch per tile size,
                                  the statistics two more launches */
};

/* Engine of later runs of the batch (the paper has no counterpart; how
 * the ensemble's device work is issued): QS_BATCH_PERSISTENT (the default)
 * or QS_BATCH_ROUNDS; anything else is QS_ERR_INVALID_ARG.  Both compute
 * the same states (per-tile arithmetic of the same plans) and the same
 * statistics partials, summed in the same order.  A change replans on the
 * next run; autotuned tile sizes are cached per engine.  Host only. */
qs_status qs_batch_set_engine(qs_batch *b, int engine);

/* After a run: tile_log2[i] (count entries, may be NULL) receives the tile
 * size of instance i's passes (0 when its list is only the Hadamard layer),
 * *run_bytes (may be NULL) the algorithmic HBM bytes of one run: 16 bytes
 * per amplitude per pass, plus the initial-state write and the statistics
 * read (8 bytes per amplitude each).  QS_ERR_INVALID_ARG before the first
 * run.  Host only. */
qs_status qs_batch_plan_info(const qs_batch *b, int *tile_log2, double *run_bytes);

qs_status qs_batch_destroy(qs_batch *b);

/* Copies the amplitudes to / from a host buffer of 2^n amplitudes in
 * canonical order (testing, checkpoints).  Synchronous. */
qs_status qs_state_copy_out(const qs_state *s, void *host_amps);
qs_status qs_state_copy_in(qs_state *s, const void *host_amps);

/* Random circuit of Sec. "Convergence to Porter-Thomas" on a rows x cols
 * grid (live sites numbered row-major are qubits 0..n-1; dead[r*cols+c] != 0
 * removes a site; dead may be NULL):
 *   cycle 0: H on every qubit;
 *   cycle t = 1..depth: CZ layout (t-1) mod 8, then on each qubit that was in
 *   a CZ at t-1 and is not in one at t: T if it is the qubit's first
 *   single-qubit gate after the H layer, else a uniform pick (SplitMix64
 *   stream seeded with `seed`, one draw per pick, top bit) from
 *   {X^1/2, Y^1/2, T} without the qubit's previous single-qubit gate.
 * The eight layouts (the paper's figure of them is not reproduced in the
 * text) are read as: H_a = horizontal edges (r,c)-(r,c+1) with
 * (c + 2r) mod 4 = a, V_a = vertical edges (r,c)-(r+1,c) with
 * (r + 2c) mod 4 = a, in the order H0 H2 V0 V2 H1 H3 V1 V3; edges touching
 * dead sites are dropped.  Within a cycle: CZs first (row-major edge order,
 * q0 < q1), then single-qubit gates by ascending qubit.
 * If out == NULL, *ngates receives the gate count; otherwise `out` must hold
 * *ngates entries on entry (capacity) and *ngates receives the count.
 * n = live sites must be 1..64. */
qs_status qs_circuit_generate(int rows, int cols, const uint8_t *dead,
                              int depth, uint64_t seed, qs_gate *out,
                              size_t *ngates);

/* Measurement support (no counterpart in the paper): the rate of fused
 * multiply-adds this GPU sustains, the denominator of the roofline of
 * arithmetic-bound kernels.  kind 0: scalar FP32, 1: packed FP32x2 (two
 * FMAs per instruction lane), 2: FP64.  Runs a few milliseconds of
 * independent FMA chains on every SM (64 warps each) on cuda_stream (NULL =
 * legacy default stream), timed with CUDA events; *fma_per_s receives FMAs
 * per second (flops / 2).  Synchronous; allocates a small output buffer
 * stream-ordered.  QS_ERR_INVALID_ARG for another kind. */
qs_status qs_alu_rate(int kind, void *cuda_stream, double *fma_per_s);

/* Build information (no counterpart in the paper).  qs_build_flags()
 * returns QS_BUILD_CHECKED for the checked build (libqs_checked.so,
 * compiled with QS_CHECKED): its kernels check their global-memory indices
 * against the state's size before each guarded access; a failed check skips
 * the access (no trap, no out-of-range access) and records a site code, and
 * the public calls that launch work (qs_apply_circuit, qs_probabilities,
 * qs_sample, qs_pt_moments, qs_cross_entropy, qs_batch_run,
 * qs_adjoint_gradient) synchronise the
 * device and return QS_ERR_INVALID_ARG naming the site.  The normal build
 * compiles the checks away. */
#define QS_BUILD_CHECKED 1
int qs_build_flags(void);

/* Checked build only: runs one guarded access one element past a small
 * device buffer, which the check catches (site 901), and returns the
 * resulting QS_ERR_INVALID_ARG -- a test of the check plumbing that touches
 * no memory out of range.  QS_ERR_UNSUPPORTED in the normal build. */
qs_status qs_check_probe(void);

#ifdef __cplusplus
}
#endif

#endif /* QS_PUBLIC_API_H_ */
