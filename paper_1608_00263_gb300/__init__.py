"""GB300 (sm_103a) state-vector library for the random-circuit sampling method of
Boixo et al., "Characterizing Quantum Supremacy in Near-Term Devices"
(arXiv:1608.00263).

Thin Python binding of the C ABI in ``include/qs.h``: the functions below
carry the C names and only marshal arguments (numpy arrays, torch tensors or
raw pointers) into ``libqs.so``.  Every step of the method runs in the
library's CUDA kernels; if the library is missing the calls raise.
"""
import ctypes

import numpy as np

from . import _native as N
from ._native import (GATE_DTYPE, QSError, QS_C64, QS_C128, QS_H, QS_X_HALF, QS_Y_HALF, QS_T,
                      QS_CZ, QS_RX, QS_RY, QS_RZ, QS_CPHASE, QS_MODE_PLAIN, QS_MODE_FUSED,
                      QS_MODE_FUSED_TC, QS_PREC_DEFAULT, QS_PREC_FP16X3, QS_PREC_BF16X3,
                      QS_PREC_BF16X6, QS_PREC_TF32X3, QS_PREC_TF32, QS_BATCH_PERSISTENT,
                      QS_BATCH_ROUNDS)

__all__ = [
    "GATE_DTYPE", "QSError", "QS_C64", "QS_C128", "QS_H", "QS_X_HALF", "QS_Y_HALF", "QS_T",
    "QS_CZ", "QS_RX", "QS_RY", "QS_RZ", "QS_CPHASE", "QS_MODE_PLAIN", "QS_MODE_FUSED",
    "QS_MODE_FUSED_TC", "QS_PREC_DEFAULT", "QS_PREC_FP16X3", "QS_PREC_BF16X3",
    "QS_PREC_BF16X6", "QS_PREC_TF32X3", "QS_PREC_TF32", "QS_BATCH_PERSISTENT", "QS_BATCH_ROUNDS",
    "qs_version", "qs_last_error", "qs_state_create", "qs_state_attach", "qs_state_destroy",
    "qs_state_amplitudes", "qs_state_reset", "qs_apply_circuit", "qs_prepare_circuit",
    "qs_plan_circuit",
    "qs_probabilities", "qs_probabilities_async", "qs_readout_share", "qs_state_sync", "qs_sample", "qs_sample_noalloc",
    "qs_cross_entropy", "qs_pt_moments",
    "qs_state_copy_out", "qs_state_copy_in", "qs_circuit_generate", "qs_adjoint_gradient",
    "qs_batch_create", "qs_batch_run", "qs_batch_state", "qs_batch_destroy", "qs_cycle_statistics",
    "qs_circuit_generate_dense", "qs_pt_convergence", "qs_noisy_circuit", "qs_batch_sample",
    "qs_batch_correlation", "qs_batch_mean_probabilities", "qs_single_error_circuit", "qs_batch_apply",
    "qs_alu_rate", "qs_batch_set_options", "qs_batch_plan_info", "qs_batch_set_engine", "qs_build_flags", "qs_check_probe",
    "library_path",
]


def library_path():
    return N.LIB_PATH


def _ptr(x):
    """Raw address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch tensor, numpy array or int address, got %r" % type(x))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(mode, precision, k, tile_log2, autotune=0):
    return N.qs_opts(mode, precision, k, tile_log2, autotune)


def _gates(gates):
    g = np.ascontiguousarray(gates)
    if g.dtype != GATE_DTYPE:
        g = g.astype(GATE_DTYPE)
    return g


def qs_version():
    return N.lib().qs_version().decode()


def qs_last_error():
    return N.lib().qs_last_error().decode()


def qs_state_create(n, dtype=QS_C64, stream=None):
    h = ctypes.c_void_p()
    N.check(N.lib().qs_state_create(n, dtype, _stream(stream), ctypes.byref(h)))
    return h.value


def qs_state_attach(n, dtype, amps, stream=None):
    h = ctypes.c_void_p()
    N.check(N.lib().qs_state_attach(n, dtype, _ptr(amps), _stream(stream), ctypes.byref(h)))
    return h.value


def qs_state_destroy(h):
    N.check(N.lib().qs_state_destroy(h))


def qs_state_amplitudes(h):
    p = ctypes.c_void_p()
    N.check(N.lib().qs_state_amplitudes(h, ctypes.byref(p)))
    return p.value


def qs_state_reset(h):
    N.check(N.lib().qs_state_reset(h))


def qs_apply_circuit(h, gates, mode=QS_MODE_FUSED, precision=QS_PREC_DEFAULT, k=0, tile_log2=0,
                     autotune=0):
    g = _gates(gates)
    o = _opts(mode, precision, k, tile_log2, autotune)
    N.check(N.lib().qs_apply_circuit(h, g.ctypes.data if g.size else None, g.size, ctypes.byref(o)))


def qs_prepare_circuit(h, gates, mode=QS_MODE_FUSED, precision=QS_PREC_DEFAULT, k=0, tile_log2=0):
    g = _gates(gates)
    o = _opts(mode, precision, k, tile_log2)
    N.check(N.lib().qs_prepare_circuit(h, g.ctypes.data if g.size else None, g.size, ctypes.byref(o)))


def qs_plan_circuit(n, dtype, gates, mode=QS_MODE_FUSED, precision=QS_PREC_DEFAULT, k=0,
                    tile_log2=0):
    g = _gates(gates)
    o = _opts(mode, precision, k, tile_log2)
    st = N.qs_plan_stats()
    N.check(N.lib().qs_plan_circuit(n, dtype, g.ctypes.data if g.size else None, g.size,
                                    ctypes.byref(o), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in N.qs_plan_stats._fields_}


def qs_probabilities(h, out, fp64=True):
    """Writes |<x|psi>|^2 into `out` (torch tensor, numpy array or address)."""
    N.check(N.lib().qs_probabilities(h, _ptr(out), 1 if fp64 else 0))
    return out


def qs_probabilities_async(h, out, fp64=True):
    """As qs_probabilities, stream-ordered; page-locked host `out` is filled
    partly by the read-out kernel and partly by the copy engine while later
    work runs: complete after qs_state_sync."""
    N.check(N.lib().qs_probabilities_async(h, _ptr(out), 1 if fp64 else 0))
    return out


def qs_readout_share(h, share=float("nan")):
    """Share of an asynchronous read-out the kernel writes into host memory
    itself: 0..1 sets it, negative restores the default 0 (all through the
    copy engine), NaN (the default argument) only reads it.  Returns the
    share in force."""
    cur = ctypes.c_double()
    N.check(N.lib().qs_readout_share(h, float(share), ctypes.byref(cur)))
    return cur.value


def qs_state_sync(h):
    """Waits for the state's stream and its asynchronous read-out copies."""
    N.check(N.lib().qs_state_sync(h))


def qs_sample(h, k, seed, out=None):
    """k samples; returns a uint64 numpy array unless `out` is given."""
    if out is None:
        out = np.empty(k, dtype=np.uint64)
    N.check(N.lib().qs_sample(h, k, seed & (2**64 - 1), _ptr(out)))
    return out


def qs_sample_noalloc(n, dtype, amps, k, seed, out, stream=None):
    """Allocation-free sampling from a state given by its device pointer;
    `out` is a device buffer of k uint64 (see include/qs.h)."""
    N.check(N.lib().qs_sample_noalloc(n, dtype, _ptr(amps), _stream(stream), k, seed & (2**64 - 1),
                                      _ptr(out)))
    return out


def qs_cross_entropy(h, samples):
    """Returns (CE, Delta H) of Eq. ae for the sample indices."""
    if isinstance(samples, np.ndarray):
        samples = np.ascontiguousarray(samples, dtype=np.uint64)
        m = samples.size
    else:
        m = samples.numel()
    ce = ctypes.c_double()
    dh = ctypes.c_double()
    N.check(N.lib().qs_cross_entropy(h, _ptr(samples), m, ctypes.byref(ce), ctypes.byref(dh)))
    return ce.value, dh.value


def qs_adjoint_gradient(h, gates, samples, mode=QS_MODE_FUSED):
    """Returns (loss, grad): the sample cross entropy and its derivative with
    respect to each gate's angle (0 for fixed gates), by the adjoint method."""
    g = _gates(gates)
    if isinstance(samples, np.ndarray):
        samples = np.ascontiguousarray(samples, dtype=np.uint64)
        m = samples.size
    else:
        m = samples.numel()
    grad = np.zeros(g.size, dtype=np.float64)
    loss = ctypes.c_double()
    o = _opts(mode, QS_PREC_DEFAULT, 0, 0)
    N.check(N.lib().qs_adjoint_gradient(h, g.ctypes.data if g.size else None, g.size, _ptr(samples), m,
                                        ctypes.byref(o), ctypes.byref(loss), grad.ctypes.data))
    return loss.value, grad


def qs_pt_moments(h, kmax=10):
    m = (ctypes.c_double * max(kmax, 1))()
    ent, uce, nrm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(N.lib().qs_pt_moments(h, kmax, m, ctypes.byref(ent), ctypes.byref(uce),
                                  ctypes.byref(nrm)))
    return {"moments": np.array(m[:kmax]), "entropy": ent.value, "uniform_ce": uce.value,
            "norm": nrm.value}


def qs_state_copy_out(h, n, dtype=QS_C64):
    out = np.empty(1 << n, dtype=np.complex64 if dtype == QS_C64 else np.complex128)
    N.check(N.lib().qs_state_copy_out(h, out.ctypes.data))
    return out


def qs_state_copy_in(h, amps):
    a = np.ascontiguousarray(amps)
    N.check(N.lib().qs_state_copy_in(h, a.ctypes.data))


def qs_circuit_generate(rows, cols, depth, seed, dead=None):
    d = None
    if dead is not None:
        d = np.ascontiguousarray(dead, dtype=np.uint8)
    cnt = ctypes.c_size_t(0)
    dp = d.ctypes.data if d is not None else None
    N.check(N.lib().qs_circuit_generate(rows, cols, dp, depth, seed & (2**64 - 1), None,
                                        ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    N.check(N.lib().qs_circuit_generate(rows, cols, dp, depth, seed & (2**64 - 1),
                                        out.ctypes.data, ctypes.byref(cnt)))
    return out


def qs_circuit_generate_dense(rows, cols, layers, seed):
    """Dense periodic-boundary random circuit (every qubit in one CZ per CZ cycle)."""
    cnt = ctypes.c_size_t(0)
    N.check(N.lib().qs_circuit_generate_dense(rows, cols, layers, seed & (2**64 - 1), None,
                                              ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    N.check(N.lib().qs_circuit_generate_dense(rows, cols, layers, seed & (2**64 - 1),
                                              out.ctypes.data, ctypes.byref(cnt)))
    return out


def qs_noisy_circuit(gates, n, r1, r2, r_init, seed):
    """One trajectory of the depolarising error model (Paulis inserted after gates)."""
    g = _gates(gates)
    gp = g.ctypes.data if g.size else None
    cnt = ctypes.c_size_t(0)
    N.check(N.lib().qs_noisy_circuit(gp, g.size, n, r1, r2, r_init, seed & (2**64 - 1), None,
                                     ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    N.check(N.lib().qs_noisy_circuit(gp, g.size, n, r1, r2, r_init, seed & (2**64 - 1),
                                     out.ctypes.data, ctypes.byref(cnt)))
    return out


def qs_batch_sample(b, k, seed, r_mes=0.0):
    """k samples of every instance (array (count, k)), measurement flips at rate r_mes."""
    count = _batch_sizes.get(b)
    if count is None:
        raise QSError(N.QS_ERR_INVALID_ARG, "unknown batch handle")
    out = np.zeros(count * k, dtype=np.uint64)
    N.check(N.lib().qs_batch_sample(b, k, seed & (2**64 - 1), float(r_mes),
                                    out.ctypes.data if out.size else None))
    return out.reshape(count, k)


def qs_single_error_circuit(gates, n, cycle, qubit, pauli):
    """The gate list with one Pauli (1 X, 2 Y, 3 Z) on `qubit` after cycle `cycle`."""
    g = _gates(gates)
    cnt = ctypes.c_size_t(g.size + 1)
    out = np.zeros(g.size + 1, dtype=GATE_DTYPE)
    N.check(N.lib().qs_single_error_circuit(g.ctypes.data if g.size else None, g.size, n, cycle, qubit, pauli,
                                            out.ctypes.data, ctypes.byref(cnt)))
    return out


def qs_batch_correlation(b, ref):
    """Pearson correlation of every instance's distribution with the reference state's."""
    count = _batch_sizes.get(b)
    if count is None:
        raise QSError(N.QS_ERR_INVALID_ARG, "unknown batch handle")
    out = np.zeros(count, dtype=np.float64)
    N.check(N.lib().qs_batch_correlation(b, ref, out.ctypes.data))
    return out


def qs_batch_mean_probabilities(b, n):
    """Mean distribution over the batch's instances (all of n qubits)."""
    out = np.zeros(1 << n, dtype=np.float64)
    N.check(N.lib().qs_batch_mean_probabilities(b, out.ctypes.data))
    return out


def qs_pt_convergence(entropy, n):
    """First index from which the entropy series stays within 4 sigma of Porter-Thomas."""
    e = np.ascontiguousarray(entropy, dtype=np.float64)
    first = ctypes.c_size_t(0)
    N.check(N.lib().qs_pt_convergence(e.ctypes.data if e.size else None, e.size, n, ctypes.byref(first)))
    return first.value


_batch_sizes = {}     # batch handle -> instance count (for output shapes)


def qs_batch_create(nqubits, stream=None):
    n = np.ascontiguousarray(nqubits, dtype=np.int32)
    h = ctypes.c_void_p()
    N.check(N.lib().qs_batch_create(int(n.size), n.ctypes.data, _stream(stream), ctypes.byref(h)))
    _batch_sizes[h.value] = int(n.size)
    return h.value


def qs_batch_run(b, gate_lists, kmax=10):
    """Runs every instance's gate list; returns an array (count, 3 + kmax):
    norm, entropy, uniform cross entropy, moments 1..kmax."""
    gl = [_gates(g) for g in gate_lists]
    offsets = np.zeros(len(gl) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([g.size for g in gl])
    gates = np.concatenate(gl) if gl else np.zeros(0, dtype=GATE_DTYPE)
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    out = np.zeros((len(gl), 3 + kmax), dtype=np.float64)
    N.check(N.lib().qs_batch_run(b, gates.ctypes.data if gates.size else None, offsets.ctypes.data, kmax,
                                 out.ctypes.data))
    return out


def qs_batch_apply(b, gate_lists):
    """Resets every instance and applies its gate list (no statistics)."""
    gl = [_gates(g) for g in gate_lists]
    offsets = np.zeros(len(gl) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([g.size for g in gl])
    gates = np.ascontiguousarray(np.concatenate(gl) if gl else np.zeros(0, dtype=GATE_DTYPE), dtype=GATE_DTYPE)
    N.check(N.lib().qs_batch_apply(b, gates.ctypes.data if gates.size else None, offsets.ctypes.data))


def qs_batch_state(b, i):
    p = ctypes.c_void_p()
    N.check(N.lib().qs_batch_state(b, i, ctypes.byref(p)))
    return p.value


def qs_batch_destroy(b):
    _batch_sizes.pop(b, None)
    N.check(N.lib().qs_batch_destroy(b))


def qs_cycle_statistics(h, gates, kmax=10, mode=QS_MODE_FUSED):
    """Statistics after every cycle: array (cycles, 4 + kmax) of cycle, norm,
    entropy, uniform cross entropy, moments 1..kmax."""
    g = _gates(gates)
    o = _opts(mode, QS_PREC_DEFAULT, 0, 0)
    cnt = ctypes.c_size_t(0)
    gp = g.ctypes.data if g.size else None
    N.check(N.lib().qs_cycle_statistics(h, gp, g.size, ctypes.byref(o), kmax, None, 0, ctypes.byref(cnt)))
    out = np.zeros((cnt.value, 4 + kmax), dtype=np.float64)
    N.check(N.lib().qs_cycle_statistics(h, gp, g.size, ctypes.byref(o), kmax, out.ctypes.data, cnt.value,
                                        ctypes.byref(cnt)))
    return out


def qs_alu_rate(kind, stream=None):
    """Fused multiply-adds per second this GPU sustains (kind 0: FP32, 1:
    packed FP32x2, 2: FP64); see include/qs.h."""
    r = ctypes.c_double()
    N.check(N.lib().qs_alu_rate(kind, _stream(stream), ctypes.byref(r)))
    return r.value


def qs_batch_set_options(b, tile_log2=0, autotune=0, mode=QS_MODE_FUSED):
    """Tile size (fixed, or autotuned per instance size) of later runs; see
    include/qs.h."""
    o = _opts(mode, QS_PREC_DEFAULT, 0, tile_log2, autotune)
    N.check(N.lib().qs_batch_set_options(b, ctypes.byref(o)))


def qs_batch_set_engine(b, engine):
    """QS_BATCH_PERSISTENT (one persistent launch per run, the default) or
    QS_BATCH_ROUNDS (lockstep rounds) for later runs; see include/qs.h."""
    N.check(N.lib().qs_batch_set_engine(b, int(engine)))


def qs_batch_plan_info(b):
    """(tile sizes per instance, algorithmic bytes of one run) of the last
    prepared run."""
    t = np.zeros(_batch_sizes[b], dtype=np.int32)
    by = ctypes.c_double()
    N.check(N.lib().qs_batch_plan_info(b, t.ctypes.data, ctypes.byref(by)))
    return t, by.value


def qs_build_flags():
    """QS_BUILD_CHECKED (1) for the checked build, else 0."""
    return int(N.lib().qs_build_flags())


def qs_check_probe():
    """Checked build: a guarded out-of-range access that the device check
    catches; raises QSError (QS_ERR_INVALID_ARG).  Normal build: raises
    QSError (QS_ERR_UNSUPPORTED)."""
    N.check(N.lib().qs_check_probe())
