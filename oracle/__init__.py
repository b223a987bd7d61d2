"""FP64 CPU oracle for the random-circuit state-vector method of arXiv:1608.00263.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by bench.py's cpu_baseline / reference arm.  The product library never
imports, links or calls anything here, and nothing here imports the product.

All arithmetic lives in ``qs_oracle.c`` (plain loops, double precision,
sequential sums in index order).  This module only marshals numpy arrays.

Parity status: gate application, statistics, sampler and cross entropy are
pinned by tests (dense Kronecker unitaries, Feynman path sums, closed forms,
brute force, published SplitMix64 outputs).  The exact CZ layouts of the
generator are a reading of a figure the paper does not include: layout
parity unpinned (soft-pinned by Table I gates per level).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

GATE_DTYPE = np.dtype([("kind", np.uint8), ("q0", np.uint8), ("q1", np.uint8),
                       ("pad", np.uint8), ("cycle", np.uint32),
                       ("theta", np.float64)])
assert GATE_DTYPE.itemsize == 16

H, X_HALF, Y_HALF, T, CZ, RX, RY, RZ, CPHASE = range(9)
TWO_QUBIT_KINDS = (CZ, CPHASE)
DIAGONAL_KINDS = (T, CZ, RZ, CPHASE)
EULER_GAMMA = 0.57721566490153286061

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.oracle_splitmix64_output.restype = ctypes.c_uint64
        lib.oracle_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_circuit_generate.restype = ctypes.c_int
        lib.oracle_circuit_generate.argtypes = [
            ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint64, P,
            ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        lib.oracle_circuit_generate_dense.restype = ctypes.c_int
        lib.oracle_circuit_generate_dense.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P, ctypes.c_size_t,
            ctypes.POINTER(ctypes.c_size_t)]
        lib.oracle_noisy_circuit.restype = ctypes.c_int
        lib.oracle_noisy_circuit.argtypes = [
            P, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_uint64, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        lib.oracle_gate_matrix.restype = ctypes.c_int
        lib.oracle_gate_matrix.argtypes = [ctypes.c_int, ctypes.c_double, P]
        lib.oracle_apply_1q.restype = ctypes.c_int
        lib.oracle_apply_1q.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_apply_controlled.restype = ctypes.c_int
        lib.oracle_apply_controlled.argtypes = [P, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, P]
        lib.oracle_state_zero.restype = None
        lib.oracle_state_zero.argtypes = [P, ctypes.c_int]
        lib.oracle_apply_circuit.restype = ctypes.c_int
        lib.oracle_apply_circuit.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t]
        lib.oracle_probabilities.restype = None
        lib.oracle_probabilities.argtypes = [P, ctypes.c_int, P]
        for name in ("oracle_norm", "oracle_entropy", "oracle_uniform_ce"):
            getattr(lib, name).restype = ctypes.c_double
            getattr(lib, name).argtypes = [P, ctypes.c_int]
        lib.oracle_moments.restype = None
        lib.oracle_moments.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_sample_uniform.restype = ctypes.c_double
        lib.oracle_sample_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_sample.restype = ctypes.c_int
        lib.oracle_sample.argtypes = [P, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint64, P]
        lib.oracle_cross_entropy.restype = ctypes.c_double
        lib.oracle_cross_entropy.argtypes = [P, ctypes.c_int, P, ctypes.c_uint64,
                                             ctypes.POINTER(ctypes.c_double)]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nq(psi):
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    return n


def splitmix64_output(seed, j):
    return int(_load().oracle_splitmix64_output(seed & (2**64 - 1), j))


def sample_uniform(seed, j):
    return float(_load().oracle_sample_uniform(seed & (2**64 - 1), j))


def grid_dead_mask(rows, cols, dead_sites=()):
    mask = np.zeros(rows * cols, dtype=np.uint8)
    for r, c in dead_sites:
        mask[r * cols + c] = 1
    return mask


def generate_circuit(rows, cols, depth, seed, dead=None):
    """Gate list of a random circuit (structured array of GATE_DTYPE)."""
    lib = _load()
    dead_arr = None if dead is None else np.ascontiguousarray(dead, dtype=np.uint8)
    dp = None if dead_arr is None else _ptr(dead_arr)
    cnt = ctypes.c_size_t(0)
    rc = lib.oracle_circuit_generate(rows, cols, dp, depth, seed, None, 0,
                                     ctypes.byref(cnt))
    if rc:
        raise ValueError("oracle_circuit_generate failed: %d" % rc)
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    rc = lib.oracle_circuit_generate(rows, cols, dp, depth, seed, _ptr(out),
                                     out.size, ctypes.byref(cnt))
    if rc:
        raise ValueError("oracle_circuit_generate failed: %d" % rc)
    return out


def generate_dense_circuit(rows, cols, layers, seed):
    """Gate list of a dense periodic-boundary circuit (appendix on denser 2D circuits)."""
    lib = _load()
    cnt = ctypes.c_size_t(0)
    if lib.oracle_circuit_generate_dense(rows, cols, layers, seed, None, 0, ctypes.byref(cnt)):
        raise ValueError("oracle_circuit_generate_dense: bad arguments")
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    if lib.oracle_circuit_generate_dense(rows, cols, layers, seed, _ptr(out), out.size,
                                         ctypes.byref(cnt)):
        raise ValueError("oracle_circuit_generate_dense failed")
    return out


def noisy_circuit(gates, n, r1, r2, r_init, seed):
    """One trajectory of the depolarising error model (see qs_oracle.c)."""
    lib = _load()
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    gp = _ptr(g) if g.size else None
    cnt = ctypes.c_size_t(0)
    if lib.oracle_noisy_circuit(gp, g.size, n, r1, r2, r_init, seed, None, 0, ctypes.byref(cnt)):
        raise ValueError("oracle_noisy_circuit: bad arguments")
    out = np.zeros(cnt.value, dtype=GATE_DTYPE)
    if lib.oracle_noisy_circuit(gp, g.size, n, r1, r2, r_init, seed, _ptr(out), out.size,
                                ctypes.byref(cnt)):
        raise ValueError("oracle_noisy_circuit failed")
    return out


FLIP_SEED_XOR = 0xD1B54A32D192ED03


def sample_at(p, seed, counters):
    """Inverse-CDF samples of p for the given draw counters: x = min{i : C_i >
    u C_{N-1}}, C the sequential FP64 cumulative sum, u = sample_uniform(seed, j)."""
    c = np.cumsum(np.asarray(p, dtype=np.float64))
    u = np.array([sample_uniform(seed, int(j)) for j in counters])
    x = np.searchsorted(c, u * c[-1], side="right")
    return np.minimum(x, len(c) - 1).astype(np.uint64)


def measurement_flips(x, n, seed, r_mes, counter):
    """Bit b of sample number `counter` flips when draw counter*64 + b of the
    stream seeded with seed ^ FLIP_SEED_XOR is below r_mes."""
    s2 = (seed ^ FLIP_SEED_XOR) & (2**64 - 1)
    x = int(x)
    for b in range(n):
        if sample_uniform(s2, counter * 64 + b) < r_mes:
            x ^= 1 << b
    return x


def eq6_fidelity(r1, r2, r_init, r_mes, g1, g2, n):
    """Eq. 6: alpha ~ exp(-r1 g1 - r2 g2 - r_init n - r_mes n)."""
    return math.exp(-r1 * g1 - r2 * g2 - r_init * n - r_mes * n)


def single_error_circuit(gates, cycle, qubit, pauli):
    """Appendix "Residual correlations after discrete errors": the circuit
    with one Pauli (1 X, 2 Y, 3 Z; written R_P(pi)) on `qubit` placed after
    every gate of cycles <= `cycle` and before the rest."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    at = int(np.sum(g["cycle"] <= cycle))
    e = np.zeros(1, dtype=GATE_DTYPE)
    e[0]["kind"] = {1: 5, 2: 6, 3: 7}[pauli]      # R_X, R_Y, R_Z
    e[0]["q0"] = qubit
    e[0]["cycle"] = cycle
    e[0]["theta"] = math.pi
    return np.concatenate([g[:at], e, g[at:]])


def pearson(p, q):
    """Correlation coefficient of two distributions over the basis states."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    dp, dq = p - p.mean(), q - q.mean()
    return float(np.sum(dp * dq) / math.sqrt(np.sum(dp * dp) * np.sum(dq * dq)))


def pt_convergence_index(entropies, n):
    """Sec. "Convergence to Porter-Thomas" (Fig. pt_depth): the first index i
    such that every entropy from i on is within 4 sigma of ln N - 1 + gamma,
    sigma = 0.75 * 2^(-n/2); len(entropies) if the last one is outside."""
    target = n * math.log(2.0) - 1.0 + EULER_GAMMA
    sigma = 0.75 * 2.0 ** (-n / 2.0)
    first = len(entropies)
    for i in range(len(entropies) - 1, -1, -1):
        if abs(entropies[i] - target) > 4.0 * sigma:
            break
        first = i
    return first


def cycle_statistics(n, gates, kmax=10):
    """Statistics after every cycle (runs of equal `cycle`): rows of
    (cycle, norm, entropy, uniform CE, moments 1..kmax), each from the
    plain definitions on the exact state after that cycle."""
    psi = zero_state(n)
    rows = []
    cyc = gates["cycle"]
    starts = [i for i in range(len(gates)) if i == 0 or cyc[i] != cyc[i - 1]]
    for ci, b in enumerate(starts):
        e = starts[ci + 1] if ci + 1 < len(starts) else len(gates)
        apply_circuit(psi, gates[b:e])
        p = probabilities(psi)
        rows.append([float(cyc[b]), norm(p), entropy(p), uniform_ce(p)] + list(moments(p, kmax)))
    return np.array(rows)


def gate_matrix(kind, theta=0.0):
    u = np.zeros(4, dtype=np.complex128)
    if _load().oracle_gate_matrix(kind, theta, _ptr(u)):
        raise ValueError("unknown gate kind %r" % kind)
    return u.reshape(2, 2)


def zero_state(n):
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().oracle_state_zero(_ptr(psi), n)
    return psi


def apply_1q(psi, k, u):
    u = np.ascontiguousarray(u, dtype=np.complex128).reshape(4)
    if _load().oracle_apply_1q(_ptr(psi), _nq(psi), k, _ptr(u)):
        raise ValueError("bad qubit")
    return psi


def apply_controlled(psi, c, t, u):
    u = np.ascontiguousarray(u, dtype=np.complex128).reshape(4)
    if _load().oracle_apply_controlled(_ptr(psi), _nq(psi), c, t, _ptr(u)):
        raise ValueError("bad qubits")
    return psi


def apply_circuit(psi, gates):
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    if _load().oracle_apply_circuit(_ptr(psi), _nq(psi), _ptr(gates), gates.size):
        raise ValueError("malformed gate list")
    return psi


def simulate(n, gates):
    """|psi> = U |0...0> for the gate list."""
    return apply_circuit(zero_state(n), gates)


def probabilities(psi):
    p = np.empty(psi.size, dtype=np.float64)
    _load().oracle_probabilities(_ptr(psi), _nq(psi), _ptr(p))
    return p


def norm(p):
    return float(_load().oracle_norm(_ptr(p), _nq(p)))


def entropy(p):
    return float(_load().oracle_entropy(_ptr(p), _nq(p)))


def uniform_ce(p):
    return float(_load().oracle_uniform_ce(_ptr(p), _nq(p)))


def moments(p, kmax=10):
    out = np.empty(kmax, dtype=np.float64)
    _load().oracle_moments(_ptr(p), _nq(p), kmax, _ptr(out))
    return out


def sample(p, m, seed):
    out = np.empty(m, dtype=np.uint64)
    rc = _load().oracle_sample(_ptr(p), _nq(p), m, seed & (2**64 - 1), _ptr(out))
    if rc:
        raise ValueError("oracle_sample failed: %d" % rc)
    return out


def cross_entropy(p, samples):
    """Returns (CE, Delta H) of Eq. ae for the given sample indices."""
    x = np.ascontiguousarray(samples, dtype=np.uint64)
    dh = ctypes.c_double(0)
    ce = _load().oracle_cross_entropy(_ptr(p), _nq(p), _ptr(x), x.size,
                                      ctypes.byref(dh))
    return float(ce), float(dh.value)
