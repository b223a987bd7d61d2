"""CPU tests of the C ABI library: it loads, exports every symbol the headers
declare, validates arguments on the host, and its host-side parts (circuit
generator, planner) agree with the oracle -- no GPU needed."""
import ctypes
import math
import glob
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native
from paper_1608_00263_gb300 import build as qs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built_library():
    qs_build.build()
    return _native.lib()


def header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(qs_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the binding knows every one of them
    assert not [n for n in names if n not in _native.SIGNATURES]


def test_version_string():
    assert "sm_103a" in qs.qs_version()


def test_state_calls_reject_a_null_state_on_the_host():
    # argument checks run before any device call, so they hold without a GPU
    for call in (lambda: qs.qs_readout_share(None, 0.5), lambda: qs.qs_readout_share(None),
                 lambda: qs.qs_state_sync(None)):
        with pytest.raises(qs.QSError) as e:
            call()
        assert e.value.status == _native.QS_ERR_INVALID_ARG


GRIDS = [(4, 5, None), (5, 6, None), (2, 2, None), (1, 9, None), (3, 4, [(2, 3)]),
         (6, 6, [(0, 0), (5, 5)]), (4, 6, [(3, 4), (3, 5)])]


@pytest.mark.parametrize("rows,cols,dead_sites", GRIDS)
def test_generator_matches_oracle_bit_exact(rows, cols, dead_sites):
    dead = O.grid_dead_mask(rows, cols, dead_sites or ())
    for seed in (0, 1, 2**63 + 5, 12345678901):
        for depth in (0, 1, 9, 40):
            a = qs.qs_circuit_generate(rows, cols, depth, seed, dead)
            b = O.generate_circuit(rows, cols, depth, seed, dead)
            assert a.tobytes() == b.tobytes()


def test_generator_rejects_bad_arguments():
    with pytest.raises(qs.QSError):
        qs.qs_circuit_generate(0, 5, 3, 0)
    with pytest.raises(qs.QSError):
        qs.qs_circuit_generate(2, 2, -1, 0)
    with pytest.raises(qs.QSError):
        qs.qs_circuit_generate(2, 2, 3, 0, np.ones(4, dtype=np.uint8))   # no live site
    # too small an output buffer
    cnt = ctypes.c_size_t(3)
    out = np.zeros(3, dtype=qs.GATE_DTYPE)
    st = _native.lib().qs_circuit_generate(2, 2, None, 4, 0, out.ctypes.data, ctypes.byref(cnt))
    assert st == _native.QS_ERR_INVALID_ARG
    assert cnt.value > 3


def _gate(kind, q0, q1=0, theta=0.0):
    g = np.zeros(1, dtype=qs.GATE_DTYPE)
    g[0] = (kind, q0, q1, 0, 0, theta)
    return g


@pytest.mark.parametrize("bad", [
    _gate(9, 0), _gate(qs.QS_H, 12), _gate(qs.QS_CZ, 3, 3), _gate(qs.QS_CZ, 1, 12),
    _gate(qs.QS_RX, 1, 0, float("nan"))])
def test_planner_validates_gates(bad):
    with pytest.raises(qs.QSError) as e:
        qs.qs_plan_circuit(12, qs.QS_C64, bad)
    assert e.value.status == _native.QS_ERR_INVALID_ARG


def test_planner_rejects_bad_sizes():
    g = qs.qs_circuit_generate(3, 4, 5, 0)
    for n in (0, 35):
        with pytest.raises(qs.QSError):
            qs.qs_plan_circuit(n, qs.QS_C64, g)
    with pytest.raises(qs.QSError):
        qs.qs_plan_circuit(12, 7, g)


def test_planner_stats():
    g = qs.qs_circuit_generate(5, 6, 40, 0)
    st = qs.qs_plan_circuit(30, qs.QS_C64, g)
    assert st["gates"] == len(g)
    assert 5 <= st["passes"] <= 25
    assert st["phases"] >= st["passes"]
    assert st["ops"] == len(g)
    assert st["bytes"] == st["passes"] * 2 * 8 * 2**30
    plain = qs.qs_plan_circuit(30, qs.QS_C64, g, mode=qs.QS_MODE_PLAIN)
    assert plain["passes"] == len(g)
    # appendix specialisation: T moves half the bytes, CZ a quarter
    kinds = g["kind"]
    N8 = 8 * 2**30
    expect = (np.sum(kinds == qs.QS_T) * N8 + np.sum(kinds == qs.QS_CZ) * N8 / 2
              + np.sum((kinds != qs.QS_T) & (kinds != qs.QS_CZ)) * 2 * N8)
    assert plain["bytes"] == expect


@pytest.fixture(scope="module")
def emulator():
    src = os.path.join(ROOT, "tests", "plan_emulator.cpp")
    host = os.path.join(ROOT, "paper_1608_00263_gb300", "csrc", "qs_host.cpp")
    d = tempfile.mkdtemp(prefix="qs_emul_")
    so = os.path.join(d, "libemul.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                    src, host, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.emul_f16.restype = ctypes.c_uint16
    lib.emul_f16.argtypes = [ctypes.c_double]
    lib.emulate_plan_mode.restype = ctypes.c_int
    lib.emulate_plan_mode.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.emul_bf16.restype = ctypes.c_uint16
    lib.emul_bf16.argtypes = [ctypes.c_double]
    lib.emul_tf32.restype = ctypes.c_uint32
    lib.emul_tf32.argtypes = [ctypes.c_double]
    lib.emulate_plan_prec.restype = ctypes.c_int
    lib.emulate_plan_prec.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.check_plan_order.restype = ctypes.c_int
    lib.check_plan_order.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]
    lib.check_plan_against.restype = ctypes.c_int
    lib.check_plan_against.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]
    lib.emulate_plan_look.restype = ctypes.c_int
    lib.emulate_plan_look.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    lib.emulate_work.restype = ctypes.c_int
    lib.emulate_work.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_int)]
    lib.emul_fold.restype = ctypes.c_int
    lib.emul_fold.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                              ctypes.c_void_p, ctypes.c_void_p]
    lib.emulate_plan.restype = ctypes.c_int
    lib.emulate_plan.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_int)]
    return lib


def _emulate(lib, n, gates, t, r, c):
    psi = O.zero_state(n)
    passes = ctypes.c_int(0)
    g = np.ascontiguousarray(gates, dtype=qs.GATE_DTYPE)
    assert lib.emulate_plan(n, g.ctypes.data, g.size, t, r, c, psi.ctypes.data,
                            ctypes.byref(passes)) == 0
    return psi, passes.value


def random_gates(rng, n, count):
    g = np.zeros(count, dtype=qs.GATE_DTYPE)
    for i in range(count):
        k = int(rng.integers(0, 9))
        g[i]["kind"] = k
        if k in (qs.QS_CZ, qs.QS_CPHASE):
            a, b = rng.choice(n, size=2, replace=False)
            g[i]["q0"], g[i]["q1"] = a, b
        else:
            g[i]["q0"] = rng.integers(0, n)
        g[i]["theta"] = rng.uniform(-3, 3)
    return g


@pytest.mark.parametrize("n,t,r,c", [(10, 7, 5, 5), (12, 8, 3, 2), (11, 11, 5, 5),
                                     (13, 9, 4, 4), (9, 6, 5, 0), (14, 10, 5, 5), (12, 5, 5, 4)])
def test_plan_semantics_random_gates(emulator, n, t, r, c):
    rng = np.random.default_rng(n * 100 + t)
    g = random_gates(rng, n, 300)
    psi, passes = _emulate(emulator, n, g, t, r, c)
    ref = O.simulate(n, g)
    assert np.max(np.abs(psi - ref)) < 1e-12
    assert passes >= 1


@pytest.mark.parametrize("n,t,r,c,seed", [(10, 6, 4, 2, 0), (12, 7, 5, 3, 1), (9, 5, 3, 0, 2), (13, 8, 5, 5, 3)])
def test_plan_semantics_diagonal_heavy(emulator, n, t, r, c, seed):
    """Mostly diagonal gates: a pending diagonal gate holds back only later
    non-diagonal gates on its qubits, so diagonal gates overtake it inside
    passes and phases; the plan must still give the circuit's state."""
    rng = np.random.default_rng(seed)
    g = np.zeros(400, dtype=qs.GATE_DTYPE)
    diag = [qs.QS_T, qs.QS_CZ, qs.QS_RZ, qs.QS_CPHASE]
    dense = [qs.QS_H, qs.QS_X_HALF, qs.QS_Y_HALF, qs.QS_RX, qs.QS_RY]
    for i in range(g.size):
        k = int(rng.choice(diag)) if rng.random() < 0.75 else int(rng.choice(dense))
        g[i]["kind"] = k
        if k in (qs.QS_CZ, qs.QS_CPHASE):
            g[i]["q0"], g[i]["q1"] = rng.choice(n, size=2, replace=False)
        else:
            g[i]["q0"] = rng.integers(0, n)
        g[i]["theta"] = rng.uniform(-3, 3)
    psi, passes = _emulate(emulator, n, g, t, r, c)
    ref = O.simulate(n, g)
    assert np.max(np.abs(psi - ref)) < 1e-12


@pytest.mark.parametrize("rows,cols,depth,t", [(4, 5, 25, 13), (4, 4, 30, 9), (3, 5, 40, 10)])
def test_plan_semantics_random_circuits(emulator, rows, cols, depth, t):
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 3)
    psi, passes = _emulate(emulator, n, g, t, 5, 5)
    ref = O.simulate(n, g)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_fp16_split_conversion_matches_numpy(emulator):
    rng = np.random.default_rng(4)
    vals = np.concatenate([
        rng.normal(size=2000), rng.normal(size=2000) * 1e-5, rng.normal(size=500) * 1e-7,
        rng.uniform(-70000, 70000, 500), [0.0, -0.0, 65504.0, 65519.99, 65520.0, 6.1e-5, 5.96e-8,
                                           2.98e-8, 2.99e-8, 1 + 2**-11, 1 + 3 * 2**-11]])
    got = np.array([emulator.emul_f16(float(v)) for v in vals], dtype=np.uint16)
    # numpy rounds float64 -> float16 to nearest even (IEEE)
    ref = vals.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("rows,cols,depth,seed", [(3, 5, 25, 0), (2, 7, 30, 1), (4, 4, 40, 2)])
def test_tc_plan_semantics(emulator, rows, cols, depth, seed):
    """Tensor-core block phases: the block unitaries (realified, FP16 hi + lo)
    reproduce the circuit to the split's precision (~2^-22 per block)."""
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, seed)
    psi = O.zero_state(n)
    passes = ctypes.c_int(0)
    tcp = ctypes.c_int(0)
    gg = np.ascontiguousarray(g, dtype=qs.GATE_DTYPE)
    assert emulator.emulate_plan_mode(n, gg.ctypes.data, gg.size, 13, 5, 5, qs.QS_MODE_FUSED_TC,
                                      psi.ctypes.data, ctypes.byref(passes), ctypes.byref(tcp)) == 0
    ref = O.simulate(n, g)
    err = np.linalg.norm(psi - ref) / np.linalg.norm(ref)
    assert tcp.value > 0
    assert err < 1e-5, err


@pytest.mark.parametrize("rows,cols,corners,depth,seed", [
    (4, 7, False, 40, 0), (5, 6, False, 40, 0), (5, 6, False, 40, 1), (5, 6, False, 40, 2),
    (6, 6, True, 40, 0)])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_full_size_plans_keep_circuit_order(emulator, rows, cols, corners, depth, seed, dtype):
    """The plans the library builds for 28-, 30- and 34-qubit circuits (with
    the deeper tile lookahead those sizes use) apply every gate once, keep
    every pair of non-commuting gates in circuit order, and carry consistent
    tile / register maps and deferred-factor counts: a symbolic check that
    needs no state."""
    dead = O.grid_dead_mask(rows, cols, [(0, 0), (rows - 1, cols - 1)] if corners else [])
    n = rows * cols - int(dead.sum())
    g = np.ascontiguousarray(qs.qs_circuit_generate(rows, cols, depth, seed, dead), dtype=qs.GATE_DTYPE)
    passes = ctypes.c_int(0)
    rc = emulator.check_plan_order(n, dtype, qs.QS_MODE_FUSED, g.ctypes.data, g.size, ctypes.byref(passes))
    assert rc == 0, rc
    assert passes.value == qs.qs_plan_circuit(n, dtype, g)["passes"]


def test_plan_order_check_catches_a_swapped_pair(emulator):
    """The symbolic check itself: the plan of a circuit in which an X^1/2 or
    Y^1/2 gate was moved before the CZ on its qubit that precedes it is not
    a valid plan of the original circuit."""
    g = np.ascontiguousarray(qs.qs_circuit_generate(3, 4, 12, 0), dtype=qs.GATE_DTYPE)
    passes = ctypes.c_int(0)
    assert emulator.check_plan_order(12, qs.QS_C64, qs.QS_MODE_FUSED, g.ctypes.data, g.size,
                                     ctypes.byref(passes)) == 0
    i = next(k for k in range(1, g.size) if int(g[k]["kind"]) in (qs.QS_X_HALF, qs.QS_Y_HALF)
             and any(int(g[j]["kind"]) == qs.QS_CZ and g[k]["q0"] in (g[j]["q0"], g[j]["q1"])
                     for j in range(k)))
    j = max(j for j in range(i) if int(g[j]["kind"]) == qs.QS_CZ and g[i]["q0"] in (g[j]["q0"], g[j]["q1"]))
    sw = g.copy()
    sw[[i, j]] = sw[[j, i]]
    rc = emulator.check_plan_against(12, qs.QS_C64, qs.QS_MODE_FUSED, sw.ctypes.data, g.ctypes.data,
                                     g.size, ctypes.byref(passes))
    assert rc == -10, rc


@pytest.mark.parametrize("look", [(8, 8), (64, 64)])
@pytest.mark.parametrize("rows,cols,depth,t,seed", [(4, 5, 25, 13, 0), (4, 4, 40, 10, 1), (3, 6, 30, 11, 2)])
def test_plan_semantics_deep_lookahead(emulator, look, rows, cols, depth, t, seed):
    """The tile lookahead of large states (8 additions among 8 candidates at
    28-31 qubits, every addition and candidate from 32 on), run on states
    small enough to emulate numerically: the plan reproduces the oracle."""
    n = rows * cols
    g = np.ascontiguousarray(qs.qs_circuit_generate(rows, cols, depth, seed), dtype=qs.GATE_DTYPE)
    psi = O.zero_state(n)
    passes = ctypes.c_int(0)
    assert emulator.emulate_plan_look(n, g.ctypes.data, g.size, t, 5, 5, look[0], look[1],
                                      psi.ctypes.data, ctypes.byref(passes)) == 0
    ref = O.simulate(n, g)
    assert np.max(np.abs(psi - ref)) < 1e-12


def _round_frac_exact(x, frac):
    """Round-to-nearest-even of x to `frac` fraction bits, in exact rational
    arithmetic (an independent restatement of the rounding rule)."""
    from fractions import Fraction
    if x == 0:
        return 0.0
    m, e = math.frexp(abs(x))               # |x| = m 2^e, m in [0.5, 1)
    q = Fraction(2) ** (e - 1 - frac)       # spacing of representable values
    v = Fraction(abs(x)) / q
    f = math.floor(v)
    r = v - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return math.copysign(float(f * q), x)


def test_bf16_and_tf32_rounding(emulator):
    """Host splitting of the tensor-core block matrices: BF16 and TF32
    rounding (nearest, ties to even) against exact rational rounding, and
    BF16 against torch's float32 -> bfloat16 conversion."""
    import struct
    import torch
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.normal(size=3000), rng.normal(size=500) * 1e-6,
                           [1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -11, 1 + 3 * 2 ** -11, -0.75, 0.0]])
    for v in vals:
        b = emulator.emul_bf16(float(v))
        bf = struct.unpack("<f", struct.pack("<I", b << 16))[0]
        assert bf == _round_frac_exact(float(v), 7), v
        t = emulator.emul_tf32(float(v))
        assert t & 0x1FFF == 0
        tf = struct.unpack("<f", struct.pack("<I", t))[0]
        assert tf == _round_frac_exact(float(v), 10), v
    f32 = vals.astype(np.float32)
    ref = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([emulator.emul_bf16(float(v)) for v in f32], dtype=np.uint16)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec,bound", [(qs.QS_PREC_FP16X3, 1e-6), (qs.QS_PREC_BF16X3, 2e-4),
                                        (qs.QS_PREC_BF16X6, 1e-7), (qs.QS_PREC_TF32X3, 1e-6),
                                        (qs.QS_PREC_TF32, 5e-3)])
def test_tc_plan_semantics_every_precision(emulator, prec, bound):
    """Tensor-core block phases in every operand precision: the stored block
    terms (decoded and summed in FP64) reproduce the circuit within the
    precision's split error."""
    rows, cols, depth, seed = 4, 4, 40, 2
    n = rows * cols
    g = np.ascontiguousarray(qs.qs_circuit_generate(rows, cols, depth, seed), dtype=qs.GATE_DTYPE)
    psi = O.zero_state(n)
    passes, tcp = ctypes.c_int(0), ctypes.c_int(0)
    assert emulator.emulate_plan_prec(n, g.ctypes.data, g.size, 13, 5, 5, qs.QS_MODE_FUSED_TC, prec,
                                      psi.ctypes.data, ctypes.byref(passes), ctypes.byref(tcp)) == 0
    ref = O.simulate(n, g)
    err = np.linalg.norm(psi - ref) / np.linalg.norm(ref)
    assert tcp.value > 0
    assert err < bound, err


def _work_batch():
    """Mixed instances for the persistent-engine work list: 5..19 qubits
    (17: two 2^16-amplitude initial and statistics chunks; 19: also two
    2^18-amplitude items per pass), one list that is only the Hadamard
    layer, one without the leading layer (|0...0> start), one depth-3
    circuit among deep ones."""
    def circ(n, depth, seed):
        rows = 1 if n < 4 else (2 if n < 9 else 4)
        cols = -(-n // rows)
        dead = np.zeros(rows * cols, dtype=np.uint8)
        dead[n:] = 1
        return O.generate_circuit(rows, cols, depth, seed, dead)
    spec = [(19, 10, 1), (5, 8, 2), (12, 20, 3), (9, 16, 4), (17, 3, 5), (14, 25, 6), (6, 10, 7), (13, 14, 8)]
    ns, gl = [], []
    for n, depth, seed in spec:
        ns.append(n)
        gl.append(circ(n, depth, seed))
    ns.append(11)
    gl.append(circ(11, 9, 9)[:11])            # the Hadamard layer only
    ns.append(10)
    gl.append(circ(10, 12, 10)[1:])           # no leading layer: starts in |0...0>
    return ns, gl


def _emulate_work(lib, ns, gl, workers, seed, corrupt=0):
    g = np.ascontiguousarray(np.concatenate(gl), dtype=qs.GATE_DTYPE)
    offs = np.zeros(len(gl) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([x.size for x in gl])
    nq = np.array(ns, dtype=np.int32)
    psi = np.zeros(sum(1 << n for n in ns), dtype=np.complex128)
    sums = np.full((len(ns), 12), np.nan)
    cnt = ctypes.c_int(0)
    rc = lib.emulate_work(len(ns), nq.ctypes.data, g.ctypes.data, offs.ctypes.data, workers, seed, corrupt,
                          psi.ctypes.data, sums.ctypes.data, ctypes.byref(cnt))
    return rc, psi, sums, cnt.value


@pytest.mark.parametrize("workers,seed", [(1, 0), (3, 11), (16, 12), (304, 13)])
def test_persistent_work_list_matches_oracle_in_any_dependency_order(emulator, workers, seed):
    """The persistent ensemble engine's work list (the library's own
    build_work): every item in bounds, every state and pass covered exactly
    once, each item's need equal to its instance's items in earlier levels
    (all earlier in the list), and, run under a randomized schedule of
    concurrent workers that follows the device protocol (take in list
    order, wait for done >= need, run, count), states equal to the oracle's
    and statistics sums equal to the oracle's probabilities' sums."""
    ns, gl = _work_batch()
    rc, psi, sums, nitems = _emulate_work(emulator, ns, gl, workers, seed)
    assert rc == 0
    at = 0
    for i, (n, g) in enumerate(zip(ns, gl)):
        ref = O.simulate(n, g)
        if g.size >= n and np.all(g["kind"][:n] == qs.QS_H):
            # the uniform start 2^(-n/2) is written as the kernel writes it,
            # rounded to FP32: the whole state carries that factor
            v = 2.0 ** (-n / 2)
            ref = ref * (float(np.float32(v)) / v)
        got = psi[at:at + (1 << n)]
        at += 1 << n
        assert np.max(np.abs(got - ref)) < 1e-12, i
        N = float(1 << n)
        y = O.probabilities(ref) * N
        with np.errstate(divide="ignore", invalid="ignore"):
            ly = np.log(y)
            expect = [y.sum(), np.sum(np.where(y > 0, y * ly, 0.0)), ly.sum()] + \
                     [np.sum(y ** k) for k in range(2, 11)]
        for k in range(12):
            if k == 2 and y.min() < 1e-8:
                continue      # sum ln y over amplitudes at rounding level: ill-conditioned
            if np.isfinite(expect[k]):
                assert sums[i, k] == pytest.approx(expect[k], rel=1e-9, abs=1e-9), (i, k)
            else:
                assert sums[i, k] == expect[k], (i, k)
    assert nitems > 0


@pytest.mark.parametrize("corrupt", [1, 2])
def test_persistent_work_list_check_catches_a_wrong_need(emulator, corrupt):
    """A planted off-by-one in one item's need (lowered: the item could run
    before its pass's inputs are complete; raised: it waits for an item of
    its own level) fails the level check."""
    ns, gl = _work_batch()
    rc, _, _, _ = _emulate_work(emulator, ns, gl, 4, 0, corrupt)
    assert rc == -4


@pytest.mark.parametrize("dtype,t", [(qs.QS_C64, 5), (qs.QS_C64, 6), (qs.QS_C128, 4), (qs.QS_C128, 5)])
def test_smallest_tiles_plan(dtype, t):
    """A tile of as many qubits as the register set still leaves a free
    tile bit beside the always-resident low qubits, so the planner makes
    progress (the plan's semantics at t = 5, c = 4 are emulated above)."""
    g = O.generate_circuit(3, 4, 12, 4)
    st = qs.qs_plan_circuit(12, dtype, g, tile_log2=t)
    assert st["tile_log2"] == t and st["passes"] >= 2 and st["gates"] == g.size


def _lib_fold(emulator, g):
    g = np.ascontiguousarray(g)
    rest = np.zeros(max(len(g), 1), dtype=qs.GATE_DTYPE)
    nrest = ctypes.c_int()
    nb = np.zeros(34, dtype=np.uint64)
    m = np.zeros(3, dtype=np.uint64)
    nf = emulator.emul_fold(g.ctypes.data if len(g) else None, len(g), rest.ctypes.data, ctypes.byref(nrest),
                            nb.ctypes.data, m.ctypes.data)
    return nf, rest[:nrest.value], nb, m


def _random_list(rng, n, count):
    kinds = [qs.QS_H, qs.QS_X_HALF, qs.QS_Y_HALF, qs.QS_T, qs.QS_T, qs.QS_T, qs.QS_CZ, qs.QS_CZ, qs.QS_CZ,
             qs.QS_RX, qs.QS_RZ, qs.QS_CPHASE]
    g = np.zeros(count, dtype=qs.GATE_DTYPE)
    for i in range(count):
        k = kinds[int(rng.integers(len(kinds)))]
        g[i]["kind"] = k
        a, b = rng.choice(n, size=2, replace=False)
        g[i]["q0"] = a
        g[i]["q1"] = b if k in (qs.QS_CZ, qs.QS_CPHASE) else 0
        g[i]["theta"] = rng.uniform(-3, 3) if k in (qs.QS_RX, qs.QS_RZ, qs.QS_CPHASE) else 0.0
    return g


def test_library_fold_rule_matches_the_bench_accounting(emulator):
    """The library's diagonal-prefix fold (qs_host.cpp) keeps exactly the
    gates the bench's accounting mirror keeps, on random lists and on the
    bench's circuits."""
    import bench
    rng = np.random.default_rng(41)
    lists = [_random_list(rng, 6, c) for c in (0, 1, 5, 20, 60) for _ in range(8)]
    lists += [qs.qs_circuit_generate(5, 6, 40, s)[30:] for s in range(3)]
    for g in lists:
        nf, rest, _, _ = _lib_fold(emulator, g)
        nf_b, rest_b = bench.fold_diagonal_prefix(qs, g)
        assert nf == nf_b and rest.tobytes() == rest_b.tobytes()


@pytest.mark.parametrize("seed", range(6))
def test_library_fold_masks_give_the_oracle_state(emulator, seed):
    """The fold masks the library hands to the first pass (CZ partners as
    XOR-accumulated qubit masks, T counts mod 8 as three bit masks) give
    2^(-n/2) e^{i pi k(x)/4}, k = 4 (CZ pairs set in x) + (T counts set in
    x): the oracle's state after the Hadamard layer and the folded gates,
    with repeated T and repeated (cancelling) CZ pairs in the list."""
    rng = np.random.default_rng(500 + seed)
    n = 7
    g = _random_list(rng, n, 40)
    nf, rest, nb, m = _lib_fold(emulator, g)
    layer = np.zeros(n, dtype=qs.GATE_DTYPE)
    layer["kind"], layer["q0"] = qs.QS_H, np.arange(n)
    keep = np.zeros(len(g), dtype=bool)
    j = 0
    for i in range(len(g)):
        if j < len(rest) and g[i].tobytes() == rest[j].tobytes():
            keep[i] = True
            j += 1
    assert j == len(rest) and (~keep).sum() == nf
    psi = O.simulate(n, np.concatenate([layer, g[~keep]]))
    x = np.arange(1 << n, dtype=np.uint64)
    bit = lambda v, q: (v >> np.uint64(q)) & np.uint64(1)
    k = np.zeros(1 << n, dtype=np.int64)
    for i in range(n):
        for j2 in range(i + 1, n):
            if (int(nb[i]) >> j2) & 1:
                assert (int(nb[j2]) >> i) & 1                 # symmetric
                k += 4 * (bit(x, i) * bit(x, j2)).astype(np.int64)
        c = ((int(m[0]) >> i) & 1) + 2 * ((int(m[1]) >> i) & 1) + 4 * ((int(m[2]) >> i) & 1)
        k += c * bit(x, i).astype(np.int64)
    want = 2.0 ** (-n / 2) * np.exp(1j * np.pi * (k % 8) / 4)
    assert np.max(np.abs(psi - want)) < 1e-13
