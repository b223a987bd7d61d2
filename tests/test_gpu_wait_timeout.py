"""Bounded waits: the tensor-core pass's mbarrier wait, run on an mbarrier
that nothing arrives at, and the persistent ensemble kernel's dependency
wait, run on a completion counter that nothing increments, give up after
their time limits and say so, without a fault; the context stays usable
afterwards (a circuit still matches the oracle).  The failures are made by
leaving the barrier without an arrival and the counter below its target: no
GPU fault, trap or endless loop is involved."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe():
    qs_build.build()
    d = tempfile.mkdtemp(prefix="qs_wait_")
    so = os.path.join(d, "libwait.so")
    subprocess.run([qs_build._nvcc(), "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                    "-gencode", qs_build.GENCODE, "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "wait_probe.cu"), "-o", so, "-lcudart"], check=True)
    lib = ctypes.CDLL(so)
    lib.wait_probe.restype = ctypes.c_int
    lib.wait_probe.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_ulonglong)]
    lib.flag_probe.restype = ctypes.c_int
    lib.flag_probe.argtypes = [ctypes.c_ulonglong, ctypes.c_uint, ctypes.c_uint, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_ulonglong)]
    return lib


def run(lib, limit_ns, arrive):
    ok, el = ctypes.c_int(-1), ctypes.c_ulonglong(0)
    assert lib.wait_probe(limit_ns, arrive, ctypes.byref(ok), ctypes.byref(el)) == 0
    return ok.value, el.value


def test_wait_gives_up_after_its_limit_and_context_survives(probe):
    ok, el = run(probe, 20_000_000, 0)            # nothing arrives: 20 ms limit
    assert ok == 0
    assert 20_000_000 <= el < 2_000_000_000
    ok, el = run(probe, 20_000_000, 1)            # the phase has completed
    assert ok == 1 and el < 20_000_000
    # the context is still usable: a circuit through the library matches the oracle
    n = 12
    g = qs.qs_circuit_generate(3, 4, 12, 5)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED)
        psi = qs.qs_state_copy_out(h, n)
    finally:
        qs.qs_state_destroy(h)
    ref = O.simulate(n, g)
    assert np.linalg.norm(psi.astype(complex) - ref) / np.linalg.norm(ref) < 1e-5


def test_counter_wait_gives_up_after_its_limit_reports_abort_and_context_survives(probe):
    def flag(limit_ns, value, abort):
        r, el = ctypes.c_int(-1), ctypes.c_ulonglong(0)
        assert probe.flag_probe(limit_ns, value, abort, ctypes.byref(r), ctypes.byref(el)) == 0
        return r.value, el.value
    r, el = flag(20_000_000, 0, 0)               # nothing increments the counter
    assert r == 1
    assert 20_000_000 <= el < 2_000_000_000
    r, el = flag(20_000_000, 1, 0)               # the counter is at its target
    assert r == 0 and el < 20_000_000
    r, el = flag(20_000_000, 0, 1)               # another CTA's wait ran out
    assert r == 2 and el < 20_000_000
    n = 12
    g = qs.qs_circuit_generate(3, 4, 12, 6)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED)
        psi = qs.qs_state_copy_out(h, n)
    finally:
        qs.qs_state_destroy(h)
    ref = O.simulate(n, g)
    assert np.linalg.norm(psi.astype(complex) - ref) / np.linalg.norm(ref) < 1e-5
