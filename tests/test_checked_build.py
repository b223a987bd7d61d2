"""The checked build (libqs_checked.so, QS_CHECKED): device-side index checks
that turn an out-of-range global index into QS_ERR_INVALID_ARG instead of an
access.

CPU: both libraries export every declared symbol and report their build
flags; the binding selects the checked library under QS_CHECKED=1; the
normal build's check probe answers QS_ERR_UNSUPPORTED without touching a GPU.
GPU: the check probe's guarded one-past-the-end access is caught (site 901)
and the context stays usable; the parity suite's small cases pass in the
checked build with no check firing.
"""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_1608_00263_gb300 import _native
from paper_1608_00263_gb300 import build as qs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1608_00263_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    qs_build.build(checked=True)


def _load(path):
    lib = ctypes.CDLL(path)
    lib.qs_build_flags.restype = ctypes.c_int
    lib.qs_check_probe.restype = ctypes.c_int
    return lib


def test_both_builds_export_every_declared_symbol_and_report_their_flags():
    from test_host_abi import header_functions
    names = header_functions()
    for path, flags in ((qs_build.LIB, 0), (qs_build.LIB_CHECKED, 1)):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                             check=True).stdout
        exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
        assert not [n for n in names if n not in exported], path
        assert _load(path).qs_build_flags() == flags


def test_normal_build_probe_is_unsupported_without_device_work():
    assert _load(qs_build.LIB).qs_check_probe() == _native.QS_ERR_UNSUPPORTED


def test_binding_selects_the_checked_library_from_the_environment():
    code = ("import paper_1608_00263_gb300 as qs, paper_1608_00263_gb300._native as N;"
            "print(N.LIB_PATH); print(qs.qs_build_flags())")
    env = dict(os.environ, QS_CHECKED="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True).stdout.split()
    assert out[0].endswith("libqs_checked.so") and out[1] == "1"
    env["QS_CHECKED"] = "0"
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True).stdout.split()
    assert out[0].endswith("libqs.so") and out[1] == "0"


@pytest.mark.gpu
def test_checked_probe_catches_the_guarded_access_and_the_context_survives():
    code = """
import numpy as np, torch
import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native as N
assert torch.cuda.is_available() and qs.qs_build_flags() == 1
try:
    qs.qs_check_probe()
    raise SystemExit("probe did not report")
except qs.QSError as e:
    assert e.status == N.QS_ERR_INVALID_ARG and "901" in str(e), e
g = qs.qs_circuit_generate(3, 5, 20, 0)
h = qs.qs_state_create(15, qs.QS_C64)
qs.qs_apply_circuit(h, g)
psi = qs.qs_state_copy_out(h, 15)
ref = O.simulate(15, g)
assert np.linalg.norm(psi - ref) / np.linalg.norm(ref) < 1e-5
qs.qs_state_destroy(h)
print("CHECKED_OK")
"""
    env = dict(os.environ, QS_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert "CHECKED_OK" in r.stdout, r.stdout + r.stderr


@pytest.mark.gpu
def test_parity_small_cases_pass_in_the_checked_build():
    """The small parity cases (plain and fused forms, both dtypes, the
    tensor-core form, statistics, sampler, cross entropy) run against the
    oracle with every device check armed; none may fire."""
    env = dict(os.environ, QS_CHECKED="1", PYTHONPATH=ROOT)
    sel = ("random_gates or grid_4x5_depth25 or probabilities or pt_moments or sampler or "
           "cross_entropy or tc_form_vs_oracle or cycle_statistics")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                        "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider", "-k", sel],
                       env=env, capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0 and " passed" in r.stdout, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.gpu
def test_batch_engines_pass_in_the_checked_build():
    """The persistent ensemble engine (whole-CTA and grouped pass bodies for
    tiles of 5 to 13 qubits, dependency waits) and the lockstep engine with
    every device check armed: the same states and statistics as each other
    and the oracle, and no check fires."""
    env = dict(os.environ, QS_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_batch.py"),
                        "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider", "-k",
                        "persistent_and_lockstep or initial_states"],
                       env=env, capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0 and " passed" in r.stdout, r.stdout[-3000:] + r.stderr[-2000:]
