"""Host-side accounting of bench.py (no GPU): the leading Hadamard layer is
recognised as the library recognises it, the launches and algorithmic bytes of
an apply follow the library's handling of that layer (generated by the first
fused pass, a uniform fill before plain kernels or alone), the roofline's
traffic record is tied to the kernel source, and the kernel-launch count of a
step adds up."""
import hashlib
import json
import os

import numpy as np

import bench
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def setup_module(_):
    qs_build.build()


def test_leading_layer_recognition():
    n = 12
    g = qs.qs_circuit_generate(3, 4, 10, 3)
    assert bench.leading_h_layer(qs, g, n) == n
    perm = g.copy()
    perm[:n] = g[:n][::-1]
    assert bench.leading_h_layer(qs, perm, n) == n          # any qubit order
    dup = g.copy()
    dup["q0"][1] = dup["q0"][0]
    assert bench.leading_h_layer(qs, dup, n) == 0           # a repeated qubit
    assert bench.leading_h_layer(qs, g[1:], n) == 0         # a missing qubit
    assert bench.leading_h_layer(qs, g[:n - 1], n) == 0


def test_applied_plan_counts_the_leading_layer():
    n = 20
    g = qs.qs_circuit_generate(4, 5, 25, 0)
    N = 1 << n
    # plain: a uniform fill (8 N written), then one kernel per gate
    rest = qs.qs_plan_circuit(n, qs.QS_C64, g[n:], mode=qs.QS_MODE_PLAIN)
    ap = bench.applied_plan(qs, n, g, qs.QS_MODE_PLAIN)
    assert ap["passes"] == rest["passes"] and ap["launches"] == rest["passes"] + 1
    assert ap["bytes"] == rest["bytes"] + 8.0 * N
    # fused: no fill launch; 16 N per pass, 8 N for the first (it only
    # writes); the diagonal prefix after the layer is folded into that pass
    nf, folded = bench.fold_diagonal_prefix(qs, g[n:])
    assert nf > 0 and len(folded) == len(g) - n - nf
    rest = qs.qs_plan_circuit(n, qs.QS_C64, folded, mode=qs.QS_MODE_FUSED)
    ap = bench.applied_plan(qs, n, g, qs.QS_MODE_FUSED)
    assert ap["passes"] == rest["passes"] and ap["launches"] == rest["passes"]
    assert ap["bytes"] == 16.0 * N * ap["passes"] - 8.0 * N
    # the layer alone: one fill
    ap = bench.applied_plan(qs, n, g[:n], qs.QS_MODE_FUSED)
    assert ap["launches"] == 1 and ap["passes"] == 0 and ap["bytes"] == 8.0 * N


def test_traffic_record_matches_kernel_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    src = open(os.path.join(ROOT, "paper_1608_00263_gb300", "csrc", "qs_fused.cu"), "rb").read()
    digest = hashlib.sha1(src).hexdigest()
    for mode in ("fused", "tc"):
        t = bench.load_traffic(mode, 30)
        if rec.get(mode, {}).get("source_sha1") != digest:
            assert t is None, mode                  # a stale capture is never reported
            continue
        # the captured launch (a pass after the first) scaled to 30 qubits:
        # within 5 % of its algorithmic 16 bytes per amplitude
        assert abs(t[0] / (16.0 * 2**30) - 1) < 0.05
        assert "16 bytes per amplitude" in t[1]


def test_kernel_launches_per_step():
    # passes + read-out + statistics (2) + sampler (5) + cross entropy (4)
    assert bench.kernel_launches_per_step(10) == 10 + 1 + 2 + 5 + 4
