"""Digital error model (Sec. "Characterizing quantum supremacy", simulations
with errors; Eq. 6): noisy trajectories on the CPU -- library and oracle
agree bit for bit, the inserted errors follow the model's rates, and the
oracle's cross entropy difference of noisy samples tracks Eq. 6."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()


def test_zero_rates_keep_the_circuit():
    g = qs.qs_circuit_generate(3, 4, 12, 2)
    for seed in (0, 5):
        assert qs.qs_noisy_circuit(g, 12, 0.0, 0.0, 0.0, seed).tobytes() == g.tobytes()
        assert O.noisy_circuit(g, 12, 0.0, 0.0, 0.0, seed).tobytes() == g.tobytes()


@pytest.mark.parametrize("rates", [(0.001, 0.01, 0.01), (0.05, 0.2, 0.1), (1.0, 1.0, 1.0), (0.3, 0.0, 0.5)])
def test_library_matches_oracle_bit_exact(rates):
    r1, r2, ri = rates
    g = qs.qs_circuit_generate(4, 5, 20, 9)
    for seed in range(20):
        a = qs.qs_noisy_circuit(g, 20, r1, r2, ri, seed)
        b = O.noisy_circuit(g, 20, r1, r2, ri, seed)
        assert a.tobytes() == b.tobytes()


def test_rejects_bad_rates():
    g = qs.qs_circuit_generate(2, 2, 3, 0)
    for bad in ((-0.1, 0, 0), (0, 1.5, 0), (0, 0, float("nan"))):
        with pytest.raises(qs.QSError):
            qs.qs_noisy_circuit(g, 4, *bad, 0)


def test_error_statistics_follow_the_model():
    """Errors after one-qubit gates occur at rate r1 with X, Y, Z equally
    likely; after CZs at rate r2 with the 15 two-qubit Paulis equally likely;
    initialisation flips at rate r_init."""
    n = 12
    g = qs.qs_circuit_generate(3, 4, 10, 1)
    one = int(np.sum(g["kind"] != qs.QS_CZ))
    two = int(np.sum(g["kind"] == qs.QS_CZ))
    r1, r2, ri = 0.2, 0.3, 0.25
    T = 400
    n1 = n2 = ninit = 0
    kinds1 = np.zeros(3)
    pairs = np.zeros(16)
    for seed in range(T):
        h = O.noisy_circuit(g, n, r1, r2, ri, seed)
        # walk the trajectory: initial Paulis, then gate, then its errors
        i = 0
        while i < len(h) and h[i]["kind"] == qs.QS_RX and h[i]["theta"] == math.pi and i < n:
            ninit += 1
            i += 1
        for x in g:
            assert h[i].tobytes() == x.tobytes()
            i += 1
            errs = []
            while i < len(h) and h[i]["theta"] == math.pi and h[i]["kind"] in (qs.QS_RX, qs.QS_RY, qs.QS_RZ):
                errs.append(h[i])
                i += 1
            if x["kind"] == qs.QS_CZ:
                if errs:
                    n2 += 1
                    code = {int(e["q0"]): int(e["kind"]) - qs.QS_RX + 1 for e in errs}
                    a, b = code.get(int(x["q0"]), 0), code.get(int(x["q1"]), 0)
                    pairs[4 * a + b] += 1
            elif errs:
                assert len(errs) == 1 and errs[0]["q0"] == x["q0"]
                n1 += 1
                kinds1[int(errs[0]["kind"]) - qs.QS_RX] += 1
        assert i == len(h)
    def within(count, trials, p):
        return abs(count - trials * p) < 5 * math.sqrt(trials * p * (1 - p))
    assert within(n1, T * one, r1)
    assert within(n2, T * two, r2)
    assert within(ninit, T * n, ri)
    # uniform choices: chi-square with generous bounds
    e1 = n1 / 3
    assert np.sum((kinds1 - e1) ** 2 / e1) < 20
    assert pairs[0] == 0
    e2 = n2 / 15
    assert np.sum((pairs[1:] - e2) ** 2 / e2) < 45


def test_measurement_flip_rule():
    x = O.measurement_flips(0, 20, 3, 0.0, 7)
    assert x == 0
    x = O.measurement_flips(0, 20, 3, 1.0, 7)
    assert x == (1 << 20) - 1
    flips = [bin(O.measurement_flips(0, 16, 11, 0.25, j)).count("1") for j in range(400)]
    assert abs(np.mean(flips) - 4.0) < 5 * math.sqrt(16 * 0.25 * 0.75 / 400)


def cross_entropy_difference(p_ideal, samples, n):
    ce = -np.mean(np.log(p_ideal[np.asarray(samples, dtype=np.int64)]))
    return n * math.log(2) + O.EULER_GAMMA - ce


@pytest.mark.parametrize("r", [0.0, 0.01])
def test_eq6_tracks_cross_entropy_difference(r):
    """Eqs. 5, aap and 6 (Fig. sva): with r2 = r_init = r_mes = r, r1 = r/10,
    the cross entropy difference of one sample per noisy trajectory tracks
    exp(-r1 g1 - r2 g2 - r_init n - r_mes n).  10 qubits, depth 25."""
    rows, cols, depth = 2, 5, 25
    n = rows * cols
    g = O.generate_circuit(rows, cols, depth, 4)
    g1 = int(np.sum(g["kind"] != qs.QS_CZ))
    g2 = int(np.sum(g["kind"] == qs.QS_CZ))
    p_ideal = O.probabilities(O.simulate(n, g))
    r1, r2, ri, rm = r / 10, r, r, r
    T = 3000
    samples = []
    for t in range(T):
        h = O.noisy_circuit(g, n, r1, r2, ri, 1000 + t)
        p = O.probabilities(O.simulate(n, h))
        x = int(O.sample_at(p, 77, [t])[0])
        samples.append(O.measurement_flips(x, n, 77, rm, t))
    dh = cross_entropy_difference(p_ideal, samples, n)
    alpha = O.eq6_fidelity(r1, r2, ri, rm, g1, g2, n)
    sigma = 1.3 / math.sqrt(T)
    # the paper finds a good agreement up to small residual correlations
    assert abs(dh - alpha) < 0.06 + 3 * sigma, (dh, alpha)
