"""Single discrete errors (Fig. 1error; appendix "Residual correlations after
discrete errors"): the insertion rule agrees with the oracle, and the oracle's
correlations obey the cases the appendix explains (phase flips at the end and
bit flips right after the H layer change nothing) and the near-uniform
average over error locations."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()


def test_insertion_matches_oracle():
    g = qs.qs_circuit_generate(3, 4, 10, 2)
    for cycle in (0, 1, 5, 10, 11):
        for q in (0, 7, 11):
            for pauli in (1, 2, 3):
                a = qs.qs_single_error_circuit(g, 12, cycle, q, pauli)
                b = O.single_error_circuit(g, cycle, q, pauli)
                assert a.tobytes() == b.tobytes()
    with pytest.raises(qs.QSError):
        qs.qs_single_error_circuit(g, 12, 3, 12, 1)
    with pytest.raises(qs.QSError):
        qs.qs_single_error_circuit(g, 12, 3, 0, 4)


@pytest.fixture(scope="module")
def deep():
    rows, cols, depth = 3, 4, 24
    n = rows * cols
    g = O.generate_circuit(rows, cols, depth, 3)
    return n, depth, g, O.probabilities(O.simulate(n, g))


def test_phase_flip_at_the_end_changes_nothing(deep):
    n, depth, g, p = deep
    for q in range(n):
        pe = O.probabilities(O.simulate(n, O.single_error_circuit(g, depth, q, 3)))
        assert np.allclose(pe, p, atol=1e-14)
        assert O.pearson(p, pe) == pytest.approx(1.0, abs=1e-12)


def test_bit_flip_after_hadamards_changes_nothing(deep):
    n, depth, g, p = deep
    for q in range(n):
        pe = O.probabilities(O.simulate(n, O.single_error_circuit(g, 0, q, 1)))
        assert np.allclose(pe, p, atol=1e-14)


def test_bit_flip_at_the_end_permutes(deep):
    n, depth, g, p = deep
    idx = np.arange(1 << n)
    for q in (0, 5, 11):
        pe = O.probabilities(O.simulate(n, O.single_error_circuit(g, depth, q, 1)))
        assert np.allclose(pe, p[idx ^ (1 << q)], atol=1e-14)


def test_mid_circuit_errors_decorrelate_and_average_to_uniform(deep):
    """Errors in the bulk of a deep circuit leave little correlation, and the
    distribution averaged over error locations is close to uniform."""
    n, depth, g, p = deep
    N = 1 << n
    corr, acc, cnt = [], np.zeros(N), 0
    for cycle in range(4, depth - 6):
        for q in range(n):
            for pauli in (1, 3):
                pe = O.probabilities(O.simulate(n, O.single_error_circuit(g, cycle, q, pauli)))
                corr.append(O.pearson(p, pe))
                acc += pe
                cnt += 1
    corr = np.abs(np.array(corr))
    assert np.median(corr) < 0.1
    avg = acc / cnt
    # Porter-Thomas: N sum p^2 - 1 ~ 1; the error average is far flatter
    assert N * np.sum(p * p) - 1 > 0.6
    assert N * np.sum(avg * avg) - 1 < 0.1
    assert abs(O.pearson(p, avg)) < 0.1


def test_average_over_all_locations_keeps_residual_correlation(deep):
    """Fig. 1error: averaged over every location (all cycles, qubits, X and Z)
    the distribution is nearly flat but keeps a positive correlation with
    p_U, from the errors near the ends that change little."""
    n, depth, g, p = deep
    N = 1 << n
    acc, cnt = np.zeros(N), 0
    for cycle in range(depth + 1):
        for q in range(n):
            for pauli in (1, 3):
                acc += O.probabilities(O.simulate(n, O.single_error_circuit(g, cycle, q, pauli)))
                cnt += 1
    avg = acc / cnt
    c = O.pearson(p, avg)
    assert 0.05 < c < 0.9
    assert N * np.sum(avg * avg) - 1 < 0.5 * (N * np.sum(p * p) - 1)
