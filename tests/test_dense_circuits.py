"""Denser periodic-boundary circuits (appendix "Depth to reach Porter-Thomas
for denser 2D circuits") and the 4-sigma convergence criterion (Sec.
"Convergence to Porter-Thomas", Fig. pt_depth): generator rules and
library/oracle agreement on the CPU, oracle pins on small exact states."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()


TORI = [(2, 2), (2, 4), (4, 4), (4, 6), (6, 4), (6, 6), (8, 8)]


@pytest.mark.parametrize("rows,cols", TORI)
def test_dense_generator_matches_oracle_bit_exact(rows, cols):
    for seed in (0, 7, 2**63 + 11):
        for layers in (0, 1, 2, 5, 24):
            a = qs.qs_circuit_generate_dense(rows, cols, layers, seed)
            b = O.generate_dense_circuit(rows, cols, layers, seed)
            assert a.tobytes() == b.tobytes()


def torus_neighbours(rows, cols, a, b):
    ra, ca, rb, cb = a // cols, a % cols, b // cols, b % cols
    dr, dc = (ra - rb) % rows, (ca - cb) % cols
    return (dr == 0 and dc in (1, cols - 1)) or (dc == 0 and dr in (1, rows - 1))


@pytest.mark.parametrize("rows,cols", [(4, 4), (4, 6), (6, 6)])
def test_dense_rules(rows, cols):
    n = rows * cols
    layers = 17
    g = O.generate_dense_circuit(rows, cols, layers, 3)
    assert np.all(g["kind"][:n] == qs.QS_H) and np.all(g["cycle"][:n] == 0)
    pairs_by_layer = {}
    prev = [None] * n
    for lay in range(1, layers + 1):
        one = g[g["cycle"] == 2 * lay - 1]
        cz = g[g["cycle"] == 2 * lay]
        # every qubit in exactly one CZ, nearest neighbours on the torus
        assert np.all(cz["kind"] == qs.QS_CZ)
        touched = np.concatenate([cz["q0"], cz["q1"]])
        assert sorted(touched.tolist()) == list(range(n))
        for x in cz:
            assert torus_neighbours(rows, cols, int(x["q0"]), int(x["q1"]))
        pairs_by_layer[lay] = sorted((int(x["q0"]), int(x["q1"])) for x in cz)
        # single-qubit gates: none in layer 1 (previous cycle is the H
        # cycle), then on every qubit; T first, never the previous gate again
        if lay == 1:
            assert one.size == 0
            continue
        assert sorted(one["q0"].tolist()) == list(range(n))
        for x in one:
            q, k = int(x["q0"]), int(x["kind"])
            assert k in (qs.QS_X_HALF, qs.QS_Y_HALF, qs.QS_T)
            if prev[q] is None:
                assert k == qs.QS_T
            else:
                assert k != prev[q]
            prev[q] = k
    # four distinct matchings, period 4 in layers
    assert len({tuple(pairs_by_layer[l]) for l in range(1, 5)}) == 4
    for l in range(5, layers + 1):
        assert pairs_by_layer[l] == pairs_by_layer[l - 4]


def test_dense_rejects_bad_tori():
    for rows, cols in ((3, 4), (4, 5), (1, 4), (2, 1), (10, 10)):
        with pytest.raises(qs.QSError):
            qs.qs_circuit_generate_dense(rows, cols, 3, 0)
        with pytest.raises(ValueError):
            O.generate_dense_circuit(rows, cols, 3, 0)
    with pytest.raises(qs.QSError):
        qs.qs_circuit_generate_dense(4, 4, -1, 0)


def test_convergence_index_matches_oracle_definition():
    n = 12
    h_pt = n * math.log(2) - 1 + O.EULER_GAMMA
    tol = 4 * 0.75 * 2 ** (-n / 2)
    rng = np.random.default_rng(5)
    cases = [[], [h_pt], [h_pt + 2 * tol], [h_pt + 2 * tol, h_pt, h_pt + 0.5 * tol],
             [h_pt, h_pt + 1.5 * tol, h_pt - 0.2 * tol]]
    for _ in range(50):
        cases.append(list(h_pt + tol * rng.uniform(-3, 3, size=rng.integers(1, 30))))
    for e in cases:
        assert qs.qs_pt_convergence(e, n) == O.pt_convergence_index(e, n)
    assert qs.qs_pt_convergence([h_pt] * 5, n) == 0
    assert qs.qs_pt_convergence([h_pt] * 4 + [h_pt + 2 * tol], n) == 5


def test_dense_early_layers_exactly_uniform():
    """Layers 1 and 2 hold only CZ and T after the H cycle (diagonal gates):
    the output distribution stays exactly uniform."""
    rows, cols = 4, 4
    n = rows * cols
    g = O.generate_dense_circuit(rows, cols, 2, 1)
    stats = O.cycle_statistics(n, g, kmax=3)
    for row in stats:
        assert abs(row[2] - n * math.log(2)) < 1e-9          # entropy ln N
        assert abs(row[4 + 1] - 1.0) < 1e-9                   # N sum p^2 = 1


def test_dense_deep_layers_reach_porter_thomas():
    """Deep dense circuits: the entropy of each instance sits within 4 sigma
    of ln N - 1 + gamma (sigma = 0.75 2^(-n/2)) from some layer on, and the
    second normalised moment is near 2 (Porter-Thomas)."""
    rows, cols = 4, 4
    n = rows * cols
    firsts = []
    for seed in range(3):
        g = O.generate_dense_circuit(rows, cols, 24, seed)
        stats = O.cycle_statistics(n, g, kmax=2)
        ent = stats[stats[:, 0] % 2 == 0][:, 2]          # after each layer's CZ cycle
        first = O.pt_convergence_index(list(ent), n)
        assert first < len(ent) - 4, (seed, first)
        firsts.append(first)
        assert abs(stats[-1, 5] - 2.0) < 8 * math.sqrt(20 / 2**n) + 0.05
    # the circuits need a few non-diagonal layers before converging
    assert min(firsts) >= 3
