"""Random-circuit generator rules (Sec. "Convergence to Porter-Thomas", Fig.
two_dimers caption) checked on the oracle's generator.

The layout figure is not available, so the exact eight CZ layouts are a
reading; the constraints the text states are checked exactly, and the
gates-per-level counts of Table I serve as a soft pin of the reading.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _live_coords(rows, cols, dead):
    coords = []
    for r in range(rows):
        for c in range(cols):
            if dead is None or not dead[r * cols + c]:
                coords.append((r, c))
    return coords


CASES = [(4, 5, None), (5, 6, None), (3, 4, None), (2, 2, None), (1, 7, None),
         (6, 6, O.grid_dead_mask(6, 6, [(0, 0), (5, 5)])),
         (4, 6, O.grid_dead_mask(4, 6, [(3, 4), (3, 5)]))]


@pytest.mark.parametrize("rows,cols,dead", CASES)
@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_generator_rules(rows, cols, dead, seed):
    depth = 33
    g = O.generate_circuit(rows, cols, depth, seed, dead)
    coords = _live_coords(rows, cols, dead)
    n = len(coords)
    assert all(int(x["q0"]) < n for x in g)
    # cycle 0: H on every qubit, nothing else
    c0 = g[g["cycle"] == 0]
    assert sorted(int(x["q0"]) for x in c0) == list(range(n))
    assert all(int(x["kind"]) == O.H for x in c0)
    assert np.all(np.diff(g["cycle"].astype(int)) >= 0)
    in_cz = [set() for _ in range(depth + 1)]
    edges_seen = {}
    last = {}
    for t in range(1, depth + 1):
        cyc = g[g["cycle"] == t]
        czs = [(int(x["q0"]), int(x["q1"])) for x in cyc if int(x["kind"]) == O.CZ]
        ones = [(int(x["q0"]), int(x["kind"])) for x in cyc if int(x["kind"]) != O.CZ]
        # within a cycle: CZs first, then single-qubit gates by qubit
        kinds = [int(x["kind"]) for x in cyc]
        assert kinds == sorted(kinds, key=lambda k: 0 if k == O.CZ else 1)
        assert [q for q, _ in ones] == sorted(q for q, _ in ones)
        for a, b in czs:
            ra, ca = coords[a]
            rb, cb = coords[b]
            assert abs(ra - rb) + abs(ca - cb) == 1, "CZ on nearest neighbours"
            assert a < b
            in_cz[t].update((a, b))
            edges_seen.setdefault((a, b), []).append(t)
        # no two CZs of a cycle act on neighbouring qubits
        for (a, b) in czs:
            for (c, d) in czs:
                if (a, b) == (c, d):
                    continue
                for u in (a, b):
                    for v in (c, d):
                        ru, cu = coords[u]
                        rv, cv = coords[v]
                        assert abs(ru - rv) + abs(cu - cv) > 1
        for q, kind in ones:
            assert kind in (O.X_HALF, O.Y_HALF, O.T)
            assert q in in_cz[t - 1] and q not in in_cz[t]
            if q not in last:
                assert kind == O.T, "first single-qubit gate after H is T"
            else:
                assert kind != last[q], "differs from the previous gate"
            last[q] = kind
        # every qubit that left a CZ gets a gate
        assert set(q for q, _ in ones) == (in_cz[t - 1] - in_cz[t])
    # fixed rotation of eight layouts: each edge recurs with period 8
    for times in edges_seen.values():
        assert all(b - a == 8 for a, b in zip(times, times[1:]))
    if rows > 1 and cols > 1:
        # every nearest-neighbour edge of the grid is used within 8 cycles
        idx = {rc: i for i, rc in enumerate(coords)}
        all_edges = set()
        for (r, c) in coords:
            for (r2, c2) in ((r, c + 1), (r + 1, c)):
                if (r2, c2) in idx:
                    all_edges.add((idx[(r, c)], idx[(r2, c2)]))
        assert set(edges_seen) == all_edges


def test_random_choice_is_uniform_over_two_allowed_gates():
    counts = {}
    for seed in range(40):
        g = O.generate_circuit(5, 6, 40, seed)
        last = {}
        for x in g[g["cycle"] > 0]:
            k = int(x["kind"])
            if k == O.CZ:
                continue
            q = int(x["q0"])
            if q in last:
                counts[(last[q], k)] = counts.get((last[q], k), 0) + 1
            last[q] = k
    for prev in (O.X_HALF, O.Y_HALF, O.T):
        pair = [counts.get((prev, k), 0) for k in (O.X_HALF, O.Y_HALF, O.T) if k != prev]
        tot = sum(pair)
        assert tot > 500
        assert abs(pair[0] / tot - 0.5) < 4 * 0.5 / np.sqrt(tot)


def test_seed_determinism_and_sensitivity():
    a = O.generate_circuit(4, 5, 25, 3)
    b = O.generate_circuit(4, 5, 25, 3)
    c = O.generate_circuit(4, 5, 25, 4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_gates_per_level_table_one_soft_pin():
    rows = []
    with open(os.path.join(GOLDEN, "table1_gates_per_level.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                r, c, n, gpl = line.split()
                rows.append((int(r), int(c), int(n), float(gpl)))
    for r, c, n, gpl in rows:
        vals = []
        for seed in range(5):
            g = O.generate_circuit(r, c, 25, seed)
            vals.append((np.sum(g["kind"] != O.H) / 25, len(g) / 25))
        excl = np.mean([v[0] for v in vals])
        incl = np.mean([v[1] for v in vals])
        # the printed value lies between the counts without and with the
        # H layer, within 5 %
        assert excl * 0.95 <= gpl <= incl * 1.05, (r, c, excl, incl, gpl)
