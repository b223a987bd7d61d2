"""The diagonal prefix folded into a circuit's initial state (CPU).

After a leading layer of H on every qubit of |0...0>, a T or CZ gate none of
whose qubits has yet met a non-diagonal gate commutes with every gate before
it, so it can act first, on the uniform superposition, where the whole
prefix is the phase e^{i pi k(x) / 4} with k = 4 (CZ pairs set in x) + (T
counts of the qubits set in x), mod 8 (T = diag(1, e^{i pi / 4}), CZ =
diag(1, 1, 1, -1); Sec. "Random circuits" gate set).  Checked on the oracle:
moving the folded gates to the front leaves the state unchanged, and the
state after the layer and the folded gates is that closed form.  The rule is
the bench's mirror of the library's (`bench.fold_diagonal_prefix`); the
library's own fold is compared with the oracle on the GPU."""
import numpy as np
import pytest

import bench
import oracle as O
import paper_1608_00263_gb300 as qs


def gate(kind, q0, q1=0, theta=0.0):
    g = np.zeros(1, dtype=qs.GATE_DTYPE)
    g["kind"], g["q0"], g["q1"], g["theta"] = kind, q0, q1, theta
    return g


def cat(*gs):
    return np.concatenate(gs)


def test_partition_of_a_hand_built_list():
    g = cat(gate(qs.QS_T, 0), gate(qs.QS_CZ, 0, 1), gate(qs.QS_X_HALF, 1), gate(qs.QS_T, 1),
            gate(qs.QS_CZ, 1, 2), gate(qs.QS_CZ, 0, 2), gate(qs.QS_Y_HALF, 0), gate(qs.QS_T, 0),
            gate(qs.QS_RZ, 2, theta=0.3), gate(qs.QS_T, 2))
    nf, rest = bench.fold_diagonal_prefix(qs, g)
    # folded: T0, CZ(0,1), CZ(0,2) (neither qubit touched yet), T2 (RZ is
    # diagonal and touches nothing); kept: X1/2 on 1 and what follows it on 1,
    # Y1/2 on 0 and the T after it, RZ
    assert nf == 4
    assert rest["kind"].tolist() == [qs.QS_X_HALF, qs.QS_T, qs.QS_CZ, qs.QS_Y_HALF, qs.QS_T, qs.QS_RZ]
    assert rest["q0"].tolist() == [1, 1, 1, 0, 0, 2]


def _folded_gates(g):
    nf, rest = bench.fold_diagonal_prefix(qs, g)
    # the folded gates in order: those not kept (lists here have no repeats
    # of a kept gate before its folded twin)
    kept_idx, j = [], 0
    for i in range(len(g)):
        if j < len(rest) and g[i].tobytes() == rest[j].tobytes():
            kept_idx.append(i)
            j += 1
    assert j == len(rest)
    mask = np.ones(len(g), dtype=bool)
    mask[kept_idx] = False
    assert mask.sum() == nf
    return g[mask], rest


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 3, 8, 0), (3, 3, 10, 1), (3, 4, 12, 2), (2, 4, 6, 7)])
def test_folded_gates_commute_to_the_front(rows, cols, depth, seed):
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, seed)
    assert bench.leading_h_layer(qs, g, n) == n
    folded, rest = _folded_gates(g[n:])
    assert len(folded) > 0
    a = O.simulate(n, g)
    b = O.simulate(n, cat(g[:n], folded, rest))
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 3, 8, 0), (3, 3, 10, 1), (3, 4, 12, 2)])
def test_state_after_the_folded_prefix_is_the_closed_form(rows, cols, depth, seed):
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, seed)
    folded, _ = _folded_gates(g[n:])
    psi = O.simulate(n, cat(g[:n], folded))
    x = np.arange(1 << n, dtype=np.int64)
    bit = lambda q: (x >> q) & 1
    k = np.zeros(1 << n, dtype=np.int64)
    for r in folded:
        if r["kind"] == qs.QS_T:
            k += bit(int(r["q0"]))
        else:
            assert r["kind"] == qs.QS_CZ
            k += 4 * bit(int(r["q0"])) * bit(int(r["q1"]))
    want = 2.0 ** (-n / 2) * np.exp(1j * np.pi * (k % 8) / 4)
    assert np.max(np.abs(psi - want)) < 1e-14
