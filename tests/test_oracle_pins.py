"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: gate application is checked
against dense Kronecker-product unitaries and against the Feynman path sum of
Eqs. path1/phX/phT/phCZ; statistics against Porter-Thomas closed forms
(Eqs. eu, eue, the moment limit k! of Sec. "Convergence to Porter-Thomas")
and exact special cases; the sampler against brute-force CDF inversion, a
chi-square test and the alpha = 1 case of Eq. pal; SplitMix64 against its
published output sequence.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import oracle as O

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


# --------------------------------------------------------------------------
# helpers independent of the oracle's index arithmetic
# --------------------------------------------------------------------------
def embed(n, ops):
    """Full 2^n operator: tensor product over qubits n-1 .. 0 (bit j of the
    basis index is qubit j, so qubit n-1 is the leftmost factor)."""
    m = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        m = np.kron(m, ops.get(q, I2))
    return m


def dense_unitary(n, gates):
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        u = O.gate_matrix(int(g["kind"]), float(g["theta"]))
        if int(g["kind"]) in O.TWO_QUBIT_KINDS:
            c, t = int(g["q0"]), int(g["q1"])
            G = embed(n, {}) - embed(n, {c: P1}) + embed(n, {c: P1, t: u})
        else:
            G = embed(n, {int(g["q0"]): u})
        U = G @ U
    return U


def random_gate_list(rng, n, count):
    gates = np.zeros(count, dtype=O.GATE_DTYPE)
    for i in range(count):
        kind = int(rng.integers(0, 9))
        gates[i]["kind"] = kind
        if kind in O.TWO_QUBIT_KINDS:
            a, b = rng.choice(n, size=2, replace=False)
            gates[i]["q0"], gates[i]["q1"] = a, b
        else:
            gates[i]["q0"] = rng.integers(0, n)
        gates[i]["theta"] = rng.uniform(-np.pi, np.pi)
    return gates


def ideal_probabilities(rows, cols, depth, seed):
    g = O.generate_circuit(rows, cols, depth, seed)
    psi = O.simulate(rows * cols, g)
    return O.probabilities(psi)


# --------------------------------------------------------------------------
# gate matrices
# --------------------------------------------------------------------------
def test_gate_matrices_unitary():
    for kind in range(9):
        for theta in (0.0, 0.3, -2.1, np.pi):
            u = O.gate_matrix(kind, theta)
            assert np.allclose(u.conj().T @ u, I2, atol=1e-15)


def test_rotation_gates_are_exponentials_of_paulis():
    # R_P(theta) = exp(-i theta/2 P): reduces to scipy's matrix exponential.
    for theta in (0.0, 0.37, 1.9, -2.6):
        for kind, P in ((O.RX, PX), (O.RY, PY), (O.RZ, PZ)):
            assert np.allclose(O.gate_matrix(kind, theta),
                               scipy.linalg.expm(-0.5j * theta * P), atol=1e-14)
        # CPHASE(phi): target phase e^{i phi} when control and target are 1
        assert np.allclose(O.gate_matrix(O.CPHASE, theta),
                           np.diag([1, np.exp(1j * theta)]), atol=1e-15)


def test_fixed_gates_match_paper_definitions():
    s = 1 / np.sqrt(2)
    # X^1/2, Y^1/2 are pi/2 rotations: squares are the Paulis up to phase,
    # and they equal the rotation matrices at theta = pi/2.
    X2 = O.gate_matrix(O.X_HALF)
    Y2 = O.gate_matrix(O.Y_HALF)
    assert np.allclose(X2 @ X2, -1j * PX, atol=1e-15)
    assert np.allclose(Y2 @ Y2, -1j * PY, atol=1e-15)
    assert np.allclose(X2, scipy.linalg.expm(-0.25j * np.pi * PX), atol=1e-15)
    assert np.allclose(Y2, scipy.linalg.expm(-0.25j * np.pi * PY), atol=1e-15)
    # T = diag(1, e^{i pi/4}); T^8 = I, T^4 = Z
    T = O.gate_matrix(O.T)
    assert np.allclose(T, np.diag([1, np.exp(0.25j * np.pi)]), atol=1e-15)
    assert np.allclose(np.linalg.matrix_power(T, 4), PZ, atol=1e-15)
    # H: Hadamard, H Z H = X
    Hm = O.gate_matrix(O.H)
    assert np.allclose(Hm, s * np.array([[1, 1], [1, -1]]), atol=1e-15)
    assert np.allclose(Hm @ PZ @ Hm, PX, atol=1e-15)
    # CZ on the target when the control is set: Z
    assert np.allclose(O.gate_matrix(O.CZ), PZ, atol=0)


# --------------------------------------------------------------------------
# gate application vs dense Kronecker unitaries
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_apply_matches_dense_unitary_random_gates(n):
    rng = np.random.default_rng(100 + n)
    gates = random_gate_list(rng, n, 40) if n > 1 else \
        np.array([g for g in random_gate_list(rng, 2, 60)
                  if int(g["kind"]) not in O.TWO_QUBIT_KINDS
                  and int(g["q0"]) == 0][:20], dtype=O.GATE_DTYPE)
    U = dense_unitary(n, gates)
    assert np.allclose(U.conj().T @ U, np.eye(1 << n), atol=1e-12)
    psi = O.simulate(n, gates)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    assert np.max(np.abs(psi - U @ e0)) < 1e-12
    # and on a random input state (every column of U, not only the first)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    w = O.apply_circuit(v.copy(), gates)
    assert np.max(np.abs(w - U @ v)) < 1e-11


def test_apply_matches_dense_unitary_generated_circuit():
    g = O.generate_circuit(2, 4, 16, 7)
    U = dense_unitary(8, g)
    psi = O.simulate(8, g)
    assert np.max(np.abs(psi - U[:, 0])) < 1e-12
    assert np.max(np.abs(U.conj().T @ U - np.eye(256))) < 1e-12


# --------------------------------------------------------------------------
# Feynman path sum, Eqs. path1 / phX / phT / phCZ
# --------------------------------------------------------------------------
def feynman_state(n, gates):
    """<x|psi> = sum over spin paths of prod(1/sqrt2 per two-sparse gate) *
    exp(i pi/4 H_s(x)).  Spin s = +1 is |0>, -1 is |1>.  Phase rules:
    X^1/2 adds pi/2 when the spin does not flip; Y^1/2 adds pi on the
    transition |1> -> |0>; T adds pi/4 on |1>; CZ adds pi on |11>.  The H
    layer acts on |0> and adds no phase.  The current spin of a qubit at a
    T or CZ is the one after its latest two-sparse gate."""
    two_sparse = (O.H, O.X_HALF, O.Y_HALF)
    seq = [[] for _ in range(n)]           # per qubit: kinds of two-sparse gates
    for g in gates:
        if int(g["kind"]) in two_sparse:
            seq[int(g["q0"])].append(int(g["kind"]))
    # free spins: every two-sparse output except the last one of each qubit
    free = [(j, k) for j in range(n) for k in range(len(seq[j]) - 1)]
    G = len(free)
    ngates2 = sum(len(s) for s in seq)
    amp = np.zeros(1 << n, dtype=complex)
    paths = np.array(list(itertools.product((1, -1), repeat=G)), dtype=int) \
        if G else np.zeros((1, 0), dtype=int)
    for x in range(1 << n):
        # spins[j][k]: array over paths
        spins = []
        col = 0
        for j in range(n):
            row = []
            for k in range(len(seq[j])):
                if k == len(seq[j]) - 1:
                    xb = (x >> j) & 1
                    row.append(np.full(paths.shape[0], 1 - 2 * xb))
                else:
                    row.append(paths[:, col])
                    col += 1
            spins.append(row)
        if any(len(s) == 0 for s in seq):
            # a qubit with no two-sparse gate stays |0>
            if any(len(seq[j]) == 0 and (x >> j) & 1 for j in range(n)):
                continue
        phase = np.zeros(paths.shape[0])        # in units of pi/4
        pos = [-1] * n                          # index of current spin
        for g in gates:
            kind = int(g["kind"])
            if kind in two_sparse:
                j = int(g["q0"])
                k = pos[j] + 1
                prev = np.ones(paths.shape[0], dtype=int) if k == 0 else spins[j][k - 1]
                cur = spins[j][k]
                if kind == O.X_HALF:
                    phase += 2 * (1 + prev * cur) / 2
                elif kind == O.Y_HALF:
                    phase += 4 * ((1 - prev) / 2) * ((1 + cur) / 2)
                pos[j] = k
            elif kind == O.T:
                j = int(g["q0"])
                cur = spins[j][pos[j]] if pos[j] >= 0 else np.ones(paths.shape[0])
                phase += 1 * (1 - cur) / 2
            elif kind == O.CZ:
                a, b = int(g["q0"]), int(g["q1"])
                sa = spins[a][pos[a]] if pos[a] >= 0 else np.ones(paths.shape[0])
                sb = spins[b][pos[b]] if pos[b] >= 0 else np.ones(paths.shape[0])
                phase += 4 * ((1 - sa) / 2) * ((1 - sb) / 2)
            else:
                raise AssertionError("path sum covers the paper's gate set only")
        # the phase takes one of 8 values, multiples of pi/4
        assert np.allclose(phase, np.round(phase))
        amp[x] = 2.0 ** (-ngates2 / 2) * np.sum(np.exp(0.25j * np.pi * phase))
    return amp


@pytest.mark.parametrize("rows,cols,depth,seed", [
    (2, 2, 10, 1), (2, 2, 12, 5), (1, 4, 11, 3), (1, 3, 14, 9), (1, 2, 16, 2)])
def test_oracle_matches_feynman_path_sum(rows, cols, depth, seed):
    g = O.generate_circuit(rows, cols, depth, seed)
    kinds = set(int(k) for k in g["kind"])
    assert kinds & {O.X_HALF, O.Y_HALF}, "circuit must contain two-sparse gates"
    n = rows * cols
    path = feynman_state(n, g)
    assert abs(np.vdot(path, path).real - 1) < 1e-12
    psi = O.simulate(n, g)
    i = int(np.argmax(np.abs(psi)))
    ph = psi[i] / path[i]
    assert abs(abs(ph) - 1) < 1e-12
    assert np.max(np.abs(psi - ph * path)) < 1e-12


# --------------------------------------------------------------------------
# invariants and exact special cases
# --------------------------------------------------------------------------
def test_norm_conserved_and_time_reversal():
    g = O.generate_circuit(3, 4, 30, 11)
    psi = O.simulate(12, g)
    p = O.probabilities(psi)
    assert abs(O.norm(p) - 1) < 1e-13
    # apply the inverse gates in reverse order: back to |0...0>
    for gate in g[::-1]:
        u = O.gate_matrix(int(gate["kind"]), float(gate["theta"])).conj().T
        if int(gate["kind"]) in O.TWO_QUBIT_KINDS:
            O.apply_controlled(psi, int(gate["q0"]), int(gate["q1"]), u)
        else:
            O.apply_1q(psi, int(gate["q0"]), u)
    e0 = np.zeros_like(psi)
    e0[0] = 1
    assert np.max(np.abs(psi - e0)) < 1e-13


def test_cz_is_symmetric_in_its_qubits():
    rng = np.random.default_rng(3)
    v = rng.normal(size=64) + 1j * rng.normal(size=64)
    a = O.apply_controlled(v.copy(), 1, 4, O.gate_matrix(O.CZ))
    b = O.apply_controlled(v.copy(), 4, 1, O.gate_matrix(O.CZ))
    assert np.array_equal(a, b)


def test_early_cycles_uniform_distribution():
    # Before any X^1/2 / Y^1/2 acts the circuit is H-layer + diagonal gates,
    # so p = 1/N exactly, entropy = ln N, N sum p^2 = 1 (Sec. "Convergence to
    # Porter-Thomas": first cycles do not change the output entropy).
    g = O.generate_circuit(4, 4, 20, 4)
    first = next(i for i, x in enumerate(g) if int(x["kind"]) in (O.X_HALF, O.Y_HALF))
    assert first > 16
    assert all(int(x["kind"]) in (O.H, O.T, O.CZ) for x in g[:first])
    p = O.probabilities(O.simulate(16, g[:first]))
    N = 1 << 16
    assert np.max(np.abs(p * N - 1)) < 1e-12
    assert abs(O.entropy(p) - 16 * math.log(2)) < 1e-10
    m = O.moments(p, 4)
    assert np.allclose(m, 1.0, atol=1e-10)
    assert abs(O.uniform_ce(p) - 16 * math.log(2)) < 1e-10


def test_clifford_variant_is_flat():
    # Replace T by S (up to phase RZ(pi/2)): an H/X^1/2/Y^1/2/S/CZ circuit
    # outputs a stabilizer state, uniform over its support, so
    # H = -ln sum p^2 and N^{k-1} sum p^k = (N sum p^2)^{k-1}.
    g = O.generate_circuit(3, 4, 24, 8)
    g = g.copy()
    for x in g:
        if int(x["kind"]) == O.T:
            x["kind"] = O.RZ
            x["theta"] = np.pi / 2
    p = O.probabilities(O.simulate(12, g))
    support = p[p > 1e-12]
    assert np.allclose(support, support[0], rtol=1e-9)
    m = O.moments(p, 6)
    assert abs(O.entropy(p) + math.log(np.sum(p ** 2))) < 1e-9
    for k in range(1, 7):
        assert m[k - 1] == pytest.approx(m[1] ** (k - 1), rel=1e-9)


# --------------------------------------------------------------------------
# Porter-Thomas closed forms for deep circuits
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def deep_p():
    # 4 x 4 grid, depth 40: deep in the Porter-Thomas regime
    return [ideal_probabilities(4, 4, 40, s) for s in range(3)]


def test_entropy_porter_thomas(deep_p):
    n = 16
    sigma = 0.75 * 2.0 ** (-n / 2)          # spread quoted in the paper
    for p in deep_p:
        assert abs(O.entropy(p) - (n * math.log(2) - 1 + O.EULER_GAMMA)) < 4 * sigma


def test_uniform_cross_entropy_porter_thomas(deep_p):
    n = 16
    N = 2.0 ** n
    sd = math.sqrt(math.pi ** 2 / 6 / N)    # sd of mean of ln(Np), Np ~ Exp(1)
    for p in deep_p:
        assert abs(O.uniform_ce(p) - (n * math.log(2) + O.EULER_GAMMA)) < 5 * sd


def test_moments_porter_thomas(deep_p):
    N = 2.0 ** 16
    for p in deep_p:
        m = O.moments(p, 10)
        assert m[0] == pytest.approx(1.0, abs=1e-12)
        for k in range(2, 11):
            rel_sd = math.sqrt((math.factorial(2 * k) - math.factorial(k) ** 2) / N) \
                / math.factorial(k)
            assert abs(m[k - 1] / math.factorial(k) - 1) < 5 * rel_sd + 0.01, k


def test_second_moment_haar_mean():
    # E[sum p^2] = 2/(N+1) (Haar) -- averaged over instances
    vals = [np.sum(ideal_probabilities(3, 4, 40, s) ** 2) for s in range(8)]
    N = 2 ** 12
    assert np.mean(vals) * (N + 1) / 2 == pytest.approx(1.0, abs=0.05)


# --------------------------------------------------------------------------
# SplitMix64 and the sampler
# --------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014).
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [O.splitmix64_output(0, j) for j in range(5)] == expected


def test_sampler_is_cdf_inversion():
    rng = np.random.default_rng(5)
    p = rng.random(32)
    p[[3, 7, 8, 20]] = 0.0                  # zero entries are never chosen
    p /= 1.3                                # unnormalised on purpose
    m = 4000
    x = O.sample(p, m, 77)
    C = np.cumsum(p)
    for j in range(m):
        u = O.sample_uniform(77, j)
        expect = next(i for i in range(32) if C[i] > u * C[-1])
        assert x[j] == expect
    assert not np.isin(x, [3, 7, 8, 20]).any()


def test_sample_uniforms_are_uniform():
    u = np.array([O.sample_uniform(123, j) for j in range(20000)])
    assert u.min() >= 0 and u.max() < 1
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = np.sum((hist - 1000) ** 2 / 1000)
    assert chi2 < 60                         # 19 dof, p ~ 1e-6


def test_sampler_chi_square_and_cross_entropy():
    p = ideal_probabilities(4, 4, 30, 2)
    m = 200000
    x = O.sample(p, m, 1000)
    # coarse bins on the top 6 index bits
    bins = (x >> np.uint64(10)).astype(np.int64)
    counts = np.bincount(bins, minlength=64)
    expected = m * p.reshape(64, -1).sum(axis=1)
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 140                        # 63 dof, p ~ 1e-7
    # Eq. ae on ideal samples: Delta H ~ 1, error ~ kappa/sqrt(m)
    ce, dh = O.cross_entropy(p, x)
    assert abs(dh - 1) < 0.02
    assert ce == pytest.approx(-np.mean(np.log(p[x])), rel=1e-12)
    # uniform samples give Delta H ~ 0 (Eq. 5)
    xu = np.arange(0, 1 << 16, dtype=np.uint64)
    _, dh0 = O.cross_entropy(p, xu)
    assert abs(dh0 - (O.uniform_ce(p) * -1 + 16 * math.log(2) + O.EULER_GAMMA)) < 1e-9
    assert abs(dh0) < 0.02


def test_sampled_log_probability_histogram_eq_pal():
    # Eq. pal with alpha = 1: z = ln(N p(x)) over ideal samples has density
    # e^{z - e^z} (1 + (e^z - 1)) = e^{2z - e^z}; its CDF is
    # 1 - (1 + e^z) e^{-e^z}.
    p = ideal_probabilities(4, 4, 30, 6)
    x = O.sample(p, 100000, 9)
    z = np.sort(np.log(p[x] * (1 << 16)))
    F = 1 - (1 + np.exp(z)) * np.exp(-np.exp(z))
    emp = np.arange(1, z.size + 1) / z.size
    ks = np.max(np.abs(emp - F))
    assert ks < 0.012


def test_shifted_amplitudes_equal_shifted_circuits():
    """The adjoint tests form a shifted circuit's amplitudes from two FP64
    states (R_P(theta + d) = R_P(theta) R_P(d), CPHASE(phi + d) = CPHASE(phi)
    (1 + (e^{id} - 1) Pi_11)); that must equal evolving the shifted circuit
    from scratch, for every parameter kind and several shifts."""
    from adjoint_reference import PARAM, _shifted_amplitudes, parameterised_circuit
    n = 10
    nominal, noisy, idx = parameterised_circuit(2, 5, 12, 4, 13)
    xi = np.arange(1 << n, dtype=np.int64)
    psi_final = O.simulate(n, noisy)
    kinds_seen = set()
    picks = [int(k) for kind in PARAM for k in idx[noisy["kind"][idx] == kind][:3]]
    for k in picks:
        kinds_seen.add(int(noisy[k]["kind"]))
        amp = _shifted_amplitudes(n, noisy, k, xi, O.simulate(n, noisy[:k]), psi_final)
        for d in (np.pi / 2, -np.pi / 2, 0.3):
            gs = noisy.copy()
            gs[k]["theta"] += d
            assert np.max(np.abs(amp(d) - O.simulate(n, gs))) < 1e-12
    assert kinds_seen == set(PARAM)


def test_shift_and_fd_gradients_agree_with_plain_shifted_circuits():
    """The one-suffix-per-parameter gradients equal the parameter shift taken
    by evolving the two shifted circuits from scratch, and central
    differences agree with both (12 qubits, every parameter kind)."""
    from adjoint_reference import (oracle_fd_grad, oracle_shift_and_fd, oracle_shift_grad,
                                   parameterised_circuit)
    n = 12
    nominal, noisy, idx = parameterised_circuit(3, 4, 16, 3, 7)
    x = O.sample(O.probabilities(O.simulate(n, nominal)), 5000, 8)
    subset = idx[::9]
    ps, fd = oracle_shift_and_fd(n, noisy, x, subset)
    direct = np.array([oracle_shift_grad(n, noisy, x, int(k)) for k in subset])
    fd_direct = np.array([oracle_fd_grad(n, noisy, x, int(k)) for k in subset[:6]])
    scale = np.max(np.abs(direct))
    assert np.max(np.abs(ps - direct)) < 1e-12 * scale
    assert np.max(np.abs(fd[:6] - fd_direct)) < 1e-8 * scale
    assert np.max(np.abs(fd - ps)) < 1e-6 * scale
