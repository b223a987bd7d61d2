"""Oracle-side gradients for the adjoint tests (test infrastructure).

Parameter shift: for R_P(theta) = exp(-i theta/2 P) and for CPHASE(phi)
(generator Pi_11 = 1/2 + (Pi_11 - 1/2), eigenvalues shifted to +-1/2) the
probability of every basis state obeys dp/dtheta = [p(theta + pi/2) -
p(theta - pi/2)] / 2, so dL/dtheta = -(1/m) sum_j (dp_j/dtheta) / p_j for
L = -(1/m) sum_j ln p(x_j).  Everything here evolves states with the FP64
oracle; nothing calls the CUDA library except its host-side circuit
generator.
"""
import numpy as np

import oracle as O
import paper_1608_00263_gb300 as qs

from seeded_inputs import normals

PARAM = (qs.QS_RX, qs.QS_RY, qs.QS_RZ, qs.QS_CPHASE)


def parameterised_circuit(rows, cols, depth, seed, noise_seed, dead=None):
    """The random circuit with every single-qubit gate replaced by R_P(theta)
    (X^1/2 -> RX(pi/2), Y^1/2 -> RY(pi/2), T -> RZ(pi/4)) and every CZ by
    CPHASE(pi); the H layer stays fixed.  Angles get 0.05 N(0,1) noise."""
    g = qs.qs_circuit_generate(rows, cols, depth, seed, dead).copy()
    nominal = g.copy()
    for x in nominal:
        k = int(x["kind"])
        if k == qs.QS_X_HALF:
            x["kind"], x["theta"] = qs.QS_RX, np.pi / 2
        elif k == qs.QS_Y_HALF:
            x["kind"], x["theta"] = qs.QS_RY, np.pi / 2
        elif k == qs.QS_T:
            x["kind"], x["theta"] = qs.QS_RZ, np.pi / 4
        elif k == qs.QS_CZ:
            x["kind"], x["theta"] = qs.QS_CPHASE, np.pi
    idx = np.nonzero(np.isin(nominal["kind"], PARAM))[0]
    noisy = nominal.copy()
    noisy["theta"][idx] += 0.05 * np.array(normals(noise_seed, idx.size))
    return nominal, noisy, idx


def oracle_loss(n, gates, x):
    p = O.probabilities(O.simulate(n, gates))
    return -np.mean(np.log(p[x.astype(np.int64)]))


def oracle_shift_grad(n, gates, x, k):
    xi = x.astype(np.int64)
    p0 = O.probabilities(O.simulate(n, gates))[xi]
    gp, gm = gates.copy(), gates.copy()
    gp[k]["theta"] += np.pi / 2
    gm[k]["theta"] -= np.pi / 2
    pp = O.probabilities(O.simulate(n, gp))[xi]
    pm = O.probabilities(O.simulate(n, gm))[xi]
    return -np.mean((pp - pm) / 2 / p0)


def oracle_fd_grad(n, gates, x, k, h=1e-4):
    gp, gm = gates.copy(), gates.copy()
    gp[k]["theta"] += h
    gm[k]["theta"] -= h
    return (oracle_loss(n, gp, x) - oracle_loss(n, gm, x)) / (2 * h)


def _shifted_amplitudes(n, gates, k, xi, psi_prefix, psi_final):
    """Amplitudes at the sample indices of the circuit with parameter k moved
    by delta, for any delta, from two FP64 states: a = psi(theta)[x] and
    b = phi[x] with phi = U_{>k} G_k (Q psi_{<k}), where Q = P for
    R_P(theta) (R_P(theta + delta) = R_P(theta) R_P(delta) and R_P(delta) =
    cos(delta/2) - i sin(delta/2) P) and Q = Pi_11 for CPHASE (CPHASE(phi +
    delta) = CPHASE(phi) (1 + (e^{i delta} - 1) Pi_11)).  Returns a function
    delta -> amplitudes."""
    g = gates[k]
    kind = int(g["kind"])
    phi = psi_prefix.copy()
    if kind == qs.QS_CPHASE:
        idx = np.arange(phi.size, dtype=np.int64)
        keep = ((idx >> int(g["q0"])) & 1) & ((idx >> int(g["q1"])) & 1)
        phi[keep == 0] = 0
        del idx, keep
    else:
        pauli = {qs.QS_RX: [[0, 1], [1, 0]], qs.QS_RY: [[0, -1j], [1j, 0]],
                 qs.QS_RZ: [[1, 0], [0, -1]]}[kind]
        O.apply_1q(phi, int(g["q0"]), np.array(pauli, dtype=np.complex128))
    O.apply_circuit(phi, gates[k:])
    a, b = psi_final[xi], phi[xi]
    if kind == qs.QS_CPHASE:
        return lambda d: a + (np.exp(1j * d) - 1) * b
    return lambda d: np.cos(d / 2) * a - 1j * np.sin(d / 2) * b


def oracle_shift_and_fd(n, gates, x, subset, h=1e-4):
    """Parameter-shift and central-difference gradients of L = -(1/m) sum ln
    p(x_j) for the parameters in `subset`, from FP64 oracle states: one
    forward sweep keeps the prefix state, and each parameter costs one
    suffix evolution (see _shifted_amplitudes)."""
    xi = x.astype(np.int64)
    psi_final = O.simulate(n, gates)
    p0 = np.abs(psi_final[xi]) ** 2
    psi = O.zero_state(n)
    pos = 0
    ps, fd = {}, {}
    for k in sorted(int(k) for k in subset):
        O.apply_circuit(psi, gates[pos:k])
        pos = k
        amp = _shifted_amplitudes(n, gates, k, xi, psi, psi_final)
        pp, pm = np.abs(amp(np.pi / 2)) ** 2, np.abs(amp(-np.pi / 2)) ** 2
        ps[k] = -np.mean((pp - pm) / 2 / p0)
        lp = -np.mean(np.log(np.abs(amp(h)) ** 2))
        lm = -np.mean(np.log(np.abs(amp(-h)) ** 2))
        fd[k] = (lp - lm) / (2 * h)
    return (np.array([ps[int(k)] for k in subset]), np.array([fd[int(k)] for k in subset]))


