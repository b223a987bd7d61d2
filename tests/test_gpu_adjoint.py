"""Adjoint gradient of the sample cross entropy vs exact parameter-shift
gradients and central finite differences from the FP64 oracle.

Parameter shift: for R_P(theta) = exp(-i theta/2 P) and for CPHASE(phi)
(generator Pi_11 = 1/2 + (Pi_11 - 1/2), eigenvalues shifted to +-1/2) the
probability of every basis state obeys dp/dtheta = [p(theta + pi/2) -
p(theta - pi/2)] / 2, so dL/dtheta = -(1/m) sum_j (dp_j/dtheta) / p_j.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build

from seeded_inputs import normals

pytestmark = pytest.mark.gpu

PARAM = (qs.QS_RX, qs.QS_RY, qs.QS_RZ, qs.QS_CPHASE)


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    import torch
    assert torch.cuda.is_available()


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


def gpu_grad(n, gates, x, dtype, mode=qs.QS_MODE_FUSED):
    h = qs.qs_state_create(n, dtype)
    try:
        return qs.qs_adjoint_gradient(h, gates, x, mode=mode)
    finally:
        qs.qs_state_destroy(h)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_all_parameters_12_qubits(dtype):
    n = 12
    nominal, noisy, idx = parameterised_circuit(3, 4, 16, 3, 7)
    x = O.sample(O.probabilities(O.simulate(n, nominal)), 20000, 8)
    loss, grad = gpu_grad(n, noisy, x, dtype)
    assert loss == pytest.approx(oracle_loss(n, noisy, x), rel=1e-6)
    ref = np.array([oracle_shift_grad(n, noisy, x, int(k)) for k in idx])
    fd = np.array([oracle_fd_grad(n, noisy, x, int(k)) for k in idx[:20]])
    assert np.max(np.abs(ref[:20] - fd)) < 1e-6 * max(1.0, np.max(np.abs(ref)))
    tol = 1e-9 if dtype == qs.QS_C128 else 1e-4
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(grad[idx] - ref)) < tol * scale
    fixed = np.setdiff1d(np.arange(noisy.size), idx)
    assert np.all(grad[fixed] == 0)


def test_plain_and_tc_forward_give_the_same_gradient():
    n = 14
    nominal, noisy, idx = parameterised_circuit(2, 7, 20, 5, 9)
    x = O.sample(O.probabilities(O.simulate(n, nominal)), 5000, 8)
    _, g_fused = gpu_grad(n, noisy, x, qs.QS_C64, qs.QS_MODE_FUSED)
    _, g_plain = gpu_grad(n, noisy, x, qs.QS_C64, qs.QS_MODE_PLAIN)
    scale = np.max(np.abs(g_plain))
    assert np.max(np.abs(g_fused - g_plain)) < 1e-4 * scale


def test_grid_4x6_depth30_subset():
    """24 qubits, depth 30 (the adjoint configuration): loss over 1e5 samples
    of the nominal circuit; parameter shift from the FP64 oracle on a seeded
    subset of parameters."""
    n = 24
    nominal, noisy, idx = parameterised_circuit(4, 6, 30, 0, 7)
    pnom = O.probabilities(O.simulate(n, nominal))
    x = O.sample(pnom, 100000, 8)
    del pnom
    loss, grad = gpu_grad(n, noisy, x, qs.QS_C64)
    assert loss == pytest.approx(oracle_loss(n, noisy, x), rel=1e-5)
    rng = np.random.default_rng(64)
    subset = rng.choice(idx, size=3, replace=False)
    ref = np.array([oracle_shift_grad(n, noisy, x, int(k)) for k in subset])
    scale = max(np.max(np.abs(ref)), 1e-3)
    assert np.max(np.abs(grad[subset] - ref)) < 1e-3 * scale, (grad[subset], ref)


def test_torch_autograd_binding():
    import torch
    from paper_1608_00263_gb300.autograd import circuit_cross_entropy
    n = 10
    nominal, noisy, idx = parameterised_circuit(2, 5, 12, 2, 11)
    x = O.sample(O.probabilities(O.simulate(n, nominal)), 4000, 8)
    theta = torch.tensor(noisy["theta"][idx], dtype=torch.float64, requires_grad=True)
    h = qs.qs_state_create(n, qs.QS_C128)
    try:
        loss = circuit_cross_entropy(theta, h, noisy, idx, x)
        loss.backward()
    finally:
        qs.qs_state_destroy(h)
    ref = np.array([oracle_shift_grad(n, noisy, x, int(k)) for k in idx])
    assert float(loss.detach()) == pytest.approx(oracle_loss(n, noisy, x), rel=1e-10)
    assert np.max(np.abs(theta.grad.numpy() - ref)) < 1e-9 * np.max(np.abs(ref))
