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

from adjoint_reference import (PARAM, oracle_fd_grad, oracle_loss, oracle_shift_and_fd,
                               oracle_shift_grad, parameterised_circuit)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    import torch
    assert torch.cuda.is_available()


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
    of the nominal circuit; on a seeded subset of 64 parameters the FP32
    adjoint gradient matches the FP64 oracle's parameter-shift gradient and
    its central differences (h = 1e-4) within 1e-4 of the largest gradient;
    four of them are also checked by evolving the shifted circuits from
    scratch."""
    n = 24
    nominal, noisy, idx = parameterised_circuit(4, 6, 30, 0, 7)
    pnom = O.probabilities(O.simulate(n, nominal))
    x = O.sample(pnom, 100000, 8)
    del pnom
    loss, grad = gpu_grad(n, noisy, x, qs.QS_C64)
    assert loss == pytest.approx(oracle_loss(n, noisy, x), rel=1e-5)
    rng = np.random.default_rng(64)
    subset = rng.choice(idx, size=64, replace=False)
    ref, fd = oracle_shift_and_fd(n, noisy, x, subset)
    scale = np.max(np.abs(ref))
    # central differences carry an O(h^2) truncation error (measured 7e-8
    # absolute here): the same absolute bound as at 12 qubits
    assert np.max(np.abs(fd - ref)) < 1e-6 * max(1.0, scale), np.max(np.abs(fd - ref))
    for k, r in zip(subset[:4], ref[:4]):
        assert oracle_shift_grad(n, noisy, x, int(k)) == pytest.approx(r, rel=1e-9, abs=1e-12 * scale)
    err = np.abs(grad[subset] - ref)
    assert np.max(err) < 1e-4 * scale, (np.max(err) / scale, grad[subset][np.argmax(err)], ref[np.argmax(err)])
    assert np.max(np.abs(grad[subset] - fd)) < 1e-4 * scale + 1e-6


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


def test_torch_autograd_binding_keeps_theta_device():
    """theta on the GPU: loss and gradient come back on the GPU."""
    import torch
    from paper_1608_00263_gb300.autograd import circuit_cross_entropy
    n = 8
    nominal, noisy, idx = parameterised_circuit(2, 4, 10, 3, 5)
    x = O.sample(O.probabilities(O.simulate(n, nominal)), 2000, 8)
    theta = torch.tensor(noisy["theta"][idx], dtype=torch.float32, device="cuda", requires_grad=True)
    h = qs.qs_state_create(n, qs.QS_C128)
    try:
        loss = circuit_cross_entropy(theta, h, noisy, idx, x)
        loss.backward()
    finally:
        qs.qs_state_destroy(h)
    assert loss.device.type == "cuda" and theta.grad.device.type == "cuda"
    ref = np.array([oracle_shift_grad(n, noisy, x, int(k)) for k in idx])
    assert np.max(np.abs(theta.grad.cpu().numpy() - ref)) < 1e-5 * np.max(np.abs(ref))
