"""Noisy trajectories and the batched sampler on the GPU: every trajectory's
state and every sample against the FP64 oracle, mixed instance sizes
(including instances shorter than one sampler chunk), and the cross entropy
difference of noisy samples against Eq. 6 (Fig. sva / Fig. pal setting)."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import build as qs_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    import torch
    assert torch.cuda.is_available()


def device_state(b, i, n):
    import torch
    ptr = qs.qs_batch_state(b, i)

    class _A:
        __cuda_array_interface__ = {"shape": (2 << n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_A(), device="cuda").cpu().numpy().view(np.complex64)


def check_samples(got, p_ref, p_dev, n, seed, k, i, r_mes):
    """Sample j of instance i: identical to the oracle's rule on the oracle
    state, except where rounding moves a CDF boundary (the FP32 state, and
    the FP32 prefix sums inside a 256-amplitude chunk); such a sample, with
    its measurement flips undone, must still invert the GPU state's CDF
    within that rounding (1e-6 of the total)."""
    mism = 0
    c = np.cumsum(p_dev)
    tol = 1e-6 * c[-1]
    for j in range(k):
        ctr = i * k + j
        want = O.measurement_flips(int(O.sample_at(p_ref, seed, [ctr])[0]), n, seed, r_mes, ctr)
        if int(got[j]) != want:
            mism += 1
            x = int(got[j]) ^ O.measurement_flips(0, n, seed, r_mes, ctr)
            t = O.sample_uniform(seed, ctr) * c[-1]
            lo = c[x - 1] if x > 0 else 0.0
            assert lo - tol <= t <= c[x] + tol, (i, j, int(got[j]), want, t, lo, c[x])
    return mism


def test_trajectories_and_batch_samples_match_oracle():
    rows, cols, depth = 3, 4, 16
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 6)
    T, k, seed, r_mes = 48, 32, 5, 0.03
    lists = [qs.qs_noisy_circuit(g, n, 0.02, 0.1, 0.05, 100 + t) for t in range(T)]
    assert sum(len(h) > len(g) for h in lists) > T // 2      # most trajectories have errors
    b = qs.qs_batch_create([n] * T)
    try:
        qs.qs_batch_apply(b, lists)
        got = qs.qs_batch_sample(b, k, seed, r_mes)
        assert got.shape == (T, k)
        mism = 0
        for t in range(T):
            ref = O.simulate(n, lists[t])
            psi = device_state(b, t, n)
            err = np.linalg.norm(psi.astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (t, err)
            mism += check_samples(got[t], O.probabilities(ref), np.abs(psi.astype(complex)) ** 2, n,
                                  seed, k, t, r_mes)
        assert mism <= 0.01 * T * k
    finally:
        qs.qs_batch_destroy(b)


def test_batch_sampler_mixed_sizes():
    """Instances of 5..13 qubits (chunks of 256 amplitudes never straddle
    instances; states below 256 amplitudes form one short chunk)."""
    sizes = [(1, 5), (1, 7), (2, 4), (3, 3), (2, 5), (3, 4), (1, 13)]
    gl, ns = [], []
    for s, (r, c) in enumerate(sizes):
        gl.append(qs.qs_circuit_generate(r, c, 12, s))
        ns.append(r * c)
    k, seed = 64, 9
    b = qs.qs_batch_create(ns)
    try:
        qs.qs_batch_run(b, gl, kmax=0)
        got = qs.qs_batch_sample(b, k, seed, 0.0)
        mism = 0
        for i, (n, g) in enumerate(zip(ns, gl)):
            ref = O.simulate(n, g)
            psi = device_state(b, i, n)
            assert np.all(got[i] < (1 << n))
            mism += check_samples(got[i], O.probabilities(ref), np.abs(psi.astype(complex)) ** 2, n,
                                  seed, k, i, 0.0)
        assert mism <= 0.01 * len(ns) * k
    finally:
        qs.qs_batch_destroy(b)


@pytest.mark.parametrize("r", [0.0, 0.005])
def test_noisy_cross_entropy_tracks_eq6(r):
    """Fig. pal setting: 5 x 4 qubits, depth 40, r2 = r_init = r_mes = r, r1 = r/10.
    One sample per trajectory; Delta H (Eq. 5) of the samples under the ideal
    circuit's distribution against Eq. 6."""
    rows, cols, depth = 4, 5, 40
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 0)
    g1 = int(np.sum(g["kind"] != qs.QS_CZ))
    g2 = int(np.sum(g["kind"] == qs.QS_CZ))
    r1, r2, ri, rm = r / 10, r, r, r
    T = 2048
    lists = [qs.qs_noisy_circuit(g, n, r1, r2, ri, 5000 + t) for t in range(T)]
    b = qs.qs_batch_create([n] * T)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_batch_apply(b, lists)
        x = qs.qs_batch_sample(b, 1, 123, rm).reshape(-1)
        qs.qs_apply_circuit(h, g)
        ce, dh = qs.qs_cross_entropy(h, x)
    finally:
        qs.qs_batch_destroy(b)
        qs.qs_state_destroy(h)
    alpha = O.eq6_fidelity(r1, r2, ri, rm, g1, g2, n)
    assert abs(dh - alpha) < 0.06 + 3 * 1.3 / math.sqrt(T), (dh, alpha)
