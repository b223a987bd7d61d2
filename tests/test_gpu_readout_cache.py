"""Fused read-out of complex64 states: probabilities, statistics partials and
sampler chunk sums come from one pass and are cached for the state as it is;
every change of the amplitudes invalidates the cache, and a state whose
memory the caller can reach is never served from it.  Checked against the
FP64 oracle (Sec. cqs: p_U, entropy, moments, sampling) and for bitwise
agreement between cached and freshly formed results."""
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


def check_stats(r, p):
    assert r["norm"] == pytest.approx(O.norm(p), abs=2.1e-5)
    assert r["entropy"] == pytest.approx(O.entropy(p), rel=1e-6)
    assert r["uniform_ce"] == pytest.approx(O.uniform_ce(p), rel=1e-6)
    for k, v in enumerate(O.moments(p, 10)):
        assert r["moments"][k] == pytest.approx(v, rel=1e-5), k


def same(a, b):
    return a["norm"] == b["norm"] and a["entropy"] == b["entropy"] and a["uniform_ce"] == b["uniform_ce"] \
        and list(a["moments"]) == list(b["moments"])


def test_cache_follows_every_change_of_the_state():
    import torch
    n = 16
    g1, g2 = qs.qs_circuit_generate(4, 4, 20, 1), qs.qs_circuit_generate(4, 4, 20, 2)
    p1, p2 = O.probabilities(O.simulate(n, g1)), O.probabilities(O.simulate(n, g2))
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g1)
        fresh = qs.qs_pt_moments(h, 10)                 # read-out pass without p
        check_stats(fresh, p1)
        out = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        qs.qs_probabilities(h, out, fp64=True)          # read-out pass with p
        assert same(qs.qs_pt_moments(h, 10), fresh)     # served from the cache
        x1 = qs.qs_sample(h, 4096, 7)
        x1b = qs.qs_sample(h, 4096, 7)                  # scanned offsets reused
        assert np.array_equal(x1, x1b)
        # a new circuit: statistics and samples follow it
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g2)
        check_stats(qs.qs_pt_moments(h, 10), p2)
        x2 = qs.qs_sample(h, 4096, 7)
        assert (p2[x2.astype(np.int64)] > 0).all()
        assert not np.array_equal(x1, x2)
        # copy_in: the statistics are those of the copied state
        psi1 = O.simulate(n, g1).astype(np.complex64)
        qs.qs_state_copy_in(h, psi1)
        check_stats(qs.qs_pt_moments(h, 10), p1)
        x1c = qs.qs_sample(h, 4096, 7)
        assert np.mean(x1c == x1) > 0.99            # equal but where rounding moves a boundary
        assert (p1[x1c.astype(np.int64)] > 0).all()
        # reset alone: |0...0>
        qs.qs_state_reset(h)
        r0 = qs.qs_pt_moments(h, 2)
        assert r0["norm"] == 1.0 and abs(r0["entropy"]) < 1e-12
        assert np.all(qs.qs_sample(h, 16, 3) == 0)
    finally:
        qs.qs_state_destroy(h)


def test_reachable_state_is_never_served_from_the_cache():
    import torch
    n = 14
    g = qs.qs_circuit_generate(2, 7, 16, 4)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g)
        qs.qs_pt_moments(h, 4)
        ptr = qs.qs_state_amplitudes(h)

        class _A:
            __cuda_array_interface__ = {"shape": (2 << n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
        amps = torch.as_tensor(_A(), device="cuda")
        amps.zero_()
        amps[2 * 5] = 1.0                               # the caller writes |5>
        torch.cuda.synchronize()
        r = qs.qs_pt_moments(h, 2)
        assert r["norm"] == 1.0 and abs(r["entropy"]) < 1e-12
        assert np.all(qs.qs_sample(h, 8, 1) == 5)
    finally:
        qs.qs_state_destroy(h)


@pytest.mark.parametrize("n", [1, 3, 5, 7, 8])
def test_small_states_partial_chunks(n):
    """States of fewer than 256 amplitudes: one partial chunk."""
    import torch
    rng = np.random.default_rng(n)
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n))
    psi /= np.linalg.norm(psi)
    psi64 = psi.astype(np.complex64)
    p = np.abs(psi64.astype(complex)) ** 2
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_state_copy_in(h, psi64)
        for fp64, dt in ((True, torch.float64), (False, torch.float32)):
            out = torch.empty(1 << n, dtype=dt, device="cuda")
            qs.qs_probabilities(h, out, fp64=fp64)
            torch.cuda.synchronize()
            assert np.allclose(out.cpu().numpy(), p, rtol=2e-7, atol=0)
        check_stats(qs.qs_pt_moments(h, 10), p)
        x = qs.qs_sample(h, 2000, 11)
        assert x.max() < (1 << n) and (p[x.astype(np.int64)] > 0).all()
        # sample j inverts the CDF of the state at the oracle's uniform
        C = np.cumsum(p)
        for j in range(0, 2000, 97):
            t = O.sample_uniform(11, j) * C[-1]
            xj = int(x[j])
            lo = C[xj - 1] if xj else 0.0
            assert lo - 1e-6 <= t <= C[xj] + 1e-6
    finally:
        qs.qs_state_destroy(h)
