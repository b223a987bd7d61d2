"""qs_sample_noalloc: the sampler variant that allocates no memory.

It exists for callers that cannot allocate device memory while they run, for
example a host application or framework that gives all GPU memory to its own
pool or fixes its memory budget up front.  Its scratch is a fixed 8 MiB array
compiled into the library, so it only takes states of up to 28 qubits.  Its
samples must equal qs_sample's for the same state and seed, call after call,
although every call reuses the same scratch array, and they must be the
oracle's inverse-CDF samples of the same probabilities.

This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native
from paper_1608_00263_gb300 import build as qs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    return _native.lib()


@pytest.mark.parametrize("n", [0, 29, -1])
def test_noalloc_rejects_sizes_outside_1_to_28_before_any_device_work(n):
    # the size check comes first, so this runs without a GPU; the pointers
    # are never dereferenced
    with pytest.raises(qs.QSError) as e:
        qs.qs_sample_noalloc(n, qs.QS_C64, 1 << 20, 10, 1, 1 << 21)
    assert e.value.status == _native.QS_ERR_INVALID_ARG
    assert "28" in str(e.value)


def test_noalloc_rejects_a_bad_dtype_before_any_device_work():
    with pytest.raises(qs.QSError) as e:
        qs.qs_sample_noalloc(10, 7, 1 << 20, 10, 1, 1 << 21)
    assert e.value.status == _native.QS_ERR_INVALID_ARG


def _justified(p, x, seed, bound):
    """Every sample x_j satisfies the inversion C_{x-1} <= u_j C_{N-1} < C_x
    of the FP64 cumulative sum of p within `bound`."""
    C = np.cumsum(p)
    u = np.array([O.sample_uniform(seed, j) for j in range(x.size)])
    target = u * C[-1]
    xi = x.astype(np.int64)
    lo = np.where(xi > 0, C[np.maximum(xi - 1, 0)], 0.0)
    ok = (lo - bound <= target) & (target < C[xi] + bound)
    assert ok.all(), np.nonzero(~ok)[0][:10]


def _state(n, dtype, cseed):
    """A random-circuit state of n qubits (grids 1 x n up to 4 x 7)."""
    rows = 1 if n < 4 else (2 if n < 9 else 4)
    cols = (n + rows - 1) // rows
    dead = np.zeros(rows * cols, dtype=np.uint8)
    dead[n:] = 1
    gates = qs.qs_circuit_generate(rows, cols, 25, cseed, dead)
    h = qs.qs_state_create(n, dtype)
    qs.qs_apply_circuit(h, gates)
    return h


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_noalloc_matches_qs_sample_and_oracle_on_consecutive_calls(dtype):
    import torch
    assert torch.cuda.is_available()
    m = 50000
    # largest state first (its chunk sums fill the scratch exactly), then
    # smaller ones, down to a single partial 256-amplitude chunk
    runs = [(28, 5, 1000), (20, 3, 1001), (16, 8, 77), (7, 2, 5), (3, 4, 9)]
    for n, cseed, seed in runs:
        if n == 28 and dtype == qs.QS_C128:
            continue        # 4 GiB; the complex64 run covers the full scratch
        h = _state(n, dtype, cseed)
        try:
            ref = qs.qs_sample(h, m, seed)
            psi = qs.qs_state_copy_out(h, n, dtype).astype(np.complex128)
            amps = qs.qs_state_amplitudes(h)
            out = torch.empty(m, dtype=torch.int64, device="cuda")
            for call in range(2):
                out.fill_(-1)
                qs.qs_sample_noalloc(n, dtype, amps, m, seed + call, out)
                torch.cuda.synchronize()
                got = out.cpu().numpy().view(np.uint64)
                expect = ref if call == 0 else qs.qs_sample(h, m, seed + call)
                assert np.array_equal(got, expect), (n, call)
                # the oracle's sampler on the same probabilities: identical
                # up to targets that land within rounding of a CDF boundary
                # (complex64: |psi|^2 and the in-chunk prefix sums are FP32,
                # so within 256 2^-22 of a 256-amplitude chunk's mass)
                p = psi.real ** 2 + psi.imag ** 2
                xo = O.sample(p, m, seed + call)
                if dtype == qs.QS_C128:
                    assert np.mean(got != xo) <= 1e-5, (n, call, np.mean(got != xo))
                else:
                    chunk = p.reshape(-1, min(256, p.size)).sum(1).max()
                    _justified(p, got, seed + call, 256 * 2.0 ** -22 * chunk)
                    assert np.mean(got != xo) <= 0.05, (n, call, np.mean(got != xo))
        finally:
            qs.qs_state_destroy(h)
