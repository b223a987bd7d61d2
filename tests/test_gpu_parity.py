"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: state L2 error relative to the oracle <= 1e-5 for complex64
paths and <= 1e-12 for complex128; entropy and cross entropy within 1e-6
relative; samples identical to the oracle's for complex128 (up to 1e-5 m
boundary cases), and for complex64 every sample must satisfy the oracle's
CDF-inversion condition within the CDF error bound.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native
from paper_1608_00263_gb300 import build as qs_build

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C64: 1e-5, qs.QS_C128: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return _native.lib()


def gpu_run(n, gates, dtype, mode=qs.QS_MODE_FUSED, tile=0):
    h = qs.qs_state_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, gates, mode=mode, tile_log2=tile)
        return qs.qs_state_copy_out(h, n, dtype)
    finally:
        qs.qs_state_destroy(h)


def rel_l2(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b) / np.linalg.norm(b))


def random_gates(rng, n, count):
    g = np.zeros(count, dtype=qs.GATE_DTYPE)
    for i in range(count):
        k = int(rng.integers(0, 9)) if n > 1 else int(rng.choice([0, 1, 2, 3, 5, 6, 7]))
        g[i]["kind"] = k
        if k in (qs.QS_CZ, qs.QS_CPHASE):
            a, b = rng.choice(n, size=2, replace=False)
            g[i]["q0"], g[i]["q1"] = a, b
        else:
            g[i]["q0"] = rng.integers(0, n)
        g[i]["theta"] = rng.uniform(-3, 3)
    return g


# --------------------------------------------------------------------------
# state evolution
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [1, 3, 12, 20])
def test_create_is_basis_zero(dtype, n):
    h = qs.qs_state_create(n, dtype)
    try:
        psi = qs.qs_state_copy_out(h, n, dtype)
    finally:
        qs.qs_state_destroy(h)
    ref = np.zeros(1 << n)
    ref[0] = 1
    assert np.array_equal(psi, ref)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [1, 2, 3, 6, 12, 15])
def test_plain_random_gates(dtype, n):
    rng = np.random.default_rng(7 * n + dtype)
    g = random_gates(rng, n, 150)
    ref = O.simulate(n, g)
    psi = gpu_run(n, g, dtype, mode=qs.QS_MODE_PLAIN)
    assert rel_l2(psi, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n,tile", [(4, 0), (5, 0), (6, 0), (9, 0), (13, 0), (14, 0),
                                    (16, 9), (17, 12), (18, 0)])
def test_fused_random_gates(dtype, n, tile):
    rb = 5 if dtype == qs.QS_C64 else 4
    if tile and not (rb <= tile <= rb + 8):
        pytest.skip("tile outside the kernel's range")
    rng = np.random.default_rng(11 * n + dtype)
    g = random_gates(rng, n, 250)
    ref = O.simulate(n, g)
    psi = gpu_run(n, g, dtype, tile=tile)
    assert rel_l2(psi, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("mode", [qs.QS_MODE_PLAIN, qs.QS_MODE_FUSED])
@pytest.mark.parametrize("seed", [0, 1])
def test_grid_4x5_depth25(dtype, mode, seed):
    g = qs.qs_circuit_generate(4, 5, 25, seed)
    ref = O.simulate(20, g)
    psi = gpu_run(20, g, dtype, mode=mode)
    assert rel_l2(psi, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_fused_t_valued_phases(dtype):
    """Phases equal to the T phase e^{i pi/4} on one or two qubits (RZ(pi/4),
    CPHASE(pi/4)) next to H, T and CZ: the staged T form on one register bit
    and the general form on two."""
    n = 12
    rng = np.random.default_rng(3)
    g = np.zeros(400, dtype=qs.GATE_DTYPE)
    for i in range(400):
        k = [qs.QS_H, qs.QS_T, qs.QS_CZ, qs.QS_RZ, qs.QS_CPHASE, qs.QS_X_HALF][i % 6]
        g[i]["kind"] = k
        a, b = rng.choice(n, size=2, replace=False)
        g[i]["q0"], g[i]["q1"] = a, b
        g[i]["theta"] = math.pi / 4
    ref = O.simulate(n, g)
    assert rel_l2(gpu_run(n, g, dtype), ref) < TOL[dtype]


def test_grid_4x6_depth30_c64():
    g = qs.qs_circuit_generate(4, 6, 30, 5)
    ref = O.simulate(24, g)
    for mode in (qs.QS_MODE_PLAIN, qs.QS_MODE_FUSED):
        assert rel_l2(gpu_run(24, g, qs.QS_C64, mode=mode), ref) < 1e-5


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_leading_hadamard_layer_only_from_basis_zero(dtype):
    """A circuit opening with H on every qubit is written as the uniform
    state only when the state is |0...0>: a second apply, an explicit reset,
    a reset after the caller took the pointer, and a reset that is read
    before any apply all give the oracle's result."""
    n = 12
    g = qs.qs_circuit_generate(3, 4, 10, 3)
    perm = g.copy()
    perm[:n] = g[:n][::-1]                      # the H layer in another qubit order
    h = qs.qs_state_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, g)
        qs.qs_apply_circuit(h, perm)             # not from |0...0>: no fold
        ref2 = O.simulate(n, np.concatenate([g, perm]))
        assert rel_l2(qs.qs_state_copy_out(h, n, dtype), ref2) < TOL[dtype]
        qs.qs_state_reset(h)
        host = np.empty(1 << n, dtype=np.float64)
        qs.qs_probabilities(h, host, fp64=True)  # a deferred reset is written before the read
        assert host[0] == 1 and np.count_nonzero(host) == 1
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, perm)
        assert rel_l2(qs.qs_state_copy_out(h, n, dtype), O.simulate(n, perm)) < TOL[dtype]
        # every form starts from the uniform fill (the old contents are not used)
        modes = [qs.QS_MODE_PLAIN, qs.QS_MODE_FUSED] + ([qs.QS_MODE_FUSED_TC] if dtype == qs.QS_C64 else [])
        ref = O.simulate(n, g)
        for md in modes:
            qs.qs_state_reset(h)
            qs.qs_apply_circuit(h, g, mode=md)
            assert rel_l2(qs.qs_state_copy_out(h, n, dtype), ref) < TOL[dtype], md
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g[:n])            # the layer alone: exactly uniform
        psi = qs.qs_state_copy_out(h, n, dtype)
        assert np.allclose(psi, 2.0 ** (-n / 2), rtol=1e-6, atol=0)
        qs.qs_state_amplitudes(h)                # the caller can now write the memory
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g)
        assert rel_l2(qs.qs_state_copy_out(h, n, dtype), O.simulate(n, g)) < TOL[dtype]
    finally:
        qs.qs_state_destroy(h)


@pytest.mark.parametrize("dtype,mode,n,tile", [(qs.QS_C64, qs.QS_MODE_FUSED, 20, 0), (qs.QS_C64, qs.QS_MODE_FUSED, 16, 9),
                                              (qs.QS_C128, qs.QS_MODE_FUSED, 20, 0),
                                              (qs.QS_C64, qs.QS_MODE_FUSED_TC, 20, 0)])
def test_leading_layer_generated_by_the_first_pass_is_exact(dtype, mode, n, tile):
    """Applied to |0...0> in one call, a circuit's leading Hadamard layer is
    generated by the first fused pass in shared memory (the state is not
    written first); applied alone it is a uniform fill.  Both give the same
    state bit for bit, and the oracle's.  (A Y^1/2 on every qubit after the
    layer leaves no diagonal prefix to fold.)"""
    rows, cols = (4, n // 4)
    g0 = qs.qs_circuit_generate(rows, cols, 20, 7)
    yh = np.zeros(n, dtype=qs.GATE_DTYPE)
    yh["kind"], yh["q0"] = qs.QS_Y_HALF, np.arange(n)
    g = np.concatenate([g0[:n], yh, g0[n:]])
    h = qs.qs_state_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, g, mode=mode, tile_log2=tile)
        one = qs.qs_state_copy_out(h, n, dtype)
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g[:n], mode=mode, tile_log2=tile)     # the fill
        qs.qs_apply_circuit(h, g[n:], mode=mode, tile_log2=tile)
        two = qs.qs_state_copy_out(h, n, dtype)
    finally:
        qs.qs_state_destroy(h)
    assert np.array_equal(one, two)
    assert rel_l2(one, O.simulate(n, g)) < (1e-5 if dtype == qs.QS_C64 else 1e-12)


@pytest.mark.parametrize("dtype,n,tile,mixed", [(qs.QS_C64, 20, 0, False), (qs.QS_C64, 16, 9, False),
                                                (qs.QS_C64, 12, 0, True), (qs.QS_C64, 13, 13, False),
                                                (qs.QS_C128, 20, 0, False), (qs.QS_C128, 12, 0, True)])
def test_diagonal_prefix_folded_into_the_first_pass(dtype, n, tile, mixed):
    """After the leading Hadamard layer, the T and CZ gates that reach the
    uniform state before any non-diagonal gate on their qubits are formed as
    its phases by the first fused pass instead of running as ops: the state
    matches the oracle's, and the unfolded evolution (the layer applied
    alone, then the rest) to rounding.  `mixed`: a random gate mix after the
    layer (repeated T on a qubit, cancelling CZ pairs, RZ and CPHASE left in
    the list, the full interpreter)."""
    rng = np.random.default_rng(300 + n)
    if mixed:
        layer = np.zeros(n, dtype=qs.GATE_DTYPE)
        layer["kind"], layer["q0"] = qs.QS_H, rng.permutation(n)
        pre = np.zeros(6, dtype=qs.GATE_DTYPE)
        pre["kind"] = [qs.QS_T, qs.QS_T, qs.QS_T, qs.QS_CZ, qs.QS_CZ, qs.QS_T]
        pre["q0"] = [0, 0, 1, 2, 2, 3]
        pre["q1"] = [0, 0, 0, 3, 3, 0]
        g = np.concatenate([layer, pre, random_gates(rng, n, 80)])
    else:
        g = qs.qs_circuit_generate(4, n // 4, 16, 11) if n % 4 == 0 else qs.qs_circuit_generate(1, n, 16, 11)
    assert bench_fold(g[n:]) > 0
    ref = O.simulate(n, g)
    h = qs.qs_state_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED, tile_log2=tile)
        one = qs.qs_state_copy_out(h, n, dtype)
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g[:n], mode=qs.QS_MODE_FUSED, tile_log2=tile)
        qs.qs_apply_circuit(h, g[n:], mode=qs.QS_MODE_FUSED, tile_log2=tile)
        two = qs.qs_state_copy_out(h, n, dtype)
    finally:
        qs.qs_state_destroy(h)
    assert rel_l2(one, ref) < TOL[dtype]
    assert rel_l2(one, two.astype(np.complex128)) < (5e-6 if dtype == qs.QS_C64 else 1e-13)


def bench_fold(g):
    import bench
    return bench.fold_diagonal_prefix(qs, g)[0]


def test_invalid_gate_launches_nothing():
    n = 10
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        good = qs.qs_circuit_generate(2, 5, 6, 1)
        bad = good.copy()
        bad[-1]["q0"] = 10
        with pytest.raises(qs.QSError) as e:
            qs.qs_apply_circuit(h, bad)
        assert e.value.status == _native.QS_ERR_INVALID_ARG
        psi = qs.qs_state_copy_out(h, n)
        assert psi[0] == 1 and np.count_nonzero(psi) == 1
        qs.qs_apply_circuit(h, good[:0])          # empty gate list is a no-op
        assert qs.qs_state_copy_out(h, n)[0] == 1
    finally:
        qs.qs_state_destroy(h)


def test_attach_torch_tensor():
    import torch
    n = 14
    amps = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    amps[0] = 1
    g = qs.qs_circuit_generate(2, 7, 12, 4)
    h = qs.qs_state_attach(n, qs.QS_C64, amps)
    try:
        qs.qs_apply_circuit(h, g)
        torch.cuda.synchronize()
    finally:
        qs.qs_state_destroy(h)
    psi = amps.cpu().numpy().view(np.complex64)
    assert rel_l2(psi, O.simulate(n, g)) < 1e-5


# --------------------------------------------------------------------------
# statistics, probabilities, sampler, cross entropy
# --------------------------------------------------------------------------
@pytest.fixture(scope="module", params=[qs.QS_C64, qs.QS_C128])
def state20(request):
    dtype = request.param
    g = qs.qs_circuit_generate(4, 5, 25, 0)
    ref = O.simulate(20, g)
    h = qs.qs_state_create(20, dtype)
    qs.qs_apply_circuit(h, g)
    yield dtype, h, ref, O.probabilities(ref)
    qs.qs_state_destroy(h)


def test_probabilities(state20):
    import torch
    dtype, h, ref, p = state20
    tol = 1e-5 if dtype == qs.QS_C64 else 1e-12
    out = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    qs.qs_probabilities(h, out, fp64=True)
    torch.cuda.synchronize()
    pd = out.cpu().numpy()
    assert np.sum(np.abs(pd - p)) < 2 * tol
    # element by element: the read-out forms |psi|^2 of the state it holds
    # (complex64: one FP32 FMA of the products, widened exactly to FP64, so
    # within 2^-22 relative; complex128: FP64 throughout) ...
    psi = qs.qs_state_copy_out(h, 20, dtype).astype(np.complex128)
    pg = psi.real ** 2 + psi.imag ** 2
    rtol = 2.0 ** -22 if dtype == qs.QS_C64 else 1e-15
    assert np.all(np.abs(pd - pg) <= rtol * pg + 1e-300), np.max(np.abs(pd - pg) / pg)
    # ... and each probability differs from the oracle's only by what that
    # amplitude's own error allows: |p - p_ref| <= (2 |psi_ref| + |d|) |d|
    d = np.abs(psi - ref)
    allow = rtol * pg + (2 * np.abs(ref) + d) * d * (1 + 1e-9) + 1e-300
    assert np.all(np.abs(pd - p) <= allow)
    host = np.empty(1 << 20, dtype=np.float64)
    qs.qs_probabilities(h, host, fp64=True)
    assert np.array_equal(host, pd)
    host32 = np.empty(1 << 20, dtype=np.float32)
    qs.qs_probabilities(h, host32, fp64=False)
    assert np.sum(np.abs(host32 - p)) < 1e-5
    # page-locked host output is written by the kernel directly
    pinned = torch.full((1 << 20,), -1.0, dtype=torch.float64).pin_memory()
    qs.qs_probabilities(h, pinned, fp64=True)
    assert np.array_equal(pinned.numpy(), pd)
    pinned32 = torch.full((1 << 20,), -1.0, dtype=torch.float32).pin_memory()
    qs.qs_probabilities(h, pinned32, fp64=False)
    assert np.array_equal(pinned32.numpy(), host32)


def test_probabilities_async_overlaps_next_circuit():
    """Asynchronous read-out to page-locked host memory: each buffer holds the
    probabilities of the state at its call, although the next circuit runs
    while the copy is in flight; a synchronous read-out into the same buffer
    lands after an earlier asynchronous one."""
    import torch
    n = 20
    g1, g2 = qs.qs_circuit_generate(4, 5, 25, 1), qs.qs_circuit_generate(4, 5, 25, 2)
    p1, p2 = O.probabilities(O.simulate(n, g1)), O.probabilities(O.simulate(n, g2))
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        a = torch.full((1 << n,), -1.0, dtype=torch.float64).pin_memory()
        b = torch.full((1 << n,), -1.0, dtype=torch.float32).pin_memory()
        qs.qs_apply_circuit(h, g1)
        qs.qs_probabilities_async(h, a, fp64=True)
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g2)
        qs.qs_probabilities_async(h, b, fp64=False)
        qs.qs_state_sync(h)
        assert np.sum(np.abs(a.numpy() - p1)) < 2e-5
        assert np.sum(np.abs(b.numpy() - p2)) < 2e-5
        ref32 = np.empty(1 << n, dtype=np.float32)
        qs.qs_probabilities(h, ref32, fp64=False)
        assert np.array_equal(b.numpy(), ref32)
        # device and pageable outputs behave as qs_probabilities
        d = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        qs.qs_probabilities_async(h, d, fp64=True)
        pg = np.empty(1 << n, dtype=np.float64)
        qs.qs_probabilities_async(h, pg, fp64=True)
        qs.qs_state_sync(h)
        assert np.array_equal(d.cpu().numpy(), pg)
        assert np.allclose(pg, ref32, rtol=2.0 ** -22, atol=0)
        # async (state of g2) then, after g1, sync into the same buffer
        qs.qs_probabilities_async(h, a, fp64=True)
        qs.qs_state_reset(h)
        qs.qs_apply_circuit(h, g1)
        qs.qs_probabilities(h, a, fp64=True)
        qs.qs_state_sync(h)
        assert np.sum(np.abs(a.numpy() - p1)) < 2e-5
    finally:
        qs.qs_state_destroy(h)


@pytest.mark.parametrize("n", [5, 8, 20])
def test_async_readout_equals_sync_at_every_share(n):
    """The read-out kernel writes a share of the probabilities (whole groups
    of 256 from index 0) into the page-locked host memory itself and the copy
    engine moves the rest: with none, part or all written directly, over
    consecutive calls, the host memory receives exactly what
    qs_probabilities writes (FP64 and FP32 output).  A state of fewer than
    256 amplitudes is never split."""
    import torch
    rng = np.random.default_rng(100 + n)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        assert qs.qs_readout_share(h) == 0.0
        for share in (0.3, 1.0, 0.7, -1.0):
            qs.qs_readout_share(h, share)
            for c in range(2):
                qs.qs_state_reset(h)
                qs.qs_apply_circuit(h, random_gates(rng, n, 40))
                for fp64 in (True, False):
                    dt = torch.float64 if fp64 else torch.float32
                    got = torch.full((1 << n,), -1.0, dtype=dt).pin_memory()
                    qs.qs_probabilities_async(h, got, fp64=fp64)
                    want = np.empty(1 << n, dtype=np.float64 if fp64 else np.float32)
                    qs.qs_probabilities(h, want, fp64=fp64)
                    qs.qs_state_sync(h)
                    assert np.array_equal(got.numpy(), want), (share, c, fp64)
            assert qs.qs_readout_share(h) == max(share, 0.0)
        with pytest.raises(qs.QSError):
            qs.qs_readout_share(h, 1.5)
    finally:
        qs.qs_state_destroy(h)


def test_pt_moments(state20):
    dtype, h, ref, p = state20
    r = qs.qs_pt_moments(h, 10)
    tol = 1e-6 if dtype == qs.QS_C64 else 1e-11
    # the state tolerance (L2 <= TOL) bounds the norm: |S - 1| <= 2 TOL + TOL^2
    assert r["norm"] == pytest.approx(O.norm(p), abs=2.001 * TOL[dtype])
    assert r["entropy"] == pytest.approx(O.entropy(p), rel=tol)
    assert r["uniform_ce"] == pytest.approx(O.uniform_ce(p), rel=tol)
    mo = O.moments(p, 10)
    mtol = 1e-5 if dtype == qs.QS_C64 else 1e-10
    for k in range(10):
        assert r["moments"][k] == pytest.approx(mo[k], rel=mtol), k


def _check_samples_justified(p_oracle, x, seed, bound):
    C = np.cumsum(p_oracle)          # numpy's pairwise sum; bound covers the order
    total = C[-1]
    idx = np.arange(x.size)
    u = np.array([O.sample_uniform(seed, int(j)) for j in idx])
    target = u * total
    lo = np.where(x > 0, C[np.maximum(x.astype(np.int64) - 1, 0)], 0.0)
    hi = C[x.astype(np.int64)]
    ok = (lo - bound <= target) & (target < hi + bound)
    assert ok.all(), np.nonzero(~ok)[0][:10]
    assert (p_oracle[x.astype(np.int64)] > 0).all()


def test_sampler(state20):
    dtype, h, ref, p = state20
    m = 100000
    seed = 1000
    x = qs.qs_sample(h, m, seed)
    xo = O.sample(p, m, seed)
    mismatch = int(np.sum(x != xo))
    if dtype == qs.QS_C128:
        assert mismatch <= max(1, int(1e-5 * m))
        _check_samples_justified(p, x, seed, 1e-12)
    else:
        psi = qs.qs_state_copy_out(h, 20, dtype)
        pg = np.abs(psi.astype(np.complex128)) ** 2
        # the FP32 state's probabilities differ from the exact ones by up to
        # ||pg - p||_1 in total, which bounds the CDF difference: a sample may
        # differ from the oracle's only where u lands within that bound of a
        # boundary; the count itself follows the state's rounding
        bound = np.sum(np.abs(pg - p)) + 1e-12
        assert mismatch <= 0.05 * m
        _check_samples_justified(p, x, seed, bound)
    # into a device buffer too
    import torch
    xd = torch.empty(m, dtype=torch.int64, device="cuda")
    qs.qs_sample(h, m, seed, out=xd)
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy().view(np.uint64), x)


def test_cross_entropy(state20):
    dtype, h, ref, p = state20
    xo = O.sample(p, 100000, 1000)
    ce, dh = qs.qs_cross_entropy(h, xo)
    ce_o, dh_o = O.cross_entropy(p, xo)
    assert ce == pytest.approx(ce_o, rel=1e-6 if dtype == qs.QS_C64 else 1e-12)
    assert dh == pytest.approx(dh_o, abs=2e-5 if dtype == qs.QS_C64 else 1e-10)
    assert abs(dh - 1) < 0.03                      # Eq. ae on ideal samples


def test_cross_entropy_rejects_out_of_range(state20):
    dtype, h, ref, p = state20
    with pytest.raises(qs.QSError) as e:
        qs.qs_cross_entropy(h, np.array([0, 1 << 20], dtype=np.uint64))
    assert e.value.status == _native.QS_ERR_INVALID_ARG


def test_sampler_edge_cases():
    n = 7
    h = qs.qs_state_create(n, qs.QS_C128)
    try:
        # basis state: every sample is index 0
        assert np.array_equal(qs.qs_sample(h, 50, 3), np.zeros(50, dtype=np.uint64))
        # a state with zero entries: never sampled
        v = np.zeros(1 << n, dtype=np.complex128)
        v[[5, 77, 127]] = [0.6, 0.0 + 0.8j, 0.0]
        qs.qs_state_copy_in(h, v)
        x = qs.qs_sample(h, 2000, 9)
        assert set(np.unique(x)) <= {5, 77}
        assert np.array_equal(x, O.sample(np.abs(v) ** 2, 2000, 9))
        # zero state: refused
        qs.qs_state_copy_in(h, np.zeros(1 << n, dtype=np.complex128))
        with pytest.raises(qs.QSError):
            qs.qs_sample(h, 10, 1)
        r = qs.qs_pt_moments(h, 2)
        assert r["norm"] == 0 and math.isinf(r["uniform_ce"])
    finally:
        qs.qs_state_destroy(h)


# --------------------------------------------------------------------------
# full sizes: properties that hold at any size
# --------------------------------------------------------------------------
def inverse_circuit(g):
    inv = g[::-1].copy()
    for x in inv:
        k = int(x["kind"])
        if k == qs.QS_X_HALF:
            x["kind"], x["theta"] = qs.QS_RX, -np.pi / 2
        elif k == qs.QS_Y_HALF:
            x["kind"], x["theta"] = qs.QS_RY, -np.pi / 2
        elif k == qs.QS_T:
            x["kind"], x["theta"] = qs.QS_RZ, -np.pi / 4      # T^dagger up to phase
        elif k in (qs.QS_RX, qs.QS_RY, qs.QS_RZ, qs.QS_CPHASE):
            x["theta"] = -x["theta"]
    return inv


def test_full_size_30_qubits():
    import torch
    n = 30
    g = qs.qs_circuit_generate(5, 6, 40, 0)
    h = qs.qs_state_create(n, qs.QS_C64)
    h2 = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED)
        qs.qs_apply_circuit(h2, g, mode=qs.QS_MODE_PLAIN)
        pa = qs.qs_state_amplitudes(h)
        pb = qs.qs_state_amplitudes(h2)
        # fused vs plain (two independent CUDA paths), on the device
        diff = _device_rel_l2(pa, pb, n)
        assert diff < 1e-5
        # tensor-core form vs plain
        qs.qs_state_reset(h2)
        qs.qs_apply_circuit(h2, g, mode=qs.QS_MODE_FUSED_TC)
        assert _device_rel_l2(pb, pa, n) < 1e-5
        r = qs.qs_pt_moments(h, 10)
        assert abs(r["norm"] - 1) < 1e-5
        N = 2.0 ** n
        sigma = 0.75 * 2.0 ** (-n / 2)
        assert abs(r["entropy"] - (n * math.log(2) - 1 + O.EULER_GAMMA)) < 4 * sigma
        assert abs(r["uniform_ce"] - (n * math.log(2) + O.EULER_GAMMA)) < 5 * math.sqrt(1.645 / N)
        assert abs(r["moments"][1] - 2) < 0.01
        x = qs.qs_sample(h, 1000000, 1000)
        ce, dh = qs.qs_cross_entropy(h, x)
        assert abs(dh - 1) < 4 * 0.8 / 1000 + 0.002
        # time reversal: U^dagger U |0> = |0> up to a global phase
        qs.qs_apply_circuit(h, inverse_circuit(g))
        probs = torch.empty(1 << n, dtype=torch.float32, device="cuda")
        qs.qs_probabilities(h, probs, fp64=False)
        torch.cuda.synchronize()
        assert float(probs[0]) > 1 - 2e-5
        del probs
    finally:
        qs.qs_state_destroy(h)
        qs.qs_state_destroy(h2)


def _device_rel_l2(pa, pb, n):
    """||a - b|| / ||b|| of two complex64 device states, computed with torch
    views of the raw buffers (test-side arithmetic only)."""
    import torch
    N = 1 << n
    ta = _view(pa, 2 * N)
    tb = _view(pb, 2 * N)
    num = den = 0.0
    step = 1 << 26
    for i in range(0, 2 * N, step):
        a, b = ta[i:i + step].double(), tb[i:i + step].double()
        num += float(torch.sum((a - b) ** 2))
        den += float(torch.sum(b ** 2))
    return math.sqrt(num / den)


def _view(ptr, count):
    import torch
    # wrap a raw device pointer as a float32 tensor (no copy)
    class _Arr:
        __cuda_array_interface__ = {"shape": (count,), "typestr": "<f4", "data": (ptr, False),
                                    "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


# --------------------------------------------------------------------------
# tensor-core form (FP16x3 block products, FP32 accumulation)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rows,cols,depth,seed", [(4, 4, 40, 0), (4, 5, 25, 1), (3, 5, 30, 2)])
def test_tc_form_vs_oracle(rows, cols, depth, seed):
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, seed)
    st = qs.qs_plan_circuit(n, qs.QS_C64, g, mode=qs.QS_MODE_FUSED_TC)
    ref = O.simulate(n, g)
    psi = gpu_run(n, g, qs.QS_C64, mode=qs.QS_MODE_FUSED_TC)
    assert rel_l2(psi, ref) < 1e-5, st


def test_tc_form_random_gates():
    rng = np.random.default_rng(17)
    n = 15
    # dense random circuits on few qubits give the planner blocks worth taking
    g = random_gates(rng, 6, 400)
    g = np.concatenate([g, random_gates(rng, n, 200)])
    ref = O.simulate(n, g)
    psi = gpu_run(n, g, qs.QS_C64, mode=qs.QS_MODE_FUSED_TC)
    assert rel_l2(psi, ref) < 1e-5


PRECISIONS = [(qs.QS_PREC_FP16X3, 1e-5), (qs.QS_PREC_BF16X6, 1e-5), (qs.QS_PREC_TF32X3, 1e-5),
              (qs.QS_PREC_BF16X3, None), (qs.QS_PREC_TF32, None)]


@pytest.mark.parametrize("prec,tol", PRECISIONS)
@pytest.mark.parametrize("rows,cols,depth,seed", [(4, 5, 25, 1), (4, 6, 30, 5)])
def test_tc_precisions_vs_oracle(prec, tol, rows, cols, depth, seed):
    """Every operand precision of the tensor-core form against the FP64
    oracle: FP16x3, BF16x6 and TF32x3 within the 1e-5 state bound; BF16x3
    (~16 bits) and plain TF32 (~11 bits) are lossy, and their error is only
    reported (and bounded loosely, so that a broken form still fails)."""
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, seed)
    st = qs.qs_plan_circuit(n, qs.QS_C64, g, mode=qs.QS_MODE_FUSED_TC, precision=prec)
    ref = O.simulate(n, g)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED_TC, precision=prec)
        err = rel_l2(qs.qs_state_copy_out(h, n), ref)
    finally:
        qs.qs_state_destroy(h)
    print("tc precision %d, %d qubits: relative L2 error %.3e (%d passes)" % (prec, n, err, st["passes"]))
    assert err < (tol if tol else 5e-2), err


def test_tc_precision_out_of_range_is_rejected():
    g = qs.qs_circuit_generate(3, 5, 10, 0)
    h = qs.qs_state_create(15, qs.QS_C64)
    try:
        with pytest.raises(qs.QSError) as e:
            qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED_TC, precision=6)
        assert e.value.status == _native.QS_ERR_INVALID_ARG
    finally:
        qs.qs_state_destroy(h)


def test_tc_form_24_qubits():
    g = qs.qs_circuit_generate(4, 6, 30, 5)
    ref = O.simulate(24, g)
    assert rel_l2(gpu_run(24, g, qs.QS_C64, mode=qs.QS_MODE_FUSED_TC), ref) < 1e-5


def test_tc_form_rejects_complex128():
    g = qs.qs_circuit_generate(4, 4, 20, 0)
    h = qs.qs_state_create(16, qs.QS_C128)
    try:
        # complex128 plans carry no tensor-core phases: same result as fused
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED_TC)
        psi = qs.qs_state_copy_out(h, 16, qs.QS_C128)
    finally:
        qs.qs_state_destroy(h)
    assert rel_l2(psi, O.simulate(16, g)) < 1e-12


def test_full_size_34_qubits():
    """6x6 grid minus two opposite corners, depth 40, complex64 in place
    (137 GB).  The FP64 oracle would need 275 GB of host memory, so the
    checks are properties that hold at any size."""
    import torch
    torch.cuda.empty_cache()
    n = 34
    dead = O.grid_dead_mask(6, 6, [(0, 0), (5, 5)])
    g = qs.qs_circuit_generate(6, 6, 40, 0, dead)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        # before the first X^1/2 / Y^1/2 the distribution is exactly uniform
        first = next(i for i, x in enumerate(g) if int(x["kind"]) in (qs.QS_X_HALF, qs.QS_Y_HALF))
        qs.qs_apply_circuit(h, g[:first])
        r = qs.qs_pt_moments(h, 4)
        assert abs(r["norm"] - 1) < 1e-5
        assert abs(r["entropy"] - n * math.log(2)) < 1e-6 * n
        assert np.allclose(r["moments"], 1.0, atol=1e-5)
        # the whole circuit: norm and Porter-Thomas entropy (Sec. pt: spread
        # 0.75 2^{-n/2}; the FP32 state adds up to ~5e-5 absolute)
        qs.qs_apply_circuit(h, g[first:])
        r = qs.qs_pt_moments(h, 10)
        assert abs(r["norm"] - 1) < 2e-5
        sigma = 0.75 * 2.0 ** (-n / 2)
        assert abs(r["entropy"] - (n * math.log(2) - 1 + O.EULER_GAMMA)) < 4 * sigma + 5e-5
        assert abs(r["moments"][1] - 2) < 0.01
        x = qs.qs_sample(h, 1000000, 1000)
        ce, dh = qs.qs_cross_entropy(h, x)
        assert abs(dh - 1) < 4 * 0.8 / 1000 + 0.002
        # time reversal through both fused forms: U_tc^dagger ... U |0> = |0>
        qs.qs_apply_circuit(h, inverse_circuit(g), mode=qs.QS_MODE_FUSED_TC)
        qs.qs_apply_circuit(h, g, mode=qs.QS_MODE_FUSED_TC)
        qs.qs_apply_circuit(h, inverse_circuit(g), mode=qs.QS_MODE_FUSED)
        # probability of |0...0>: the first amplitude, read through a view
        t = _view(qs.qs_state_amplitudes(h), 2)
        p0 = float(t[0]) ** 2 + float(t[1]) ** 2
        assert p0 > 1 - 1e-4, p0
    finally:
        qs.qs_state_destroy(h)


# --------------------------------------------------------------------------
# statistics after every cycle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [qs.QS_MODE_FUSED, qs.QS_MODE_PLAIN])
def test_cycle_statistics_vs_oracle(mode):
    n = 16
    g = qs.qs_circuit_generate(4, 4, 30, 4)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        st = qs.qs_cycle_statistics(h, g, kmax=3, mode=mode)
    finally:
        qs.qs_state_destroy(h)
    assert st.shape == (31, 7)
    psi = O.zero_state(n)
    for c in range(31):
        O.apply_circuit(psi, g[g["cycle"] == c])
        p = O.probabilities(psi)
        assert st[c, 0] == c
        assert st[c, 2] == pytest.approx(O.entropy(p), rel=1e-6, abs=1e-6)
        assert np.allclose(st[c, 4:], O.moments(p, 3), rtol=1e-5)
    # Sec. pt: the H layer gives the uniform distribution, the first cycles
    # are diagonal, later the entropy approaches ln N - 1 + gamma
    assert st[0, 2] == pytest.approx(n * math.log(2), abs=1e-6)
    assert abs(st[-1, 2] - (n * math.log(2) - 1 + O.EULER_GAMMA)) < 0.01


@pytest.mark.parametrize("dtype,mode", [(qs.QS_C64, qs.QS_MODE_FUSED), (qs.QS_C128, qs.QS_MODE_FUSED),
                                        (qs.QS_C64, qs.QS_MODE_FUSED_TC)])
def test_autotuned_apply_matches_oracle(dtype, mode):
    """qs_opts.autotune = 1: the library times the candidate forms on a
    scratch copy and applies the circuit with the fastest; the result is the
    oracle's, the state's own contents before the call are respected (two
    circuits in a row), and a second call reuses the cached choice."""
    n = 16
    g1 = qs.qs_circuit_generate(4, 4, 20, 3)
    g2 = qs.qs_circuit_generate(4, 4, 12, 4)[16:]          # no leading H layer
    h = qs.qs_state_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, g1, mode=mode, autotune=1)
        qs.qs_apply_circuit(h, g2, mode=mode, autotune=1)
        ref = O.simulate(n, np.concatenate([g1, g2]))
        assert rel_l2(qs.qs_state_copy_out(h, n, dtype), ref) < TOL[dtype]
        with pytest.raises(qs.QSError) as e:
            qs.qs_apply_circuit(h, g2, mode=mode, autotune=1, tile_log2=10)
        assert e.value.status == _native.QS_ERR_INVALID_ARG
    finally:
        qs.qs_state_destroy(h)
