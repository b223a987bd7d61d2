"""Batched ensemble (qs_batch_*): every instance against the FP64 oracle on
a small ensemble, and the full 4096-instance ensemble (n 12..24, depth
10..40) against properties and Porter-Thomas closed forms."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native as N
from paper_1608_00263_gb300 import build as qs_build

from seeded_inputs import ensemble_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    import torch
    assert torch.cuda.is_available()


def instance(s):
    n, depth, rows, cols, dead = ensemble_instance(s)
    g = qs.qs_circuit_generate(rows, cols, depth, s, np.array(dead, dtype=np.uint8))
    return n, depth, g


def device_state(b, i, n):
    import torch
    ptr = qs.qs_batch_state(b, i)

    class _A:
        __cuda_array_interface__ = {"shape": (2 << n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_A(), device="cuda").cpu().numpy().view(np.complex64)


def test_small_ensemble_matches_oracle():
    seeds = [s for s in range(200) if ensemble_instance(s)[0] <= 17][:24]
    inst = [instance(s) for s in seeds]
    b = qs.qs_batch_create([x[0] for x in inst])
    try:
        st = qs.qs_batch_run(b, [x[2] for x in inst], kmax=4)
        st2 = qs.qs_batch_run(b, [x[2] for x in inst], kmax=4)      # graph replay
        assert np.array_equal(st, st2)
        for i, (n, depth, g) in enumerate(inst):
            ref = O.simulate(n, g)
            psi = device_state(b, i, n)
            err = np.linalg.norm(psi.astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (i, n, depth, err)
            p = O.probabilities(ref)
            assert abs(st[i, 0] - 1) < 2e-5
            assert st[i, 1] == pytest.approx(O.entropy(p), rel=1e-6)
            assert st[i, 2] == pytest.approx(O.uniform_ce(p), rel=1e-6)
            assert np.allclose(st[i, 3:], O.moments(p, 4), rtol=1e-5)
    finally:
        qs.qs_batch_destroy(b)


def test_batch_initial_states_with_and_without_hadamard_layer():
    """Instances opening with H on every qubit start from the uniform state
    (Sec. pt, cycle 0) and plan the rest; the others start from |0...0>:
    a list that is only the layer, a layer missing one qubit, a layer after a
    T gate, a layer with a repeated qubit, and the empty list."""
    n = 12
    g = qs.qs_circuit_generate(3, 4, 10, 3)
    assert np.all(g["kind"][:n] == qs.QS_H)
    t0 = g[n:n + 1].copy()
    t0["kind"], t0["q0"], t0["theta"] = qs.QS_T, 5, 0.0
    dup = g.copy()
    dup["q0"][1] = dup["q0"][0]
    lists = [g, g[:n], g[1:], np.concatenate([t0, g]), dup, g[:0]]
    b = qs.qs_batch_create([n] * len(lists))
    try:
        for rep in range(2):                                       # capture, then replay
            qs.qs_batch_apply(b, lists)
            for i, gl in enumerate(lists):
                ref = O.simulate(n, gl)
                psi = device_state(b, i, n)
                err = np.linalg.norm(psi.astype(complex) - ref) / np.linalg.norm(ref)
                assert err < 1e-5, (rep, i, err)
    finally:
        qs.qs_batch_destroy(b)


def test_ensemble_4096():
    import torch
    torch.cuda.empty_cache()
    inst = [instance(s) for s in range(4096)]
    ns = np.array([x[0] for x in inst])
    depths = np.array([x[1] for x in inst])
    b = qs.qs_batch_create(ns)
    try:
        st = qs.qs_batch_run(b, [x[2] for x in inst], kmax=10)
        # every state normalised to the FP32 evolution's accuracy
        assert np.max(np.abs(st[:, 0] - 1)) < 2e-5
        # deep instances: entropy and moments at their Porter-Thomas values
        # (Sec. "Convergence to Porter-Thomas": convergence within ~10 cycles
        # for the paper's grids; spread 0.75 2^{-n/2} between states)
        deep = depths >= 30
        assert deep.sum() > 1000
        pt = ns * math.log(2) - 1 + O.EULER_GAMMA
        z = (st[:, 1] - pt) / (0.75 * 2.0 ** (-ns / 2))
        assert np.mean(np.abs(z[deep]) < 4) > 0.95, np.percentile(np.abs(z[deep]), [50, 90, 99])
        ipr2 = st[:, 4]
        assert abs(np.mean(ipr2[deep]) - 2) < 0.02
        ce_pt = ns * math.log(2) + O.EULER_GAMMA
        assert abs(np.mean(st[deep, 2] - ce_pt[deep])) < 0.01
        # a random subset of the small instances against the oracle
        rng = np.random.default_rng(1)
        small = np.nonzero(ns <= 16)[0]
        for i in rng.choice(small, size=8, replace=False):
            n, depth, g = inst[i]
            p = O.probabilities(O.simulate(n, g))
            assert st[i, 1] == pytest.approx(O.entropy(p), rel=1e-6)
    finally:
        qs.qs_batch_destroy(b)


def test_autotuned_ensemble_matches_oracle_and_reports_its_choices():
    """qs_batch_set_options(autotune=1): the tile size per instance size is
    chosen by timing the batch's own rounds (9..13 qubits, at most n); the
    run still matches the oracle instance by instance, every instance of one
    size uses the same tile, and the run reports its algorithmic bytes."""
    seeds = [s for s in range(300) if ensemble_instance(s)[0] <= 16][:20]
    inst = [instance(s) for s in seeds]
    b = qs.qs_batch_create([x[0] for x in inst])
    try:
        with pytest.raises(qs.QSError):
            qs.qs_batch_plan_info(b)                     # nothing prepared yet
        with pytest.raises(qs.QSError):
            qs.qs_batch_set_options(b, mode=qs.QS_MODE_FUSED_TC)
        with pytest.raises(qs.QSError):
            qs.qs_batch_set_options(b, tile_log2=14)
        qs.qs_batch_set_options(b, autotune=1)
        st = qs.qs_batch_run(b, [x[2] for x in inst], kmax=2)
        tiles, run_bytes = qs.qs_batch_plan_info(b)
        by_n = {}
        for i, (n, depth, g) in enumerate(inst):
            assert min(9, n) <= tiles[i] <= min(13, n), (n, tiles[i])
            assert by_n.setdefault(n, tiles[i]) == tiles[i]
            ref = O.simulate(n, g)
            err = np.linalg.norm(device_state(b, i, n).astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (i, n, err)
            assert st[i, 1] == pytest.approx(O.entropy(O.probabilities(ref)), rel=1e-6)
        assert run_bytes >= 16 * sum(1 << x[0] for x in inst)
        # a fixed tile size for every instance
        qs.qs_batch_set_options(b, tile_log2=10)
        qs.qs_batch_run(b, [x[2] for x in inst], kmax=2)
        tiles, _ = qs.qs_batch_plan_info(b)
        assert np.all(tiles == 10)
        for i, (n, depth, g) in enumerate(inst[:5]):
            ref = O.simulate(n, g)
            err = np.linalg.norm(device_state(b, i, n).astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (i, n, err)
    finally:
        qs.qs_batch_destroy(b)


def _mixed_instances():
    """5..19 qubits, shallow and deep: with a fixed tile size t < 13 every
    pass runs in thread groups of 2^(t-5) threads (t = 5: one thread, t = 9:
    half a warp, t = 12: four warps); 13-qubit tiles take the whole CTA; 19
    qubits give two 2^18-amplitude work items per pass."""
    out = []
    for k, (n, depth) in enumerate([(19, 12), (5, 8), (12, 20), (9, 16), (17, 3), (14, 25), (6, 10),
                                    (13, 14), (11, 18), (16, 9)]):
        rows = 1 if n < 4 else (2 if n < 9 else 4)
        cols = -(-n // rows)
        dead = np.zeros(rows * cols, dtype=np.uint8)
        dead[n:] = 1
        out.append((n, depth, qs.qs_circuit_generate(rows, cols, depth, 100 + k, dead)))
    return out


@pytest.mark.parametrize("tile", [0, 5, 7, 9, 10, 12])
def test_persistent_and_lockstep_engines_agree_with_each_other_and_the_oracle(tile):
    """The persistent engine (one launch, grouped passes, dependency waits)
    against the lockstep rounds on the same plans: identical states and
    statistics (the same per-tile arithmetic and the same partials summed in
    the same order), and both against the FP64 oracle."""
    inst = _mixed_instances()
    if tile:
        inst = [x for x in inst if x[0] >= tile]
    b = qs.qs_batch_create([x[0] for x in inst])
    try:
        if tile:
            qs.qs_batch_set_options(b, tile_log2=tile)
        gl = [x[2] for x in inst]
        res = {}
        for engine in (qs.QS_BATCH_ROUNDS, qs.QS_BATCH_PERSISTENT):
            qs.qs_batch_set_engine(b, engine)
            st = qs.qs_batch_run(b, gl, kmax=6)
            st2 = qs.qs_batch_run(b, gl, kmax=6)               # graph replay
            assert np.array_equal(st, st2)
            res[engine] = (st, [device_state(b, i, x[0]) for i, x in enumerate(inst)])
        st_r, psi_r = res[qs.QS_BATCH_ROUNDS]
        st_p, psi_p = res[qs.QS_BATCH_PERSISTENT]
        assert np.array_equal(st_r, st_p)
        for i, (n, depth, g) in enumerate(inst):
            assert np.array_equal(psi_r[i], psi_p[i]), (i, n, depth)
            ref = O.simulate(n, g)
            err = np.linalg.norm(psi_p[i].astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (i, n, depth, err)
            p = O.probabilities(ref)
            assert st_p[i, 1] == pytest.approx(O.entropy(p), rel=1e-6)
            assert np.allclose(st_p[i, 3:], O.moments(p, 6), rtol=1e-5)
    finally:
        qs.qs_batch_destroy(b)


def test_engine_choice_is_validated_and_autotuned_per_engine():
    inst = _mixed_instances()[:4]
    b = qs.qs_batch_create([x[0] for x in inst])
    try:
        with pytest.raises(qs.QSError) as e:
            qs.qs_batch_set_engine(b, 2)
        assert e.value.status == N.QS_ERR_INVALID_ARG
        qs.qs_batch_set_engine(b, qs.QS_BATCH_PERSISTENT)
        qs.qs_batch_set_options(b, autotune=1)
        qs.qs_batch_run(b, [x[2] for x in inst], kmax=2)
        tiles, _ = qs.qs_batch_plan_info(b)
        for i, (n, depth, g) in enumerate(inst):
            assert min(9, n) <= tiles[i] <= min(13, n)
            ref = O.simulate(n, g)
            err = np.linalg.norm(device_state(b, i, n).astype(complex) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (i, n, err)
    finally:
        qs.qs_batch_destroy(b)
