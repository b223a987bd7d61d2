"""Single-error sweep on the GPU (Fig. 1error, Figs. zcorr / xcorr): one
batch instance per error location, correlations with the ideal output and
the error-averaged distribution against the FP64 oracle."""
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


def test_single_error_sweep_matches_oracle():
    rows, cols, depth = 3, 4, 16
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 8)
    locs = [(c, q, pauli) for c in range(depth + 1) for q in range(n) for pauli in (1, 3)]
    lists = [qs.qs_single_error_circuit(g, n, c, q, pauli) for c, q, pauli in locs]
    b = qs.qs_batch_create([n] * len(lists))
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        qs.qs_batch_run(b, lists, kmax=0)
        qs.qs_apply_circuit(h, g)
        corr = qs.qs_batch_correlation(b, h)
        avg = qs.qs_batch_mean_probabilities(b, n)
    finally:
        qs.qs_batch_destroy(b)
        qs.qs_state_destroy(h)
    p = O.probabilities(O.simulate(n, g))
    acc = np.zeros(1 << n)
    for i, (c, q, pauli) in enumerate(locs):
        pe = O.probabilities(O.simulate(n, O.single_error_circuit(g, c, q, pauli)))
        acc += pe
        assert abs(corr[i] - O.pearson(p, pe)) < 2e-5, (c, q, pauli, corr[i])
    assert np.allclose(avg, acc / len(locs), rtol=2e-5, atol=1e-12)
    # the appendix's exact cases: Z at the end, X after the H layer
    for i, (c, q, pauli) in enumerate(locs):
        if (pauli == 3 and c == depth) or (pauli == 1 and c == 0):
            assert corr[i] > 1 - 1e-5
