"""Dense periodic-boundary circuits on the GPU: per-cycle statistics against
the FP64 oracle and the 4-sigma convergence layer of Fig. pt_depth /
appendix pt_nc, for both evolution forms."""
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


@pytest.mark.parametrize("mode", [qs.QS_MODE_FUSED, qs.QS_MODE_PLAIN])
@pytest.mark.parametrize("rows,cols,seed", [(4, 4, 0), (4, 4, 5), (4, 6, 1)])
def test_dense_cycle_statistics_and_convergence(mode, rows, cols, seed):
    n = rows * cols
    layers = 20
    g = qs.qs_circuit_generate_dense(rows, cols, layers, seed)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        st = qs.qs_cycle_statistics(h, g, kmax=3, mode=mode)
    finally:
        qs.qs_state_destroy(h)
    ref = O.cycle_statistics(n, g, kmax=3)
    assert st.shape == ref.shape
    assert np.array_equal(st[:, 0], ref[:, 0])
    assert np.allclose(st[:, 2], ref[:, 2], rtol=1e-6, atol=1e-6)      # entropy
    assert np.allclose(st[:, 4:], ref[:, 4:], rtol=1e-5)               # moments
    # convergence layer: entropies after each layer's CZ cycle
    e_gpu = st[st[:, 0] % 2 == 0][:, 2]
    e_ref = ref[ref[:, 0] % 2 == 0][:, 2]
    i_gpu = qs.qs_pt_convergence(e_gpu, n)
    i_ref = O.pt_convergence_index(list(e_ref), n)
    if i_gpu != i_ref:
        # only an entropy within rounding of the 4-sigma edge may flip it
        edge = 4 * 0.75 * 2 ** (-n / 2)
        h_pt = n * math.log(2) - 1 + O.EULER_GAMMA
        for i in range(min(i_gpu, i_ref), max(i_gpu, i_ref)):
            assert abs(abs(e_ref[i] - h_pt) - edge) < 1e-5
