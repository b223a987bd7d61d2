"""qs_sample_noalloc: the sampler variant that allocates no memory.

It exists for callers that cannot allocate device memory while they run (for
example code recording a CUDA graph, or a host application that gives all
GPU memory to its own pool).  Its scratch is a fixed 8 MiB array compiled
into the library, so it only takes states of up to 28 qubits.  Its samples
must equal qs_sample's for the same state and seed, call after call, even
though every call reuses the same scratch array.

This file is named to be collected last.
"""
import numpy as np
import pytest

import paper_1608_00263_gb300 as qs
from paper_1608_00263_gb300 import _native
from paper_1608_00263_gb300 import build as qs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    qs_build.build()
    return _native.lib()


def test_noalloc_rejects_more_than_28_qubits_before_any_device_work():
    # the size check comes first, so this runs without a GPU; the pointers
    # are never dereferenced
    with pytest.raises(qs.QSError) as e:
        qs.qs_sample_noalloc(29, qs.QS_C64, 1 << 20, 10, 1, 1 << 21)
    assert e.value.status == _native.QS_ERR_INVALID_ARG
    assert "28" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_noalloc_matches_qs_sample_on_consecutive_calls(dtype):
    import torch
    assert torch.cuda.is_available()
    m = 50000
    runs = [(20, (4, 5, 25, 3), 1000), (16, (4, 4, 30, 8), 77)]   # large state first, then small
    for n, (rows, cols, depth, cseed), seed in runs:
        gates = qs.qs_circuit_generate(rows, cols, depth, cseed)
        h = qs.qs_state_create(n, dtype)
        try:
            qs.qs_apply_circuit(h, gates)
            ref = qs.qs_sample(h, m, seed)
            amps = qs.qs_state_amplitudes(h)
            out = torch.empty(m, dtype=torch.int64, device="cuda")
            for call in range(2):
                out.fill_(-1)
                qs.qs_sample_noalloc(n, dtype, amps, m, seed + call, out)
                torch.cuda.synchronize()
                expect = ref if call == 0 else qs.qs_sample(h, m, seed + call)
                assert np.array_equal(out.cpu().numpy().view(np.uint64), expect), (n, call)
        finally:
            qs.qs_state_destroy(h)
