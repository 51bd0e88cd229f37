"""The allocation-free PMEASURE entry point against the regular one (GPU).

qsim_probabilities_noalloc serves callers that cannot allocate device memory when they
need the read-out (graph capture, no device synchronisation allowed, fixed memory
budgets): its scratch is a fixed device array inside the library. This file is collected
last so that a run stopping at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


def noalloc(qs, st, qubits):
    import torch
    out = torch.full((1 << len(qubits),), -1.0, dtype=torch.float64, device="cuda")
    q = np.array(qubits, dtype=np.int32)
    rc = qs.lib().qsim_probabilities_noalloc(
        ctypes.c_void_p(st.tensor.data_ptr()), st.n, st.dtype, q.ctypes.data_as(ctypes.c_void_p),
        len(qubits), ctypes.c_void_p(out.data_ptr()), st.stream)
    qs._check(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_matches_regular_probabilities_twice(qs, dtype):
    rng = np.random.default_rng(4242)
    n = 15
    for call, qubits in enumerate(([14, 0, 7], [1, 3, 5, 7, 9, 11, 13, 0, 2, 4])):
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        psi /= np.linalg.norm(psi)
        st = qs.State(n, dtype)
        st.from_numpy(psi)  # identity layout: array bit positions are the qubit numbers
        ref = st.probabilities(qubits)
        got = noalloc(qs, st, qubits)
        assert np.max(np.abs(got - ref)) <= 1e-13, (call, qubits)
        st.close()


def test_noalloc_rejects_too_many_qubits(qs):
    st = qs.State(12, "c64")
    q = np.arange(11, dtype=np.int32)
    import torch
    out = torch.zeros(1 << 11, dtype=torch.float64, device="cuda")
    rc = qs.lib().qsim_probabilities_noalloc(
        ctypes.c_void_p(st.tensor.data_ptr()), 12, st.dtype, q.ctypes.data_as(ctypes.c_void_p), 11,
        ctypes.c_void_p(out.data_ptr()), st.stream)
    assert rc == 1
    assert "at most 10" in qs.qsim_last_error()
