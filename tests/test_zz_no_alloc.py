"""The allocation-free PMEASURE entry point against the regular one (GPU).

qsim_probabilities_noalloc serves callers that cannot allocate device memory when they
need the read-out (no device synchronisation allowed, fixed memory budgets): its scratch is a fixed device array inside the library. This file is collected
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


def test_noalloc_smaller_call_after_a_larger_one(qs):
    # the shared scratch keeps the previous call's partial histograms: a call with fewer
    # blocks and fewer bins after a wide one must not read any of them
    rng = np.random.default_rng(4243)
    for n, qubits in ((15, [1, 3, 5, 7, 9, 11, 13, 0, 2, 4]), (9, [8, 2]), (15, [6])):
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        psi /= np.linalg.norm(psi)
        st = qs.State(n, "c128")
        st.from_numpy(psi)
        got = noalloc(qs, st, qubits)
        assert np.max(np.abs(got - st.probabilities(qubits))) <= 1e-13, (n, qubits)
        st.close()


@pytest.mark.parametrize("dtype,fuse,tol", [("c128", 4, 1e-12), ("c64", 5, 1e-6)])
def test_noalloc_after_a_fused_circuit_and_canonicalize_vs_oracle(qs, dtype, fuse, tol):
    # the documented path for a library state: a fused circuit leaves a complex128 state in
    # the split format, a complex64 state (tensor-core path) in a permuted qubit layout;
    # qsim_canonicalize restores plain amplitudes in logical order, and the allocation-free
    # read-out then matches the FP64 oracle
    import oracle
    import synth
    n = 14
    ops = synth.random_circuit(n, 12, seed=14)
    st = qs.State(n, dtype)
    st.run_circuit(ops, fuse=fuse, remap=True)
    stats = st.stats()
    assert stats["fused_blocks"] > 0
    if dtype == "c64":
        assert stats["epilogue_remaps"] + stats["remaps"] > 0
    st.canonicalize()
    ref_state = oracle.run(n, ops)
    for qubits in ([0, 13, 6], [12, 1, 4, 9, 3], [7]):
        got = noalloc(qs, st, qubits)
        ref = oracle.probabilities(ref_state, n, qubits)
        assert np.max(np.abs(got - ref)) <= tol, qubits
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
