"""Full-size parity: the 28- and 32-qubit workloads through the C ABI.

At 28 qubits the FP64 oracle evolves the whole state (about two minutes per circuit on the
host cores), so the GPU results are compared amplitude by amplitude: the 28-qubit depth-40
random circuit per gate and fused, in complex128 (max|d amp| <= 1e-12) and complex64
(max|d amp| <= 1e-6, fidelity >= 1 - 1e-6), and the QFT + depth-30 random recipe through the
tensor-core fused path at 28 qubits. At 32 qubits (32 GiB) the oracle cannot hold the state:
the QFT of a basis state is checked on sampled amplitudes against its closed form
(magnitude 2^-n/2, phase 2 pi x y / 2^n at the bit-reversed index), and the norm by the
FP64 reduction.
"""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N = 28


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


@pytest.fixture(scope="module")
def rqc28():
    ops = synth.random_circuit(N, 40, seed=0)
    assert synth.count_gates(ops) == 1714
    return ops, oracle.run(N, ops)


@pytest.fixture(scope="module")
def qft_rqc28():
    ops = synth.qft_circuit(N) + synth.random_circuit(N, 30, seed=3)
    return ops, oracle.run(N, ops)


def compare(got, ref, chunk=1 << 24):
    """max |got - ref| and the fidelity |<ref|got>|^2 / (<got|got><ref|ref>), chunked."""
    worst, dot, gg, rr = 0.0, 0j, 0.0, 0.0
    for i in range(0, ref.size, chunk):
        g = got[i:i + chunk].astype(np.complex128)
        r = ref[i:i + chunk]
        worst = max(worst, float(np.max(np.abs(g - r))))
        dot += np.vdot(r, g)
        gg += float(np.vdot(g, g).real)
        rr += float(np.vdot(r, r).real)
    return worst, abs(dot) ** 2 / (gg * rr)


def run_gpu(qs, ops, dtype, fuse, merge=False):
    import torch
    st = qs.State(N, dtype)
    st.run_circuit(ops, fuse=fuse, remap=True, merge_diagonals=merge)
    stats = st.stats()
    got = st.to_numpy()
    st.close()
    del st
    torch.cuda.empty_cache()
    return got, stats


@pytest.mark.parametrize("fuse,merge", [(0, False), (0, True), (5, False)])
def test_rqc28_complex128_vs_oracle(qs, rqc28, fuse, merge):
    ops, ref = rqc28
    got, stats = run_gpu(qs, ops, "c128", fuse, merge)
    worst, fid = compare(got, ref)
    assert worst <= 1e-12, worst
    assert fid >= 1 - 1e-12
    assert stats["gates"] == 1714
    if merge:  # the T gates and CZ layers run as table sweeps
        assert stats["diag_sweeps"] > 0 and stats["diag_gates"] > 2 * stats["diag_sweeps"]


@pytest.mark.parametrize("fuse,merge", [(0, False), (0, True), (4, False), (5, False)])
def test_rqc28_complex64_vs_oracle(qs, rqc28, fuse, merge):
    # fuse 4 and 5 run on the tensor cores (3xTF32) with the remap folded into the epilogue
    ops, ref = rqc28
    got, stats = run_gpu(qs, ops, "c64", fuse, merge)
    assert (stats["diag_sweeps"] > 0) == merge
    worst, fid = compare(got, ref)
    assert worst <= 1e-6, worst
    assert fid >= 1 - 1e-6, fid
    if fuse:
        assert stats["fused_blocks"] > 0


@pytest.mark.parametrize("fuse", [4, 5])
def test_qft_plus_random_28q_fused_tensor_cores_vs_oracle(qs, qft_rqc28, fuse):
    ops, ref = qft_rqc28
    got, stats = run_gpu(qs, ops, "c64", fuse)
    worst, fid = compare(got, ref)
    assert stats["fused_blocks"] > 0
    assert worst <= 1e-6, worst
    assert fid >= 1 - 1e-6, fid


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-6)])
def test_qft_plus_random_28q_per_gate_merged_diagonals_vs_oracle(qs, qft_rqc28, dtype, tol):
    # the QFT's controlled-phase ladders share their target: groups of up to 10 qubits
    ops, ref = qft_rqc28
    got, stats = run_gpu(qs, ops, dtype, 0, merge=True)
    worst, fid = compare(got, ref)
    assert stats["diag_sweeps"] > 0
    assert worst <= tol, worst
    assert fid >= 1 - tol, fid


def bitrev(y, n):
    return int(format(y, "0%db" % n)[::-1], 2)


def test_qft32_of_basis_state_closed_form_on_samples(qs):
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << 32) + (2 << 30):
        pytest.skip("needs 34 GiB of free device memory")
    n, x = 32, 0x9E3779B9
    ops = [("X", (q,), ()) for q in range(n) if (x >> q) & 1] + synth.qft_circuit(n)
    st = qs.State(n, "c64")
    st.run_circuit(ops, fuse=5, remap=True)
    assert st.stats()["fused_blocks"] > 0
    assert abs(st.norm() - 1) <= 1e-6
    rng = np.random.default_rng(11)
    idx = [0, (1 << n) - 1] + [int(v) for v in rng.integers(0, 1 << n, size=2000)]
    got = np.array([st.amplitude(i) for i in idx])
    Nn = 1 << n
    ref = np.array([np.exp(2j * math.pi * ((x * bitrev(i, n)) % Nn) / Nn) / math.sqrt(Nn) for i in idx])
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.max(rel) <= 1e-3, np.max(rel)
    fid_s = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert fid_s >= 1 - 1e-6, fid_s
    st.close()
    del st
    torch.cuda.empty_cache()
