"""Partial amplitude mode (Section 2.2, Eq. 4) on the GPU against the FP64 oracle.

Small circuits: every amplitude against the oracle's full-state simulation (complex128
within 1e-12, complex64 within 1e-6). A 40-qubit circuit (two 20-qubit blocks, five gates
across the line): sampled amplitudes against the oracle's own partial-mode recombination,
which never holds the 2^40 state.
"""

import numpy as np
import pytest

import oracle
import synth

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


TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.mark.parametrize("n,depth,cross,cut,dtype,fuse", [
    (10, 6, 4, 0, "c128", 0), (12, 5, 5, 7, "c128", 4), (14, 6, 3, 0, "c64", 5), (16, 4, 6, 0, "c64", 0),
    (16, 5, 2, 6, "c128", 5), (13, 4, 0, 0, "c64", 4)])
def test_partial_all_amplitudes_vs_full_oracle(qs, n, depth, cross, cut, dtype, fuse):
    ops = synth.partial_circuit(n, depth, cross, seed=n + cross, cut=cut or None)
    ref = oracle.run(n, ops)
    got, info = qs.qsim_partial_amplitudes(n, ops, np.arange(1 << n, dtype=np.uint64), cut=cut, dtype=dtype,
                                           fuse=fuse, remap=True)
    assert info["decomposed"] == cross and info["subcircuits"] == 2 ** (cross + 1)
    assert np.max(np.abs(got - ref)) <= TOL[dtype], np.max(np.abs(got - ref))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_partial_multi_controlled_crossings_vs_oracle(qs, dtype):
    n = 10
    ops = synth.partial_circuit(n, 3, 1, 9)
    ops += [("TOFFOLI", (0, 2, 7), ()), ("TOFFOLI", (1, 6, 3), ()), ("TOFFOLI", (4, 8, 2), ()),
            ("CONTROL", (1,), ()), ("ISWAP", (5, 9), ()), ("RX", (6,), (0.3,)), ("ENDCONTROL", (), ()),
            ("CONTROL", (7,), ()), ("CNOT", (0, 3), ()), ("ENDCONTROL", (), ())]
    ops += synth.partial_circuit(n, 2, 2, 10)
    ref = oracle.run(n, ops)
    got, info = qs.qsim_partial_amplitudes(n, ops, np.arange(1 << n, dtype=np.uint64), dtype=dtype, fuse=4)
    assert info["decomposed"] == 9
    assert np.max(np.abs(got - ref)) <= TOL[dtype]


@pytest.mark.parametrize("dtype,fuse", [("c64", 5), ("c128", 0)])
def test_partial_40_qubits_sampled_vs_oracle_partial(qs, dtype, fuse):
    n, cut = 40, 20
    ops = synth.partial_circuit(n, 4, 5, seed=40)
    rng = np.random.default_rng(5)
    xs = np.concatenate([[0, (1 << n) - 1], rng.integers(0, 1 << n, size=300, dtype=np.uint64)]).astype(np.uint64)
    ref = oracle.partial_amplitudes(n, ops, xs, cut=cut)
    got, info = qs.qsim_partial_amplitudes(n, ops, xs, cut=cut, dtype=dtype, fuse=fuse, remap=True)
    assert info["decomposed"] == 5 and info["slots"] == 6
    # amplitudes are ~2^-20: the sampled mean |d|^2 times 2^40 estimates the squared error
    # norm of the whole state, held to the same bound as the small cases
    d = np.abs(got - ref)
    assert np.sqrt(np.mean(d ** 2) * 2.0 ** n) <= TOL[dtype], np.sqrt(np.mean(d ** 2) * 2.0 ** n)
    assert np.max(d) <= 10 * TOL[dtype] * 2.0 ** (-n / 2)
    assert np.sqrt(np.mean(np.abs(ref) ** 2) * 2.0 ** n) == pytest.approx(1.0, rel=0.25)


def test_partial_rejections(qs):
    with pytest.raises(qs.QsimError):
        qs.qsim_partial_amplitudes(6, [("H", (0,), ()), ("SWAP", (1, 5), ())], [0])
    with pytest.raises(qs.QsimError):
        qs.qsim_partial_amplitudes(6, [("H", (0,), ())], [1 << 6])
    got, info = qs.qsim_partial_amplitudes(6, [("H", (0,), ())], [])
    assert got.size == 0 and info["decomposed"] == 0


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_partial_smallest_split_vs_oracle(qs, dtype):
    # two 1-qubit blocks joined by a CNOT and a CR (the smallest cut), all four amplitudes
    ops = [("H", (0,), ()), ("RY", (1,), (0.4,)), ("CNOT", (0, 1), ()), ("T", (1,), ()), ("CR", (1, 0), (0.7,)),
           ("H", (1,), ())]
    ref = oracle.run(2, ops)
    got, info = qs.qsim_partial_amplitudes(2, ops, np.arange(4, dtype=np.uint64), dtype=dtype)
    assert info["cut"] == 1 and info["decomposed"] == 2
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
