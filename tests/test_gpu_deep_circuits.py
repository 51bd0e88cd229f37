"""The FP64-accurate split format (complex128 on the FP32 pipe) on deep circuits.

Each split update keeps about 48 significant bits (a few units of 2^-48 relative to the
terms of the update, from roundings with no preferred sign; the matrices are carried in
three floats, exactly the FP64 entries), so the error against the FP64 oracle grows like the
square root of the number of gates. These tests run circuits four to ten times deeper
than the 28-qubit depth-40 workload (up to about 9,900 gates) per gate and fused at every
width k = 2..5 on CUDA cores, and hold them to the complex128 bar of max |d amp| <= 1e-12.
A state takes at most 4096 split sweeps between exact values (reset, host copy); past that
budget it runs on FP64 instructions, which the tests check as well.
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


@pytest.fixture(scope="module")
def deep14():
    ops = synth.random_circuit(14, 400, seed=400)
    return ops, oracle.run(14, ops)


@pytest.mark.parametrize("fuse", [0, 2, 3, 4, 5])
def test_deep_14q_depth400_complex128_vs_oracle(qs, deep14, fuse):
    # per gate the 8226 sweeps exceed the split format's budget of 4096 (the run takes FP64
    # instructions); fused, the same gates fit in far fewer split sweeps
    ops, ref = deep14
    st = qs.State(14, "c128")
    st.run_circuit(ops, fuse=fuse, remap=True)
    stats = st.stats()
    got = st.to_numpy()
    err = float(np.max(np.abs(got - ref)))
    print("14 qubits, %d gates, fuse %d: %d sweeps, FP64 fallback %d, max|d amp| = %.3e"
          % (synth.count_gates(ops), fuse, stats["sweeps"], stats["fp64_fallback"], err))
    assert stats["fp64_fallback"] == (1 if stats["sweeps"] > 4096 else 0)
    assert err <= 1e-12
    # the norm moves by at most 2 sum |a_i| |d a_i| <= 2 sqrt(2^n) max |d a_i|
    assert abs(st.norm() - 1) <= 2 * 2 ** (14 / 2) * 1e-12
    st.close()


@pytest.mark.parametrize("fuse", [0, 4])
def test_deep_20q_depth160_complex128_vs_oracle(qs, fuse):
    n = 20
    ops = synth.random_circuit(n, 160, seed=160)
    ref = oracle.run(n, ops)
    st = qs.State(n, "c128")
    st.run_circuit(ops, fuse=fuse, remap=True)
    err = float(np.max(np.abs(st.to_numpy() - ref)))
    print("20 qubits, %d gates, fuse %d: max|d amp| = %.3e" % (synth.count_gates(ops), fuse, err))
    assert err <= 1e-12
    st.close()


def concentrated(rounds):
    # circuit then inverse, repeated: the state returns to |0...0> after every pair, so the
    # largest amplitude is 1 at the end of each round (the hard case for a bound relative to
    # the amplitudes)
    n = 10
    ops = synth.random_circuit(n, 20, seed=10)
    return n, (ops + synth.inverse_ops(ops)) * rounds


def test_deep_concentrated_state_within_the_split_budget(qs):
    # 6 rounds = 3696 split sweeps, under the budget of 4096
    n, seq = concentrated(6)
    st = qs.State(n, "c128")
    st.run_circuit(seq, fuse=0)
    assert st.stats()["fp64_fallback"] == 0
    got = st.to_numpy()
    err = float(np.max(np.abs(got - oracle.run(n, seq))))
    print("10 qubits, %d gates in the split format, concentrated: max|d amp| = %.3e" % (synth.count_gates(seq), err))
    assert err <= 1e-12
    assert abs(got[0] - 1) <= 1e-12
    st.close()


def test_deep_concentrated_state_past_the_budget_takes_fp64(qs):
    # 16 rounds (9856 sweeps) in one run: the state switches to FP64 instructions; after a
    # reset it is back in the split format
    n, seq = concentrated(16)
    st = qs.State(n, "c128")
    st.run_circuit(seq, fuse=0)
    assert st.stats()["fp64_fallback"] == 1
    got = st.to_numpy()
    err = float(np.max(np.abs(got - oracle.run(n, seq))))
    print("10 qubits, %d gates with the FP64 fallback, concentrated: max|d amp| = %.3e"
          % (synth.count_gates(seq), err))
    assert err <= 1e-12
    assert abs(got[0] - 1) <= 1e-12
    st.reset()
    st.run_circuit(seq[:100], fuse=0)
    assert st.stats()["fp64_fallback"] == 0
    st.close()


def test_split_budget_counts_single_gate_calls(qs):
    # qsim_apply_gate spends the same budget: 4096 split sweeps, then FP64 instructions,
    # with the result still matching the oracle
    n = 6
    rng = np.random.default_rng(6)
    st = qs.State(n, "c128")
    psi = oracle.zero_state(n)
    h = oracle.gate_matrix("H")[1]
    for i in range(4200):
        t = int(rng.integers(n))
        st.apply_gate([t], h)
        oracle.apply(psi, n, [t], [], h)
    st.run_circuit([("T", (0,), ())])
    oracle.apply(psi, n, [0], [], oracle.gate_matrix("T")[1])
    assert st.stats()["fp64_fallback"] == 1
    assert np.max(np.abs(st.to_numpy() - psi)) <= 1e-12
    st.close()
