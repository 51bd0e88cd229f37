"""GPU parity: the CUDA library through its C ABI against the FP64 oracle.

Tolerances: complex128 states must match the oracle within max|d amp| <= 1e-12, complex64
states within 1e-6 (and fidelity >= 1 - 1e-6 for whole circuits).
"""

import math

import numpy as np
import pytest

import oracle
import synth
from oracle.script import parse_script

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


def rand_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def rand_unitary(d, rng):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def start(qs, n, dtype, rng):
    psi = rand_state(n, rng)
    if dtype == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    st = qs.State(n, dtype)
    st.from_numpy(psi)
    return st, psi.copy()


ONE_Q = ["H", "X", "Y", "Z", "S", "T", "SX", "SY", "RZ", "RY", "GEN"]


def one_q_matrix(name, rng):
    if name == "GEN":
        return rand_unitary(2, rng)
    if name in ("RZ", "RY"):
        return oracle.gate_matrix(name, (rng.uniform(-3, 3),))[1]
    return oracle.gate_matrix(name)[1]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_single_qubit_every_target_and_class(qs, dtype, n):
    rng = np.random.default_rng(1000 + n)
    st, psi = start(qs, n, dtype, rng)
    for t in range(n):
        others = [q for q in range(n) if q != t]
        ctl_sets = [[]]
        if others:
            ctl_sets += [[others[0]], [others[-1]]]
        if len(others) >= 2:
            ctl_sets.append(list(rng.choice(others, size=2, replace=False)))
        for ctl in ctl_sets:
            for name in ONE_Q:
                m = one_q_matrix(name, rng)
                st.apply_gate([t], m, [int(c) for c in ctl])
                oracle.apply(psi, n, [t], [int(c) for c in ctl], m)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - psi)) <= TOL[dtype]


TWO_Q = ["SWAP", "ISWAP", "CZ", "CR", "CNOT", "GEN"]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [2, 4, 7])
def test_two_qubit_every_pair(qs, dtype, n):
    rng = np.random.default_rng(2000 + n)
    st, psi = start(qs, n, dtype, rng)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            others = [q for q in range(n) if q not in (a, b)]
            ctl = [others[(a + b) % len(others)]] if others and (a + 2 * b) % 3 == 0 else []
            for name in TWO_Q:
                m = rand_unitary(4, rng) if name == "GEN" else oracle.gate_matrix(name, (0.7,))[1]
                st.apply_gate([a, b], m, ctl)
                oracle.apply(psi, n, [a, b], ctl, m)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - psi)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_three_qubit_matrix_and_toffoli(qs, dtype):
    rng = np.random.default_rng(3)
    n = 9
    st, psi = start(qs, n, dtype, rng)
    ops = []
    for _ in range(6):
        qs_ = [int(x) for x in rng.choice(n, size=3, replace=False)]
        ops.append(("TOFFOLI", tuple(qs_), ()))
        u = rand_unitary(8, rng)
        qs2 = [int(x) for x in rng.choice(n, size=3, replace=False)]
        ops.append(("MATRIX", tuple(qs2), (), u))
    st.run_circuit(ops)
    for op in ops:
        if op[0] == "TOFFOLI":
            oracle.apply(psi, n, [op[1][2]], list(op[1][:2]), oracle.gate_matrix("X")[1])
        else:
            oracle.apply(psi, n, list(op[1]), [], op[3])
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - psi)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_apply_fused_random_unitaries(qs, dtype, k):
    rng = np.random.default_rng(40 + k)
    n = 13
    st, psi = start(qs, n, dtype, rng)
    for rep in range(4):
        qubits = [int(x) for x in rng.choice(n, size=k, replace=False)]
        if rep == 0:
            qubits = list(range(k))  # the low qubits (tensor-core placement)
        u = rand_unitary(1 << k, rng)
        st.apply_fused(qubits, u)
        oracle.apply(psi, n, qubits, [], u)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - psi)) <= TOL[dtype]


def run_both(qs, n, ops, dtype, **kw):
    st = qs.State(n, dtype)
    st.run_circuit(ops, **kw)
    return st.to_numpy().astype(np.complex128), oracle.run(n, ops), st


@pytest.mark.parametrize("fuse", [0, 2, 3, 4, 5])
def test_random_circuit_12q_depth20_c128(qs, fuse):
    ops = synth.random_circuit(12, 20, seed=0)
    assert synth.count_gates(ops) == 372
    got, ref, st = run_both(qs, 12, ops, "c128", fuse=fuse)
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert st.stats()["gates"] == 372


@pytest.mark.parametrize("fuse", [0, 4, 5])
def test_random_circuit_12q_c64(qs, fuse):
    ops = synth.random_circuit(12, 20, seed=0)
    got, ref, _ = run_both(qs, 12, ops, "c64", fuse=fuse)
    assert np.max(np.abs(got - ref)) <= 1e-6
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_graph_capture_matches_direct(qs, dtype):
    ops = synth.random_circuit(14, 6, seed=9)
    a = qs.State(14, dtype)
    a.run_circuit(ops, fuse=0)
    b = qs.State(14, dtype)
    b.run_circuit(ops, fuse=0, use_graph=True)
    b.reset()
    b.run_circuit(ops, fuse=0, use_graph=True)  # replay of the cached graph
    assert np.array_equal(a.to_numpy(), b.to_numpy())


def test_appendix_a2_example_through_the_abi(qs):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "appendix_a2_example.txt")
    text = open(path).read()
    n, ops, pm, _ = parse_script(text)
    expected = {}
    for line in text.splitlines():
        if line.startswith("#@expected"):
            k, v = line[len("#@expected"):].split(":")
            expected[k.strip()] = float(v)
    for dtype in ("c128", "c64"):
        st = qs.State(n, dtype)
        st.run_circuit(ops)
        probs = st.probabilities(pm)
        for s, p in enumerate(probs):
            assert abs(p - expected[format(s, "03b")]) <= 1e-6


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_readouts_24q_vs_oracle(qs, dtype):
    # 24 qubits: the histogram splits each thread's index range over several blocks (no
    # listed bit or one above the thread bits) or takes it whole; complex64 sums its
    # squares exactly in FP32 pairs, so both formats match the FP64 oracle to 1e-12
    rng = np.random.default_rng(79)
    n = 24
    st, psi = start(qs, n, dtype, rng)
    for qubits in ([0], [23], [5, 3], [23, 0, 17, 5], list(range(14, 24)), [1, 3, 5, 7, 9, 11, 13, 15],
                   [16, 2, 20, 9, 11, 0]):
        got = st.probabilities(qubits)
        ref = oracle.probabilities(psi, n, qubits)
        assert np.max(np.abs(got - ref)) <= 1e-12, qubits
    # the other read-outs at this size: complex64 sums run on the FP32 pipe in exact pairs
    # (per-qubit sums over segments of 4096 amplitudes, two per warp at 24 qubits)
    assert abs(st.norm() - oracle.norm2(psi, n)) <= 1e-12
    assert np.max(np.abs(st.expect_z() - oracle.z_expectations(psi, n))) <= 1e-12
    other, psi2 = start(qs, n, dtype, np.random.default_rng(80))
    assert abs(st.inner(other) - oracle.inner(psi, psi2, n)) <= 1e-12
    other.close()
    st.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_wide_pmeasure_vs_oracle(qs, dtype):
    # twelve to twenty listed qubits at 20 qubits (up to 5 lane bits + 20 listed thread bits
    # and 2^20 bins: the whole distribution)
    rng = np.random.default_rng(81)
    n = 20
    st, psi = start(qs, n, dtype, rng)
    for qubits in (list(range(8, 20)), [19, 0, 7, 3, 12, 1, 15, 9, 4, 18, 2, 11], list(range(13)),
                   list(range(7, 20)), list(range(19, -1, -1)), [int(x) for x in rng.permutation(20)[:17]]):
        got = st.probabilities(qubits)
        ref = oracle.probabilities(psi, n, qubits)
        assert np.max(np.abs(got - ref)) <= 1e-12, qubits
    st.close()


def test_pmeasure_output_larger_than_the_scratch(qs):
    # 22 listed qubits of 22: 2^22 bins (32 MiB) go to a buffer of their own
    rng = np.random.default_rng(82)
    n = 22
    st, psi = start(qs, n, "c64", rng)
    qubits = [int(x) for x in rng.permutation(n)]
    got = st.probabilities(qubits)
    ref = oracle.probabilities(psi, n, qubits)
    assert np.max(np.abs(got - ref)) <= 1e-12
    st.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_readouts_vs_oracle(qs, dtype):
    rng = np.random.default_rng(77)
    n = 14
    st, psi = start(qs, n, dtype, rng)
    tol = 1e-13 if dtype == "c128" else 1e-12
    assert abs(st.norm() - oracle.norm2(psi, n)) <= tol
    for qubits in ([0], [13], [3, 1], [1, 3], [12, 0, 5], list(range(6)), [13, 2, 7, 9, 4, 0, 11, 1],
                   list(range(13))):
        got = st.probabilities(qubits)
        ref = oracle.probabilities(psi, n, qubits)
        assert np.max(np.abs(got - ref)) <= tol, qubits
    assert np.max(np.abs(st.expect_z() - oracle.z_expectations(psi, n))) <= 1e-12
    for idx in (0, 1, 5, (1 << n) - 1, 12345):
        assert abs(st.amplitude(idx) - psi[idx]) <= 1e-15
    other, psi2 = start(qs, n, dtype, np.random.default_rng(78))
    ip = st.inner(other)
    assert abs(ip - oracle.inner(psi, psi2, n)) <= 1e-12
    f = st.fidelity(other)
    ref_f = abs(oracle.inner(psi, psi2, n)) ** 2 / (oracle.norm2(psi, n) * oracle.norm2(psi2, n))
    assert abs(f - ref_f) <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [5, 12, 17])
def test_sample_vs_oracle(qs, dtype, n):
    rng = np.random.default_rng(500 + n)
    st, psi = start(qs, n, dtype, rng)
    shots, seed = 3000, 0xC0FFEE + n
    got = st.sample(shots, seed).astype(np.int64)
    u = oracle.sample_draws(seed, shots)
    ref = oracle.sample(psi, n, u).astype(np.int64)
    cdf = np.cumsum(np.abs(psi) ** 2)
    target = u * cdf[-1]
    j = np.clip(np.searchsorted(cdf, target), 1, len(cdf) - 1)
    gap = np.minimum(np.abs(cdf[j] - target), np.abs(cdf[j - 1] - target))
    near = gap < 1e-9 * max(1.0, cdf[-1])
    mism = got != ref
    assert not np.any(mism & ~near), np.nonzero(mism & ~near)
    # marginal sampling keeps the listed bits of the full-index draw
    qubits = [n - 1, 0, 2]
    marg = st.sample(shots, seed, qubits=qubits).astype(np.int64)
    ref_m = np.array([oracle.project_bits(i, qubits) for i in ref])
    assert np.sum(marg != ref_m) <= np.sum(near)


def test_full_size_28q_compute_uncompute(qs):
    # the 28-qubit depth-40 random circuit then its inverse returns |0...0>
    import torch
    ops = synth.random_circuit(28, 40, seed=0)
    assert synth.count_gates(ops) == 1714
    for dtype, bound in (("c128", 1e-12), ("c64", 1e-6)):
        st = qs.State(28, dtype)
        st.run_circuit(ops)
        norm_mid = st.norm()
        st.run_circuit(synth.inverse_ops(ops))
        a0 = st.amplitude(0)
        assert abs(norm_mid - 1) <= bound
        assert 1 - abs(a0) ** 2 <= bound, (dtype, a0)
        assert abs(st.norm() - 1) <= bound
        del st
        torch.cuda.empty_cache()


def mixed_circuit(n, length, seed):
    """Every gate kind of the App. A-1 library, CONTROL blocks with one or two extra
    controls, DAGGER blocks and gates whose qubits exceed a 5-qubit window."""
    rng = np.random.default_rng(seed)
    one = ["H", "X", "Y", "Z", "S", "T", "SX", "SY"]
    rot = ["RX", "RY", "RZ"]
    ops = []

    def pick(k):
        return tuple(int(x) for x in rng.choice(n, size=k, replace=False))

    def gate():
        r = rng.integers(0, 9)
        if r == 0:
            return [(one[rng.integers(len(one))], pick(1), ())]
        if r == 1:
            return [(rot[rng.integers(3)], pick(1), (float(rng.uniform(-3, 3)),))]
        if r == 2:
            return [("U4", pick(1), tuple(float(x) for x in rng.uniform(-3, 3, size=4)))]
        if r == 3:
            return [(["CNOT", "CZ", "SWAP", "ISWAP"][rng.integers(4)], pick(2), ())]
        if r == 4:
            return [("CR", pick(2), (float(rng.uniform(-3, 3)),))]
        if r == 5:
            return [("TOFFOLI", pick(3), ())]
        def controlled(ctrls, inner):  # CONTROL markers nest, one qubit each
            return ([("CONTROL", (c,), ()) for c in ctrls] + inner +
                    [("ENDCONTROL", (), ())] * len(ctrls))

        if r == 6:  # one or two extra controls around a one- or two-qubit gate
            qs_ = pick(4)
            nc = int(rng.integers(1, 3))
            inner = [("CNOT", qs_[nc:nc + 2], ())] if rng.integers(2) else [("H", qs_[nc:nc + 1], ())]
            return controlled(qs_[:nc], inner)
        if r == 7:  # an adjoint block
            return [("DAGGER", (), ()), ("T", pick(1), ()), ("CR", pick(2), (0.7,)), ("ENDDAGGER", (), ())]
        # four controls on a two-qubit gate: six qubits, wider than any fusion window
        qs_ = pick(6)
        return controlled(qs_[:4], [("CZ", qs_[4:6], ())])

    for _ in range(length):
        ops += gate()
    return ops


@pytest.mark.parametrize("n", [9, 14])
@pytest.mark.parametrize("dtype,fuse", [("c128", 0), ("c128", 3), ("c128", 5), ("c64", 0), ("c64", 4), ("c64", 5)])
def test_all_gate_kinds_per_gate_and_fused_vs_oracle(qs, n, dtype, fuse):
    # n = 9 fuses on CUDA cores (below the tensor-core tile), n = 14 on the tensor cores for
    # complex64; complex128 always fuses in the split format on CUDA cores
    ops = mixed_circuit(n, 120, seed=n + fuse)
    got, ref, st = run_both(qs, n, ops, dtype, fuse=fuse)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    if dtype == "c64":
        fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
        assert fid >= 1 - 1e-6
    if fuse:
        assert st.stats()["fused_blocks"] > 0


def test_edge_cases(qs):
    # one qubit; an instruction list made only of markers; invalid input is rejected
    st = qs.State(1, "c128")
    st.run_circuit([("DAGGER", (), ()), ("ENDDAGGER", (), ())])
    assert st.amplitude(0) == 1.0
    st.run_circuit([("H", (0,), ())])
    assert abs(st.amplitude(1) - math.sqrt(0.5)) < 1e-14  # split format: 48-bit significand
    with pytest.raises(qs.QsimError):
        st.run_circuit([("H", (1,), ())])
    with pytest.raises(qs.QsimError):
        st.run_circuit([("CNOT", (0, 0), ())])
    with pytest.raises(qs.QsimError):
        st.run_circuit([("DAGGER", (), ()), ("H", (0,), ())])
    assert st.amplitude(0) != 0  # unchanged by the rejected calls


@pytest.mark.parametrize("fuse", [4, 5])
def test_qft_plus_random_fused_tensor_cores_vs_oracle(qs, fuse):
    # the QFT + depth-30 random recipe at a size the oracle finishes in seconds
    n = 20
    ops = synth.qft_circuit(n) + synth.random_circuit(n, 30, seed=2)
    got, ref, st = run_both(qs, n, ops, "c64", fuse=fuse)
    assert st.stats()["fused_blocks"] > 0
    assert np.max(np.abs(got - ref)) <= 1e-6
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6
    assert abs(np.vdot(got, got).real - 1) <= 1e-6


@pytest.mark.parametrize("lo_smem", [False, True])
def test_fused_row_phases_vs_oracle(qs, lo_smem):
    # diagonal gates on qubits outside a fused block's window run as row phases in that
    # block: the QFT's controlled phases, RZ with a generic angle, T, and a doubly
    # controlled Z (three-qubit entries); the result must still match the oracle
    n = 20
    ops = [("H", (q,), ()) for q in range(n)] + synth.qft_circuit(n)
    ops += [("RZ", (15,), (0.7310254,)), ("CONTROL", (3,), ()), ("CZ", (17, 19), ()),
            ("ENDCONTROL", (), ()), ("T", (18,), ()), ("CR", (16, 12), (-1.234,))]
    ops += synth.random_circuit(n, 6, seed=9)
    st = qs.State(n, "c64")
    st.set_tc_lo_smem(lo_smem)
    st.run_circuit(ops, fuse=5)
    stats = st.stats()
    got = st.to_numpy().astype(np.complex128)
    ref = oracle.run(n, ops)
    assert stats["phase_gates"] > 0 and stats["fused_blocks"] > 0
    assert np.max(np.abs(got - ref)) <= 1e-6
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert fid >= 1 - 1e-6


@pytest.mark.parametrize("fuse", [4, 5])
def test_fused_low_part_in_tensor_or_shared_memory_agree(qs, fuse):
    # the low TF32 part of each tile in tensor memory (five or eight loads in flight) or
    # in shared memory (three): the same products in the same order, bit-identical states
    n = 20
    ops = synth.qft_circuit(n) + synth.random_circuit(n, 30, seed=2)
    ref = oracle.run(n, ops)
    outs = []
    for lo_smem in (False, True):
        st = qs.State(n, "c64")
        st.set_tc_lo_smem(lo_smem)
        st.run_circuit(ops, fuse=fuse)
        assert st.stats()["fused_blocks"] > 0
        outs.append(st.to_numpy().astype(np.complex128))
        st.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0] - ref)) <= 1e-6


def test_autotuned_width_matches_oracle(qs):
    # fuse = -1: the device microbenchmarks price every candidate plan and the cheapest
    # runs; whatever it picks, the result must match the oracle
    t = qs.qsim_autotune()
    for key in ("gbs_pair_c64", "gbs_pair_df_c128", "gbs_fused_k5", "gbs_remap", "gbs_fused_df_k3"):
        assert t[key] > 0, key
    ops = synth.random_circuit(14, 12, seed=7)
    got, ref, st = run_both(qs, 14, ops, "c128", fuse=-1)
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert st.stats()["predicted_ms"] > 0
    got, ref, st = run_both(qs, 14, ops, "c64", fuse=-1)
    assert np.max(np.abs(got - ref)) <= 1e-6


def compute_uncompute(qs, n, ops, dtype, fuse):
    import torch
    st = qs.State(n, dtype)
    st.run_circuit(ops, fuse=fuse)
    norm_mid = st.norm()
    st.run_circuit(synth.inverse_ops(ops), fuse=fuse)
    a0 = st.amplitude(0)
    norm_end = st.norm()
    stats = st.stats()
    st.close()
    del st
    torch.cuda.empty_cache()
    return norm_mid, a0, norm_end, stats


def test_full_size_28q_fused_compute_uncompute(qs):
    ops = synth.random_circuit(28, 40, seed=0)
    norm_mid, a0, norm_end, stats = compute_uncompute(qs, 28, ops, "c64", 5)
    assert stats["fused_blocks"] > 0
    assert abs(norm_mid - 1) <= 1e-6 and abs(norm_end - 1) <= 1e-6
    assert abs(a0) ** 2 / norm_end >= 1 - 1e-6


def test_full_size_32q_qft_random_fused(qs):
    # 32-qubit complex64 (32 GiB): QFT(32) + depth-30 random, fused into 5-qubit unitaries
    ops = synth.qft_circuit(32) + synth.random_circuit(32, 30, seed=3)
    norm_mid, a0, norm_end, stats = compute_uncompute(qs, 32, ops, "c64", 5)
    assert abs(norm_mid - 1) <= 1e-6 and abs(norm_end - 1) <= 1e-6
    assert abs(a0) ** 2 / norm_end >= 1 - 1e-6


def test_full_size_34q_random_fused(qs):
    # the largest single state: 34-qubit complex64 (128 GiB), depth 24, remaps + fusion
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << 34) + (4 << 30):
        pytest.skip("needs 132 GiB of free device memory")
    ops = synth.random_circuit(34, 24, seed=4)
    norm_mid, a0, norm_end, stats = compute_uncompute(qs, 34, ops, "c64", 5)
    assert stats["remaps"] + stats["epilogue_remaps"] > 0
    assert abs(norm_mid - 1) <= 1e-6 and abs(norm_end - 1) <= 1e-6
    assert abs(a0) ** 2 / norm_end >= 1 - 1e-6


def test_fused_without_renormalisation_drift_is_small_and_fidelity_holds(qs):
    # the raw bias of FP32 tensor-core accumulation (round toward zero), no correction
    ops = synth.random_circuit(28, 40, seed=0)
    st = qs.State(28, "c64")
    st.run_circuit(ops, fuse=5, renorm=False)
    drift = 1 - st.norm()
    st.run_circuit(synth.inverse_ops(ops), fuse=5, renorm=False)
    a0 = st.amplitude(0)
    assert 0 <= drift <= 5e-5
    assert abs(a0) ** 2 / st.norm() >= 1 - 1e-6


def test_fused_renormalisation_keeps_the_input_norm(qs):
    # renormalisation is relative to the state's norm before the first fused block
    n = 16
    rng = np.random.default_rng(31)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi *= 2.0 / np.linalg.norm(psi)  # norm^2 = 4
    ops = synth.random_circuit(n, 12, seed=5)
    st = qs.State(n, "c64")
    st.from_numpy(psi)
    st.run_circuit(ops, fuse=5)
    assert abs(st.norm() / 4.0 - 1) <= 1e-6
    ref = oracle.run(n, ops, psi=psi.astype(np.complex64).astype(np.complex128))
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 2e-6


@pytest.mark.parametrize("n", [3, 9])
def test_fp64_native_kernels_match_oracle(qs, n):
    # the FP64-instruction kernels on plain doubles (qsim_set_option FP64_NATIVE)
    rng = np.random.default_rng(900 + n)
    psi = rand_state(n, rng)
    st = qs.State(n, "c128")
    st.set_fp64_native(True)
    st.from_numpy(psi)
    for t in range(n):
        for name in ONE_Q:
            m = one_q_matrix(name, rng)
            ctl = [(t + 1) % n] if n > 1 and name in ("H", "GEN") else []
            st.apply_gate([t], m, ctl)
            oracle.apply(psi, n, [t], ctl, m)
    ops = synth.random_circuit(n, 6, seed=n)
    st.run_circuit(ops)
    psi = oracle.run(n, ops, psi=psi)
    assert np.max(np.abs(st.to_numpy() - psi)) <= 1e-12


def test_split_format_round_trip_and_readouts(qs):
    # complex128 states switch to the split format for gates and back for read-outs
    n = 13
    rng = np.random.default_rng(17)
    psi = rand_state(n, rng)
    st = qs.State(n, "c128")
    st.from_numpy(psi)
    st.apply_gate([3], oracle.gate_matrix("H")[1])
    oracle.apply(psi, n, [3], [], oracle.gate_matrix("H")[1])
    assert abs(st.amplitude(77) - psi[77]) <= 1e-15        # read while split
    assert abs(st.norm() - oracle.norm2(psi, n)) <= 1e-13   # converts to plain
    st.apply_gate([5], oracle.gate_matrix("SX")[1])          # converts back
    oracle.apply(psi, n, [5], [], oracle.gate_matrix("SX")[1])
    st.canonicalize()
    import torch
    raw = st.tensor.cpu().numpy()                             # plain complex128 again
    assert np.max(np.abs(raw - psi)) <= 1e-14


def test_bounded_wait_reports_timeout_and_context_survives(qs):
    # a device wait that nothing releases runs out after 50 ms and is reported
    import ctypes
    rc = qs.lib().qsim_selftest_bounded_wait(50, None)
    assert rc == 4  # QSIM_ETIMEOUT
    assert "bounded wait" in qs.qsim_last_error()
    ops = synth.random_circuit(12, 4, seed=1)
    got, ref, _ = run_both(qs, 12, ops, "c64", fuse=5)   # the context is still usable
    assert np.max(np.abs(got - ref)) <= 1e-6
    del ctypes


@pytest.mark.parametrize("dtype,fuse", [("c64", 5), ("c128", 4), ("c128", 0), ("c64", -1)])
def test_repeated_circuit_reuses_the_last_plan(qs, dtype, fuse):
    # the same gate list from the same layout takes the state's last plan (bit-identical
    # result); a changed matrix, or a different layout, is planned afresh
    n = 16
    tol = 1e-12 if dtype == "c128" else 1e-6
    ops = synth.random_circuit(n, 8, seed=77)
    ref = oracle.run(n, ops)
    st = qs.State(n, dtype)
    st.run_circuit(ops, fuse=fuse, remap=True)
    first = st.to_numpy()
    assert st.stats()["plan_reused"] == 0
    st.reset()
    st.run_circuit(ops, fuse=fuse, remap=True)
    again = st.to_numpy()
    assert st.stats()["plan_reused"] == 1
    assert np.array_equal(first, again)
    assert np.max(np.abs(again - ref)) <= tol
    ops2 = ops[:-1] + [("RZ", (3,), (0.123,))]
    st.reset()
    st.run_circuit(ops2, fuse=fuse, remap=True)
    assert st.stats()["plan_reused"] == 0
    assert np.max(np.abs(st.to_numpy() - oracle.run(n, ops2))) <= tol
    st.reset()
    st.run_circuit(ops, fuse=fuse, remap=True)
    st.run_circuit(ops, fuse=fuse, remap=True)  # from wherever the first run left the layout
    assert np.max(np.abs(st.to_numpy() - oracle.run(n, ops + ops))) <= 2 * tol
    st.reset()
    st.run_circuit(ops, fuse=fuse, remap=True, use_graph=True)
    st.reset()
    st.run_circuit(ops, fuse=fuse, remap=True, use_graph=True)
    assert np.max(np.abs(st.to_numpy() - ref)) <= tol
    st.close()


def test_async_host_copy_matches_the_synchronous_one(qs):
    # qsim_copy_to_host_async queues the restore of logical order and the copy; after
    # qsim_synchronize the pinned buffer holds what qsim_copy_to_host returns
    import ctypes
    import torch
    n = 16
    ops = synth.random_circuit(n, 10, seed=16)
    st = qs.State(n, "c64")
    st.run_circuit(ops, fuse=5, remap=True)
    pinned = torch.empty(1 << n, dtype=torch.complex64, pin_memory=True)
    qs._check(qs.lib().qsim_copy_to_host_async(st.handle, ctypes.c_void_p(pinned.data_ptr())))
    st.synchronize()
    got = pinned.numpy().copy()
    assert np.array_equal(got, st.to_numpy())
    assert np.max(np.abs(got.astype(np.complex128) - oracle.run(n, ops))) <= 1e-6
    st.close()
