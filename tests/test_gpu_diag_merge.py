"""GPU parity of the merged diagonal sweep (qsim_run_opts.merge_diagonals) against the oracle.

Per-gate runs with merging group the diagonal gates that commute past the gates between
them and apply each group as one table sweep. The oracle applies the instruction list gate
by gate (Eq. 2 / Eq. 3), in its own order, so these tests also check that the planner only
moves gates past gates they commute with. Tolerances as everywhere: complex128 (split
format and FP64 instructions) max|d amp| <= 1e-12, complex64 1e-6.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-6, "native": 1e-12}


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


def diagonal_heavy(n, length, seed):
    """Mostly diagonal gates (Z, S, T, RZ, CZ, CR, controlled and adjoint diagonals) with
    some non-diagonal gates (H, SX, RX, CNOT) that break and reorder the groups."""
    rng = np.random.default_rng(seed)
    ops = []

    def pick(k):
        return tuple(int(x) for x in rng.choice(n, size=k, replace=False))

    kinds = [0, 1, 2, 3] + ([4, 5] if n >= 2 else []) + ([6, 7, 8] if n >= 3 else []) + ([9] if n >= 4 else [])
    for _ in range(length):
        r = kinds[int(rng.integers(len(kinds)))]
        if r == 0:
            ops.append((["Z", "S", "T"][rng.integers(3)], pick(1), ()))
        elif r == 1:
            ops.append(("RZ", pick(1), (float(rng.uniform(-3, 3)),)))
        elif r == 2:
            ops.append((["H", "SX"][rng.integers(2)], pick(1), ()))
        elif r == 3:
            ops.append(("RX", pick(1), (float(rng.uniform(-3, 3)),)))
        elif r == 4:
            ops.append(("CZ", pick(2), ()))
        elif r == 5:
            ops.append(("CR", pick(2), (float(rng.uniform(-3, 3)),)))
        elif r == 6:  # a controlled RZ: a diagonal whose first entry is not 1
            q = pick(3)
            ops += [("CONTROL", (q[0],), ()), ("RZ", q[1:2], (float(rng.uniform(-3, 3)),)), ("ENDCONTROL", (), ())]
        elif r == 7:  # an adjoint block of diagonals
            ops += [("DAGGER", (), ()), ("T", pick(1), ()), ("CR", pick(2), (0.3,)), ("ENDDAGGER", (), ())]
        elif r == 8:
            ops.append(("CNOT", pick(2), ()))
        else:  # a doubly controlled CZ: four qubits in one group
            q = pick(4)
            ops += [("CONTROL", (q[0],), ()), ("CONTROL", (q[1],), ()), ("CZ", q[2:4], ()),
                    ("ENDCONTROL", (), ()), ("ENDCONTROL", (), ())]
    return ops


def make_state(qs, n, kind, rng):
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    if kind == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    st = qs.State(n, "c128" if kind == "native" else kind)
    if kind == "native":
        st.set_fp64_native(True)
    st.from_numpy(psi)
    return st, psi


@pytest.mark.parametrize("kind", ["c128", "c64", "native"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 14])
def test_merged_diagonals_vs_oracle(qs, kind, n):
    # n = 1, 2 put every table bit inside one 32-byte chunk (and n = 1 runs the one-amplitude
    # complex64 path); n = 14 needs groups to split at 10 qubits
    rng = np.random.default_rng(4000 + n)
    st, psi = make_state(qs, n, kind, rng)
    ops = diagonal_heavy(n, 150, seed=n)
    st.run_circuit(ops, merge_diagonals=True)
    ref = oracle.run(n, ops, psi=psi)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[kind]
    stats = st.stats()
    if n >= 3:
        assert stats["diag_sweeps"] > 0
        assert stats["diag_gates"] >= 2 * stats["diag_sweeps"]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_brick_layers_merge_into_few_sweeps(qs, dtype):
    # the random-circuit recipe: after each layer of single-qubit gates, the T gates and the
    # whole CZ brick layer of 14 qubits run as two table sweeps (10 + 4 qubits) or so
    n = 14
    ops = synth.random_circuit(n, 12, seed=7)
    st = qs.State(n, dtype)
    st.run_circuit(ops, merge_diagonals=True)
    ref = oracle.run(n, ops)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    stats = st.stats()
    plain = qs.qsim_plan_dry_run(n, dtype, ops, fuse=0)
    assert stats["sweeps"] < plain["sweeps"]
    assert stats["diag_gates"] > stats["diag_sweeps"]


def test_merged_plan_under_graph_capture_and_reuse(qs):
    n = 10
    ops = diagonal_heavy(n, 80, seed=11)
    ref = oracle.run(n, ops)
    st = qs.State(n, "c128")
    for use_graph in (False, False, True, True):  # reused plan; then captured, then replayed
        st.reset()
        st.run_circuit(ops, merge_diagonals=True, use_graph=use_graph)
        got = st.to_numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert st.stats()["diag_sweeps"] > 0
    st.close()


def test_deep_repetition_of_merged_groups_stays_within_1e12(qs):
    # the same groups applied over and over: the table entries are the exact products of
    # the FP64 entries, so their rounding does not add up coherently beyond the per-gate
    # path's; 14 qubits, 30 repetitions of a block and its inverse (4020 gates, about 2300
    # sweeps: inside the split format's budget of 4096)
    n = 14
    block = synth.random_circuit(n, 2, seed=5)
    ops = (block + synth.inverse_ops(block)) * 30
    st = qs.State(n, "c128")
    st.run_circuit(ops, merge_diagonals=True)
    assert st.stats()["fp64_fallback"] == 0
    got = st.to_numpy()
    ref = oracle.zero_state(n)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_autotuned_width_with_merging_matches_oracle(qs, dtype):
    # fuse = -1 plans every candidate width, the per-gate candidate with table sweeps
    n = 12
    ops = synth.random_circuit(n, 20, seed=21)
    st = qs.State(n, dtype)
    st.run_circuit(ops, fuse=-1, merge_diagonals=True)
    got = st.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - oracle.run(n, ops))) <= TOL[dtype]
    assert st.stats()["predicted_ms"] > 0
    st.close()
