"""Host-side planning of the merged diagonal sweep (qsim_run_opts.merge_diagonals), through
qsim_plan_dry_run: no device is touched. The GPU tests check the numbers; these check the
grouping rule: a diagonal gate joins an open group of at most 10 qubits, a non-diagonal gate
closes only the groups that share a qubit with it, and a group runs as one table sweep only
when its per-gate sweeps would move more bytes."""

import numpy as np

import synth


def q():
    import paper_2008_07140_gb300 as qs
    return qs


def cz_ladder(qubits):
    return [("CZ", (a, a + 1), ()) for a in qubits]


def test_groups_hold_at_most_ten_qubits():
    # twelve commuting CZs on 24 qubits: two groups of five (ten qubits each) become table
    # sweeps; the last two CZs (a quarter of the state each) stay per-gate sweeps
    ops = cz_ladder(range(0, 24, 2))
    st = q().qsim_plan_dry_run(24, "c64", ops, fuse=0, merge_diagonals=True)
    assert st["diag_sweeps"] == 2 and st["diag_gates"] == 10
    assert st["sweeps"] == 4


def test_non_diagonal_gate_closes_only_the_groups_it_touches():
    # group A on qubits 0..9, group B on 10..19; H on qubit 0 closes A only, and the CZs
    # after it on 10..19 still join B
    ops = cz_ladder(range(0, 10, 2)) + cz_ladder(range(10, 20, 2)) + [("H", (0,), ())]
    ops += [("S", (a,), ()) for a in range(10, 20)]
    st = q().qsim_plan_dry_run(24, "c64", ops, fuse=0, merge_diagonals=True)
    assert st["diag_sweeps"] == 2
    assert st["diag_gates"] == 5 + 5 + 10
    assert st["sweeps"] == 3  # A, the H, B


def test_a_few_high_phases_stay_per_gate():
    # a T and a CZ on high qubits move half and a quarter of the state: cheaper than one
    # table sweep over the whole state
    ops = [("T", (20,), ()), ("CZ", (21, 22), ())]
    st = q().qsim_plan_dry_run(24, "c64", ops, fuse=0, merge_diagonals=True)
    assert st["diag_sweeps"] == 0 and st["sweeps"] == 2
    # on low qubits each phase sweep moves whole 64-byte segments: one table sweep
    ops = [("T", (0,), ()), ("T", (1,), ())]
    st = q().qsim_plan_dry_run(24, "c64", ops, fuse=0, merge_diagonals=True)
    assert st["diag_sweeps"] == 1 and st["sweeps"] == 1


def test_controls_count_toward_the_group_and_wide_gates_pass():
    # a diagonal with controls on more than 10 qubits cannot join a group: it runs as its
    # own sweep and closes nothing
    ctl = [("CONTROL", (c,), ()) for c in range(2, 12)]
    ops = cz_ladder([12, 14]) + ctl + [("Z", (0,), ())] + [("ENDCONTROL", (), ())] * 10 + cz_ladder([16, 18])
    st = q().qsim_plan_dry_run(24, "c64", ops, fuse=0, merge_diagonals=True)
    assert st["diag_sweeps"] == 1 and st["diag_gates"] == 4
    assert st["sweeps"] == 2


def test_merging_is_off_by_default_and_in_fused_plans():
    ops = synth.random_circuit(14, 10, seed=3)
    plain = q().qsim_plan_dry_run(14, "c64", ops, fuse=0)
    assert plain["diag_sweeps"] == 0 and plain["sweeps"] == synth.count_gates(ops)
    fused = q().qsim_plan_dry_run(14, "c64", ops, fuse=5, merge_diagonals=True)
    assert fused["diag_sweeps"] == 0
    merged = q().qsim_plan_dry_run(14, "c128", ops, fuse=0, merge_diagonals=True)
    assert merged["sweeps"] < plain["sweeps"] and merged["diag_gates"] >= 2 * merged["diag_sweeps"] > 0
    assert np.isfinite(merged["bytes"])
