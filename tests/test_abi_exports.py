"""The C-ABI library builds, loads and exports every entry point its header declares.

Runs without a GPU: it only loads libqsim.so and calls host-side entry points (the gate
library, the version string, argument validation that fails before any device work).
"""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsim.h")


@pytest.fixture(scope="module")
def qs():
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qsim_create", "qsim_apply_gate", "qsim_apply_fused", "qsim_run_circuit",
                     "qsim_amplitude", "qsim_probabilities", "qsim_sample"):
        assert required in names


def test_every_declared_symbol_is_exported(qs):
    lib = ctypes.CDLL(qs.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []
    assert sorted(qs.EXPORTS) == declared_functions()


def test_version_and_error_string(qs):
    assert "sm_103a" in qs.qsim_version()
    assert isinstance(qs.qsim_last_error(), str)


GATES = [("H", ()), ("X", ()), ("Y", ()), ("Z", ()), ("S", ()), ("T", ()), ("SX", ()), ("SY", ()),
         ("RX", (0.7,)), ("RY", (-1.3,)), ("RZ", (2.1,)), ("U4", (0.3, 1.1, -0.7, 2.5)),
         ("CNOT", ()), ("CZ", ()), ("CR", (0.9,)), ("SWAP", ()), ("ISWAP", ()), ("TOFFOLI", ())]


@pytest.mark.parametrize("name,params", GATES)
def test_host_gate_library_matches_oracle(qs, name, params):
    k, m = qs.qsim_gate_matrix(name, params)
    k_ref, m_ref = oracle.gate_matrix(name, params)
    assert k == k_ref
    assert np.max(np.abs(m - m_ref)) < 1e-15


def test_invalid_arguments_rejected_without_device_work(qs):
    lib = qs.lib()
    h = ctypes.c_void_p()
    assert lib.qsim_create(0, 0, None, ctypes.byref(h)) == 1  # n out of range
    assert lib.qsim_create(5, 7, None, ctypes.byref(h)) == 1  # unknown dtype
    assert lib.qsim_create(41, 0, None, ctypes.byref(h)) == 1
    assert lib.qsim_apply_gate(None, None, 1, None, 0, None) == 1
    assert "NULL" in qs.qsim_last_error() or "state" in qs.qsim_last_error()
    # a caller's buffer must be 256-byte aligned (checked before anything touches it)
    assert lib.qsim_wrap(ctypes.c_void_p(0x10010), 8, 0, None, ctypes.byref(h)) == 1
    assert "aligned" in qs.qsim_last_error()


def test_planner_dry_run_host_only(qs):
    # host-side planning: every gate is accounted for, fusion cuts the sweeps, and the
    # remap-in-epilogue scheme leaves few stand-alone remaps (no device needed)
    import synth
    ops = synth.random_circuit(28, 40, seed=0)
    per_gate = qs.qsim_plan_dry_run(28, "c64", ops, fuse=0)
    assert per_gate["gates"] == 1714 and per_gate["sweeps"] == 1714 and per_gate["remaps"] == 0
    # front-greedy fusion over qubit windows: about 12 gates per sweep at k = 4, 17 at k = 5
    for k, most in ((4, 160), (5, 115)):
        st = qs.qsim_plan_dry_run(28, "c64", ops, fuse=k)
        assert st["gates"] == 1714
        assert st["fused_blocks"] > 0 and st["sweeps"] <= most
        assert st["remaps"] <= 8
    c128 = qs.qsim_plan_dry_run(28, "c128", ops, fuse=5)
    assert c128["remaps"] == 0  # complex128 fuses on CUDA cores, no tensor-core layout


def test_qft_plan_uses_row_phases(qs):
    # diagonal gates whose qubits all lie outside a fused block's window travel with that
    # block as row phases: a 20-qubit QFT (210 gates) plans into a few dozen sweeps
    import synth
    st = qs.qsim_plan_dry_run(20, "c64", synth.qft_circuit(20), fuse=5)
    assert st["gates"] == 210 and st["sweeps"] <= 40 and st["phase_gates"] >= 50
    # no row phases off the tensor-core path
    assert qs.qsim_plan_dry_run(20, "c128", synth.qft_circuit(20), fuse=5)["phase_gates"] == 0


def test_ctypes_struct_layouts_match_the_header(tmp_path):
    # the binding's ctypes mirrors have the header's field offsets and sizes (gcc compiles a
    # probe that prints offsetof / sizeof for every field)
    import ctypes
    import subprocess
    import paper_2008_07140_gb300 as q
    mirrors = {"qsim_op": q.Op, "qsim_run_opts": q.RunOpts, "qsim_traj_batch": q.TrajBatch,
               "qsim_run_stats": q.RunStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qsim.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, field, v = line.split()
            got[(cname, field)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


@pytest.mark.parametrize("n,depth,cross,cut,seed", [(8, 8, 2, 0, 1), (9, 5, 3, 3, 2), (10, 6, 4, 0, 3),
                                                    (12, 4, 5, 7, 4), (11, 3, 0, 0, 5)])
def test_partial_plan_counts_match_the_oracle(n, depth, cross, cut, seed):
    import synth
    import paper_2008_07140_gb300 as q
    ops = synth.partial_circuit(n, depth, cross, seed, cut=cut or None)
    info = q.qsim_partial_plan(n, ops, cut=cut)
    ct, c, circuits = oracle.partial_decompose(n, ops, cut=cut or None)
    assert info["cut"] == ct and info["decomposed"] == c == cross
    assert info["subcircuits"] == 2 * len(circuits) == 2 ** (c + 1)
    assert info["segment_runs"] == sum(2 * 2 ** s for s in range(c + 1))  # prefix sharing
    assert info["slots"] == c + 1
    # each block's segments form one plan: transitions into the next segment run in the
    # previous segment's last epilogue, so at most the very first block of each side needs a
    # stand-alone remap
    assert info["sweeps"] > 0 and info["remaps"] <= 2


def test_partial_plan_multi_controlled_and_rejections():
    import paper_2008_07140_gb300 as q
    ops = [("H", (0,), ()), ("TOFFOLI", (0, 2, 6), ()), ("TOFFOLI", (1, 5, 3), ()), ("TOFFOLI", (4, 6, 2), ()),
           ("CONTROL", (1,), ()), ("ISWAP", (5, 7), ()), ("ENDCONTROL", (), ()), ("CR", (7, 0), (0.4,))]
    assert q.qsim_partial_plan(8, ops)["decomposed"] == oracle.partial_decompose(8, ops)[1] == 5
    for gate in [("SWAP", (1, 5), ()), ("ISWAP", (2, 4), ())]:
        with pytest.raises(q.QsimError):
            q.qsim_partial_plan(6, [("H", (0,), ()), gate])
    with pytest.raises(q.QsimError):
        q.qsim_partial_plan(6, [("H", (0,), ())], cut=6)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7])
def test_partial_plan_on_tiny_blocks(n):
    # blocks of one to three qubits: the fusion width clamps to the block and the plan
    # still counts every segment run
    import synth
    import paper_2008_07140_gb300 as q
    ops = synth.partial_circuit(n, 3, 2, seed=n)
    info = q.qsim_partial_plan(n, ops)
    assert info["cut"] == n // 2 and info["decomposed"] == 2
    assert info["segment_runs"] == 14 and info["sweeps"] > 0 and info["remaps"] == 0
    assert info["gates_applied"] <= info["gates_unshared"]


@pytest.mark.parametrize("kw", [dict(noise={"phase_damping": 1.5}), dict(noise={"bit_flip": -0.1}),
                                dict(p_depol=2.0), dict(gamma=-0.5)])
def test_trajectory_arguments_rejected_on_the_host(kw):
    # argument checks run before any device work, so they hold without a GPU
    import ctypes
    import paper_2008_07140_gb300 as q
    with pytest.raises(q.QsimError) as e:
        q.qsim_run_trajectories([(4, [("H", (0,), ())])], [0], 1, stream=ctypes.c_void_p(0), **kw)
    assert e.value.status == 1  # QSIM_EINVAL


def test_trajectory_batch_struct_rejects_unknown_channel_bits_and_kron():
    import ctypes
    import paper_2008_07140_gb300 as q
    lib = q.lib()
    arr, keep = q.ops_to_c([("H", (0,), ())])
    ops_ptrs = (ctypes.POINTER(q.Op) * 1)(ctypes.cast(arr, ctypes.POINTER(q.Op)))
    widths = (ctypes.c_int32 * 1)(4)
    nops = (ctypes.c_size_t * 1)(1)
    tp = (ctypes.c_int32 * 1)(0)
    zexp = np.zeros(24)
    for channels, kron in ((1 << 6, 0), (1, 2)):
        b = q.TrajBatch(1, widths, ops_ptrs, nops, 1, tp, 1, channels, 0, (ctypes.c_double * 6)(0.1, 0, 0, 0, 0, 0),
                        kron, 0, 0)
        st = lib.qsim_run_trajectories(ctypes.byref(b), ctypes.c_void_p(0), zexp.ctypes.data_as(ctypes.c_void_p),
                                       None, None, None)
        assert st == 1, (channels, kron)
    del keep


def test_partial_amplitudes_arguments_rejected_on_the_host():
    import ctypes
    import paper_2008_07140_gb300 as q
    ops = [("H", (0,), ()), ("CNOT", (0, 3), ())]
    for bad in (dict(indices=[1 << 6]), dict(indices=[0], dtype=7)):
        with pytest.raises((q.QsimError, KeyError)):
            q.qsim_partial_amplitudes(6, ops, bad["indices"], dtype=bad.get("dtype", "c64"), stream=ctypes.c_void_p(0))
    with pytest.raises(q.QsimError):
        q.qsim_partial_amplitudes(6, [("SWAP", (1, 4), ())], [0], stream=ctypes.c_void_p(0))


def test_trajectory_plan_arguments_rejected_on_the_host():
    # qsim_traj_prepare checks the batch and the kept list before any device work
    import ctypes
    import paper_2008_07140_gb300 as q
    progs = [(4, [("H", (0,), ())])]
    lib = q.lib()
    bt = q._Batch(progs, [0, 0], 1, 0.1, 0.0, 0, 0, None, None, False)
    for keep in ([2], [0, 0], [-1]):  # out of range, repeated, negative
        kp = (ctypes.c_int32 * len(keep))(*keep)
        h = ctypes.c_void_p()
        assert lib.qsim_traj_prepare(ctypes.byref(bt.b), kp, len(keep), ctypes.c_void_p(0), ctypes.byref(h)) == 1
        assert not h.value
    assert lib.qsim_traj_prepare(ctypes.byref(bt.b), None, 0, ctypes.c_void_p(0), None) == 1
    with pytest.raises(q.QsimError):
        q.TrajPlan(progs, [0], 1, p_depol=1.5, stream=ctypes.c_void_p(0))
    assert lib.qsim_traj_launch(None, None) == 1
    assert lib.qsim_traj_set_seed(None, 5) == 1
    assert lib.qsim_traj_state(None, 0, None, None) == 1


def test_expand_reproduces_the_oracle_on_the_host():
    # the gate list qsim_expand returns (blocks expanded, CNOT / CZ / CR / TOFFOLI in
    # (target, controls) form), applied by the oracle's Eq. 2 / Eq. 3 loops, gives the
    # oracle's own run of the instruction list
    import oracle
    import synth
    import paper_2008_07140_gb300 as q
    n = 7
    ops = synth.qft_circuit(n) + synth.random_circuit(n, 3, seed=12)
    ops += [("DAGGER", (), ()), ("TOFFOLI", (0, 5, 3), ()), ("U4", (2,), (0.3, -1.1, 0.7, 2.0)),
            ("ENDDAGGER", (), ()), ("CONTROL", (6,), ()), ("ISWAP", (1, 4), ()), ("CONTROL", (2,), ()),
            ("RX", (0,), (0.4,)), ("ENDCONTROL", (), ()), ("ENDCONTROL", (), ()), ("CZ", (4, 6), ())]
    gates = q.qsim_expand(n, ops)
    psi = oracle.zero_state(n)
    for targets, controls, m, _ in gates:
        oracle.apply(psi, n, list(targets), list(controls), m)
    assert np.max(np.abs(psi - oracle.run(n, ops))) <= 1e-14
    kinds = [k for _, _, _, k in gates]
    assert "CNOT" in kinds and "TOFFOLI" in kinds
    assert all(len(t) == 1 for t, c, _, k in gates if k in ("CNOT", "CZ", "CR", "TOFFOLI"))
    with pytest.raises(q.QsimError):
        q.qsim_expand(n, [("H", (n,), ())])
    with pytest.raises(q.QsimError):
        q.qsim_expand(n, [("DAGGER", (), ()), ("H", (0,), ())])
