"""The instruction-script front end (Appendix A-1) of the library: parsing on the host, and
the Appendix A-2 worked example plus a script with mid-circuit MEASURE run on the GPU
against the printed output and the FP64 oracle."""

import math
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2008_07140_gb300 import script

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_a2_example.txt")


def expected_a2():
    out = {}
    for line in open(GOLDEN).read().splitlines():
        if line.startswith("#@expected"):
            k, v = line[len("#@expected"):].split(":")
            out[k.strip()] = float(v)
    return out


def test_parse_the_appendix_a2_script():
    prog = script.parse(open(GOLDEN).read())
    names = [i.op for i in prog]
    assert names[:2] == ["QINIT", "CREG"] and prog[0].qubits == (5,) and prog[1].qubits == (3,)
    assert names[-1] == "PMEASURE" and prog[-1].qubits == (4, 3, 0)
    assert names.count("DAGGER") == 1 and names.count("ENDDAGGER") == 1
    cr = [i for i in prog if i.op == "CR"]
    assert abs(cr[0].params[0] - math.pi / 2) < 1e-15 and abs(cr[1].params[0] - math.pi / 4) < 1e-15
    ry = [i for i in prog if i.op == "RY"]
    assert abs(ry[0].params[0] + math.pi / 4) < 1e-15


@pytest.mark.parametrize("text,value", [("pi", math.pi), ('"-pi/4"', -math.pi / 4), ("3*pi/8", 3 * math.pi / 8),
                                        ("-(pi/4)+pi", 0.75 * math.pi), ("0.5", 0.5), ("2*(1+pi)", 2 * (1 + math.pi))])
def test_angle_expressions(text, value):
    prog = script.parse("QINIT 1\nRZ 0," + text)
    assert abs(prog[1].params[0] - value) < 1e-15


@pytest.mark.parametrize("text", ["QINIT 2\nFOO 0", "QINIT 2\nMEASURE 0,1", "QINIT 2\nRZ 0,pi/", "QINIT 2\nCNOT 0",
                                  "QINIT 2\nH x", "QINIT 2\nPMEASURE"])
def test_parse_errors(text):
    with pytest.raises(script.ScriptError):
        script.parse(text)


def fmt(op):
    name, qubits, params = op
    args = [str(q) for q in qubits] + ['"%r"' % p for p in params]
    return name + (" " + ",".join(args) if args else "")


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,fuse", [("c128", 0), ("c128", 5), ("c64", 5)])
def test_appendix_a2_script_end_to_end_on_the_gpu(dtype, fuse):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    res = script.run_script(open(GOLDEN).read(), dtype=dtype, fuse=fuse)
    exp = expected_a2()
    assert res.n == 5 and res.cregs == [None, None, None]
    # the printed probabilities carry 6 significant digits (the exact 0.8200825 is printed
    # 0.820082): compare the unrounded values within one unit of the last printed digit
    qubits, probs = res.pmeasure[0]
    for s, p in enumerate(probs):
        key = format(s, "0%db" % len(qubits))
        assert abs(p - exp[key]) <= 1e-6, (key, p, exp[key])
    assert [l.split(":")[0] for l in res.pmeasure_lines()] == sorted(exp)
    res.state.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_mid_circuit_measure_script_vs_oracle(dtype):
    # gates, MEASURE, more gates, MEASURE, PMEASURE: outcomes, registers and the final
    # probabilities against the oracle replaying the same draws
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 8
    part1 = synth.random_circuit(n, 6, seed=11)
    part2 = synth.random_circuit(n, 5, seed=12)
    draws = [0.37, 0.81]
    text = "\n".join(["QINIT %d" % n, "CREG 2"] + [fmt(o) for o in part1] + ["MEASURE 3,$0"] +
                     [fmt(o) for o in part2] + ["MEASURE 6,$1", "PMEASURE 0,3,6,7"])
    res = script.run_script(text, dtype=dtype, fuse=5, draws=draws)
    psi = oracle.run(n, part1)
    r0, _, psi = oracle.measure(psi, n, 3, draws[0])
    psi = oracle.run(n, part2, psi)
    r1, _, psi = oracle.measure(psi, n, 6, draws[1])
    ref = oracle.probabilities(psi, n, [0, 3, 6, 7])
    assert res.cregs == [r0, r1]
    qubits, probs = res.pmeasure[0]
    assert qubits == (0, 3, 6, 7)
    tol = 1e-12 if dtype == "c128" else 1e-6
    assert np.max(np.abs(probs - ref)) <= tol
    assert abs(res.state.norm() - 1) <= tol
    res.state.close()


@pytest.mark.parametrize("draws", [[], [0.5], [0.2, 1.0]])
def test_measure_draws_are_checked_before_any_device_work(draws):
    text = "QINIT 2\nCREG 2\nH 0\nMEASURE 0,$0\nMEASURE 1,$1"
    with pytest.raises(script.ScriptError):
        script.run_script(text, draws=draws)


ALL_KINDS = """%Configure
QINIT 4
CREG 2
%Operate
H 0
X 1
Y 2
Z 3
S 0
T 1
SX 2
SY 3
RX 0,"pi/3"
RY 1,-pi/4
RZ 2,"3*pi/8"
U4 3,"pi/2","pi/3","-pi/5","pi/7"
CNOT 0,1
CZ 1,2
SWAP 2,3
ISWAP 0,3
CR 1,3,"pi/16"
TOFFOLI 0,1,2
DAGGER
  H 1
  CONTROL 3
    RX 0,"2*(1+pi)"
  ENDCONTROL
ENDDAGGER
%Measure
MEASURE 1,$0
PMEASURE 3,0
"""


@pytest.mark.parametrize("which", ["a2", "all_kinds"])
def test_front_end_reads_scripts_as_the_oracle_reader_does(which):
    # two independent readers of the App. A-1 format: the same gates, qubits and angles
    from oracle.script import parse_script
    text = open(GOLDEN).read() if which == "a2" else ALL_KINDS
    n, ops, pm, measures = parse_script(text)
    prog = script.parse(text)
    gates = [i for i in prog if i.op not in ("QINIT", "CREG", "MEASURE", "PMEASURE")]
    assert [i.op for i in prog if i.op == "QINIT"] == ["QINIT"] and prog[0].qubits == (n,)
    assert len(gates) == len(ops)
    for ins, (name, qubits, params) in zip(gates, ops):
        assert ins.op == name and tuple(ins.qubits) == tuple(qubits), (ins, name, qubits)
        assert len(ins.params) == len(params)
        assert all(abs(a - b) < 1e-15 for a, b in zip(ins.params, params)), (ins, params)
    assert [(i.qubits[0], i.creg) for i in prog if i.op == "MEASURE"] == measures
    pms = [list(i.qubits) for i in prog if i.op == "PMEASURE"]
    assert (pms[-1] if pms else None) == pm
