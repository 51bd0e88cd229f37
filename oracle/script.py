"""Reader for the instruction-script format of Appendix A-1 (test infrastructure only).

Turns a script (``%Configure`` / ``%Operate`` / ``%Measure`` sections, one instruction per
line) into the oracle's gate list plus the QINIT width and the PMEASURE qubit list. It is
used to replay the worked example of Appendix A-2 against its printed output.
Angles are written as quoted expressions such as "pi/2" or "-pi/4".
"""

import ast
import math
import operator

_BINOPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
           ast.Div: operator.truediv, ast.Pow: operator.pow}


def _angle(text):
    text = text.strip().strip('"').strip()

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
            return float(node.value)
        if isinstance(node, ast.Name) and node.id.lower() == "pi":
            return math.pi
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            v = ev(node.operand)
            return -v if isinstance(node.op, ast.USub) else v
        if isinstance(node, ast.BinOp) and type(node.op) in _BINOPS:
            return _BINOPS[type(node.op)](ev(node.left), ev(node.right))
        raise ValueError("bad angle expression %r" % text)

    return ev(ast.parse(text, mode="eval"))


_ONE_Q = {"H", "X", "Y", "Z", "S", "T", "SX", "SY"}
_ROT = {"RX", "RY", "RZ"}
_TWO_Q = {"CNOT", "CZ", "SWAP", "ISWAP"}


def parse_script(text):
    """Returns (n_qubits, ops, pmeasure_qubits, measures)."""
    n = None
    ops = []
    pmeasure = None
    measures = []
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line or line.startswith("%"):
            continue
        head, _, rest = line.partition(" ")
        head = head.upper()
        args = [a.strip() for a in rest.split(",")] if rest.strip() else []
        if head == "QINIT":
            n = int(args[0])
        elif head == "CREG":
            pass
        elif head in _ONE_Q:
            ops.append((head, (int(args[0]),), ()))
        elif head in _ROT:
            ops.append((head, (int(args[0]),), (_angle(args[1]),)))
        elif head == "U4":
            ops.append((head, (int(args[0]),), tuple(_angle(a) for a in args[1:])))
        elif head in _TWO_Q:
            ops.append((head, (int(args[0]), int(args[1])), ()))
        elif head == "CR":
            ops.append((head, (int(args[0]), int(args[1])), (_angle(args[2]),)))
        elif head == "TOFFOLI":
            ops.append((head, (int(args[0]), int(args[1]), int(args[2])), ()))
        elif head in ("DAGGER", "ENDDAGGER"):
            ops.append((head, (), ()))
        elif head in ("CONTROL", "ENDCONTROL"):
            ops.append((head, tuple(int(a) for a in args), ()))
        elif head == "PMEASURE":
            pmeasure = [int(a) for a in args]
        elif head == "MEASURE":
            measures.append((int(args[0]), int(args[1].lstrip("$"))))
        else:
            raise ValueError("unknown instruction %r" % head)
    if n is None:
        raise ValueError("script has no QINIT")
    return n, ops, pmeasure, measures
