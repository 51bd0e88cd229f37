"""Instruction scripts (Appendix A-1) run on the GPU through the C ABI.

A script holds one instruction per line. QINIT n and CREG m configure the quantum and
classical registers; gate instructions and DAGGER / CONTROL blocks operate on the state;
MEASURE i, $j measures qubit i into classical register j (the state collapses and keeps
evolving); PMEASURE i, j, ... reads the probabilities of the listed qubits without changing
the state. Section headers ('%...') and comments ('#...') are skipped. Angles are
arithmetic expressions of numbers and pi, optionally quoted ("pi/2", -pi/4, 3*pi/8).

    parse(text)                       -> list of Instr (host only)
    run_script(text, dtype, fuse, draws) -> ScriptResult (runs on the GPU)

MEASURE draws come from `draws`, an iterable of floats in [0, 1) used in script order (by
default a seeded numpy generator); the outcome rule is the library's (qsim_measure).
"""

from dataclasses import dataclass, field

import numpy as np

# name -> (qubits, angle parameters)
_GATES = {
    "H": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0), "S": (1, 0), "T": (1, 0),
    "SX": (1, 0), "SY": (1, 0),
    "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1), "U4": (1, 4),
    "CNOT": (2, 0), "CZ": (2, 0), "SWAP": (2, 0), "ISWAP": (2, 0), "CR": (2, 1),
    "TOFFOLI": (3, 0),
}


class ScriptError(ValueError):
    pass


@dataclass
class Instr:
    op: str                 # instruction name, upper case
    qubits: tuple = ()
    params: tuple = ()
    creg: int = -1          # MEASURE target register
    line: int = 0


@dataclass
class ScriptResult:
    n: int
    cregs: list
    pmeasure: list = field(default_factory=list)  # (qubits, probabilities) per PMEASURE
    state: object = None

    def pmeasure_lines(self, k=0):
        """The k-th PMEASURE in the layout of Appendix A-2: 'bits: probability', 6 significant
        digits."""
        qubits, probs = self.pmeasure[k]
        m = len(qubits)
        return ["%s: %.6g" % (format(s, "0%db" % m), p) for s, p in enumerate(probs)]


class _Angle:
    """Recursive-descent reader for angle expressions: sums of products of factors, a factor
    being a number, pi, a parenthesised expression or a signed factor."""

    def __init__(self, text):
        self.s = text.replace(" ", "")
        self.i = 0

    def value(self):
        v = self._sum()
        if self.i != len(self.s):
            raise ScriptError("bad angle expression %r" % self.s)
        return v

    def _peek(self):
        return self.s[self.i] if self.i < len(self.s) else ""

    def _sum(self):
        v = self._product()
        while self._peek() in ("+", "-"):
            op = self._peek()
            self.i += 1
            w = self._product()
            v = v + w if op == "+" else v - w
        return v

    def _product(self):
        v = self._factor()
        while self._peek() in ("*", "/"):
            op = self._peek()
            self.i += 1
            w = self._factor()
            v = v * w if op == "*" else v / w
        return v

    def _factor(self):
        c = self._peek()
        if c in ("+", "-"):
            self.i += 1
            f = self._factor()
            return f if c == "+" else -f
        if c == "(":
            self.i += 1
            v = self._sum()
            if self._peek() != ")":
                raise ScriptError("unbalanced parenthesis in %r" % self.s)
            self.i += 1
            return v
        if self.s[self.i:self.i + 2].lower() == "pi":
            self.i += 2
            return float(np.pi)
        j = self.i
        while self.i < len(self.s) and (self.s[self.i].isdigit() or self.s[self.i] in ".eE"):
            self.i += 1
        if j == self.i:
            raise ScriptError("bad angle expression %r" % self.s)
        return float(self.s[j:self.i])


def _angle(tok):
    return _Angle(tok.strip().strip('"').strip("'")).value()


def _int(tok, what, lineno):
    try:
        return int(tok)
    except ValueError:
        raise ScriptError("line %d: %s %r is not an integer" % (lineno, what, tok)) from None


def parse(text):
    out = []
    for lineno, raw in enumerate(text.splitlines(), 1):
        body = raw.split("#", 1)[0].strip()
        if not body or body.startswith("%"):
            continue
        name, _, rest = body.partition(" ")
        name = name.upper()
        args = [a.strip() for a in rest.split(",")] if rest.strip() else []
        if name in ("QINIT", "CREG"):
            if len(args) != 1:
                raise ScriptError("line %d: %s takes one number" % (lineno, name))
            out.append(Instr(name, (_int(args[0], "size", lineno),), line=lineno))
        elif name in _GATES:
            nq, npar = _GATES[name]
            if len(args) != nq + npar:
                raise ScriptError("line %d: %s takes %d qubits and %d angles" % (lineno, name, nq, npar))
            qs = tuple(_int(a, "qubit", lineno) for a in args[:nq])
            out.append(Instr(name, qs, tuple(_angle(a) for a in args[nq:]), line=lineno))
        elif name in ("DAGGER", "ENDDAGGER", "ENDCONTROL"):
            out.append(Instr(name, line=lineno))
        elif name == "CONTROL":
            if len(args) != 1:
                raise ScriptError("line %d: CONTROL takes one qubit" % lineno)
            out.append(Instr(name, (_int(args[0], "qubit", lineno),), line=lineno))
        elif name == "MEASURE":
            if len(args) != 2 or not args[1].startswith("$"):
                raise ScriptError("line %d: MEASURE takes a qubit and a $register" % lineno)
            out.append(Instr(name, (_int(args[0], "qubit", lineno),),
                             creg=_int(args[1][1:], "register", lineno), line=lineno))
        elif name == "PMEASURE":
            if not args:
                raise ScriptError("line %d: PMEASURE needs qubits" % lineno)
            out.append(Instr(name, tuple(_int(a, "qubit", lineno) for a in args), line=lineno))
        else:
            raise ScriptError("line %d: unknown instruction %r" % (lineno, name))
    return out


def run_script(text, dtype="c128", fuse=0, draws=None, seed=20080714):
    """Run a script on the GPU; returns a ScriptResult with the State left open."""
    from . import State
    prog = parse(text)
    n = None
    cregs = []
    if draws is None:
        rng = np.random.default_rng(seed)
        draws = iter(lambda: float(rng.random()), None)
    else:
        draws = list(draws)
        need = sum(1 for ins in prog if ins.op == "MEASURE")
        if len(draws) < need:
            raise ScriptError("%d MEASURE instructions but %d draws" % (need, len(draws)))
        if any(not 0.0 <= u < 1.0 for u in draws):
            raise ScriptError("MEASURE draws must lie in [0, 1)")
        draws = iter(draws)
    st = None
    result = None
    pending = []
    depth = 0  # open DAGGER / CONTROL blocks

    def flush():
        if pending:
            st.run_circuit(list(pending), fuse=fuse)
            pending.clear()

    for ins in prog:
        if ins.op == "QINIT":
            if st is not None:
                raise ScriptError("line %d: QINIT given twice" % ins.line)
            n = ins.qubits[0]
            st = State(n, dtype)
            result = ScriptResult(n=n, cregs=cregs, state=st)
            continue
        if ins.op == "CREG":
            cregs.extend([None] * ins.qubits[0])
            continue
        if st is None:
            raise ScriptError("line %d: %s before QINIT" % (ins.line, ins.op))
        if ins.op in ("DAGGER", "CONTROL"):
            depth += 1
        elif ins.op in ("ENDDAGGER", "ENDCONTROL"):
            depth -= 1
        if ins.op in ("MEASURE", "PMEASURE"):
            if depth:
                raise ScriptError("line %d: %s inside a DAGGER or CONTROL block" % (ins.line, ins.op))
            flush()
            if ins.op == "MEASURE":
                if not 0 <= ins.creg < len(cregs):
                    raise ScriptError("line %d: register $%d not allocated by CREG" % (ins.line, ins.creg))
                u = next(draws, None)
                if u is None:
                    raise ScriptError("line %d: no draw left for MEASURE" % ins.line)
                r, _ = st.measure(ins.qubits[0], u)
                cregs[ins.creg] = r
            else:
                result.pmeasure.append((ins.qubits, st.probabilities(list(ins.qubits))))
            continue
        pending.append((ins.op, ins.qubits, ins.params))
    if st is None:
        raise ScriptError("the script has no QINIT")
    flush()
    return result
