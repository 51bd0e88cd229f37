"""Random-circuit and QFT gate-list generators (names, qubits and angles only).

Random-circuit recipe (a stand-in for the paper's Google-prescription random circuits,
Section 3.1, whose circuit files are not available): for cycle c = 0..d-1, every qubit q
gets one gate drawn from {H, SX, SY, T} (draw mod 4), then CZ acts on the neighbour
pairs (q, q+1) with q = c (mod 2) and q + 1 < n (a one-dimensional brick). A CNOT ladder
CNOT(q, q+1), q = 0..n-2, and a controlled-phase layer CR(q, q+1, pi / 2^((q mod 4)+1))
are appended. For n = 12, d = 20 this gives 372 gates; for n = 28, d = 40, 1714 gates.

The QFT (without the final swaps, so its output is bit-reversed) is the textbook
ladder: for q = n-1 down to 0: H(q), then CR(j, q, pi / 2^(q-j)) for j = q-1 down to 0.
"""

import math

MASK64 = (1 << 64) - 1

# The random single-qubit set of the synthetic circuits. SX and SY are the principal
# square roots of X and Y; neither is in the paper's instruction set.
RQC_1Q_SET = ("H", "SX", "SY", "T")


class SplitMix64:
    """SplitMix64 stream: state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        return self.next() % m


def random_circuit(n: int, depth: int, seed: int, tail: bool = True):
    """Gate list of the synthetic random circuit on n qubits (see module docstring)."""
    if n < 1 or depth < 0:
        raise ValueError("need n >= 1 and depth >= 0")
    rng = SplitMix64(seed * 0x1000193 + n * 0x100 + depth)
    ops = []
    for c in range(depth):
        for q in range(n):
            ops.append((RQC_1Q_SET[rng.below(4)], (q,), ()))
        for q in range(c % 2, n - 1, 2):
            ops.append(("CZ", (q, q + 1), ()))
    if tail:
        for q in range(n - 1):
            ops.append(("CNOT", (q, q + 1), ()))
        for q in range(n - 1):
            ops.append(("CR", (q, q + 1), (math.pi / 2 ** ((q % 4) + 1),)))
    return ops


def partial_circuit(n: int, depth: int, crossings: int, seed: int, cut: int = None):
    """Two-block circuit of the partial-amplitude shape (Section 2.2): `depth` layers of
    random one-qubit gates and CZ ladders that stay inside the upper block (qubits
    [0, cut)) or the lower block ([cut, n)), plus `crossings` gates across the dividing
    line (CZ, CNOT with the control above, CNOT with the control below, CR, in turn; the
    pair drawn from the two blocks), placed after evenly spaced layers. cut defaults to
    n // 2."""
    cut = n // 2 if cut is None else cut
    if not 1 <= cut < n or depth < 1 or crossings < 0:
        raise ValueError("need 1 <= cut < n, depth >= 1, crossings >= 0")
    rng = SplitMix64(seed * 0x2000193 + n * 0x100 + depth * 7 + crossings)
    at = [((k + 1) * depth) // (crossings + 1) for k in range(crossings)]
    ops = []
    k = 0
    for c in range(depth):
        for q in range(n):
            ops.append((RQC_1Q_SET[rng.below(4)], (q,), ()))
        for lo, hi in ((0, cut), (cut, n)):
            for q in range(lo + c % 2, hi - 1, 2):
                ops.append(("CZ", (q, q + 1), ()))
        while k < crossings and at[k] == c:
            a = rng.below(cut)
            b = cut + rng.below(n - cut)
            kind = k % 4
            if kind == 0:
                ops.append(("CZ", (a, b), ()))
            elif kind == 1:
                ops.append(("CNOT", (a, b), ()))
            elif kind == 2:
                ops.append(("CNOT", (b, a), ()))
            else:
                ops.append(("CR", (b, a), (math.pi / 2 ** (1 + k % 3),)))
            k += 1
    return ops


def qft_circuit(n: int):
    """QFT on n qubits without the closing swaps (output in bit-reversed order)."""
    ops = []
    for q in range(n - 1, -1, -1):
        ops.append(("H", (q,), ()))
        for j in range(q - 1, -1, -1):
            ops.append(("CR", (j, q), (math.pi / 2 ** (q - j),)))
    return ops


def inverse_ops(ops):
    """Wrap a gate list in the paper's DAGGER ... ENDDAGGER markers (Appendix A-1)."""
    return [("DAGGER", (), ())] + list(ops) + [("ENDDAGGER", (), ())]


BLOCK_MARKERS = ("DAGGER", "ENDDAGGER", "CONTROL", "ENDCONTROL")


def count_gates(ops) -> int:
    """Number of listed gates (block markers are not gates)."""
    return sum(1 for op in ops if op[0] not in BLOCK_MARKERS)


def trajectory_widths(count: int, lo: int, hi: int, seed: int):
    """Per-trajectory qubit counts drawn uniformly from [lo, hi]."""
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    return [lo + rng.below(hi - lo + 1) for _ in range(count)]
