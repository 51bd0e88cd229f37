"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the simulation method. It only emits gate *lists*:
tuples ``(name, qubits, params)`` with gate names from the paper's instruction set
(Appendix A-1) plus the random-circuit single-qubit set {H, SX, SY, T}. Each side
(the FP64 oracle and the CUDA library) turns names into matrices with its own code.

Random draws come from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), a counter-style
64-bit mixer chosen because it is short enough to state exactly.
"""

from .circuits import (  # noqa: F401
    SplitMix64,
    random_circuit,
    partial_circuit,
    qft_circuit,
    inverse_ops,
    count_gates,
    trajectory_widths,
    RQC_1Q_SET,
    BLOCK_MARKERS,
)
