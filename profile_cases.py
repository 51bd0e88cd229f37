"""Small, self-contained launch cases for profiling single kernels under ncu.

    python profile_cases.py pair c64     # k_pair, 26 qubits, target 14
    python profile_cases.py pair c128
    python profile_cases.py fused c64    # fused k = 5 on qubits 0..4
    python profile_cases.py remap c64    # 5-pair remap sweep
    python profile_cases.py perm c64 28  # X (permutation class), target 14
    python profile_cases.py pair c128 28 native   # FP64-instruction kernel
    python profile_cases.py circuit c64 28  # the 28-qubit depth-40
        # circuit, fused (k = 5): tile plans with remaps in the epilogue and row phases
    python profile_cases.py qft c64 26     # QFT(n) + depth-30 random circuit, fused
        # (k = 5): launches that carry many row phases (the QFT's controlled phases)
    python profile_cases.py traj c64 20     # one trajectory launch:
        # 152 noisy trajectories (one per SM) of a depth-20 random circuit on n qubits
    python profile_cases.py diag c64 28     # merged diagonal sweep: T on qubits 0..9 and
        # CZ on (0, 1) ... (8, 9) as one table sweep over 10 qubits
    python profile_cases.py pergate c64 28  # the depth-40 random circuit per gate with the
        # merged diagonal sweeps (merge_diagonals)
    python profile_cases.py readouts c64 28 # norm, inner product, per-qubit Z, PMEASURE of
        # qubits 0..9 and 18..27, 1024 samples, after the depth-40 random circuit (fused)
    python profile_cases.py partial c64 48  # partial amplitude mode:
        # two-block circuit, depth 10, six gates across the line, 2^20 amplitudes; prints
        # the wall time of each of two calls

Each case builds the library if needed, runs three launches of the kernel on a 26-qubit
state (512 MiB complex64 / 1 GiB complex128, larger than L2) and exits 0.
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv):
    import torch
    from paper_2008_07140_gb300 import build
    build.build()
    from paper_2008_07140_gb300 import State
    case = argv[1] if len(argv) > 1 else "pair"
    dtype = argv[2] if len(argv) > 2 else "c64"
    n = int(argv[3]) if len(argv) > 3 else 26
    rng = np.random.default_rng(1)
    if case == "traj":
        from synth import random_circuit
        from paper_2008_07140_gb300 import qsim_run_trajectories
        prog = [(n, random_circuit(n, 20, seed=n))]
        qsim_run_trajectories(prog, [0] * 152, 1, 1e-3, 5e-4, shots=0)
        torch.cuda.synchronize()
        print("ok", case, n)
        return
    if case == "partial":
        import time
        from synth import partial_circuit
        from paper_2008_07140_gb300 import qsim_partial_amplitudes
        ops = partial_circuit(n, 10, 6, seed=n)
        xs = rng.integers(0, 1 << n, size=1 << 20, dtype=np.uint64)
        for _ in range(2):
            t0 = time.perf_counter()
            _, info = qsim_partial_amplitudes(n, ops, xs, dtype=dtype, fuse=5, remap=True)
            print("wall %.2f ms" % ((time.perf_counter() - t0) * 1e3), info)
        print("ok", case, dtype, n)
        return
    st = State(n, dtype)
    if len(argv) > 4 and argv[4] == "native":
        st.set_fp64_native(True)
    if case == "pair":
        z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        u, _ = np.linalg.qr(z)
        for _ in range(3):
            st.apply_gate([14], u)
    elif case == "perm":
        x = np.array([[0.0, 1.0], [1.0, 0.0]])
        for _ in range(3):
            st.apply_gate([14], x)
    elif case == "fused":
        z = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
        u, _ = np.linalg.qr(z)
        for _ in range(3):
            st.apply_fused([4, 3, 2, 1, 0], u)
    elif case == "remap":
        z = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
        u, _ = np.linalg.qr(z)
        for rep in range(3):
            base = 8 + 5 * (rep % 2)
            st.apply_fused([base, base + 1, base + 2, base + 3, base + 4], u)
    elif case == "circuit":
        from synth import random_circuit
        st.run_circuit(random_circuit(n, 40, seed=0), fuse=5, remap=True)
    elif case == "pergate":
        from synth import random_circuit
        st.run_circuit(random_circuit(n, 40, seed=0), fuse=0, merge_diagonals=True)
    elif case == "readouts":
        from synth import random_circuit
        fuse = 5 if dtype == "c64" else 4
        other = State(n, dtype)
        st.run_circuit(random_circuit(n, 40, seed=11), fuse=fuse, remap=True)
        other.run_circuit(random_circuit(n, 20, seed=12), fuse=fuse, remap=True)
        st.canonicalize()
        other.canonicalize()
        for _ in range(2):
            st.norm()
            st.inner(other)
            st.expect_z()
            st.probabilities(list(range(10)))
            st.probabilities(list(range(n - 10, n)))
            st.sample(1024, 7)
    elif case == "diag":
        ops = [("T", (q,), ()) for q in range(10)] + [("CZ", (q, q + 1), ()) for q in range(0, 10, 2)]
        for _ in range(3):
            st.run_circuit(ops, merge_diagonals=True)
    elif case == "qft":
        from synth import qft_circuit, random_circuit
        st.run_circuit(qft_circuit(n) + random_circuit(n, 30, seed=3), fuse=5, remap=True)
    else:
        raise SystemExit("unknown case %r" % case)
    torch.cuda.synchronize()
    print("ok", case, dtype, n, st.norm())


if __name__ == "__main__":
    main(sys.argv)
