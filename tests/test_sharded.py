"""A state split over 2^g shards by its top index bits (Section 2.2, step 2), on the host.

The shard planner and both executors run here on host shards whose local arithmetic is the
FP64 oracle's Eq. 2 / Eq. 3 loops on each shard's 2^(n-g) amplitudes: swapping a global
qubit in (Section 3.1's pairwise exchange of half shards), skipping shards under a global
control and folding diagonal gates on global qubits must reproduce the oracle's run of the
whole state. The distributed executor runs as two gloo ranks on CPU.
"""

import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2008_07140_gb300 import sharded

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class HostHalf:
    def __init__(self, view):
        self.view = view

    def tensor(self):
        import torch
        return torch.from_numpy(self.view.view(np.float64))

    def set_tensor(self, t):
        self.view[:] = t.numpy().view(np.complex128)

    def copy_out(self):
        return self.view.copy()

    def copy_in(self, src):
        self.view[:] = src


class HostShard:
    """A shard in host memory; gates by the oracle's loops on the shard alone."""

    def __init__(self, L, first):
        self.L = L
        self.psi = np.zeros(1 << L, dtype=np.complex128)
        if first:
            self.psi[0] = 1.0

    def apply(self, targets, controls, m):
        oracle.apply(self.psi, self.L, list(targets), list(controls), m)

    def half(self, v):
        h = 1 << (self.L - 1)
        return HostHalf(self.psi[v * h:(v + 1) * h])

    def sync(self):
        pass

    def to_numpy(self):
        return self.psi


def mixed_ops(n, seed):
    """QFT, a random circuit and every gate kind, CONTROL and DAGGER blocks included."""
    rng = np.random.default_rng(seed)
    ops = synth.qft_circuit(n) + synth.random_circuit(n, 4, seed=seed)
    for _ in range(40):
        q = [int(x) for x in rng.choice(n, size=3, replace=False)]
        kind = int(rng.integers(8))
        if kind == 0:
            ops.append(("TOFFOLI", tuple(q), ()))
        elif kind == 1:
            ops.append(("SWAP", tuple(q[:2]), ()))
        elif kind == 2:
            ops.append(("ISWAP", tuple(q[:2]), ()))
        elif kind == 3:
            ops += [("CONTROL", (q[0],), ()), ("RX", (q[1],), (0.37,)), ("ENDCONTROL", (), ())]
        elif kind == 4:
            ops += [("DAGGER", (), ()), ("CR", tuple(q[:2]), (1.1,)), ("SY", (q[2],), ()), ("ENDDAGGER", (), ())]
        elif kind == 5:
            ops.append(("U4", (q[0],), (0.3, -1.2, 0.8, 2.1)))
        elif kind == 6:
            ops.append(("CZ", tuple(q[:2]), ()))
        else:
            ops.append(("RZ", (q[0],), (-0.61,)))
    return ops


def host_gates(n, ops):
    """(targets, controls, matrix) from the oracle's expansion with controlled gates split
    into (target, controls) form here, so that the test does not need the CUDA library."""
    out = []
    for qubits, controls, m in oracle.expand(ops):
        qubits, controls, m = list(qubits), list(controls), np.asarray(m)
        # peel leading control qubits of P0 (x) I + P1 (x) U' matrices (CNOT, CZ, CR, TOFFOLI)
        while len(qubits) > 1:
            d = m.shape[0] // 2
            if not (np.allclose(m[:d, :d], np.eye(d)) and np.allclose(m[:d, d:], 0) and np.allclose(m[d:, :d], 0)):
                break
            controls.append(qubits.pop(0))
            m = m[d:, d:]
        out.append((qubits, controls, m))
    return out


@pytest.mark.parametrize("n,g", [(5, 1), (7, 2), (8, 3), (9, 1)])
def test_local_shards_reproduce_the_oracle(n, g):
    ops = mixed_ops(n, seed=n + g)
    gates = host_gates(n, ops)
    L = n - g
    shards = [HostShard(L, r == 0) for r in range(1 << g)]
    ex = sharded.LocalShards(n, g, shards)
    ex.run_gates(gates)
    got = ex.to_numpy()
    ref = oracle.run(n, ops)
    assert np.max(np.abs(got - ref)) <= 1e-13
    assert ex.planner.exchanges > 0  # gates on global qubits took exchanges
    # the planner's layout is a permutation and every global qubit swap was paired
    assert sorted(ex.planner.pos) == list(range(n))
    assert all(ex.planner.at[ex.planner.pos[q]] == q for q in range(n))


def test_diagonal_and_controlled_gates_on_global_qubits_take_no_exchange():
    # after a Hadamard layer (which swaps the global qubits in and out), controls and
    # diagonal targets on whatever qubits are global then are resolved per shard
    n, g = 6, 2
    first = [("H", (q,), ()) for q in range(n)]
    ex = sharded.LocalShards(n, g, [HostShard(n - g, r == 0) for r in range(1 << g)])
    ex.run_gates(host_gates(n, first))
    before = ex.planner.exchanges
    a, b = ex.planner.at[n - 2], ex.planner.at[n - 1]  # the qubits on global bits now
    lo = [q for q in range(n) if q not in (a, b)]
    second = [("CZ", (b, lo[1]), ()), ("CR", (a, b), (0.4,)), ("T", (b,), ()), ("CNOT", (a, lo[0]), ()),
              ("RZ", (a,), (0.9,)), ("TOFFOLI", (b, a, lo[2]), ()), ("CONTROL", (b,), ()), ("S", (a,), ()),
              ("ENDCONTROL", (), ()), ("CZ", (a, b), ())]
    ex.run_gates(host_gates(n, second))
    assert ex.planner.exchanges == before
    assert np.max(np.abs(ex.to_numpy() - oracle.run(n, first + second))) <= 1e-14


def test_exchange_count_follows_the_schedule():
    # a Hadamard on each global qubit, twice: the first swaps it in, the second finds it local
    n, g = 8, 2
    ops = [("H", (6,), ()), ("H", (7,), ()), ("H", (6,), ()), ("H", (7,), ())]
    ex = sharded.LocalShards(n, g, [HostShard(n - g, r == 0) for r in range(4)])
    ex.run_gates(host_gates(n, ops))
    assert ex.planner.exchanges == 2
    assert np.max(np.abs(ex.to_numpy() - oracle.run(n, ops))) <= 1e-15


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ops = mixed_ops(n, seed=77)
    gates = host_gates(n, ops)
    g = world.bit_length() - 1
    sh = sharded.DistShard(n, HostShard(n - g, rank == 0))
    sh.run_gates(gates)
    full = sh.gather()
    results[rank] = (full.tobytes(), sh.planner.exchanges)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_dist_shards_gloo_reproduce_the_oracle(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    n = 7
    with ctx.Manager() as mgr:
        results = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, n, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        ref = oracle.run(n, mixed_ops(n, seed=77))
        for r in range(world):
            full = np.frombuffer(results[r][0], dtype=np.complex128)
            assert np.max(np.abs(full - ref)) <= 1e-13
            assert results[r][1] > 0
