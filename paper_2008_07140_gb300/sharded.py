"""One n-qubit state split over G = 2^g shards by its top g index bits (Section 2.2, step 2).

Shard r holds the 2^L amplitudes (L = n - g) whose index has r in its top g bits; inside a
shard the index bits are the L "local" positions. A logical qubit sits either at a local
position (0..L-1) or at a global one (L..n-1, bit j = position - L of the shard number).
The layout starts as the identity and changes only through swaps.

How a gate runs (the gate list comes from qsim_expand: targets, controls, matrix):

* every qubit local: each shard applies it to its own amplitudes;
* a control on a global qubit: the shards whose bit is 0 skip the gate, the others apply
  it with their local controls only;
* a diagonal gate with a target on a global qubit: the shard's bit selects the diagonal
  entries, which leaves a diagonal gate on the local targets (or a phase on the whole
  shard under the local controls);
* any other gate on a global target: the global qubit is first swapped with a local one.
  The local qubit whose next use is furthest away is moved to the top local position L - 1
  (a local SWAP gate when it is not already there), then shards r and r ^ 2^j exchange
  halves: shard r keeps the half whose top local bit equals its own bit j and sends the
  other half to its partner, which sends back the matching half (Section 3.1 measures this
  pairwise exchange as the dominant cost of a gate on a global qubit). Afterwards position
  L - 1 holds the formerly global qubit and global bit j the formerly local one.

The schedule depends only on the gate list and the layout, so every shard takes the same
decisions without talking to the others; the only data exchanged are the half shards.

Execution is split from planning: ``ShardPlanner`` turns gates into steps (a local gate for
every shard, or an exchange of global bit j); an executor runs the steps on its shards.
``DistShard`` runs one shard per process with torch.distributed point-to-point transfers
(NCCL between GPUs, gloo on CPU); ``LocalShards`` runs all shards of one state in one
process and swaps the halves itself (a single GPU or host memory). The local arithmetic is
the backend's: ``QsimShard`` holds the shard in the CUDA library (every gate one of its
kernels); other backends only need ``apply``, ``half`` and ``to_numpy``.
"""

import bisect
import math

import numpy as np

from . import State, qsim_expand

_SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


class LocalGate:
    """A gate in local positions for every shard: shard r applies it when its bits at
    `need_one` are all 1; `diag_bits` lists (target index, global bit j) of targets that sit
    on global qubits (diagonal gates only), whose matrix index bit is the shard's bit j."""

    def __init__(self, targets, controls, m, need_one=(), diag_bits=()):
        self.targets = list(targets)
        self.controls = list(controls)
        self.m = np.asarray(m, dtype=np.complex128)
        self.need_one = list(need_one)
        self.diag_bits = list(diag_bits)

    def for_shard(self, r):
        """(local targets, local controls, matrix) for shard r, or None when it skips."""
        if any(not (r >> j) & 1 for j in self.need_one):
            return None
        if not self.diag_bits:
            return self.targets, self.controls, self.m
        nt = len(self.targets)
        fixed = {ti: (r >> j) & 1 for ti, j in self.diag_bits}
        free = [ti for ti in range(nt) if ti not in fixed]
        d = np.diag(self.m)
        sub = np.zeros(1 << len(free), dtype=np.complex128)
        for s in range(1 << len(free)):
            idx = 0
            for ti in range(nt):  # target ti is bit nt - 1 - ti of the matrix index
                bit = fixed[ti] if ti in fixed else (s >> (len(free) - 1 - free.index(ti))) & 1
                idx |= bit << (nt - 1 - ti)
            sub[s] = d[idx]
        if free:
            return [self.targets[ti] for ti in free], self.controls, np.diag(sub)
        return None if sub[0] == 1 else ("phase", self.controls, sub[0])


class ShardPlanner:
    """Layout and schedule of an n-qubit state over 2^g shards (no data, no device)."""

    def __init__(self, n, g):
        if g < 0 or g >= n:
            raise ValueError("need 0 <= g < n")
        self.n, self.g, self.L = n, g, n - g
        self.pos = list(range(n))  # logical qubit -> position
        self.at = list(range(n))   # position -> logical qubit
        self.exchanges = 0
        self.local_swaps = 0

    def _swap_positions(self, a, b):
        qa, qb = self.at[a], self.at[b]
        self.at[a], self.at[b] = qb, qa
        self.pos[qa], self.pos[qb] = b, a

    def plan(self, gates):
        """Steps for a gate list [(targets, controls, matrix), ...] (logical qubits):
        ("gate", LocalGate) and ("exchange", j)."""
        steps = []
        occ = [[] for _ in range(self.n)]  # gate indices using each logical qubit
        for k, (t, c, _) in enumerate(gates):
            for q in set(t) | set(c):
                occ[q].append(k)

        def next_use(q, i):
            j = bisect.bisect_right(occ[q], i)
            return occ[q][j] if j < len(occ[q]) else len(gates) + q  # never again: furthest

        for i, (targets, controls, m) in enumerate(gates):
            m = np.asarray(m, dtype=np.complex128)
            diagonal = np.count_nonzero(m - np.diag(np.diag(m))) == 0
            glob_t = [q for q in targets if self.pos[q] >= self.L]
            if glob_t and not diagonal:
                busy = set(targets) | set(controls)
                for q in glob_t:
                    cand = [p for p in range(self.L) if self.at[p] not in busy]
                    if not cand:
                        raise ValueError("gate %d: no free local qubit to swap with" % i)
                    v = max(cand, key=lambda p: (next_use(self.at[p], i), p))
                    top = self.L - 1
                    if v != top:  # bring the victim to the top local position
                        steps.append(("gate", LocalGate([v, top], [], _SWAP)))
                        self.local_swaps += 1
                        self._swap_positions(v, top)
                    j = self.pos[q] - self.L
                    steps.append(("exchange", j))
                    self.exchanges += 1
                    self._swap_positions(top, self.pos[q])
            t_loc, diag_bits = [], []
            for ti, q in enumerate(targets):
                p = self.pos[q]
                if p >= self.L:
                    diag_bits.append((ti, p - self.L))
                t_loc.append(p if p < self.L else -1)
            c_loc = [self.pos[c] for c in controls if self.pos[c] < self.L]
            need_one = [self.pos[c] - self.L for c in controls if self.pos[c] >= self.L]
            steps.append(("gate", LocalGate(t_loc, c_loc, m, need_one, diag_bits)))
        return steps


def _apply_local(backend, spec, L):
    """Apply one shard's share of a LocalGate through the backend."""
    if spec is None:
        return
    targets, controls, m = spec
    if targets == "phase":  # a phase on the shard under the local controls
        ph = m
        spare = next(p for p in range(L) if p not in controls)
        backend.apply([spare], controls, np.diag([ph, ph]))
        return
    backend.apply(targets, controls, m)


class LocalShards:
    """All 2^g shards of one state in one process; exchanges swap the halves in place."""

    def __init__(self, n, g, backends):
        if len(backends) != 1 << g:
            raise ValueError("need 2^g shard backends")
        self.planner = ShardPlanner(n, g)
        self.shards = backends

    def run_gates(self, gates):
        P = self.planner
        for kind, arg in P.plan(gates):
            if kind == "gate":
                for r, b in enumerate(self.shards):
                    _apply_local(b, arg.for_shard(r), P.L)
            else:
                j = arg
                for r, b in enumerate(self.shards):
                    partner = r ^ (1 << j)
                    if partner < r:
                        continue
                    # r has bit j = 0: it keeps its half 0 and gives half 1; the partner
                    # (bit j = 1) gives its half 0
                    mine, theirs = b.half(1), self.shards[partner].half(0)
                    tmp = mine.copy_out()
                    mine.copy_in(theirs.copy_out())
                    theirs.copy_in(tmp)
        for b in self.shards:
            b.sync()

    def to_numpy(self):
        """The whole state in logical index order (host)."""
        P = self.planner
        parts = np.concatenate([b.to_numpy() for b in self.shards])  # physical order
        return _to_logical(parts, P)


class DistShard:
    """This process's shard of a state spread over a torch.distributed group of 2^g ranks."""

    def __init__(self, n, backend, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        world = dist.get_world_size(group)
        g = int(round(math.log2(world)))
        if 1 << g != world:
            raise ValueError("the group size must be a power of two")
        self.rank = dist.get_rank(group)
        self.planner = ShardPlanner(n, g)
        self.shard = backend

    def run_gates(self, gates):
        P = self.planner
        for kind, arg in P.plan(gates):
            if kind == "gate":
                _apply_local(self.shard, arg.for_shard(self.rank), P.L)
            else:
                self._exchange(arg)
        self.shard.sync()

    def _exchange(self, j):
        dist = self.dist
        partner = self.rank ^ (1 << j)
        b = (self.rank >> j) & 1
        half = self.shard.half(1 - b)
        send = half.tensor()
        recv = send.clone()
        peer = partner if self.group is None else dist.get_global_rank(self.group, partner)
        reqs = dist.batch_isend_irecv([dist.P2POp(dist.isend, send, peer, self.group),
                                       dist.P2POp(dist.irecv, recv, peer, self.group)])
        for q in reqs:
            q.wait()
        half.set_tensor(recv)

    def gather(self):
        """The whole state on every rank, in logical order (host; small states only)."""
        import torch
        dist = self.dist
        mine = torch.from_numpy(np.ascontiguousarray(self.shard.to_numpy()).view(np.float64).copy())
        parts = [torch.zeros_like(mine) for _ in range(dist.get_world_size(self.group))]
        dist.all_gather(parts, mine, group=self.group)
        phys = np.concatenate([p.numpy().view(np.complex128) for p in parts])
        return _to_logical(phys, self.planner)


def _to_logical(phys, P):
    """Reorder a state from physical positions (position p = index bit p) to logical order."""
    n = P.n
    t = phys.reshape([2] * n)  # axis a <-> position n - 1 - a
    # logical qubit q is at position pos[q]: axis of q = n - 1 - pos[q]
    axes = [n - 1 - P.pos[n - 1 - a] for a in range(n)]
    return np.ascontiguousarray(np.transpose(t, axes)).reshape(-1)


class _Half:
    """Half of a shard held by the CUDA library (a view of its device buffer)."""

    def __init__(self, view):
        self.view = view

    def tensor(self):
        import torch
        return torch.view_as_real(self.view).contiguous() if self.view.is_complex() else self.view

    def set_tensor(self, t):
        import torch
        self.view.copy_(torch.view_as_complex(t) if self.view.is_complex() else t)

    def copy_out(self):
        return self.view.clone()

    def copy_in(self, src):
        self.view.copy_(src)


class QsimShard:
    """A shard held by the CUDA library: a qsim state of L qubits on the current device.
    Gates run as its kernels; a half is a view of its buffer after qsim_canonicalize
    (plain amplitudes in local index order)."""

    def __init__(self, L, dtype="c128", first=True):
        """The shard of |0...0>: amplitude 1 at local index 0 of the first shard, zeros in
        every other one."""
        self.L = L
        self.st = State(L, dtype)
        if not first:
            self.st.tensor.zero_()

    def apply(self, targets, controls, m):
        m = np.asarray(m, dtype=np.complex128)
        if len(targets) <= 2:
            self.st.apply_gate(list(targets), m, list(controls))
        else:
            self.st.run_circuit([("MATRIX", tuple(targets), (), m)] if not controls else
                                [("CONTROL", tuple(controls), ())] + [("MATRIX", tuple(targets), (), m)] +
                                [("ENDCONTROL", (), ())])

    def half(self, v):
        self.st.canonicalize()
        h = 1 << (self.L - 1)
        return _Half(self.st.tensor[v * h:(v + 1) * h])

    def sync(self):
        self.st.canonicalize()

    def to_numpy(self):
        return self.st.to_numpy().astype(np.complex128)

    def close(self):
        self.st.close()


def expand_for_shards(n, ops):
    """The gate list of `ops` as (targets, controls, matrix) triples (qsim_expand)."""
    return [(t, c, m) for t, c, m, _ in qsim_expand(n, ops)]
