"""Python binding of libqsim, the GB300 full-amplitude state-vector library.

Argument marshalling only: every step of the computation runs in the CUDA library
(``csrc/``) behind the C ABI declared in ``include/qsim.h``. The functions below carry the
same names as the C entry points. PyTorch is used for device memory and streams: a
``State`` can own a torch tensor that holds its amplitudes, and calls are ordered on the
current torch CUDA stream.

The library must have been built (``paper_2008_07140_gb300.build.build()`` or
``__graft_entry__.build()``); importing the binding without it raises at first use.
There is no CPU fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsim.so")

QSIM_C64 = 0
QSIM_C128 = 1
DTYPES = {"c64": QSIM_C64, "c128": QSIM_C128, QSIM_C64: QSIM_C64, QSIM_C128: QSIM_C128}

STATUS = {0: "QSIM_OK", 1: "QSIM_EINVAL", 2: "QSIM_ENOMEM", 3: "QSIM_ECUDA", 4: "QSIM_ETIMEOUT",
          5: "QSIM_EUNSUPPORTED"}

OP_KINDS = {"MATRIX": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "T": 6, "SX": 7, "SY": 8,
            "RX": 9, "RY": 10, "RZ": 11, "U4": 12, "CNOT": 13, "CZ": 14, "CR": 15, "SWAP": 16,
            "ISWAP": 17, "TOFFOLI": 18, "DAGGER": 32, "ENDDAGGER": 33, "CONTROL": 34,
            "ENDCONTROL": 35}

# C-ABI symbols declared in include/qsim.h (checked by the export test)
EXPORTS = ["qsim_create", "qsim_wrap", "qsim_destroy", "qsim_reset", "qsim_set_stream",
           "qsim_synchronize", "qsim_canonicalize", "qsim_apply_gate", "qsim_apply_fused",
           "qsim_run_circuit", "qsim_last_run_stats", "qsim_amplitude", "qsim_probabilities",
           "qsim_sample", "qsim_measure", "qsim_norm", "qsim_inner", "qsim_fidelity", "qsim_expect_z",
           "qsim_copy_to_host", "qsim_copy_from_host", "qsim_gate_matrix", "qsim_last_error",
           "qsim_version", "qsim_probabilities_noalloc", "qsim_set_option",
           "qsim_run_trajectories", "qsim_autotune", "qsim_selftest_bounded_wait",
           "qsim_plan_dry_run", "qsim_partial_plan", "qsim_partial_amplitudes", "qsim_traj_prepare",
           "qsim_traj_set_seed", "qsim_traj_launch", "qsim_traj_results", "qsim_traj_state",
           "qsim_traj_destroy", "qsim_expand", "qsim_copy_to_host_async"]

TRAJ_MAX_QUBITS = 24


class QsimError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nq", ctypes.c_int32), ("qubits", ctypes.c_int32 * 3),
                ("nc", ctypes.c_int32), ("controls", ctypes.POINTER(ctypes.c_int32)),
                ("params", ctypes.c_double * 4), ("matrix", ctypes.POINTER(ctypes.c_double))]


class RunOpts(ctypes.Structure):
    _fields_ = [("fuse", ctypes.c_int32), ("remap", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("no_renorm", ctypes.c_int32), ("merge_diagonals", ctypes.c_int32)]


class TrajBatch(ctypes.Structure):
    _fields_ = [("nprog", ctypes.c_int32), ("prog_qubits", ctypes.POINTER(ctypes.c_int32)),
                ("prog_ops", ctypes.POINTER(ctypes.POINTER(Op))), ("prog_nops", ctypes.POINTER(ctypes.c_size_t)),
                ("ntraj", ctypes.c_int32), ("traj_prog", ctypes.POINTER(ctypes.c_int32)),
                ("seed", ctypes.c_uint64), ("channels", ctypes.c_uint32), ("noisy_kinds", ctypes.c_uint32),
                ("p", ctypes.c_double * 6), ("kron", ctypes.c_int32), ("shots", ctypes.c_int32),
                ("event_cap", ctypes.c_int32)]


# Eq. (5) channels by number (QSIM_NOISE_*), in the order they run at a noisy site
NOISE_CHANNELS = ("depolarizing", "amplitude_damping", "bit_flip", "phase_flip", "bit_phase_flip",
                  "phase_damping")


class PartialOpts(ctypes.Structure):
    _fields_ = [("cut", ctypes.c_int32), ("dtype", ctypes.c_int32), ("fuse", ctypes.c_int32),
                ("remap", ctypes.c_int32)]


class PartialInfo(ctypes.Structure):
    _fields_ = [("cut", ctypes.c_int32), ("decomposed", ctypes.c_int32), ("subcircuits", ctypes.c_int64),
                ("segment_runs", ctypes.c_int64), ("slots", ctypes.c_int32), ("gates_applied", ctypes.c_double),
                ("gates_unshared", ctypes.c_double), ("sweeps", ctypes.c_int64), ("remaps", ctypes.c_int64)]


class RunStats(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("fused_blocks", ctypes.c_int64), ("remaps", ctypes.c_int64),
                ("kernels", ctypes.c_int64), ("bytes", ctypes.c_double),
                ("fuse_width", ctypes.c_int64), ("predicted_ms", ctypes.c_double),
                ("phase_gates", ctypes.c_int64), ("epilogue_remaps", ctypes.c_int64),
                ("plan_reused", ctypes.c_int64), ("fp64_fallback", ctypes.c_int64),
                ("upload_bytes", ctypes.c_int64), ("diag_sweeps", ctypes.c_int64),
                ("diag_gates", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libqsim (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqsim.so is not built; run paper_2008_07140_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)
        sig = {
            "qsim_create": [I, I, P, ctypes.POINTER(P)],
            "qsim_wrap": [P, I, I, P, ctypes.POINTER(P)],
            "qsim_reset": [P], "qsim_set_stream": [P, P], "qsim_synchronize": [P],
            "qsim_canonicalize": [P],
            "qsim_apply_gate": [P, P, I, P, I, P],
            "qsim_apply_fused": [P, P, I, P],
            "qsim_run_circuit": [P, P, ctypes.c_size_t, P],
            "qsim_last_run_stats": [P, P],
            "qsim_amplitude": [P, U64, P],
            "qsim_probabilities": [P, P, I, P],
            "qsim_sample": [P, P, I, U64, U64, P],
            "qsim_measure": [P, I, ctypes.c_double, ctypes.POINTER(I), D],
            "qsim_norm": [P, D], "qsim_inner": [P, P, P], "qsim_fidelity": [P, P, D],
            "qsim_expect_z": [P, P], "qsim_copy_to_host": [P, P], "qsim_copy_from_host": [P, P],
            "qsim_copy_to_host_async": [P, P],
            "qsim_gate_matrix": [I, P, ctypes.POINTER(I), P],
            "qsim_probabilities_noalloc": [P, I, I, P, I, P, P],
            "qsim_set_option": [P, I, I],
            "qsim_run_trajectories": [P, P, P, P, P, P],
            "qsim_traj_prepare": [P, P, ctypes.c_int32, P, ctypes.POINTER(P)],
            "qsim_traj_set_seed": [P, U64],
            "qsim_traj_launch": [P, P],
            "qsim_traj_results": [P, P, P, P, P, P],
            "qsim_traj_state": [P, ctypes.c_int32, P, P],
            "qsim_partial_plan": [I, P, ctypes.c_size_t, I, P],
            "qsim_partial_amplitudes": [I, P, ctypes.c_size_t, P, P, ctypes.c_size_t, P, P, P],
            "qsim_autotune": [P, P, I],
            "qsim_selftest_bounded_wait": [I, P],
            "qsim_plan_dry_run": [I, I, P, ctypes.c_size_t, P, P],
            "qsim_expand": [I, P, ctypes.c_size_t, P, ctypes.c_size_t, P, ctypes.c_size_t, P, ctypes.c_size_t,
                            P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.qsim_destroy.argtypes = [P]
        L.qsim_destroy.restype = None
        L.qsim_traj_destroy.argtypes = [P]
        L.qsim_traj_destroy.restype = None
        L.qsim_last_error.restype = ctypes.c_char_p
        L.qsim_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise QsimError(status, lib().qsim_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---- same-name wrappers ---------------------------------------------------------------

def qsim_version():
    return lib().qsim_version().decode()


def qsim_last_error():
    return lib().qsim_last_error().decode()


def qsim_gate_matrix(name, params=()):
    p = np.zeros(4)
    p[:len(params)] = params
    out = np.zeros(2 * 64)
    k = ctypes.c_int()
    _check(lib().qsim_gate_matrix(OP_KINDS[name.upper()], _ptr(p), ctypes.byref(k), _ptr(out)))
    d = 1 << k.value
    m = out[:2 * d * d].reshape(d, d, 2)
    return k.value, m[..., 0] + 1j * m[..., 1]


def ops_to_c(ops):
    """Marshal a gate list [(name, qubits, params)] or [(name, qubits, params, matrix)]
    into a ctypes array of qsim_op; returns (array, keep-alive list)."""
    arr = (Op * max(len(ops), 1))()
    keep = []
    for i, op in enumerate(ops):
        name, qubits, params = op[0], op[1], op[2]
        o = arr[i]
        o.kind = OP_KINDS[name.upper()]
        o.nq = len(qubits)
        for j, q in enumerate(qubits):
            o.qubits[j] = q
        for j, v in enumerate(params):
            o.params[j] = v
        if len(op) > 3 and op[3] is not None:
            m = np.ascontiguousarray(np.asarray(op[3], dtype=np.complex128)).view(np.float64)
            keep.append(m)
            o.matrix = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return arr, keep


class GateRec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nt", ctypes.c_int32), ("targets", ctypes.c_int32 * 5),
                ("nc", ctypes.c_int32), ("ctrl_off", ctypes.c_int32), ("mat_off", ctypes.c_int64)]


def qsim_expand(n, ops):
    """The gate list qsim_run_circuit applies (blocks expanded, controlled gates in
    (target, controls) form): a list of (targets, controls, matrix, kind name)."""
    arr, keep = ops_to_c(ops)
    sizes = (ctypes.c_size_t * 3)()
    _check(lib().qsim_expand(n, arr, len(ops), None, 0, None, 0, None, 0, sizes))
    ng, nc, nm = sizes[0], sizes[1], sizes[2]
    recs = (GateRec * max(ng, 1))()
    ctl = np.zeros(max(nc, 1), dtype=np.int32)
    mats = np.zeros(2 * max(nm, 1))
    _check(lib().qsim_expand(n, arr, len(ops), recs, ng, _ptr(ctl), nc, _ptr(mats), nm, sizes))
    del keep
    names = {v: k for k, v in OP_KINDS.items()}
    out = []
    for i in range(ng):
        r = recs[i]
        d = 1 << r.nt
        m = mats[2 * r.mat_off:2 * (r.mat_off + d * d)].reshape(d, d, 2)
        out.append((tuple(r.targets[:r.nt]), tuple(int(c) for c in ctl[r.ctrl_off:r.ctrl_off + r.nc]),
                    m[..., 0] + 1j * m[..., 1], names.get(r.kind, "MATRIX")))
    return out


def qsim_plan_dry_run(n, dtype, ops, fuse=5, remap=True, merge_diagonals=False):
    """Host-only planning statistics of a circuit (no device needed)."""
    arr, keep = ops_to_c(ops)
    o = RunOpts(fuse, 1 if remap else 0, 0, 0, 1 if merge_diagonals else 0)
    st = RunStats()
    _check(lib().qsim_plan_dry_run(n, DTYPES[dtype], arr, len(ops), ctypes.byref(o), ctypes.byref(st)))
    del keep
    return {f: getattr(st, f) for f, _ in RunStats._fields_}


def qsim_autotune(stream=None):
    """Device microbenchmarks of the autotuner; returns the measured table as a dict."""
    out = np.zeros(11)
    if stream is None:
        stream = _current_stream()
    _check(lib().qsim_autotune(stream, _ptr(out), 11))
    keys = ["gbs_pair_c64", "gbs_pair_df_c128", "gbs_fused_k4", "gbs_fused_k5", "gbs_remap", "launch_us",
            "pair_blocks_per_sm", "gbs_fused_df_k2", "gbs_fused_df_k3", "gbs_fused_df_k4", "gbs_fused_df_k5"]
    return {k: float(v) for k, v in zip(keys, out)}


class _Batch:
    """A qsim_traj_batch with the arrays it points to kept alive."""

    def __init__(self, programs, traj_prog, seed, p_depol=0.0, gamma=0.0, shots=0, event_cap=0, noise=None,
                 noisy=None, kron=False):
        chans = {}
        if p_depol != 0:  # 0 disables; anything else goes to the library's range check
            chans[0] = p_depol
        if gamma != 0:
            chans[1] = gamma
        for name, p in (noise or {}).items():
            chans[NOISE_CHANNELS.index(name)] = p
        mask = sum(1 << c for c in chans)
        pv = (ctypes.c_double * 6)(*[chans.get(c, 0.0) for c in range(6)])
        kinds = 0 if noisy is None else sum(1 << OP_KINDS[name.upper()] for name in noisy)
        if noisy is not None and kinds == 0:
            mask = 0  # no gate class is noisy
        nprog = len(programs)
        self.arrays, self.keeps = [], []
        for _, ops in programs:
            arr, keep = ops_to_c(ops)
            self.arrays.append(arr)
            self.keeps.append(keep)
        self.ops_ptrs = (ctypes.POINTER(Op) * nprog)(*[ctypes.cast(a, ctypes.POINTER(Op)) for a in self.arrays])
        self.widths = (ctypes.c_int32 * nprog)(*[w for w, _ in programs])
        self.nops = (ctypes.c_size_t * nprog)(*[len(ops) for _, ops in programs])
        self.ntraj = len(traj_prog)
        self.tp = (ctypes.c_int32 * self.ntraj)(*traj_prog)
        self.shots, self.event_cap = shots, event_cap
        self.b = TrajBatch(nprog, self.widths, self.ops_ptrs, self.nops, self.ntraj, self.tp, seed, mask, kinds,
                           pv, 1 if kron else 0, shots, event_cap)

    def outputs(self):
        return (np.zeros((self.ntraj, TRAJ_MAX_QUBITS)), np.zeros(max(self.shots, 1), dtype=np.uint64),
                np.zeros((self.ntraj, max(self.event_cap, 1)), dtype=np.uint32),
                np.zeros(self.ntraj, dtype=np.int32))

    def unpack(self, zexp, samples, events, nev):
        ev_lists = []
        for t in range(self.ntraj):
            lst = []
            for e in range(min(int(nev[t]), self.event_cap)):
                c = int(events[t, e])
                lst.append((c >> 12, (c >> 6) & 63, (c >> 2) & 15, c & 3))
            ev_lists.append(lst)
        return zexp, samples[:self.shots], ev_lists, nev


def qsim_run_trajectories(programs, traj_prog, seed, p_depol=0.0, gamma=0.0, shots=0, event_cap=0, stream=None,
                          noise=None, noisy=None, kron=False):
    """Run noisy trajectories. programs: list of (n_qubits, gate list). Depolarizing runs
    with p_depol and amplitude damping with gamma when they are not 0; `noise` maps further
    channel names (NOISE_CHANNELS) to their p; `noisy` is the set of instruction names
    whose gates are noisy (None: every gate); kron selects joint two-qubit draws. Returns
    (zexp [ntraj, n_max], samples [shots], events list per trajectory as tuples
    (gate, qubit, channel, branch), event counts)."""
    bt = _Batch(programs, traj_prog, seed, p_depol, gamma, shots, event_cap, noise, noisy, kron)
    zexp, samples, events, nev = bt.outputs()
    if stream is None:
        stream = _current_stream()
    _check(lib().qsim_run_trajectories(ctypes.byref(bt.b), stream, _ptr(zexp), _ptr(samples), _ptr(events),
                                       _ptr(nev)))
    return bt.unpack(zexp, samples, events, nev)


class TrajPlan:
    """A prepared trajectory batch (qsim_traj_prepare): launch() records one kernel launch
    on the stream (capturable into a CUDA graph), results() reads the outputs back, state(i)
    the final state of the i-th kept trajectory. Same arguments as qsim_run_trajectories,
    plus `keep`, the trajectories whose final states stay on the device."""

    def __init__(self, programs, traj_prog, seed, p_depol=0.0, gamma=0.0, shots=0, event_cap=0, noise=None,
                 noisy=None, kron=False, keep=(), stream=None):
        self.batch = _Batch(programs, traj_prog, seed, p_depol, gamma, shots, event_cap, noise, noisy, kron)
        self.keep = list(keep)
        self.keep_w = [programs[traj_prog[t]][0] for t in self.keep]
        kp = (ctypes.c_int32 * max(len(self.keep), 1))(*self.keep)
        self.handle = ctypes.c_void_p()
        self.stream = _current_stream() if stream is None else stream
        _check(lib().qsim_traj_prepare(ctypes.byref(self.batch.b), kp, len(self.keep), self.stream,
                                       ctypes.byref(self.handle)))

    def set_seed(self, seed):
        _check(lib().qsim_traj_set_seed(self.handle, seed))

    def launch(self, stream=None):
        _check(lib().qsim_traj_launch(self.handle, self.stream if stream is None else stream))

    def results(self, stream=None):
        zexp, samples, events, nev = self.batch.outputs()
        _check(lib().qsim_traj_results(self.handle, self.stream if stream is None else stream, _ptr(zexp),
                                       _ptr(samples), _ptr(events), _ptr(nev)))
        return self.batch.unpack(zexp, samples, events, nev)

    def state(self, i, stream=None):
        out = np.zeros(1 << self.keep_w[i], dtype=np.complex64)
        _check(lib().qsim_traj_state(self.handle, i, self.stream if stream is None else stream, _ptr(out)))
        return out

    def close(self):
        if self.handle:
            lib().qsim_traj_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _info_dict(info):
    return {k: getattr(info, k) for k, _ in PartialInfo._fields_}


def qsim_partial_plan(n, ops, cut=0):
    """Host-only decomposition of the partial amplitude mode (Section 2.2): the plan's
    cut, decomposed-gate count c, 2^(c+1) sub-circuits, segment runs and slots."""
    arr, keep = ops_to_c(ops)
    info = PartialInfo()
    _check(lib().qsim_partial_plan(n, arr, len(ops), cut, ctypes.byref(info)))
    del keep
    return _info_dict(info)


def qsim_partial_amplitudes(n, ops, indices, cut=0, dtype="c128", fuse=0, remap=False, stream=None):
    """Amplitudes <x|psi> for the indices x by the partial amplitude mode on the GPU.
    Returns (complex128 array, plan info dict)."""
    arr, keep = ops_to_c(ops)
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.zeros(2 * max(len(idx), 1))
    o = PartialOpts(cut, DTYPES[dtype], fuse, 1 if remap else 0)
    info = PartialInfo()
    if stream is None:
        stream = _current_stream()
    _check(lib().qsim_partial_amplitudes(n, arr, len(ops), ctypes.byref(o), _ptr(idx), len(idx), _ptr(out),
                                         ctypes.byref(info), stream))
    del keep
    return out[:2 * len(idx)].view(np.complex128), _info_dict(info)


class State:
    """An n-qubit state on the current CUDA device (a torch tensor holds the amplitudes)."""

    def __init__(self, n, dtype="c64", stream=None, tensor=None):
        import torch
        self.n = n
        self.dtype = DTYPES[dtype]
        tdt = torch.complex64 if self.dtype == QSIM_C64 else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        self.tensor = tensor
        self.stream = stream if stream is not None else _current_stream()
        h = ctypes.c_void_p()
        _check(lib().qsim_wrap(ctypes.c_void_p(tensor.data_ptr()), n, self.dtype, self.stream,
                               ctypes.byref(h)))
        self.handle = h
        _check(lib().qsim_reset(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().qsim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- gates
    def apply_gate(self, targets, matrix, controls=()):
        m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128)).view(np.float64)
        t = np.array(targets, dtype=np.int32)
        c = np.array(controls, dtype=np.int32) if len(controls) else np.zeros(1, dtype=np.int32)
        _check(lib().qsim_apply_gate(self.handle, _ptr(t), len(targets), _ptr(c), len(controls), _ptr(m)))

    def apply_fused(self, qubits, u):
        m = np.ascontiguousarray(np.asarray(u, dtype=np.complex128)).view(np.float64)
        q = np.array(qubits, dtype=np.int32)
        _check(lib().qsim_apply_fused(self.handle, _ptr(q), len(qubits), _ptr(m)))

    def run_circuit(self, ops, fuse=0, remap=True, use_graph=False, renorm=True, merge_diagonals=False):
        arr, keep = ops_to_c(ops)
        o = RunOpts(fuse, 1 if remap else 0, 1 if use_graph else 0, 0 if renorm else 1,
                    1 if merge_diagonals else 0)
        _check(lib().qsim_run_circuit(self.handle, arr, len(ops), ctypes.byref(o)))
        del keep

    def stats(self):
        st = RunStats()
        _check(lib().qsim_last_run_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in RunStats._fields_}

    def reset(self):
        _check(lib().qsim_reset(self.handle))

    def set_fp64_native(self, on=True):
        """complex128 only: run gates with FP64 instructions on plain doubles (default:
        the FP64-accurate split format on the FP32 pipe)."""
        _check(lib().qsim_set_option(self.handle, 1, 1 if on else 0))

    def set_tc_lo_smem(self, on=True):
        """complex64 fused tensor-core apply: keep the low TF32 part of each tile in shared
        memory (three loads in flight) instead of tensor memory (the default)."""
        _check(lib().qsim_set_option(self.handle, 2, 1 if on else 0))

    def synchronize(self):
        _check(lib().qsim_synchronize(self.handle))

    def canonicalize(self):
        _check(lib().qsim_canonicalize(self.handle))

    # -- read-outs
    def amplitude(self, index):
        out = np.zeros(2)
        _check(lib().qsim_amplitude(self.handle, index, _ptr(out)))
        return complex(out[0], out[1])

    def probabilities(self, qubits):
        q = np.array(qubits, dtype=np.int32)
        out = np.zeros(1 << len(qubits))
        _check(lib().qsim_probabilities(self.handle, _ptr(q), len(qubits), _ptr(out)))
        return out

    def sample(self, shots, seed, qubits=None):
        out = np.zeros(shots, dtype=np.uint64)
        if qubits:
            q = np.array(qubits, dtype=np.int32)
            _check(lib().qsim_sample(self.handle, _ptr(q), len(qubits), shots, seed, _ptr(out)))
        else:
            _check(lib().qsim_sample(self.handle, None, 0, shots, seed, _ptr(out)))
        return out

    def measure(self, qubit, u):
        """MEASURE (App. A-1): returns (outcome, its probability); the state collapses."""
        r = ctypes.c_int()
        pr = ctypes.c_double()
        _check(lib().qsim_measure(self.handle, qubit, float(u), ctypes.byref(r), ctypes.byref(pr)))
        return r.value, pr.value

    def norm(self):
        out = ctypes.c_double()
        _check(lib().qsim_norm(self.handle, ctypes.byref(out)))
        return out.value

    def inner(self, other):
        out = np.zeros(2)
        _check(lib().qsim_inner(self.handle, other.handle, _ptr(out)))
        return complex(out[0], out[1])

    def fidelity(self, other):
        out = ctypes.c_double()
        _check(lib().qsim_fidelity(self.handle, other.handle, ctypes.byref(out)))
        return out.value

    def expect_z(self):
        out = np.zeros(self.n)
        _check(lib().qsim_expect_z(self.handle, _ptr(out)))
        return out

    def to_numpy(self):
        dt = np.complex64 if self.dtype == QSIM_C64 else np.complex128
        out = np.zeros(1 << self.n, dtype=dt)
        _check(lib().qsim_copy_to_host(self.handle, _ptr(out)))
        return out

    def from_numpy(self, psi):
        dt = np.complex64 if self.dtype == QSIM_C64 else np.complex128
        a = np.ascontiguousarray(psi, dtype=dt)
        _check(lib().qsim_copy_from_host(self.handle, _ptr(a)))
        self.synchronize()
