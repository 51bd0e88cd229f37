"""FP64 CPU oracle for the full-amplitude state-vector method.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run anything in this package. The CUDA library never
calls it, and the two share no code; the one common input is the gate-name list made by
the seeded generators in ``synth``.

What it computes (paper: Wang et al., "A quantum circuit simulator and its applications
on Sunway TaihuLight supercomputer"):

* gate matrices of the instruction set (Appendix A-1), plus SX and SY for the random
  circuits (principal square roots, not in the paper);
* DAGGER / CONTROL block expansion (Appendix A-1);
* state evolution by Eq. (2) / Eq. (3) and the k-qubit generalisation (``qsim_oracle.c``);
* PMEASURE probabilities (Appendix A-1, outcome strings as printed in Appendix A-2) and
  MEASURE with collapse (Appendix A-1);
* sampling, Z expectations, norm and inner products;
* the partial amplitude mode (Section 2.2): crossing controlled gates split by Eq. (4),
  2^(c+1) sub-circuits simulated independently and recombined;
* the noisy-gate procedure of Section 2.4 with the six Kraus sets of Eq. (5) (per qubit,
  or jointly over the Kronecker products for two-qubit gates; noise on chosen gate
  classes), driven by Philox4x32-10 draws; and an exact density-matrix evolution for
  small n.

Parity status of each function is listed in ``parity_status``; every entry is pinned by
a ``-m "not gpu"`` test in ``tests/test_oracle_pins.py`` unless it says otherwise.
"""

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

parity_status = {
    "gate_matrix": "pinned (unitarity, SX^2 = X, SY^2 = Y, Appendix A-2 example)",
    "apply": "pinned (Kronecker brute force n <= 10, GHZ, QFT closed form)",
    "expand": "pinned (circuit then DAGGER returns |0..0>, Appendix A-2 example)",
    "probabilities": "pinned (Appendix A-2 printed output, brute force marginals)",
    "sample": "pinned (brute-force inverse CDF on tiny states)",
    "philox": "pinned (Random123 known-answer vectors, cuRAND host generator stream)",
    "trajectory": "pinned (density-matrix average within 3 sigma for all six Eq. 5 channels, per "
                  "qubit and Kronecker joint draws; p = 0 reduces to noiseless; phase-damping "
                  "branch states in closed form; branch frequencies binomial 4 sigma)",
    "density_matrix": "pinned (trace 1, Kraus completeness, noiseless = pure state, one-qubit "
                      "closed forms of every channel)",
    "inner": "pinned (closed forms <i0|0> = -i, <0|i0> = i, <+^n|0^n> = 2^(-n/2), a phase; "
             "numpy.vdot on random states)",
    "reduced_density": "pinned (numpy transpose-and-contract construction, every placement of "
                       "one to three qubits)",
    "measure": "pinned (Bell-state outcomes and collapse, Kronecker-built projectors)",
    "partial_decompose": "pinned (recombined state = full simulation for CZ / CNOT / CR / "
                         "TOFFOLI / CONTROL crossings, 2^(c+1) sub-circuits, SWAP rejected)",
    "partial_amplitudes": "pinned (equal to the full simulation at sampled indices)",
}


def build(force: bool = False) -> str:
    """Compile ``qsim_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i = ctypes.c_int
        u64 = ctypes.c_uint64
        lib.or_apply_1q.argtypes = [P, i, i, u64, P]
        lib.or_apply_kq.argtypes = [P, i, P, i, u64, P]
        lib.or_norm2.argtypes = [P, i]
        lib.or_norm2.restype = ctypes.c_double
        lib.or_reduced_density.argtypes = [P, i, P, i, P]
        lib.or_inner.argtypes = [P, P, i, P]
        lib.or_probabilities.argtypes = [P, i, P, i, P]
        lib.or_z_sums.argtypes = [P, i, P]
        lib.or_sample.argtypes = [P, i, P, ctypes.c_int64, P]
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_philox_many.argtypes = [P, ctypes.c_int64, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------------------
# Gate library (Appendix A-1). Matrices are complex128, row-major; for multi-qubit gates
# the first listed qubit is the most significant bit of the row/column index.
# --------------------------------------------------------------------------------------

def gate_matrix(name, params=()):
    """Matrix of a named gate; returns (number of qubits the matrix acts on, matrix)."""
    name = name.upper()
    s2 = math.sqrt(2.0) / 2.0
    if name == "H":
        return 1, np.array([[s2, s2], [s2, -s2]], dtype=complex)
    if name == "X":
        return 1, np.array([[0, 1], [1, 0]], dtype=complex)
    if name == "Y":
        return 1, np.array([[0, -1j], [1j, 0]], dtype=complex)
    if name == "Z":
        return 1, np.array([[1, 0], [0, -1]], dtype=complex)
    if name == "S":
        return 1, np.array([[1, 0], [0, 1j]], dtype=complex)
    if name == "T":
        return 1, np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=complex)
    if name == "SX":  # principal square root of X (random-circuit set; not in the paper)
        return 1, 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=complex)
    if name == "SY":  # principal square root of Y (random-circuit set; not in the paper)
        return 1, 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=complex)
    if name == "RX":
        th = params[0]
        c, s = math.cos(th / 2), math.sin(th / 2)
        return 1, np.array([[c, -1j * s], [-1j * s, c]], dtype=complex)
    if name == "RY":
        th = params[0]
        c, s = math.cos(th / 2), math.sin(th / 2)
        return 1, np.array([[c, -s], [s, c]], dtype=complex)
    if name == "RZ":
        th = params[0]
        return 1, np.array([[np.exp(-0.5j * th), 0], [0, np.exp(0.5j * th)]], dtype=complex)
    if name == "U4":
        if len(params) == 8:  # four complex elements given as (re, im) pairs
            u = [complex(params[2 * j], params[2 * j + 1]) for j in range(4)]
            return 1, np.array([[u[0], u[1]], [u[2], u[3]]], dtype=complex)
        a, b, g, d = params  # angle form
        c, s = math.cos(g / 2), math.sin(g / 2)
        return 1, np.array(
            [[np.exp(1j * (a - b / 2 - d / 2)) * c, -np.exp(1j * (a - b / 2 + d / 2)) * s],
             [np.exp(1j * (a + b / 2 - d / 2)) * s, np.exp(1j * (a + b / 2 + d / 2)) * c]],
            dtype=complex)
    if name == "CNOT":
        m = np.eye(4, dtype=complex)
        m[2:, 2:] = [[0, 1], [1, 0]]
        return 2, m
    if name == "CZ":
        return 2, np.diag([1, 1, 1, -1]).astype(complex)
    if name == "CR":
        return 2, np.diag([1, 1, 1, np.exp(1j * params[0])]).astype(complex)
    if name == "SWAP":
        return 2, np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    if name == "ISWAP":
        return 2, np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]],
                           dtype=complex)
    if name == "TOFFOLI":
        m = np.eye(8, dtype=complex)
        m[6:, 6:] = [[0, 1], [1, 0]]
        return 3, m
    raise ValueError("unknown gate %r" % name)


BLOCK_MARKERS = ("DAGGER", "ENDDAGGER", "CONTROL", "ENDCONTROL")


def expand(ops, names=False):
    """Flatten DAGGER / CONTROL blocks (Appendix A-1) into (qubits, controls, matrix), or
    (instruction name, qubits, controls, matrix) with names=True.

    DAGGER ... ENDDAGGER: the block M becomes M^dagger, i.e. its gates in reverse order,
    each conjugate-transposed. CONTROL i ... ENDCONTROL: qubit i becomes an extra control
    of every gate in the block. Both nest.
    """
    def parse(pos, end_marker):
        items = []
        while pos < len(ops):
            name, qubits, params = ops[pos]
            uname = name.upper()
            if uname == "DAGGER":
                inner, pos = parse(pos + 1, "ENDDAGGER")
                items.append(("dagger", inner))
            elif uname == "CONTROL":
                inner, pos = parse(pos + 1, "ENDCONTROL")
                items.append(("control", tuple(qubits), inner))
            elif uname in ("ENDDAGGER", "ENDCONTROL"):
                if uname != end_marker:
                    raise ValueError("unbalanced %s" % uname)
                return items, pos + 1
            else:
                k, m = gate_matrix(uname, params)
                if len(qubits) != k:
                    raise ValueError("%s acts on %d qubits" % (uname, k))
                items.append(("gate", tuple(qubits), m, uname))
                pos += 1
                continue
            continue
        if end_marker is not None:
            raise ValueError("missing %s" % end_marker)
        return items, pos

    def flatten(items, dag, ctrls):
        # Under an odd number of enclosing DAGGERs the items run in reverse order and
        # each is replaced by its adjoint; a nested DAGGER flips the parity again.
        out = []
        for it in (reversed(items) if dag else items):
            if it[0] == "gate":
                m = it[2].conj().T if dag else it[2]
                out.append((it[3], it[1], tuple(ctrls), m) if names else (it[1], tuple(ctrls), m))
            elif it[0] == "dagger":
                out.extend(flatten(it[1], not dag, ctrls))
            else:
                out.extend(flatten(it[2], dag, ctrls + list(it[1])))
        return out

    items, _ = parse(0, None)
    return flatten(items, False, [])


# --------------------------------------------------------------------------------------
# State evolution
# --------------------------------------------------------------------------------------

def zero_state(n):
    """QINIT n: |0...0> (Appendix A-1)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply(psi, n, qubits, controls, m):
    """Apply matrix m on `qubits` with `controls` (Eq. 2 / Eq. 3 and their k-qubit form)."""
    lib = _load()
    qubits = [int(q) for q in qubits]
    controls = [int(c) for c in controls]
    allq = qubits + controls
    if len(set(allq)) != len(allq) or any(q < 0 or q >= n for q in allq):
        raise ValueError("qubits must be distinct and in [0, n)")
    cmask = 0
    for c in controls:
        cmask |= 1 << c
    m = np.ascontiguousarray(m, dtype=np.complex128)
    if len(qubits) == 1:
        lib.or_apply_1q(_ptr(psi), n, qubits[0], cmask, _ptr(m))
    else:
        qs = np.array(qubits, dtype=np.int32)
        lib.or_apply_kq(_ptr(psi), n, _ptr(qs), len(qubits), cmask, _ptr(m))
    return psi


def run(n, ops, psi=None):
    """Evolve |0..0> (or psi) under the gate list `ops`; returns the final state."""
    if psi is None:
        psi = zero_state(n)
    for qubits, controls, m in expand(ops):
        apply(psi, n, qubits, controls, m)
    return psi


def norm2(psi, n):
    return _load().or_norm2(_ptr(psi), n)


def inner(a, b, n):
    out = np.zeros(2)
    _load().or_inner(_ptr(a), _ptr(b), n, _ptr(out))
    return complex(out[0], out[1])


def probabilities(psi, n, qubits):
    """PMEASURE: out[s], s = sum_j bit(qubits[j]) << (m-1-j) (first qubit leftmost)."""
    qs = np.array(qubits, dtype=np.int32)
    out = np.zeros(1 << len(qubits))
    _load().or_probabilities(_ptr(psi), n, _ptr(qs), len(qubits), _ptr(out))
    return out


def z_expectations(psi, n):
    """<Z_q> for every qubit, normalised by the state's norm."""
    out = np.zeros(n)
    _load().or_z_sums(_ptr(psi), n, _ptr(out))
    return out / norm2(psi, n)


def measure(psi, n, q, u):
    """MEASURE (App. A-1): measure qubit q and keep the post-measurement state. The outcome
    is the smallest r with u < P(0) + ... + P(r), P the marginal of q relative to the norm
    (the same branch rule as sampling and the noise draws); the state is projected onto it
    and renormalised. Returns (r, P(r), new state)."""
    bit = (np.arange(1 << n) >> q) & 1
    w = np.abs(psi) ** 2
    p = [float(w[bit == 0].sum()), float(w[bit == 1].sum())]
    tot = p[0] + p[1]
    r = 0 if u * tot < p[0] else 1
    out = np.where(bit == r, psi / math.sqrt(p[r]), 0.0).astype(np.complex128)
    return r, p[r] / tot, out


def project_bits(index, qubits):
    m = len(qubits)
    return sum(((int(index) >> q) & 1) << (m - 1 - j) for j, q in enumerate(qubits))


def sample(psi, n, u):
    """Basis indices by inverse CDF in index order, one per draw u in [0, 1)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(len(u), dtype=np.uint64)
    _load().or_sample(_ptr(psi), n, _ptr(u), len(u), _ptr(out))
    return out


# --------------------------------------------------------------------------------------
# Philox4x32-10 and the draw layout shared (by specification, not by code) with the GPU
# --------------------------------------------------------------------------------------

SAMPLE_TAG = 0x53414D50  # counter word 3 of a sampling draw


def philox(ctr, key):
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def philox_many(ctrs, key):
    c = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _load().or_philox_many(_ptr(c), len(c), _ptr(k), _ptr(out))
    return out


def seed_key(seed):
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def u01(x0, x1):
    """53-bit double in [0, 1) from two 32-bit words: ((x0 << 32 | x1) >> 11) * 2^-53."""
    return float((((int(x0) << 32) | int(x1)) >> 11)) * (2.0 ** -53)


def sample_draws(seed, shots):
    """Draw u_j for shot j: Philox(key = seed, counter = (j_lo, j_hi, 0, SAMPLE_TAG))."""
    ctrs = np.zeros((shots, 4), dtype=np.uint32)
    j = np.arange(shots, dtype=np.uint64)
    ctrs[:, 0] = (j & 0xFFFFFFFF).astype(np.uint32)
    ctrs[:, 1] = (j >> 32).astype(np.uint32)
    ctrs[:, 3] = SAMPLE_TAG
    x = philox_many(ctrs, seed_key(seed)).astype(np.uint64)
    return (((x[:, 0] << np.uint64(32)) | x[:, 1]) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


# --------------------------------------------------------------------------------------
# Noise (Section 2.4, Eq. 5)
# --------------------------------------------------------------------------------------

def kraus(channel, p):
    """Kraus operators of Eq. (5), in the order printed there."""
    I = np.eye(2, dtype=complex)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
    Z = np.array([[1, 0], [0, -1]], dtype=complex)
    if channel == "bit_flip":
        return [math.sqrt(p) * I, math.sqrt(1 - p) * X]
    if channel == "phase_flip":
        return [math.sqrt(p) * I, math.sqrt(1 - p) * Z]
    if channel == "bit_phase_flip":
        return [math.sqrt(p) * I, math.sqrt(1 - p) * Y]
    if channel == "amplitude_damping":
        return [np.array([[1, 0], [0, math.sqrt(1 - p)]], dtype=complex),
                np.array([[0, math.sqrt(p)], [0, 0]], dtype=complex)]
    if channel == "phase_damping":
        return [np.array([[1, 0], [0, math.sqrt(1 - p)]], dtype=complex),
                np.array([[0, 0], [0, math.sqrt(p)]], dtype=complex)]
    if channel == "depolarizing":
        return [math.sqrt(1 - 3 * p / 4) * I, math.sqrt(p) / 2 * X,
                math.sqrt(p) / 2 * Y, math.sqrt(p) / 2 * Z]
    raise ValueError(channel)


# Channel numbers: the order in which the channels run at one noisy site.
NOISE_CHANNELS = ("depolarizing", "amplitude_damping", "bit_flip", "phase_flip", "bit_phase_flip",
                  "phase_damping")
KRON_SITE = 0x4B524F4E  # counter word 2 of a joint two-qubit draw


def noise_sites(qubits, controls):
    """Qubits that get noise after a gate: every qubit it touches, ascending."""
    return sorted(set(qubits) | set(controls))


def noise_ctr(traj, gate, site, channel):
    """Counter of one noise draw: (trajectory, gate index, site, channel); the site is the
    qubit, or KRON_SITE for the joint draw of a two-qubit gate."""
    return (traj & 0xFFFFFFFF, gate & 0xFFFFFFFF, site & 0xFFFFFFFF, channel & 0xFFFFFFFF)


def noise_list(p_depol=0.0, gamma=0.0, noise=None):
    """[(channel number, name, p)] in channel order: depolarizing with p_depol and amplitude
    damping with gamma when they are > 0, then every entry {name: p} of `noise` (which
    may also name those two)."""
    chans = {}
    if p_depol > 0:
        chans["depolarizing"] = p_depol
    if gamma > 0:
        chans["amplitude_damping"] = gamma
    for name, p in (noise or {}).items():
        if name not in NOISE_CHANNELS:
            raise ValueError(name)
        if not 0.0 <= p <= 1.0:
            raise ValueError("p of %s outside [0, 1]" % name)
        chans[name] = p
    return [(c, name, chans[name]) for c, name in enumerate(NOISE_CHANNELS) if name in chans]


def reduced_density(psi, n, qs):
    """rho[r, c] = sum over the other qubits of psi_(r, rest) conj(psi_(c, rest)), qs[0] the
    most significant bit of r and c; ||(K on qs) psi||^2 = tr(K rho K^dag)."""
    k = len(qs)
    q = np.array(qs, dtype=np.int32)
    out = np.zeros((1 << k, 1 << k), dtype=np.complex128)
    _load().or_reduced_density(_ptr(psi), n, _ptr(q), k, _ptr(out))
    return out


def trajectory(n, ops, seed, traj, p_depol=0.0, gamma=0.0, near_tie=1e-9, noise=None, noisy=None,
               kron=False):
    """One Monte-Carlo trajectory of the noisy-gate procedure (Section 2.4).

    After each gate U (applied first) whose instruction name is in `noisy` (every gate when
    `noisy` is None), the channels of noise_list(p_depol, gamma, noise) act on every qubit
    the gate touches: for each such qubit q in ascending order and each channel in
    channel order,
      1. every Kraus operator K_i of Eq. (5) acts on the state: p_i = ||K_i psi||^2 /
         ||psi||^2, computed as tr(K_i rho K_i^dag) / tr(rho) from the reduced density
         matrix rho of q;
      2. a draw u = U01(Philox(seed, (traj, gate, q, channel)));
      3. the smallest i with u < p_1 + ... + p_i;
      4. psi <- K_i psi, normalised to ||psi||^2 = 1.
    With kron=True a two-qubit gate on qubits a < b instead draws once per channel, from
    (traj, gate, KRON_SITE, channel), over the Kronecker products K_i (x) K_j of Eq. (5)'s
    two-qubit rule, ordered i-major, K_i acting on b (the more significant bit) and K_j
    on a.
    Returns (final state, events (gate, qubit, channel, branch) with branch > 0 in gate
    order, number of draws within `near_tie` of a cumulative-probability boundary).
    """
    key = seed_key(seed)
    psi = zero_state(n)
    chans = noise_list(p_depol, gamma, noise)
    events = []
    ties = 0

    def choose(qs, Ks, u):
        rho = reduced_density(psi, n, qs)
        tot = float(np.real(np.trace(rho)))
        probs = [float(np.real(np.trace(K @ rho @ K.conj().T))) / tot for K in Ks]
        cdf = np.cumsum(probs)
        # smallest i with u < cdf_i; past the end (cdf rounded below u), the last branch of
        # positive probability
        br = next((i for i, c in enumerate(cdf) if u < c), max(i for i, q in enumerate(probs) if q > 0))
        tie = min((abs(u - c) for c in cdf[:-1]), default=1.0) < near_tie
        apply(psi, n, qs, [], Ks[br])
        psi[:] /= math.sqrt(norm2(psi, n))
        return br, tie

    def draw(g, site, c):
        x = philox(noise_ctr(traj, g, site, c), key)
        return u01(x[0], x[1])

    for g, (name, qubits, controls, m) in enumerate(expand(ops, names=True)):
        apply(psi, n, qubits, controls, m)
        if not chans or (noisy is not None and name not in noisy):
            continue
        sites = noise_sites(qubits, controls)
        if kron and len(sites) == 2:
            a, b = sites
            for c, cname, p in chans:
                Ks = kraus(cname, p)
                s = len(Ks)
                br, tie = choose([b, a], [np.kron(Ks[i], Ks[j]) for i in range(s) for j in range(s)],
                                 draw(g, KRON_SITE, c))
                ties += tie
                for q, bq in ((a, br % s), (b, br // s)):
                    if bq > 0:
                        events.append((g, q, c, bq))
            continue
        for q in sites:
            for c, cname, p in chans:
                br, tie = choose([q], kraus(cname, p), draw(g, q, c))
                ties += tie
                if br > 0:
                    events.append((g, q, c, br))
    return psi, events, ties


def trajectory_sample_draw(seed, traj, ngates):
    """Draw for the one shot taken from a trajectory: counter (traj, ngates, 0, SAMPLE_TAG)."""
    x = philox((traj & 0xFFFFFFFF, ngates & 0xFFFFFFFF, 0, SAMPLE_TAG), seed_key(seed))
    return u01(x[0], x[1])


# --------------------------------------------------------------------------------------
# Partial amplitude mode (Section 2.2, Eq. 4)
# --------------------------------------------------------------------------------------

def _peel_control(qubits, m):
    """If m (on `qubits`, the first the most significant index bit) has the form
    P0 (x) I + P1 (x) U' in its first qubit, return U' on qubits[1:]; else None."""
    d = m.shape[0] // 2
    if (np.allclose(m[:d, :d], np.eye(d), atol=1e-14) and np.allclose(m[:d, d:], 0, atol=1e-14)
            and np.allclose(m[d:, :d], 0, atol=1e-14)):
        return m[d:, d:]
    return None


def _first_to_front(qubits, m, j):
    """m re-indexed so that qubits[j] becomes the first (most significant) qubit."""
    k = len(qubits)
    order = [qubits[j]] + [q for i, q in enumerate(qubits) if i != j]
    perm = np.zeros((1 << k, 1 << k))
    for new in range(1 << k):
        old = 0
        for pos, q in enumerate(order):
            bit = (new >> (k - 1 - pos)) & 1
            old |= bit << (k - 1 - qubits.index(q))
        perm[old, new] = 1.0
    return order, perm.T @ m @ perm


def partial_decompose(n, ops, cut=None):
    """Steps 1 and 2 of the partial amplitude mode (Section 2.2).

    The dividing line lies between qubits cut - 1 and cut (default n // 2, the middle):
    the upper block is qubits [0, cut), the lower block [cut, n). A gate that crosses the
    line must be a controlled gate: qubits are taken, in listed order, as controls while
    the matrix has the controlled form P0 (x) I + P1 (x) U' in them and the rest still
    crosses the line; then its targets T lie on one side and its controls C on the other
    side split it by Eq. (4), extended to several controls:
        gate = (I - P_C) (x) I  +  P_C (x) U'',
    P_C the projector on C = 1...1 and U'' the gate on T with its controls on T's side.
    Each decomposition doubles the list of circuits (bit 0: the first term, bit 1: the
    second). Returns (cut, c, circuits), circuits[b] = (upper gates, lower gates) for
    b in [0, 2^c), bit k of b the term taken at the k-th decomposed gate, each gate
    (qubits, controls, matrix) in the block's own numbering (upper q -> q, lower
    q -> q - cut). Raises ValueError for a crossing gate without that form (SWAP).
    """
    cut = n // 2 if cut is None else cut
    if not 1 <= cut < n:
        raise ValueError("cut must lie in [1, n)")
    side = lambda q: 0 if q < cut else 1
    local = lambda q: q if q < cut else q - cut
    circuits = [([], [])]
    c = 0
    for qubits, controls, m in expand(ops):
        qubits, controls = list(qubits), list(controls)
        touched = qubits + controls
        if len({side(q) for q in touched}) == 1:
            s = side(touched[0])
            g = ([local(q) for q in qubits], [local(q) for q in controls], m)
            for blocks in circuits:
                blocks[s].append(g)
            continue
        # take listed qubits as controls while the targets still cross the line
        while len({side(q) for q in qubits}) > 1:
            u = _peel_control(qubits, m)
            if u is None:
                raise ValueError("a gate on %s crosses the dividing line and is not controlled" % (qubits,))
            controls.append(qubits[0])
            qubits, m = qubits[1:], u
        ts = side(qubits[0])
        far = [q for q in controls if side(q) != ts]
        near = [q for q in controls if side(q) == ts]
        k = len(far)
        proj = np.zeros((1 << k, 1 << k), dtype=complex)
        proj[-1, -1] = 1.0  # P_C
        rest = np.eye(1 << k, dtype=complex) - proj  # I - P_C
        far_l = [local(q) for q in far]
        term1_target = ([local(q) for q in qubits], [local(q) for q in near], m)
        doubled = []
        for bit in (0, 1):
            for up, lo in circuits:
                blocks = [list(up), list(lo)]
                blocks[1 - ts].append((far_l, [], rest if bit == 0 else proj))
                if bit == 1:
                    blocks[ts].append(term1_target)
                doubled.append((blocks[0], blocks[1]))
        circuits = doubled
        c += 1
    # each doubling appends the bit-1 copies after the bit-0 ones, so the k-th
    # decomposition is bit k of the index
    return cut, c, circuits


def _run_gates(n, gates):
    """Step 3: a sub-circuit simulated in the full amplitude mode from |0...0>."""
    psi = zero_state(n)
    for qubits, controls, m in gates:
        apply(psi, n, qubits, controls, m)
    return psi


def partial_state(n, ops, cut=None):
    """Step 4: psi[x] = sum_b upper_b[x mod 2^cut] lower_b[x >> cut] (small n)."""
    cut, c, circuits = partial_decompose(n, ops, cut)
    psi = np.zeros(1 << n, dtype=complex)
    for up, lo in circuits:
        u = _run_gates(cut, up)
        l = _run_gates(n - cut, lo)
        psi += np.kron(l, u)  # index (x_lower << cut) | x_upper
    return psi


def partial_amplitudes(n, ops, xs, cut=None):
    """Amplitudes <x|psi> for the indices xs by steps 1-4, without the full state."""
    cut, c, circuits = partial_decompose(n, ops, cut)
    xs = np.asarray(xs, dtype=np.uint64)
    xu = (xs & np.uint64((1 << cut) - 1)).astype(np.int64)
    xl = (xs >> np.uint64(cut)).astype(np.int64)
    out = np.zeros(len(xs), dtype=complex)
    for up, lo in circuits:
        out += _run_gates(cut, up)[xu] * _run_gates(n - cut, lo)[xl]
    return out


def _embed(n, qubits, m):
    """2^n x 2^n operator of m on `qubits` (first listed = MSB), via a dense index map."""
    k = len(qubits)
    dim = 1 << n
    full = np.zeros((dim, dim), dtype=complex)
    for i in range(dim):
        r = sum(((i >> q) & 1) << (k - 1 - j) for j, q in enumerate(qubits))
        base = i
        for q in qubits:
            base &= ~(1 << q)
        for c in range(1 << k):
            jdx = base
            for j, q in enumerate(qubits):
                if (c >> (k - 1 - j)) & 1:
                    jdx |= 1 << q
            full[jdx, i] = m[c, r]
    return full


def _controlled(m, nc):
    """Matrix of m with nc extra controls listed first (identity unless all are 1)."""
    k = int(round(math.log2(m.shape[0])))
    dim = 1 << (k + nc)
    full = np.eye(dim, dtype=complex)
    full[dim - (1 << k):, dim - (1 << k):] = m
    return full


def density_matrix(n, ops, p_depol=0.0, gamma=0.0, noise=None, noisy=None):
    """Exact FP64 density-matrix evolution rho <- sum_i K_i (U rho U^dag) K_i^dag.

    The same channels, gates and order as `trajectory`: after each noisy gate, for each
    touched qubit ascending, the channels of noise_list(p_depol, gamma, noise) in channel
    order (the Kronecker two-qubit sets give the same map: sum_ij (K_i (x) K_j) rho
    (K_i (x) K_j)^dag is the two one-qubit maps in turn). Small n only (dense 2^n x 2^n).
    """
    dim = 1 << n
    rho = np.zeros((dim, dim), dtype=complex)
    rho[0, 0] = 1.0
    chans = noise_list(p_depol, gamma, noise)
    for name, qubits, controls, m in expand(ops, names=True):
        U = _embed(n, list(controls) + list(qubits), _controlled(m, len(controls)))
        rho = U @ rho @ U.conj().T
        if noisy is not None and name not in noisy:
            continue
        for q in noise_sites(qubits, controls):
            for _, ch, p in chans:
                acc = np.zeros_like(rho)
                for K in kraus(ch, p):
                    Kf = _embed(n, [q], K)
                    acc += Kf @ rho @ Kf.conj().T
                rho = acc
    return rho


def z_from_density(rho, n):
    diag = np.real(np.diag(rho))
    idx = np.arange(len(diag))
    return np.array([np.sum(diag * (1 - 2 * ((idx >> q) & 1))) for q in range(n)])
