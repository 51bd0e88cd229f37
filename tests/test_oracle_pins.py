"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests calls the CUDA library. Each checks the oracle against something
other than itself: the worked example printed in Appendix A-2, closed forms (GHZ, QFT,
Z-Y-Z decomposition), Kronecker-product operators built independently with numpy,
published Philox known-answer vectors, a library Philox stream, Kraus completeness
(Eq. 5) and an exact density-matrix evolution.
"""

import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.script import parse_script

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# --------------------------------------------------------------------------------------
# Independent Kronecker-product construction (numpy.kron only; qubit n-1 leftmost)
# --------------------------------------------------------------------------------------

I2 = np.eye(2, dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def kron_chain(ops_by_qubit, n):
    full = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        full = np.kron(full, ops_by_qubit.get(q, I2))
    return full


def kron_gate(n, qubits, controls, m):
    """Dense operator of gate m on `qubits` (first = MSB of m's index) with controls."""
    k = len(qubits)
    dim = 1 << k
    u_part = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(dim):
        for c in range(dim):
            if m[r, c] == 0:
                continue
            ops = {}
            for j, q in enumerate(qubits):
                a = (r >> (k - 1 - j)) & 1
                b = (c >> (k - 1 - j)) & 1
                e = np.zeros((2, 2), dtype=complex)
                e[a, b] = 1.0
                ops[q] = e
            for cq in controls:
                ops[cq] = P1
            u_part += m[r, c] * kron_chain(ops, n)
    proj = kron_chain({cq: P1 for cq in controls}, n)
    return np.eye(1 << n, dtype=complex) - proj + u_part


def random_unitary(dim, rng):
    z = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------------------
# Appendix A-2 worked example
# --------------------------------------------------------------------------------------

def load_a2():
    text = open(os.path.join(GOLDEN, "appendix_a2_example.txt")).read()
    expected = {}
    for line in text.splitlines():
        if line.startswith("#@expected"):
            bits, val = line[len("#@expected"):].split(":")
            expected[bits.strip()] = float(val)
    return text, expected


def test_appendix_a2_printed_probabilities():
    text, expected = load_a2()
    n, ops, pm, _ = parse_script(text)
    assert n == 5 and pm == [4, 3, 0]
    psi = oracle.run(n, ops)
    probs = oracle.probabilities(psi, n, pm)
    for s, p in enumerate(probs):
        key = format(s, "03b")
        assert abs(p - expected[key]) <= 1e-6, (key, p, expected[key])
    assert abs(probs.sum() - 1.0) < 1e-12  # PMEASURE probabilities sum to 1


def test_appendix_a2_string_order_matters():
    # The printed strings fix the bit order: the first listed qubit is the leftmost
    # character. Reading the qubit list the other way round must not match.
    text, expected = load_a2()
    n, ops, pm, _ = parse_script(text)
    psi = oracle.run(n, ops)
    probs_rev = oracle.probabilities(psi, n, pm[::-1])
    mismatch = max(abs(probs_rev[s] - expected[format(s, "03b")]) for s in range(8))
    assert mismatch > 1e-3


# --------------------------------------------------------------------------------------
# Gate library (Appendix A-1)
# --------------------------------------------------------------------------------------

ALL_GATES = [("H", ()), ("X", ()), ("Y", ()), ("Z", ()), ("S", ()), ("T", ()),
             ("SX", ()), ("SY", ()), ("RX", (0.7,)), ("RY", (-1.3,)), ("RZ", (2.1,)),
             ("U4", (0.3, 1.1, -0.7, 2.5)), ("CNOT", ()), ("CZ", ()), ("CR", (0.9,)),
             ("SWAP", ()), ("ISWAP", ()), ("TOFFOLI", ())]


@pytest.mark.parametrize("name,params", ALL_GATES)
def test_gate_unitary(name, params):
    k, m = oracle.gate_matrix(name, params)
    assert m.shape == (1 << k, 1 << k)
    assert np.allclose(m.conj().T @ m, np.eye(1 << k), atol=1e-14)


def test_gate_closed_forms():
    X = oracle.gate_matrix("X")[1]
    Y = oracle.gate_matrix("Y")[1]
    Z = oracle.gate_matrix("Z")[1]
    S = oracle.gate_matrix("S")[1]
    T = oracle.gate_matrix("T")[1]
    H = oracle.gate_matrix("H")[1]
    SX = oracle.gate_matrix("SX")[1]
    SY = oracle.gate_matrix("SY")[1]
    assert np.allclose(SX @ SX, X, atol=1e-15)
    assert np.allclose(SY @ SY, Y, atol=1e-15)
    assert np.allclose(T @ T, S, atol=1e-15) and np.allclose(S @ S, Z, atol=1e-15)
    assert np.allclose(H @ Z @ H, X, atol=1e-15)
    assert np.allclose(X @ Y, 1j * Z, atol=1e-15)
    # Rotations: R_P(pi) = -i P; R_P(a) R_P(b) = R_P(a + b)
    for name, P in (("RX", X), ("RY", Y), ("RZ", Z)):
        assert np.allclose(oracle.gate_matrix(name, (math.pi,))[1], -1j * P, atol=1e-15)
        ab = oracle.gate_matrix(name, (0.4,))[1] @ oracle.gate_matrix(name, (0.5,))[1]
        assert np.allclose(ab, oracle.gate_matrix(name, (0.9,))[1], atol=1e-15)
    # U4 angle form = e^{i alpha} RZ(beta) RY(gamma) RZ(delta) (Z-Y-Z decomposition)
    a, b, g, d = 0.3, 1.1, -0.7, 2.5
    zyz = (np.exp(1j * a) * oracle.gate_matrix("RZ", (b,))[1]
           @ oracle.gate_matrix("RY", (g,))[1] @ oracle.gate_matrix("RZ", (d,))[1])
    assert np.allclose(oracle.gate_matrix("U4", (a, b, g, d))[1], zyz, atol=1e-15)
    # CNOT, CZ, CR, TOFFOLI are controlled forms of X, Z, phase, X (first qubit = control)
    assert np.allclose(oracle.gate_matrix("CNOT")[1], kron_gate(2, [0], [1], X), atol=0)
    assert np.allclose(oracle.gate_matrix("CZ")[1], kron_gate(2, [0], [1], Z), atol=0)
    ph = np.diag([1, np.exp(0.9j)])
    assert np.allclose(oracle.gate_matrix("CR", (0.9,))[1], kron_gate(2, [0], [1], ph), atol=1e-15)
    assert np.allclose(oracle.gate_matrix("TOFFOLI")[1], kron_gate(3, [0], [2, 1], X), atol=0)


# --------------------------------------------------------------------------------------
# Eq. (2) / (3) and the k-qubit apply against Kronecker brute force
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_apply_1q_all_targets_vs_kron(n):
    rng = np.random.default_rng(100 + n)
    for t in range(n):
        others = [q for q in range(n) if q != t]
        for nc in range(min(2, len(others)) + 1):
            ctrls = list(rng.choice(others, size=nc, replace=False)) if nc else []
            u = random_unitary(2, rng)
            psi = random_state(n, rng)
            ref = kron_gate(n, [t], ctrls, u) @ psi
            got = oracle.apply(psi.copy(), n, [t], ctrls, u)
            assert np.max(np.abs(got - ref)) < 1e-14, (n, t, ctrls)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_apply_2q_all_pairs_vs_kron(n):
    rng = np.random.default_rng(200 + n)
    for q0 in range(n):
        for q1 in range(n):
            if q0 == q1:
                continue
            others = [q for q in range(n) if q not in (q0, q1)]
            ctrls = [others[0]] if others and (q0 + q1) % 2 else []
            m = random_unitary(4, rng)
            psi = random_state(n, rng)
            ref = kron_gate(n, [q0, q1], ctrls, m) @ psi
            got = oracle.apply(psi.copy(), n, [q0, q1], ctrls, m)
            assert np.max(np.abs(got - ref)) < 1e-14, (q0, q1, ctrls)


def test_apply_kq_vs_kron():
    rng = np.random.default_rng(7)
    n = 8
    for k in (3, 4, 5):
        for _ in range(3):
            qs = list(rng.choice(n, size=k, replace=False))
            m = random_unitary(1 << k, rng)
            psi = random_state(n, rng)
            ref = kron_gate(n, qs, [], m) @ psi
            got = oracle.apply(psi.copy(), n, qs, [], m)
            assert np.max(np.abs(got - ref)) < 1e-13


def test_circuit_vs_kron_product_n10():
    n = 10
    ops = synth.random_circuit(n, 3, seed=5)
    full = np.eye(1 << n, dtype=complex)
    for qubits, controls, m in oracle.expand(ops):
        full = kron_gate(n, list(qubits), list(controls), m) @ full
    ref = full[:, 0]
    got = oracle.run(n, ops)
    assert np.max(np.abs(got - ref)) < 1e-13


# --------------------------------------------------------------------------------------
# Closed forms and invariants
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz(n):
    ops = [("H", (0,), ())] + [("CNOT", (q, q + 1), ()) for q in range(n - 1)]
    psi = oracle.run(n, ops)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


def test_bell_with_control_block():
    # CONTROL 0 ... ENDCONTROL around X 1 is CNOT 0,1 (Appendix A-1)
    ops = [("H", (0,), ()), ("CONTROL", (0,), ()), ("X", (1,), ()), ("ENDCONTROL", (0,), ())]
    psi = oracle.run(2, ops)
    assert np.allclose(psi, [1 / math.sqrt(2), 0, 0, 1 / math.sqrt(2)], atol=1e-15)


def bitrev(y, n):
    return int(format(y, "0%db" % n)[::-1], 2)


@pytest.mark.parametrize("n,x", [(3, 5), (6, 0), (6, 37), (9, 301)])
def test_qft_of_basis_state(n, x):
    ops = [("X", (q,), ()) for q in range(n) if (x >> q) & 1] + synth.qft_circuit(n)
    psi = oracle.run(n, ops)
    N = 1 << n
    assert np.allclose(np.abs(psi), N ** -0.5, atol=1e-14)  # uniform magnitudes
    for y in range(N):
        ref = np.exp(2j * math.pi * x * y / N) / math.sqrt(N)
        assert abs(psi[bitrev(y, n)] - ref) < 1e-13
    # the same transform via the library FFT (numpy.fft.ifft * sqrt(N) is the +i DFT)
    e = np.zeros(N, dtype=complex)
    e[x] = 1
    dft = np.fft.ifft(e) * math.sqrt(N)
    assert np.max(np.abs(psi[[bitrev(y, n) for y in range(N)]] - dft)) < 1e-13


@pytest.mark.parametrize("n,depth", [(4, 8), (12, 20)])
def test_norm_and_circuit_then_dagger(n, depth):
    ops = synth.random_circuit(n, depth, seed=3)
    psi = oracle.run(n, ops)
    assert abs(oracle.norm2(psi, n) - 1.0) < 1e-13
    back = oracle.run(n, ops + synth.inverse_ops(ops))
    assert abs(back[0] - 1.0) < 1e-12 and np.max(np.abs(back[1:])) < 1e-12


def test_nested_dagger_and_control_expansion():
    ops = [("RX", (0,), (0.3,)), ("CNOT", (0, 1), ()), ("RZ", (1,), (1.2,))]
    twice = [("DAGGER", (), ())] + [("DAGGER", (), ())] + ops + [("ENDDAGGER", (), ())] * 2
    a = oracle.expand(ops)
    b = oracle.expand(twice)
    assert len(a) == len(b)
    for (qa, ca, ma), (qb, cb, mb) in zip(a, b):
        assert qa == qb and ca == cb and np.allclose(ma, mb, atol=0)
    ctl = oracle.expand([("CONTROL", (2,), ()), ("CONTROL", (3,), ())] + ops +
                        [("ENDCONTROL", (3,), ()), ("ENDCONTROL", (2,), ())])
    assert all(c == (2, 3) for _, c, _ in ctl)


def test_expand_dagger_order_and_adjoint():
    ops = [("RX", (0,), (0.3,)), ("S", (1,), ())]
    out = oracle.expand([("DAGGER", (), ())] + ops + [("ENDDAGGER", (), ())])
    assert [q for q, _, _ in out] == [(1,), (0,)]
    assert np.allclose(out[0][2], np.diag([1, -1j]), atol=0)
    assert np.allclose(out[1][2], oracle.gate_matrix("RX", (-0.3,))[1], atol=1e-15)


# --------------------------------------------------------------------------------------
# Readouts
# --------------------------------------------------------------------------------------

def test_probabilities_vs_bruteforce():
    rng = np.random.default_rng(3)
    n = 7
    psi = random_state(n, rng)
    for qs in ([0], [6], [3, 1], [1, 3], [6, 0, 2], list(range(n))):
        got = oracle.probabilities(psi, n, qs)
        ref = np.zeros(1 << len(qs))
        for i in range(1 << n):
            s = 0
            for j, q in enumerate(qs):
                s = (s << 1) | ((i >> q) & 1)
            ref[s] += abs(psi[i]) ** 2
        assert np.max(np.abs(got - ref)) < 1e-15
        assert abs(got.sum() - 1) < 1e-14


def test_z_expectations_closed_form():
    # product state RY(theta_q)|0> on each qubit: <Z_q> = cos(theta_q)
    n = 6
    th = [0.1 * (q + 1) for q in range(n)]
    psi = oracle.run(n, [("RY", (q,), (th[q],)) for q in range(n)])
    assert np.allclose(oracle.z_expectations(psi, n), np.cos(th), atol=1e-14)


def inner_closed_forms(inner):
    """Closed forms of <a|b> = sum conj(a_i) b_i that fix which side is conjugated, the sign
    of the imaginary part and the normalisation; returns the list of failures."""
    bad = []
    n = 3
    zero = oracle.zero_state(n)
    i_zero = 1j * zero
    # <i 0|0> = -i and <0|i 0> = +i: only the first argument is conjugated
    if abs(inner(i_zero, zero, n) - (-1j)) > 1e-15:
        bad.append("<i0|0>")
    if abs(inner(zero, i_zero, n) - 1j) > 1e-15:
        bad.append("<0|i0>")
    # <+^n|0^n> = 2^(-n/2) (H on every qubit, built here without the oracle)
    for m in (1, 4, 9):
        plus = np.full(1 << m, 2.0 ** (-m / 2), dtype=complex)
        if abs(inner(plus, oracle.zero_state(m), m) - 2.0 ** (-m / 2)) > 1e-15:
            bad.append("<+|0> n=%d" % m)
    # <a|e^{i phi} a> = e^{i phi} ||a||^2 for a random a
    rng = np.random.default_rng(21)
    a = random_state(6, rng) * 1.7
    phi = 0.8134
    if abs(inner(a, np.exp(1j * phi) * a, 6) - np.exp(1j * phi) * 1.7 ** 2) > 1e-13:
        bad.append("phase")
    return bad


def test_inner_closed_forms_and_library_vdot():
    # the checker of qsim_inner / qsim_fidelity: closed forms, then numpy.vdot (a library
    # routine the oracle does not call) on random states of several sizes
    assert inner_closed_forms(oracle.inner) == []
    rng = np.random.default_rng(22)
    for n in (1, 5, 12):
        a = random_state(n, rng)
        b = random_state(n, rng) * (0.3 - 0.9j)
        assert abs(oracle.inner(a, b, n) - np.vdot(a, b)) <= 1e-14
        assert abs(oracle.inner(a, b, n) - np.conj(oracle.inner(b, a, n))) <= 1e-15
        assert abs(oracle.inner(a, a, n) - oracle.norm2(a, n)) <= 1e-14


def test_reduced_density_vs_numpy_contraction():
    # rho of the listed qubits (first = most significant) by numpy: move their axes to the
    # front of the 2^n tensor and contract the rest; every placement of 1..3 qubits
    rng = np.random.default_rng(23)
    n = 6
    psi = random_state(n, rng)
    t = psi.reshape([2] * n)  # axis a <-> qubit n - 1 - a
    for k in (1, 2, 3):
        for qs in ([0, 1, 2][:k], [5, 0, 3][:k], [2, 4, 1][:k], [3, 5, 0][:k]):
            axes = [n - 1 - q for q in qs]
            rest = [a for a in range(n) if a not in axes]
            A = np.transpose(t, axes + rest).reshape(1 << k, -1)
            assert np.max(np.abs(oracle.reduced_density(psi, n, qs) - A @ A.conj().T)) <= 1e-15, qs
    # a product state |1> (x) |+>: rho of qubit 1 = |1><1|, of qubit 0 = |+><+|
    prod = np.zeros(4, dtype=complex)
    prod[2] = prod[3] = math.sqrt(0.5)
    assert np.allclose(oracle.reduced_density(prod, 2, [1]), [[0, 0], [0, 1]], atol=1e-16)
    assert np.allclose(oracle.reduced_density(prod, 2, [0]), [[0.5, 0.5], [0.5, 0.5]], atol=1e-16)


def test_pin_catches_a_conjugation_swap_in_inner(monkeypatch):
    # an inner product that conjugates b instead of a (or flips the imaginary part's sign)
    # fails the closed forms
    real = oracle.inner
    monkeypatch.setattr(oracle, "inner", lambda a, b, n: real(b, a, n))
    assert "<i0|0>" in inner_closed_forms(oracle.inner)
    monkeypatch.setattr(oracle, "inner", lambda a, b, n: np.conj(real(a, b, n)))
    assert "<0|i0>" in inner_closed_forms(oracle.inner)


def test_sample_vs_library_inverse_cdf():
    rng = np.random.default_rng(9)
    n = 6
    psi = random_state(n, rng)
    u = oracle.sample_draws(seed=1234, shots=500)
    assert np.all((u >= 0) & (u < 1))
    got = oracle.sample(psi, n, u)
    cdf = np.cumsum(np.abs(psi) ** 2)
    ref = np.searchsorted(cdf, u * cdf[-1], side="right")
    assert np.array_equal(got.astype(np.int64), ref)


# --------------------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------------------

# Known-answer vectors distributed with the Random123 library (Salmon et al., SC'11):
# (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(ctr, key, out):
    assert tuple(oracle.philox(ctr, key)) == out


def _load_curand():
    for cand in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so",
                 ctypes.util.find_library("curand")):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


def test_philox_vs_curand_host_generator():
    lib = _load_curand()
    if lib is None:
        pytest.skip("libcurand not loadable")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    seed = 0x0123456789ABCDEF
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
    count = 4 * 64
    buf = (ctypes.c_uint32 * count)()
    assert lib.curandGenerate(gen, buf, ctypes.c_size_t(count)) == 0
    lib.curandDestroyGenerator(gen)
    # the host generator's j-th block of four words is counter (0, 0, j, 0) (one
    # subsequence per block) under key (seed_lo, seed_hi)
    ctrs = np.zeros((64, 4), dtype=np.uint32)
    ctrs[:, 2] = np.arange(64)
    ours = oracle.philox_many(ctrs, oracle.seed_key(seed)).reshape(-1)
    assert np.array_equal(ours, np.frombuffer(buf, dtype=np.uint32))


def test_u01_range_and_resolution():
    assert oracle.u01(0, 0) == 0.0
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u01(0, 1 << 11) == 2.0 ** -53


# --------------------------------------------------------------------------------------
# Noise (Section 2.4, Eq. 5)
# --------------------------------------------------------------------------------------

CHANNELS = ["bit_flip", "phase_flip", "bit_phase_flip", "amplitude_damping",
            "phase_damping", "depolarizing"]


@pytest.mark.parametrize("channel", CHANNELS)
@pytest.mark.parametrize("p", [0.0, 0.2, 1.0])
def test_kraus_completeness(channel, p):
    ks = oracle.kraus(channel, p)
    acc = sum(k.conj().T @ k for k in ks)
    assert np.allclose(acc, np.eye(2), atol=1e-15)


def test_kraus_noise_limits():
    # flips are noiseless at p = 1, damping and depolarizing at p = 0 (Eq. 5 remark)
    rho = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, 0.7]])
    for ch, p in (("bit_flip", 1.0), ("phase_flip", 1.0), ("bit_phase_flip", 1.0),
                  ("amplitude_damping", 0.0), ("phase_damping", 0.0), ("depolarizing", 0.0)):
        out = sum(k @ rho @ k.conj().T for k in oracle.kraus(ch, p))
        assert np.allclose(out, rho, atol=1e-15), ch
    # full depolarizing (p = 1) sends any state to I/2
    out = sum(k @ rho @ k.conj().T for k in oracle.kraus("depolarizing", 1.0))
    assert np.allclose(out, np.eye(2) / 2, atol=1e-15)
    # full amplitude damping sends any state to |0><0|
    out = sum(k @ rho @ k.conj().T for k in oracle.kraus("amplitude_damping", 1.0))
    assert np.allclose(out, [[1, 0], [0, 0]], atol=1e-15)


def test_trajectory_noiseless_limit_is_exact():
    n = 6
    ops = synth.random_circuit(n, 5, seed=2)
    psi, events, _ = oracle.trajectory(n, ops, seed=1, traj=0, p_depol=0.0, gamma=0.0)
    assert events == []
    assert np.array_equal(psi, oracle.run(n, ops))


def test_density_matrix_noiseless_is_pure_state():
    n = 4
    ops = synth.random_circuit(n, 4, seed=8)
    rho = oracle.density_matrix(n, ops, 0.0, 0.0)
    psi = oracle.run(n, ops)
    assert np.allclose(rho, np.outer(psi, psi.conj()), atol=1e-14)


def test_density_matrix_is_a_state():
    rho = oracle.density_matrix(4, synth.random_circuit(4, 3, seed=4), 0.1, 0.2)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.allclose(rho, rho.conj().T, atol=1e-15)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-13


def test_trajectory_average_matches_density_matrix():
    # Monte-Carlo unravelling of Section 2.4 vs the exact channel evolution (3 sigma)
    n, depth = 8, 4
    p, gamma = 0.06, 0.08
    ops = synth.random_circuit(n, depth, seed=21)
    exact = oracle.z_from_density(oracle.density_matrix(n, ops, p, gamma), n)
    T = 300
    zs = np.array([oracle.z_expectations(
        oracle.trajectory(n, ops, seed=77, traj=t, p_depol=p, gamma=gamma)[0], n)
        for t in range(T)])
    mean = zs.mean(axis=0)
    sigma = zs.std(axis=0, ddof=1) / math.sqrt(T)
    assert np.all(np.abs(mean - exact) <= 3 * sigma + 1e-12), (mean, exact, sigma)
    # and the noise is visible: the noiseless values differ from the exact noisy ones
    clean = oracle.z_expectations(oracle.run(n, ops), n)
    assert np.max(np.abs(clean - exact)) > 0.05


def test_depolarizing_branch_frequencies():
    # state-independent branch weights (1 - 3p/4, p/4, p/4, p/4): binomial 4 sigma
    p = 0.2
    key = oracle.seed_key(99)
    draws = 20000
    ctrs = np.array([oracle.noise_ctr(0, g, 0, 0) for g in range(draws)], dtype=np.uint32)
    x = oracle.philox_many(ctrs, key)
    u = np.array([oracle.u01(a, b) for a, b in x[:, :2]])
    c1 = 1 - 3 * p / 4
    counts = [np.sum(u < c1), np.sum((u >= c1) & (u < c1 + p / 4)),
              np.sum((u >= c1 + p / 4) & (u < c1 + p / 2)), np.sum(u >= c1 + p / 2)]
    for cnt, w in zip(counts, [c1, p / 4, p / 4, p / 4]):
        assert abs(cnt - draws * w) < 4 * math.sqrt(draws * w * (1 - w))


def test_measure_bell_state_and_projector():
    # MEASURE (App. A-1) on a Bell state: either outcome with probability 1/2, the partner
    # qubit then follows with certainty; on a random state the collapsed state equals the
    # Kronecker-built projector |r><r| on qubit q applied and normalised
    bell = oracle.run(2, [("H", (0,), ()), ("CNOT", (0, 1), ())])
    r, pr, post = oracle.measure(bell, 2, 0, 0.3)
    assert r == 0 and abs(pr - 0.5) < 1e-15
    assert np.allclose(post, [1, 0, 0, 0], atol=1e-15)
    r, pr, post = oracle.measure(bell, 2, 0, 0.7)
    assert r == 1 and abs(pr - 0.5) < 1e-15
    assert np.allclose(post, [0, 0, 0, 1], atol=1e-15)
    r2, pr2, _ = oracle.measure(post, 2, 1, 0.999)
    assert r2 == 1 and abs(pr2 - 1.0) < 1e-15
    rng = np.random.default_rng(21)
    n = 4
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for q in range(n):
        for u in (0.05, 0.5, 0.95):
            r, pr, post = oracle.measure(psi, n, q, u)
            proj = kron_chain({q: np.diag([1.0 - r, float(r)]).astype(complex)}, n)
            v = proj @ psi
            p_ref = np.vdot(v, v).real / np.vdot(psi, psi).real
            assert abs(pr - p_ref) < 1e-13
            p0 = 1 - p_ref if r == 1 else p_ref
            assert (r == 0) == (u < p0)
            assert np.max(np.abs(post - v / np.linalg.norm(v))) < 1e-13


# ---- the six Eq. (5) channels, Kronecker joint draws, noisy gate classes -----------------

def one_qubit_channel_closed_form(name, p, r):
    """The channel map of Eq. (5) on a 2x2 density matrix r, written out by hand."""
    r00, r01, r10, r11 = r[0, 0], r[0, 1], r[1, 0], r[1, 1]
    if name == "bit_flip":        # p r + (1-p) X r X
        return np.array([[p * r00 + (1 - p) * r11, p * r01 + (1 - p) * r10],
                         [p * r10 + (1 - p) * r01, p * r11 + (1 - p) * r00]])
    if name == "phase_flip":      # p r + (1-p) Z r Z
        return np.array([[r00, (2 * p - 1) * r01], [(2 * p - 1) * r10, r11]])
    if name == "bit_phase_flip":  # p r + (1-p) Y r Y, Y r Y = [[r11, -r10], [-r01, r00]]
        return np.array([[p * r00 + (1 - p) * r11, p * r01 - (1 - p) * r10],
                         [p * r10 - (1 - p) * r01, p * r11 + (1 - p) * r00]])
    if name == "amplitude_damping":
        return np.array([[r00 + p * r11, math.sqrt(1 - p) * r01], [math.sqrt(1 - p) * r10, (1 - p) * r11]])
    if name == "phase_damping":
        return np.array([[r00, math.sqrt(1 - p) * r01], [math.sqrt(1 - p) * r10, r11]])
    if name == "depolarizing":    # (1 - 3p/4) r + p/4 (X r X + Y r Y + Z r Z) = (1-p) r + p/2 I
        return (1 - p) * r + p / 2 * np.eye(2)
    raise ValueError(name)


@pytest.mark.parametrize("name,p", [("bit_flip", 0.7), ("phase_flip", 0.3), ("bit_phase_flip", 0.9),
                                    ("amplitude_damping", 0.35), ("phase_damping", 0.6), ("depolarizing", 0.4)])
def test_density_matrix_one_qubit_closed_forms(name, p):
    # noise only after the T gate (gate class selection): the state before it is pure
    ops = [("RY", (0,), (0.7,)), ("T", (0,), ())]
    psi = oracle.run(1, ops)
    r = np.outer(psi, psi.conj())
    rho = oracle.density_matrix(1, ops, noise={name: p}, noisy={"T"})
    assert np.allclose(rho, one_qubit_channel_closed_form(name, p, r), atol=1e-15)
    # and every gate noisy: the channel acts after RY as well
    psi_ry = oracle.run(1, ops[:1])
    r1 = one_qubit_channel_closed_form(name, p, np.outer(psi_ry, psi_ry.conj()))
    T = oracle.gate_matrix("T", ())[1]
    r2 = one_qubit_channel_closed_form(name, p, T @ r1 @ T.conj().T)
    assert np.allclose(oracle.density_matrix(1, ops, noise={name: p}), r2, atol=1e-15)


def average_density(n, ops, T, seed, **kw):
    acc = np.zeros((1 << n, 1 << n), dtype=complex)
    for t in range(T):
        psi = oracle.trajectory(n, ops, seed, t, **kw)[0]
        acc += np.outer(psi, psi.conj())
    return acc / T


@pytest.mark.parametrize("kron", [False, True])
@pytest.mark.parametrize("noise,noisy", [
    ({"bit_flip": 0.85}, None), ({"phase_flip": 0.8}, None), ({"bit_phase_flip": 0.85}, None),
    ({"phase_damping": 0.25}, None),
    ({"depolarizing": 0.05, "amplitude_damping": 0.1, "bit_flip": 0.95, "phase_flip": 0.95,
      "bit_phase_flip": 0.95, "phase_damping": 0.1}, None),
    ({"amplitude_damping": 0.3, "phase_damping": 0.2}, {"CZ", "CNOT", "ISWAP", "SWAP"})])
def test_trajectory_average_is_the_density_matrix(noise, noisy, kron):
    # For pure samples psi_t, E ||psi psi^dag - rho||_F^2 = 1 - tr rho^2, so the average of T
    # of them lies within ||.||_F^2 ~ (1 - tr rho^2) / T of rho; a wrong operator, branch
    # order or missing renormalisation is off by O(1)
    n, T = 4, 400
    ops = synth.random_circuit(n, 3, seed=31)
    exact = oracle.density_matrix(n, ops, noise=noise, noisy=noisy)
    avg = average_density(n, ops, T, 0xC0FFEE, noise=noise, noisy=noisy, kron=kron)
    expected = (1 - np.real(np.trace(exact @ exact))) / T
    dev = np.linalg.norm(avg - exact) ** 2
    assert dev <= 3 * expected, (dev, expected)
    clean = oracle.run(n, ops)
    assert np.linalg.norm(np.outer(clean, clean.conj()) - exact) ** 2 > 30 * expected  # visible


def test_phase_damping_branches_closed_form():
    # H|0> then phase damping: K2 = diag(0, sqrt p) is taken with probability p |b|^2 = p / 2
    # and leaves |1>; K1 leaves (|0> + sqrt(1-p)|1>) / sqrt(2 - p)
    p, T = 0.3, 4000
    ops = [("H", (0,), ())]
    k1 = np.array([1, math.sqrt(1 - p)]) / math.sqrt(2 - p)
    hits = 0
    for t in range(T):
        psi, ev, _ = oracle.trajectory(1, ops, 5, t, noise={"phase_damping": p})
        if ev:
            assert ev == [(0, 0, 5, 1)]
            assert np.allclose(psi, [0, 1], atol=1e-15)
            hits += 1
        else:
            assert np.allclose(psi, k1, atol=1e-15)
    assert abs(hits - T * p / 2) < 4 * math.sqrt(T * p / 2 * (1 - p / 2))


@pytest.mark.parametrize("name,c,pauli", [("bit_flip", 2, "X"), ("phase_flip", 3, "Z"), ("bit_phase_flip", 4, "Y")])
def test_flip_branch_frequencies_and_states(name, c, pauli):
    # K1 = sqrt(p) I, K2 = sqrt(1-p) P: P is applied with probability 1 - p whatever the
    # state (p is the probability of no flip, as printed), leaving P|psi> normalised
    p, T = 0.8, 4000
    ops = [("RY", (0,), (1.1,))]
    psi0 = oracle.run(1, ops)
    P = oracle.gate_matrix(pauli, ())[1]
    hits = 0
    for t in range(T):
        psi, ev, _ = oracle.trajectory(1, ops, 6, t, noise={name: p})
        if ev:
            assert ev == [(0, 0, c, 1)]
            assert np.allclose(psi, P @ psi0, atol=1e-15)
            hits += 1
        else:
            assert np.allclose(psi, psi0, atol=1e-15)
    assert abs(hits - T * (1 - p)) < 4 * math.sqrt(T * p * (1 - p))


def test_kron_joint_depolarizing_frequencies():
    # a CNOT draws one number over the 16 products K_i (x) K_j: outcome (i, j) has
    # probability w_i w_j, w = (1 - 3p/4, p/4, p/4, p/4)
    p, T = 0.5, 6000
    w = [1 - 3 * p / 4, p / 4, p / 4, p / 4]
    counts = np.zeros((4, 4))
    for t in range(T):
        _, ev, _ = oracle.trajectory(2, [("CNOT", (1, 0), ())], 8, t, noise={"depolarizing": p}, kron=True)
        i = next((b for g, q, c, b in ev if q == 1), 0)
        j = next((b for g, q, c, b in ev if q == 0), 0)
        assert all(g == 0 and c == 0 for g, q, c, b in ev)
        counts[i, j] += 1
    for i in range(4):
        for j in range(4):
            pij = w[i] * w[j]
            assert abs(counts[i, j] - T * pij) < 4 * math.sqrt(T * pij * (1 - pij)), (i, j)


def test_noise_only_on_the_chosen_gate_classes():
    n = 5
    ops = synth.random_circuit(n, 4, seed=12)
    names = [e[0] for e in oracle.expand(ops, names=True)]
    noisy = {"CZ", "T"}
    total = 0
    for t in range(50):
        _, ev, _ = oracle.trajectory(n, ops, 3, t, noise={"bit_flip": 0.5, "phase_damping": 0.5}, noisy=noisy)
        assert all(names[g] in noisy for g, _, _, _ in ev)
        total += len(ev)
    assert total > 0


# ---- partial amplitude mode (Section 2.2, Eq. 4) -----------------------------------------

def test_eq4_cz_is_projector_sum():
    # CZ^{i,j} = P0^i (x) I^j + P1^i (x) Z^j (Eq. 4), i the more significant index bit
    P0 = np.diag([1.0, 0.0])
    P1 = np.diag([0.0, 1.0])
    Z = np.diag([1.0, -1.0])
    cz = oracle.gate_matrix("CZ", ())[1]
    assert np.allclose(cz, np.kron(P0, np.eye(2)) + np.kron(P1, Z), atol=0)


@pytest.mark.parametrize("n,depth,cross,cut,seed", [(8, 8, 2, None, 1), (9, 5, 3, 3, 2), (10, 6, 4, None, 3),
                                                    (12, 4, 5, 7, 4), (11, 3, 0, None, 5)])
def test_partial_recombination_equals_full_simulation(n, depth, cross, cut, seed):
    ops = synth.partial_circuit(n, depth, cross, seed, cut=cut)
    ref = oracle.run(n, ops)
    got = oracle.partial_state(n, ops, cut=cut)
    assert np.max(np.abs(got - ref)) <= 1e-13
    ct, c, circuits = oracle.partial_decompose(n, ops, cut=cut)
    assert c == cross and len(circuits) == 2 ** c  # 2^(c+1) sub-circuits
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, 1 << n, size=50)
    assert np.max(np.abs(oracle.partial_amplitudes(n, ops, xs, cut=cut) - ref[xs])) <= 1e-13


def test_partial_multi_controlled_crossings():
    # TOFFOLI with both controls above the line, with the controls split across it, and a
    # CONTROL block whose control sits on the other side of a two-qubit target gate
    n = 8
    ops = synth.partial_circuit(n, 3, 1, 9)
    ops += [("TOFFOLI", (0, 2, 6), ()), ("TOFFOLI", (1, 5, 3), ()), ("TOFFOLI", (4, 6, 2), ()),
            ("CONTROL", (1,), ()), ("ISWAP", (5, 7), ()), ("RX", (6,), (0.3,)), ("ENDCONTROL", (), ()),
            ("CONTROL", (6,), ()), ("CNOT", (0, 3), ()), ("ENDCONTROL", (), ())]
    ops += synth.partial_circuit(n, 2, 2, 10)
    got = oracle.partial_state(n, ops)
    assert np.max(np.abs(got - oracle.run(n, ops))) <= 1e-13
    assert oracle.partial_decompose(n, ops)[1] == 1 + 6 + 2


def test_partial_fig1_shape():
    # 8 qubits, 8 layers, the blocks joined by CZ gates after layers 7 and 8: four circuits,
    # eight 4-qubit sub-circuits, 2^7 stored amplitudes instead of 2^8
    ops = synth.partial_circuit(8, 8, 0, 11)
    ops += [("CZ", (3, 4), ()), ("H", (3,), ()), ("H", (4,), ()), ("CZ", (2, 5), ())]
    cut, c, circuits = oracle.partial_decompose(8, ops)
    assert cut == 4 and c == 2 and len(circuits) == 4
    assert 2 * len(circuits) * (1 << 4) == 1 << 7
    assert np.max(np.abs(oracle.partial_state(8, ops) - oracle.run(8, ops))) <= 1e-13


@pytest.mark.parametrize("gate", [("SWAP", (1, 5), ()), ("ISWAP", (2, 4), ())])
def test_partial_rejects_uncontrolled_crossing(gate):
    with pytest.raises(ValueError):
        oracle.partial_decompose(6, [("H", (0,), ()), gate])


# ---- the pins catch planted mistakes (each plants one in the oracle, on the CPU) ---------

def test_pin_catches_the_usual_flip_convention(monkeypatch):
    # the textbook convention (sqrt(1-p) I, sqrt(p) X) instead of Eq. 5's sqrt(p) I: the
    # one-qubit closed form no longer holds
    real = oracle.kraus

    def swapped(channel, p):
        if channel == "bit_flip":
            return [math.sqrt(1 - p) * np.eye(2), math.sqrt(p) * np.array([[0, 1], [1, 0]], dtype=complex)]
        return real(channel, p)

    monkeypatch.setattr(oracle, "kraus", swapped)
    ops = [("RY", (0,), (0.7,)), ("T", (0,), ())]
    psi = oracle.run(1, ops)
    r = np.outer(psi, psi.conj())
    rho = oracle.density_matrix(1, ops, noise={"bit_flip": 0.7}, noisy={"T"})
    assert not np.allclose(rho, one_qubit_channel_closed_form("bit_flip", 0.7, r), atol=1e-6)


def test_pin_catches_swapped_projectors(monkeypatch):
    # Eq. 4 with the projectors exchanged (P1 (x) I + P0 (x) U): the recombined state is no
    # longer the full simulation
    real_decompose = oracle.partial_decompose

    def is_projector(q, cs, m):
        d = np.diag(m)
        return len(q) == 1 and not cs and np.allclose(m, np.diag(d)) and sorted(np.round(d.real, 12)) == [0.0, 1.0]

    def swap(gates):
        return [(q, cs, np.diag(np.diag(m)[::-1]) if is_projector(q, cs, m) else m) for q, cs, m in gates]

    def bad_decompose(n, ops, cut=None):
        cut_, c, circuits = real_decompose(n, ops, cut)
        return cut_, c, [(swap(up), swap(lo)) for up, lo in circuits]

    monkeypatch.setattr(oracle, "partial_decompose", bad_decompose)
    n = 8
    ops = synth.partial_circuit(n, 4, 2, 1)
    assert np.max(np.abs(oracle.partial_state(n, ops) - oracle.run(n, ops))) > 1e-3


def test_pin_catches_a_missing_renormalisation(monkeypatch):
    # dropping step 3's normalisation leaves unnormalised trajectory states: the averaged
    # density matrix misses the exact one by far more than the statistical bound
    real_norm2 = oracle.norm2
    monkeypatch.setattr(oracle, "norm2", lambda psi, n: 1.0 if psi.size == 1 << 4 else real_norm2(psi, n))
    n, T = 4, 200
    ops = synth.random_circuit(n, 3, seed=31)
    noise = {"amplitude_damping": 0.3}
    exact = oracle.density_matrix(n, ops, noise=noise)
    avg = average_density(n, ops, T, 0xC0FFEE, noise=noise)
    expected = (1 - np.real(np.trace(exact @ exact))) / T
    assert np.linalg.norm(avg - exact) ** 2 > 3 * expected


def test_noisy_class_inside_blocks_is_the_instruction_kind():
    # CONTROL 1 { H 0 } and DAGGER { T 0 }: with noisy = {"H"} the channel follows the
    # controlled H on both qubits it touches and nothing else; with noisy = {"T"} it follows
    # the adjoint T (which stays of kind T)
    ops = [("RY", (0,), (0.9,)), ("RY", (1,), (1.3,)), ("CONTROL", (1,), ()), ("H", (0,), ()),
           ("ENDCONTROL", (), ()), ("DAGGER", (), ()), ("T", (0,), ()), ("ENDDAGGER", (), ())]
    p = 0.3
    K = oracle.kraus("phase_damping", p)

    def channel(rho, q):
        return sum(oracle._embed(2, [q], k) @ rho @ oracle._embed(2, [q], k).conj().T for k in K)

    def unitary(rho, sub):
        psi_ops = sub
        U = np.column_stack([oracle.run(2, [("X", (j,), ()) for j in range(2) if (c >> j) & 1] + psi_ops)
                             for c in range(4)])
        return U @ rho @ U.conj().T

    rho0 = np.zeros((4, 4), dtype=complex)
    rho0[0, 0] = 1
    r = unitary(rho0, ops[:2])
    r = unitary(r, ops[2:5])
    r_h = channel(channel(r, 0), 1)
    expect_h = unitary(r_h, ops[5:])
    got_h = oracle.density_matrix(2, ops, noise={"phase_damping": p}, noisy={"H"})
    assert np.allclose(got_h, expect_h, atol=1e-14)
    expect_t = channel(unitary(r, ops[5:]), 0)
    got_t = oracle.density_matrix(2, ops, noise={"phase_damping": p}, noisy={"T"})
    assert np.allclose(got_t, expect_t, atol=1e-14)
    assert not np.allclose(got_h, got_t, atol=1e-6)
