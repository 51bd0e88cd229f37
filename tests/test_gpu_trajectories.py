"""Noisy trajectories (Section 2.4, Eq. 5) on the GPU against the FP64 oracle.

The GPU and the oracle draw the same Philox4x32-10 numbers, so each trajectory takes the
same branches (near-ties, where a draw lies within 1e-9 of a probability boundary, may
differ and are allowed); Z expectations and samples then match up to the complex64
precision of the GPU state. The average over trajectories matches the exact FP64 density
matrix within 3 sigma.
"""

import math
import warnings

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


# FP32 bar of the trajectory states: max |d amp| and |d <Z>| against the FP64 oracle
STATE_TOL = 1e-6


def check_against_oracle(qs, programs, traj_prog, seed, p, gamma, **noise_kw):
    """Every trajectory against oracle.trajectory: the same branch events, the final state
    (normalised, kept on the device) and <Z> within STATE_TOL. Trajectories with a near-tie
    draw are skipped; returns (compared, event counts)."""
    ntraj = len(traj_prog)
    plan = qs.TrajPlan(programs, traj_prog, seed, p, gamma, shots=ntraj, event_cap=256, keep=range(ntraj),
                       **noise_kw)
    plan.launch()
    zexp, samples, events, nev = plan.results()
    compared = 0
    for t in range(ntraj):
        w, ops = programs[traj_prog[t]]
        psi, ev_ref, ties = oracle.trajectory(w, ops, seed, t, p, gamma, **noise_kw)
        if ties:
            continue
        compared += 1
        assert events[t] == ev_ref, (t, events[t], ev_ref)
        got = plan.state(t).astype(np.complex128)
        assert np.max(np.abs(got - psi)) <= STATE_TOL, t
        zr = oracle.z_expectations(psi, w)
        assert np.max(np.abs(zexp[t, :w] - zr)) <= STATE_TOL
    plan.close()
    return compared, nev


@pytest.mark.parametrize("p,gamma", [(0.05, 0.05), (0.0, 0.1), (0.08, 0.0)])
def test_windowed_runs_match_oracle_branch_by_branch(qs, p, gamma):
    # from 17 qubits on, runs are chosen over qubit windows and apply commuting gates out of
    # list order between state-dependent draws; branches and Z expectations must still be
    # the oracle's (gamma = 0.05 makes state-dependent draws frequent)
    programs = [(w, synth.random_circuit(w, 4, seed=w)) for w in (17, 18)]
    traj_prog = [0, 1, 0, 1]
    compared, nev = check_against_oracle(qs, programs, traj_prog, 0x5EED17, p, gamma)
    assert compared >= 3
    assert sum(nev) > 0


@pytest.mark.parametrize("p,gamma", [(0.05, 0.05), (0.0, 0.1), (0.08, 0.0), (0.0, 0.0)])
def test_trajectories_match_oracle_branch_by_branch(qs, p, gamma):
    widths = [10, 11, 13, 15]  # 15 lives in global memory, the others in shared memory
    programs = [(w, synth.random_circuit(w, 5, seed=w)) for w in widths]
    ntraj = 12
    traj_prog = [t % len(widths) for t in range(ntraj)]
    seed = 0xABCDEF12345
    zexp, samples, events, nev = qs.qsim_run_trajectories(programs, traj_prog, seed, p, gamma,
                                                          shots=ntraj, event_cap=256)
    for t in range(ntraj):
        w, ops = programs[traj_prog[t]]
        psi, ev_ref, ties = oracle.trajectory(w, ops, seed, t, p, gamma)
        if ties == 0:
            assert events[t] == ev_ref, (t, events[t], ev_ref)
            zr = oracle.z_expectations(psi, w)
            assert np.max(np.abs(zexp[t, :w] - zr)) <= STATE_TOL
            assert np.all(zexp[t, w:] == 0)
            u = oracle.trajectory_sample_draw(seed, t, len(oracle.expand(ops)))
            ref = int(oracle.sample(psi, w, np.array([u]))[0])
            cdf = np.cumsum(np.abs(psi) ** 2)
            j = np.clip(np.searchsorted(cdf, u * cdf[-1]), 1, len(cdf) - 1)
            if min(abs(cdf[j] - u * cdf[-1]), abs(cdf[j - 1] - u * cdf[-1])) > 1e-6:
                assert int(samples[t]) == ref
    if p == 0 and gamma == 0:
        assert all(n == 0 for n in nev)
    else:
        assert sum(nev) > 0


def test_trajectory_average_matches_density_matrix_8q(qs):
    n, depth = 8, 4
    p, gamma = 0.06, 0.08
    ops = synth.random_circuit(n, depth, seed=21)
    exact = oracle.z_from_density(oracle.density_matrix(n, ops, p, gamma), n)
    T = 2000
    zexp, _, _, _ = qs.qsim_run_trajectories([(n, ops)], [0] * T, 4242, p, gamma)
    z = zexp[:, :n]
    mean = z.mean(axis=0)
    sigma = z.std(axis=0, ddof=1) / math.sqrt(T)
    assert np.all(np.abs(mean - exact) <= 3 * sigma + 1e-12), (mean, exact, sigma)
    clean = oracle.z_expectations(oracle.run(n, ops), n)
    assert np.max(np.abs(clean - exact)) > 0.05  # the noise is visible


def test_trajectory_batch_of_uneven_widths_runs(qs):
    # the uneven-width batch shape (widths 14..22 drawn per trajectory) at a reduced count,
    # run from two host threads at once on their own streams (the first launch on a device
    # sets the kernel's shared-memory limit there): both equal a run from one thread
    import threading
    import torch
    widths = synth.trajectory_widths(64, 14, 22, seed=7)
    progs = sorted(set(widths))
    programs = [(w, synth.random_circuit(w, 20, seed=w)) for w in progs]
    traj_prog = [progs.index(w) for w in widths]
    zexp, samples, _, nev = qs.qsim_run_trajectories(programs, traj_prog, 99, 1e-3, 5e-4, shots=64)
    for t, w in enumerate(widths):
        assert np.all(np.abs(zexp[t, :w]) <= 1 + 1e-6)
        assert int(samples[t]) < (1 << w)
    res = [None, None]

    def worker(i):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            res[i] = qs.qsim_run_trajectories(programs, traj_prog, 99, 1e-3, 5e-4, shots=64)

    th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for r in res:
        assert np.array_equal(r[0], zexp) and np.array_equal(r[1], samples) and np.array_equal(r[3], nev)


def test_trajectory_launch_captured_in_a_graph(qs):
    # qsim_traj_launch records into a CUDA graph; replays give bit-identical <Z>, samples
    # and events to a direct launch, and a new seed set between replays gives the results
    # of a direct run with that seed
    import torch
    widths = [12, 15, 17]
    programs = [(w, synth.random_circuit(w, 6, seed=w)) for w in widths]
    traj_prog = [t % 3 for t in range(24)]
    plan = qs.TrajPlan(programs, traj_prog, 2024, 0.02, 0.03, shots=24, event_cap=64, keep=[0, 1, 2])
    plan.launch()
    direct = plan.results()
    states = [plan.state(i) for i in range(3)]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.launch(stream=qs._current_stream())
    g.replay()
    replay = plan.results(stream=qs._current_stream())
    assert np.array_equal(direct[0], replay[0]) and np.array_equal(direct[1], replay[1])
    assert direct[2] == replay[2] and np.array_equal(direct[3], replay[3])
    for i in range(3):
        assert np.array_equal(states[i], plan.state(i))
    plan.set_seed(77)
    g.replay()
    reseeded = plan.results(stream=qs._current_stream())
    ref = qs.qsim_run_trajectories(programs, traj_prog, 77, 0.02, 0.03, shots=24, event_cap=64)
    assert np.array_equal(reseeded[0], ref[0]) and np.array_equal(reseeded[1], ref[1])
    assert reseeded[2] == ref[2]
    assert not np.array_equal(reseeded[0], direct[0])
    plan.close()


def test_trajectory_batch_of_the_bench_shape_vs_oracle(qs):
    # the bench's batch (2048 trajectories, widths drawn uniformly from 14..22, one seeded
    # depth-20 random circuit per width, depolarizing p = 1e-3 and amplitude damping
    # gamma = 5e-4 after every gate on each touched qubit, one shot from each of the first
    # 1024 trajectories), one launch; for every width the first trajectory of that width
    # against the oracle (branches, final state, <Z>, its shot under the near-tie rule)
    widths = synth.trajectory_widths(2048, 14, 22, seed=0)
    progs = sorted(set(widths))
    assert progs == list(range(14, 23))
    programs = [(w, synth.random_circuit(w, 20, seed=w)) for w in progs]
    traj_prog = [progs.index(w) for w in widths]
    picked = [widths.index(w) for w in progs]
    assert max(picked) < 1024  # every picked trajectory also gives one of the 1024 shots
    seed, p, gamma = 0x5EED2048, 1e-3, 5e-4
    plan = qs.TrajPlan(programs, traj_prog, seed, p, gamma, shots=1024, event_cap=64, keep=picked)
    plan.launch()
    zexp, samples, events, nev = plan.results()
    assert sum(nev) > 0
    for t in range(1024):
        assert int(samples[t]) < (1 << widths[t])
    compared = near_shots = 0
    for i, t in enumerate(picked):
        w, ops = programs[traj_prog[t]]
        psi, ev_ref, ties = oracle.trajectory(w, ops, seed, t, p, gamma)
        if ties:
            continue
        compared += 1
        assert events[t] == ev_ref, (w, t, events[t], ev_ref)
        got = plan.state(i).astype(np.complex128)
        assert np.max(np.abs(got - psi)) <= STATE_TOL, w
        assert np.max(np.abs(zexp[t, :w] - oracle.z_expectations(psi, w))) <= STATE_TOL, w
        u = oracle.trajectory_sample_draw(seed, t, len(oracle.expand(ops)))
        ref = int(oracle.sample(psi, w, np.array([u]))[0])
        cdf = np.cumsum(np.abs(psi) ** 2)
        j = np.clip(np.searchsorted(cdf, u * cdf[-1]), 1, len(cdf) - 1)
        if min(abs(cdf[j] - u * cdf[-1]), abs(cdf[j - 1] - u * cdf[-1])) > 1e-6:
            assert int(samples[t]) == ref, (w, t)
        else:
            near_shots += 1
    plan.close()
    msg = "bench-shape batch: %d of %d widths compared branch by branch, %d near-tie shots" % (
        compared, len(progs), near_shots)
    print(msg)
    warnings.warn(msg)  # shown in the run's warnings summary
    assert compared >= len(progs) - 1


ALL_SIX = {"depolarizing": 0.04, "amplitude_damping": 0.05, "bit_flip": 0.96, "phase_flip": 0.95,
           "bit_phase_flip": 0.96, "phase_damping": 0.06}


@pytest.mark.parametrize("noise,noisy,kron", [
    ({"bit_flip": 0.9}, None, False),
    ({"phase_flip": 0.9, "bit_phase_flip": 0.9}, None, False),
    ({"phase_damping": 0.1}, None, False),
    ({"phase_damping": 0.1}, None, True),
    ({"depolarizing": 0.08, "amplitude_damping": 0.06}, None, True),
    (ALL_SIX, None, False),
    (ALL_SIX, None, True),
    ({"depolarizing": 0.05, "phase_damping": 0.1}, {"CZ", "ISWAP", "T"}, False)])
def test_all_eq5_channels_match_oracle_branch_by_branch(qs, noise, noisy, kron):
    # every channel of Eq. 5, per-qubit and joint (Kronecker) draws, noise on chosen gate
    # classes; widths in shared memory (10, 13), global memory (15) and windowed runs (17)
    widths = [10, 13, 15, 17]
    programs = [(w, synth.random_circuit(w, 4, seed=w + 100)) for w in widths]
    traj_prog = [0, 1, 2, 3, 0, 1, 2, 3]
    compared, nev = check_against_oracle(qs, programs, traj_prog, 0xFEED5, 0.0, 0.0, noise=noise, noisy=noisy,
                                         kron=kron)
    assert compared >= 6
    assert sum(nev) > 0


def test_flip_channels_at_p_one_are_noiseless(qs):
    # Eq. 5's flips put sqrt(p) on the identity: p = 1 never flips
    n = 9
    ops = synth.random_circuit(n, 3, seed=5)
    zexp, _, _, nev = qs.qsim_run_trajectories([(n, ops)], [0] * 8, 17, event_cap=8,
                                               noise={"bit_flip": 1.0, "phase_flip": 1.0, "bit_phase_flip": 1.0})
    assert all(v == 0 for v in nev)
    clean = oracle.z_expectations(oracle.run(n, ops), n)
    assert np.max(np.abs(zexp[:, :n] - clean)) <= STATE_TOL


def test_all_channels_average_matches_density_matrix_8q(qs):
    n, depth = 8, 4
    ops = synth.random_circuit(n, depth, seed=23)
    noise = {"depolarizing": 0.05, "amplitude_damping": 0.06, "bit_flip": 0.97, "phase_flip": 0.97,
             "bit_phase_flip": 0.97, "phase_damping": 0.08}
    exact = oracle.z_from_density(oracle.density_matrix(n, ops, noise=noise), n)
    T = 2000
    for kron in (False, True):
        zexp, _, _, _ = qs.qsim_run_trajectories([(n, ops)], [0] * T, 4243, noise=noise, kron=kron)
        z = zexp[:, :n]
        mean = z.mean(axis=0)
        sigma = z.std(axis=0, ddof=1) / math.sqrt(T)
        assert np.all(np.abs(mean - exact) <= 3 * sigma + 1e-12), (kron, mean, exact, sigma)
    clean = oracle.z_expectations(oracle.run(n, ops), n)
    assert np.max(np.abs(clean - exact)) > 0.05


@pytest.mark.parametrize("kw", [dict(noise={"phase_damping": 1.5}), dict(noise={"bit_flip": -0.1}),
                                dict(p_depol=2.0)])
def test_bad_noise_parameters_are_rejected(qs, kw):
    with pytest.raises(Exception):
        qs.qsim_run_trajectories([(4, [("H", (0,), ())])], [0], 1, **kw)


def test_trajectory_extreme_widths_vs_oracle(qs):
    # the narrowest state (2 qubits) and the widest (QSIM_TRAJ_MAX_QUBITS = 24, in global
    # memory with windowed runs) against the oracle, branch by branch
    programs = [(2, synth.random_circuit(2, 6, seed=2)), (24, synth.random_circuit(24, 1, seed=24, tail=False))]
    traj_prog = [0, 0, 0, 1]
    compared, nev = check_against_oracle(qs, programs, traj_prog, 0xE0E0, 0.06, 0.08)
    assert compared >= 3
    assert sum(nev) > 0
    with pytest.raises(qs.QsimError):
        qs.qsim_run_trajectories([(25, [("H", (0,), ())])], [0], 1)
