"""Benchmark: state-vector gates/s and HBM GB/s on the 28-qubit depth-40 random circuit.

One step = one run of the whole circuit (1714 listed gates) on a state reset to |0...0>,
inputs resident in HBM. Paths: per-gate FP64 (complex128), per-gate FP32 (complex64) and
fused FP32 (complex64, k-qubit unitaries composed in FP64 on the host, applied by the
fused kernel). The headline `value` is the fused FP32 path; the other paths are reported
beside it. The state (2 GiB / 4 GiB) is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own circuit instance (seed = rank) on its own GPU, with
no collective on the data path (weak scaling); rank 0 prints one JSON line.
"""

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS = 28
DEPTH = 40
METRIC = "state-vector gates/s and HBM GB/s (% of peak), fused FP32 vs per-gate FP64"
# DRAM bytes (read + write) of one k_fused_tc<5> launch on the 28-qubit state, from one ncu
# capture of the current kernel (--set full on the profile case `fused c64 28`); None when
# the kernel has changed since the counters were taken.
FUSED_TRAFFIC_BYTES = 2.147630e9 + 2.086106e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest value over all ranks (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank, ms, world):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank / (max_over_ranks(ms, world) * 1e-3)


def time_path(qs, torch, ops, dtype, fuse, steps, warmup, world, use_graph=False, native=False, merge=False):
    """Device time of `steps` circuit runs (events on the state's stream)."""
    st = qs.State(N_QUBITS, dtype)
    if native:
        st.set_fp64_native(True)
    for _ in range(warmup):
        st.reset()
        st.run_circuit(ops, fuse=fuse, remap=True, use_graph=use_graph, merge_diagonals=merge)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        st.reset()
        st.run_circuit(ops, fuse=fuse, remap=True, use_graph=use_graph, merge_diagonals=merge)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / steps
    stats = st.stats()
    norm = st.norm()
    del st
    torch.cuda.empty_cache()
    return ms, stats, norm


def time_kernel(qs, torch, dtype, reps=20, native=False):
    """Average duration of the dominant per-gate kernel (generic 1-qubit pair sweep on a
    middle target) measured with CUDA events; returns (ms, algorithmic bytes)."""
    import numpy as np
    st = qs.State(N_QUBITS, dtype)
    if native:
        st.set_fp64_native(True)
    rng = np.random.default_rng(5)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u, _ = np.linalg.qr(z)
    for _ in range(3):
        st.apply_gate([14], u)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        st.apply_gate([14], u)
    e1.record()
    torch.cuda.synchronize()
    B = 16 if dtype == "c128" else 8
    del st
    torch.cuda.empty_cache()
    return e0.elapsed_time(e1) / reps, 2 * B * (1 << N_QUBITS)


def time_targets(qs, torch, dtype, reps=20, n=N_QUBITS):
    """Per-gate sweep bandwidth for each target position 0..n-1 and each gate class: a
    random 1-qubit unitary (generic), a real rotation RY (real), T = diag(1, e^(i pi/4))
    (diagonal: only the amplitudes with the target bit set change) and X (permutation).
    CUDA events over `reps` launches per (class, target); algorithmic bytes per class."""
    import numpy as np
    st = qs.State(n, dtype)
    rng = np.random.default_rng(6)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    gen, _ = np.linalg.qr(z)
    th = 0.37
    classes = {"generic": (gen, 1.0),
               "real": (np.array([[np.cos(th / 2), -np.sin(th / 2)], [np.sin(th / 2), np.cos(th / 2)]]), 1.0),
               "diagonal": (np.diag([1.0, np.exp(0.25j * np.pi)]), 0.5),
               "permutation": (np.array([[0.0, 1.0], [1.0, 0.0]]), 1.0)}
    B = 16 if dtype == "c128" else 8
    out = {}
    for name, (u, frac) in classes.items():
        row = []
        for t in range(n):
            st.apply_gate([t], u)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                st.apply_gate([t], u)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row.append(round(frac * 2 * B * (1 << n) / (ms * 1e-3) / 1e9, 1))
        out[name] = row
    # the diagonal class at DRAM-sector granularity: where the two halves of a pair share a
    # 32-byte sector (2^t B < 32) the untouched half is read and written all the same
    out["diagonal_sector_bytes"] = [round(v * (2.0 if (1 << t) * B < 32 else 1.0), 1)
                                    for t, v in enumerate(out["diagonal"])]
    st.close()
    del st
    torch.cuda.empty_cache()
    return out


def time_diag_merge(qs, torch, dtype, hbm_peak, reps=10):
    """The merged diagonal sweep against the per-gate sweeps it replaces: T on qubits 0..9
    and CZ on (0, 1), (2, 3), ..., (8, 9) of the 28-qubit state, 15 diagonal gates on low
    qubits, where a per-gate phase sweep moves whole 32-byte sectors. CUDA events around
    `reps` runs of the 15 gates, per gate and merged (one table sweep over 10 qubits)."""
    ops = [("T", (q,), ()) for q in range(10)] + [("CZ", (q, q + 1), ()) for q in range(0, 10, 2)]
    B = 16 if dtype == "c128" else 8
    out = {"gates": len(ops)}
    for merge in (False, True):
        st = qs.State(N_QUBITS, dtype)
        for _ in range(2):
            st.run_circuit(ops, merge_diagonals=merge)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            st.run_circuit(ops, merge_diagonals=merge)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        stats = st.stats()
        st.close()
        del st
        torch.cuda.empty_cache()
        out["merged" if merge else "per_gate"] = {"ms": ms, "sweeps": stats["sweeps"],
                                                  "diag_sweeps": stats["diag_sweeps"]}
    m = out["merged"]
    m["achieved_gbs"] = 2 * B * (1 << N_QUBITS) / (m["ms"] * 1e-3) / 1e9
    m["frac"] = m["achieved_gbs"] / hbm_peak
    out["speedup"] = out["per_gate"]["ms"] / m["ms"]
    return out


def readout_report(qs, torch, hbm_peak, reps=5):
    """The read-outs (Section 2.1's norm / PMEASURE / sampling, fidelity) on 28-qubit states
    after the random circuit: host wall time per call (each call returns its result to the
    host, so it includes the synchronisation), median of `reps`, and the algorithmic bytes
    (each state read once) over that time as a fraction of the measured HBM bandwidth."""
    import statistics
    import synth
    ops = synth.random_circuit(N_QUBITS, DEPTH, seed=11)
    out = {}
    for dtype in ("c64", "c128"):
        B = 16 if dtype == "c128" else 8
        st, other = qs.State(N_QUBITS, dtype), qs.State(N_QUBITS, dtype)
        st.run_circuit(ops, fuse=5 if dtype == "c64" else 4, remap=True)
        other.run_circuit(ops[: len(ops) // 2], fuse=5 if dtype == "c64" else 4, remap=True)
        st.canonicalize()
        other.canonicalize()
        torch.cuda.synchronize()
        one = B * (1 << N_QUBITS)
        calls = {"norm": (st.norm, one), "inner": (lambda: st.inner(other), 2 * one),
                 "expect_z": (st.expect_z, one),
                 "probabilities_q0_9": (lambda: st.probabilities(list(range(10))), one),
                 "probabilities_q18_27": (lambda: st.probabilities(list(range(18, 28))), one),
                 "sample_1024": (lambda: st.sample(1024, 7), 2 * one)}
        rep = {}
        for name, (fn, nbytes) in calls.items():
            fn()
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                fn()
                ts.append((time.perf_counter() - t0) * 1e3)
            ms = statistics.median(ts)
            rep[name] = {"ms": ms, "bytes": nbytes, "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak}
        out[dtype] = rep
        st.close()
        other.close()
        del st, other
        torch.cuda.empty_cache()
    return out


def time_fused_kernel(qs, torch, k=5, reps=20):
    """Average duration of the fused tensor-core kernel (k-qubit unitary on qubits 0..k-1
    of the 28-qubit complex64 state) with CUDA events; returns (ms, algorithmic bytes)."""
    import numpy as np
    st = qs.State(N_QUBITS, "c64")
    rng = np.random.default_rng(6)
    z = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    u, _ = np.linalg.qr(z)
    q = list(range(k - 1, -1, -1))
    for _ in range(3):
        st.apply_fused(q, u)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        st.apply_fused(q, u)
    e1.record()
    torch.cuda.synchronize()
    del st
    torch.cuda.empty_cache()
    return e0.elapsed_time(e1) / reps, 2 * 8 * (1 << N_QUBITS)


def e2e_path(qs, torch, ops, dtype, fuse, steps, readout=10):
    """One end-to-end step through the C ABI as the paper's programs use the simulator
    (QINIT, the gates, PMEASURE): qsim_reset sets |0...0> on the device, qsim_run_circuit
    takes the gate list from host memory (the plan's matrices go host-to-device from the
    state's pinned staging buffer), and qsim_probabilities of `readout` qubits brings 2^readout
    FP64 probabilities back (device-to-host, synchronising). `steps` (>= 5) steps after one
    warm-up; per step the wall time and CUDA events on the state's stream. Returns (median
    step seconds, host-to-device bytes, device-to-host bytes, report)."""
    import numpy as np
    st = qs.State(N_QUBITS, dtype)
    qubits = list(range(readout))

    def one_step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[0].record()
        st.reset()
        st.run_circuit(ops, fuse=fuse, remap=True)
        ev[1].record()
        probs = st.probabilities(qubits)  # synchronises the stream
        ev[2].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return wall, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), probs

    one_step()  # warm-up (plans the circuit; later steps reuse the plan)
    walls, dev, rd = [], [], []
    for _ in range(max(5, steps)):
        w, d, r, probs = one_step()
        walls.append(w)
        dev.append(d)
        rd.append(r)
    up = st.stats()["upload_bytes"]
    ok = abs(float(np.sum(probs)) - 1.0) < 1e-3
    st.close()
    del st
    torch.cuda.empty_cache()
    med = float(np.median(walls))
    rep = {"steps": len(walls), "median_ms": 1e3 * med, "min_ms": 1e3 * min(walls), "max_ms": 1e3 * max(walls),
           "step_ms": [round(1e3 * w, 2) for w in walls],
           "device_reset_circuit_ms_median": float(np.median(dev)), "readout_ms_median": float(np.median(rd)),
           "final_probabilities_sum_ok": ok,
           "step": "qsim_reset, qsim_run_circuit (gate list from host), qsim_probabilities of qubits "
                   "0..%d (%d FP64 values to the host)" % (readout - 1, 1 << readout)}
    return med, up, 8 << readout, rep


def state_io_path(qs, torch, ops, dtype, fuse, steps):
    """Same circuit through the C ABI with the whole state in host buffers, `steps` (>= 5) steps
    after one warm-up: pinned host -> device copy of the initial state, the circuit, the
    restore of logical qubit order, device -> host copy of the final state. Per step the
    wall time and the phases: CUDA events on the state's stream around each call (h2d,
    device, restore, d2h) and the host time the circuit call takes to plan and launch.
    Returns (median step seconds, bytes each way, norm check, report dict)."""
    import numpy as np
    nbytes = (16 if dtype == "c128" else 8) << N_QUBITS
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    host_in = torch.zeros(1 << N_QUBITS, dtype=tdt, pin_memory=True)
    host_in[0] = 1.0
    host_out = torch.empty(1 << N_QUBITS, dtype=tdt, pin_memory=True)
    st = qs.State(N_QUBITS, dtype)
    lib = qs.lib()
    pin_in = ctypes.c_void_p(host_in.data_ptr())
    pin_out = ctypes.c_void_p(host_out.data_ptr())

    def one_step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[0].record()
        qs._check(lib.qsim_copy_from_host(st.handle, pin_in))
        ev[1].record()
        h0 = time.perf_counter()
        st.run_circuit(ops, fuse=fuse, remap=True)
        host_launch = time.perf_counter() - h0
        ev[2].record()
        qs._check(lib.qsim_canonicalize(st.handle))
        ev[3].record()
        qs._check(lib.qsim_copy_to_host(st.handle, pin_out))  # synchronises the stream
        ev[4].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ph = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        return wall, {"h2d_ms": ph[0], "device_ms": ph[1], "restore_ms": ph[2], "d2h_ms": ph[3],
                      "plan_launch_host_ms": 1e3 * host_launch}

    one_step()  # warm-up (plans the circuit; later steps reuse the plan)
    walls, phases = [], []
    for _ in range(max(5, steps)):
        w, ph = one_step()
        walls.append(w)
        phases.append(ph)
    ok = abs(float(np.sum(np.abs(host_out.numpy()) ** 2)) - 1.0) < 1e-3
    st.close()
    del st
    torch.cuda.empty_cache()
    med = float(np.median(walls))
    dev_keys = ("h2d_ms", "device_ms", "restore_ms", "d2h_ms")
    sums = [sum(p[k] for k in dev_keys) for p in phases]  # stream time of each step
    gaps = [1e3 * w - t for w, t in zip(walls, sums)]     # wall time the stream was not busy
    rep = {"steps": len(walls), "median_ms": 1e3 * med, "min_ms": 1e3 * min(walls), "max_ms": 1e3 * max(walls),
           "step_ms": [round(1e3 * w, 2) for w in walls],
           "phases_median_ms": {k: float(np.median([p[k] for p in phases])) for k in phases[0]},
           "phases_ms_per_step": [{k: round(v, 2) for k, v in p.items()} for p in phases],
           "phases_sum_median_ms": float(np.median(sums)),
           "phases_sum_ms_per_step": [round(t, 2) for t in sums],
           "host_gap_median_ms": float(np.median(gaps))}
    return med, nbytes, ok, rep


def trajectory_batch(qs, torch, world, rank):
    """2048 noisy trajectories (widths drawn from 14..22, depth-20 random circuits per width,
    depolarizing p = 1e-3 and amplitude damping gamma = 5e-4 after every gate on each
    touched qubit), one persistent launch; wall time of the whole C call (programs up,
    kernel, results down), best of 2 after one warm-up."""
    import synth
    widths = synth.trajectory_widths(2048, 14, 22, seed=rank)
    progs = sorted(set(widths))
    programs = [(w, synth.random_circuit(w, 20, seed=w)) for w in progs]
    traj_prog = [progs.index(w) for w in widths]
    gates = {w: synth.count_gates(ops) for w, ops in programs}
    qs.qsim_run_trajectories(programs, traj_prog, 1, 1e-3, 5e-4, shots=1024)
    best = None
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        zexp, samples, _, nev = qs.qsim_run_trajectories(programs, traj_prog, 1 + rep, 1e-3, 5e-4, shots=1024)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    total_gates = sum(gates[w] for w in widths)
    amp_updates = sum(gates[w] * (1 << w) for w in widths)
    # algorithmic FP32 flops: a gate on k qubits is 2^k complex multiply-adds (8 flops each)
    # per amplitude (the random circuits have no blocks, so op[1] lists every touched qubit)
    flops_w = {w: sum(8 * (1 << len(op[1])) for op in ops if op[0] not in synth.BLOCK_MARKERS) * (1 << w)
               for w, ops in programs}
    flops = sum(flops_w[w] for w in widths)
    return {"trajectories": len(widths), "widths": "14..22 (uniform draw)", "depth": 20,
            "p_depol": 1e-3, "gamma": 5e-4, "shots": 1024, "seconds": best,
            "trajectories_per_s": len(widths) / best, "gate_applications_per_s": total_gates / best,
            "amplitude_updates_per_s": amp_updates / best, "algorithmic_flops": flops,
            "branch_events": int(sum(nev)),
            "launches": 1}


def partial_amplitude_mode(qs, torch):
    """Partial amplitude mode (Section 2.2): a 48-qubit two-block circuit (24 + 24 qubits,
    depth 10, six controlled gates across the dividing line, so 2^7 sub-circuits), 2^20
    requested amplitudes; wall time of the whole C call (indices up, prefix-shared
    sub-circuit runs through the fused engine, FP64 gather, amplitudes down), best of 2
    after one warm-up."""
    import numpy as np
    import synth
    n, depth, cross = 48, 10, 6
    ops = synth.partial_circuit(n, depth, cross, seed=48)
    xs = np.random.default_rng(48).integers(0, 1 << n, size=1 << 20, dtype=np.uint64)
    _, info = qs.qsim_partial_amplitudes(n, ops, xs, dtype="c64", fuse=5, remap=True)
    best = None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qs.qsim_partial_amplitudes(n, ops, xs, dtype="c64", fuse=5, remap=True)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    gate_amps = info["gates_applied"] * (1 << 24)
    return {"qubits": n, "cut": info["cut"], "depth": depth, "decomposed": info["decomposed"],
            "subcircuits": info["subcircuits"], "segment_runs": info["segment_runs"],
            "gate_applications": info["gates_applied"],
            "gate_applications_unshared": info["gates_unshared"], "sweeps": info["sweeps"],
            "standalone_remaps": info["remaps"], "amplitudes": int(xs.size),
            "dtype": "c64", "fuse": 5, "seconds": best, "amplitudes_per_s": xs.size / best,
            "gate_amplitude_updates_per_s": gate_amps / best}


def spread_sample(gates, count):
    """`count` gates taken at evenly spaced positions of the whole list, in list order."""
    count = max(1, min(count, len(gates)))
    return [gates[(i * len(gates)) // count] for i in range(count)]


def cpu_baseline(ops, count=200):
    """The FP64 oracle as it stands, on this host's cores: `count` gates spread evenly over
    the circuit (one-, two-qubit and controlled gates in the circuit's mix) applied to a
    28-qubit complex128 state, timed; the sample is the whole of the timed work."""
    import oracle
    gates = oracle.expand(ops)
    sample = spread_sample(gates, count)
    psi = oracle.zero_state(N_QUBITS)
    oracle.apply(psi, N_QUBITS, *sample[0])  # first touch of the 4 GiB state, untimed
    t0 = time.perf_counter()
    for qubits, controls, m in sample:
        oracle.apply(psi, N_QUBITS, qubits, controls, m)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    del psi
    return {"value": len(sample) / dt, "unit": "gates/s", "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": "%d of the %d gates of the %d-qubit depth-%d circuit, evenly spaced over it, "
                      "complex128, %.1f s" % (len(sample), len(gates), N_QUBITS, DEPTH, dt)}


def timed_run(torch, st, ops, fuse, renorm=True):
    """One run of `ops` from |0...0> on the state, CUDA events on its stream; returns ms."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st.reset()
    e0.record()
    st.run_circuit(ops, fuse=fuse, remap=True, renorm=renorm)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def path_entry(st, ngates, ms, hbm_peak):
    stats = st.stats()
    gbs = stats["bytes"] / (ms * 1e-3) / 1e9
    return {"gates_per_s": ngates / (ms * 1e-3), "ms": ms, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
            "sweeps": stats["sweeps"], "fused_blocks": stats["fused_blocks"], "remaps": stats["remaps"],
            "epilogue_remaps": stats["epilogue_remaps"], "phase_gates": stats["phase_gates"],
            "fuse_width": stats["fuse_width"]}


def largest_state_report(qs, torch, hbm_peak, local):
    """The largest single state: a 34-qubit complex64 random circuit of depth 24 (128 GiB),
    fused with the autotuned width (remaps included) against the plain per-gate path on the
    same circuit; fused: one warm-up and one timed run, then the inverse circuit and the
    FP64 compute-uncompute fidelity; per gate: one timed run."""
    import synth
    n, depth = 34, 24
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << n) + (4 << 30):
        return {"skipped": "needs 132 GiB of free device memory, %.1f GiB free" % (free / 2 ** 30)}
    ops = synth.random_circuit(n, depth, seed=4)
    ngates = synth.count_gates(ops)
    st = qs.State(n, "c64")
    out = {"workload": "random circuit, 34 qubits, depth 24, %d gates, complex64 (128 GiB)" % ngates}
    with ClockSampler(local) as clk:
        st.reset()
        st.run_circuit(ops, fuse=-1, remap=True)  # warm-up (autotuner, plan)
        ms = timed_run(torch, st, ops, -1)
        fused = path_entry(st, ngates, ms, hbm_peak)
        fused["norm_after"] = st.norm()
        st.run_circuit(synth.inverse_ops(ops), fuse=-1, remap=True)
        fused["uncompute_fidelity"] = abs(st.amplitude(0)) ** 2 / st.norm()
        out["fused_autotuned"] = fused
        ms = timed_run(torch, st, ops, 0)
        plain = path_entry(st, ngates, ms, hbm_peak)
        plain["norm_after"] = st.norm()
        out["per_gate_fp32"] = plain
    out["clocks"] = clk.summary()
    out["fused_vs_per_gate"] = out["fused_autotuned"]["gates_per_s"] / out["per_gate_fp32"]["gates_per_s"]
    st.close()
    del st
    torch.cuda.empty_cache()
    return out


def qft32_report(qs, torch, hbm_peak, local):
    """Precision + fusion at scale: a 32-qubit complex64 state (32 GiB) through QFT(32) and
    a depth-30 random circuit, fused at k = 4 and 5 on the tensor cores (and at k = 5 with
    the renormalisation off, for the raw FP64 norm drift), against the plain per-gate path;
    FP64 norm drift after the circuit and the fidelity of circuit then inverse with
    |0...0>."""
    import synth
    n = 32
    ops = synth.qft_circuit(n) + synth.random_circuit(n, 30, seed=3)
    inv = synth.inverse_ops(ops)
    ngates = synth.count_gates(ops)
    st = qs.State(n, "c64")
    out = {"workload": "QFT(32) + random depth 30, %d gates, complex64 (32 GiB)" % ngates}
    with ClockSampler(local) as clk:
        for name, fuse, renorm in (("fused_k4", 4, True), ("fused_k5", 5, True), ("fused_k5_no_renorm", 5, False),
                                   ("per_gate_fp32", 0, True)):
            if fuse:
                st.reset()
                st.run_circuit(ops, fuse=fuse, remap=True, renorm=renorm)  # warm-up (plan)
            ms = timed_run(torch, st, ops, fuse, renorm)
            entry = path_entry(st, ngates, ms, hbm_peak)
            entry["norm_drift"] = st.norm() - 1.0
            if fuse:
                st.run_circuit(inv, fuse=fuse, remap=True, renorm=renorm)
                entry["uncompute_fidelity"] = abs(st.amplitude(0)) ** 2 / st.norm()
                entry["uncompute_norm_drift"] = st.norm() - 1.0
            out[name] = entry
    out["clocks"] = clk.summary()
    out["fused_k5_vs_per_gate"] = out["fused_k5"]["gates_per_s"] / out["per_gate_fp32"]["gates_per_s"]
    st.close()
    del st
    torch.cuda.empty_cache()
    return out


def per_gate_fp64_30q_report(qs, torch, hbm_peak, local):
    """The per-gate FP64-accurate path at 30 qubits (complex128, 16 GiB, split format): the
    30-qubit depth-40 random circuit, one sweep per gate (one timed run after a warm-up on
    its first 64 gates), and every target position 0..29 of each gate class (5 launches
    each)."""
    import synth
    n = 30
    ops = synth.random_circuit(n, DEPTH, seed=0)
    ngates = synth.count_gates(ops)
    out = {"workload": "random circuit, 30 qubits, depth 40, %d gates, complex128 (16 GiB), per gate" % ngates}
    with ClockSampler(local) as clk:
        st = qs.State(n, "c128")
        st.run_circuit(ops[:64], fuse=0)
        ms = timed_run(torch, st, ops, 0)
        out["per_gate_fp64"] = path_entry(st, ngates, ms, hbm_peak)
        out["per_gate_fp64"]["norm_after"] = st.norm()
        out["per_gate_fp64"]["dtype"] = "f64-accurate split (FP32 pipe)"
        st.close()
        del st
        torch.cuda.empty_cache()
        tg = time_targets(qs, torch, "c128", reps=5, n=n)
    out["clocks"] = clk.summary()
    out["per_target_gbs"] = tg
    out["per_target_min_frac"] = {c: min(v) / hbm_peak for c, v in tg.items()}
    torch.cuda.empty_cache()
    return out


def arm_config(args, world):
    return {"workload": "random circuit, 28 qubits, depth 40, 1714 gates",
            "qubits": N_QUBITS, "depth": DEPTH, "gate_set": "H SX SY T + CZ brick + CNOT ladder + CR layer",
            "fuse": args.fuse, "parallelism": "replicas" if world > 1 else "single",
            "l2": "state (2-4 GiB) larger than L2, no flush"}


REF_SAMPLE = 32  # gates per reference step, evenly spaced over the 28-qubit circuit


def run_reference(args, world, rank):
    """The FP64 oracle as it stands on the host cores. One step = the same REF_SAMPLE gates,
    evenly spaced over the 28-qubit depth-40 circuit (its mix of one-, two-qubit and
    controlled gates), applied to one 4 GiB complex128 state; every step is timed whole, so
    ms_per_step is a measured time and `value` = sample gates / measured time."""
    if rank != 0:
        return
    import oracle
    import synth
    ops = synth.random_circuit(N_QUBITS, DEPTH, seed=0)
    gates = oracle.expand(ops)
    sample = spread_sample(gates, REF_SAMPLE)
    psi = oracle.zero_state(N_QUBITS)
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for qubits, controls, m in sample:
            oracle.apply(psi, N_QUBITS, qubits, controls, m)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = len(sample) / (ms * 1e-3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = ("%d of the %d gates of the %d-qubit depth-%d circuit, evenly spaced over it, complex128, per step"
            % (len(sample), len(gates), N_QUBITS, DEPTH))
    cfg = arm_config(args, world)
    cfg["step"] = desc
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "gates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "gates/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fuse", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="leave out the 30-, 32- and 34-qubit reports of the bench line")
    ap.add_argument("--workload", default="rqc28", choices=["rqc28", "rqc34", "qft32", "fp64_30q"],
                    help="rqc34 / qft32 / fp64_30q: print only that report instead of the bench line")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    from paper_2008_07140_gb300 import build as qbuild
    if rank == 0 or not qbuild.up_to_date():
        qbuild.build()
    barrier(world)
    import paper_2008_07140_gb300 as qs

    hbm_peak, peak_src = measured_peaks()
    reports = {"rqc34": largest_state_report, "qft32": qft32_report, "fp64_30q": per_gate_fp64_30q_report}
    if args.workload in reports:
        if rank == 0:
            print(json.dumps(reports[args.workload](qs, torch, hbm_peak, local)), flush=True)
        return
    ops = synth.random_circuit(N_QUBITS, DEPTH, seed=rank)
    ngates = synth.count_gates(ops)

    # headline first: fused FP32, timed with clocks sampled
    with ClockSampler(local) as clk:
        ms, stats, norm = time_path(qs, torch, ops, "c64", args.fuse, args.steps, args.warmup, world)
    ms = max_over_ranks(ms, world)
    value = world * ngates / (ms * 1e-3)
    gbs = stats["bytes"] / (ms * 1e-3) / 1e9
    paths = {"fused_fp32": {"gates_per_s": value, "ms_per_step": ms, "hbm_gbs": gbs,
                            "hbm_frac": gbs / hbm_peak, "sweeps": stats["sweeps"],
                            "fused_blocks": stats["fused_blocks"], "remaps": stats["remaps"],
                            "norm_after": norm, "dtype": "f32"}}

    # secondary paths (fewer steps)
    sub_steps = max(1, min(args.steps, 2))
    for name, dtype, fuse, native, merge in (
            ("per_gate_fp64", "c128", 0, False, False), ("per_gate_fp32", "c64", 0, False, False),
            ("per_gate_fp64_merged_diagonals", "c128", 0, False, True),
            ("per_gate_fp32_merged_diagonals", "c64", 0, False, True),
            ("per_gate_fp64_native_instructions", "c128", 0, True, False),
            ("fused_fp64_autotuned", "c128", -1, False, False)):
        pms, pstats, pnorm = time_path(qs, torch, ops, dtype, fuse, sub_steps, 1, world, native=native, merge=merge)
        pms = max_over_ranks(pms, world)
        pgbs = pstats["bytes"] / (pms * 1e-3) / 1e9
        paths[name] = {"gates_per_s": world * ngates / (pms * 1e-3), "ms_per_step": pms,
                       "hbm_gbs": pgbs, "hbm_frac": pgbs / hbm_peak, "sweeps": pstats["sweeps"],
                       "fuse_width": pstats["fuse_width"], "norm_after": pnorm,
                       "dtype": ("f64 (FP64 instructions)" if native else "f64-accurate split (FP32 pipe)")
                       if dtype == "c128" else "f32"}
        if merge:
            paths[name]["diag_sweeps"] = pstats["diag_sweeps"]
            paths[name]["diag_gates"] = pstats["diag_gates"]

    # per-gate sweep bandwidth at every target position, per gate class
    for name, dtype in (("per_gate_fp64", "c128"), ("per_gate_fp32", "c64")):
        tg = time_targets(qs, torch, dtype)
        paths[name]["per_target_gbs"] = tg
        paths[name]["per_target_min_frac"] = {c: min(v) / hbm_peak for c, v in tg.items()}

    # dominant kernel of the headline path, live (and the per-gate sweeps beside it)
    fms, fbytes = time_fused_kernel(qs, torch, 5)
    kms, kbytes = time_kernel(qs, torch, "c64")
    kms64, kbytes64 = time_kernel(qs, torch, "c128")
    kms64n, kbytes64n = time_kernel(qs, torch, "c128", native=True)
    achieved = fbytes / (fms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": FUSED_TRAFFIC_BYTES,
            "kernel": "k_fused_tc<5>: 3xTF32 fused 5-qubit unitary, complex64, 28 qubits, %.3f ms" % fms,
            "algorithmic_bytes": fbytes, "peak_source": peak_src + " hbm_gbs (copy)",
            "other_kernels": {
                "k_pair_c64": {"achieved": kbytes / (kms * 1e-3) / 1e9,
                               "frac": kbytes / (kms * 1e-3) / 1e9 / hbm_peak, "ms": kms},
                "k_pair_df_c128_split": {"achieved": kbytes64 / (kms64 * 1e-3) / 1e9,
                                         "frac": kbytes64 / (kms64 * 1e-3) / 1e9 / hbm_peak,
                                         "ms": kms64},
                "k_pair_c128_fp64_instructions": {"achieved": kbytes64n / (kms64n * 1e-3) / 1e9,
                                                  "frac": kbytes64n / (kms64n * 1e-3) / 1e9 / hbm_peak,
                                                  "ms": kms64n},
                "k_diag_c64_merged_low_diagonals": time_diag_merge(qs, torch, "c64", hbm_peak),
                "k_diag_df_c128_merged_low_diagonals": time_diag_merge(qs, torch, "c128", hbm_peak)}}

    # end to end through the C ABI: |0...0> on the device, the gate list from the host, PMEASURE
    # of ten qubits back; beside it the same circuit with the whole 2 GiB state copied in and out
    e2e_dt, h2d, d2h, e2e_rep = e2e_path(qs, torch, ops, "c64", args.fuse, args.steps)
    e2e = {"value": world * ngates / max_over_ranks(e2e_dt, world), "unit": "gates/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    e2e.update(e2e_rep)
    io_dt, nbytes, io_ok, io_rep = state_io_path(qs, torch, ops, "c64", args.fuse, args.steps)
    e2e["whole_state_io"] = dict(io_rep, value=world * ngates / max_over_ranks(io_dt, world),
                                 h2d_bytes_per_step=nbytes, d2h_bytes_per_step=nbytes, final_norm_ok=io_ok)

    with ClockSampler(local) as tclk:
        traj = trajectory_batch(qs, torch, world, rank)
    traj["clocks"] = tclk.summary()
    sm_mhz = traj["clocks"]["sm_mhz"] or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x clock
    achieved_t = traj["algorithmic_flops"] / traj["seconds"] / 1e12
    traj["roofline"] = {"bound": "alu", "achieved": achieved_t, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": achieved_t / fp32_peak,
                        "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x sampled SM clock",
                        "flops": "8 * 2^k per amplitude per gate on k qubits (k = 1, 2), all gates of "
                                 "all trajectories, over the whole call's wall time"}
    partial = partial_amplitude_mode(qs, torch)
    readouts = readout_report(qs, torch, hbm_peak)

    large = {}
    if world == 1 and not args.quick:
        large["per_gate_fp64_30q"] = per_gate_fp64_30q_report(qs, torch, hbm_peak, local)
        large["qft32_fused"] = qft32_report(qs, torch, hbm_peak, local)
        large["largest_state_34q"] = largest_state_report(qs, torch, hbm_peak, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ops)

    launches = (stats["kernels"] + 1) * args.steps
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": arm_config(args, world),
                "paths": paths,
                "fused_vs_fp64": value / paths["per_gate_fp64"]["gates_per_s"],
                "fused_vs_per_gate_fp32": value / paths["per_gate_fp32"]["gates_per_s"],
                "fused_vs_per_gate_fp32_merged_diagonals":
                    value / paths["per_gate_fp32_merged_diagonals"]["gates_per_s"],
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "noisy_trajectories": traj,
                "partial_amplitude_mode": partial, "readouts": readouts,
                "gpu_launches": launches, "clocks": clk.summary()}
        line.update(large)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
