#!/usr/bin/env python3
"""Benchmark of the state-vector hot path on GB300.

Workload (default): 30-qubit random circuit on a 5x6 grid, depth 20, sqrt(X/Y/W)
single-qubit gates and fSim(pi/2, pi/6) on four cycling edge patterns (845
gates), complex64 state (8 GiB, far larger than the 129 MB L2), fused into
blocks of at most 6 qubits applied on the tensor cores (FP16 hi+lo split).
One step = initialise |0..0>, apply every fused block, and reduce the squared
norm in FP64 -- the whole hot path.  The other workloads (per-gate path,
complex128, n=33 tensor-core vs CUDA-core blocks, adjoint gradients, the
512-circuit batch) are measured after the main line and reported under
"extras".

metric: gate-apps/s = unfused gates applied per second (whole job).
Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle (a
plain complex128 C implementation) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2111_06868_gb300 import circuits as C  # noqa: E402

METRIC = "gate-apps/s"
ARITH = {"tc_f16": "fp16 hi+lo split operands (3 products), fp32 accumulate in TMEM, fp64 norm",
         "tc_bf16": "bf16 hi+lo split operands (3 products), fp32 accumulate in TMEM, fp64 norm",
         "tc_pass": "fp16 hi+lo split operands (3 products), fp32 accumulate in TMEM, fp64 norm",
         "cuda_core": "fp32 FMA on CUDA cores, fp64 norm", "auto": "fp32 FMA on CUDA cores, fp64 norm",
         "df": "double-float (hi + lo fp32 pairs, error-free products and sums) on CUDA cores, fp64 norm",
         "tc_c128": "dense k=3,4 blocks: fp16 products of 8-bit digit slices (6 per operand), exact fp32 "
                    "accumulate per level, levels joined in 64-bit integers; other gates double-float; fp64 norm"}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


def workload(args, rank):
    if args.workload == "n30":
        circ = C.config_n30(seed=args.seed + rank)
        desc = "n=30 5x6 grid depth-20 fSim(pi/2,pi/6) random circuit, 845 gates"
    elif args.workload == "n33":
        circ = C.config_n33(seed=args.seed + rank)
        desc = "n=33 6x6-minus-3-corners depth-24 fSim random circuit, 1116 gates"
    elif args.workload == "n27":
        circ = C.random_circuit(C.grid(5, 6, first=27), 20, args.seed + rank, "fsim")
        desc = "n=27 (first 27 sites of the 5x6 grid) depth-20 fSim random circuit (profiling size)"
    elif args.workload == "n12":
        circ = C.config_small(seed=args.seed + rank)
        desc = "n=12 3x4 grid depth-10 CZ random circuit, 163 gates"
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    return circ, desc


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def fuse(hq, n, gates, kmax, args):
    """The fusion step (host): hq_fuse_beam by default (--fuse-width kept
    sequences), hq_fuse_dag on --fuse dag, hq_fuse on --fuse greedy."""
    return hq.hq_fuse(n, gates, kmax, method=args.fuse, restarts=args.fuse_restarts, width=args.fuse_width)


def kernel_sources_sha(kernel_class):
    """Hash of the sources the kernel class is built from (ties ncu traffic
    figures to the code they were measured on)."""
    import hashlib

    files = {"k_tcz": ["k_tcz.cu", "hq_tcgen05.cuh"], "k_tc": ["k_tc.cu", "hq_tcgen05.cuh"], "k_gather": ["k_apply.cu"], "k_diag": ["k_apply.cu"], "k_block": ["k_apply.cu"]}
    key = next((k for k in files if kernel_class.startswith(k)), None)
    if key is None:
        return None
    h = hashlib.sha256()
    for f in files[key] + ["hq_internal.cuh"]:
        with open(os.path.join(ROOT, "paper_2111_06868_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_class, n):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json),
    scaled by the state size; None if absent or if the kernel changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entry = json.load(f).get(kernel_class)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("source_sha") != kernel_sources_sha(kernel_class):
        return None
    return entry["dram_bytes_per_amplitude"] * (1 << n)


def block_class(qs, m, engine, tc_min_k, n=30, elem_bytes=8):
    """Which kernel libhq launches for this block (mirrors its dispatch:
    controlled gates first, tensor-core blocks of k = 4, 5 run widened to 6
    qubits when n >= 13)."""
    from paper_2111_06868_gb300 import hq

    d = m.shape[0]
    k = len(qs)
    s, mask, _ = hq.hq_gate_structure(m)
    nc = bin(mask).count("1")
    sector_bits = 2 if elem_bytes == 8 else 1
    if nc and k - nc <= 2 and any((mask >> j) & 1 and n - 1 - q >= sector_bits for j, q in enumerate(qs)):
        return f"k_ctrl_kt{k - nc}"
    df = "_df" if engine in ("df", "tc_c128") and elem_bytes == 16 else ""
    if not np.any(m[~np.eye(d, dtype=bool)]):
        return f"k_diag{df}_k{k}"
    nz = np.abs(m) > 4 * np.finfo(np.float64).eps * np.abs(m).max()
    if k <= 4 and np.all(nz.sum(axis=0) == 1) and np.all(nz.sum(axis=1) == 1):
        return f"k_mono{df}_k{k}"
    if engine == "tc_c128":
        if elem_bytes == 16 and k in (3, 4) and n >= 11:
            return "k_tcz_k4"
    elif engine.startswith("tc") and k >= max(tc_min_k, 4) and n >= k + 7:
        return f"k_tc_{engine[3:]}_k{6 if n >= 13 else k}"
    if engine in ("df", "tc_c128") and elem_bytes == 16 and k <= 4:
        return f"k_gather_df_k{k}"
    return f"k_gather_k{k}" if k <= 4 else f"k_block_k{k}"


def touched_fraction(qs, m, n, elem_bytes):
    """Fraction of the state's bytes one gate reads and writes: 2^-c for the
    controlled-gate kernel with c controls at or above the 32-byte sector,
    else 1."""
    from paper_2111_06868_gb300 import hq

    if not block_class(qs, m, "auto", 4, n, elem_bytes).startswith("k_ctrl"):
        return 1.0
    _, mask, _ = hq.hq_gate_structure(m)
    sector_bits = 2 if elem_bytes == 8 else 1
    return 2.0 ** -sum(1 for j, q in enumerate(qs) if (mask >> j) & 1 and n - 1 - q >= sector_bits)


def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo), or the platform string."""
    import platform

    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts: /proc/cpuinfo has no model name, lscpu does
        import subprocess

        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(circ, seconds: float = 12.0, single_seconds: float = 6.0):
    """The oracle as it stands over the first gates of the same circuit: on all
    host cores until ~`seconds` of CPU work (the reported rate), then on one
    thread for ~`single_seconds`; rates in unfused gate-apps/s."""
    import oracle

    cores = oracle.max_threads()
    n = circ.n

    def run(limit):
        psi = np.zeros(1 << n, np.complex128)
        psi[0] = 1.0
        done = 0
        t0 = time.perf_counter()
        for g in circ.gates:
            oracle.apply_gate(psi, n, g.qubits, g.matrix)
            done += 1
            if time.perf_counter() - t0 > limit:
                break
        return done, time.perf_counter() - t0

    done, dt = run(seconds)
    oracle.set_threads(1)
    try:
        done1, dt1 = run(single_seconds)
    finally:
        oracle.set_threads(cores)
    return {"value": done / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of {len(circ.gates)} gates of the same n={n} circuit, complex128, "
                      f"unfused, OpenMP over {cores} threads ({dt:.1f} s)",
            "single_thread": {"value": done1 / dt1, "sample": f"first {done1} gates on 1 thread ({dt1:.1f} s)"},
            # one gate touches 2^n amplitudes: the rate three qubits up is an eighth (not run: 128 GiB)
            "n33_extrapolated": {"value": done / dt / 8, "note": f"extrapolated from n={n} as rate / 2^(33-{n})"}
            if n == 30 else None,
            "cpu": cpu_model(), "nproc": os.cpu_count()}


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload, each step a
    bounded sample (the first gates of the circuit)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    circ, desc = workload(args, 0)
    n = circ.n
    cores = oracle.max_threads()
    psi = np.zeros(1 << n, np.complex128)
    psi[0] = 1.0
    per_step = args.ref_gates
    gates = circ.gates[:per_step]
    for _ in range(args.warmup):
        for g in gates:
            oracle.apply_gate(psi, n, g.qubits, g.matrix)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for g in gates:
            oracle.apply_gate(psi, n, g.qubits, g.matrix)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = f"first {per_step} gates of the n={n} circuit per step, complex128, unfused, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "gate-apps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n": n, "state": "complex128 (oracle)"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _events():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_blocks(n, blocks, engine, dtype, reps=1, tc_min_k=4):
    """Seconds per pass of `blocks` over a fresh |0..0> state (CUDA events)."""
    import torch
    from paper_2111_06868_gb300 import hq

    st = torch.empty(1 << n, dtype=dtype, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks[:2], engine=engine, tc_min_k=tc_min_k)  # warm the code paths
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        hq.hq_state_init(st)
        hq.hq_apply_blocks(st, blocks, engine=engine, tc_min_k=tc_min_k)
    e1.record()
    torch.cuda.synchronize()
    return st, e0.elapsed_time(e1) / 1e3 / reps


def measure_small_circuit(args, reps: int = 20):
    """One small circuit (n=12, 163 gates; latency-bound): per-block launches
    of the fused circuit against one persistent launch of the batch runner."""
    import torch
    from paper_2111_06868_gb300 import hq

    c12 = C.config_small(seed=0)
    st12 = torch.empty(1 << c12.n, dtype=torch.complex64, device="cuda")
    b12 = fuse(hq, c12.n, c12.gates, 4, args)
    hq.hq_state_init(st12)
    hq.hq_apply_blocks(st12, b12)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        hq.hq_state_init(st12)
        hq.hq_apply_blocks(st12, b12)
    e1.record()
    torch.cuda.synchronize()
    t_blocks = e0.elapsed_time(e1) / 1e3 / reps
    b = hq.Batch([c12], None, 12, 6, 0, 0)
    b.run()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    b.close()
    return {"gates": len(c12.gates), "fused_blocks_k4": len(b12), "apply_blocks_us": 1e6 * t_blocks,
            "batch_runner_us": 1e6 * t_batch, "gate_apps_per_s_batch_runner": len(c12.gates) / t_batch}


def measure_adjoint(dtypes=("complex64", "complex128")):
    """Adjoint gradients: n=20 ansatz, 320 angles, batch 64 (wall clock of
    one synchronous hq_adjoint_grad call after a warm-up call)."""
    import torch
    from paper_2111_06868_gb300 import hq

    ans = C.ansatz(20, 8)
    H = C.ansatz_hamiltonian(20)
    th = C.ansatz_params(ans.n_params, 64, seed=0)
    adj = {}
    for dt in dtypes:
        hq.hq_adjoint_grad(ans, H, th[:2], dtype=dt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hq.hq_adjoint_grad(ans, H, th, dtype=dt)
        t = time.perf_counter() - t0
        adj[dt] = {"grad_per_s": 64 * ans.n_params / t, "s": t}
    return adj


def measure_trajectories(args, T=8):
    """Noisy n=24 grid circuit by pure-state sampling of its Kraus channels
    (Sec. 5): depolarizing after every gate, amplitude damping (whose branch
    probabilities depend on the state) after every one-qubit gate."""
    import torch
    from paper_2111_06868_gb300 import hq

    c24 = C.random_circuit(C.layout_for(24), 12, seed=args.seed, two_qubit="cz")
    ops = C.noisy_ops(c24, p1=1e-3, p2=1e-2, gamma=1e-3)
    nch = sum(1 for o in ops if o[0] == "kraus")
    rng = np.random.default_rng(args.seed)  # the uniforms the sampling draws
    st = torch.empty(1 << 24, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_run_trajectory(st, ops, rng.random(nch))
    torch.cuda.synchronize()
    z = []
    t0 = time.perf_counter()
    for _ in range(T):
        hq.hq_state_init(st)
        hq.hq_run_trajectory(st, ops, rng.random(nch))
        z.append(hq.hq_expectation(st, [(1.0, ((0, "Z"),))]))
    dt_traj = (time.perf_counter() - t0) / T
    del st
    torch.cuda.empty_cache()
    return {"gates": len(c24.gates), "channels": nch,
            "state_dependent_channels": sum(1 for g in c24.gates if g.k == 1),
            "trajectories_per_s": 1 / dt_traj, "ms_per_trajectory": 1e3 * dt_traj,
            "z0_mean": float(np.mean(z)), "timing": "wall clock, host waits included"}


def measure_batch():
    """Batched serving load: 512 circuits, n ~ U{10..24}, one persistent
    launch replayed from a CUDA graph.  The autotuner picks the in-pass fusion
    width and the tile shape: for makespan with the largest-first queue
    (throughput), for median latency with the smallest-first queue; the
    hand-picked (13, 7) tile with 2-qubit fusion is timed beside them."""
    import torch
    from paper_2111_06868_gb300 import autotune
    from paper_2111_06868_gb300 import hq

    cs = C.config_batch(512, seed=0)
    Gb = sum(len(c.gates) for c in cs)
    states = [torch.empty(1 << c.n, dtype=torch.complex64, device="cuda") for c in cs]
    t0 = time.perf_counter()
    pick_span, tim_span = autotune.tune(cs, states, objective="makespan", small_first=0, cache_path=None)
    pick_p50, tim_p50 = autotune.tune(cs, states, objective="p50", small_first=1, cache_path=None)
    tune_s = time.perf_counter() - t0

    def run(cfg):
        b = hq.Batch(cs, states, *cfg)
        b.run()
        e0, e1 = _events()
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        lat, span = b.latencies()
        b.close()
        return {"config": list(cfg), "gate_apps_per_s": Gb / t, "s": t,
                "p50_ms": float(np.percentile(lat, 50)) / 1e3, "p99_ms": float(np.percentile(lat, 99)) / 1e3}

    res = {"circuits": len(cs), "gates": Gb, "launches_per_run": 1, "graph": True,
           "config_fields": ["tile_bits", "max_high", "ctas_per_sm", "small_first", "fuse_k"],
           "largest_first": run(pick_span), "smallest_first": run(pick_p50),
           "hand_picked_largest_first": run((13, 7, 0, 0, 2)), "hand_picked_smallest_first": run((13, 7, 0, 1, 2)),
           "tuned": {"makespan": {"choice": list(pick_span), "candidates_s": tim_span},
                     "p50": {"choice": list(pick_p50), "candidates_s": tim_p50}, "tuning_s": tune_s}}
    del states
    torch.cuda.empty_cache()
    return res


def measure_expectation(reps=5, n=30):
    """<psi|H|psi> at n=30 (complex64) for the ansatz Hamiltonian (29 ZZ and
    30 X terms: several X-mask groups, the tiled path), wall clock of the
    synchronous call."""
    import torch
    from paper_2111_06868_gb300 import hq

    H = C.ansatz_hamiltonian(n)
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st, "+")
    e = hq.hq_expectation(st, H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        e = hq.hq_expectation(st, H)
    t = (time.perf_counter() - t0) / reps
    del st
    torch.cuda.empty_cache()
    return {"n": n, "terms": len(H), "s": t, "value": e, "expected_value": 0.5 * n,
            "state": f"|+>^{n}: every ZZ term 0, every 0.5 X term 0.5"}


def measure_fp_peaks(N=8192, reps=5):
    """Non-tensor-core arithmetic peaks of this GPU, for the rooflines of the
    complex128 kernels (FP64) and the CUDA-core blocks (FP32): cuBLAS DGEMM
    and SGEMM (TF32 off) on N^3, 2 N^3 flop per product, best of `reps`
    (CUDA events)."""
    import torch

    res = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt in (("fp64_dgemm_tflops", torch.float64), ("fp32_sgemm_tflops", torch.float32)):
            a = torch.randn(N, N, dtype=dt, device="cuda")
            b = torch.randn(N, N, dtype=dt, device="cuda")
            c = a @ b
            best = 1e30
            for _ in range(reps):
                e0, e1 = _events()
                e0.record()
                c = a @ b
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            res[name] = 2 * N ** 3 / best / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    torch.cuda.empty_cache()
    res["how"] = f"torch.matmul {N}^3, 2 N^3 flop, best of {reps}, CUDA events; allow_tf32 False"
    return res


def measure_c128(args, circ):
    """Configuration 2 in complex128: per gate and fused k <= 4 on the FP64
    kernels, in double-float, and fused k <= 3, 4 on the tensor cores (exact
    digit-slice products); rates in unfused gate-apps/s, effective GB/s =
    bytes of one read and write of the state per launch."""
    import torch

    G = len(circ.gates)
    res = {"gates": G}
    st, t = _time_blocks(30, [(g.qubits, g.matrix) for g in circ.gates], "auto", torch.complex128)
    res["per_gate"] = {"launches": G, "gate_apps_per_s": G / t, "s": t, "GBps": G * 2 * (1 << 30) * 16 / t / 1e9}
    del st
    from paper_2111_06868_gb300 import hq

    b4 = fuse(hq, 30, circ.gates, 4, args)
    st, t4 = _time_blocks(30, b4, "cuda_core", torch.complex128)
    res["fused_k4"] = {"blocks": len(b4), "gate_apps_per_s": G / t4, "s": t4,
                       "GBps": len(b4) * 2 * (1 << 30) * 16 / t4 / 1e9}
    del st
    # the same in double-float arithmetic on the FP32 pipes (HQ_ENGINE_DF)
    st, t = _time_blocks(30, [(g.qubits, g.matrix) for g in circ.gates], "df", torch.complex128)
    res["per_gate_df"] = {"launches": G, "gate_apps_per_s": G / t, "s": t, "GBps": G * 2 * (1 << 30) * 16 / t / 1e9}
    del st
    for kk in (2, 3, 4):
        bk = fuse(hq, 30, circ.gates, kk, args)
        st, tk = _time_blocks(30, bk, "df", torch.complex128)
        res[f"fused_k{kk}_df"] = {"blocks": len(bk), "gate_apps_per_s": G / tk, "s": tk,
                                  "GBps": len(bk) * 2 * (1 << 30) * 16 / tk / 1e9}
        del st
    # dense 3- and 4-qubit blocks on the tensor cores as exact FP16 digit-slice
    # products (HQ_ENGINE_TC_C128), the others in double-float
    peaks, _ = load_peaks()
    for kk in (3, 4):
        bk = fuse(hq, 30, circ.gates, kk, args)
        st, tk = _time_blocks(30, bk, "tc_c128", torch.complex128)
        gbs = len(bk) * 2 * (1 << 30) * 16 / tk / 1e9
        res[f"fused_k{kk}_tc_c128"] = {"blocks": len(bk), "gate_apps_per_s": G / tk, "s": tk, "GBps": gbs,
                                       "hbm_frac": gbs / peaks["hbm_gbs"]}
        del st
    torch.cuda.empty_cache()
    return res


def measure_n28_vs_oracle(args):
    """Relative L2 error against the oracle (complex128, gate by gate) of the
    n=28 subset of the 33-qubit layout (942 gates), for every complex64 engine
    on the fused k <= 6 blocks, and max-abs error of the complex128 paths
    (per gate; fused k <= 4 in double-float and on the tensor cores); the
    oracle state is computed on the host cores (~80 s)."""
    import torch
    import oracle
    from paper_2111_06868_gb300 import hq

    c28 = C.config_n33(seed=args.seed, first=28)
    t0 = time.perf_counter()
    want = oracle.simulate(c28)
    t_or = time.perf_counter() - t0
    nw = np.linalg.norm(want)
    st = torch.empty(1 << 28, dtype=torch.complex64, device="cuda")
    errs = {}
    b28 = fuse(hq, 28, c28.gates, 6, args)
    for eng in ("tc_f16", "tc_bf16", "cuda_core"):
        hq.hq_state_init(st)
        hq.hq_apply_blocks(st, b28, engine=eng, tc_min_k=4)
        errs[eng] = float(np.linalg.norm(st.cpu().numpy().astype(np.complex128) - want) / nw)
    del st
    st = torch.empty(1 << 28, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, c28.gates)
    c128 = float(np.abs(st.cpu().numpy() - want).max())
    b4 = fuse(hq, 28, c28.gates, 4, args)
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, b4, engine="df")
    c128_df = float(np.abs(st.cpu().numpy() - want).max())
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, b4, engine="tc_c128")
    c128_tc = float(np.abs(st.cpu().numpy() - want).max())
    del st
    torch.cuda.empty_cache()
    return {"gates": len(c28.gates), "blocks_k6": len(b28), "rel_l2": errs, "bar_rel_l2": 2e-5,
            "c128_per_gate_max_abs": c128, "c128_df_fused_k4_max_abs": c128_df,
            "c128_tc_c128_fused_k4_max_abs": c128_tc, "bar_max_abs": 1e-12,
            "oracle_s": t_or, "oracle_threads": oracle.max_threads()}


def measure_extras(args):
    """One measurement of every other workload (CUDA events)."""
    import torch
    from paper_2111_06868_gb300 import hq

    out = {}
    # n=30, unfused: every gate its own launch
    circ = C.config_n30(seed=args.seed)
    G = len(circ.gates)
    st, t = _time_blocks(30, [(g.qubits, g.matrix) for g in circ.gates], "auto", torch.complex64)
    out["n30_per_gate_c64"] = {"gate_apps_per_s": G / t, "s": t, "launches": G}
    del st
    # the same circuit fused into blocks of <= 4 qubits on the exact FP32
    # CUDA-core kernels (gather / monomial / diagonal; no tensor cores)
    b4 = fuse(hq, 30, circ.gates, 4, args)
    st, t4 = _time_blocks(30, b4, "cuda_core", torch.complex64)
    out["n30_fused_k4_c64_cuda_core"] = {"blocks": len(b4), "gate_apps_per_s": G / t4, "s": t4,
                                         "speedup_vs_per_gate": t / t4}
    del st
    # n=30, complex128 (FP64): the whole circuit per gate, and fused into
    # <= 4-qubit blocks on the exact kernels
    out["n30_c128"] = measure_c128(args, circ)
    torch.cuda.empty_cache()
    # n=30 QFT, unfused: 435 controlled phases (the controlled-gate kernel reads
    # and writes only the amplitudes whose controls are 1), 30 H, 15 SWAP
    qft = [(g.qubits, g.matrix) for g in C.qft_circuit(30).gates]
    for name, dt, S in (("c64", torch.complex64, 8), ("c128", torch.complex128, 16)):
        st, t = _time_blocks(30, qft, "auto", dt)
        touched = sum(touched_fraction(q, m, 30, S) for q, m in qft) * 2 * (1 << 30) * S
        out[f"n30_qft_per_gate_{name}"] = {"gates": len(qft), "gate_apps_per_s": len(qft) / t, "s": t,
                                           "touched_GBps": touched / t / 1e9,
                                           "full_pass_equivalents": touched / (2 * (1 << 30) * S)}
        del st
        torch.cuda.empty_cache()
    # n=30 <Z_0> after the circuit: Sec. 3.1 pop (light cone of qubit 0) and
    # simplify ahead of fusion, against fusing the whole circuit
    t_h = time.perf_counter()
    kept = hq.hq_simplify(30, hq.hq_pop(30, circ.gates, [0]))
    b_pop = fuse(hq, 30, kept, 6, args)
    t_h = time.perf_counter() - t_h
    b_full = fuse(hq, 30, circ.gates, 6, args)
    z0 = [(1.0, ((0, "Z"),))]
    st, t_full = _time_blocks(30, b_full, "tc_f16", torch.complex64)
    e_full = hq.hq_expectation(st, z0)
    del st
    st, t_pop = _time_blocks(30, b_pop, "tc_f16", torch.complex64)
    e_pop = hq.hq_expectation(st, z0)
    del st
    torch.cuda.empty_cache()
    out["n30_z0_light_cone"] = {"gates_full": G, "gates_kept": len(kept), "blocks_full": len(b_full),
                                "blocks_kept": len(b_pop), "s_full": t_full, "s_kept": t_pop,
                                "speedup": t_full / t_pop, "host_s": t_h, "z0_full": e_full, "z0_kept": e_pop}
    out["n24_noisy_trajectories"] = measure_trajectories(args)
    # n=15 noisy circuit at the density-matrix level (Sec. 5): rho as a
    # 30-qubit vector (8 GiB), every gate and channel as its superoperator
    # (Sec. 2 MatrixSuperGate), fused into <= 6 vector-qubit blocks on the
    # tensor cores; the same circuit and channels as the trajectories above
    c15 = C.random_circuit(C.layout_for(15), 10, seed=args.seed, two_qubit="cz")
    ops15 = C.noisy_ops(c15, p1=1e-3, p2=1e-2, gamma=1e-3)
    t_h = time.perf_counter()
    sup = [(tuple(qs) + tuple(15 + q for q in qs), hq.hq_dm_superop([m] if kind == "gate" else m))
           for kind, qs, m in ops15]
    bdm = hq.hq_fuse(30, sup, 6, method="dag", restarts=8, seed=0)  # as hq_dm_apply fuses
    t_h = time.perf_counter() - t_h
    st, t_dm = _time_blocks(30, bdm, "tc_f16", torch.complex64)
    rho = st.view(1 << 15, 1 << 15)
    tr = hq.hq_dm_expectation(rho, [(1.0, ())])
    z0 = hq.hq_dm_expectation(rho, [(1.0, ((0, "Z"),))])
    pur = hq.hq_dm_purity(rho)
    reps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        hq.hq_dm_init(rho)
        hq.hq_dm_apply(rho, ops15, k_max=6, engine="tc_f16")
    torch.cuda.synchronize()
    t_api = (time.perf_counter() - t0) / reps
    out["n15_density_matrix"] = {
        "ops": len(ops15), "gates": len(c15.gates), "channels": sum(1 for o in ops15 if o[0] == "kraus"),
        "vector_qubits": 30, "blocks": len(bdm), "device_s": t_dm, "noisy_ops_per_s": len(ops15) / t_dm,
        "GBps_per_block": 2 * 8 * 2 ** 30 * len(bdm) / t_dm / 1e9, "api_s": t_api,
        "api_note": "hq_dm_apply wall clock: host superoperators and fusion included",
        "host_superop_and_fuse_s": t_h, "trace": tr, "z0": z0, "purity": pur}
    del st, rho
    torch.cuda.empty_cache()
    # n=33: fused k <= 6 on tensor cores vs CUDA cores (64 GiB state)
    c33 = C.config_n33(seed=args.seed)
    b33 = fuse(hq, 33, c33.gates, 6, args)
    st, t_tc = _time_blocks(33, b33, "tc_f16", torch.complex64)
    nrm = hq.hq_expectation(st, [(1.0, ())])
    _, t_cc = _time_blocks(33, b33, "cuda_core", torch.complex64)
    out["n33_fused_k6"] = {"blocks": len(b33), "gates": len(c33.gates),
                           "tc_f16_gate_apps_per_s": len(c33.gates) / t_tc, "tc_f16_s": t_tc,
                           "tc_f16_GBps_per_block": len(b33) * 2 * (1 << 33) * 8 / t_tc / 1e9,
                           "cuda_core_s": t_cc, "cuda_core_gate_apps_per_s": len(c33.gates) / t_cc,
                           "tc_speedup_vs_cuda_core": t_cc / t_tc, "norm_minus_1": nrm ** 0.5 - 1}
    del st
    torch.cuda.empty_cache()
    # accuracy of every engine against the oracle on the n=28 subset
    if not args.no_oracle_check:
        out["n28_subset_vs_oracle"] = measure_n28_vs_oracle(args)
    out["adjoint_n20_batch64"] = measure_adjoint()
    out["n30_expectation_ansatz_hamiltonian"] = measure_expectation()
    out["batch512"] = measure_batch()
    out["n12_one_circuit"] = measure_small_circuit(args)
    return out


def gpu_numa_info(device_index):
    """NUMA node and local CPUs of the GPU (Linux sysfs via its PCI bus id),
    and this process's CPU affinity."""
    info = {"affinity": sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None}
    try:
        out = subprocess.run(["nvidia-smi", f"--id={device_index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True, timeout=10).stdout.strip()
        bus = out.lower()
        if bus.startswith("0000000"):
            bus = bus[4:]
        base = f"/sys/bus/pci/devices/{bus}"
        with open(f"{base}/numa_node") as f:
            info["gpu_numa_node"] = int(f.read().strip())
        with open(f"{base}/local_cpulist") as f:
            info["gpu_local_cpulist"] = f.read().strip()
        info["pci_bus_id"] = bus
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return info


def _cpulist(text):
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part.strip():
            cpus.add(int(part))
    return cpus


def measure_e2e(args, hq, circ, blocks, state, stream, engine, dist):
    """End to end through the public API, as a user of Sec. 4.2's simulate()
    gets the result: every step is one hq_simulate call (the block matrices
    go up from host memory inside it; |0..0>, the blocks and the FP64 norm)
    and the final state read back into pinned host memory, in stream order
    (with the device time of the two parts).  Also measured: the streamed
    form (two device states, each step's read-back on a second stream under
    the next step); the same with the state uploaded from pinned host memory
    (hq_state_upload: the SMs read the host buffer over the CPU-GPU link),
    hq_apply_blocks and the norm instead; the H2D and D2H copies alone
    (GB/s); the copy-engine variant that overlaps the next step's upload
    with the current step on a second stream; and a variant that runs the
    fusion of the next step's circuit on the host while the current step's
    read-back runs.  The pinned buffers are allocated (and first touched) by
    a thread bound to the GPU's local CPUs where the system reports them."""
    import torch

    n, G = circ.n, len(circ.gates)
    cdt, S = state.dtype, state.element_size()
    numa = gpu_numa_info(torch.cuda.current_device())
    old_aff = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    local = _cpulist(numa.get("gpu_local_cpulist", "")) & (old_aff or set())
    if local:
        os.sched_setaffinity(0, local)
    try:
        host_in = torch.empty(1 << n, dtype=cdt, pin_memory=True)
        host_in.zero_()
        host_in[0] = 1
        host_out = torch.empty(1 << n, dtype=cdt, pin_memory=True)
        host_out.zero_()
    finally:
        if local:
            os.sched_setaffinity(0, old_aff)
    numa["pinned_allocated_on_local_cpus"] = bool(local)
    out = torch.zeros(1, dtype=torch.float64).pin_memory()
    bufs = [state, torch.empty_like(state)]
    copy_stream = torch.cuda.Stream()

    def timed_copy(fn, reps=3):
        best = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            fn()
            c1.record(stream)
            torch.cuda.synchronize()
            best = min(best, c0.elapsed_time(c1) / 1e3)
        return best

    t_ce = timed_copy(lambda: bufs[1].copy_(host_in, non_blocking=True))
    t_sm = timed_copy(lambda: hq.hq_state_upload(bufs[1], host_in, stream=stream))
    t_d2h = timed_copy(lambda: host_out.copy_(bufs[1], non_blocking=True))
    nbytes = (1 << n) * S
    # matrices the library uploads per step: the split B operand of every tensor-core block
    tc_bytes = sum(2 * (2 * 64) ** 2 * 2 for q, m in blocks
                   if block_class(q, m, engine, args.tc_min_k, n, S).startswith("k_tc"))

    def simulate_read(steps, refuse=False):
        cur_blocks = blocks
        for s in range(steps):
            out[0] = hq.hq_simulate(state, cur_blocks, engine=engine, tc_min_k=args.tc_min_k, stream=stream)
            host_out.copy_(state, non_blocking=True)
            if refuse and s + 1 < steps:  # next step's fusion on the host, under this step's copy
                cur_blocks = fuse(hq, n, circ.gates, args.kmax, args)

    def upload(steps):
        for s in range(steps):
            hq.hq_state_upload(state, host_in, stream=stream)
            hq.hq_apply_blocks(state, blocks, engine=engine, tc_min_k=args.tc_min_k, stream=stream)
            out[0] = hq.hq_expectation(state, [(1.0, ())], stream=stream)

    def overlapped(steps, start=None):
        copied = [None, None]
        with torch.cuda.stream(copy_stream):
            if start is not None:
                copy_stream.wait_event(start)
            bufs[0].copy_(host_in, non_blocking=True)
            copied[0] = torch.cuda.Event()
            copied[0].record(copy_stream)
        for s in range(steps):
            cur = bufs[s % 2]
            stream.wait_event(copied[s % 2])
            hq.hq_apply_blocks(cur, blocks, engine=engine, tc_min_k=args.tc_min_k, stream=stream)
            if s + 1 < steps:
                nxt = (s + 1) % 2
                with torch.cuda.stream(copy_stream):
                    bufs[nxt].copy_(host_in, non_blocking=True)
                    copied[nxt] = torch.cuda.Event()
                    copied[nxt].record(copy_stream)
            out[0] = hq.hq_expectation(cur, [(1.0, ())], stream=stream)

    def simulate_pipelined(steps):
        """The same steps with two device states: step s runs on one while
        the result of step s - 1 is read back from the other on a second
        stream, into its own pinned host buffer (host_in is not needed after
        the upload variants)."""
        outs = [host_out, host_in]
        done = [None, None]
        for s in range(steps):
            cur = bufs[s % 2]
            if done[s % 2] is not None:  # that state's previous read-back has finished
                stream.wait_event(done[s % 2])
            out[0] = hq.hq_simulate(cur, blocks, engine=engine, tc_min_k=args.tc_min_k, stream=stream)
            ready = torch.cuda.Event()
            ready.record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ready)
                outs[s % 2].copy_(cur, non_blocking=True)
                done[s % 2] = torch.cuda.Event()
                done[s % 2].record(copy_stream)
        for d in done:
            if d is not None:
                stream.wait_event(d)

    def serial_breakdown(steps):
        """Device time of the hq_simulate call and of the read-back in the
        serial steps (CUDA events around each)."""
        sim, cp = [], []
        for s in range(steps):
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            out[0] = hq.hq_simulate(state, blocks, engine=engine, tc_min_k=args.tc_min_k, stream=stream)
            b.record(stream)
            host_out.copy_(state, non_blocking=True)
            c.record(stream)
            c.synchronize()
            sim.append(a.elapsed_time(b))
            cp.append(b.elapsed_time(c))
        return {"simulate_ms": statistics.mean(sim), "read_back_ms": statistics.mean(cp),
                "read_back_GBps": nbytes / statistics.mean(cp) / 1e6}

    def timed(fn, steps, **kw):
        fn(2, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if fn is overlapped:
            fn(steps, start=e0)
        else:
            fn(steps, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    e2e_steps = max(2, min(args.steps, 5))
    # the headline: one state, one stream (hq_simulate, then the read-back);
    # the streamed form beside it (its copies run beside the HBM-bound
    # blocks, and on some boxes the link then slows down several fold)
    et = timed(simulate_read, e2e_steps)
    e2e_value, et = whole_job_rate(et, G * e2e_steps, dist, "cuda")
    t_p = timed(simulate_pipelined, e2e_steps)
    t_f = timed(simulate_read, e2e_steps, refuse=True)
    t_u = timed(upload, e2e_steps)
    t_o = timed(overlapped, e2e_steps)
    breakdown = serial_breakdown(e2e_steps)
    del bufs
    return {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": tc_bytes, "d2h_bytes_per_step": nbytes + 8,
            "ms_per_step": 1e3 * et / e2e_steps, **breakdown,
            "note": "every step: hq_simulate (|0..0>, the fused blocks with their matrices uploaded from host "
                    "memory inside the call, FP64 norm read back), then the final state copied into pinned "
                    "host memory; in stream order on one stream",
            "streamed": {"value": G * e2e_steps / t_p, "ms_per_step": 1e3 * t_p / e2e_steps,
                         "note": "two device states: each step's final state read back on a second stream, "
                                 "into its own pinned host buffer, while the next step runs"},
            "h2d": {"sm_read_GBps": nbytes / t_sm / 1e9, "sm_read_ms": 1e3 * t_sm,
                    "copy_engine_GBps": nbytes / t_ce / 1e9, "copy_engine_ms": 1e3 * t_ce},
            "d2h": {"copy_engine_GBps": nbytes / t_d2h / 1e9, "copy_engine_ms": 1e3 * t_d2h},
            "numa": numa,
            "with_fusion_each_step": {"value": G * e2e_steps / t_f, "ms_per_step": 1e3 * t_f / e2e_steps,
                                      "fusion": args.fuse,
                                      "note": "the fusion of the next step on the host under the current "
                                              "step's state read-back"},
            "state_upload": {"value": G * e2e_steps / t_u, "ms_per_step": 1e3 * t_u / e2e_steps,
                             "h2d_bytes_per_step": nbytes + tc_bytes, "d2h_bytes_per_step": 8,
                             "note": "every step: hq_state_upload of the pinned host state (SM reads), "
                                     "hq_apply_blocks, FP64 norm read back"},
            "copy_engine_overlapped": {"value": G * e2e_steps / t_o, "ms_per_step": 1e3 * t_o / e2e_steps,
                                       "note": "torch copy_ from pinned memory on a second stream, the next "
                                               "step's copy overlapping the current step (two buffers)"}}


def whole_job_rate(local_seconds: float, local_units: float, dist=None, device=None):
    """Replicas: every rank processed its own units; the job rate is the sum
    of the units over the slowest rank's time (max over ranks)."""
    if dist is None:
        return local_units / local_seconds, local_seconds
    import torch

    t = torch.tensor([local_seconds, local_units], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    units = t[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return float(units.item()) / float(tmax.item()), float(tmax.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hq", choices=["hq", "reference"])
    ap.add_argument("--workload", default="n30", choices=["n30", "n33", "n27", "n12"])
    ap.add_argument("--kmax", type=int, default=6)
    ap.add_argument("--fuse", default="beam", choices=["beam", "dag", "greedy"],
                    help="hq_fuse_beam (beam search over DAG-frontier blocks), hq_fuse_dag (DAG frontier, "
                         "restarts) or hq_fuse (greedy rule)")
    ap.add_argument("--fuse-restarts", type=int, default=64)
    ap.add_argument("--fuse-width", type=int, default=128, help="kept sequences of hq_fuse_beam")
    ap.add_argument("--dtype", default="complex64", choices=["complex64", "complex128"])
    ap.add_argument("--engine", default="tc_f16", choices=["auto", "cuda_core", "tc_f16", "tc_bf16", "tc_pass", "df", "tc_c128"])
    ap.add_argument("--tc-min-k", type=int, default=4)
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' sub-measurements")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ref-gates", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true", help="skip the n=28 oracle comparison in extras")
    ap.add_argument("--expect-n", type=int, default=30, help="state size of --only expect")
    ap.add_argument("--only", choices=["adjoint", "trajectories", "batch", "expect", "peaks"],
                    help="run one of the extra workloads alone (for profiling) and print its result")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2111_06868_gb300 import build as hqbuild
    from paper_2111_06868_gb300 import hq

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        hqbuild.build()
    if dist:
        dist.barrier()
    hq.load()
    if args.only:
        if args.only == "adjoint":
            res = measure_adjoint(("complex64",))
        elif args.only == "batch":
            res = measure_batch()
        elif args.only == "expect":
            res = measure_expectation(n=args.expect_n)
        elif args.only == "peaks":
            res = measure_fp_peaks()
        else:
            res = measure_trajectories(args, T=2)
        print(json.dumps({"only": args.only, **res}))
        return

    circ, desc = workload(args, rank)
    n, G = circ.n, len(circ.gates)
    t_f = time.perf_counter()
    blocks = fuse(hq, n, circ.gates, args.kmax, args) if args.kmax > 0 else [(g.qubits, g.matrix) for g in circ.gates]
    fuse_s = time.perf_counter() - t_f
    B = len(blocks)
    cdt = torch.complex64 if args.dtype == "complex64" else torch.complex128
    S = 8 if cdt == torch.complex64 else 16
    classes = [block_class(q, m, args.engine, args.tc_min_k, n, S) for q, m in blocks]
    state = torch.empty(1 << n, dtype=cdt, device="cuda")
    stream = torch.cuda.current_stream()
    norm_term = [(1.0, ())]
    engine = args.engine

    passes = len(hq.hq_plan_passes(n, blocks)) if engine == "tc_pass" else 0

    def step():
        """One pass of the hot path through the public API: one hq_simulate
        call (Sec. 4.2 simulate: |0..0>, every fused block, the FP64 norm;
        synchronous)."""
        return hq.hq_simulate(state, blocks, engine=engine, tc_min_k=args.tc_min_k)

    def step_per_block(events):
        """The same step with one call per block, bracketed by CUDA events on
        the launching stream (per-kernel durations for the roofline)."""
        hq.hq_state_init(state)
        if engine == "tc_pass":  # the pass engine plans over the whole list: one bracket
            events[0].record(stream)
            hq.hq_apply_blocks(state, blocks, engine=engine)
            events[B].record(stream)
            return hq.hq_expectation(state, norm_term)
        for i, b in enumerate(blocks):
            events[i].record(stream)
            hq.hq_apply_blocks(state, [b], engine=engine, tc_min_k=args.tc_min_k)
        events[B].record(stream)
        return hq.hq_expectation(state, norm_term)

    for _ in range(args.warmup):
        norm = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0.record(stream)
    for s in range(args.steps):
        norm = step()
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1) / 1e3
    value, elapsed = whole_job_rate(elapsed, G * args.steps, dist, "cuda")

    # second timed pass: per-block launches bracketed by events (roofline)
    per_step_events = [[torch.cuda.Event(enable_timing=True) for _ in range(B + 1)] for _ in range(args.steps)]
    step_per_block(per_step_events[0])
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for s in range(args.steps):
        step_per_block(per_step_events[s])
    p1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per_block_step_s = p0.elapsed_time(p1) / 1e3 / args.steps

    durs = {}
    for ev in per_step_events:
        if engine == "tc_pass":  # one bracket per step; averaged over its passes
            durs.setdefault("k_pass (all passes)", []).extend([ev[0].elapsed_time(ev[B]) / 1e3 / passes] * passes)
            continue
        for i in range(B):
            durs.setdefault(classes[i], []).append(ev[i].elapsed_time(ev[i + 1]) / 1e3)
    tot = {c: sum(v) for c, v in durs.items()}
    dom = max(tot, key=tot.get)
    avg = statistics.mean(durs[dom])
    bytes_per_launch = 2 * (1 << n) * S
    peaks, peak_kind = load_peaks()
    achieved = bytes_per_launch / avg / 1e9
    per_class = {c: {"launches_per_step": len(v) // args.steps, "avg_ms": 1e3 * statistics.mean(v),
                     "GBps": bytes_per_launch / statistics.mean(v) / 1e9, "share": tot[c] / sum(tot.values())}
                 for c, v in durs.items()}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, hq, circ, blocks, state, stream, engine, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(circ)

    extras = None
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "n30":
        del state
        torch.cuda.empty_cache()
        extras = measure_extras(args)

    if rank == 0:
        # bytes a step moves: the first tensor-core block only writes (its input
        # is computed from the tokens), the last sums the norm as it writes
        first_tc = classes[0].startswith("k_tc")
        # hq_simulate runs a structured last block of 4..6 qubits on k_tc too, to fold the norm in
        last_tc = classes[-1].startswith("k_tc") or (engine in ("tc_f16", "tc_bf16") and n >= 13 and
                                                     4 <= len(blocks[-1][0]) <= 6)
        passes_rw = 2 * B - (1 if first_tc else -1) + (0 if last_tc else 1)
        eff_gbs = passes_rw * (bytes_per_launch // 2) * args.steps / (elapsed / world) / 1e9
        rec = {
            "metric": METRIC, "value": value, "unit": "gate-apps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if S == 8 else "f64", "data": "synthetic",
            "config": {"workload": desc, "n": n, "gates": G, "fused_blocks": B, "k_max": args.kmax,
                       "arith": ARITH.get(engine, engine) if (S == 8 or engine in ("df", "tc_c128")) else "fp64",
                       "note": "the n=30 circuit of the per-gate / fused k<=4 configuration, run on the "
                               "fused k<=6 tensor-core engine of the 33-qubit configuration"
                               if n == 30 and engine.startswith("tc") else None,
                       "timing": "value: one hq_simulate call per step (init folded into the first "
                                 "block, norm into the last); roofline: a second pass with hq_state_init, "
                                 "one hq_apply_blocks call per block between CUDA events, and the norm",
                       "fusion": (f"dag ({args.fuse_restarts} restarts)" if args.fuse == "dag" else
                                  f"beam (width {args.fuse_width})" if args.fuse == "beam" else args.fuse),
                       "state": args.dtype, "engine": engine, "l2": (f"state ({S * (1 << n) / 2**30:g} GiB) larger than the 129 MB L2; no flush" if S << n > 129e6
                              else f"state ({S << n} B) fits in L2 and is not flushed"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       **({"passes": passes} if engine == "tc_pass" else {})},
            "effective_GBps": eff_gbs, "roofline_frac_effective": eff_gbs / peaks["hbm_gbs"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": measured_traffic(dom, n),
                         "kernel": dom, "peak_source": peak_kind,
                         "bytes_per_launch": bytes_per_launch},
            "per_class": per_class,
            "norm2": norm, "fuse_s": fuse_s, "per_block_pass_ms_per_step": 1e3 * per_block_step_s,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "extras": extras,
            # per step: the blocks, k_init unless folded, the norm (k_expect + k_expect_final) unless folded
            "gpu_launches": args.steps * (B + (0 if first_tc else 1) + (0 if last_tc else 2)),
        }
        print(json.dumps(rec))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
