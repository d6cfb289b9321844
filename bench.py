#!/usr/bin/env python
"""Benchmark of the contraction hot path on synthetic circuits (one JSON line on rank 0).

Workloads (seeded; see paper_2108_06831_gb300/circuits.py):
  state24   (default) 24-qubit 1D brickwork, depth 20 (U3 on every qubit + alternating CZ),
            full 2^24 complex64 state per step; metric amplitudes/s
  state10   10-qubit brickwork, depth 8, a batch of 512 circuits' worth of parameter sets
  grad20    20-qubit hardware-efficient ansatz (400 parameters), TFIM energy forward plus
            adjoint gradient over a batch of 64 parameter sets; metric grads/s

Timing: W warm-up steps, then exactly K steps, each bracketed by CUDA events on the
launching stream, with a write of a buffer larger than L2 between steps (untimed); the
value is the units of all ranks over the maximum per-rank time.  Multi-GPU runs are
independent replicas (the path has no exchange step).

--impl reference times the FP64 oracle (the CPU program the parity tests use) on bounded
samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitudes/s, grads/s & % roofline; split-prec+batched vs plain FP32 at ≤1e-5 err"
# FP32 multiply-add roofline of the kernels bound by FP32 arithmetic: measured on the GPU at start-up
# (set_fp32_peak); the nominal rate from the device's SM count and maximum clock is reported beside it
FP32_ALU_PEAK_TFLOPS = None
FP32_ALU_PEAK_SRC = None
# circuits of this many qubits and more run their own generated pass kernels inside a batch (the
# library's rule for plans with generated kernels; the tuned batch builds such plans for them)
SERVE_WIDE = 19


def set_fp32_peak(tn, torch, dev):
    """The FP32 multiply-add rate measured on this GPU by the library's probe (packed FP32x2 FMA
    chains on every SM at full occupancy, CUDA events), and the nominal rate (SM count from the
    device, 128 FP32 lanes per SM, maximum SM clock from nvidia-smi) for context."""
    global FP32_ALU_PEAK_TFLOPS, FP32_ALU_PEAK_SRC
    rate, secs = tn.probe_fma_rate()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        mhz = float(subprocess.run(["nvidia-smi", "-i", str(dev.index or 0), "--query-gpu=clocks.max.sm",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                   timeout=20).stdout.strip().splitlines()[0])
    except Exception:
        mhz = float("nan")
    nominal = sms * 128 * 2 * mhz * 1e6 / 1e12
    FP32_ALU_PEAK_TFLOPS = rate
    FP32_ALU_PEAK_SRC = (f"measured FP32 FMA rate {rate:.1f} TFLOP/s (tn_probe_fma_rate: packed FP32x2 FMA chains on "
                         f"every SM, {secs * 1e3:.0f} ms launch); nominal {sms} SMs x 128 lanes x 2 flops x "
                         f"{mhz:.0f} MHz = {nominal:.1f} TFLOP/s")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="state24",
                    choices=["state24", "state10", "grad20", "gemm_fp32", "gemm_3xtf32", "gemm_bf16x3",
                             "serving512", "serving512p", "amps36", "permute28", "gemm_merge", "fig31", "fig31amps", "plan31", "q428_24"])
    ap.add_argument("--batch", type=int, default=0, help="gemm workloads: batch override (small profiling cases)")
    ap.add_argument("--legs", type=int, default=0, help="permute28: tensor legs override (small profiling cases)")
    ap.add_argument("--prec", type=int, default=1, help="amps36: GEMM precision (0 FP32, 1 3xTF32, 2 split BF16)")
    ap.add_argument("--max-log2", type=int, default=0,
                    help="amps36: cap on the largest intermediate (log2 entries; 0 = 28); below the "
                         "best order's peak the planner slices indices")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--order-trials", type=int, default=0,
                    help="amps36: orders the contraction-path search tries (0: the planner's default)")
    ap.add_argument("--order-search", type=int, default=0,
                    help="network workloads: 1 = adaptive (cross-entropy) contraction-order search")
    ap.add_argument("--lanes", type=int, default=8,
                    help="fig31amps: streams the captured graph spreads the 98 calls over")
    ap.add_argument("--no-configs", action="store_true",
                    help="state24: skip the short runs of the other configurations after the headline")
    ap.add_argument("--no-specialize", action="store_true", help="run the interpreting gate-apply kernel")
    ap.add_argument("--blocks", type=int, default=0,
                    help="state workloads: contract by uniform 2^k x 2^k blocks of k = 6 or 7 qubits, each "
                         "applied by the batched complex GEMM in --prec (0 FP32, 1 3xTF32, 2 split BF16)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="state workloads: apply the gates one by one (no precontracted two-qubit blocks)")
    return ap.parse_args()


def recorded_traffic(kernel_hash, profile="fused_gate_apply_state24.md"):
    """DRAM bytes per launch of the profiled kernel from the committed ncu summary, or None
    unless the kernel sources hash to the value recorded with that capture."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", profile)) as fh:
            m = re.search(r"traffic_bytes_per_launch=(\d+) kernel_hash=([0-9a-f]+)", fh.read())
        if m and m.group(2) == kernel_hash:
            return float(m.group(1))
    except OSError:
        pass
    return None


def file_hash(path):
    """sha256 (16 hex digits) of one source file."""
    import hashlib
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def jit_source_hash(dump_dir):
    """sha256 (16 hex digits) of the generated kernel sources written to dump_dir."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(dump_dir)):
        with open(os.path.join(dump_dir, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def max_over_ranks(total_ms, world, device):
    """The slowest rank's timed total (ms): replicas finish when the last one does."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step, steps, world, t_max_ms):
    """Units processed by all ranks per second of the slowest rank's time (weak scaling)."""
    return units_per_step * steps * world / (t_max_ms / 1000.0)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_bf16_peak():
    """Dense BF16 tensor rate (TFLOP/s, burst) and where it came from: the measured figure, else the
    fallback of an earlier GB300 measurement (1.9 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops"
    except Exception:
        return 1900.0, "fallback bf16 1900 TFLOP/s (no MEASURED_PEAKS.json)"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU) timing

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2108_06831_gb300 import circuits as C
from oracle.statevector import basis_state, apply_matrix, gate_matrix, simulate_state
from oracle import observables as OB
from oracle.tn import contract_amplitude, contract_amplitude_sweep
kind, budget = {kind!r}, {budget}
t0 = time.perf_counter()
if kind == "state":
    # whole circuits of the same family (brickwork, depth {depth}, seed {seed}), growing the width
    # while the next one (about twice the work) still fits the budget; nothing is extrapolated
    m = min(12, {n})
    while True:
        c, p = C.brickwork(m, {depth}, {seed}, parameterized=True)
        t1 = time.perf_counter()
        psi = basis_state(c.n_qubits, 0)
        for g in c.gates:
            psi = apply_matrix(psi, c.n_qubits, gate_matrix(c, g, p), g.qubits)
        dt = time.perf_counter() - t1
        if m >= {n} or time.perf_counter() - t0 + 2.2 * dt > budget:
            break
        m += 1
    out = dict(value=(1 << m) / dt, unit="amplitudes/s", seconds=dt,
               sample=f"FP64 state-vector oracle, the whole {{m}}-qubit brickwork of depth {depth} "
                      f"({{len(c.gates)}} gates, {{dt:.1f}} s; the widest that fits the time budget, "
                      f"not scaled)")
elif kind == "grad":
    c = C.hea({n}, 10)
    e = OB.expectation(c, C.tfim({n}), C.hea_params(c.n_params, 1, 4000)[0])
    dt = time.perf_counter() - t0
    out = dict(value=1.0 / (2 * dt), unit="grads/s", seconds=dt,
               sample=f"FP64 oracle expectation of one parameter set ({{dt:.1f}} s); a parameter-shift "
                      f"gradient entry costs two")
elif kind == "amps":
    c = C.grid(6, 6, {depth}, {seed})
    xs = C.random_bitstrings(36, 4096, {seed} + 1)
    done = 0
    while done < len(xs) and (done == 0 or time.perf_counter() - t0 < budget):
        contract_amplitude_sweep(c, int(xs[done]))
        done += 1
    dt = time.perf_counter() - t0
    out = dict(value=done / dt, unit="amplitudes/s", seconds=dt,
               sample=f"FP64 oracle network sweep, {{done}} of the 4096 bitstrings ({{dt:.1f}} s)")
elif kind == "serve":
    circs = [c for c in C.serving_mix(512, {seed}) if c.n_qubits <= 20]  # a sample bounded in time
    done = amps = 0
    for c in circs:
        if done and time.perf_counter() - t0 > budget:
            break
        simulate_state(c)
        done += 1
        amps += 1 << c.n_qubits
    dt = time.perf_counter() - t0
    out = dict(value=amps / dt, unit="amplitudes/s", seconds=dt,
               sample=f"FP64 state-vector oracle, the first {{done}} of the mix's circuits of at most 20 qubits "
                      f"({{dt:.1f}} s)")
elif kind == "sweep":
    pts = [(n, k) for n in range(2, 29, 2) for k in range(2, 15, 2)]
    done = amps = 0
    for i, (n, k) in enumerate(pts):
        if done and time.perf_counter() - t0 > budget:
            break
        simulate_state(C.paper_fig31(n, k, {seed} + i))
        done += 1
        amps += 1 << n
    dt = time.perf_counter() - t0
    out = dict(value=amps / dt, unit="amplitudes/s", seconds=dt,
               sample=f"FP64 state-vector oracle, the {{done}} smallest of the 98 Fig. 3.1 circuits ({{dt:.1f}} s)")
elif kind == "q428":
    from oracle.fixedpoint import apply_gate_q, quantize_matrix, ONE
    m = min(12, {n})
    while True:
        c, _ = C.brickwork(m, {depth}, {seed})
        t1 = time.perf_counter()
        re = np.zeros(1 << c.n_qubits, dtype=np.int64)
        im = np.zeros(1 << c.n_qubits, dtype=np.int64)
        re[0] = ONE
        for g in c.gates:
            Ur, Ui = quantize_matrix(gate_matrix(c, g, None))
            re, im = apply_gate_q(re, im, c.n_qubits, Ur, Ui, g.qubits)
        dt = time.perf_counter() - t1
        if m >= {n} or time.perf_counter() - t0 + 2.2 * dt > budget:
            break
        m += 1
    out = dict(value=(1 << m) / dt, unit="amplitudes/s", seconds=dt,
               sample=f"Q4.28 fixed-point oracle (numpy int64), the whole {{m}}-qubit brickwork of depth "
                      f"{depth} ({{len(c.gates)}} gates, {{dt:.1f}} s; the widest that fits the time budget, "
                      f"not scaled)")
elif kind == "sweep_amps":
    pts = [(n, k) for n in range(2, 29, 2) for k in range(2, 15, 2)]
    done = 0
    for i, (n, k) in enumerate(pts):  # one bitstring per point, until the budget is spent
        if done and time.perf_counter() - t0 > budget:
            break
        c = C.paper_fig31(n, k, {seed} + i)
        contract_amplitude(c, int(C.random_bitstrings(n, 1, {seed} + 500 + i)[0]))
        done += 1
    dt = time.perf_counter() - t0
    out = dict(value=done / dt, unit="amplitudes/s", seconds=dt,
               sample=f"FP64 oracle greedy network contraction, one amplitude of each of the first {{done}} "
                      f"of the 98 Fig. 3.1 circuits ({{dt:.1f}} s)")
print(json.dumps(out))
"""

ORACLE_KINDS = ("state", "grad", "amps", "serve", "sweep", "sweep_amps", "q428")


def run_oracle_sample(kind: str, n: int, depth: int, seed: int, budget: float, threads: int = 1):
    code = ORACLE_SNIPPET.format(root=ROOT, kind=kind, n=n, depth=depth, seed=seed, budget=budget)
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return None, r.stderr[-400:]
    return json.loads(r.stdout.strip().splitlines()[-1]), None


# ----------------------------------------------------------------------------- workloads

WORKLOADS = {
    "state24": dict(kind="state", n=24, depth=20, seed=1001, batch=1),
    # batched complex GEMM of a pairwise merge (kernel c): C[b] = A[b] B[b]^T, complex64
    # 6x6 grid, depth 12, 4096 random bitstrings, amplitudes by network contraction (64 per call)
    "amps36": dict(kind="amps", n=36, depth=12, seed=3003, batch=4096, chunk=64),
    # batched serving mix: 512 circuits, n ~ U[8, 22], depth ~ U[4, 30], half brickwork, half QFT
    "serving512": dict(kind="serve", n=0, depth=0, seed=5000, batch=512),
    # the same mix with the brickwork halves' U3 angles as parameters (gate tables built in the run)
    "serving512p": dict(kind="serve", n=0, depth=0, seed=5000, batch=512, params=True),
    "gemm_fp32": dict(kind="gemm", prec=0, M=4096, N=4096, K=4096, batch=1, n=0, depth=0, seed=7),
    "gemm_3xtf32": dict(kind="gemm", prec=1, M=4096, N=4096, K=4096, batch=1, n=0, depth=0, seed=7),
    "gemm_bf16x3": dict(kind="gemm", prec=2, M=4096, N=4096, K=4096, batch=1, n=0, depth=0, seed=7),
    # the dense merge of the 6x6 grid network (64 bitstrings): HBM-bound, 3xTF32 split on chip
    "gemm_merge": dict(kind="gemm", prec=1, M=32768, N=64, K=64, batch=64, n=0, depth=0, seed=7),
    # index permutation (kernel b) of a 2^28-leg complex64 tensor (2 GiB): low legs kept, full
    # reversal, and a seeded random permutation, one launch each per step
    "permute28": dict(kind="permute", n=28, depth=0, seed=2800, batch=1),
    "state10": dict(kind="state", n=10, depth=8, seed=1000, batch=512),
    # the paper's Fig. 3.1 test circuits: n in {2, 4, ..., 28} qubits, k in {2, 4, ..., 14} rounds,
    # full states; a step contracts all 98 of them
    "fig31": dict(kind="sweep", n=28, depth=14, seed=6000, batch=98),
    # the same 98 circuits in amplitude mode: 64 seeded bitstrings each, by network contraction
    # (3xTF32 merges, one plan per circuit sized for 64 bitstrings per call)
    "fig31amps": dict(kind="sweep_amps", n=28, depth=14, seed=6000, batch=98, chunk=64, prec=1),
    "grad20": dict(kind="grad", n=20, depth=10, seed=4000, batch=64),
    # the 24-qubit brickwork (depth 20, fixed angles) in the paper's Q4.28 fixed-point arithmetic:
    # one HBM-bound launch per gate on int32 pairs
    "q428_24": dict(kind="q428", n=24, depth=20, seed=1001, batch=1),
    # contraction-path search on the host (the paper's E1 grid): the 98 Fig. 3.1 circuits planned
    # for 64 bitstrings per call, the deterministic greedy alone against the randomised search
    "plan31": dict(kind="plan", n=28, depth=14, seed=6000, batch=98, chunk=64),
}


def plan_search_line(args, wl):
    """Host-only measurement: planning time and planned cost per Fig. 3.1 circuit, greedy alone
    (order_trials = 1) against the default search and the adaptive search; no GPU work."""
    from paper_2108_06831_gb300 import circuits as C
    from paper_2108_06831_gb300 import tn
    pts = wl.get("points") or [(n, k) for n in range(2, 29, 2) for k in range(2, 15, 2)]
    per_point, tot = {}, {"greedy": [0.0, 0.0], "search": [0.0, 0.0], "adaptive": [0.0, 0.0]}
    for i, (n, k) in enumerate(pts):
        ch = tn.CircuitHandle(C.paper_fig31(n, k, wl["seed"] + i))
        row = {}
        for name, trials, adaptive in (("greedy", 1, 0), ("search", 0, 0), ("adaptive", 0, 1)):
            t0 = time.perf_counter()
            st = tn.Plan(ch, target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=wl["chunk"],
                         precision=1, order_trials=trials, order_search=adaptive).stats()
            dt = time.perf_counter() - t0
            row[name] = {"plan_s": round(dt, 4), "cost_bytes": st["net_cost"], "largest_intermediate_log2":
                         st["net_max_log2"], "merges": st["net_merges"]}
            tot[name][0] += dt
            tot[name][1] += st["net_cost"]
        per_point[f"n{n}_k{k}"] = row
    ratios = sorted(r["greedy"]["cost_bytes"] / r["search"]["cost_bytes"] for r in per_point.values())
    return {"metric": "contraction-path search time (host), Fig. 3.1 grid", "value": tot["search"][0], "unit": "s",
            "n_gpus": 0, "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * tot["search"][0],
            "higher_is_better": False, "scaling": None, "vs_baseline": None, "dtype": "f64 (host planning)",
            "data": "synthetic", "gpu_launches": 0, "roofline": None,
            "config": {"workload": args.workload, "points": "n in 2..28 step 2, k in 2..14 step 2",
                       "bitstrings_per_call": wl["chunk"], "host_cores": os.cpu_count(),
                       "search": "256 orders per search (greedy, step-wise greedy, qubit sweep, fold-first), "
                                 "every bitstring pass size"},
            "greedy": {"seconds": tot["greedy"][0], "cost_bytes_total": tot["greedy"][1]},
            "search": {"seconds": tot["search"][0], "cost_bytes_total": tot["search"][1]},
            "adaptive": {"seconds": tot["adaptive"][0], "cost_bytes_total": tot["adaptive"][1],
                         "what": "order_search = 1: cross-entropy search over trial kind, temperature and "
                                 "bitstring-index weight, 256 orders in 4 rounds"},
            "greedy_over_search_cost": {"median": ratios[len(ratios) // 2], "max": ratios[-1], "min": ratios[0]},
            "per_point": per_point}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    if wl["kind"] == "plan":
        print(json.dumps({"impl": "reference", "unavailable": "host-only planning workload: the oracle contracts "
                          "in its own fixed order and has no order search to time"}))
        return 0
    if wl["kind"] not in ORACLE_KINDS:
        print(json.dumps({"impl": "reference", "unavailable": "kernel-level workload with no oracle counterpart "
                          "(the oracle computes states, amplitudes and expectations, not bare GEMMs or permutes)"}))
        return 0
    vals = []
    info = None
    for _ in range(args.warmup):
        run_oracle_sample(wl["kind"], wl["n"], wl["depth"], wl["seed"], 2.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        info, err = run_oracle_sample(wl["kind"], wl["n"], wl["depth"], wl["seed"], 8.0)
        if info is None:
            print(json.dumps({"impl": "reference", "unavailable": f"oracle sample failed: {err}"}))
            return 0
        vals.append(info["value"])
    wall = time.perf_counter() - t0
    unit = info["unit"]
    v = statistics.median(vals)
    sample = info["sample"] + ", 1 thread"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "q4.28 (int64 sums)" if wl["kind"] == "q428" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, **{k: wl[k] for k in ("n", "depth", "batch")}},
            "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    wl = WORKLOADS[args.workload]
    if wl["kind"] == "plan":
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(plan_search_line(args, wl)))
        return 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline runs first, in a fresh process, before this process touches the GPU
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and wl["kind"] in ORACLE_KINDS:
        info, err = run_oracle_sample(wl["kind"], wl["n"], wl["depth"], wl["seed"], 20.0)
        if info is not None:
            cpu = {"value": info["value"], "unit": info["unit"], "cores": 1, "kind": "oracle",
                   "sample": info["sample"] + ", 1 thread"}
        else:
            cpu = {"value": None, "unit": None, "cores": 1, "kind": "oracle", "sample": f"failed: {err}"}
        # the same sample with the BLAS threads on every host core (numpy tensordot / einsum)
        ncores = os.cpu_count() or 1
        info_all, _ = run_oracle_sample(wl["kind"], wl["n"], wl["depth"], wl["seed"], 20.0, threads=ncores)
        if info_all is not None:
            cpu_all = {"value": info_all["value"], "unit": info_all["unit"], "cores": ncores, "kind": "oracle",
                       "sample": info_all["sample"] + f", {ncores} BLAS threads"}

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2108_06831_gb300 import circuits as C
    from paper_2108_06831_gb300 import tn

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > L2

    hbm_peak, peak_kind = load_peaks()
    set_fp32_peak(tn, torch, dev)
    if wl["kind"] == "state":
        circ_p, params0 = C.brickwork(wl["n"], wl["depth"], wl["seed"], parameterized=True)
        circ_f, _ = C.brickwork(wl["n"], wl["depth"], wl["seed"])
        batch = wl["batch"]
        params = np.tile(params0, (batch, 1))
        spec = not args.no_specialize
        bprec = args.prec if args.blocks else 0
        ctr = tn.Contractor(circ_p, batch=batch, tile_qubits=args.tile, device=dev, specialize=spec,
                            fuse=not args.no_fuse, block_qubits=args.blocks, precision=bprec)
        p_dev = torch.as_tensor(params, device=dev)
        out = torch.empty((batch, 1 << wl["n"]), dtype=torch.complex64, device=dev)
        units_per_step = batch * (1 << wl["n"])
        unit = "amplitudes/s"

        def step():
            tn.contract_state(ctr.plan, p_dev, out, ctr.workspace)
        launches_per_step = 1 + ctr.plan.stats()["n_passes"]
        if args.blocks:  # block build + first block; per GEMM the B operand's split (tensor cores) + the GEMM
            launches_per_step = 2 + ctr.plan.stats()["n_passes"] * (2 if bprec else 1)
        import tempfile
        dump = tempfile.mkdtemp(prefix="tnq_src_")
        os.environ["TNQ_JIT_DUMP_DIR"] = dump  # the timed plan's generated sources, hashed below
        fixed = tn.Contractor(circ_f, batch=batch, tile_qubits=args.tile, device=dev, specialize=spec,
                              fuse=not args.no_fuse, block_qubits=args.blocks, precision=bprec)
        del os.environ["TNQ_JIT_DUMP_DIR"]
        kernel_hash = jit_source_hash(dump)
        import shutil
        shutil.rmtree(dump, ignore_errors=True)
        fst = fixed.plan.stats()

        def kernel_only():
            tn.contract_state(fixed.plan, None, out, fixed.workspace)
        kernel_launches = fst["n_passes"]
        alg_bytes = fst["hbm_bytes"] * batch
        alg_flops = fst["flops"] * batch
        # the circuit's own count: every one-qubit gate as a general 2x2 complex product, 14 real
        # flops per amplitude (2 complex multiplies, 1 complex add); CZ (a sign) none
        plain_flops = 14.0 * (1 << wl["n"]) * batch * sum(1 for g in circ_f.gates if len(g.qubits) == 1)
    elif wl["kind"] == "serve":
        circs = C.serving_mix(wl["batch"], wl["seed"])
        handles = [tn.CircuitHandle(c) for c in circs]
        t_tune = time.perf_counter()
        # tile sizes of the executor's circuits picked by measurement; circuits of SERVE_WIDE qubits
        # and more get generated kernels (compiled in parallel) run on side streams (untimed setup)
        bat = tn.Batch.tuned(handles)
        t_tune = time.perf_counter() - t_tune
        # the sequential comparison: each circuit on its own, wide ones through their generated kernels
        plans = [tn.Plan(h, specialize=c.n_qubits >= SERVE_WIDE) for h, c in zip(handles, circs)]
        wide_passes = sum(p.stats()["n_passes"] for p, c in zip(plans, circs) if c.n_qubits >= SERVE_WIDE)
        tiles_by_n = {}
        for c, t in zip(circs, bat.tiles):
            tiles_by_n.setdefault(c.n_qubits, set()).add(t)
        states = torch.empty(bat.state_elems, dtype=torch.complex64, device=dev)
        bws = torch.empty(bat.workspace_bytes, dtype=torch.uint8, device=dev)
        batch = len(circs)
        units_per_step = float(sum(1 << c.n_qubits for c in circs))
        unit = "amplitudes/s"
        run_params = None
        if wl.get("params"):
            # the brickwork halves' U3 angles as per-run parameters: plans at the tiles the autotuner
            # picked for the same circuits with fixed angles, gate tables built inside each run
            circs_p, params_p = C.serving_mix_params(wl["batch"], wl["seed"])
            pplans = [tn.Plan(tn.CircuitHandle(c), tile_qubits=t, specialize=c.n_qubits >= SERVE_WIDE)
                      for c, t in zip(circs_p, bat.tiles)]
            bat = tn.Batch(pplans)
            flat = np.zeros(max(bat.n_params, 1))
            for pv, off in zip(params_p, bat.param_offsets):
                flat[off:off + len(pv)] = pv
            run_params = torch.as_tensor(flat, device=dev)
            bws = torch.empty(bat.workspace_bytes, dtype=torch.uint8, device=dev)
        tn.batch_run(bat, states, bws, params=run_params)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                tn.batch_run(bat, states, bws, params=run_params)
        torch.cuda.synchronize()

        def step():
            graph.replay()
        # (gate tables +) the persistent kernel + the wide circuits' pass kernels
        launches_per_step = (2 if run_params is not None else 1) + wide_passes
        kernel_only = None
        ctr = None
        # the comparison: every circuit contracted on its own, one after another
        seq_bufs = [torch.empty(1 << c.n_qubits, dtype=torch.complex64, device=dev) for c in circs]
        seq_ws = torch.empty(16, dtype=torch.uint8, device=dev)

        def seq_step():
            for p, buf in zip(plans, seq_bufs):
                tn.contract_state(p, None, buf, seq_ws)
    elif wl["kind"] == "amps":
        circ = C.grid(6, 6, wl["depth"], wl["seed"])
        chunk = wl["chunk"]
        ctr = None
        plan = tn.Plan(tn.CircuitHandle(circ), target=tn.TARGET_AMPLITUDES, network_bitstrings=chunk,
                       precision=args.prec, max_intermediate_log2=args.max_log2, order_search=args.order_search,
                       order_trials=args.order_trials)
        nst = plan.stats()
        aws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
        xs_h = C.random_bitstrings(36, wl["batch"], wl["seed"] + 1)
        xs = torch.as_tensor(xs_h.astype(np.int64), device=dev)
        amps = torch.empty(wl["batch"], dtype=torch.complex64, device=dev)
        batch = wl["batch"]
        units_per_step = float(batch)
        unit = "amplitudes/s"

        def eager_step():
            for i in range(0, batch, chunk):
                tn.contract_amplitudes(plan, None, xs[i:i + chunk], amps[i:i + chunk], aws)
        # one call captured once as a CUDA graph (a capped plan's call is tens of thousands of small
        # launches); a step copies each chunk of bitstrings into the captured buffer and replays it
        xs_c = torch.empty(chunk, dtype=torch.int64, device=dev)
        amps_c = torch.empty(chunk, dtype=torch.complex64, device=dev)
        xs_c.copy_(xs[:chunk])
        tn.contract_amplitudes(plan, None, xs_c, amps_c, aws)
        torch.cuda.synchronize()
        amps_graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(cap):
            with torch.cuda.graph(amps_graph, stream=cap):
                tn.contract_amplitudes(plan, None, xs_c, amps_c, aws)
        torch.cuda.synchronize()

        def step():
            for i in range(0, batch, chunk):
                xs_c.copy_(xs[i:i + chunk])
                amps_graph.replay()
                amps[i:i + chunk].copy_(amps_c)
        # per pass of the network and slice: the closure kernel, one GEMM per launched merge, B's
        # split per tensor-core merge (and A's for split BF16); a sliced plan adds the FP64 slice
        # sum per slice and the final store per pass; a call runs chunk / 2^net_batch_log2 passes
        n_slices = 1 << nst["net_sliced"]
        per_pass = n_slices * (1 + nst["net_merges"] + nst["net_tensor_merges"] * (2 if args.prec == 2 else 1))
        if n_slices > 1:
            per_pass += n_slices + 1
        per_call = per_pass * (chunk >> nst["net_batch_log2"])
        launches_per_step = per_call * (batch // chunk)
        kernel_only = None
    elif wl["kind"] == "q428":
        circ, _ = C.brickwork(wl["n"], wl["depth"], wl["seed"])
        qplan = tn.Plan(tn.CircuitHandle(circ), q428=True)
        qst = torch.empty((1 << wl["n"], 2), dtype=torch.int32, device=dev)
        batch = 1
        units_per_step = float(1 << wl["n"])
        unit = "amplitudes/s"
        ctr = None

        def step():
            tn.contract_state_q428(qplan, qst)
        launches_per_step = 1 + len(circ.gates)  # basis state, then one launch per gate
        kernel_only = None
    elif wl["kind"] == "sweep_amps":
        pts = [(n, k) for n in range(2, 29, 2) for k in range(2, 15, 2)]
        chunk = wl["chunk"]
        nplans, nws, nxs, nout, plan_s = {}, {}, {}, {}, {}
        for i, (n, k) in enumerate(pts):
            t0 = time.perf_counter()
            nplans[(n, k)] = tn.Plan(tn.CircuitHandle(C.paper_fig31(n, k, wl["seed"] + i)),
                                     target=tn.TARGET_AMPLITUDES, network_bitstrings=chunk, precision=1,
                                     order_search=args.order_search)
            plan_s[(n, k)] = time.perf_counter() - t0
            nws[(n, k)] = torch.empty(max(nplans[(n, k)].workspace_bytes, 16), dtype=torch.uint8, device=dev)
            nxs[(n, k)] = torch.as_tensor(C.random_bitstrings(n, chunk, wl["seed"] + 1000 + i).astype(np.int64),
                                          device=dev)
            nout[(n, k)] = torch.empty(chunk, dtype=torch.complex64, device=dev)
        batch = len(pts)
        units_per_step = float(chunk * len(pts))
        unit = "amplitudes/s"
        ctr = None

        def eager_step():
            for key in pts:
                tn.contract_amplitudes(nplans[key], None, nxs[key], nout[key], nws[key])
        # the 98 calls (their closure kernels, merges and copies) captured once in a CUDA graph, as
        # independent chains on --lanes streams (circuit i on stream i mod lanes): the small merges of different
        # circuits run side by side instead of one launch after another; a step replays the graph
        eager_step()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        lanes = [torch.cuda.Stream(device=dev) for _ in range(args.lanes)]
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                for ln in lanes:
                    ln.wait_stream(cap)
                for i, key in enumerate(pts):
                    with torch.cuda.stream(lanes[i % len(lanes)]):
                        tn.contract_amplitudes(nplans[key], None, nxs[key], nout[key], nws[key])
                for ln in lanes:
                    cap.wait_stream(ln)
        torch.cuda.synchronize()

        def step():
            graph.replay()
        launches_per_step = 0
        for key in pts:
            st = nplans[key].stats()
            sl = 1 << st["net_sliced"]
            per_pass = sl * (1 + st["net_merges"] + st["net_tensor_merges"]) + (sl + 1 if sl > 1 else 0)
            launches_per_step += per_pass * (chunk >> st["net_batch_log2"])
        kernel_only = None
    elif wl["kind"] == "sweep":
        pts = [(n, k) for n in range(2, 29, 2) for k in range(2, 15, 2)]
        ctrs, outs = {}, {}
        for i, (n, k) in enumerate(pts):
            ctrs[(n, k)] = tn.Contractor(C.paper_fig31(n, k, wl["seed"] + i), device=dev)
            outs[(n, k)] = torch.empty(1 << n, dtype=torch.complex64, device=dev)
        batch = len(pts)
        units_per_step = float(sum(1 << n for n, _ in pts))
        unit = "amplitudes/s"

        def step():
            for key in pts:
                tn.contract_state(ctrs[key].plan, None, outs[key], ctrs[key].workspace)
        launches_per_step = sum(c.plan.stats()["n_passes"] for c in ctrs.values())
        kernel_only = None
        ctr = None
    elif wl["kind"] == "permute":
        n = args.legs or wl["n"]
        batch = 1
        g = torch.Generator(device=dev).manual_seed(wl["seed"])
        px = torch.randn(1 << n, dtype=torch.complex64, device=dev, generator=g)
        py = torch.empty_like(px)
        rng = np.random.default_rng(wl["seed"])
        high = [int(v) for v in rng.permutation(n - 5)]
        perms = [high + list(range(n - 5, n)), list(range(n))[::-1], [int(v) for v in rng.permutation(n)]]
        units_per_step = len(perms) * 16.0 * (1 << n) / 1e9  # algorithmic GB: read + write every element
        unit = "GB/s"

        def step():
            for pm in perms:
                tn.permute(n, pm, 1, px, py)
        launches_per_step = len(perms)
        kernel_only = None
        ctr = None
    elif wl["kind"] == "gemm":
        batch, M, N, K, prec = args.batch or wl["batch"], wl["M"], wl["N"], wl["K"], wl["prec"]
        g = torch.Generator(device=dev).manual_seed(wl["seed"])
        a = torch.randn((batch, M, K), dtype=torch.complex64, device=dev, generator=g)
        bm = torch.randn((batch, N, K), dtype=torch.complex64, device=dev, generator=g)
        cm = torch.empty((batch, M, N), dtype=torch.complex64, device=dev)
        wsb = tn.cgemm_workspace_bytes(prec, batch, M, N, K)
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
        units_per_step = 8.0 * batch * M * N * K / 1e12  # algorithmic TFLOP (complex, 4-multiply form)
        unit = "TFLOP/s"

        def step():
            tn.cgemm_batched(prec, batch, M, N, K, a, bm, cm, ws, wsb)
        # + B embed/split; + A split unless 3xTF32 splits A on chip (at most two 128-column tiles)
        launches_per_step = {0: 1, 1: 2 if 2 * N // 128 <= 2 else 3, 2: 3}[prec]
        kernel_only = None
        ctr = None
    else:
        circ = C.hea(wl["n"], wl["depth"])
        batch = wl["batch"]
        params = C.hea_params(circ.n_params, batch, wl["seed"])
        ctr = tn.Contractor(circ, target=tn.TARGET_EXPECTATION, batch=batch, tile_qubits=args.tile, device=dev)
        obs = tn.Observable(C.tfim(wl["n"]))
        p_dev = torch.as_tensor(params, device=dev)
        e_out = torch.empty(batch, dtype=torch.float64, device=dev)
        g_out = torch.empty((batch, circ.n_params), dtype=torch.float64, device=dev)
        units_per_step = batch * circ.n_params
        unit = "grads/s"

        def step():  # energies and their gradient: one forward, reduction, H psi, adjoint sweep
            tn.expectation_value_and_grad(ctr.plan, obs, p_dev, e_out, g_out, ctr.workspace)
        st = ctr.plan.stats()
        launches_per_step = None
        kernel_only = None
        bwd_alg_flops = (st["flops"] + st["bwd_flops"]) * batch
        # algorithmic HBM bytes of the call: the forward passes (plan stats), the H psi passes (psi
        # read and lambda written; lambda also read after the first), the adjoint passes (psi and
        # lambda read and written: 32 B per amplitude)
        obs_passes = tn.state_expectation_workspace_bytes(obs, 1) // (512 * 8)
        amps_b = float(1 << wl["n"])
        grad_alg_bytes = batch * (st["hbm_bytes"] + amps_b * (16.0 + 24.0 * (obs_passes - 1))
                                  + amps_b * 32.0 * st["n_bwd_passes"])

    def timed(fn, k):
        times = []
        for _ in range(k):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            times.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed steps are the profiler's capture range (ncu --profile-from-start off records only
    # these launches; without a profiler attached the two calls do nothing)
    torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        ms = timed(step, args.steps)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    # the arithmetic the step computes in: FP32 (complex64 states), or the tensor-core split forms
    prec_used = args.prec if (wl["kind"] == "amps" or (wl["kind"] == "state" and args.blocks)) else wl.get("prec", 0)
    dtype = {0: "f32", 1: "3xtf32 (f32 accumulate)", 2: "bf16x3 (f32 accumulate)"}[prec_used]
    if wl["kind"] == "permute":
        dtype = "c64 (data movement)"
    if wl["kind"] == "q428":
        dtype = "q4.28 (int32 pairs, int64 sums)"
    t_max = max_over_ranks(sum(ms), world, dev)
    value = whole_job_value(units_per_step, args.steps, world, t_max)
    assert tn.sync_status() == tn.OK

    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "n_qubits": wl["n"], "depth": wl["depth"], "batch": batch,
                       "tile_qubits": ctr.plan.stats()["tile_qubits"] if ctr is not None else None,
                       "specialized_kernels": bool(ctr.plan.stats()["specialized"]) if ctr is not None else None,
                       "fused_2q_blocks": ctr.plan.stats()["n_fused"] if ctr is not None and not args.blocks else None,
                       "order_search": ("adaptive" if args.order_search else "fixed mix")
                       if wl["kind"] in ("amps", "sweep_amps") else None,
                       "uniform_blocks": ({"block_qubits": args.blocks, "blocks": ctr.plan.stats()["n_fused"],
                                           "gemm_launches": ctr.plan.stats()["n_passes"]}
                                          if args.blocks and ctr is not None else None),
                       "l2": "256 MiB buffer written between timed steps (untimed)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary()}
    if launches_per_step is not None:
        line["gpu_launches"] = launches_per_step * args.steps

    # roofline of the dominant kernel (fused gate-apply): the fixed-angle plan launches only it
    if kernel_only is not None:
        for _ in range(3):
            kernel_only()
        kms = timed(kernel_only, args.steps)
        avg_launch_ms = statistics.mean(kms) / kernel_launches
        bytes_per_launch = alg_bytes / kernel_launches
        flops_per_launch = alg_flops / kernel_launches
        gbs = bytes_per_launch / (avg_launch_ms / 1000) / 1e9
        tfl = flops_per_launch / (avg_launch_ms / 1000) / 1e12
        hbm_frac = gbs / hbm_peak
        alu_frac = tfl / FP32_ALU_PEAK_TFLOPS
        if wl["kind"] == "state" and args.blocks:
            # uniform blocks: the dominant kernel is the batched complex GEMM (one launch per block);
            # the whole call (block build, clear, first block, GEMMs) is charged to the GEMMs
            if bprec == 0:
                tpk, tsrc, tk = alu_frac, FP32_ALU_PEAK_SRC, "alu"
                tpeak, tach = FP32_ALU_PEAK_TFLOPS, tfl
            else:
                bf16, bsrc = load_bf16_peak()
                products = 3 if bprec == 1 else 6
                tpeak = bf16 * (1.1 / 2.25) if bprec == 1 else bf16
                tach = products * tfl
                tpk, tk = tach / tpeak, "tensor"
                tsrc = bsrc + (" x 1.1/2.25 (TF32 nominal ratio)" if bprec == 1 else "")
            kname = ("k_cgemm_tc_stream (batched complex GEMM, tcgen05)" if bprec else "k_cgemm_fp32 (batched complex GEMM)")
            if tpk >= hbm_frac:
                line["roofline"] = {"bound": tk, "achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tpk,
                                    "traffic": None, "kernel": kname, "peak_source": tsrc,
                                    "also": {"hbm_gbs": gbs, "hbm_frac": hbm_frac, "hbm_peak": hbm_peak}}
            else:
                line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": hbm_frac, "traffic": None, "kernel": kname,
                                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                                    "also": {"tflops_executed": tach, "compute_frac": tpk, "compute_bound": tk}}
        elif alu_frac >= hbm_frac:
            line["roofline"] = {"bound": "alu", "achieved": tfl, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": alu_frac, "traffic": None,
                                "kernel": "tnq_p* (fused gate-apply pass kernels)",
                                "peak_source": FP32_ALU_PEAK_SRC,
                                "also": {"hbm_gbs": gbs, "hbm_frac": hbm_frac, "hbm_peak": hbm_peak,
                                         "hbm_peak_source": peak_kind}}
        else:
            line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
                                "traffic": None, "kernel": "tnq_p* (fused gate-apply pass kernels)",
                                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                                "also": {"tflops": tfl, "alu_frac": alu_frac}}
        if wl["kind"] == "state" and not args.blocks:
            # the same circuit applied one gate at a time, each gate a pass over the state (16 B per
            # amplitude): the traffic the fused passes avoid
            ub = 16.0 * (1 << wl["n"]) * batch * len(circ_f.gates)
            line["roofline"]["unfused_gate_by_gate"] = {
                "bytes_per_step": ub, "equivalent_gbs": ub / (t_max / args.steps / 1000.0) / 1e9,
                "passes_avoided": len(circ_f.gates) - kernel_launches}
        if args.workload == "state24" and not args.tile and not args.no_specialize and not args.no_fuse:
            line["roofline"]["traffic"] = recorded_traffic(kernel_hash)
            line["roofline"]["kernel_source_hash"] = kernel_hash
        line["roofline"]["launches_per_step"] = kernel_launches
        line["roofline"]["avg_launch_ms"] = avg_launch_ms
        if wl["kind"] == "state":
            ptf = plain_flops / kernel_launches / (avg_launch_ms / 1000) / 1e12
            line["roofline"]["executed_flops_per_step"] = alg_flops
            line["roofline"]["plain_2x2_count"] = {
                "flops_per_step": plain_flops, "tflops": ptf, "frac_of_fp32_peak": ptf / FP32_ALU_PEAK_TFLOPS,
                "note": "14 real flops per amplitude per one-qubit gate (general 2x2 complex product), "
                        "CZ none; 'achieved' counts the flops the kernels execute after the planner's "
                        "rewrites"}

    if args.workload == "state10":
        # the configuration is latency-bound: one circuit (batch 1) per call, microseconds per call
        one = tn.Contractor(circ_p, batch=1, tile_qubits=args.tile, device=dev, specialize=spec)
        p1 = torch.as_tensor(params0[None, :], device=dev)
        o1 = torch.empty((1, 1 << wl["n"]), dtype=torch.complex64, device=dev)

        def single():
            tn.contract_state(one.plan, p1, o1, one.workspace)
        for _ in range(5):
            single()
        line["config"]["us_per_circuit_batch1"] = 1000.0 * statistics.median(timed(single, 50))
        line["config"]["us_per_circuit_batched"] = 1000.0 * (t_max / args.steps) / batch

    # end to end through the public API with host buffers
    if not args.no_e2e and wl["kind"] == "state":
        # every step copies its parameters in from pinned host memory, contracts, and copies the whole
        # state back to pinned host memory.  The copy back runs on a stream of its own, from one of two
        # device (and host) buffers, so that step i's transfer overlaps step i+1's contraction; a buffer
        # is written again only after its previous transfer has completed.
        h_params = torch.as_tensor(params).pin_memory()
        h_outs = [torch.empty((batch, 1 << wl["n"]), dtype=torch.complex64).pin_memory() for _ in range(2)]
        d_outs = [out, torch.empty_like(out)]
        copy_stream = torch.cuda.Stream(device=dev)
        copied = [None, None]

        def e2e_run(k):
            for i in range(k):
                j = i % 2
                if copied[j] is not None:
                    stream.wait_event(copied[j])
                p_dev.copy_(h_params, non_blocking=True)
                tn.contract_state(ctr.plan, p_dev, d_outs[j], ctr.workspace)
                ready = torch.cuda.Event()
                ready.record(stream)
                copy_stream.wait_event(ready)
                with torch.cuda.stream(copy_stream):
                    h_outs[j].copy_(d_outs[j], non_blocking=True)
                    copied[j] = torch.cuda.Event()
                    copied[j].record(copy_stream)
            for ev in copied:  # the timed region ends with the last transfer
                if ev is not None:
                    stream.wait_event(ev)
        e2e_run(3)
        torch.cuda.synchronize()
        flush.zero_()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        e2e_run(args.steps)
        t1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = t0.elapsed_time(t1)

        def e2e_step():  # the same step with nothing overlapped: copy in, contract, copy back
            p_dev.copy_(h_params, non_blocking=True)
            tn.contract_state(ctr.plan, p_dev, out, ctr.workspace)
            h_outs[0].copy_(out, non_blocking=True)
        for _ in range(3):
            e2e_step()
        seq_ms = sum(timed(e2e_step, args.steps))
        line["e2e"] = {"value": units_per_step * args.steps / (e2e_ms / 1000), "unit": unit,
                       "sequential_value": units_per_step * args.steps / (seq_ms / 1000),
                       "h2d_bytes_per_step": int(h_params.numel() * 8),
                       "d2h_bytes_per_step": int(h_outs[0].numel() * 8),
                       "overlap": "each step's device-to-host copy runs on a second stream beside the next "
                                  "step's contraction (two output buffers)"}
    elif not args.no_e2e and wl["kind"] == "grad":
        h_params = torch.as_tensor(params).pin_memory()
        h_g = torch.empty_like(g_out, device="cpu").pin_memory()
        h_e = torch.empty_like(e_out, device="cpu").pin_memory()

        def e2e_step():
            p_dev.copy_(h_params, non_blocking=True)
            step()
            h_e.copy_(e_out, non_blocking=True)
            h_g.copy_(g_out, non_blocking=True)
        for _ in range(3):
            e2e_step()
        ems = timed(e2e_step, args.steps)
        line["e2e"] = {"value": units_per_step * args.steps / (sum(ems) / 1000), "unit": unit,
                       "h2d_bytes_per_step": int(h_params.numel() * 8),
                       "d2h_bytes_per_step": int((h_g.numel() + h_e.numel()) * 8)}
    if not args.no_e2e and wl["kind"] == "amps":
        h_xs = torch.as_tensor(xs_h.astype(np.int64)).pin_memory()
        h_amps = torch.empty(batch, dtype=torch.complex64).pin_memory()

        def e2e_step():
            xs.copy_(h_xs, non_blocking=True)
            step()
            h_amps.copy_(amps, non_blocking=True)
        for _ in range(3):
            e2e_step()
        ems = timed(e2e_step, args.steps)
        line["e2e"] = {"value": units_per_step * args.steps / (sum(ems) / 1000), "unit": unit,
                       "h2d_bytes_per_step": int(h_xs.numel() * 8), "d2h_bytes_per_step": int(h_amps.numel() * 8)}
    if not args.no_e2e and wl["kind"] == "sweep_amps":
        h_xs = {key: nxs[key].cpu().pin_memory() for key in pts}
        h_amps = {key: torch.empty(chunk, dtype=torch.complex64).pin_memory() for key in pts}

        def e2e_step():
            for key in pts:
                nxs[key].copy_(h_xs[key], non_blocking=True)
                tn.contract_amplitudes(nplans[key], None, nxs[key], nout[key], nws[key])
                h_amps[key].copy_(nout[key], non_blocking=True)
        for _ in range(3):
            e2e_step()
        ems = timed(e2e_step, args.steps)
        line["e2e"] = {"value": units_per_step * args.steps / (sum(ems) / 1000), "unit": unit,
                       "h2d_bytes_per_step": int(sum(v.numel() for v in h_xs.values()) * 8),
                       "d2h_bytes_per_step": int(sum(v.numel() for v in h_amps.values()) * 8)}
    if wl["kind"] == "amps":
        per_step_s = t_max / args.steps / 1000.0
        a = amps.cpu().numpy().astype(np.complex128)
        line["config"].update({"grid": "6x6", "bitstrings": batch, "bitstrings_per_call": wl["chunk"],
                               "precision": args.prec, "merges_per_pass": nst["net_merges"],
                               "largest_intermediate_log2": nst["net_max_log2"],
                               "max_intermediate_log2": args.max_log2 or 28, "sliced_indices": nst["net_sliced"],
                               "bitstrings_per_pass": 1 << nst["net_batch_log2"],
                               "tensor_core_merges_per_pass": nst["net_tensor_merges"]})
        line["config"]["folded_merges"] = nst["net_folded_merges"]
        line["config"]["launch"] = "each call of 64 bitstrings replays one captured CUDA graph"
        for _ in range(2):
            eager_step()
        eager_ms = statistics.mean(timed(eager_step, max(2, min(args.steps, 3))))
        line["eager"] = {"value": units_per_step / (eager_ms / 1000.0), "unit": unit, "ms_per_step": eager_ms,
                         "what": "the same calls issued one by one (no graph)"}
        # the dominant kernel: the dense merges (batch 64, M 32768, N = K = 64), HBM-bound;
        # the same GEMM shape is timed alone here with CUDA events (A read once as FP32 when
        # the split runs on chip; the epilogue of a network merge also permutes its output)
        gb, gm, gn, gk = wl["chunk"], 32768, 64, 64
        ga = torch.randn((gb, gm, gk), dtype=torch.complex64, device=dev)
        gbm = torch.randn((gb, gn, gk), dtype=torch.complex64, device=dev)
        gc = torch.empty((gb, gm, gn), dtype=torch.complex64, device=dev)
        gwsb = tn.cgemm_workspace_bytes(args.prec, gb, gm, gn, gk)
        gws = torch.empty(max(gwsb, 16), dtype=torch.uint8, device=dev)

        def merge_gemm():
            tn.cgemm_batched(args.prec, gb, gm, gn, gk, ga, gbm, gc, gws, gwsb)
        for _ in range(3):
            merge_gemm()
        kms = statistics.mean(timed(merge_gemm, args.steps))
        alg_bytes = 8.0 * gb * (gm * gk + gn * gk + gm * gn)  # complex64 A, B read, C written
        ach = alg_bytes / (kms / 1000.0) / 1e9
        if args.prec == 0:
            # plain FP32 on the CUDA cores: 8 real flops per complex multiply-add make this shape
            # ALU-bound (32 flops per byte moved), so its roof is the FP32 rate
            tfl = 8.0 * gb * gm * gn * gk / (kms / 1000.0) / 1e12
            line["roofline"] = {"bound": "alu", "achieved": tfl, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": tfl / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                                "kernel": "dense network merge GEMM (batch 64, M 32768, N 64, K 64; k_cgemm_fp32)",
                                "avg_launch_ms": kms, "peak_source": FP32_ALU_PEAK_SRC,
                                "also": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "frac": ach / hbm_peak},
                                "flops_per_s_all_merges": nst["flops"] * (batch // wl["chunk"]) / per_step_s}
        else:
            line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                                "frac": ach / hbm_peak, "traffic": None,
                                "kernel": "dense network merge GEMM (batch 64, M 32768, N 64, K 64; "
                                          + ("k_cgemm_tc_stream" if args.prec == 1 else "k_cgemm_tc + split") + ")",
                                "avg_launch_ms": kms, "algorithmic_bytes_per_launch": alg_bytes,
                                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                                "flops_per_s_all_merges": nst["flops"] * (batch // wl["chunk"]) / per_step_s}
        # Porter-Thomas check of the amplitudes: mean |a|^2 2^36 should be near 1
        line["porter_thomas_mean"] = float(np.mean(np.abs(a) ** 2) * 2.0 ** 36)
    if wl["kind"] == "grad":
        # the step is one call: forward (tnq_p*), reduction, H psi, adjoint sweep (tnq_b*, every op
        # on psi and lambda plus derivative dots); the gate work against the FP32 ALU roof
        tfl = bwd_alg_flops / (t_max / args.steps / 1000.0) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": tfl, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tfl / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                            "kernel": "tn_expectation_value_and_grad (tnq_p* forward + tnq_b* adjoint sweep)",
                            "algorithmic_flops_per_call": bwd_alg_flops,
                            "peak_source": FP32_ALU_PEAK_SRC}
        gbs = grad_alg_bytes / (t_max / args.steps / 1000.0) / 1e9
        line["roofline"]["also"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": gbs / hbm_peak, "algorithmic_bytes_per_call": grad_alg_bytes,
                                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if wl["kind"] == "serve":
        for _ in range(2):
            seq_step()
        sms = timed(seq_step, max(1, args.steps // 2))
        line["config"].update({"circuits": batch, "amplitudes_per_step": units_per_step,
                               "launch": (f"one CUDA graph: the persistent kernel for the circuits under {SERVE_WIDE} "
                                          f"qubits, beside the generated pass kernels of the "
                                          f"{sum(1 for c in circs if c.n_qubits >= SERVE_WIDE)} wider ones on 4 "
                                          f"side streams"),
                               "tiles_by_qubits": {str(k): sorted(v) for k, v in sorted(tiles_by_n.items())},
                               "autotune_seconds": round(t_tune, 1)})
        if run_params is not None:
            line["config"]["parameters"] = (f"{bat.n_params} float64 parameters (the brickwork halves' U3 angles) "
                                            f"read per run: gate tables built by one kernel inside each run")
        line["sequential"] = {"value": units_per_step / (statistics.mean(sms) / 1000.0), "unit": unit,
                              "ms_per_step": statistics.mean(sms),
                              "what": "the same circuits contracted one after another (tn_contract_state each)"}
        # the persistent executor (the step's one kernel) against the FP32 ALU roof: algorithmic
        # flops of every circuit's gates
        alg = sum(p.stats()["flops"] for p in plans)
        tfl = alg / (t_max / args.steps / 1000.0) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": tfl, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tfl / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                            "kernel": "k_batch_exec + the wide circuits' tnq_p* (one graph)",
                            "peak_source": FP32_ALU_PEAK_SRC}
        # the same step against HBM: every circuit's passes (8 B per amplitude for the first, 16 after)
        sbytes = sum(p.stats()["hbm_bytes"] for p in plans)
        gbs = sbytes / (t_max / args.steps / 1000.0) / 1e9
        line["roofline"]["also"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": gbs / hbm_peak, "algorithmic_bytes_per_step": sbytes,
                                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if wl["kind"] == "sweep":
        # amplitudes/s of every (n, k) point, each timed on its own; the roofline is the largest
        # point's (n = 28, k = 14: 2 GiB state) gate work against the FP32 ALU peak
        sweep = {}
        for key in pts:
            c = ctrs[key]

            def one():
                tn.contract_state(c.plan, None, outs[key], c.workspace)
            for _ in range(2):
                one()
            pms = statistics.mean(timed(one, max(2, args.steps)))
            sweep[f"n{key[0]}_k{key[1]}"] = round((1 << key[0]) / (pms / 1000.0), 1)
            if key == pts[-1]:
                big_ms, big_flops = pms, c.plan.stats()["flops"]
        tfl = big_flops / (big_ms / 1000.0) / 1e12
        line["config"].update({"points": "n in 2..28 step 2, k in 2..14 step 2", "circuits_per_step": batch})
        line["per_point_amplitudes_per_s"] = sweep
        line["roofline"] = {"bound": "alu", "achieved": tfl, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tfl / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                            "kernel": "tnq_p* (fused gate-apply), Fig. 3.1 circuit n=28 k=14",
                            "peak_source": FP32_ALU_PEAK_SRC}
    if wl["kind"] == "sweep_amps":
        # per point: amplitudes/s of its call timed on its own, planning time (host), plan shape;
        # roofline: the algorithmic bytes of every launched merge of the step against HBM
        per_point = {}
        for key in pts:
            pl = nplans[key]

            def one():
                tn.contract_amplitudes(pl, None, nxs[key], nout[key], nws[key])
            for _ in range(2):
                one()
            pms = statistics.mean(timed(one, max(2, args.steps)))
            st = pl.stats()
            per_point[f"n{key[0]}_k{key[1]}"] = {
                "amplitudes_per_s": round(chunk / (pms / 1000.0), 1), "plan_s": round(plan_s[key], 3),
                "merges": st["net_merges"], "bitstrings_per_pass": 1 << st["net_batch_log2"],
                "largest_intermediate_log2": st["net_max_log2"]}
        per_step_s = t_max / args.steps / 1000.0
        step_bytes = sum(nplans[key].stats()["net_bytes"] for key in pts)
        ach = step_bytes / per_step_s / 1e9
        for _ in range(2):
            eager_step()
        eager_ms = statistics.mean(timed(eager_step, max(2, args.steps)))
        line["config"].update({"points": "n in 2..28 step 2, k in 2..14 step 2", "circuits_per_step": batch,
                               "bitstrings_per_circuit": chunk, "precision": 1,
                               "launch": "the step's 98 calls replayed as one CUDA graph",
                               "planning_s_total": round(sum(plan_s.values()), 2)})
        line["eager"] = {"value": units_per_step / (eager_ms / 1000.0), "unit": unit, "ms_per_step": eager_ms,
                         "what": "the same 98 calls issued one by one (no graph)"}
        line["per_point"] = per_point
        line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": ach / hbm_peak, "traffic": None,
                            "kernel": "network merges (k_cgemm_fp32 / k_cgemm_tc*) of all 98 circuits",
                            "algorithmic_bytes_per_step": step_bytes,
                            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if wl["kind"] == "q428":
        # algorithmic bytes of the step: the basis state written, then every amplitude read and
        # written once per gate (int32 pairs); all launches of the step are of this kind
        per_step_s = t_max / args.steps / 1000.0
        qb = qplan.stats()["hbm_bytes"]
        ach = qb / per_step_s / 1e9
        # the same circuit through the FP32 path: relative 2-norm difference of the two states
        fctr = tn.Contractor(circ, device=dev)
        f32 = fctr.state(None)[0].to(torch.complex128)
        qv = (qst[:, 0].to(torch.float64) + 1j * qst[:, 1].to(torch.float64)) / float(1 << 28)
        diff = (torch.linalg.vector_norm(qv - f32) / torch.linalg.vector_norm(f32)).item()
        line["config"].update({"circuit": "brickwork, fixed angles", "arithmetic": "Q4.28: int32 values q/2^28, "
                               "exact 64-bit sums, round half up, saturating", "gates": len(circ.gates)})
        line["rel_l2_vs_fp32_path"] = diff
        qhash = file_hash(os.path.join(ROOT, "paper_2108_06831_gb300", "csrc", "k_q428.cu"))
        line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": ach / hbm_peak, "traffic": recorded_traffic(qhash, "q428_state24.md"),
                            "traffic_kernel": "k_q428_g1", "kernel_source_hash": qhash,
                            "kernel": "k_q428_g1 / k_q428_g2",
                            "algorithmic_bytes_per_step": qb, "avg_launch_ms": 1000.0 * per_step_s / launches_per_step,
                            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if not args.no_e2e and wl["kind"] == "q428":
        h_q = torch.empty((1 << wl["n"], 2), dtype=torch.int32).pin_memory()

        def e2e_step():
            tn.contract_state_q428(qplan, qst)
            h_q.copy_(qst, non_blocking=True)
        for _ in range(3):
            e2e_step()
        ems = timed(e2e_step, args.steps)
        line["e2e"] = {"value": units_per_step * args.steps / (sum(ems) / 1000), "unit": unit,
                       "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(h_q.numel() * 4)}
    if wl["kind"] == "permute":
        per_step_s = t_max / args.steps / 1000.0
        ach = units_per_step / per_step_s
        line["config"].update({"legs": n, "tensor_bytes": 8 << n,
                               "permutations": "low 5 legs kept / all legs reversed / seeded random"})
        line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": ach / hbm_peak, "traffic": None, "kernel": "k_permute",
                            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if wl["kind"] == "gemm":
        # tensor-pipe roofline of the whole call (operand split + GEMM), against the peak of the
        # arithmetic the tensor cores run: TF32 = measured bf16 peak x nominal 1.1/2.25
        bf16_peak, bf16_src = load_bf16_peak()
        per_step_s = t_max / args.steps / 1000.0
        alg = 8.0 * batch * wl["M"] * wl["N"] * wl["K"]
        alg_bytes = 8.0 * batch * (wl["M"] * wl["K"] + wl["N"] * wl["K"] + wl["M"] * wl["N"])
        hbm_ach = alg_bytes / per_step_s / 1e9
        hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
               "traffic": None, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
               "algorithmic_bytes_per_launch": alg_bytes}
        line["config"].update({"M": wl["M"], "N": wl["N"], "K": wl["K"], "precision": wl["prec"]})
        if wl["prec"] == 0:
            comp = {"bound": "alu", "achieved": alg / per_step_s / 1e12, "peak": FP32_ALU_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": alg / per_step_s / 1e12 / FP32_ALU_PEAK_TFLOPS,
                    "traffic": None, "kernel": "k_cgemm_fp32", "peak_source": FP32_ALU_PEAK_SRC}
        else:
            products = 3 if wl["prec"] == 1 else 6
            executed = products * alg  # real tensor flops: products x (2M)(2N)(2K)/... = products x 8MNK
            peak = bf16_peak * (1.1 / 2.25) if wl["prec"] == 1 else bf16_peak
            ach = executed / per_step_s / 1e12
            comp = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None,
                    "kernel": "k_cgemm_tc / k_cgemm_tc_stream (+ operand split kernels)",
                    "peak_source": bf16_src + (" x 1.1/2.25 (TF32 nominal ratio)" if wl["prec"] == 1 else "")}
        hbm["kernel"] = comp["kernel"]
        # the binding roof is the one the kernel is closest to
        line["roofline"] = dict(comp if comp["frac"] >= hbm["frac"] else hbm)
        line["roofline"]["also"] = {k: (hbm if comp["frac"] >= hbm["frac"] else comp)[k]
                                    for k in ("bound", "achieved", "peak", "unit", "frac")}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if cpu_all is not None:
        line["cpu_baseline_all_cores"] = cpu_all
    if rank == 0 and world == 1 and args.workload == "state24" and not args.no_configs and not args.blocks \
            and not args.no_fuse and not args.tile and not args.no_specialize:
        # the other configurations, each measured in its own process after this one's timed region
        # (short runs: 3 warm-up and 5 timed steps, no CPU baseline); the headline above is config 2
        torch.cuda.synchronize()
        line["other_configs"] = other_configs()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


OTHER_CONFIGS = [
    ("config 1: 10-qubit brickwork depth 8, 512 parameter sets per call", ["--workload", "state10"]),
    ("config 2, split precision on: uniform 2^6 x 2^6 blocks, 3xTF32 tensor-core GEMMs",
     ["--blocks", "6", "--prec", "1"]),
    ("config 2, split precision on: uniform 2^6 x 2^6 blocks, split-BF16 tensor-core GEMMs",
     ["--blocks", "6", "--prec", "2"]),
    ("config 3: 6x6 grid depth 12, 4096 amplitudes, 3xTF32 merges", ["--workload", "amps36", "--prec", "1"]),
    ("config 3, plain FP32 merges", ["--workload", "amps36", "--prec", "0"]),
    ("config 4: 20-qubit HEA, TFIM energy + adjoint gradient, 64 parameter sets", ["--workload", "grad20"]),
    ("config 5: 512-circuit serving mix, one CUDA graph (persistent launch + wide circuits on side streams)",
     ["--workload", "serving512"]),
]


def other_configs():
    """Short runs of the other configurations in fresh processes: value, unit, time per step,
    roofline fraction and bound of each (or the failure)."""
    out = {}
    for name, extra in OTHER_CONFIGS:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "5", "--warmup", "3",
               "--no-cpu-baseline", "--no-e2e"] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            d = json.loads(r.stdout.strip().splitlines()[-1])
            rf = d.get("roofline") or {}
            out[name] = {"value": d["value"], "unit": d["unit"], "ms_per_step": round(d["ms_per_step"], 4),
                         "dtype": d.get("dtype"), "roofline_bound": rf.get("bound"),
                         "roofline_frac": rf.get("frac"), "clocks": d.get("clocks"),
                         "args": " ".join(extra)}
            if "sequential" in d:
                out[name]["sequential_ms_per_step"] = round(d["sequential"]["ms_per_step"], 3)
        except Exception as e:  # reported, never fatal for the headline
            out[name] = {"error": f"{type(e).__name__}: {str(e)[:200]}", "args": " ".join(extra)}
    return out


if __name__ == "__main__":
    sys.exit(main())
