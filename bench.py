#!/usr/bin/env python
"""Throughput of the dense state-vector hot path on one or more GB300s.

Workload: the 30-qubit depth-20 random circuit (per layer a Haar-random
single-qubit unitary on every qubit, then CZ on a random matching of the
qubits, seed 1234): 600 single-qubit gates + 300 CZ = 900 gates on a
complex64 state of 8 GiB.  One step = the whole path over that input:
|0...0> initialisation, the 900 gates under the chosen plan, the FP64 norm,
<sum Z> and 10^6 shots sampled from the FP64 prefix of |a|^2.

Metric: gates/s (unfused gate count / step time) and the HBM GB/s of the
step (algorithmic bytes / step time).  The state (8 GiB) is far larger than
L2 (129 MB), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--plan P] [--impl reference]

Multi-GPU: the path does not shard on these one-GPU machines; under torchrun
each rank runs an independent replica of the workload (weak scaling), with a
barrier and the max over ranks of the timed region.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates/s + HBM GB/s at 30 qubits; learned-fused FP32 vs plain per-gate at 1-F≤1e-6"
N_QUBITS, DEPTH, SEED, SHOTS = 30, 20, 1234, 1_000_000
# FP32 arithmetic roofline of this GPU from its unit counts and clock:
# 152 SMs x 128 FP32 FMA lanes x 2 flop x 2.070 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12

# DRAM traffic of a kernel class from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch) as bytes per amplitude, with the SHA-256
# of the kernel's source file at capture time: reported only while that file
# is unchanged.  Captures run a 27-qubit state (1 GiB, 8x the L2; full
# captures stay at a few GB on the device) and the traffic of a launch grows
# with the state, so it is scaled by 2^n.
TRAFFIC = {
    # k_fused_tmem6, 27 qubits: dram__bytes_read.sum 1.073929 GB + dram__bytes_write.sum 1.011859 GB
    "fused_f16": {"bytes_per_amp": (1.073929e9 + 1.011859e9) / 2 ** 27,
                  "sources": [("paper_1805_00988_gb300/csrc/fused.cu",
                               "// ------------------------------------------------------------------ multi-block passes"),
                              ("paper_1805_00988_gb300/csrc/tc_ptx.cuh", None)],
                  "sha256": "b00b0177de2c9b21884416e46f6dc82c58a162dc8016cd6882d0b7ac7fc5687d"},
}


def source_digest(sources):
    """SHA-256 over the kernel sources: each file up to its marker (the device
    code; host code after it does not change a kernel's traffic)."""
    import hashlib
    h = hashlib.sha256()
    for path, until in sources:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), path), "r") as f:
            text = f.read()
        cut = text.find(until) if until else -1
        h.update(text[:cut if cut >= 0 else len(text)].encode())
    return h.hexdigest()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (a timed region ends when the slowest
    rank's does); with one rank, x itself."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank units in `seconds` (the max over ranks)."""
    return world * units_per_rank / seconds


def traffic_for(kind: str, n: int):
    """DRAM bytes of one launch of the kernel class at n qubits, or None
    when the kernel's sources changed since the capture."""
    t = TRAFFIC.get(kind)
    if not t or t["bytes_per_amp"] is None:
        return None, None
    if t["sha256"] is None or source_digest(t["sources"]) != t["sha256"]:
        return None, "kernel source changed since the last ncu capture of its traffic"
    return t["bytes_per_amp"] * 2.0 ** n, "ncu capture of one 27-qubit launch, scaled by 2^(n-27)"


# ---------------------------------------------------------------- the paper's own benchmark (opt-in)
# Algorithm 2 ("Benchmarking algorithm"): for every register size, a number of
# samples, each of a simulator type drawn at random, timing the App. A QFT
# (controlled phases then H, no final swaps) including the register's
# creation, until the device is done (§3, independence by shuffling).  The
# simulator types here are this library's plans and precisions.  Sizes start
# at 1 qubit (the algorithm's loop starts at 0, which is no register).
PAPER_TYPES = ("per_gate_c64", "per_gate_c128", "learned_c64", "staged_c64")


def paper_types(n: int):
    """The types that run an n-qubit register (register tiles need n >= 11)."""
    return [t for t in PAPER_TYPES if t != "staged_c64" or n >= 11]


def paper_sweep_schedule(max_n: int, samples: int, seed: int):
    """(n, type) in run order: n = 1 .. max_n, `samples` runs each, every run's
    type drawn at random from the types that run n qubits."""
    import random
    rng = random.Random(seed)
    return [(n, rng.choice(paper_types(n))) for n in range(1, max_n + 1) for _ in range(samples)]


def summarize_sweep(rows):
    """rows of (type, n, seconds) -> {type: {n: runs, mean / median / min ms}}."""
    out = {}
    for typ, n, sec in rows:
        out.setdefault(typ, {}).setdefault(n, []).append(sec * 1e3)
    return {typ: {str(n): {"runs": len(v), "mean_ms": statistics.fmean(v), "median_ms": statistics.median(v),
                           "min_ms": min(v)} for n, v in sorted(per.items())}
            for typ, per in sorted(out.items())}


def run_paper_sweep(args):
    """One JSON line with the sweep's rows and their summary (rank 0 only)."""
    import torch
    from paper_1805_00988_gb300 import build
    build.build()
    from paper_1805_00988_gb300 import circuits as C
    from paper_1805_00988_gb300 import costmodel, sim
    model, _ = costmodel.load()

    def opts_for(plan, n):
        if plan == "staged":
            return sim.plan_opts("staged", tile_qubits=min(13, n))
        return sim.plan_opts(plan)

    def check(st, n, dt):
        """Outside the timed region: the QFT of |0...0> is the uniform state,
        so the norm is 1 and every |a_j|^2 is 2^-n (complex64: within FP32
        rounding of ~n^2 gates)."""
        nrm = sim.sim_norm(st.h)
        p = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
        sim.sim_probabilities(st.h, p.data_ptr(), sim.SIM_F64)
        dev = float((p - 2.0 ** -n).abs().max().item()) * 2.0 ** n      # relative to 2^-n
        tol = 1e-10 if dt == "c128" else 1e-4
        return {"norm": nrm, "max_rel_dev": dev, "ok": abs(nrm - 1.0) <= tol and dev <= tol}

    def one(n, typ):
        plan, dt = typ.rsplit("_", 1)
        g = sim.to_sim_gates(C.qft_paper(n))
        o = opts_for(plan, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # sim_create allocates the register each run (the device allocation is
        # part of what the paper's script times), not a cached torch tensor
        st = sim.State(n, dt, torch_memory=False)
        if plan == "learned":
            sim.sim_set_cost_model(st.h, model)
        sim.sim_apply_circuit(st.h, g, o)
        sim.sim_synchronize(st.h)
        sec = time.perf_counter() - t0
        chk = check(st, n, dt)
        st.close()
        return sec, chk

    warm = min(12, args.paper_sweep)
    for typ in paper_types(warm):            # one untimed run per type (library and context start-up)
        one(warm, typ)
    rows, rejected = [], []
    for n, typ in paper_sweep_schedule(args.paper_sweep, args.paper_samples, SEED):
        sec, chk = one(n, typ)
        (rows if chk["ok"] else rejected).append((typ, n, sec, chk))
    print(json.dumps({"mode": "paper_qft_sweep", "circuit": "App. A QFT order (no swaps), from |0...0>",
                      "timed": ("wall time: register creation (sim_create, a device allocation each run) + the "
                                "whole QFT + device synchronisation"),
                      "checked": ("after each run, outside the timed region: norm and max |p_j - 2^-n| / 2^-n "
                                  "(uniform output), within 1e-10 (complex128) / 1e-4 (complex64); failing rows "
                                  "are rejected"),
                      "max_qubits": args.paper_sweep, "samples": args.paper_samples, "seed": SEED,
                      "summary": summarize_sweep([(t, n, sec) for t, n, sec, _ in rows]),
                      "rejected": [[t, n, round(sec * 1e3, 4), c] for t, n, sec, c in rejected],
                      "rows": [[t, n, round(sec * 1e3, 4), round(c["max_rel_dev"], 12)] for t, n, sec, c in rows]}))
    return 0


def workload_name(n, depth):
    return "haar_cz: %d qubits, depth %d (Haar U(2) on every qubit + CZ on a random matching per layer)" % (n, depth)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except Exception:
        pass
    return 0.0


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.file.read())) if len(r) >= 9]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_sample(gates, n_target, budget_s, warm_gates=0, one_thread_s=0.0):
    """Time the FP64 oracle gate by gate on this host's cores over a prefix of
    the circuit until budget_s is spent.  Runs at n_target qubits when host
    RAM allows (16 GiB state at 30 qubits), else at 28 qubits with the rate
    scaled by 2^(n - 30) (the oracle's work per gate is proportional to 2^n).
    With one_thread_s > 0 the next gates are then timed on one thread for
    that long (same state); returns that rate too (else None)."""
    import oracle
    n = n_target
    need = (2 ** n) * 16 / 2 ** 30 + 2.0
    while n > 20 and mem_available_gb() < need * 1.3:
        n -= 1
        need = (2 ** n) * 16 / 2 ** 30 + 2.0
    from paper_1805_00988_gb300 import circuits as C
    g = gates if n == n_target else C.haar_cz(n, DEPTH, seed=SEED)
    psi = oracle.basis_state(n, 0)
    for k in range(warm_gates):
        oracle.apply_circuit(psi, g[k:k + 1], inplace=True)
    done, t0 = 0, time.perf_counter()
    k = warm_gates
    while True:
        oracle.apply_circuit(psi, g[k % len(g):k % len(g) + 1], inplace=True)
        done += 1
        k += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= len(g):
            break
    rate = done / el * (2.0 ** (n - n_target))
    threads = oracle.num_threads()
    sample = "first %d gates of the %d-qubit circuit, FP64 oracle, %d host threads" % (done, n, threads)
    if n != n_target:
        sample += ", rate scaled by 2^(%d-%d) to %d qubits (host RAM %.0f GB free)" % (
            n, n_target, n_target, mem_available_gb())
    one = None
    if one_thread_s > 0:
        oracle.set_num_threads(1)
        try:
            d1, t1 = 0, time.perf_counter()
            while True:
                oracle.apply_circuit(psi, g[k % len(g):k % len(g) + 1], inplace=True)
                d1 += 1
                k += 1
                e1 = time.perf_counter() - t1
                if e1 >= one_thread_s or d1 >= len(g):
                    break
        finally:
            oracle.set_num_threads(threads)
        one = {"value": d1 / e1 * (2.0 ** (n - n_target)), "unit": "gates/s", "cores": 1,
               "sample": "gates %d..%d of the %d-qubit circuit on one host thread (%.1f s)" % (
                   k - d1, k - 1, n, e1)}
    return rate, sample, threads, done, el, one


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1805_00988_gb300 import circuits as C
    gates = C.haar_cz(N_QUBITS, DEPTH, seed=SEED)
    per_step = float(os.environ.get("QSIM_REF_STEP_SECONDS", "6"))
    rates = []
    info = None
    for i in range(args.warmup + args.steps):
        rate, sample, cores, done, el, _ = oracle_sample(gates, N_QUBITS, per_step, warm_gates=0)
        if i >= args.warmup:
            rates.append(rate)
            info = (sample, cores, done, el)
    v = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "gates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 900.0 / v * 1e3,
            "extrapolated_from_gates": info[2],
            "extrapolation": ("each step times the first %d of the 900 gates (%.1f s of CPU work); value is that "
                              "rate and ms_per_step = 900 gates at that rate" % (info[2], info[3])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(N_QUBITS, DEPTH), "n_qubits": N_QUBITS,
                                            "depth": DEPTH, "gates": 900, "state": "complex128 (host)"},
            "cpu_baseline": {"value": v, "unit": "gates/s", "cores": info[1], "kind": "oracle", "sample": info[0]},
            "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg
def load_cost_model(sim):
    """The plan cost model trained on this machine's GB300 (parameters shipped
    with the package); None when absent (the learned plan then falls back to
    the greedy fixed-k plan)."""
    from paper_1805_00988_gb300 import costmodel
    if not os.path.exists(costmodel.DEFAULT_PATH):
        return None, {"cost_model": "absent: greedy fixed-k plan used"}
    m, info = costmodel.load()
    return m, {"cost_model": info}


def infidelity_torch(a, b, chunk=1 << 26):
    """1 - |<a|b>|^2 / (<a|a><b|b>) in FP64 over two CUDA tensors (chunked)."""
    import torch
    ip = torch.zeros((), dtype=torch.complex128, device=a.device)
    na = torch.zeros((), dtype=torch.float64, device=a.device)
    nb = torch.zeros((), dtype=torch.float64, device=a.device)
    for o in range(0, a.numel(), chunk):
        x = a[o:o + chunk].to(torch.complex128)
        y = b[o:o + chunk].to(torch.complex128)
        ip += torch.vdot(x, y)
        na += torch.vdot(x, x).real
        nb += torch.vdot(y, y).real
    return float(1.0 - (ip.abs() ** 2) / (na * nb))


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1805_00988_gb300 import build
    build.build()
    from paper_1805_00988_gb300 import circuits as C
    from paper_1805_00988_gb300 import sim

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    def barrier():
        if world > 1:
            dist.barrier()

    n, depth, shots = args.qubits, args.depth, args.shots
    gates = C.haar_cz(n, depth, seed=SEED)
    sg = sim.to_sim_gates(gates)
    plan = args.plan
    opts = sim.plan_opts(plan, fuse_k=args.fuse_k, tile_qubits=args.tile)
    st = sim.State(n, "c64", device=dev)
    stream = st.stream
    model, model_info = load_cost_model(sim)
    if model is not None:
        sim.sim_set_cost_model(st.h, model)
    shot_buf = torch.empty(shots, dtype=torch.int64, device=dev)

    def step():
        sim.sim_set_basis_state(st.h, 0)
        sim.sim_apply_circuit(st.h, sg, opts)
        # 10^6 shots, the FP64 norm and <sum Z>: one pass over the state gives
        # the sampler's sub-block sums, their total and the weighted sum
        _, nrm, ez = sim.sim_sample_observe(st.h, shots, 99, shot_buf.data_ptr(), out_on_device=True)
        return nrm, ez

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clk = ClockSampler(vis.split(",")[local_rank] if vis else str(local_rank))
    sim.sim_profile_read(st.h, reset=True)
    sim.sim_profile_enable(st.h, True)
    l0 = sim.sim_launch_count(st.h)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        nrm, ez = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    launches = sim.sim_launch_count(st.h) - l0
    prof = sim.sim_profile_read(st.h, reset=True)
    sim.sim_profile_enable(st.h, False)
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps
    gates_per_s = job_rate(len(gates), world, ms_per_step / 1e3)
    step_bytes = sum(v[2] for v in prof.values()) / args.steps
    peaks, peak_kind = load_peaks()

    # roofline: the kernel class with the largest device time
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms, dbytes, dflops) = dom
    sec = dms / dl / 1e3                                   # average launch duration
    gbs = (dbytes / dl) / sec / 1e9
    tflops = (dflops / dl) / sec / 1e12
    hbm_frac = gbs / peaks["hbm_gbs"]
    if dname in ("fused", "fused_multi"):
        # tensor-core TF32 work: the measured sustained bf16 peak scaled by the
        # nominal TF32 / bf16 dense ratio (1.1 / 2.25 PFLOP/s)
        cpeak = peaks.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
        cbound, csrc = "tensor", "MEASURED_PEAKS.json bf16_tflops_sustained x (1.1 / 2.25) nominal TF32/bf16"
    elif dname == "fused_f16":
        # tensor-core FP16 work (kind::f16): the dense FP16 rate is the bf16 rate
        cpeak = peaks.get("bf16_tflops_sustained", 1700.0)
        cbound, csrc = "tensor", "MEASURED_PEAKS.json bf16_tflops_sustained (FP16 dense = bf16 dense rate)"
    else:
        cpeak = FP32_PEAK_TFLOPS
        cbound, csrc = "alu", "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz"
    cfrac = tflops / cpeak
    if cfrac > hbm_frac:
        # the binding resource is arithmetic (register 2x2 updates or tensor-core GEMMs)
        roofline = {"kernel": dname, "bound": cbound, "achieved": tflops, "peak": cpeak,
                    "unit": "TFLOP/s", "frac": cfrac, "traffic": None, "peak_source": csrc,
                    "alg_flops_per_launch": dflops / dl, "hbm": {"achieved_GBps": gbs, "peak_GBps": peaks["hbm_gbs"],
                                                                "frac": hbm_frac}}
    else:
        roofline = {"kernel": dname, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": hbm_frac, "traffic": None,
                    "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs, copy)" if peak_kind == "measured"
                                    else "fallback 6.8 TB/s"),
                    "compute": {"bound": cbound, "achieved_TFLOPs": tflops, "peak_TFLOPs": cpeak, "frac": cfrac,
                                "peak_source": csrc}}
    traffic, tsrc = traffic_for(dname, n)
    roofline["traffic"] = traffic
    if tsrc:
        roofline["traffic_source"] = tsrc
    roofline.update({"alg_bytes_per_launch": dbytes / dl, "avg_launch_ms": dms / dl, "launches": dl,
                     "timed_with": "CUDA events around every launch on the handle's stream, timed region"})
    kernels = {k: {"launches": v[0], "ms": v[1], "alg_GBps": (v[2] / (v[1] / 1e3) / 1e9) if v[1] > 0 else None,
                   "alg_TFLOPs": (v[3] / (v[1] / 1e3) / 1e12) if v[1] > 0 else None}
               for k, v in prof.items()}

    # end to end through the public API with host buffers
    host_gates = torch.empty(sg.nbytes, dtype=torch.uint8, pin_memory=True)
    hg = host_gates.numpy().view(sim.SIM_GATE_DTYPE)
    hg[:] = sg
    host_shots = torch.empty(shots, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.sim_set_basis_state(st.h, 0)
        sim.sim_apply_circuit(st.h, hg, opts)
        sim.sim_sample_observe(st.h, shots, 99, out=host_shots)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": job_rate(len(gates), world, e2e_s), "unit": "gates/s", "h2d_bytes_per_step": int(sg.nbytes),
           "d2h_bytes_per_step": int(shots * 8 + 16)}

    line = {"metric": METRIC, "value": gates_per_s, "unit": "gates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Haar/CZ circuit)",
            "precision": ("complex64 state (FP32 pairs); fused blocks: unitaries built in FP64, applied as "
                          "split-precision tensor-core GEMMs with FP32 accumulation (k = 6: FP16 hi / lo parts "
                          "of power-of-two-scaled operands, 22 significant bits per operand; k <= 5: 3xTF32); "
                          "norm, <sum Z> and the sampling prefix accumulated in FP64"),
            "config": {"workload": workload_name(n, depth), "n_qubits": n, "depth": depth,
                       "gates": int(len(gates)), "state": "complex64", "plan": plan, "tile_qubits": args.tile,
                       "shots": shots,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (%.3g GiB state vs 129 MB L2); no flush" % (2.0 ** n * 8 / 2 ** 30)},
            "hbm_gbs": world * step_bytes / (ms_per_step / 1e3) / 1e9,
            "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e, "roofline": roofline,
            "kernels": kernels, "norm": nrm, "expect_z_sum": ez}
    line["config"].update(model_info if plan == "learned" else {})
    if plan == "learned":
        line["config"]["learned_windows"] = [sim.VARIANTS[v] for v in sim.sim_last_plan(st.h)]

    # plan variants on the same workload, each with its infidelity
    if args.variants and rank == 0:
        line["variants"] = run_variants(args, sim, C, gates, sg, dev, st, peaks)

    if args.extras and rank == 0:
        st.close()
        st = None
        line["extras"] = run_extras(args, sim, C, dev, model)

    if rank == 0 and world == 1 and args.cpu_baseline:
        rate, sample, cores, done, el, one = oracle_sample(gates, n, args.cpu_seconds,
                                                           one_thread_s=args.cpu_seconds / 2)
        line["cpu_baseline"] = {"value": rate, "unit": "gates/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "seconds": el, "one_thread": one}
    if st is not None:
        st.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_variants(args, sim, C, gates, sg, dev, st_c64, peaks):
    """Each plan once warm, timed once or twice; infidelity of every complex64
    result against the complex128 per-gate state of the same circuit (the
    full-size parity test checks that state against the FP64 oracle's own
    30-qubit run: infidelity <= 1e-12)."""
    import torch
    out = {}
    stream = st_c64.stream

    def timed(st, opts, reps):
        sim.sim_set_basis_state(st.h, 0)
        sim.sim_apply_circuit(st.h, sg, opts)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            sim.sim_set_basis_state(st.h, 0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st.stream)
            sim.sim_apply_circuit(st.h, sg, opts)
            e1.record(st.stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    ref = sim.State(args.qubits, "c128", device=dev)
    t128 = timed(ref, sim.plan_opts("per_gate"), 1)
    out["per_gate_c128"] = {"ms": t128, "gates_per_s": len(gates) / (t128 / 1e3), "infidelity": 0.0,
                            "note": ("reference state for the complex64 infidelities (equal to the FP64 oracle's "
                                     "state within 1e-12 infidelity at 30 qubits: tests/test_fullsize.py)")}
    # complex128 through the tensor cores: 4-qubit fused blocks of exact
    # integer digit products (what the learned plan runs for complex128)
    st128 = sim.State(args.qubits, "c128", device=dev)
    try:
        t = timed(st128, sim.plan_opts("fused", fuse_k=4), 2)
        out["fused:4_c128"] = {"ms": t, "gates_per_s": len(gates) / (t / 1e3),
                               "infidelity": infidelity_torch(st128.tensor, ref.tensor),
                               "max_abs_diff": float((st128.tensor - ref.tensor).abs().max().item()),
                               "speedup_vs_per_gate_c128": t128 / t}
    except sim.SimError as e:
        out["fused:4_c128"] = {"error": str(e)}
    st128.close()
    for spec in args.variant_plans:
        plan, _, num = spec.partition(":")
        try:
            if plan == "fused":
                opts = sim.plan_opts(plan, fuse_k=int(num or args.fuse_k))
            else:
                opts = sim.plan_opts(plan, fuse_k=args.fuse_k, tile_qubits=int(num or 0))
            t = timed(st_c64, opts, 2)
            inf = infidelity_torch(st_c64.tensor, ref.tensor)
            out[spec + "_c64"] = {"ms": t, "gates_per_s": len(gates) / (t / 1e3), "infidelity": inf}
        except sim.SimError as e:
            out[spec + "_c64"] = {"error": str(e)}
    ref.close()
    return out


def _timed(fn, stream, reps):
    import torch
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best


def run_extras(args, sim, C, dev, model):
    """The other workloads of the hot path, one line each (device time, best
    of a few runs after a warm run)."""
    import torch
    out = {}
    # the paper's benchmark circuit: QFT at 28 qubits from a random basis state, per-gate kernels
    n = 28
    j = C.random_basis_index(n, seed=SEED)
    g = sim.to_sim_gates(C.qft(n))
    for dt in ("c64", "c128"):
        st = sim.State(n, dt, device=dev)
        res = {}
        plans = [("per_gate", sim.plan_opts("per_gate")), ("staged", sim.plan_opts("staged"))]
        if dt == "c128":
            plans.append(("fused:4", sim.plan_opts("fused", fuse_k=4)))
        for plan, o in plans:

            def run():
                sim.sim_set_basis_state(st.h, j)
                sim.sim_apply_circuit(st.h, g, o)
            run()
            ms = _timed(run, st.stream, 2)
            res[plan] = {"ms": ms, "gates_per_s": len(g) / (ms / 1e3)}
        out["qft28_" + dt] = res
        st.close()
    # launch-bound small register: 14 qubits, complex128, 20 layers of U3 on
    # every qubit + a CNOT ladder (540 gates, a 256 KiB state that stays in L2)
    n = 14
    g = sim.to_sim_gates(C.u3_cnot_ladder(n, 20, seed=SEED))
    st = sim.State(n, "c128", device=dev)
    res = {}
    for plan in ("per_gate", "staged"):
        o = sim.plan_opts(plan)

        def run():
            sim.sim_set_basis_state(st.h, 0)
            sim.sim_apply_circuit(st.h, g, o)
        run()
        ms = _timed(run, st.stream, 5)
        res[plan] = {"ms": ms, "gates_per_s": len(g) / (ms / 1e3)}
    out["u3_cnot_ladder_14q_c128"] = res
    st.close()
    # one launch per gate kind at 30 qubits (complex64): device time against the
    # algorithmic bytes of the pairs it must touch (S = state bytes): dense 2S,
    # CNOT S (control = 1 pairs), Toffoli S/2, CZ S/2 (the |11> quarter, read +
    # write), SWAP S (the |01>, |10> halves' quarter each, read + write); then a
    # single-qubit measurement (FP64 sum of one half + collapse pass)
    n = 30
    st = sim.State(n, "c64", device=dev)
    S = (2 ** n) * 8.0
    peaks, _ = load_peaks()
    kinds = {"dense_H": (C.gate("h", 17), 2 * S)}
    # permutation and phase gates with the low qubit at 3, 8, 17 (target 12) and 25:
    # a low qubit cuts the touched part of the state into runs of 2^q amplitudes
    for c in (3, 8, 17, 25):
        t = 12 if c == 17 else 17
        kinds["cnot_c%d" % c] = (C.gate("x", t, controls=(c,)), S)
        kinds["cz_c%d" % c] = (C.gate("z", t, controls=(c,)), S / 2)
        kinds["swap_%d" % c] = (C.gate("swap", t, target2=c), S)
        kinds["toffoli_c%d" % c] = (C.gate("x", t, controls=(c, 29 if c != 25 else 27)), S / 2)
    res = {}
    for name, (gate, alg) in kinds.items():
        sg = sim.to_sim_gates(gate)
        o = sim.plan_opts("per_gate")

        def run():
            for _ in range(4):
                sim.sim_apply_circuit(st.h, sg, o)
        run()
        ms = _timed(run, st.stream, 3) / 4
        gbs = alg / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "alg_GBps": gbs, "frac_of_copy_peak": gbs / peaks["hbm_gbs"]}
    sim.sim_set_basis_state(st.h, 0)
    sim.sim_apply_circuit(st.h, sim.to_sim_gates(C.concat([C.gate("h", q) for q in range(n)])), sim.plan_opts("staged"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m, p = sim.sim_measure(st.h, 11, seed=5, draw=0)
    torch.cuda.synchronize()
    res["measure_qubit"] = {"ms_wall": (time.perf_counter() - t0) * 1e3, "outcome": m, "probability": p,
                            "note": "FP64 sum over the state + collapse pass, host round trip included"}
    out["gate_kernels_30q_c64"] = res
    st.close()
    # batched variational circuits: 4096 circuits of 8..20 qubits, 4..12 layers, one graph launch;
    # tile size and CTAs per SM from the autotuner (tuned here unless cached)
    from paper_1805_00988_gb300 import autotune
    ns, offs, bg = C.variational(4096, 8, 20, 4, 12, seed=SEED)
    wl = "variational4096_8-20q_4-12l_seed%d" % SEED
    cached = autotune.batch_opts(wl)
    tuned = None
    if cached is None:
        tuned = autotune.tune_batch(ns, offs, bg, wl, reps=2)
        cached = (tuned["tile_qubits"], tuned["ctas_per_sm"])
    t0 = time.perf_counter()
    b = sim.Batch(ns, offs, bg, tile_qubits=cached[0], ctas_per_sm=cached[1])
    plan_s = time.perf_counter() - t0
    b.run()
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        b.run()
        ts.append(time.perf_counter() - t0)
    info, cfg = b.info(), b.config()
    b.close()
    tb = min(ts)
    fl_peak = FP32_PEAK_TFLOPS
    out["batched_4096"] = {"ms": tb * 1e3, "circuits_per_s": 4096 / tb, "gates_per_s": len(bg) / tb,
                           "gates": int(len(bg)), "host_plan_s": plan_s, "work_items": info["items"],
                           "persistent_ctas": info["grid"], "tile_qubits": cfg["tile_qubits"],
                           "ctas_per_sm": cfg["ctas_per_sm"],
                           "autotune": tuned["all"] if tuned else "cached",
                           "roofline": {"bound": "alu", "achieved": cfg["alg_flops"] / tb / 1e12, "peak": fl_peak,
                                        "unit": "TFLOP/s", "frac": cfg["alg_flops"] / tb / 1e12 / fl_peak,
                                        "alg_flops": cfg["alg_flops"],
                                        "peak_source": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz",
                                        "hbm": {"alg_scratch_bytes": cfg["alg_scratch_bytes"],
                                                "achieved_GBps": cfg["alg_scratch_bytes"] / tb / 1e9,
                                                "frac": cfg["alg_scratch_bytes"] / tb / 1e9 / peaks["hbm_gbs"]}},
                           "note": "wall time of sim_batch_run (graph launch + readback of 4096 <sum Z> values)"}
    # the learned plan on held-out mixed circuits (stretches of different circuit families) at
    # register sizes where the best plan changes, against every fixed variant
    from paper_1805_00988_gb300 import costmodel
    mixes = (("haar", "graph", "haar", "graph"), ("graph", "qft", "haar"), ("rev", "phase", "ladder", "graph"))
    rows = []
    for n in (18, 22, 26, 28):
        st = sim.State(n, "c64", device=dev)
        sim.sim_set_cost_model(st.h, model)
        W = costmodel.window_size(n)
        for i, kinds in enumerate(mixes):
            sgm = sim.to_sim_gates(C.segments(n, kinds, 2 * W, seed=900 + i))
            r = {"n": n, "circuit": "+".join(kinds), "gates": len(sgm),
                 "learned": costmodel.time_window(st, sgm, sim.plan_opts("learned"), 3),
                 "learned_plan": [sim.VARIANTS[int(v)] for v in sim.sim_last_plan(st.h)]}
            for v in range(sim.N_VARIANTS):
                r[sim.VARIANTS[v]] = costmodel.time_window(st, sgm, sim.variant_opts(v), 3)
            rows.append(r)
        st.close()
    names = list(sim.VARIANTS)
    out["learned_vs_fixed_heldout"] = {
        "unit": "ms (median of 3, CUDA events)", "rows": rows,
        "geomean_learned_over_fixed": {v: float(np.exp(np.mean([np.log(r["learned"] / r[v]) for r in rows])))
                                       for v in names},
        "geomean_learned_over_best_fixed": float(np.exp(np.mean([np.log(r["learned"] / min(r[v] for v in names))
                                                                 for r in rows])))}
    # density matrix of 15 qubits (a 30-qubit register, 8 GiB complex64): the 30-qubit workload's
    # gate distribution at depth 20, each layer followed by depolarizing (1e-3) and amplitude
    # damping (2e-3) on every qubit; gates as G rho G^dagger on the register, one pass per channel
    nd = 15
    gd = C.noisy_haar_cz(nd, 20, seed=SEED)
    is_ch = np.isin(gd["name"], C.CHANNEL_NAMES)
    rho = sim.DensityMatrix(nd, "c64", device=dev)
    sgd = sim.to_sim_gates(gd)
    res = {"gates": int(np.count_nonzero(~is_ch)), "channels": int(np.count_nonzero(is_ch))}
    for name, o in (("per_gate", sim.plan_opts("per_gate")), ("fused:6", sim.plan_opts("fused", fuse_k=6)),
                    ("learned", sim.plan_opts("learned"))):
        if name == "learned":
            sim.sim_set_cost_model(rho.h, model)

        def run():
            rho.set_basis(0)
            sim.sim_dm_apply_circuit(rho.h, sgd, o)
        run()
        sim.sim_profile_enable(rho.h, True)
        ms = _timed(run, rho.stream, 1)
        prof = sim.sim_profile_read(rho.h)
        sim.sim_profile_enable(rho.h, False)
        r = {"ms": ms, "ops_per_s": len(gd) / (ms / 1e3)}
        if "channel" in prof:
            cl, cms, cb, _ = prof["channel"]
            r["channel_passes"] = cl
            r["channel_ms"] = cms
            r["channel_alg_GBps"] = cb / (cms / 1e3) / 1e9
            r["channel_frac_of_copy_peak"] = r["channel_alg_GBps"] / peaks["hbm_gbs"]
        res[name] = r
    res["trace"] = rho.trace()
    res["purity"] = rho.purity()
    res["note"] = "15-qubit density matrix, complex64; ops = gates + channels; best of 1 after a warm run"
    out["noisy_haar_cz_15q_density"] = res
    rho.close()
    # 33 qubits, depth 24 (64 GiB complex64): learned plan vs greedy register tiles and greedy fixed-k fused blocks, then 10^6 shots
    if args.c5:
        n5 = 33
        g5 = sim.to_sim_gates(C.haar_cz(n5, 24, seed=SEED))
        st = sim.State(n5, "c64", device=dev)
        res = {}
        for name, o in (("greedy_staged13", sim.plan_opts("staged", tile_qubits=13)),
                        ("greedy_fused5", sim.plan_opts("fused", fuse_k=5)),
                        ("greedy_fused6", sim.plan_opts("fused", fuse_k=6)),
                        ("learned", sim.plan_opts("learned"))):
            if name == "learned":
                sim.sim_set_cost_model(st.h, model)

            def run():
                sim.sim_set_basis_state(st.h, 0)
                sim.sim_apply_circuit(st.h, g5, o)
            run()
            ms = _timed(run, st.stream, 1)
            res[name] = {"ms": ms, "gates_per_s": len(g5) / (ms / 1e3)}
        res["learned"]["windows"] = [sim.VARIANTS[v] for v in sim.sim_last_plan(st.h)]
        shots = torch.empty(1_000_000, dtype=torch.int64, device=dev)
        ms = _timed(lambda: sim.sim_sample(st.h, 1_000_000, 7, shots.data_ptr(), out_on_device=True), st.stream, 2)
        res["sample_1e6_shots_ms"] = ms
        res["norm"] = st.norm2()
        out["haar_cz_33q_depth24"] = res
        st.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plan", default="learned")
    ap.add_argument("--fuse-k", type=int, default=5)
    ap.add_argument("--tile", type=int, default=0, help="tile qubits of the staged plan (0 = library default)")
    ap.add_argument("--qubits", type=int, default=N_QUBITS)
    ap.add_argument("--depth", type=int, default=DEPTH)
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--variant-plans", default="per_gate,staged:13,fused:4,fused:5,fused:6,learned")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-c5", dest="c5", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--paper-sweep", type=int, default=0,
                    help="instead of the timed step: the paper's QFT sweep up to this many qubits (rank 0)")
    ap.add_argument("--paper-samples", type=int, default=5)
    args = ap.parse_args()
    args.variant_plans = [p for p in args.variant_plans.split(",") if p]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.paper_sweep > 0:
        return run_paper_sweep(args) if rank == 0 else 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
