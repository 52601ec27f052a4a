"""Autotuner for plan variants and tile sizes.

``tune(n, dtype, gates)`` times every feasible variant (per-gate, staged with
11/12/13-qubit tiles, fused with k = 3..6) of a circuit on this GPU with CUDA
events (best of ``reps`` after a warm run) and returns the fastest; results
are cached in a JSON file keyed by "n/dtype/workload".  ``best_opts`` reads
the cache.  ``tune_batch`` does the same for a batch of small circuits: the
persistent kernel's register-tile size (11, 12 or 13 qubits) and its CTAs
per SM; ``batch_opts`` reads that choice back for sim.Batch.  Timing only:
the library does all the work through the C ABI.
"""
from __future__ import annotations

import json
import os

from . import sim

CACHE = os.environ.get("QSIM_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "qsim_gb300", "autotune.json"))

CANDIDATES = [("per_gate", {}), ("staged", {"tile_qubits": 11}), ("staged", {"tile_qubits": 12}),
              ("staged", {"tile_qubits": 13}), ("fused", {"fuse_k": 3}), ("fused", {"fuse_k": 4}),
              ("fused", {"fuse_k": 5}), ("fused", {"fuse_k": 6})]


def feasible(n: int, dtype: str, plan: str, kw: dict) -> bool:
    if plan == "staged":
        t = kw["tile_qubits"]
        return n >= t and (dtype == "c64" or t <= 12)
    if plan == "fused":
        return dtype == "c64" and n >= kw["fuse_k"] + 7
    return True


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def key(n: int, dtype: str, workload: str) -> str:
    return "%d/%s/%s" % (n, dtype, workload)


def tune(n: int, dtype: str, gates, workload: str, reps: int = 3, start_basis: int = 0):
    """Time all feasible candidates; cache and return {"plan", "opts", "ms", "all"}."""
    import torch
    sg = sim.to_sim_gates(gates)
    st = sim.State(n, dtype)
    times = {}
    for plan, kw in CANDIDATES:
        if not feasible(n, dtype, plan, kw):
            continue
        o = sim.plan_opts(plan, **kw)
        best = None
        for r in range(reps + 1):
            sim.sim_set_basis_state(st.h, start_basis)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st.stream)
            sim.sim_apply_circuit(st.h, sg, o)
            e1.record(st.stream)
            e1.synchronize()
            if r > 0:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        times[plan + (":%d" % list(kw.values())[0] if kw else "")] = best
    st.close()
    win = min(times, key=times.get)
    plan, _, num = win.partition(":")
    opts = {"plan": plan}
    if plan == "staged":
        opts["tile_qubits"] = int(num)
    elif plan == "fused":
        opts["fuse_k"] = int(num)
    res = {"plan": plan, "opts": opts, "ms": times[win], "all": times}
    d = _load()
    d[key(n, dtype, workload)] = res
    _store(d)
    return res


BATCH_TILES = (11, 12, 13)


def tune_batch(n_qubits, offsets, gates, workload: str, reps: int = 3, tiles=BATCH_TILES):
    """Time one batch of circuits (sim_batch_run wall time, best of ``reps``
    after a warm run) under every tile size and every CTA count per SM that
    fits; cache and return {"tile_qubits", "ctas_per_sm", "ms", "all"}."""
    import time
    times = {}
    for m in tiles:
        per_sm = 1
        while True:
            try:
                b = sim.Batch(n_qubits, offsets, gates, tile_qubits=m, ctas_per_sm=per_sm)
            except sim.SimError:
                break                      # more CTAs than fit on an SM
            b.run()
            best = None
            for _ in range(reps):
                t0 = time.perf_counter()
                b.run()
                t = (time.perf_counter() - t0) * 1e3
                best = t if best is None else min(best, t)
            b.close()
            times["%d/%d" % (m, per_sm)] = best
            per_sm += 1
    win = min(times, key=times.get)
    m, per_sm = (int(x) for x in win.split("/"))
    res = {"tile_qubits": m, "ctas_per_sm": per_sm, "ms": times[win], "all": times}
    d = _load()
    d["batch/" + workload] = res
    _store(d)
    return res


def batch_opts(workload: str):
    """Cached (tile_qubits, ctas_per_sm) of a batch workload, or None."""
    r = _load().get("batch/" + workload)
    return (r["tile_qubits"], r["ctas_per_sm"]) if r else None


def best_opts(n: int, dtype: str, workload: str):
    """Cached sim_plan_opts for (n, dtype, workload), or None."""
    r = _load().get(key(n, dtype, workload))
    if not r:
        return None
    o = dict(r["opts"])
    return sim.plan_opts(o.pop("plan"), **o)
