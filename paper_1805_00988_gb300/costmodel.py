"""Training of the plan cost model on timings the simulator itself produces.

``collect`` cuts circuits of several families into the windows the learned
plan uses, runs every window under every feasible plan variant on the GPU
(CUDA events, median of repeats) and records the library's feature row for
it; the target is log(milliseconds per 2^30 amplitudes) -- the time scaled
to a 30-qubit state, so that a register a few qubits larger than any timed
one is predicted from the per-amplitude cost the model has seen.  ``train`` fits the MLP with the
library's own kernels (sim_mlp_train); ``save`` / ``load`` keep the
parameters as JSON.  Everything here drives the C ABI; no simulation
arithmetic happens in Python.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import circuits as C
from . import sim

HIDDEN = 64
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_params.json")


def window_size(n: int) -> int:
    """Gates per window of the learned plan (matches the library)."""
    return max(64, 8 * n)


def families(n: int, seed: int):
    rng = np.random.default_rng(seed)
    yield "haar_cz", C.haar_cz(n, 16, seed=seed)
    yield "qft", C.qft(n)
    yield "u3_ladder", C.u3_cnot_ladder(n, 8, seed=seed)
    yield "variational", C.variational_layered(n, 8, rng)
    yield "random", C.random_gates(n, 12 * n, seed=seed)
    yield "phase", C.phase_polynomial(n, 12 * n, seed=seed)
    yield "reversible", C.reversible(n, 12 * n, seed=seed)
    yield "graph", C.graph_state(n, 12 * n, seed=seed)


def time_window(st, sg, opts, reps: int) -> float:
    import torch
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st.stream)
        sim.sim_apply_circuit(st.h, sg, opts)
        e1.record(st.stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def target(ms: float, n: int) -> float:
    """The regression target: log of the time scaled to 2^30 amplitudes."""
    return math.log(max(ms, 1e-4)) - (n - 30) * math.log(2.0)


def collect(n_list=(24, 26, 28), reps: int = 3, seed: int = 7, max_windows: int = 6, log=None):
    """Returns X (rows x features, float32), T (``target``, float32), meta.

    Rows: every window of the first ``max_windows`` of each family's circuit
    under every feasible variant, and the span of all those windows as one
    segment under every variant but per-gate (the learned plan compares the
    per-window choice with one variant over the whole circuit)."""
    X, T, meta = [], [], []

    def row(st, n, fam, w0, seg, v):
        f = sim.sim_plan_features(n, sim.SIM_C64, seg, v)
        if f is None:
            return
        ms = time_window(st, seg, sim.variant_opts(v), reps)
        X.append(f)
        T.append(target(ms, n))
        meta.append((n, fam, w0, v, ms))
        if log:
            log("n=%d %-11s w0=%4d len=%5d %-9s %.3f ms" % (n, fam, w0, len(seg), sim.VARIANTS[v], ms))

    for n in n_list:
        st = sim.State(n, "c64")
        for fam, g in families(n, seed + n):
            sg = sim.to_sim_gates(g)
            W = window_size(n)
            span = min(len(sg), W * max_windows)
            for w0 in range(0, span, W):
                for v in range(sim.N_VARIANTS):
                    row(st, n, fam, w0, sg[w0:w0 + W], v)
            if span > W:
                for v in range(1, sim.N_VARIANTS):
                    row(st, n, fam, -1, sg[:span], v)
        st.close()
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32), meta


def init_params(seed: int, d_in: int = sim.N_FEATURES, hidden: int = HIDDEN) -> np.ndarray:
    """He-normal weights, zero biases, in the library's parameter order."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((d_in, hidden)).ravel() * math.sqrt(2.0 / d_in), np.zeros(hidden),
             rng.standard_normal((hidden, hidden)).ravel() * math.sqrt(2.0 / hidden), np.zeros(hidden),
             rng.standard_normal((hidden, 1)).ravel() * math.sqrt(2.0 / hidden), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(X, T, steps: int = 3000, lr: float = 3e-3, seed: int = 11, model=None):
    m = model or sim.MLP(sim.N_FEATURES, HIDDEN)
    m.set_params(init_params(seed))
    loss = m.train(X, T, steps=steps, lr=lr)
    return m, loss


def save(model, path: str = DEFAULT_PATH, info=None):
    with open(path, "w") as f:
        json.dump({"d_in": model.d_in, "hidden": model.hidden, "params": model.get_params().tolist(),
                   "info": info or {}}, f)


def load(path: str = DEFAULT_PATH):
    with open(path) as f:
        d = json.load(f)
    m = sim.MLP(d["d_in"], d["hidden"])
    m.set_params(np.array(d["params"], dtype=np.float32))
    return m, d.get("info", {})


def main(argv=None):
    import argparse
    import time
    ap = argparse.ArgumentParser(description="collect timings on this GPU and train the plan cost model")
    ap.add_argument("--n", default="26,28,30,32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--windows", type=int, default=6)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=DEFAULT_PATH)
    a = ap.parse_args(argv)
    t0 = time.time()
    X, T, meta = collect(tuple(int(v) for v in a.n.split(",")), reps=a.reps, max_windows=a.windows,
                         log=lambda s: print(s, flush=True))
    t1 = time.time()
    m, loss = train(X, T, steps=a.steps)
    pred = m.forward(X)
    rmse = float(np.sqrt(np.mean((pred - T) ** 2)))
    import torch
    info = {"rows": int(len(X)), "n": a.n, "train_mse": float(loss), "rmse_log_ms": rmse,
            "collect_s": t1 - t0, "gpu": torch.cuda.get_device_name(0)}
    save(m, a.out, info)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
