"""Seeded synthetic circuit and state generators.

This module only *describes* inputs: gate lists (name, qubits, angles or an
explicit 2x2 matrix), basis indices and random states.  It holds none of the
simulation arithmetic (no gate matrices for named gates, no state updates);
the CUDA library and the CPU oracle each turn a gate record into a matrix on
their own.  Both sides consume the same arrays, so their parity never depends
on matching random-number streams.

Gate records use ``GATE_DTYPE``:

    name     gate name: x y z h s sdg t tdg rx ry rz p u3 u swap
    target   target qubit (qubit t is bit t of the amplitude index)
    target2  second qubit of a swap, else -1
    nctrl    number of control qubits (0..2); the update applies only where
             every control bit is 1 (the controlled gate of §2.3)
    ctrl     control qubits (unused slots -1)
    params   angles (theta, phi, lambda) for rx/ry/rz/p/u3
    mat      explicit 2x2 matrix [[A, B], [C, D]] as (re, im) pairs, name 'u'

Noise channels (density matrices only) use the same records: name one of
``CHANNEL_NAMES`` (dep = depolarizing, adamp = amplitude damping, pdamp =
phase damping, bflip = bit flip, pflip = phase flip), the qubit in target and
the channel's parameter in params[0].

Workloads (sizes and distributions of the paper's QFT benchmark, App. A, and
of the dense random / variational circuits the simulator is measured on):

    u3_cnot_ladder   layers of U3 on every qubit then a CNOT ladder
    qft              textbook QFT (H + controlled phase, then qubit reversal)
    qft_paper        the App. A benchmark ordering (no final swaps)
    haar_cz          layers of Haar-random 1q unitaries + CZ on a random matching
    phase_polynomial diagonal gates only (controlled phases, RZ, P, T, S, Z)
    reversible       permutation gates only (X, CNOT, Toffoli, SWAP)
    graph_state      H on every qubit, then CZ on random edges (cluster states)
    segments         consecutive stretches of the above (mixed circuits)
    variational      batched RY/RZ layers + CZ ring, uneven qubit counts
    bernstein_vazirani   the App. C worked example
    noisy            layers of a circuit, each followed by channels on every qubit
    random_noisy     random gates with random channels in between (parity sweeps)
"""
from __future__ import annotations

import math

import numpy as np

GATE_DTYPE = np.dtype([
    ("name", "U5"),
    ("target", "<i4"),
    ("target2", "<i4"),
    ("nctrl", "<i4"),
    ("ctrl", "<i4", (2,)),
    ("params", "<f8", (3,)),
    ("mat", "<f8", (8,)),
])

GATE_NAMES = ("u", "x", "y", "z", "h", "s", "sdg", "t", "tdg",
              "rx", "ry", "rz", "p", "u3", "swap")
CHANNEL_NAMES = ("dep", "adamp", "pdamp", "bflip", "pflip")

# inverse of each named gate, with the map on its angles
_INVERSE = {"x": "x", "y": "y", "z": "z", "h": "h", "s": "sdg", "sdg": "s",
            "t": "tdg", "tdg": "t", "rx": "rx", "ry": "ry", "rz": "rz",
            "p": "p", "u3": "u3", "u": "u", "swap": "swap"}


def empty(m: int) -> np.ndarray:
    g = np.zeros(m, dtype=GATE_DTYPE)
    g["target2"] = -1
    g["ctrl"] = -1
    return g


def gate(name: str, target: int, controls=(), params=(), mat=None, target2: int = -1) -> np.ndarray:
    """One gate record (a length-1 array)."""
    g = empty(1)
    g["name"] = name
    g["target"] = target
    g["target2"] = target2
    g["nctrl"] = len(controls)
    for i, c in enumerate(controls):
        g["ctrl"][0, i] = c
    for i, p in enumerate(params):
        g["params"][0, i] = p
    if mat is not None:
        m = np.asarray(mat, dtype=np.complex128).reshape(2, 2)
        g["mat"][0] = [m[0, 0].real, m[0, 0].imag, m[0, 1].real, m[0, 1].imag,
                       m[1, 0].real, m[1, 0].imag, m[1, 1].real, m[1, 1].imag]
    return g


def concat(parts) -> np.ndarray:
    parts = [p for p in parts if len(p)]
    if not parts:
        return empty(0)
    return np.concatenate(parts)


def inverse(circ: np.ndarray) -> np.ndarray:
    """The inverse circuit: reversed order, each gate replaced by its inverse."""
    inv = circ[::-1].copy()
    for k in range(len(inv)):
        nm = str(inv["name"][k])
        inv["name"][k] = _INVERSE[nm]
        th, ph, la = inv["params"][k]
        if nm in ("rx", "ry", "rz", "p"):
            inv["params"][k] = (-th, 0.0, 0.0)
        elif nm == "u3":
            inv["params"][k] = (-th, -la, -ph)
        elif nm == "u":
            m = inv["mat"][k]
            a, b, c, d = (complex(m[0], m[1]), complex(m[2], m[3]),
                          complex(m[4], m[5]), complex(m[6], m[7]))
            # conjugate transpose
            a, b, c, d = a.conjugate(), c.conjugate(), b.conjugate(), d.conjugate()
            inv["mat"][k] = [a.real, a.imag, b.real, b.imag, c.real, c.imag, d.real, d.imag]
    return inv


def haar_unitary_2x2(rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed U(2): QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def u3_cnot_ladder(n: int = 14, layers: int = 20, seed: int = 1234) -> np.ndarray:
    """Layers of U3(theta, phi, lambda) on every qubit, angles i.i.d. uniform
    in [0, 2 pi) drawn layer-major then qubit then (theta, phi, lambda), each
    layer followed by CNOT(control q, target q + 1) for q = 0 .. n - 2."""
    rng = np.random.default_rng(seed)
    m = layers * (n + n - 1)
    g = empty(m)
    k = 0
    for _ in range(layers):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            g["name"][k] = "u3"
            g["target"][k] = q
            g["params"][k] = ang[q]
            k += 1
        for q in range(n - 1):
            g["name"][k] = "x"
            g["target"][k] = q + 1
            g["nctrl"][k] = 1
            g["ctrl"][k, 0] = q
            k += 1
    return g


def qft(n: int, swaps: bool = True) -> np.ndarray:
    """Textbook quantum Fourier transform with qubit n-1 the most significant
    bit: for q = n-1 .. 0, H(q) then controlled-phase pi / 2^(q-m) with
    control m, target q, for m = q-1 .. 0; then SWAP(q, n-1-q) for q < n/2.
    The result maps |j> to sum_k e^{2 pi i j k / 2^n} |k> / sqrt(2^n)."""
    parts = []
    for q in range(n - 1, -1, -1):
        parts.append(gate("h", q))
        for m in range(q - 1, -1, -1):
            parts.append(gate("p", q, controls=(m,), params=(math.pi / float(2 ** (q - m)),)))
    if swaps:
        for q in range(n // 2):
            parts.append(gate("swap", q, target2=n - 1 - q))
    return concat(parts)


def qft_paper(n: int) -> np.ndarray:
    """The QFT benchmark circuit of §3 (App. A), built from the QFT's
    structure (§2: a Hadamard per qubit, and between every pair of qubits
    k < j a controlled phase of angle pi / 2^(j - k)): qubit j, taken from
    qubit 0 upwards, first receives the phases it shares with each lower
    qubit, then its Hadamard; no final swaps.  A controlled phase is
    symmetric in its two qubits; here the higher qubit is the control.  The
    circuit equals F P, the QFT of the bit-reversed input."""
    pair_phase = {(k, j): math.pi / float(2 ** (j - k)) for j in range(n) for k in range(j)}
    stages = [[gate("p", k, controls=(j,), params=(pair_phase[(k, j)],)) for k in range(j)] + [gate("h", j)]
              for j in range(n)]
    return concat([g for stage in stages for g in stage])


def phase_polynomial(n: int, m: int, seed: int) -> np.ndarray:
    """m diagonal gates (a phase polynomial, the shape of the cost layers of
    QAOA and IQP circuits and of Trotterised ZZ couplings): each gate is,
    with probability 1/2, a controlled phase P(theta) on a random pair of
    qubits, else one of RZ(theta), P(theta), T, S, Z on a random qubit;
    angles uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    singles = ("rz", "p", "t", "s", "z")
    g = empty(m)
    for k in range(m):
        qs = rng.permutation(n)
        th = rng.uniform(0.0, 2.0 * math.pi)
        if rng.random() < 0.5 and n >= 2:
            g["name"][k] = "p"
            g["target"][k] = qs[0]
            g["nctrl"][k] = 1
            g["ctrl"][k, 0] = qs[1]
        else:
            g["name"][k] = singles[int(rng.integers(0, len(singles)))]
            g["target"][k] = qs[0]
        g["params"][k, 0] = th
    return g


def reversible(n: int, m: int, seed: int) -> np.ndarray:
    """m permutation gates (the reversible-logic part of arithmetic and
    oracle circuits): X, CNOT, Toffoli (two controls) and SWAP in equal
    shares, on random distinct qubits."""
    rng = np.random.default_rng(seed)
    g = empty(m)
    for k in range(m):
        qs = rng.permutation(n)
        kind = int(rng.integers(0, 4 if n >= 3 else 2))
        if kind == 3 and n >= 2:
            g["name"][k] = "swap"
            g["target"][k] = qs[0]
            g["target2"][k] = qs[1]
            continue
        g["name"][k] = "x"
        g["target"][k] = qs[0]
        nc = min(kind, n - 1) if kind < 3 else 0
        g["nctrl"][k] = nc
        for c in range(nc):
            g["ctrl"][k, c] = qs[1 + c]
    return g


def graph_state(n: int, m: int, seed: int) -> np.ndarray:
    """m gates of graph-state (cluster-state) preparation, the entangling
    stage of measurement-based and IQP-type circuits: H on every qubit, then
    CZ on random edges, with a Z or S on a random qubit every eighth gate."""
    rng = np.random.default_rng(seed)
    g = empty(m)
    for k in range(m):
        if k < min(n, m):
            g["name"][k] = "h"
            g["target"][k] = k
            continue
        qs = rng.permutation(n)
        if k % 8 == 0 or n < 2:
            g["name"][k] = "z" if rng.random() < 0.5 else "s"
            g["target"][k] = qs[0]
            continue
        g["name"][k] = "z"
        g["target"][k] = qs[0]
        g["nctrl"][k] = 1
        g["ctrl"][k, 0] = qs[1]
    return g


def segments(n: int, kinds, seg_gates: int, seed: int) -> np.ndarray:
    """A circuit made of consecutive segments of about seg_gates gates each,
    of the given kinds: "haar" (layers of haar_cz), "phase"
    (phase_polynomial), "qft" (the textbook QFT, whatever its length),
    "ladder" (layers of u3_cnot_ladder), "rev" (reversible: X / CNOT /
    Toffoli / SWAP), "graph" (graph-state preparation: H, then CZ edges).  Circuits whose best plan differs from one stretch of
    gates to the next."""
    parts = []
    for i, kind in enumerate(kinds):
        sd = seed * 101 + i
        if kind == "haar":
            parts.append(haar_cz(n, max(1, round(seg_gates / (n + n // 2))), seed=sd))
        elif kind == "phase":
            parts.append(phase_polynomial(n, seg_gates, seed=sd))
        elif kind == "qft":
            parts.append(qft(n))
        elif kind == "ladder":
            parts.append(u3_cnot_ladder(n, max(1, round(seg_gates / (2 * n - 1))), seed=sd))
        elif kind == "rev":
            parts.append(reversible(n, seg_gates, seed=sd))
        elif kind == "graph":
            parts.append(graph_state(n, seg_gates, seed=sd))
        else:
            raise ValueError(kind)
    return concat(parts)


def random_basis_index(n: int, seed: int = 1234) -> int:
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 2 ** n))


def random_matching(rng: np.random.Generator, n: int):
    """floor(n/2) disjoint random pairs over qubits 0..n-1 (one qubit idle if
    n is odd)."""
    perm = rng.permutation(n)
    return [(int(perm[2 * i]), int(perm[2 * i + 1])) for i in range(n // 2)]


def haar_cz(n: int = 30, depth: int = 20, seed: int = 1234) -> np.ndarray:
    """Per layer: a Haar-random U(2) on every qubit (qubit order), then CZ on
    the pairs of a random matching (control = first, target = second of each
    drawn pair)."""
    rng = np.random.default_rng(seed)
    npair = n // 2
    g = empty(depth * (n + npair))
    k = 0
    for _ in range(depth):
        for q in range(n):
            u = haar_unitary_2x2(rng)
            g["name"][k] = "u"
            g["target"][k] = q
            g["mat"][k] = [u[0, 0].real, u[0, 0].imag, u[0, 1].real, u[0, 1].imag,
                           u[1, 0].real, u[1, 0].imag, u[1, 1].real, u[1, 1].imag]
            k += 1
        for (a, b) in random_matching(rng, n):
            g["name"][k] = "z"
            g["target"][k] = b
            g["nctrl"][k] = 1
            g["ctrl"][k, 0] = a
            k += 1
    return g


def variational_layered(n: int, layers: int, rng: np.random.Generator) -> np.ndarray:
    """One variational circuit: per layer RY(theta_q) then RZ(phi_q) on each
    qubit q (angles uniform in [0, 2 pi)), then CZ(q, q+1 mod n) for every q."""
    ring = n if n > 2 else n - 1
    g = empty(layers * (2 * n + ring))
    k = 0
    for _ in range(layers):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 2))
        for q in range(n):
            g["name"][k] = "ry"
            g["target"][k] = q
            g["params"][k, 0] = ang[q, 0]
            k += 1
            g["name"][k] = "rz"
            g["target"][k] = q
            g["params"][k, 0] = ang[q, 1]
            k += 1
        for q in range(ring):
            g["name"][k] = "z"
            g["target"][k] = (q + 1) % n
            g["nctrl"][k] = 1
            g["ctrl"][k, 0] = q
            k += 1
    return g


def variational(count: int = 4096, nmin: int = 8, nmax: int = 20, lmin: int = 4, lmax: int = 12,
                seed: int = 1234):
    """A batch of variational circuits with qubit counts uniform in
    [nmin, nmax] and layer counts uniform in [lmin, lmax].  Returns
    (nqubits int32[count], offsets int64[count+1], gates GATE_DTYPE[...])."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count).astype(np.int32)
    ls = rng.integers(lmin, lmax + 1, size=count).astype(np.int32)
    parts = [variational_layered(int(ns[i]), int(ls[i]), rng) for i in range(count)]
    offs = np.zeros(count + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    return ns, offs, concat(parts)


def bernstein_vazirani(n: int = 14, a: int = 101) -> np.ndarray:
    """App. C: H on every qubit, the inner-product oracle as Z on each qubit i
    with bit i of a set, H on every qubit."""
    parts = [gate("h", i) for i in range(n)]
    parts += [gate("z", i) for i in range(n) if (a >> i) & 1]
    parts += [gate("h", i) for i in range(n)]
    return concat(parts)


def random_gates(n: int, m: int, seed: int, names=None, max_ctrl: int = 2) -> np.ndarray:
    """m random gates over n qubits: random names, targets, up to max_ctrl
    controls, random angles and (for 'u') Haar matrices.  Used for parity
    sweeps over every placement."""
    rng = np.random.default_rng(seed)
    names = names or GATE_NAMES
    g = empty(m)
    for k in range(m):
        nm = names[int(rng.integers(0, len(names)))]
        if nm == "swap" and n < 2:
            nm = "h"
        qs = rng.permutation(n)
        g["name"][k] = nm
        g["target"][k] = qs[0]
        used = 1
        if nm == "swap":
            g["target2"][k] = qs[1]
            used = 2
        nc = int(rng.integers(0, min(max_ctrl, n - used) + 1))
        g["nctrl"][k] = nc
        for c in range(nc):
            g["ctrl"][k, c] = qs[used + c]
        g["params"][k] = rng.uniform(0.0, 2.0 * math.pi, size=3)
        if nm == "u":
            u = haar_unitary_2x2(rng)
            g["mat"][k] = [u[0, 0].real, u[0, 0].imag, u[0, 1].real, u[0, 1].imag,
                           u[1, 0].real, u[1, 0].imag, u[1, 1].real, u[1, 1].imag]
    return g


def random_state(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """A random unit vector of 2^n amplitudes (complex normal entries,
    normalised in FP64)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    v /= np.sqrt(np.vdot(v, v).real)
    return v.astype(dtype)


def channel(name: str, target: int, p: float) -> np.ndarray:
    """One noise-channel record (density matrices only)."""
    if name not in CHANNEL_NAMES:
        raise ValueError(name)
    g = empty(1)
    g["name"][0] = name
    g["target"][0] = target
    g["params"][0, 0] = p
    return g


def noisy(gates: np.ndarray, n: int, per_layer: int, channels=(("dep", 1e-3),)) -> np.ndarray:
    """`gates` cut into layers of per_layer gates, each layer followed by every
    (name, p) channel of `channels` on every qubit 0..n-1."""
    parts = []
    for f in range(0, len(gates), per_layer):
        parts.append(gates[f:f + per_layer])
        for name, p in channels:
            for q in range(n):
                parts.append(channel(name, q, p))
    return concat(parts)


def noisy_haar_cz(n: int, depth: int, seed: int, channels=(("dep", 1e-3), ("adamp", 2e-3))) -> np.ndarray:
    """haar_cz(n, depth) with the given channels on every qubit after each
    layer (a layer = n Haar gates + the matching's n // 2 CZ)."""
    return noisy(haar_cz(n, depth, seed=seed), n, n + n // 2, channels)


def random_noisy(n: int, m: int, seed: int, p_channel: float = 0.3) -> np.ndarray:
    """m records: random gates (random_gates), each followed with probability
    p_channel by a random channel on a random qubit, parameter uniform in
    [0, 0.5)."""
    rng = np.random.default_rng(seed)
    g = random_gates(n, m, seed=seed + 1)
    parts = []
    for k in range(m):
        parts.append(g[k:k + 1])
        if rng.random() < p_channel:
            parts.append(channel(CHANNEL_NAMES[int(rng.integers(0, len(CHANNEL_NAMES)))],
                                 int(rng.integers(0, n)), float(rng.uniform(0.0, 0.5))))
    return concat(parts)
