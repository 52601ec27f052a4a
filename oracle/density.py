"""FP64 density-matrix oracle: mixed states and noise channels.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use
it; it shares no code with the CUDA library.

The paper names density matrices as one output a simulator can give (§1);
this module writes the standard definitions out with dense matrices, slow and
plain, for registers of up to about 10 qubits:

  state        rho, a 2^n x 2^n complex matrix; rho[r, c] is the coefficient
               of |r><c|, qubit t = bit t of r and c (the state-vector
               convention of the rest of the oracle).  A pure state psi gives
               rho = |psi><psi|, i.e. rho[r, c] = psi_r conj(psi_c).
  gate         rho -> G rho G^dagger, G the gate embedded in the whole register
               (§1.3.2: the tensor product of the gate with identities; a
               controlled gate acts where every control bit is 1, §2.3).
  channel      rho -> sum_m K_m rho K_m^dagger (Kraus form), each K_m embedded
               like a gate.
  probability  p_j = <j|rho|j> = Re rho[j, j] (§1.3.3 with M_j = |j><j|).
  measurement  §1.3.3: p(m) = tr(M_m rho M_m^dagger) with M_m the projector
               on qubit q = m; post-state M_m rho M_m / p(m).
  sampling     inverse CDF over p_j, the rule of the state-vector oracle
               (orc_sample_weights: smallest j whose compensated prefix
               exceeds u_s times the total), p_j below zero counted as zero.

Named channels follow Nielsen & Chuang, *Quantum Computation and Quantum
Information*, §8.3: depolarizing(p) maps rho to (1 - p) rho + p I / 2;
amplitude damping (gamma) and phase damping (lambda) as their Kraus pairs;
bit flip and phase flip with probability p.
"""
from __future__ import annotations

import numpy as np

from . import gate_matrix, sample_weights, uniform

_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)     # |1><1|


def _nq(rho: np.ndarray) -> int:
    d = rho.shape[0]
    n = d.bit_length() - 1
    if rho.shape != (d, d) or d != (1 << n):
        raise ValueError("rho must be 2^n x 2^n")
    return n


def kron_register(n: int, factors: dict) -> np.ndarray:
    """The n-qubit operator with factors[q] on qubit q and identity on the
    others (qubit n - 1 is the leftmost Kronecker factor: qubit t = bit t)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        out = np.kron(out, factors.get(q, _I2))
    return out


def embed(n: int, U: np.ndarray, target: int, controls=()) -> np.ndarray:
    """U on `target`, applied where every control bit is 1 (§2.3):
    G = (1 - P) + P (U on target), P the projector on controls all 1."""
    P = kron_register(n, {c: _P1 for c in controls})
    full = kron_register(n, {target: U})
    eye = np.eye(1 << n, dtype=np.complex128)
    return eye - P + P @ full


def swap_operator(n: int, a: int, b: int, controls=()) -> np.ndarray:
    """The permutation |..x_a..x_b..> -> |..x_b..x_a..> where every control
    bit is 1, identity elsewhere, written out basis state by basis state."""
    d = 1 << n
    G = np.zeros((d, d), dtype=np.complex128)
    for j in range(d):
        k = j
        if all((j >> c) & 1 for c in controls):
            ba, bb = (j >> a) & 1, (j >> b) & 1
            k = j & ~((1 << a) | (1 << b)) | (bb << a) | (ba << b)
        G[k, j] = 1.0
    return G


def gate_operator(n: int, g) -> np.ndarray:
    """The whole-register operator of one gate record (circuits.GATE_DTYPE)."""
    name = str(g["name"])
    ctrl = tuple(int(c) for c in g["ctrl"][: int(g["nctrl"])])
    if name == "swap":
        return swap_operator(n, int(g["target"]), int(g["target2"]), ctrl)
    U = gate_matrix(name, tuple(g["params"]), np.asarray(g["mat"], dtype=np.float64))
    return embed(n, U, int(g["target"]), ctrl)


def pure(psi: np.ndarray) -> np.ndarray:
    """|psi><psi|."""
    psi = np.asarray(psi, dtype=np.complex128)
    return np.outer(psi, psi.conj())


def basis(n: int, j: int = 0) -> np.ndarray:
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[j, j] = 1.0
    return rho


# record names of noise channels (the input format's channel records) -> kind
CHANNELS = {"dep": "depolarizing", "adamp": "amplitude_damping", "pdamp": "phase_damping",
            "bflip": "bit_flip", "pflip": "phase_flip"}


def apply_circuit(rho: np.ndarray, gates) -> np.ndarray:
    """rho -> G rho G^dagger for each gate record in order; a channel record
    (name in CHANNELS, parameter params[0]) applies its Kraus map there."""
    n = _nq(rho)
    out = np.array(rho, dtype=np.complex128)
    for g in gates:
        name = str(g["name"])
        if name in CHANNELS:
            out = apply_kraus(out, kraus(CHANNELS[name], float(g["params"][0])), int(g["target"]))
            continue
        G = gate_operator(n, g)
        out = G @ out @ G.conj().T
    return out


# ---------------------------------------------------------------- channels
def kraus(kind: str, p: float):
    """Kraus operators of a named single-qubit channel (Nielsen & Chuang §8.3)."""
    if kind == "depolarizing":
        return [np.sqrt(1.0 - 0.75 * p) * _I2, np.sqrt(p / 4.0) * _X, np.sqrt(p / 4.0) * _Y, np.sqrt(p / 4.0) * _Z]
    if kind == "amplitude_damping":
        return [np.array([[1, 0], [0, np.sqrt(1.0 - p)]], dtype=np.complex128),
                np.array([[0, np.sqrt(p)], [0, 0]], dtype=np.complex128)]
    if kind == "phase_damping":
        return [np.array([[1, 0], [0, np.sqrt(1.0 - p)]], dtype=np.complex128),
                np.array([[0, 0], [0, np.sqrt(p)]], dtype=np.complex128)]
    if kind == "bit_flip":
        return [np.sqrt(1.0 - p) * _I2, np.sqrt(p) * _X]
    if kind == "phase_flip":
        return [np.sqrt(1.0 - p) * _I2, np.sqrt(p) * _Z]
    raise ValueError(kind)


def apply_kraus(rho: np.ndarray, ks, target: int) -> np.ndarray:
    """rho -> sum_m K_m rho K_m^dagger, every K_m on qubit `target`."""
    n = _nq(rho)
    out = np.zeros_like(rho, dtype=np.complex128)
    for K in ks:
        E = kron_register(n, {target: np.asarray(K, dtype=np.complex128)})
        out += E @ rho @ E.conj().T
    return out


# ---------------------------------------------------------------- observables
def probabilities(rho: np.ndarray) -> np.ndarray:
    return np.real(np.diag(rho)).copy()


def trace(rho: np.ndarray) -> float:
    return float(np.sum(np.real(np.diag(rho))))


def purity(rho: np.ndarray) -> float:
    """tr(rho^2)."""
    return float(np.real(np.trace(rho @ rho)))


def expect_z_sum(rho: np.ndarray) -> float:
    """<sum_i Z_i> = sum_j p_j (n - 2 popcount j) (Z_i: +1 on bit i = 0)."""
    n = _nq(rho)
    p = probabilities(rho)
    w = np.array([n - 2 * bin(j).count("1") for j in range(1 << n)], dtype=np.float64)
    return float(np.sum(p * w))


def measure(rho: np.ndarray, q: int, seed: int, draw: int = 0):
    """Measure qubit q (§1.3.3); returns (outcome, probability, post-state).
    Outcome 0 iff p0 > u (p0 + p1), u = the oracle's SplitMix64 draw."""
    n = _nq(rho)
    P1 = kron_register(n, {q: _P1})
    P0 = np.eye(1 << n, dtype=np.complex128) - P1
    p0 = float(np.real(np.trace(P0 @ rho @ P0)))
    p1 = float(np.real(np.trace(P1 @ rho @ P1)))
    u = uniform(seed, draw)
    m = 0 if p0 > u * (p0 + p1) else 1
    P = P1 if m else P0
    pm = p1 if m else p0
    return m, pm / (p0 + p1), (P @ rho @ P) / pm


def sample(rho: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Shots from p_j = Re rho[j, j] (negative values, which only rounding
    produces for a physical rho, count as zero); rho is unchanged."""
    p = np.maximum(probabilities(rho), 0.0)
    return sample_weights(p, shots, seed)
