"""CPU FP64 oracle for dense state-vector gate application.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this package.  It
shares no code with the CUDA library: the arithmetic lives in
``qsim_oracle.c`` (plain C, FP64), compiled here with gcc; ``mlp.py`` holds
the numpy FP64 oracle of the cost model's network (forward, backward,
Adam); ``density.py`` the numpy FP64 density-matrix oracle (gates, noise
channels, measurement and sampling of mixed states, dense matrices).

States are numpy complex128 arrays of 2^n amplitudes (amplitude j <-> |j>,
qubit t = bit t of j).  Gate lists are structured arrays with the fields of
``paper_1805_00988_gb300.circuits.GATE_DTYPE``; this wrapper maps gate names
to the oracle's own kind codes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqsim_oracle.so")

# oracle kind codes (the enum at the top of qsim_oracle.c)
KINDS = {"u": 0, "x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8,
         "rx": 9, "ry": 10, "rz": 11, "p": 12, "u3": 13, "swap": 14}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qsim_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.orc_apply_circuit.argtypes = [i32, P, i64, P, P, P, P, P, P, P]
            lib.orc_apply_circuit.restype = i32
            lib.orc_gate_matrix.argtypes = [i32, P, P, P]
            lib.orc_gate_matrix.restype = i32
            lib.orc_basis_state.argtypes = [i32, P, u64]
            lib.orc_probabilities.argtypes = [i32, P, P]
            lib.orc_norm2.argtypes = [i32, P]
            lib.orc_norm2.restype = f64
            lib.orc_prob_one.argtypes = [i32, P, i32]
            lib.orc_prob_one.restype = f64
            lib.orc_splitmix64.argtypes = [u64]
            lib.orc_splitmix64.restype = u64
            lib.orc_uniform.argtypes = [u64, u64]
            lib.orc_uniform.restype = f64
            lib.orc_measure.argtypes = [i32, P, i32, u64, u64, P]
            lib.orc_measure.restype = i32
            lib.orc_sample.argtypes = [i32, P, u64, u64, P]
            lib.orc_sample.restype = i32
            lib.orc_sample_weights.argtypes = [u64, P, u64, u64, P]
            lib.orc_sample_weights.restype = i32
            lib.orc_expect_z_sum.argtypes = [i32, P]
            lib.orc_expect_z_sum.restype = f64
            lib.orc_infidelity.argtypes = [i32, P, P]
            lib.orc_infidelity.restype = f64
            lib.orc_num_threads.restype = i32
            lib.orc_set_num_threads.argtypes = [i32]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nqubits(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    """Threads of the oracle's per-gate loops from now on (results do not
    depend on it; reductions are serial)."""
    _load().orc_set_num_threads(int(t))


def gate_matrix(name: str, params=(0.0, 0.0, 0.0), mat=None) -> np.ndarray:
    """The oracle's 2x2 matrix for a named gate, as a complex128 2x2 array."""
    lib = _load()
    p = np.zeros(3, dtype=np.float64)
    p[: len(params)] = params
    m = np.zeros(8, dtype=np.float64) if mat is None else np.ascontiguousarray(mat, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    if lib.orc_gate_matrix(KINDS[name], _ptr(p), _ptr(m), _ptr(out)) != 0:
        raise ValueError(name)
    return (out[0::2] + 1j * out[1::2]).reshape(2, 2)


def basis_state(n: int, j: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    _load().orc_basis_state(n, _ptr(psi), j)
    return psi


def apply_circuit(psi: np.ndarray, gates: np.ndarray, inplace: bool = False) -> np.ndarray:
    """Apply the gate list in order to a copy of psi (complex128); returns it.
    With inplace=True psi (a C-contiguous complex128 array) is updated and
    returned."""
    lib = _load()
    if inplace:
        if psi.dtype != np.complex128 or not psi.flags["C_CONTIGUOUS"]:
            raise ValueError("inplace needs a C-contiguous complex128 array")
        out = psi
    else:
        out = np.array(psi, dtype=np.complex128, copy=True, order="C")
    n = _nqubits(out)
    m = len(gates)
    kind = np.array([KINDS[str(x)] for x in gates["name"]], dtype=np.int32)
    target = np.ascontiguousarray(gates["target"], dtype=np.int32)
    target2 = np.ascontiguousarray(gates["target2"], dtype=np.int32)
    nctrl = np.ascontiguousarray(gates["nctrl"], dtype=np.int32)
    ctrl = np.ascontiguousarray(gates["ctrl"], dtype=np.int32)
    params = np.ascontiguousarray(gates["params"], dtype=np.float64)
    mat = np.ascontiguousarray(gates["mat"], dtype=np.float64)
    rc = lib.orc_apply_circuit(n, _ptr(out), m, _ptr(kind), _ptr(target), _ptr(target2),
                               _ptr(nctrl), _ptr(ctrl), _ptr(params), _ptr(mat))
    if rc != 0:
        raise ValueError("invalid gate %d" % (-rc - 1))
    return out


def probabilities(psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    p = np.zeros(psi.size, dtype=np.float64)
    _load().orc_probabilities(_nqubits(psi), _ptr(psi), _ptr(p))
    return p


def norm2(psi: np.ndarray) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().orc_norm2(_nqubits(psi), _ptr(psi)))


def prob_one(psi: np.ndarray, q: int) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().orc_prob_one(_nqubits(psi), _ptr(psi), q))


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def uniform(seed: int, s: int) -> float:
    return float(_load().orc_uniform(seed & 0xFFFFFFFFFFFFFFFF, s))


def measure(psi: np.ndarray, q: int, seed: int, draw: int = 0):
    """Measure qubit q; returns (outcome, probability, collapsed state)."""
    out = np.array(psi, dtype=np.complex128, copy=True, order="C")
    p = ctypes.c_double(0.0)
    m = _load().orc_measure(_nqubits(out), _ptr(out), q, seed, draw, ctypes.byref(p))
    return int(m), float(p.value), out


def sample(psi: np.ndarray, shots: int, seed: int) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(shots, dtype=np.uint64)
    if _load().orc_sample(_nqubits(psi), _ptr(psi), shots, seed, _ptr(out)) != 0:
        raise MemoryError("oracle sample")
    return out


def sample_weights(p: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Inverse-CDF shots over non-negative weights p (the rule of sample())."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(shots, dtype=np.uint64)
    if _load().orc_sample_weights(p.size, _ptr(p), shots, seed, _ptr(out)) != 0:
        raise MemoryError("oracle sample_weights")
    return out


def expect_z_sum(psi: np.ndarray) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().orc_expect_z_sum(_nqubits(psi), _ptr(psi)))


def infidelity(a: np.ndarray, b: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    return float(_load().orc_infidelity(_nqubits(a), _ptr(a), _ptr(b)))
