"""Thin ctypes binding of the C ABI in include/qsim_gb300.h.

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Importing this module loads ``_lib/libqsim_gb300.so`` and raises
ImportError when it has not been built (``python -m
paper_1805_00988_gb300.build``); there is no CPU fallback.

The module-level functions keep the C names (``sim_create``,
``sim_apply_gate`` ...).  ``State`` is a small convenience wrapper whose state
buffer is a PyTorch CUDA tensor (PyTorch supplies device memory and the
stream; the library never sees a torch type).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqsim_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libqsim_gb300.so is not built (run python -m paper_1805_00988_gb300.build); "
                      "the simulator has no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

SIM_C64, SIM_C128 = 0, 1
SIM_F32, SIM_F64 = 0, 1
SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ETIMEOUT, SIM_EUNSUPPORTED = range(6)
SIM_PLAN_PER_GATE, SIM_PLAN_STAGED, SIM_PLAN_FUSED, SIM_PLAN_LEARNED = range(4)
PLANS = {"per_gate": 0, "staged": 1, "fused": 2, "learned": 3}
CUDA_STREAM_LEGACY = 1      # cudaStreamLegacy

GATE_KINDS = {"u": 0, "x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8,
              "rx": 9, "ry": 10, "rz": 11, "p": 12, "u3": 13, "swap": 14,
              # noise channels (density-matrix handles only), parameter in params[0]
              "dep": 16, "adamp": 17, "pdamp": 18, "bflip": 19, "pflip": 20}
SIM_CHANNELS = {"depolarizing": 0, "amplitude_damping": 1, "phase_damping": 2, "bit_flip": 3, "phase_flip": 4}

# struct sim_gate (112 bytes)
SIM_GATE_DTYPE = np.dtype([
    ("kind", "<i4"), ("target", "<i4"), ("target2", "<i4"), ("n_controls", "<i4"),
    ("controls", "<i4", (2,)), ("params", "<f8", (3,)), ("matrix", "<f8", (8,)),
])
assert SIM_GATE_DTYPE.itemsize == 112


class sim_plan_opts(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_int32), ("fuse_k", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32), ("flags", ctypes.c_int32)]


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("status %d: %s" % (status, msg))
        self.status = status


P = ctypes.c_void_p
_i32, _u64, _sz = ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("sim_create", [_i32, _i32, P, ctypes.POINTER(P)])
_sig("sim_create_from_buffer", [_i32, _i32, P, _sz, P, ctypes.POINTER(P)])
_sig("sim_destroy", [P])
_sig("sim_state_info", [P, P, P, P, P])
_sig("sim_synchronize", [P])
_sig("sim_set_basis_state", [P, _u64])
_sig("sim_load_state", [P, P, _i32])
_sig("sim_copy_state", [P, P, _i32])
_sig("sim_apply_gate", [P, P, _i32, P, _i32])
_sig("sim_apply_circuit", [P, P, _sz, P])
_sig("sim_probabilities", [P, P, _i32])
_sig("sim_norm", [P, P])
_sig("sim_measure", [P, _i32, _u64, _u64, P, P])
_sig("sim_sample", [P, _u64, _u64, P, _i32])
_sig("sim_sample_observe", [P, _u64, _u64, P, _i32, P, P])
_sig("sim_expect_z_sum", [P, P])
_sig("sim_profile_enable", [P, _i32])
_sig("sim_profile_read", [P, _i32, P, P, P, P, _i32])
_sig("sim_launch_count", [P, P])
_sig("sim_kernel_class_name", [_i32], ctypes.c_char_p)
_sig("sim_num_kernel_classes", [], _i32)
_sig("sim_last_error", [], ctypes.c_char_p)
_sig("sim_version", [], ctypes.c_char_p)


def last_error() -> str:
    return _lib.sim_last_error().decode()


def check(status: int):
    if status != SIM_OK:
        raise SimError(status, last_error())


def lib_handle():
    """The loaded ctypes library (for callers that need a raw entry point)."""
    return _lib


# ---------------------------------------------------------------- raw entry points
def sim_create(n: int, dtype: int = SIM_C64, stream: int = 0) -> int:
    h = P()
    check(_lib.sim_create(n, dtype, P(stream or None), ctypes.byref(h)))
    return h.value


def sim_create_from_buffer(n: int, dtype: int, dev_ptr: int, nbytes: int, stream: int = 0) -> int:
    h = P()
    check(_lib.sim_create_from_buffer(n, dtype, P(dev_ptr), nbytes, P(stream or None), ctypes.byref(h)))
    return h.value


def sim_destroy(h: int):
    check(_lib.sim_destroy(P(h)))
    _COST_MODELS.pop(h, None)


def sim_synchronize(h: int):
    check(_lib.sim_synchronize(P(h)))


def sim_set_basis_state(h: int, j: int):
    check(_lib.sim_set_basis_state(P(h), j))


def sim_load_state(h: int, src, src_is_host: bool = True):
    check(_lib.sim_load_state(P(h), P(src), int(src_is_host)))


def sim_copy_state(h: int, dst, dst_is_host: bool = True):
    check(_lib.sim_copy_state(P(h), P(dst), int(dst_is_host)))


def sim_apply_gate(h: int, U, target: int, controls=()):
    u = np.zeros(8, dtype=np.float64)
    m = np.asarray(U, dtype=np.complex128).reshape(2, 2)
    u[0::2] = m.reshape(-1).real
    u[1::2] = m.reshape(-1).imag
    c = (ctypes.c_int * 2)(*(list(controls) + [-1, -1])[:2])
    check(_lib.sim_apply_gate(P(h), u.ctypes.data_as(P), target, c, len(controls)))


def to_sim_gates(gates: np.ndarray) -> np.ndarray:
    """Convert a circuits.GATE_DTYPE array into struct sim_gate records."""
    out = np.zeros(len(gates), dtype=SIM_GATE_DTYPE)
    if len(gates) == 0:
        return out
    names = gates["name"]
    kinds = np.zeros(len(gates), dtype=np.int32)
    for nm, code in GATE_KINDS.items():
        kinds[names == nm] = code
    known = np.isin(names, list(GATE_KINDS))
    if not np.all(known):
        raise ValueError("unknown gate name %r" % names[~known][0])
    out["kind"] = kinds
    out["target"] = gates["target"]
    out["target2"] = gates["target2"]
    out["n_controls"] = gates["nctrl"]
    out["controls"] = gates["ctrl"]
    out["params"] = gates["params"]
    out["matrix"] = gates["mat"]
    return out


SIM_FLAG_MULTI_BLOCK_PASSES = 1


def plan_opts(plan="per_gate", fuse_k=0, tile_qubits=0, flags=0) -> sim_plan_opts:
    p = PLANS[plan] if isinstance(plan, str) else int(plan)
    return sim_plan_opts(p, fuse_k, tile_qubits, flags)


def sim_apply_circuit(h: int, sim_gates: np.ndarray, opts: sim_plan_opts = None):
    g = np.ascontiguousarray(sim_gates, dtype=SIM_GATE_DTYPE)
    check(_lib.sim_apply_circuit(P(h), g.ctypes.data_as(P), len(g),
                                 ctypes.byref(opts) if opts is not None else None))


def sim_probabilities(h: int, dev_out: int, out_real: int = SIM_F64):
    check(_lib.sim_probabilities(P(h), P(dev_out), out_real))


def sim_norm(h: int) -> float:
    r = ctypes.c_double()
    check(_lib.sim_norm(P(h), ctypes.byref(r)))
    return r.value


def sim_expect_z_sum(h: int) -> float:
    r = ctypes.c_double()
    check(_lib.sim_expect_z_sum(P(h), ctypes.byref(r)))
    return r.value


_sig("sim_norm_expect_z", [P, P, P])


def sim_norm_expect_z(h: int):
    """(norm, <sum Z>) from one pass over the state."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(_lib.sim_norm_expect_z(P(h), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sim_measure(h: int, qubit: int, seed: int, draw: int = 0):
    m = ctypes.c_int()
    p = ctypes.c_double()
    check(_lib.sim_measure(P(h), qubit, seed, draw, ctypes.byref(m), ctypes.byref(p)))
    return m.value, p.value


def sim_sample(h: int, shots: int, seed: int, out=None, out_on_device: bool = False):
    """Host output: returns a numpy uint64 array (or fills ``out``).  Device
    output: ``out`` is a device pointer (int) to shots uint64."""
    if out_on_device:
        check(_lib.sim_sample(P(h), shots, seed, P(out), 1))
        return out
    arr = np.empty(shots, dtype=np.uint64) if out is None else out
    check(_lib.sim_sample(P(h), shots, seed, arr.ctypes.data_as(P), 0))
    return arr


_sig("sim_plan_describe", [_i32, _i32, P, _sz, P, P, P, P, P, _sz, P])


def sim_sample_observe(h: int, shots: int, seed: int, out=None, out_on_device: bool = False):
    """Shots as sim_sample draws them, plus (norm, <sum Z>) of the same state:
    returns (shots, norm, expz); for complex64 from 13 qubits all three come
    from one pass over the state."""
    a, b = ctypes.c_double(), ctypes.c_double()
    if out_on_device:
        check(_lib.sim_sample_observe(P(h), shots, seed, P(out), 1, ctypes.byref(a), ctypes.byref(b)))
        return out, a.value, b.value
    arr = np.empty(shots, dtype=np.uint64) if out is None else out
    check(_lib.sim_sample_observe(P(h), shots, seed, arr.ctypes.data_as(P), 0, ctypes.byref(a), ctypes.byref(b)))
    return arr, a.value, b.value


SIM_TILE_OP_DTYPE = np.dtype([("kind", "<i4"), ("arg", "<i4"), ("thr_c", "<u4"), ("plain", "<i4"),
                              ("out_c", "<u8"), ("km_c", "<u8"), ("km_t", "<u8"), ("thr_t", "<u4"),
                              ("pad", "<u4"), ("out_t", "<u8"), ("m", "<f8", (8,))])
SIM_TILE_PASS_INFO = 24
_sig("sim_plan_staged_ops", [_i32, _i32, P, _sz, _i32, P, _sz, P, _sz, P, P])


def sim_plan_staged_ops(n: int, dtype: int, sim_gates: np.ndarray, tile_qubits: int = 0):
    """The staged plan's encoded op records and per-pass geometry (host only):
    returns (ops as SIM_TILE_OP_DTYPE records, info as an int32 array of
    shape (passes, SIM_TILE_PASS_INFO))."""
    g = np.ascontiguousarray(sim_gates, dtype=SIM_GATE_DTYPE)
    nops, npass = ctypes.c_size_t(), ctypes.c_size_t()
    check(_lib.sim_plan_staged_ops(n, dtype, g.ctypes.data_as(P), len(g), tile_qubits, None, 0, None, 0,
                                   ctypes.byref(nops), ctypes.byref(npass)))
    ops = np.zeros(nops.value, dtype=SIM_TILE_OP_DTYPE)
    info = np.zeros((npass.value, SIM_TILE_PASS_INFO), dtype=np.int32)
    check(_lib.sim_plan_staged_ops(n, dtype, g.ctypes.data_as(P), len(g), tile_qubits, ops.ctypes.data_as(P),
                                   len(ops), info.ctypes.data_as(P), info.size, ctypes.byref(nops),
                                   ctypes.byref(npass)))
    return ops, info


def sim_plan_describe(n: int, dtype: int, sim_gates: np.ndarray, opts: sim_plan_opts):
    """Host-only: (passes, ops, layout_changes, order) of the staged schedule."""
    g = np.ascontiguousarray(sim_gates, dtype=SIM_GATE_DTYPE)
    passes, ops, lc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ln = ctypes.c_size_t()
    check(_lib.sim_plan_describe(n, dtype, g.ctypes.data_as(P), len(g), ctypes.byref(opts), ctypes.byref(passes),
                                 ctypes.byref(ops), ctypes.byref(lc), None, 0, ctypes.byref(ln)))
    order = np.zeros(ln.value, dtype=np.int32)
    check(_lib.sim_plan_describe(n, dtype, g.ctypes.data_as(P), len(g), ctypes.byref(opts), None, None, None,
                                 order.ctypes.data_as(P), len(order), ctypes.byref(ln)))
    return passes.value, ops.value, lc.value, order


def sim_profile_enable(h: int, on: bool = True):
    check(_lib.sim_profile_enable(P(h), int(on)))


def sim_profile_read(h: int, reset: bool = True):
    k = _lib.sim_num_kernel_classes()
    launches = (ctypes.c_uint64 * k)()
    ms = (ctypes.c_double * k)()
    nbytes = (ctypes.c_double * k)()
    flops = (ctypes.c_double * k)()
    check(_lib.sim_profile_read(P(h), k, launches, ms, nbytes, flops, int(reset)))
    return {_lib.sim_kernel_class_name(i).decode(): (int(launches[i]), float(ms[i]), float(nbytes[i]),
                                                     float(flops[i]))
            for i in range(k) if launches[i]}


def sim_launch_count(h: int) -> int:
    r = ctypes.c_uint64()
    check(_lib.sim_launch_count(P(h), ctypes.byref(r)))
    return r.value


def sim_version() -> str:
    return _lib.sim_version().decode()


# ---------------------------------------------------------------- convenience wrapper
class State:
    """An n-qubit register whose amplitudes live in a PyTorch CUDA tensor.

    dtype: "c64" (complex64) or "c128" (complex128).  Starts in |0...0>.
    """

    def __init__(self, n: int, dtype: str = "c64", device=None, torch_memory: bool = True):
        import torch
        self.n = n
        self.dtype = SIM_C128 if dtype in ("c128", SIM_C128, np.complex128) else SIM_C64
        self._torch = torch
        dev = torch.device(device or "cuda")
        self.stream = torch.cuda.current_stream(dev)
        # torch's default stream has handle 0; the ABI reads 0 as "make your
        # own stream", so the legacy default stream is passed explicitly.
        self.stream_handle = self.stream.cuda_stream or CUDA_STREAM_LEGACY
        tdt = torch.complex128 if self.dtype == SIM_C128 else torch.complex64
        if torch_memory:
            self.tensor = torch.empty(2 ** n, dtype=tdt, device=dev)
            self.h = sim_create_from_buffer(n, self.dtype, self.tensor.data_ptr(),
                                            self.tensor.numel() * self.tensor.element_size(),
                                            self.stream_handle)
            sim_set_basis_state(self.h, 0)
        else:
            self.tensor = None
            self.h = sim_create(n, self.dtype, self.stream_handle)

    def close(self):
        if getattr(self, "h", None):
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def np_dtype(self):
        return np.complex128 if self.dtype == SIM_C128 else np.complex64

    def set_basis(self, j: int = 0):
        sim_set_basis_state(self.h, j)

    def load(self, psi: np.ndarray):
        a = np.ascontiguousarray(psi, dtype=self.np_dtype)
        assert a.size == 2 ** self.n
        sim_load_state(self.h, a.ctypes.data, True)

    def state(self) -> np.ndarray:
        out = np.empty(2 ** self.n, dtype=self.np_dtype)
        sim_copy_state(self.h, out.ctypes.data, True)
        return out

    def apply(self, gates: np.ndarray, plan="per_gate", **kw):
        sim_apply_circuit(self.h, to_sim_gates(gates), plan_opts(plan, **kw))

    def apply_gate(self, U, target, controls=()):
        sim_apply_gate(self.h, U, target, controls)

    def probabilities(self, f64: bool = True):
        t = self._torch.empty(2 ** self.n, dtype=self._torch.float64 if f64 else self._torch.float32,
                              device=self.tensor.device if self.tensor is not None else "cuda")
        sim_probabilities(self.h, t.data_ptr(), SIM_F64 if f64 else SIM_F32)
        sim_synchronize(self.h)
        return t.cpu().numpy()

    def norm2(self) -> float:
        return sim_norm(self.h)

    def expect_z_sum(self) -> float:
        return sim_expect_z_sum(self.h)

    def measure(self, qubit: int, seed: int, draw: int = 0):
        return sim_measure(self.h, qubit, seed, draw)

    def sample(self, shots: int, seed: int) -> np.ndarray:
        return sim_sample(self.h, shots, seed)

    def synchronize(self):
        sim_synchronize(self.h)


# ---------------------------------------------------------------- density matrices
_sig("sim_dm_create", [_i32, _i32, P, ctypes.POINTER(P)])
_sig("sim_dm_create_from_buffer", [_i32, _i32, P, _sz, P, ctypes.POINTER(P)])
_sig("sim_dm_info", [P, P])
_sig("sim_dm_set_basis_state", [P, _u64])
_sig("sim_dm_set_pure", [P, P])
_sig("sim_dm_apply_circuit", [P, P, _sz, P])
_sig("sim_channel_kraus", [_i32, ctypes.c_double, P, P])
_sig("sim_dm_apply_kraus", [P, _i32, P, _i32])
_sig("sim_dm_apply_channel", [P, _i32, ctypes.c_double, _i32])
_sig("sim_dm_probabilities", [P, P, _i32])
_sig("sim_dm_trace", [P, P])
_sig("sim_dm_purity", [P, P])
_sig("sim_dm_expect_z_sum", [P, P])
_sig("sim_dm_measure", [P, _i32, _u64, _u64, P, P])
_sig("sim_dm_sample", [P, _u64, _u64, P, _i32])


def _mat8(K) -> np.ndarray:
    m = np.asarray(K, dtype=np.complex128).reshape(2, 2).reshape(-1)
    out = np.zeros(8, dtype=np.float64)
    out[0::2] = m.real
    out[1::2] = m.imag
    return out


def sim_channel_kraus(kind: str, p: float):
    """The library's Kraus operators of a named channel, as 2x2 complex arrays."""
    buf = np.zeros(32, dtype=np.float64)
    cnt = ctypes.c_int()
    check(_lib.sim_channel_kraus(SIM_CHANNELS[kind], float(p), buf.ctypes.data_as(P), ctypes.byref(cnt)))
    return [(buf[8 * m:8 * m + 8:2] + 1j * buf[8 * m + 1:8 * m + 8:2]).reshape(2, 2) for m in range(cnt.value)]


def sim_dm_apply_circuit(h: int, sim_gates: np.ndarray, opts: sim_plan_opts = None):
    g = np.ascontiguousarray(sim_gates, dtype=SIM_GATE_DTYPE)
    check(_lib.sim_dm_apply_circuit(P(h), g.ctypes.data_as(P), len(g),
                                    ctypes.byref(opts) if opts is not None else None))


def _dm_scalar(fn, h):
    r = ctypes.c_double()
    check(fn(P(h), ctypes.byref(r)))
    return r.value


class DensityMatrix:
    """A density matrix of n qubits (a 2n-qubit register whose amplitude
    (r << n) | c is rho[r][c]) in a PyTorch CUDA tensor.  Starts in
    |0...0><0...0|."""

    def __init__(self, n: int, dtype: str = "c64", device=None):
        import torch
        self.n = n
        self.dtype = SIM_C128 if dtype in ("c128", SIM_C128, np.complex128) else SIM_C64
        self._torch = torch
        dev = torch.device(device or "cuda")
        self.stream = torch.cuda.current_stream(dev)
        self.stream_handle = self.stream.cuda_stream or CUDA_STREAM_LEGACY
        tdt = torch.complex128 if self.dtype == SIM_C128 else torch.complex64
        self.tensor = torch.empty(4 ** n, dtype=tdt, device=dev)
        h = P()
        check(_lib.sim_dm_create_from_buffer(n, self.dtype, P(self.tensor.data_ptr()),
                                             self.tensor.numel() * self.tensor.element_size(),
                                             P(self.stream_handle), ctypes.byref(h)))
        self.h = h.value
        self.set_basis(0)

    def close(self):
        if getattr(self, "h", None):
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def np_dtype(self):
        return np.complex128 if self.dtype == SIM_C128 else np.complex64

    def set_basis(self, j: int = 0):
        check(_lib.sim_dm_set_basis_state(P(self.h), j))

    def set_pure(self, psi_state: "State"):
        check(_lib.sim_dm_set_pure(P(self.h), P(psi_state.h)))

    def load(self, rho: np.ndarray):
        a = np.ascontiguousarray(np.asarray(rho).reshape(-1), dtype=self.np_dtype)
        assert a.size == 4 ** self.n
        sim_load_state(self.h, a.ctypes.data, True)

    def matrix(self) -> np.ndarray:
        out = np.empty(4 ** self.n, dtype=self.np_dtype)
        sim_copy_state(self.h, out.ctypes.data, True)
        return out.reshape(2 ** self.n, 2 ** self.n)

    def apply(self, gates: np.ndarray, plan="per_gate", **kw):
        sim_dm_apply_circuit(self.h, to_sim_gates(gates), plan_opts(plan, **kw))

    def apply_kraus(self, kraus_ops, target: int):
        k = np.concatenate([_mat8(K) for K in kraus_ops])
        check(_lib.sim_dm_apply_kraus(P(self.h), target, k.ctypes.data_as(P), len(kraus_ops)))

    def apply_channel(self, kind: str, p: float, target: int):
        check(_lib.sim_dm_apply_channel(P(self.h), SIM_CHANNELS[kind], float(p), target))

    def probabilities(self, f64: bool = True):
        t = self._torch.empty(2 ** self.n, dtype=self._torch.float64 if f64 else self._torch.float32,
                              device=self.tensor.device)
        check(_lib.sim_dm_probabilities(P(self.h), P(t.data_ptr()), SIM_F64 if f64 else SIM_F32))
        sim_synchronize(self.h)
        return t.cpu().numpy()

    def trace(self) -> float:
        return _dm_scalar(_lib.sim_dm_trace, self.h)

    def purity(self) -> float:
        return _dm_scalar(_lib.sim_dm_purity, self.h)

    def expect_z_sum(self) -> float:
        return _dm_scalar(_lib.sim_dm_expect_z_sum, self.h)

    def measure(self, qubit: int, seed: int, draw: int = 0):
        m = ctypes.c_int()
        p = ctypes.c_double()
        check(_lib.sim_dm_measure(P(self.h), qubit, seed, draw, ctypes.byref(m), ctypes.byref(p)))
        return m.value, p.value

    def sample(self, shots: int, seed: int) -> np.ndarray:
        arr = np.empty(shots, dtype=np.uint64)
        check(_lib.sim_dm_sample(P(self.h), shots, seed, arr.ctypes.data_as(P), 0))
        return arr

    def synchronize(self):
        sim_synchronize(self.h)


# ---------------------------------------------------------------- batches
class BatchOpts(ctypes.Structure):
    _fields_ = [("tile_qubits", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


_sig("sim_batch_create", [_i32, P, P, P, P, ctypes.POINTER(P)])
_sig("sim_batch_create_opts", [_i32, P, P, P, ctypes.POINTER(BatchOpts), P, ctypes.POINTER(P)])
_sig("sim_batch_config", [P, ctypes.POINTER(BatchOpts), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double)])
_sig("sim_batch_run", [P, P, _i32])
_sig("sim_batch_info", [P, P, P, P, P, P])
_sig("sim_batch_destroy", [P])


class Batch:
    """Many independent circuits, each from |0...0>, returning <sum_i Z_i>
    per circuit (one persistent launch replayed from a CUDA graph).
    tile_qubits (11..13, 0 = 13) and ctas_per_sm (0 = as many as fit) set the
    launch configuration (sim_batch_create_opts)."""

    def __init__(self, n_qubits, offsets, gates, stream: int = 0, tile_qubits: int = 0, ctas_per_sm: int = 0):
        self.n = np.ascontiguousarray(n_qubits, dtype=np.int32)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        sg = np.ascontiguousarray(to_sim_gates(gates) if gates.dtype != SIM_GATE_DTYPE else gates,
                                  dtype=SIM_GATE_DTYPE)
        h = P()
        o = BatchOpts(int(tile_qubits), int(ctas_per_sm))
        check(_lib.sim_batch_create_opts(len(self.n), self.n.ctypes.data_as(P), self.offsets.ctypes.data_as(P),
                                         sg.ctypes.data_as(P), ctypes.byref(o), P(stream or CUDA_STREAM_LEGACY),
                                         ctypes.byref(h)))
        self.h = h.value

    def config(self):
        o = BatchOpts()
        fl, sb = ctypes.c_double(), ctypes.c_double()
        check(_lib.sim_batch_config(P(self.h), ctypes.byref(o), ctypes.byref(fl), ctypes.byref(sb)))
        return {"tile_qubits": o.tile_qubits, "ctas_per_sm": o.ctas_per_sm, "alg_flops": fl.value,
                "alg_scratch_bytes": sb.value}

    def run(self) -> np.ndarray:
        out = np.zeros(len(self.n), dtype=np.float64)
        check(_lib.sim_batch_run(P(self.h), out.ctypes.data_as(P), 0))
        return out

    def info(self):
        items, passes, ops, nbytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        grid = ctypes.c_int()
        check(_lib.sim_batch_info(P(self.h), ctypes.byref(items), ctypes.byref(passes), ctypes.byref(ops),
                                  ctypes.byref(nbytes), ctypes.byref(grid)))
        return {"items": items.value, "passes": passes.value, "ops": ops.value, "device_bytes": nbytes.value,
                "grid": grid.value}

    def close(self):
        if getattr(self, "h", None):
            check(_lib.sim_batch_destroy(P(self.h)))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- cost model
_sig("sim_mlp_param_count", [_i32, _i32])
_sig("sim_mlp_create", [_i32, _i32, P, ctypes.POINTER(P)])
_sig("sim_mlp_destroy", [P])
_sig("sim_mlp_set_params", [P, P])
_sig("sim_mlp_get_params", [P, P])
_sig("sim_mlp_forward", [P, P, ctypes.c_int64, P, _i32])
_sig("sim_mlp_loss_grad", [P, P, P, ctypes.c_int64, _i32, P, P])
_sig("sim_mlp_train", [P, P, P, ctypes.c_int64, _i32, ctypes.c_float, _i32, P])
_sig("sim_set_cost_model", [P, P])
_sig("sim_plan_features", [_i32, _i32, P, _sz, _i32, P])
_sig("sim_last_plan", [P, P, _sz, P])

N_FEATURES = 16
N_VARIANTS = 7
VARIANTS = ["per_gate", "staged:12", "staged:13", "fused:3", "fused:4", "fused:5", "fused:6"]


def variant_opts(v: int) -> sim_plan_opts:
    name, _, num = VARIANTS[v].partition(":")
    if name == "fused":
        return plan_opts("fused", fuse_k=int(num))
    return plan_opts(name, tile_qubits=int(num or 0))


def sim_plan_features(n: int, dtype: int, sim_gates: np.ndarray, variant: int):
    """Feature row of the cost model, or None if the variant is not feasible."""
    g = np.ascontiguousarray(sim_gates, dtype=SIM_GATE_DTYPE)
    out = np.zeros(N_FEATURES, dtype=np.float32)
    rc = _lib.sim_plan_features(n, dtype, g.ctypes.data_as(P), len(g), variant, out.ctypes.data_as(P))
    if rc == SIM_EUNSUPPORTED:
        return None
    check(rc)
    return out


class MLP:
    """The plan cost model (parameters live on the GPU)."""

    def __init__(self, d_in: int = N_FEATURES, hidden: int = 64, stream: int = 0):
        self.d_in, self.hidden = d_in, hidden
        self.n_params = _lib.sim_mlp_param_count(d_in, hidden)
        h = P()
        check(_lib.sim_mlp_create(d_in, hidden, P(stream or CUDA_STREAM_LEGACY), ctypes.byref(h)))
        self.h = h.value

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.n_params
        check(_lib.sim_mlp_set_params(P(self.h), t.ctypes.data_as(P)))

    def get_params(self):
        t = np.zeros(self.n_params, dtype=np.float32)
        check(_lib.sim_mlp_get_params(P(self.h), t.ctypes.data_as(P)))
        return t

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(len(X), dtype=np.float32)
        check(_lib.sim_mlp_forward(P(self.h), X.ctypes.data_as(P), len(X), y.ctypes.data_as(P), 0))
        return y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = ctypes.c_float()
        g = np.zeros(self.n_params, dtype=np.float32)
        check(_lib.sim_mlp_loss_grad(P(self.h), X.ctypes.data_as(P), T.ctypes.data_as(P), len(X), 0,
                                     ctypes.byref(loss), g.ctypes.data_as(P)))
        return loss.value, g

    def train(self, X, T, steps: int, lr: float):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = ctypes.c_float()
        check(_lib.sim_mlp_train(P(self.h), X.ctypes.data_as(P), T.ctypes.data_as(P), len(X), steps,
                                 ctypes.c_float(lr), 0, ctypes.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            check(_lib.sim_mlp_destroy(P(self.h)))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# handle -> the MLP object its SIM_PLAN_LEARNED consults: the library keeps
# only the pointer, so the binding holds the Python object (and with it the
# model's device memory) until the handle is destroyed or given another model
_COST_MODELS = {}


def sim_set_cost_model(h: int, mlp):
    check(_lib.sim_set_cost_model(P(h), P(mlp.h if mlp is not None else None)))
    if mlp is None:
        _COST_MODELS.pop(h, None)
    else:
        _COST_MODELS[h] = mlp


def sim_last_plan(h: int):
    n = ctypes.c_size_t()
    check(_lib.sim_last_plan(P(h), None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int32)
    check(_lib.sim_last_plan(P(h), out.ctypes.data_as(P), n.value, ctypes.byref(n)))
    return out
