"""CPU-side checks of the boundary: the library builds, loads without a GPU,
and exports every entry point include/qsim_gb300.h declares; the Python
binding's struct layout matches the header."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_00988_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char \*|void)\s*\*?\s*(sim_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_paper_api():
    names = declared_functions()
    for required in ("sim_create", "sim_apply_gate", "sim_apply_circuit", "sim_probabilities",
                     "sim_measure", "sim_sample", "sim_norm", "sim_expect_z_sum"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_without_gpu(lib):
    lib.sim_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sim_version()
    lib.sim_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.sim_last_error(), bytes)


def test_invalid_arguments_rejected_before_cuda(lib):
    h = ctypes.c_void_p()
    lib.sim_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.sim_create(0, 0, None, ctypes.byref(h)) == 1          # SIM_EINVAL
    assert lib.sim_create(35, 0, None, ctypes.byref(h)) == 1
    assert lib.sim_create(4, 7, None, ctypes.byref(h)) == 1
    lib.sim_apply_gate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    assert lib.sim_apply_gate(None, None, 0, None, 0) == 1


def test_binding_struct_layout_and_conversion():
    from paper_1805_00988_gb300 import circuits as C
    from paper_1805_00988_gb300 import sim
    assert sim.SIM_GATE_DTYPE.itemsize == 112
    assert sim.SIM_GATE_DTYPE.fields["params"][1] == 24
    assert sim.SIM_GATE_DTYPE.fields["matrix"][1] == 48
    g = C.concat([C.gate("h", 3), C.gate("x", 1, controls=(0, 2)), C.gate("swap", 0, target2=4),
                  C.gate("u3", 2, params=(0.1, 0.2, 0.3))])
    s = sim.to_sim_gates(g)
    assert list(s["kind"]) == [4, 1, 14, 13]
    assert list(s["n_controls"]) == [0, 2, 0, 0]
    assert list(s["controls"][1]) == [0, 2]
    assert s["target2"][2] == 4
    np.testing.assert_array_equal(s["params"][3], [0.1, 0.2, 0.3])
    with pytest.raises(ValueError):
        bad = C.gate("h", 0)
        bad["name"] = "zz"
        sim.to_sim_gates(bad)


def test_gate_kind_codes_match_header():
    from paper_1805_00988_gb300 import sim
    src = open(os.path.join(ROOT, "include", "qsim_gb300.h")).read()
    codes = dict((k.lower(), int(v)) for k, v in re.findall(r"SIM_GATE_(\w+)\s*=\s*(\d+)", src))
    # channel records carry short names in the binding
    short = {"ch_depolarizing": "dep", "ch_amplitude_damping": "adamp", "ch_phase_damping": "pdamp",
             "ch_bit_flip": "bflip", "ch_phase_flip": "pflip"}
    assert {short.get(k, k): v for k, v in codes.items()} == sim.GATE_KINDS
    chan = dict((k.lower(), int(v)) for k, v in re.findall(r"SIM_CHANNEL_(\w+)\s*=\s*(\d+)", src))
    assert chan == sim.SIM_CHANNELS
    for k, v in sim.SIM_CHANNELS.items():
        assert codes["ch_" + k] == 16 + v


def test_channel_kraus_matches_oracle_without_gpu(lib, orc):
    """sim_channel_kraus is host code: its Kraus operators equal the oracle's
    (Nielsen & Chuang §8.3) for every named channel, and bad arguments are
    rejected."""
    from oracle import density
    P = ctypes.c_void_p
    lib.sim_channel_kraus.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
    names = ["depolarizing", "amplitude_damping", "phase_damping", "bit_flip", "phase_flip"]
    for kind, name in enumerate(names):
        for p in (0.0, 0.17, 1.0):
            buf = np.zeros(32)
            cnt = ctypes.c_int()
            assert lib.sim_channel_kraus(kind, p, buf.ctypes.data_as(P), ctypes.byref(cnt)) == 0
            got = [(buf[8 * m:8 * m + 8:2] + 1j * buf[8 * m + 1:8 * m + 8:2]).reshape(2, 2) for m in range(cnt.value)]
            want = density.kraus(name, p)
            assert len(got) == len(want)
            for a, b in zip(got, want):
                assert np.max(np.abs(a - b)) < 1e-15, (name, p)
    buf = np.zeros(32)
    cnt = ctypes.c_int()
    assert lib.sim_channel_kraus(9, 0.1, buf.ctypes.data_as(P), ctypes.byref(cnt)) == 1
    assert lib.sim_channel_kraus(0, 1.5, buf.ctypes.data_as(P), ctypes.byref(cnt)) == 1
    lib.sim_dm_create.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)]
    h = P()
    assert lib.sim_dm_create(18, 0, None, ctypes.byref(h)) == 1
    assert lib.sim_dm_create(0, 0, None, ctypes.byref(h)) == 1
