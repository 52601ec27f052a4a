"""sim_norm_noalloc: the norm of a caller's state buffer for callers that
cannot allocate device memory when they need it (all free memory held by
another allocator, or no entry into the device allocator allowed).  It uses
only a fixed scratch array compiled into the library.

Checked through the C ABI against sim_norm (the handle-based entry point) on
two calls in a row, within the reduction tolerance of the other tests
(1e-12 absolute on a unit-norm state), for both dtypes.  This file is
collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import build
    build.build()
    from paper_1805_00988_gb300 import sim as S
    lib = S.lib_handle()
    lib.sim_norm_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.sim_norm_noalloc.restype = ctypes.c_int
    return S


@pytest.mark.parametrize("dt,n", [("c64", 17), ("c128", 15), ("c64", 3), ("c64", 23), ("c128", 22)])
def test_noalloc_norm_matches_sim_norm_twice(gsim, orc, dt, n):
    """n = 22, 23: thousands of amplitudes per block, so every thread of the
    partial-sum kernel runs its strided loop many times.  Also against the
    oracle's compensated FP64 sum of the same (copied) state."""
    lib = gsim.lib_handle()
    st = gsim.State(n, dt)
    st.apply(C.random_gates(n, 80, seed=n))
    st.synchronize()
    ref = st.norm2()
    ref_orc = orc.norm2(st.state().astype(np.complex128))
    for _ in range(2):
        out = ctypes.c_double(-1.0)
        rc = lib.sim_norm_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n,
                                  gsim.SIM_C128 if dt == "c128" else gsim.SIM_C64,
                                  ctypes.c_void_p(st.stream_handle), ctypes.byref(out))
        assert rc == gsim.SIM_OK, gsim.last_error()
        assert abs(out.value - ref) <= 1e-12
        assert abs(out.value - ref_orc) <= 1e-12
    st.close()


def test_noalloc_norm_of_a_scaled_state(gsim):
    """A second, different state right after the first: the shared scratch
    holds nothing over from the previous call."""
    import torch
    lib = gsim.lib_handle()
    v = torch.full((2 ** 12,), 0.5 + 0.5j, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    out = ctypes.c_double()
    assert lib.sim_norm_noalloc(ctypes.c_void_p(v.data_ptr()), 12, gsim.SIM_C64, ctypes.c_void_p(1),
                                ctypes.byref(out)) == gsim.SIM_OK
    assert abs(out.value - 2 ** 12 * 0.5) <= 1e-9


def test_noalloc_norm_rejects_sizes_beyond_its_maximum(gsim):
    import torch
    lib = gsim.lib_handle()
    v = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = ctypes.c_double()
    rc = lib.sim_norm_noalloc(ctypes.c_void_p(v.data_ptr()), 35, gsim.SIM_C64, None, ctypes.byref(out))
    assert rc == gsim.SIM_EINVAL
    assert "stated maximum" in gsim.last_error()
