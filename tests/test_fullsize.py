"""The timed workload at its full size: 30 qubits, depth 20, complex64, the
learned plan with the shipped cost model -- the configuration bench.py times.
The oracle cannot re-simulate 900 gates on 2^30 amplitudes in seconds, so it
checks what it can compute from the GPU's final state: the FP64 norm, <sum Z>
and sampled shots (same state, same u_s); the state itself is checked by the
mirror circuit returning to |0...0>."""
import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

N, DEPTH, SEED = 30, 20, 1234


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim
    return sim


@pytest.mark.gpu
def test_timed_workload_observables_match_oracle(gsim, orc):
    from paper_1805_00988_gb300 import costmodel
    model, _ = costmodel.load()
    g = C.haar_cz(N, DEPTH, seed=SEED)
    st = gsim.State(N, "c64")
    gsim.sim_set_cost_model(st.h, model)
    st.apply(g, plan="learned")
    nrm, ez = st.norm2(), st.expect_z_sum()
    shots = st.sample(4096, seed=SEED)
    psi = st.state().astype(np.complex128)

    ref_n = orc.norm2(psi)
    assert abs(nrm - ref_n) <= 1e-12 * ref_n
    assert abs(nrm - 1.0) <= 1e-4
    # both sides sum 2^30 FP64 terms of weight up to 30 in different orders
    assert abs(ez - orc.expect_z_sum(psi)) <= 1e-9 * N

    ref = orc.sample(psi, 4096, seed=SEED)
    diff = np.nonzero(shots != ref)[0]
    if len(diff):
        c = np.cumsum(np.abs(psi) ** 2)
        for s in diff:
            t = orc.uniform(SEED, int(s)) * c[-1]
            assert np.min(np.abs(c - t)) <= 1e-12 * c[-1], (s, shots[s], ref[s])
    assert len(diff) <= 2
    del psi

    st.apply(C.inverse(g), plan="learned")
    a0 = complex(st.tensor[0].item())
    assert abs(abs(a0) ** 2 - 1.0) < 1e-4
    st.close()
