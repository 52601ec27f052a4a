"""GPU parity of density matrices and noise channels against the FP64
density-matrix oracle (oracle/density.py), through the C ABI.

The GPU holds rho of n qubits as a 2n-qubit register and applies each gate
G on qubit t as G on register qubit t + n and conj(G) on register qubit t,
so every plan of the state-vector path runs it; channels are one 4 x 4
superoperator pass each.  Tolerances are those of the state-vector tests,
element-wise relative to max|rho|: complex128 1e-11; complex64 per-gate and
register tiles 1e-5 (FP32 rounding per gate); complex64 fused blocks 1e-4
(the 3xTF32 / FP16-split bound derived in tests/test_fused.py).
"""
import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as s
    return s


@pytest.fixture(scope="module")
def dm(orc):
    from oracle import density
    return density


def random_rho(n, seed):
    rng = np.random.default_rng(seed)
    d = 1 << n
    G = rng.standard_normal((d, 3)) + 1j * rng.standard_normal((d, 3))
    rho = G @ G.conj().T
    return rho / np.trace(rho).real


TOL = {"c128": 1e-11, "c64": 1e-5, "c64_fused": 1e-4}


def close(got, ref, tol):
    err = np.max(np.abs(got.astype(np.complex128) - ref))
    assert err <= tol * np.max(np.abs(ref)), (err, tol)


PLANS = [("per_gate", {}), ("staged", {}), ("fused", {"fuse_k": 3}), ("fused", {"fuse_k": 4}),
         ("fused", {"fuse_k": 5}), ("fused", {"fuse_k": 6}), ("learned", {})]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("plan,kw", PLANS, ids=[p + str(k.get("fuse_k", "")) for p, k in PLANS])
def test_noisy_circuit_matches_oracle(sim, dm, dt, plan, kw):
    """Random gates (up to two controls, swaps) with random channels between
    them, from a random mixed state; n = 7 (a 14-qubit register: fused
    blocks of k <= 6 span several tiles)."""
    if dt == "c128" and plan == "fused" and kw["fuse_k"] != 4:
        pytest.skip("complex128 fused blocks are 4-qubit")
    n = 7
    g = C.random_noisy(n, 60, seed=11)
    rho0 = random_rho(n, seed=3)
    st = sim.DensityMatrix(n, dt)
    if plan == "learned":
        from paper_1805_00988_gb300 import costmodel
        model, _ = costmodel.load()
        sim.sim_set_cost_model(st.h, model)
        st._model = model
    st.load(rho0)
    st.apply(g, plan=plan, **kw)
    ref = dm.apply_circuit(rho0.astype(np.complex64).astype(np.complex128) if dt == "c64" else rho0, g)
    tol = TOL[dt] if dt == "c128" or plan in ("per_gate", "staged") else TOL["c64_fused"]
    close(st.matrix(), ref, tol)
    st.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_every_channel_on_every_qubit(sim, dm, dt, n):
    """Each named channel and a random non-trace-preserving Kraus map on every
    qubit (column qubit 0, the 16-byte-vector case, included)."""
    rng = np.random.default_rng(n)
    rho = random_rho(n, seed=n + 40)
    st = sim.DensityMatrix(n, dt)
    st.load(rho)
    ref = rho.astype(np.complex64).astype(np.complex128) if dt == "c64" else rho.copy()
    for t in range(n):
        for kind in ("depolarizing", "amplitude_damping", "phase_damping", "bit_flip", "phase_flip"):
            p = float(rng.uniform(0.05, 0.9))
            st.apply_channel(kind, p, t)
            ref = dm.apply_kraus(ref, dm.kraus(kind, p), t)
        ks = [rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)) for _ in range(3)]
        ks = [k * 0.4 for k in ks]
        st.apply_kraus(ks, t)
        ref = dm.apply_kraus(ref, ks, t)
    close(st.matrix(), ref, TOL[dt])
    st.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_observables_match_oracle(sim, dm, orc, dt):
    """Probabilities, trace, purity, <sum Z>, sampling (index-exact on the
    GPU's own rho, up to shots on a prefix boundary) and measurement (outcome,
    probability and post-state) against the oracle."""
    n = 8
    g = C.random_noisy(n, 50, seed=21)
    st = sim.DensityMatrix(n, dt)
    st.apply(g, plan="per_gate")
    rho = st.matrix().astype(np.complex128)
    tol = 1e-12
    np.testing.assert_allclose(st.probabilities(), dm.probabilities(rho), rtol=0, atol=tol)
    assert abs(st.trace() - dm.trace(rho)) < tol
    assert abs(st.purity() - np.sum(np.abs(rho) ** 2)) < tol
    assert abs(st.purity() - dm.purity(rho)) < (1e-6 if dt == "c64" else 1e-12)
    assert abs(st.expect_z_sum() - dm.expect_z_sum(rho)) < 1e-11
    shots = st.sample(20000, seed=9)
    ref_shots = dm.sample(rho, 20000, seed=9)
    assert np.count_nonzero(shots != ref_shots) <= 2
    for q in (0, 3, 7):
        rho = st.matrix().astype(np.complex128)
        m, p = st.measure(q, seed=5, draw=q)
        m2, p2, post = dm.measure(rho, q, seed=5, draw=q)
        assert m == m2 and abs(p - p2) < 1e-12
        close(st.matrix(), post, TOL[dt])
    st.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_pure_state_density_follows_the_state(sim, dm, orc, dt):
    """rho = |psi><psi| (sim_dm_set_pure), gates on rho = the outer product of
    the gates applied to psi; the diagonal samples like the state."""
    n = 6
    psi = C.random_state(n, seed=8)
    g = C.random_gates(n, 80, seed=8)
    s = sim.State(n, dt)
    s.load(psi)
    st = sim.DensityMatrix(n, dt)
    st.set_pure(s)
    close(st.matrix(), dm.pure(s.state().astype(np.complex128)), TOL[dt])
    st.apply(g, plan="per_gate")
    s.apply(g, plan="per_gate")
    ref = dm.pure(orc.apply_circuit(psi.astype(s.np_dtype).astype(np.complex128), g))
    close(st.matrix(), ref, TOL[dt])
    assert abs(st.purity() - 1.0) < (1e-5 if dt == "c64" else 1e-12)
    st.close()
    s.close()


@pytest.mark.parametrize("dt,k", [("c64", 3), ("c64", 6), ("c128", 4)])
def test_fused_plan_absorbs_channels(sim, dm, dt, k):
    """Under the fused plan the channels ride inside the tensor-core blocks
    (no channel pass is launched) and the result still matches the oracle;
    per gate, every channel is its own pass."""
    n = 7
    g = C.noisy_haar_cz(n, 3, seed=5, channels=(("dep", 0.05), ("adamp", 0.1), ("pdamp", 0.07)))
    n_ch = int(np.count_nonzero(np.isin(g["name"], C.CHANNEL_NAMES)))
    rho0 = random_rho(n, seed=12)
    ref = dm.apply_circuit(rho0.astype(np.complex64).astype(np.complex128) if dt == "c64" else rho0, g)
    for plan, kw in (("fused", {"fuse_k": k}), ("per_gate", {})):
        st = sim.DensityMatrix(n, dt)
        st.load(rho0)
        sim.sim_profile_enable(st.h, True)
        st.apply(g, plan=plan, **kw)
        prof = sim.sim_profile_read(st.h)
        launched = prof.get("channel", (0,))[0]
        assert launched == (0 if plan == "fused" else n_ch), (plan, prof)
        tol = TOL["c128"] if dt == "c128" else (TOL["c64_fused"] if plan == "fused" else TOL["c64"])
        close(st.matrix(), ref, tol)
        st.close()


def test_basis_state_and_errors(sim):
    import ctypes
    st = sim.DensityMatrix(3, "c64")
    st.set_basis(5)
    m = st.matrix()
    assert m[5, 5] == 1 and np.count_nonzero(m) == 1
    lib = sim.lib_handle()
    # state-vector calls refuse a density handle and vice versa
    assert lib.sim_norm(ctypes.c_void_p(st.h), ctypes.byref(ctypes.c_double())) == sim.SIM_EINVAL
    assert lib.sim_set_basis_state(ctypes.c_void_p(st.h), 0) == sim.SIM_EINVAL
    with pytest.raises(sim.SimError):
        sim.sim_apply_circuit(st.h, sim.to_sim_gates(C.gate("h", 0)))
    s = sim.State(3, "c64")
    assert lib.sim_dm_trace(ctypes.c_void_p(s.h), ctypes.byref(ctypes.c_double())) == sim.SIM_EINVAL
    # channel records belong to density handles only
    with pytest.raises(sim.SimError):
        s.apply(C.channel("dep", 0, 0.1))
    with pytest.raises(sim.SimError):
        st.apply(C.channel("dep", 3, 0.1))          # qubit out of range
    with pytest.raises(sim.SimError):
        st.apply(C.channel("adamp", 0, 1.5))        # parameter out of [0, 1]
    with pytest.raises(sim.SimError):
        st.apply_channel("depolarizing", 0.1, 3)
    st.close()
    s.close()


def test_full_size_noisy_register(sim, dm):
    """15 qubits (a 30-qubit register, 8 GiB complex64): a noisy Haar/CZ
    circuit through the learned plan against the same circuit in complex128
    through 4-qubit fused blocks (themselves checked against the oracle
    above), element-wise on every entry; trace 1, Hermitian on sampled
    entries, purity below 1."""
    import torch
    from paper_1805_00988_gb300 import costmodel
    n = 15
    g = C.noisy_haar_cz(n, 3, seed=1234)
    a = sim.DensityMatrix(n, "c64")
    model, _ = costmodel.load()
    sim.sim_set_cost_model(a.h, model)
    a.apply(g, plan="learned")
    b = sim.DensityMatrix(n, "c128")
    b.apply(g, plan="fused", fuse_k=4)
    torch.cuda.synchronize()
    assert abs(a.trace() - 1.0) < 1e-5 and abs(b.trace() - 1.0) < 1e-12
    pa, pb = a.purity(), b.purity()
    assert pb < 1.0 and abs(pa - pb) < 1e-5
    ta = a.tensor.view(2 ** n, 2 ** n)
    tb = b.tensor.view(2 ** n, 2 ** n)
    err = 0.0
    for r0 in range(0, 2 ** n, 2048):
        err = max(err, float((ta[r0:r0 + 2048].to(torch.complex128) - tb[r0:r0 + 2048]).abs().max()))
    assert err <= 1e-4 * float(tb.diagonal().abs().max())
    rng = np.random.default_rng(0)
    r = torch.tensor(rng.integers(0, 2 ** n, 4096), device=tb.device)
    c = torch.tensor(rng.integers(0, 2 ** n, 4096), device=tb.device)
    assert float((tb[r, c] - tb[c, r].conj()).abs().max()) <= 1e-12 * float(tb.diagonal().abs().max())
    a.close()
    b.close()


def test_maximum_density_matrix_17_qubits(sim):
    """The largest density matrix (17 qubits: a 34-qubit register, 128 GiB in
    complex64): H on the top qubit and a depolarizing channel (p = 0.2)
    there; the trace is 1, the diagonal 1/2 on |0...0> and |10...0>, and the
    purity that of a Bloch vector of length 1 - p: (1 + (1 - p)^2) / 2."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 140 * 2 ** 30:
        pytest.skip("needs 140 GiB of free device memory")
    n = 17
    import ctypes
    P = ctypes.c_void_p
    h = P()
    lib = sim.lib_handle()
    assert lib.sim_dm_create(n, sim.SIM_C64, P(1), ctypes.byref(h)) == sim.SIM_OK, sim.last_error()
    lib_h = h.value
    try:
        gh = sim.to_sim_gates(C.concat([C.gate("h", n - 1), C.channel("dep", n - 1, 0.2)]))
        sim.sim_dm_apply_circuit(lib_h, gh, sim.plan_opts("per_gate"))
        tr, pu = ctypes.c_double(), ctypes.c_double()
        assert lib.sim_dm_trace(P(lib_h), ctypes.byref(tr)) == sim.SIM_OK
        assert lib.sim_dm_purity(P(lib_h), ctypes.byref(pu)) == sim.SIM_OK
        assert abs(tr.value - 1.0) < 1e-6
        # |+><+| depolarized with p: Bloch vector length 1 - p, purity (1 + (1 - p)^2) / 2
        assert abs(pu.value - (1 + 0.8 ** 2) / 2) < 1e-6
        p = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
        assert lib.sim_dm_probabilities(P(lib_h), P(p.data_ptr()), sim.SIM_F64) == sim.SIM_OK
        torch.cuda.synchronize()
        assert abs(float(p[0]) - 0.5) < 1e-6 and abs(float(p[1 << (n - 1)]) - 0.5) < 1e-6
        assert float(p.sum()) == pytest.approx(1.0, abs=1e-6)
    finally:
        sim.sim_destroy(lib_h)
