"""The fused plan: gates grouped into blocks of at most k qubits, each block's
2^k x 2^k unitary formed in FP64 on the GPU and applied with split-precision
tensor-core GEMMs (complex64 states): 3xTF32 for k <= 5, FP16 hi / lo parts
of operands scaled by powers of two for k = 6 (the same 22 significant
bits).

Tolerance: infidelity <= 1e-6 (the bound the fused path is held to).
Element-wise: 3xTF32 keeps the low parts of both operands with 11 mantissa
bits and drops lo x lo, so a product carries a relative error of about 2^-21
and a block output (a sum of 2^(k+1) products) about 2^-21 sqrt(2^(k+1));
over B blocks errors add like a random walk, so after a few hundred blocks
|psi - ref| <= 1e-4 max|ref| holds with margin."""
import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C


def test_block_counts_cpu():
    from paper_1805_00988_gb300 import sim
    g = sim.to_sim_gates(C.haar_cz(30, 20, seed=1234))
    desc = {k: sim.sim_plan_describe(30, 0, g, sim.plan_opts("fused", fuse_k=k)) for k in (3, 4, 5, 6)}
    blocks = [desc[k][1] for k in (3, 4, 5, 6)]
    # larger blocks never need more of them
    assert blocks == sorted(blocks, reverse=True)
    assert blocks[-1] < 900
    # the plans the timed runs use (depth 3 after a first group at depth 2);
    # the planner's bound pruning must not change them
    assert desc[5][1] == 73 and desc[6][1] == 54
    # one pass per block by default; with multi-block passes k = 5 pairs blocks
    for k in (3, 4, 5, 6):
        assert desc[k][0] == desc[k][1]
    multi = sim.sim_plan_describe(30, 0, g, sim.plan_opts("fused", fuse_k=5, flags=sim.SIM_FLAG_MULTI_BLOCK_PASSES))
    assert multi[1] == desc[5][1] and multi[0] < multi[1]


def test_planner_concurrent_calls_cpu():
    """The depth-3 block planner spreads its triple search over the host
    thread pool; host threads planning at the same time (the binding releases
    the GIL in the call) get the same plans as one thread alone."""
    import threading
    from paper_1805_00988_gb300 import sim
    circ = {n: sim.to_sim_gates(C.haar_cz(n, 8, seed=n)) for n in (20, 24, 26)}
    ref = {(n, k): sim.sim_plan_describe(n, 0, g, sim.plan_opts("fused", fuse_k=k))[:2]
           for n, g in circ.items() for k in (5, 6)}
    got, errs = [], []

    def worker(seed):
        try:
            for i in range(6):
                n = (20, 24, 26)[(seed + i) % 3]
                k = 5 + (seed + i) % 2
                got.append(((n, k), sim.sim_plan_describe(n, 0, circ[n], sim.plan_opts("fused", fuse_k=k))[:2]))
        except Exception as e:          # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=worker, args=(s,)) for s in range(6)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not errs and len(got) == 36
    for key, r in got:
        assert r == ref[key], (key, r, ref[key])


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as S
    return S


def check(orc, got, ref):
    got = got.astype(np.complex128)
    err = np.max(np.abs(got - ref))
    assert err <= 1e-4 * np.max(np.abs(ref)), err
    assert orc.infidelity(ref, got) <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_fused_single_block(gsim, orc, k):
    """One Hadamard on each of k qubits: one block, one GEMM."""
    n = k + 8
    g = C.concat([C.gate("h", q) for q in range(k)])
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=k)
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=k)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n,k", [(10, 3), (11, 4), (12, 5), (12, 4), (13, 5), (14, 6), (16, 3), (18, 5), (20, 6)])
def test_fused_random_circuits(gsim, orc, n, k):
    g = C.concat([C.random_gates(n, 300, seed=n * 10 + k), C.qft(n)])
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=n)
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=k)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("qubits", [(0, 1, 2, 3, 4, 5), (10, 11, 12, 13, 14, 15), (0, 3, 7, 9, 12, 15),
                                    (1, 2, 5, 8, 11, 14)])
def test_fused_k6_block_placements(gsim, orc, qubits):
    """k = 6 on one block per placement, 16 qubits.  Qubits 0..5: a tile is a
    single 64 KB run and every low tile bit is a block bit (the converters'
    largest bank-spreading permutation); 10..15: 64 runs of 1 KB; the mixed
    placements with and without qubit 0 take the consumer's 16-byte and
    8-byte stores."""
    n = 16
    q = list(qubits)
    g = C.concat([C.gate("h", t) for t in q] +
                 [C.gate("z", q[i + 1], controls=(q[i],)) for i in range(5)] +
                 [C.gate("rx", t, params=(0.3 + 0.1 * i,)) for i, t in enumerate(q)] +
                 [C.gate("x", q[5], controls=(q[0],)), C.gate("t", q[2])])
    blocks = gsim.sim_plan_describe(n, 0, gsim.to_sim_gates(g), gsim.plan_opts("fused", fuse_k=6))[1]
    assert blocks == 1
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=sum(q))
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=6)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_fused_many_tiles_per_cta(gsim, orc, k):
    """24 qubits: every CTA of the persistent kernel streams many tiles, so
    the stage ring and both accumulators wrap around many times."""
    n = 24
    g = C.concat([C.random_gates(n, 120, seed=40 + k), C.haar_cz(n, 2, seed=k)])
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=7 + k)
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=k)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("k", [4, 6])
def test_fused_haar_cz_20q(gsim, orc, k):
    n = 20
    g = C.haar_cz(n, 20, seed=1234)
    st = gsim.State(n, "c64")
    st.apply(g, plan="fused", fuse_k=k)
    check(orc, st.state(), orc.apply_circuit(orc.basis_state(n, 0), g))
    st.close()


@pytest.mark.gpu
def test_fused_rejects_c128_k5_and_small(gsim):
    """complex128 runs 4-qubit blocks only (tests/test_fused_c128.py); a
    register below k + 7 qubits has no full tile."""
    st = gsim.State(12, "c128")
    with pytest.raises(gsim.SimError) as e:
        st.apply(C.qft(12), plan="fused", fuse_k=5)
    assert e.value.status == gsim.SIM_EUNSUPPORTED
    st.close()
    st = gsim.State(9, "c64")
    with pytest.raises(gsim.SimError):
        st.apply(C.qft(9), plan="fused", fuse_k=4)
    st.close()


def wide_range_state(n, lo, hi, seed):
    """Amplitudes of modulus 2^u, u uniform in [lo, hi], with uniform phases."""
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(lo, hi, 1 << n))
    return (mag * np.exp(2j * np.pi * rng.uniform(0.0, 1.0, 1 << n))).astype(np.complex64)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["norm1e-3", "norm1e-6", "span2^-40..2^-5", "norm1e6", "x4", "norm1e-30"])
def test_fused_k6_state_magnitudes(gsim, orc, case):
    """k = 6 splits the state into FP16 parts after scaling it by a power of two
    chosen from its norm (no amplitude exceeds the norm), so the result is the
    plain product of the gates (Algorithm 1, gate after gate) at every scale of
    the input: states of norm 1e-3, 1e-6, 1e-30 and 1e6, a state scaled by 4,
    and one whose amplitudes spread over 2^-40 .. 2^-5.  Element by element
    against the oracle on the same complex64 input, and the infidelity held to
    1e-10 (a 22-bit split gives about 1e-13 per block; the required bound is
    1e-6) -- the precision must not depend on the magnitude."""
    n = 18
    g = C.haar_cz(n, 4, seed=31)
    if case.startswith("span"):
        psi = wide_range_state(n, -40.0, -5.0, seed=5)
    else:
        scale = {"norm1e-3": 1e-3, "norm1e-6": 1e-6, "norm1e6": 1e6, "x4": 4.0, "norm1e-30": 1e-30}[case]
        psi = (C.random_state(n, seed=9).astype(np.complex128) * scale).astype(np.complex64)
    st = gsim.State(n, "c64")
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=6)
    got = st.state().astype(np.complex128)
    ref = orc.apply_circuit(psi.astype(np.complex128), g)
    err = np.max(np.abs(got - ref))
    assert err <= 1e-5 * np.max(np.abs(ref)), err
    assert orc.infidelity(ref, got) <= 1e-10
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("factor", [8.0, 1e-3])
def test_fused_k6_non_unitary_gates(gsim, orc, factor):
    """Gate matrices need not be unitary.  k = 6 scales each block's W by a
    power of two from a bound on its entries (the product of the gates'
    spectral norms), so blocks of gates scaled by 8 (entries up to 8^m) or by
    1e-3 are applied like unitary ones."""
    n = 16
    rng = np.random.default_rng(17)
    parts = []
    for layer in range(2):
        for q in range(6):
            u = C.haar_unitary_2x2(rng) * factor
            parts.append(C.gate("u", q, mat=u))
        parts.append(C.gate("z", 1, controls=(0,)))
    g = C.concat(parts)
    assert gsim.sim_plan_describe(n, 0, gsim.to_sim_gates(g), gsim.plan_opts("fused", fuse_k=6))[1] == 1
    psi = C.random_state(n, seed=3)
    st = gsim.State(n, "c64")
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=6)
    got = st.state().astype(np.complex128)
    ref = orc.apply_circuit(psi.astype(np.complex128), g)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert orc.infidelity(ref, got) <= 1e-10
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("k", [5, 6])
def test_fused_haar_cz_30q_vs_c128(gsim, k):
    import torch
    n = 30
    g = C.haar_cz(n, 20, seed=1234)
    a = gsim.State(n, "c64")
    a.apply(g, plan="fused", fuse_k=k)
    b = gsim.State(n, "c128")
    b.apply(g, plan="staged")
    ip = torch.zeros((), dtype=torch.complex128, device="cuda")
    for o in range(0, 2 ** n, 1 << 26):
        ip += torch.vdot(a.tensor[o:o + (1 << 26)].to(torch.complex128), b.tensor[o:o + (1 << 26)])
    assert 1.0 - abs(ip.item()) ** 2 / a.norm2() <= 1e-6
    a.close()
    b.close()


def test_block_planner_handles_gates_wider_than_k_cpu():
    """A SWAP with two controls lowers to an X with three controls (4 qubits):
    wider than a k = 3 block, it must become its own per-gate step."""
    from paper_1805_00988_gb300 import sim
    g = C.concat([C.gate("swap", 0, target2=1, controls=(2, 3)), C.gate("h", 4),
                  C.random_gates(10, 200, seed=3)])
    blocks = sim.sim_plan_describe(10, 0, sim.to_sim_gates(g), sim.plan_opts("fused", fuse_k=3))[0]
    assert blocks >= 2


@pytest.mark.gpu
@pytest.mark.parametrize("where", ["first", "late"])
def test_fused_wide_gates(gsim, orc, where):
    """A gate wider than k runs as its own per-gate launch between blocks,
    first or deep inside the circuit (then in a later group of the
    plan-as-you-launch pipeline)."""
    n = 12
    wide = C.gate("swap", 0, target2=5, controls=(2, 9))
    g = (C.concat([wide, C.random_gates(n, 100, seed=8)]) if where == "first" else
         C.concat([C.random_gates(n, 150, seed=8), wide, C.random_gates(n, 100, seed=9), wide]))
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=2)
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=3)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [12, 16, 22])
def test_fused_multi_block_passes(gsim, orc, n):
    """Pairs of blocks applied to one tile kept in shared memory: the tile's
    12 qubits hold both blocks' qubits and qubit 0 (loaded with 16-byte async
    copies); every pair, and the single blocks between them, against the
    oracle."""
    g = C.concat([C.haar_cz(n, 8, seed=n), C.random_gates(n, 150, seed=n + 1)])
    opts = dict(plan="fused", fuse_k=5, flags=gsim.SIM_FLAG_MULTI_BLOCK_PASSES)
    passes, blocks = gsim.sim_plan_describe(n, 0, gsim.to_sim_gates(g), gsim.plan_opts(**opts))[:2]
    assert passes < blocks
    st = gsim.State(n, "c64")
    psi = C.random_state(n, seed=n + 2)
    st.load(psi)
    st.apply(g, **opts)
    check(orc, st.state(), orc.apply_circuit(psi.astype(np.complex64).astype(np.complex128), g))
    st.close()
