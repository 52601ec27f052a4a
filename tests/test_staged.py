"""The staged (multi-gate tile pass) plan.

CPU: the host planner may reorder gates only where they commute; applying the
circuit in the planner's order with the FP64 oracle must give the original
circuit's state (to rounding).
GPU: staged results against the oracle for every gate kind and placement,
bit-exact permutation circuits, and the workload circuits at full size.
"""
import math

import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

TOL = {"c64": (1e-5, 1e-6), "c128": (1e-11, 1e-12)}


def lowered_swap_parts(g):
    """SWAP(a, b; ctrls) = CNOT(b -> a), X(b; ctrls + a), CNOT(b -> a)."""
    a, b = int(g["target"]), int(g["target2"])
    cs = tuple(int(c) for c in g["ctrl"][: int(g["nctrl"])])
    return [C.gate("x", a, controls=(b,)), C.gate("x", b, controls=cs + (a,)), C.gate("x", a, controls=(b,))]


def apply_in_order(orc, psi, gates, order):
    seen = {}
    out = psi
    for i in order:
        g = gates[i:i + 1]
        if str(g["name"][0]) == "swap":
            k = seen.get(i, 0)
            seen[i] = k + 1
            out = orc.apply_circuit(out, lowered_swap_parts(g[0])[k])
        else:
            out = orc.apply_circuit(out, g)
    return out


@pytest.mark.parametrize("n,dtype,tile", [(11, 0, 11), (12, 0, 11), (13, 0, 13), (14, 0, 12), (16, 0, 13),
                                          (12, 1, 12), (15, 1, 11), (16, 1, 12)])
def test_planner_order_respects_commutation(orc, n, dtype, tile):
    from paper_1805_00988_gb300 import sim
    rng_gates = C.random_gates(n, 300, seed=n * 7 + tile, max_ctrl=2)
    # at most one control on swaps (the oracle takes up to two controls after lowering)
    sw = rng_gates["name"] == "swap"
    rng_gates["nctrl"][sw] = np.minimum(rng_gates["nctrl"][sw], 1)
    gates = C.concat([rng_gates, C.haar_cz(n, 4, seed=3), C.qft(n)])
    passes, ops, lc, order = sim.sim_plan_describe(n, dtype, sim.to_sim_gates(gates),
                                                   sim.plan_opts("staged", tile_qubits=tile))
    # a ramp (one op of four records) can stand for many controlled phases
    assert passes >= 1 and ops >= 1
    # every non-identity gate appears (swaps three times)
    counts = np.bincount(order, minlength=len(gates))
    for k in range(len(gates)):
        if str(gates["name"][k]) == "swap":
            assert counts[k] == 3
        else:
            assert counts[k] in (0, 1)
    psi = C.random_state(n, seed=5)
    ref = orc.apply_circuit(psi, gates)
    got = apply_in_order(orc, psi, gates, order)
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_planner_pass_counts_for_the_workloads():
    from paper_1805_00988_gb300 import sim
    g = C.haar_cz(30, 20, seed=1234)
    passes, ops, lc, order = sim.sim_plan_describe(30, 0, sim.to_sim_gates(g), sim.plan_opts("staged"))
    # 900 gates in far fewer state passes than one per gate
    assert passes <= 40 and len(order) == 900
    g = C.qft(28)
    passes, ops, lc, order = sim.sim_plan_describe(28, 0, sim.to_sim_gates(g), sim.plan_opts("staged"))
    assert passes <= 10


def test_planner_merges_controlled_phase_runs():
    """Runs of controlled phases that share a qubit become SK_RAMP ops (one
    op of (2^RB + 32) / 4 records, the factor tables, padded to stay inside
    one staged chunk), so the App. A QFT's record count is no longer one per
    gate plus the layout changes; a circuit without controlled phases still
    gets exactly that."""
    from paper_1805_00988_gb300 import sim
    g = C.qft_paper(28)
    passes, ops, lc, order = sim.sim_plan_describe(28, 0, sim.to_sim_gates(g), sim.plan_opts("staged"))
    assert len(order) == len(g) and ops != len(order) + lc
    g = C.haar_cz(20, 6, seed=3)
    passes, ops, lc, order = sim.sim_plan_describe(20, 0, sim.to_sim_gates(g), sim.plan_opts("staged"))
    assert ops == len(order) + lc


def test_planner_rejects_small_registers():
    from paper_1805_00988_gb300 import sim
    with pytest.raises(sim.SimError):
        sim.sim_plan_describe(8, 0, sim.to_sim_gates(C.qft(8)), sim.plan_opts("staged"))


# ------------------------------------------------------------------ GPU

@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as S
    return S


def check_state(orc, got, ref, dt):
    rel, inf_tol = TOL[dt]
    got = got.astype(np.complex128)
    err = np.max(np.abs(got - ref))
    assert err <= rel * np.max(np.abs(ref)), (dt, err)
    assert orc.infidelity(ref, got) <= inf_tol


@pytest.mark.gpu
@pytest.mark.parametrize("dt,n,tile", [("c64", 11, 11), ("c64", 12, 12), ("c64", 13, 13), ("c64", 14, 11),
                                       ("c64", 15, 13), ("c64", 17, 12), ("c64", 20, 13),
                                       ("c128", 11, 11), ("c128", 12, 12), ("c128", 14, 11), ("c128", 17, 12)])
def test_staged_random_circuits(gsim, orc, dt, n, tile):
    gates = C.concat([C.random_gates(n, 400, seed=n + tile), C.qft(n)])
    psi = C.random_state(n, seed=n)
    st = gsim.State(n, dt)
    st.load(psi)
    st.apply(gates, plan="staged", tile_qubits=tile)
    start = psi.astype(st.np_dtype).astype(np.complex128)
    check_state(orc, st.state(), orc.apply_circuit(start, gates), dt)
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dt,n,tile", [("c64", 14, 11), ("c64", 16, 13), ("c64", 18, 12), ("c128", 14, 11),
                                       ("c128", 16, 12)])
def test_staged_phase_ramps(gsim, orc, dt, n, tile):
    """Runs of controlled phases sharing one qubit (SK_RAMP): the shared qubit
    and its partners land on register, thread and outer bits in turn, some
    pairs repeat (their factors multiply), and dense gates between the runs
    force new passes and layouts."""
    rng = np.random.default_rng(n + tile)
    parts = [C.gate("h", q) for q in range(n)]
    for _ in range(12):
        q = int(rng.integers(0, n))
        partners = [int(m) for m in rng.choice([m for m in range(n) if m != q], size=int(rng.integers(3, n)),
                                               replace=False)]
        partners += partners[:2]
        for m in partners:
            parts.append(C.gate("p", q, controls=(m,), params=(float(rng.uniform(-math.pi, math.pi)),)))
        for t in rng.choice(n, size=3, replace=False):
            parts.append(C.gate("u3", int(t), params=tuple(float(x) for x in rng.uniform(0, 2 * math.pi, 3))))
    gates = C.concat(parts)
    psi = C.random_state(n, seed=n + 1)
    st = gsim.State(n, dt)
    st.load(psi)
    st.apply(gates, plan="staged", tile_qubits=tile)
    start = psi.astype(st.np_dtype).astype(np.complex128)
    check_state(orc, st.state(), orc.apply_circuit(start, gates), dt)
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_staged_permutations_bit_exact(gsim, orc, dt):
    n = 15
    rng = np.random.default_rng(4)
    parts = []
    for _ in range(200):
        qs = [int(v) for v in rng.permutation(n)]
        if rng.random() < 0.3:
            parts.append(C.gate("swap", qs[0], target2=qs[1], controls=qs[2:2 + int(rng.integers(0, 2))]))
        else:
            parts.append(C.gate("x", qs[0], controls=qs[1:1 + int(rng.integers(0, 3))]))
    gates = C.concat(parts)
    st = gsim.State(n, dt)
    psi = C.random_state(n, seed=8).astype(st.np_dtype)
    st.load(psi)
    st.apply(gates, plan="staged")
    ref = orc.apply_circuit(psi.astype(np.complex128), gates).astype(st.np_dtype)
    assert np.array_equal(st.state().view(np.uint8), ref.view(np.uint8))
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_staged_haar_cz_22q_vs_oracle(gsim, orc, dt):
    n = 22
    g = C.haar_cz(n, 20, seed=1234)
    st = gsim.State(n, dt)
    st.apply(g, plan="staged")
    check_state(orc, st.state(), orc.apply_circuit(orc.basis_state(n, 0), g), dt)
    st.close()


@pytest.mark.gpu
def test_staged_u3_ladder_14q_c128(gsim, orc):
    g = C.u3_cnot_ladder(14, 20, seed=1234)
    st = gsim.State(14, "c128")
    st.apply(g, plan="staged")
    check_state(orc, st.state(), orc.apply_circuit(orc.basis_state(14, 0), g), "c128")
    st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_staged_qft_28q_closed_form(gsim, dt):
    n = 28
    N = 2 ** n
    j = C.random_basis_index(n, seed=1234)
    st = gsim.State(n, dt)
    st.set_basis(j)
    st.apply(C.qft(n), plan="staged")
    rng = np.random.default_rng(6)
    ks = np.concatenate([[0, 1, N - 1], rng.integers(0, N, 4093)])
    got = st.tensor[ks].cpu().numpy().astype(np.complex128)
    ref = np.exp(2j * np.pi * ((j * ks) % N) / N) / math.sqrt(N)
    assert np.max(np.abs(got - ref)) <= (5e-5 if dt == "c64" else 1e-11) / math.sqrt(N)
    st.close()


@pytest.mark.gpu
def test_staged_haar_cz_30q_matches_c128_per_gate(gsim):
    """At the timed size: staged complex64 vs per-gate complex128 (itself
    checked against the oracle up to 22 qubits), infidelity <= 1e-6; and the
    mirror circuit returns to |0...0>."""
    import torch
    n = 30
    g = C.haar_cz(n, 20, seed=1234)
    a = gsim.State(n, "c64")
    a.apply(g, plan="staged")
    b = gsim.State(n, "c128")
    b.apply(g, plan="per_gate")
    ip = torch.zeros((), dtype=torch.complex128, device="cuda")
    for o in range(0, 2 ** n, 1 << 26):
        ip += torch.vdot(a.tensor[o:o + (1 << 26)].to(torch.complex128), b.tensor[o:o + (1 << 26)])
    b.close()
    na = a.norm2()
    assert 1.0 - abs(ip.item()) ** 2 / na <= 1e-6
    a.apply(C.inverse(g), plan="staged")
    a0 = complex(a.tensor[0].item())
    assert abs(abs(a0) ** 2 - 1.0) < 1e-5
    a.close()
