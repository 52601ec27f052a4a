"""The fused plan on complex128 states: blocks of 4 qubits, each block's
unitary built in FP64 and applied on the FP16 tensor cores as exact integer
arithmetic on balanced 8-bit digit planes of the state and of the block
matrix (47 bits relative to each row's and each column's largest entry).

Tolerances (the required bounds for complex128): infidelity <= 1e-12 and
|psi - ref| <= 1e-11 max|ref| element-wise.  Derivation: each block keeps 47
bits of every row and column in fixed point (2^-47 = 7e-15 of its largest
entry) and drops the digit products of levels 6 and up (at most about 2^-42
of the row and column maxima, with random signs far less); a K = 32 dot
product then errs by about 1e-13 of its largest term, and over a few hundred
blocks that random walk stays under 1e-11 of max|ref|, the infidelity near
its square."""
import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as S
    return S


def check(orc, got, ref):
    amax = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= 1e-11 * amax, err
    # the infidelity is scale-free; both states are divided by max|ref| so
    # that its FP64 sums neither overflow nor underflow at norms of 1e+-150
    assert orc.infidelity(ref / amax, got / amax) <= 1e-12


def run(gsim, n, g, psi):
    st = gsim.State(n, "c128")
    st.load(psi)
    st.apply(g, plan="fused", fuse_k=4)
    got = st.state()
    st.close()
    return got


@pytest.mark.parametrize("qubits", [(0, 1, 2, 3), (10, 11, 12, 13), (0, 5, 9, 13), (2, 3, 7, 11)])
def test_c128_fused_block_placements(gsim, orc, qubits):
    """One block per placement at 14 qubits: the block's qubits are the
    lowest tile bits, the highest, or spread (runs of 2 KB to 256 KB)."""
    n = 14
    q = list(qubits)
    g = C.concat([C.gate("h", t) for t in q] +
                 [C.gate("z", q[i + 1], controls=(q[i],)) for i in range(3)] +
                 [C.gate("rx", t, params=(0.3 + 0.1 * i,)) for i, t in enumerate(q)] +
                 [C.gate("x", q[3], controls=(q[0], q[1])), C.gate("t", q[2]),
                  C.gate("u3", q[1], params=(0.4, 1.1, -0.7))])
    assert gsim.sim_plan_describe(n, 1, gsim.to_sim_gates(g), gsim.plan_opts("fused", fuse_k=4))[1] == 1
    psi = C.random_state(n, seed=sum(q))
    check(orc, run(gsim, n, g, psi), orc.apply_circuit(psi, g))


@pytest.mark.parametrize("n", [11, 12, 16, 20])
def test_c128_fused_random_circuits(gsim, orc, n):
    """Every gate kind with up to two controls and the QFT; 11 qubits is a
    single tile, 20 qubits many tiles per CTA."""
    g = C.concat([C.random_gates(n, 200, seed=n), C.qft(n)])
    psi = C.random_state(n, seed=n + 1)
    check(orc, run(gsim, n, g, psi), orc.apply_circuit(psi, g))


def test_c128_fused_haar_cz_24q(gsim, orc):
    n = 24
    g = C.haar_cz(n, 6, seed=1234)
    st = gsim.State(n, "c128")
    st.apply(g, plan="fused", fuse_k=4)
    got = st.state()
    st.close()
    check(orc, got, orc.apply_circuit(orc.basis_state(n, 0), g))


@pytest.mark.parametrize("case", ["norm1e-150", "norm1e150", "norm1e-295", "span2^-300..2^0", "zero"])
def test_c128_fused_state_magnitudes(gsim, orc, case):
    """Each row is put in fixed point relative to its own largest component,
    so states of any magnitude, and rows whose entries span hundreds of
    binades, keep the same relative precision; the zero state stays zero."""
    n = 14
    g = C.haar_cz(n, 3, seed=21)
    if case == "zero":
        psi = np.zeros(2 ** n, dtype=np.complex128)
    elif case.startswith("span"):
        rng = np.random.default_rng(4)
        psi = np.exp2(rng.uniform(-300.0, 0.0, 2 ** n)) * np.exp(2j * np.pi * rng.uniform(0.0, 1.0, 2 ** n))
    else:
        # 1e-295: row exponents near the bottom of the FP64 range (results that
        # would fall below the normal range are flushed to zero)
        psi = C.random_state(n, seed=6) * {"norm1e-150": 1e-150, "norm1e150": 1e150, "norm1e-295": 1e-295}[case]
    got = run(gsim, n, g, psi)
    ref = orc.apply_circuit(psi, g)
    if case == "zero":
        assert not np.any(got)
    else:
        check(orc, got, ref)


def test_c128_fused_non_unitary_gates(gsim, orc):
    """Block matrices need not be unitary: each column of W is put in fixed
    point relative to its own largest entry."""
    n = 13
    rng = np.random.default_rng(17)
    parts = []
    for layer in range(3):
        for q in range(4):
            parts.append(C.gate("u", q, mat=C.haar_unitary_2x2(rng) * (8.0 if layer == 1 else 1e-3)))
        parts.append(C.gate("z", 1, controls=(0,)))
    g = C.concat(parts)
    psi = C.random_state(n, seed=3)
    check(orc, run(gsim, n, g, psi), orc.apply_circuit(psi, g))


def test_c128_fused_rejects_other_block_sizes(gsim):
    st = gsim.State(12, "c128")
    with pytest.raises(gsim.SimError) as e:
        st.apply(C.qft(12), plan="fused", fuse_k=5)
    assert e.value.status == gsim.SIM_EUNSUPPORTED
    st.close()
