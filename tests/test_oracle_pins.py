"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's loop: the brute-force checks build the
full 2^n x 2^n operator by Kronecker products (§1.3.2, the U_t embedding),
the gate matrices are pinned by group relations and by scipy's matrix
exponential, and the workloads by their closed forms (App. C, QFT).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from paper_1805_00988_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

I2 = np.eye(2, dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def kron_list(factors):
    """Kronecker product with factors listed for qubit n-1 (left) ... qubit 0 (right)."""
    out = np.array([[1.0 + 0j]])
    for f in factors:
        out = np.kron(out, f)
    return out


def full_operator(n, U, target, controls=()):
    """I + (prod_c |1><1|_c) (x) (U - I)_target as a 2^n x 2^n matrix."""
    fac = []
    for q in range(n - 1, -1, -1):
        if q == target:
            fac.append(U - I2)
        elif q in controls:
            fac.append(P1)
        else:
            fac.append(I2)
    return np.eye(2 ** n, dtype=complex) + kron_list(fac)


def swap_operator(n, a, b, controls=()):
    """SWAP = (II + XX + YY + ZZ)/2 on qubits a, b, optionally controlled."""
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
    Z = np.array([[1, 0], [0, -1]], dtype=complex)
    S = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for Pm in (I2, X, Y, Z):
        fac = []
        for q in range(n - 1, -1, -1):
            fac.append(Pm if q in (a, b) else I2)
        S += kron_list(fac)
    S /= 2
    if not controls:
        return S
    fac = [P1 if q in controls else I2 for q in range(n - 1, -1, -1)]
    Pc = kron_list(fac)
    return np.eye(2 ** n) + Pc @ (S - np.eye(2 ** n))


def gate_full_operator(orc, n, g):
    nm = str(g["name"])
    ctrl = tuple(int(c) for c in g["ctrl"][: int(g["nctrl"])])
    if nm == "swap":
        return swap_operator(n, int(g["target"]), int(g["target2"]), ctrl)
    U = orc.gate_matrix(nm, g["params"], g["mat"])
    return full_operator(n, U, int(g["target"]), ctrl)


# ---------------------------------------------------------------- matrices

def test_gate_matrices_pauli_relations(orc):
    X, Y, Z = (orc.gate_matrix(k) for k in ("x", "y", "z"))
    H, S, T = (orc.gate_matrix(k) for k in ("h", "s", "t"))
    Sdg, Tdg = orc.gate_matrix("sdg"), orc.gate_matrix("tdg")
    np.testing.assert_allclose(X @ Y, 1j * Z, atol=1e-15)
    np.testing.assert_allclose(Y @ Z, 1j * X, atol=1e-15)
    np.testing.assert_allclose(Z @ X, 1j * Y, atol=1e-15)
    np.testing.assert_allclose(H @ H, I2, atol=1e-15)
    np.testing.assert_allclose(H @ X @ H, Z, atol=1e-15)
    np.testing.assert_allclose(S @ S, Z, atol=1e-15)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)
    np.testing.assert_allclose(S @ Sdg, I2, atol=1e-15)
    np.testing.assert_allclose(T @ Tdg, I2, atol=1e-15)
    # Z leaves |0> alone and flips the sign of |1> (gate table, §1.3.2)
    assert Z[0, 0] == 1 and Z[1, 1] == -1


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, math.pi, 5.9])
def test_rotations_are_matrix_exponentials(orc, theta):
    X, Y, Z = (orc.gate_matrix(k) for k in ("x", "y", "z"))
    for name, Pm in (("rx", X), ("ry", Y), ("rz", Z)):
        ref = scipy.linalg.expm(-0.5j * theta * Pm)
        np.testing.assert_allclose(orc.gate_matrix(name, (theta,)), ref, atol=1e-14)
    # P(l) = e^{i l / 2} RZ(l); U3 special cases
    np.testing.assert_allclose(orc.gate_matrix("p", (theta,)),
                               np.exp(0.5j * theta) * orc.gate_matrix("rz", (theta,)), atol=1e-14)
    np.testing.assert_allclose(orc.gate_matrix("u3", (theta, 0.0, 0.0)), orc.gate_matrix("ry", (theta,)),
                               atol=1e-14)
    np.testing.assert_allclose(orc.gate_matrix("u3", (theta, -math.pi / 2, math.pi / 2)),
                               orc.gate_matrix("rx", (theta,)), atol=1e-14)
    # U3(0, 0, l) = P(l)
    np.testing.assert_allclose(orc.gate_matrix("u3", (0.0, 0.0, theta)), orc.gate_matrix("p", (theta,)),
                               atol=1e-14)


def test_u3_unitary_and_euler_form(orc):
    rng = np.random.default_rng(7)
    for _ in range(20):
        th, ph, la = rng.uniform(0, 2 * math.pi, 3)
        U = orc.gate_matrix("u3", (th, ph, la))
        np.testing.assert_allclose(U.conj().T @ U, I2, atol=1e-14)
        # U3 = e^{i(ph+la)/2} RZ(ph) RY(th) RZ(la)
        ref = np.exp(0.5j * (ph + la)) * (orc.gate_matrix("rz", (ph,)) @ orc.gate_matrix("ry", (th,))
                                          @ orc.gate_matrix("rz", (la,)))
        np.testing.assert_allclose(U, ref, atol=1e-14)


def test_explicit_matrix_passes_through(orc):
    rng = np.random.default_rng(3)
    U = C.haar_unitary_2x2(rng)
    g = C.gate("u", 0, mat=U)
    np.testing.assert_array_equal(orc.gate_matrix("u", mat=g["mat"][0]), U)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_every_gate_kind_and_placement_vs_kronecker(orc, n):
    rng = np.random.default_rng(100 + n)
    psi = C.random_state(n, seed=n)
    for name in C.GATE_NAMES:
        if name == "swap" and n < 2:
            continue
        for _ in range(6):
            qs = rng.permutation(n)
            used = 2 if name == "swap" else 1
            nc = int(rng.integers(0, min(2, n - used) + 1))
            g = C.gate(name, int(qs[0]), controls=tuple(int(c) for c in qs[used:used + nc]),
                       params=tuple(rng.uniform(0, 2 * math.pi, 3)),
                       mat=C.haar_unitary_2x2(rng), target2=int(qs[1]) if name == "swap" else -1)
            got = orc.apply_circuit(psi, g)
            ref = gate_full_operator(orc, n, g[0]) @ psi
            np.testing.assert_allclose(got, ref, atol=1e-14, rtol=0)


def test_random_circuit_vs_kronecker_product(orc):
    n = 6
    g = C.random_gates(n, 60, seed=11)
    psi = C.random_state(n, seed=12)
    M = np.eye(2 ** n, dtype=complex)
    for k in range(len(g)):
        M = gate_full_operator(orc, n, g[k]) @ M
    np.testing.assert_allclose(orc.apply_circuit(psi, g), M @ psi, atol=1e-13, rtol=0)


def test_tensor_product_order(orc):
    # §1.3.1: |1> (x) |0> = |10> = |2>; with qubit t = bit t, X on qubit 1 of |00> gives |2>
    psi = orc.apply_circuit(orc.basis_state(2, 0), C.gate("x", 1))
    assert psi[2] == 1 and np.count_nonzero(psi) == 1


def test_algorithm1_operand_order(orc):
    # Alg. 1: v_a <- G00 v_a + G01 v_b ; v_b <- G10 v_a + G11 v_b, with old values
    U = np.array([[1 + 2j, 3 - 1j], [0.5j, -2 + 0.25j]])
    psi = np.array([2 - 1j, 0.5 + 3j])
    got = orc.apply_circuit(psi, C.gate("u", 0, mat=U))
    np.testing.assert_allclose(got, U @ psi, atol=1e-15)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 4, 9])
def test_hadamard_layer_closed_form(orc, n):
    hs = C.concat([C.gate("h", q) for q in range(n)])
    psi = orc.apply_circuit(orc.basis_state(n, 0), hs)
    np.testing.assert_allclose(psi, np.full(2 ** n, 2 ** (-n / 2)), atol=1e-15)
    a = (2 ** n) // 3
    psi = orc.apply_circuit(orc.basis_state(n, a), hs)
    x = np.arange(2 ** n)
    sign = np.array([(-1) ** bin(a & int(v)).count("1") for v in x])
    np.testing.assert_allclose(psi, sign * 2 ** (-n / 2), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 10])
def test_qft_closed_form(orc, n):
    N = 2 ** n
    for j in (0, 1, N // 3, N - 1):
        psi = orc.apply_circuit(orc.basis_state(n, j), C.qft(n))
        k = np.arange(N)
        ref = np.exp(2j * np.pi * j * k / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, ref, atol=1e-13)


def bitrev(j, n):
    return int(format(j, "0%db" % n)[::-1], 2)


@pytest.mark.parametrize("n", [2, 5, 7])
def test_paper_qft_is_fourier_of_bit_reversed_input(orc, n):
    N = 2 ** n
    for j in (1, N // 3, N - 2):
        psi = orc.apply_circuit(orc.basis_state(n, j), C.qft_paper(n))
        k = np.arange(N)
        ref = np.exp(2j * np.pi * bitrev(j, n) * k / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, ref, atol=1e-13)


def test_ghz_and_bell(orc):
    n = 7
    g = C.concat([C.gate("h", 0)] + [C.gate("x", q + 1, controls=(q,)) for q in range(n - 1)])
    psi = orc.apply_circuit(orc.basis_state(n, 0), g)
    ref = np.zeros(2 ** n, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15)
    # Bell state (|00> + |11>)/sqrt(2) of §1.3.1
    psi = orc.apply_circuit(orc.basis_state(2, 0), C.concat([C.gate("h", 0), C.gate("x", 1, controls=(0,))]))
    np.testing.assert_allclose(psi, np.array([1, 0, 0, 1]) / math.sqrt(2), atol=1e-15)


def test_bernstein_vazirani_worked_example(orc):
    fx = dict(line.split() for line in open(os.path.join(GOLDEN, "bernstein_vazirani.txt"))
              if line.strip() and not line.startswith("#"))
    n, a, shots, expect = int(fx["n"]), int(fx["a"]), int(fx["samples"]), int(fx["expected_outcome"])
    psi = orc.apply_circuit(orc.basis_state(n, 0), C.bernstein_vazirani(n, a))
    p = orc.probabilities(psi)
    assert abs(p[a] - 1.0) < 1e-12
    s = orc.sample(psi, shots, seed=2018)
    assert np.all(s == expect)


# ---------------------------------------------------------------- invariants

def test_norm_preserved_and_inverse_returns(orc):
    n = 9
    g = C.random_gates(n, 300, seed=5)
    psi = C.random_state(n, seed=6)
    out = orc.apply_circuit(psi, g)
    assert abs(orc.norm2(out) - 1.0) < 1e-13
    back = orc.apply_circuit(out, C.inverse(g))
    np.testing.assert_allclose(back, psi, atol=1e-13)


def test_haar_cz_circuit_norm(orc):
    g = C.haar_cz(n=8, depth=6, seed=9)
    psi = orc.apply_circuit(orc.basis_state(8, 0), g)
    assert abs(orc.norm2(psi) - 1.0) < 1e-13
    back = orc.apply_circuit(psi, C.inverse(g))
    assert abs(back[0] - 1.0) < 1e-13


@pytest.mark.parametrize("name,ctrls", [("x", 0), ("x", 1), ("x", 2), ("swap", 0), ("swap", 1)])
def test_permutations_bit_exact(orc, name, ctrls):
    n = 6
    rng = np.random.default_rng(21)
    psi = C.random_state(n, seed=22)
    for _ in range(10):
        qs = [int(v) for v in rng.permutation(n)]
        if name == "x":
            t, cs = qs[0], qs[1:1 + ctrls]
            g = C.gate("x", t, controls=cs)
            idx = np.arange(2 ** n)
            cm = sum(1 << c for c in cs)
            src = np.where((idx & cm) == cm, idx ^ (1 << t), idx)
        else:
            a, b, cs = qs[0], qs[1], qs[2:2 + ctrls]
            g = C.gate("swap", a, controls=cs, target2=b)
            idx = np.arange(2 ** n)
            cm = sum(1 << c for c in cs)
            differ = ((idx >> a) & 1) != ((idx >> b) & 1)
            src = np.where(((idx & cm) == cm) & differ, idx ^ ((1 << a) | (1 << b)), idx)
        got = orc.apply_circuit(psi, g)
        assert np.array_equal(got, psi[src])       # bit-exact


# ---------------------------------------------------------------- measurement

def test_probabilities_and_norm(orc):
    psi = C.random_state(10, seed=31) * 1.7
    p = orc.probabilities(psi)
    np.testing.assert_allclose(p, np.abs(psi) ** 2, rtol=1e-15)
    assert abs(orc.norm2(psi) - 1.7 ** 2) < 1e-12


def test_single_qubit_measure_definition(orc):
    # §1.3.3: alpha|0> + beta|1>: p(0) = |alpha|^2, post-state |0> or |1>
    alpha, beta = 0.6, 0.8j
    psi = np.array([alpha, beta])
    ones = 0
    draws = 4000
    for d in range(draws):
        m, p, post = orc.measure(psi, 0, seed=77, draw=d)
        if m == 0:
            assert abs(p - 0.36) < 1e-15
            np.testing.assert_allclose(post, [1, 0], atol=1e-15)
        else:
            assert abs(p - 0.64) < 1e-15
            np.testing.assert_allclose(post, [0, 1j], atol=1e-15)
        ones += m
    sigma = math.sqrt(draws * 0.64 * 0.36)
    assert abs(ones - 0.64 * draws) < 4 * sigma


def test_multi_qubit_collapse_projector(orc):
    n, q = 6, 3
    psi = C.random_state(n, seed=41)
    m, p, post = orc.measure(psi, q, seed=5, draw=0)
    proj = full_operator(n, P1 if m == 1 else P0, q) - 0 * I2[0, 0]
    # full_operator(n, P, q) = I + (P - I) on qubit q = the projector embedded
    ref = proj @ psi
    pref = np.vdot(ref, ref).real
    assert abs(p - pref) < 1e-14
    np.testing.assert_allclose(post, ref / math.sqrt(pref), atol=1e-14)


def test_sampling_distribution_and_support(orc):
    n = 5
    psi = C.random_state(n, seed=51)
    psi[[3, 17]] = 0                    # zero-probability outcomes are never drawn
    psi /= np.linalg.norm(psi)
    shots = 200000
    s = orc.sample(psi, shots, seed=99)
    assert not np.any((s == 3) | (s == 17))
    counts = np.bincount(s.astype(np.int64), minlength=2 ** n)
    p = np.abs(psi) ** 2
    m = p > 0
    chi2 = np.sum((counts[m] - shots * p[m]) ** 2 / (shots * p[m]))
    dof = int(m.sum()) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    # the state is unchanged and sampling is reproducible
    np.testing.assert_array_equal(orc.sample(psi, 1000, seed=99), s[:1000])


def test_sampling_two_outcomes_follows_uniform_draw(orc):
    psi = np.array([0.5, math.sqrt(0.75)])
    s = orc.sample(psi, 1000, seed=3)
    u = np.array([orc.uniform(3, k) for k in range(1000)])
    # inverse CDF: outcome 0 exactly when u < p0 (away from the boundary)
    assert np.array_equal(s == 0, u < 0.25)


def test_splitmix64_published_vectors(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for st, out in rows:
        assert orc.splitmix64(int(st, 16)) == int(out, 16)
    u = [orc.uniform(1234, k) for k in range(20000)]
    assert 0.0 <= min(u) and max(u) < 1.0
    assert abs(np.mean(u) - 0.5) < 0.01


def test_expect_z_sum(orc):
    n = 7
    assert abs(orc.expect_z_sum(orc.basis_state(n, 0)) - n) < 1e-15
    assert abs(orc.expect_z_sum(orc.basis_state(n, 2 ** n - 1)) + n) < 1e-15
    th = np.linspace(0.1, 3.0, n)
    g = C.concat([C.gate("ry", q, params=(th[q],)) for q in range(n)])
    psi = orc.apply_circuit(orc.basis_state(n, 0), g)
    assert abs(orc.expect_z_sum(psi) - np.sum(np.cos(th))) < 1e-13


def test_variational_single_layer_closed_form(orc):
    # one layer of RY, RZ then the CZ ring: RZ and CZ are diagonal, so
    # <Z_i> = cos(theta_i) and <sum Z> = sum_i cos(theta_i)
    rng = np.random.default_rng(8)
    n = 8
    g = C.variational_layered(n, 1, rng)
    psi = orc.apply_circuit(orc.basis_state(n, 0), g)
    th = g["params"][g["name"] == "ry"][:, 0]
    assert abs(orc.expect_z_sum(psi) - np.sum(np.cos(th))) < 1e-13


def test_infidelity(orc):
    a = C.random_state(6, seed=1)
    assert abs(orc.infidelity(a, a)) < 1e-15
    assert abs(orc.infidelity(a, np.exp(0.7j) * 3 * a)) < 1e-14
    b = np.zeros_like(a)
    b[0] = 1
    c = np.zeros_like(a)
    c[1] = 1
    assert abs(orc.infidelity(b, c) - 1.0) < 1e-15


def test_invalid_gates_rejected(orc):
    psi = orc.basis_state(3, 0)
    for g in (C.gate("x", 3), C.gate("x", 0, controls=(0,)), C.gate("x", 0, controls=(1, 1)),
              C.gate("swap", 1, target2=1)):
        with pytest.raises(ValueError):
            orc.apply_circuit(psi, g)


def test_state_memory_sizes_of_section_2_1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "state_memory.txt"))
            if l.strip() and not l.startswith("#")]
    for n, nbytes in rows:
        assert (2 ** int(n)) * np.dtype(np.complex64).itemsize == int(nbytes)
