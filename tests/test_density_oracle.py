"""Pins of the density-matrix oracle (oracle/density.py) against what the
mathematics fixes, none of them re-typing its code:

* gates on a pure state: |psi><psi| evolves into |G psi><G psi|, with the
  state-vector oracle (itself pinned by brute-force Kronecker operators)
  giving G psi;
* channels: the element-wise closed forms of Nielsen & Chuang §8.3 for
  depolarizing, amplitude damping, phase damping, bit flip and phase flip,
  their action on one factor of a product state, trace preservation,
  Hermiticity and positivity of random CPTP maps, composition of
  depolarizing maps, the maximally mixed state;
* measurement (§1.3.3) against the state-vector oracle on pure states and
  on a Bell state; sampling against a hand-computed inverse CDF and against
  the state-vector sampler; <sum Z> and purity closed forms.
"""
import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C


@pytest.fixture(scope="module")
def dm(orc):
    from oracle import density
    return density


def random_rho(rng, d, rank=None):
    """A random density matrix of dimension d: G G^dagger / tr, G Ginibre."""
    r = rank or d
    G = rng.standard_normal((d, r)) + 1j * rng.standard_normal((d, r))
    rho = G @ G.conj().T
    return rho / np.trace(rho).real


def test_gates_on_pure_state(orc, dm):
    for n, seed in ((1, 1), (3, 2), (5, 3)):
        g = C.random_gates(n, 40, seed=seed)
        psi = C.random_state(n, seed=seed + 10)
        got = dm.apply_circuit(dm.pure(psi), g)
        ref = dm.pure(orc.apply_circuit(psi, g))
        assert np.max(np.abs(got - ref)) < 1e-13


def test_gates_on_mixed_state_are_a_mixture(orc, dm):
    """A mixture sum_k w_k |psi_k><psi_k| evolves term by term."""
    rng = np.random.default_rng(4)
    n = 4
    g = C.random_gates(n, 30, seed=7)
    psis = [C.random_state(n, seed=20 + k) for k in range(3)]
    w = rng.dirichlet(np.ones(3))
    rho = sum(wk * dm.pure(p) for wk, p in zip(w, psis))
    ref = sum(wk * dm.pure(orc.apply_circuit(p, g)) for wk, p in zip(w, psis))
    assert np.max(np.abs(dm.apply_circuit(rho, g) - ref)) < 1e-13


@pytest.mark.parametrize("p", [0.0, 0.1, 0.5, 1.0])
def test_named_channels_closed_forms(dm, p):
    rng = np.random.default_rng(int(p * 100) + 1)
    r = random_rho(rng, 2)
    a, b, c, d = r[0, 0], r[0, 1], r[1, 0], r[1, 1]
    s = np.sqrt(1.0 - p)
    forms = {
        "depolarizing": (1 - p) * r + p * np.eye(2) / 2,
        "amplitude_damping": np.array([[a + p * d, s * b], [s * c, (1 - p) * d]]),
        "phase_damping": np.array([[a, s * b], [s * c, d]]),
        "bit_flip": np.array([[(1 - p) * a + p * d, (1 - p) * b + p * c],
                              [(1 - p) * c + p * b, (1 - p) * d + p * a]]),
        "phase_flip": np.array([[a, (1 - 2 * p) * b], [(1 - 2 * p) * c, d]]),
    }
    for kind, want in forms.items():
        got = dm.apply_kraus(r, dm.kraus(kind, p), 0)
        assert np.max(np.abs(got - want)) < 1e-15, kind


@pytest.mark.parametrize("t", [0, 1, 2])
def test_channel_acts_on_one_factor(dm, t):
    """E on qubit t of rho2 (x) rho1 (x) rho0 (qubit 2 the leftmost factor)
    replaces rho_t by E(rho_t), from the amplitude-damping closed form."""
    rng = np.random.default_rng(9)
    rs = [random_rho(rng, 2) for _ in range(3)]
    g = 0.3
    r = rs[t]
    rs_out = list(rs)
    rs_out[t] = np.array([[r[0, 0] + g * r[1, 1], np.sqrt(1 - g) * r[0, 1]],
                          [np.sqrt(1 - g) * r[1, 0], (1 - g) * r[1, 1]]])
    rho = np.kron(rs[2], np.kron(rs[1], rs[0]))
    want = np.kron(rs_out[2], np.kron(rs_out[1], rs_out[0]))
    got = dm.apply_kraus(rho, dm.kraus("amplitude_damping", g), t)
    assert np.max(np.abs(got - want)) < 1e-15


def test_random_cptp_preserves_trace_hermiticity_positivity(dm):
    rng = np.random.default_rng(5)
    n = 3
    rho = random_rho(rng, 8)
    for t in range(n):
        # Kraus operators from a random isometry V (6 x 2): sum K^dag K = V^dag V = I
        G = rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))
        V, _ = np.linalg.qr(G)
        ks = [V[2 * i:2 * i + 2, :] for i in range(3)]
        assert np.max(np.abs(sum(K.conj().T @ K for K in ks) - np.eye(2))) < 1e-14
        out = dm.apply_kraus(rho, ks, t)
        assert abs(np.trace(out).real - 1.0) < 1e-14
        assert np.max(np.abs(out - out.conj().T)) < 1e-15
        assert np.min(np.linalg.eigvalsh(out)) > -1e-14


def test_depolarizing_composes(dm):
    rng = np.random.default_rng(6)
    rho = random_rho(rng, 4)
    p1, p2 = 0.2, 0.35
    two = dm.apply_kraus(dm.apply_kraus(rho, dm.kraus("depolarizing", p1), 1), dm.kraus("depolarizing", p2), 1)
    one = dm.apply_kraus(rho, dm.kraus("depolarizing", 1 - (1 - p1) * (1 - p2)), 1)
    assert np.max(np.abs(two - one)) < 1e-15


def test_full_depolarizing_gives_maximally_mixed(orc, dm):
    n = 3
    psi = C.random_state(n, seed=3)
    rho = dm.pure(psi)
    assert abs(dm.purity(rho) - 1.0) < 1e-13
    for t in range(n):
        rho = dm.apply_kraus(rho, dm.kraus("depolarizing", 1.0), t)
    assert np.max(np.abs(rho - np.eye(8) / 8)) < 1e-15
    assert abs(dm.purity(rho) - 1 / 8) < 1e-15
    assert abs(dm.expect_z_sum(rho)) < 1e-15
    assert abs(dm.trace(rho) - 1.0) < 1e-15


def test_expect_z_and_purity_of_product_state(dm):
    rng = np.random.default_rng(8)
    rs = [random_rho(rng, 2) for _ in range(3)]
    rho = np.kron(rs[2], np.kron(rs[1], rs[0]))
    want = sum((r[0, 0] - r[1, 1]).real for r in rs)
    assert abs(dm.expect_z_sum(rho) - want) < 1e-14
    assert abs(dm.purity(rho) - np.prod([np.trace(r @ r).real for r in rs])) < 1e-14


def test_measure_pure_matches_state_oracle(orc, dm):
    n = 4
    for q in range(n):
        for draw in range(3):
            psi = C.random_state(n, seed=q * 10 + draw)
            m, p, post = orc.measure(psi, q, seed=77, draw=draw)
            m2, p2, rho = dm.measure(dm.pure(psi), q, seed=77, draw=draw)
            assert (m, round(p, 12)) == (m2, round(p2, 12))
            assert np.max(np.abs(rho - dm.pure(post))) < 1e-13


def test_measure_bell_state(orc, dm):
    bell = np.zeros(4, dtype=complex)
    bell[0] = bell[3] = 2 ** -0.5
    for draw in range(8):
        m, p, rho = dm.measure(dm.pure(bell), 0, seed=5, draw=draw)
        assert abs(p - 0.5) < 1e-15
        want = np.zeros((4, 4))
        want[3 * m, 3 * m] = 1.0
        assert np.max(np.abs(rho - want)) < 1e-15


def test_sample_weights_inverse_cdf_by_hand(orc):
    p = np.array([0.25, 0.0, 0.5, 0.25])
    shots = orc.sample_weights(p, 400, seed=13)
    for s, j in enumerate(shots):
        u = orc.uniform(13, s)
        want = 0 if u < 0.25 else (2 if u < 0.75 else 3)
        assert j == want
    assert 1 not in set(shots.tolist())


def test_sample_pure_matches_state_sampler(orc, dm):
    n = 6
    psi = C.random_state(n, seed=31)
    a = dm.sample(dm.pure(psi), 3000, seed=4)
    b = orc.sample(psi, 3000, seed=4)
    # the two weights may differ in the last bit (a fused multiply-add in the
    # C oracle); only a shot on a prefix boundary can then move
    assert np.count_nonzero(a != b) <= 2
