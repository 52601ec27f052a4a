"""Batched circuits in one persistent launch: <sum Z> per circuit against the
oracle, against the closed form of one-layer variational circuits, bit-
reproducible reruns, and the bounded-wait timeout path (injected on the host).

Tolerance: the states are complex64; <sum Z> = sum_x p_x (n - 2 popcount x)
with |weights| <= n and p accurate to ~1e-6 relative, so |error| <= 1e-5 n."""
import math
import os

import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C


def test_batch_create_rejects_bad_input_cpu():
    from paper_1805_00988_gb300 import sim
    g = C.gate("h", 0)
    with pytest.raises(sim.SimError) as e:
        sim.Batch([0], [0, 1], g)
    assert e.value.status == sim.SIM_EINVAL
    with pytest.raises(sim.SimError):
        sim.Batch([3], [0, 1], C.gate("h", 3))           # target out of range
    with pytest.raises(sim.SimError):
        sim.Batch([3, 3], [0, 1, 0], C.gate("h", 0))     # decreasing offsets
    for bad in ({"tile_qubits": 10}, {"tile_qubits": 14}, {"ctas_per_sm": -1}):
        with pytest.raises(sim.SimError) as e:
            sim.Batch([3], [0, 1], g, **bad)
        assert e.value.status == sim.SIM_EINVAL


def test_batch_planning_for_every_tile_size_cpu():
    """Host planning of circuits below, at and above each tile size ends
    (without a GPU the call then fails at the first CUDA call; with one, the
    batch is built and released)."""
    from paper_1805_00988_gb300 import sim
    ns, offs, parts = mixed_batch(12, seed=8)
    ns[0], ns[1] = 11, 12
    parts[0], parts[1] = C.random_gates(11, 30, seed=1), C.random_gates(12, 30, seed=2)
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    for tile in (11, 12, 13):
        try:
            sim.Batch(ns, offs, C.concat(parts), tile_qubits=tile).close()
        except sim.SimError as e:
            assert e.status in (sim.SIM_ECUDA, sim.SIM_ENOMEM), e


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as S
    return S


def oracle_expz(orc, n, gates):
    return orc.expect_z_sum(orc.apply_circuit(orc.basis_state(n, 0), gates))


@pytest.mark.gpu
def test_batch_mixed_sizes_and_kinds(gsim, orc):
    rng = np.random.default_rng(3)
    ns, parts = [], []
    for i in range(40):
        n = int(rng.integers(2, 18))
        if i % 3 == 0:
            g = C.random_gates(n, 60, seed=i)
        else:
            g = C.variational_layered(n, int(rng.integers(1, 5)), rng)
        ns.append(n)
        parts.append(g)
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    b = gsim.Batch(ns, offs, C.concat(parts))
    got = b.run()
    for i, (n, g) in enumerate(zip(ns, parts)):
        assert abs(got[i] - oracle_expz(orc, n, g)) <= 1e-5 * n, (i, n)
    # reruns are bit-identical
    assert np.array_equal(b.run(), got)
    b.close()


@pytest.mark.gpu
def test_batch_one_layer_closed_form_full_size(gsim):
    """4096 circuits of 8..20 qubits, one RY/RZ layer + CZ ring:
    <sum Z> = sum_i cos(theta_i) exactly (RZ and CZ are diagonal)."""
    ns, offs, g = C.variational(4096, 8, 20, 1, 1, seed=77)
    b = gsim.Batch(ns, offs, g)
    got = b.run()
    th = g["params"][:, 0]
    ref = np.array([np.sum(np.cos(th[offs[i]:offs[i + 1]][g["name"][offs[i]:offs[i + 1]] == "ry"]))
                    for i in range(len(ns))])
    assert np.max(np.abs(got - ref) / ns) <= 1e-5
    b.close()


@pytest.mark.gpu
def test_batch_variational_4096_sampled_vs_oracle(gsim, orc):
    """The timed batch (4096 circuits, 8..20 qubits, 4..12 layers): a seeded
    sample of circuits (including the largest ones) against the oracle."""
    ns, offs, g = C.variational(4096, 8, 20, 4, 12, seed=1234)
    b = gsim.Batch(ns, offs, g)
    got = b.run()
    rng = np.random.default_rng(9)
    pick = list(rng.choice(4096, 24, replace=False)) + list(np.nonzero(ns == 20)[0][:3])
    for i in pick:
        gi = g[offs[i]:offs[i + 1]]
        assert abs(got[i] - oracle_expz(orc, int(ns[i]), gi)) <= 1e-5 * ns[i], (i, ns[i])
    b.close()


@pytest.mark.gpu
def test_batch_wait_timeout_is_reported(gsim, orc):
    """A dependency that is never published (injected on the host) makes the
    bounded device wait give up: SIM_ETIMEOUT, and the context stays usable."""
    ns, offs, g = C.variational(8, 15, 16, 2, 3, seed=5)
    os.environ["QSIM_INJECT_BATCH_STALL"] = "1"
    try:
        b = gsim.Batch(ns, offs, g)
    finally:
        del os.environ["QSIM_INJECT_BATCH_STALL"]
    with pytest.raises(gsim.SimError) as e:
        b.run()
    assert e.value.status == gsim.SIM_ETIMEOUT
    b.close()
    b = gsim.Batch(ns, offs, g)
    got = b.run()
    gi = g[offs[0]:offs[1]]
    assert abs(got[0] - oracle_expz(orc, int(ns[0]), gi)) <= 1e-5 * ns[0]
    b.close()


def mixed_batch(count, seed, nmax=18):
    rng = np.random.default_rng(seed)
    ns, parts = [], []
    for i in range(count):
        n = int(rng.integers(2, nmax + 1))
        g = C.random_gates(n, 40, seed=seed + i) if i % 3 == 0 else C.variational_layered(n, int(rng.integers(1, 5)), rng)
        ns.append(n)
        parts.append(g)
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    return ns, offs, parts


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [11, 12, 13])
def test_batch_tile_sizes_and_cta_counts(gsim, orc, tile):
    """Every register-tile size and the smallest and largest CTA count per
    SM give the oracle's <sum Z> (circuits of 2..18 qubits: below, at and
    above the tile size, so single-tile and multi-pass circuits both run)."""
    ns, offs, parts = mixed_batch(30, seed=tile)
    ref = [oracle_expz(orc, n, g) for n, g in zip(ns, parts)]
    gates = C.concat(parts)
    b = gsim.Batch(ns, offs, gates, tile_qubits=tile)
    most = b.config()["ctas_per_sm"]
    assert b.config()["tile_qubits"] == tile and most >= 2
    got_most = b.run()
    b.close()
    b = gsim.Batch(ns, offs, gates, tile_qubits=tile, ctas_per_sm=1)
    assert b.config()["ctas_per_sm"] == 1
    got_one = b.run()
    b.close()
    for i, n in enumerate(ns):
        assert abs(got_most[i] - ref[i]) <= 1e-5 * n, (i, n)
        assert abs(got_one[i] - ref[i]) <= 1e-5 * n, (i, n)
    with pytest.raises(gsim.SimError):
        gsim.Batch(ns, offs, gates, tile_qubits=tile, ctas_per_sm=most + 1)


@pytest.mark.gpu
def test_autotuned_batch_choice_is_used(gsim, orc, tmp_path, monkeypatch):
    """The autotuner times every (tile size, CTAs per SM) on a batch and
    caches the fastest; a batch built from the cached choice runs with it and
    still matches the oracle."""
    from paper_1805_00988_gb300 import autotune as A
    monkeypatch.setattr(A, "CACHE", str(tmp_path / "tune.json"))
    ns, offs, parts = mixed_batch(60, seed=4)
    gates = C.concat(parts)
    r = A.tune_batch(ns, offs, gates, "mixed60", reps=2)
    assert r["ms"] == min(r["all"].values())
    assert {"11/1", "12/1", "13/1", "13/2"} <= set(r["all"])
    tile, per_sm = A.batch_opts("mixed60")
    assert (tile, per_sm) == (r["tile_qubits"], r["ctas_per_sm"])
    b = gsim.Batch(ns, offs, gates, tile_qubits=tile, ctas_per_sm=per_sm)
    cfg = b.config()
    assert (cfg["tile_qubits"], cfg["ctas_per_sm"]) == (tile, per_sm)
    got = b.run()
    b.close()
    for i, (n, g) in enumerate(zip(ns, parts)):
        assert abs(got[i] - oracle_expz(orc, n, g)) <= 1e-5 * n, (i, n)


@pytest.mark.gpu
def test_batch_algorithmic_counts(gsim):
    """sim_batch_config's algorithmic flops and scratch bytes: an 8-qubit
    circuit of one H (16 flops per amplitude, 2^8 amplitudes) lives in one
    tile and touches no scratch; a 16-qubit circuit that needs two passes
    moves its 2^16-amplitude state out once and back once."""
    b = gsim.Batch([8], [0, 1], C.gate("h", 3))
    cfg = b.config()
    b.close()
    assert cfg["alg_flops"] == 16.0 * 2 ** 8 and cfg["alg_scratch_bytes"] == 0.0
    g = C.concat([C.gate("h", q) for q in range(16)])
    b = gsim.Batch([16], [0, 16], g, tile_qubits=13)
    info, cfg = b.info(), b.config()
    b.close()
    assert cfg["alg_flops"] == 16 * 16.0 * 2 ** 16
    assert cfg["alg_scratch_bytes"] == 2.0 * (info["passes"] - 1) * 8 * 2 ** 16 and info["passes"] >= 2
