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
