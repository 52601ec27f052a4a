"""Autotuner: candidate feasibility (CPU) and a tuning round on the GPU whose
cached choice is the fastest measured candidate."""
import json
import os

import pytest

from paper_1805_00988_gb300 import circuits as C


def test_feasibility_cpu():
    from paper_1805_00988_gb300 import autotune as A
    assert A.feasible(20, "c64", "staged", {"tile_qubits": 13})
    assert not A.feasible(20, "c128", "staged", {"tile_qubits": 13})
    assert not A.feasible(9, "c64", "staged", {"tile_qubits": 11})
    assert A.feasible(12, "c64", "fused", {"fuse_k": 5})
    assert not A.feasible(11, "c64", "fused", {"fuse_k": 5})
    assert not A.feasible(20, "c128", "fused", {"fuse_k": 3})


@pytest.mark.gpu
def test_tune_caches_fastest(tmp_path, monkeypatch):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import autotune as A
    monkeypatch.setattr(A, "CACHE", str(tmp_path / "tune.json"))
    r = A.tune(20, "c64", C.haar_cz(20, 6, seed=3), "haar_cz_d6", reps=2)
    assert r["ms"] == min(r["all"].values())
    d = json.load(open(tmp_path / "tune.json"))
    assert "20/c64/haar_cz_d6" in d
    o = A.best_opts(20, "c64", "haar_cz_d6")
    assert o is not None
