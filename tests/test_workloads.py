"""The seeded input generator: shapes, determinism and the physical recipe."""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W


def test_config_sizes():
    assert W.a5b5_10k().n_beads == 10_000
    assert W.a10b10_1m().n_beads == 1_000_000
    assert W.ternary_8m().n_beads == 8_100_000
    reps = W.replica_set()
    assert len(reps) == 64
    for r in reps:
        assert 20_000 <= r.n_beads <= 100_000 and r.n_beads % 20 == 0
        assert r.mesh == round((r.n_beads / 3) ** (1 / 3))
    assert reps[0].chi[0][1] == pytest.approx(0.2) and reps[-1].chi[0][1] == pytest.approx(2.0)


def test_generate_is_seeded_and_well_formed():
    w = W.diblock(50, 3, 4, 6.0, 6, 1.0)
    a, b = W.generate(w), W.generate(w)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    c = W.generate(w, seed=7)
    assert not np.array_equal(a["pos"], c["pos"])
    n = w.n_beads
    assert a["pos"].shape == (n, 3) and a["pos"].dtype == np.float32
    assert a["vel"].shape == (n, 3) and a["vel"].dtype == np.float32
    assert a["type"].tolist()[:7] == [0, 0, 0, 1, 1, 1, 1]
    assert a["bonds"].shape == (50 * 6, 2)
    d = a["pos"][a["bonds"][:, 1]].astype(np.float64) - a["pos"][a["bonds"][:, 0]]
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 0.7, atol=1e-5)
    np.testing.assert_allclose(a["vel"].astype(np.float64).mean(axis=0), 0.0, atol=1e-6)


def test_ternary_blend_layout():
    w = W.Workload("t", [(3, [0] * 20), (3, [1] * 20), (30, [2])], 10.0, 10, 3,
                   [[0, 1.2, 0.3], [1.2, 0, 0.8], [0.3, 0.8, 0]], 0.05, 5, 10)
    d = W.generate(w)
    assert d["type"].tolist().count(2) == 30
    assert d["bonds"].shape[0] == 6 * 19
    assert np.all(d["bonds"][:, 1] == d["bonds"][:, 0] + 1)
