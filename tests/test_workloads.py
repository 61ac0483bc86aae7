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


def test_chains_with_bounded_bond_angles():
    """with_bond_angles: bonds of walk_step, every bond angle in 100..140
    degrees, the same draw for the same seed, topology and velocities kept."""
    w = W.diblock(50, 6, 4, 8.0, 8, 1.0)
    d = W.generate(w)
    a = W.with_bond_angles(w, d)
    b = W.with_bond_angles(w, d)
    assert np.array_equal(a["pos"], b["pos"])
    assert not np.array_equal(a["pos"], W.with_bond_angles(w, d, seed=1)["pos"])
    for k in ("vel", "type", "bonds"):
        assert np.array_equal(a[k], d[k])
    x = a["pos"].astype(np.float64).reshape(50, 10, 3)
    assert np.array_equal(x[:, 0], d["pos"].astype(np.float64).reshape(50, 10, 3)[:, 0])
    r = np.linalg.norm(x[:, 1:] - x[:, :-1], axis=-1)
    np.testing.assert_allclose(r, w.walk_step, rtol=1e-5)
    u, v = x[:, :-2] - x[:, 1:-1], x[:, 2:] - x[:, 1:-1]
    c = np.sum(u * v, -1) / np.linalg.norm(u, axis=-1) / np.linalg.norm(v, axis=-1)
    theta = np.degrees(np.arccos(np.clip(c, -1, 1)))
    assert theta.min() >= 100.0 - 1e-3 and theta.max() <= 140.0 + 1e-3
