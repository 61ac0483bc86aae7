"""The largest system the library accepts: 2^24 - 1 beads.

The fixed-point density adds 2^39 per bead, so the whole-mesh sum of a
species stays below 2^63 only for fewer than 2^24 beads (HPF_MAX_BEADS; one
more is rejected on the host, tests/test_abi.py).  At the limit the mesh
must still be the exact scatter (bit for bit against the oracle's own
scatter, and each species summing to N_K 2^39), the field force of sampled
beads must match the oracle's, and steps must run without raising the
overflow or range flags.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = (1 << 24) - 1


def test_maximum_bead_count(hpf_gpu, orc):
    rng = np.random.default_rng(7)
    box = float((N / 3.0) ** (1.0 / 3.0))
    mesh = 178
    types = (rng.random(N) < 0.5).astype(np.int32)
    pos = rng.uniform(0.0, box, size=(N, 3)).astype(np.float32)
    vel = rng.normal(size=(N, 3)).astype(np.float32)
    bonds = np.zeros((0, 2), np.int32)
    pp = dict(n_beads=N, n_species=2, mesh=mesh, box=box, chi=[[0.0, 1.0], [1.0, 0.0]],
              field_every=5, sort_every=0)
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    s.set_state(pos, vel, types, bonds)
    D = s.scatter_density()
    op = orc.make_params(**pp)
    Do = orc.scatter(op, pos, types)
    assert np.array_equal(D, Do)
    for k in range(2):
        assert int(D[k].sum(dtype=np.int64)) == int(np.count_nonzero(types == k)) << 39
    F = s.forces(1)
    Vo, Go = orc.field(op, Do)
    sample = rng.choice(N, size=4000, replace=False)
    Fo = orc.field_force(op, pos[sample], types[sample], Go)
    rms = np.sqrt(np.mean(np.sum(Fo ** 2, axis=1)))
    err = np.linalg.norm(F[sample] - Fo, axis=1)
    assert np.all(err <= 1e-5 * (np.linalg.norm(Fo, axis=1) + rms))
    s.step(5)
    p5, v5, step = s.get_state()
    assert step == 5 and np.all(np.isfinite(p5)) and np.all(np.isfinite(v5))
    s.close()
