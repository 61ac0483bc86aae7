"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bars: the density mesh bit-exact; per-bead force within
1e-5 (|F_oracle| + F_rms); 10-step positions and velocities within 1e-4;
FP64 observables within 1e-12 relative where both sides start from the same
bits (bond, field energy) and 1e-7 where the FP32 force enters (kinetic).
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BEAD = 1 << 39


def thermal(data, sigma=0.05, seed=5):
    """Generated chains have every bond at exactly r0 (zero bond force); a seeded
    jitter gives the bonds thermal-size stretches so force bars are meaningful."""
    rng = np.random.default_rng(seed)
    d = dict(data)
    d["pos"] = (data["pos"] + rng.normal(0.0, sigma, data["pos"].shape)).astype(np.float32)
    return d


def make(hpf, w: W.Workload, data=None, **over):
    pp = w.params()
    pp.update(over)
    data = W.generate(w) if data is None else data
    sys_ = hpf.System(hpf.make_params(**pp))
    sys_.set_state(data["pos"], data["vel"], data["type"], data["bonds"], over.get("step", 0))
    return sys_, data, pp


def oparams(orc, pp):
    return orc.make_params(**pp)


def force_ok(F, Fo, rel=1e-5):
    F = F.astype(np.float64)
    rms = np.sqrt(np.mean(np.sum(Fo ** 2, axis=1))) if len(Fo) else 0.0
    err = np.linalg.norm(F - Fo, axis=1)
    bound = rel * (np.linalg.norm(Fo, axis=1) + rms)
    return np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300))) if len(Fo) else 0.0


SMALL = [
    W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600"),
    W.diblock(37, 3, 2, 5.1, 5, 2.0, name="odd_185"),
    W.Workload("aniso", [(40, [0, 1, 2, 1]), (90, [2])], 7.0, 7, 3,
               [[0, 1.2, 0.3], [1.2, 0, 0.8], [0.3, 0.8, 0]], 0.05, 3, 10),
]


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_scatter_bit_exact(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w)
    D = s.scatter_density()
    Do = orc.scatter(oparams(orc, pp), d["pos"], d["type"])
    np.testing.assert_array_equal(D, Do)
    assert int(D.sum()) == w.n_beads * BEAD


def test_scatter_edge_positions_bit_exact(hpf_gpu, orc):
    """Beads on nodes, on cell faces, far outside the box, at -0.0 and at L."""
    M, L = 6, 6.6
    h = L / M
    pts = [(0, 0, 0), (-0.0, 1e-30, -1e-30), (L, L, L), (h, 2 * h, 3 * h), (-3 * L - 0.01, 7.7 * L, -0.5),
           (0.5 * h, 0.5 * h, 0.5 * h), (np.nextafter(np.float32(L), 0), 0.1, 4.0),
           (-1e-7, -1e-7, 1e-7), (123.456, -654.321, 99.0)]
    pos = np.array(pts, dtype=np.float32)
    n = len(pos)
    types = (np.arange(n) % 2).astype(np.int32)
    w = W.diblock(1, 1, 1, L, M, 1.0)
    pp = w.params()
    pp["n_beads"] = n
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    s.set_state(pos, np.zeros_like(pos), types, np.zeros((0, 2), np.int32))
    np.testing.assert_array_equal(s.scatter_density(), orc.scatter(oparams(orc, pp), pos, types))


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_field_matches_oracle(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w)
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    Vo, Go = orc.field(op, Do)
    Fm = s.field(D_in=Do)
    scale = np.max(np.abs(Go)) + 1e-30
    np.testing.assert_allclose(Fm[..., :3], Go, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(Fm[..., 3], Vo, rtol=1e-5, atol=1e-6 * (np.max(np.abs(Vo)) + 1))


@pytest.mark.parametrize("tile", list(range(8)))
def test_every_field_tile_matches_the_oracle(hpf_gpu, orc, tile):
    """Each candidate of the autotuner (TMA-staged, plain-staged, untiled, node
    pairs) computes the same field, on an even and an odd mesh, and the
    candidates agree bit for bit."""
    for mesh in (10, 9):
        w = W.diblock(80, 5, 5, float(mesh) * 1.03, mesh, 1.4)
        s, d, pp = make(hpf_gpu, w)
        s.force_field_tile(tile)
        op = oparams(orc, pp)
        Do = orc.scatter(op, d["pos"], d["type"])
        Vo, Go = orc.field(op, Do)
        Fm = s.field(D_in=Do)
        scale = np.max(np.abs(Go)) + 1e-30
        np.testing.assert_allclose(Fm[..., :3], Go, rtol=1e-5, atol=1e-6 * scale)
        np.testing.assert_allclose(Fm[..., 3], Vo, rtol=1e-5, atol=1e-6 * (np.max(np.abs(Vo)) + 1))
        r, _, _ = make(hpf_gpu, w)
        r.force_field_tile(6)
        assert np.array_equal(Fm, r.field(D_in=Do))


@pytest.mark.parametrize("mesh,tma", [(8, True), (7, False), (70, True)])
def test_field_tiles_autotuned_and_staged(hpf_gpu, orc, mesh, tma):
    """The stencil's tile shape comes from the autotuner; even-x meshes are
    staged by TMA (zero-filled halo faces patched with periodic images)."""
    w = W.diblock(60, 5, 5, float(mesh) * 0.97, mesh, 1.0)
    s, d, pp = make(hpf_gpu, w)
    assert s.field_tile() == ((0, 0, 0), False)
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    Vo, Go = orc.field(op, Do)
    Fm = s.field(D_in=Do)
    shape, staged = s.field_tile()
    assert shape in [(32, 8, 4), (32, 8, 8), (16, 16, 4), (64, 4, 4), (16, 16, 8), (32, 4, 8),
                     (0, 0, 0), (2, 1, 1)]
    assert staged == (tma and shape not in ((0, 0, 0), (2, 1, 1)))
    scale = np.max(np.abs(Go)) + 1e-30
    np.testing.assert_allclose(Fm[..., :3], Go, rtol=1e-5, atol=1e-6 * scale)


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
@pytest.mark.parametrize("which", [1, 2, 3])
def test_forces_match_oracle(hpf_gpu, orc, w, which):
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)))
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    Vo, Go = orc.field(op, Do)
    Fo = np.zeros((w.n_beads, 3))
    if which & 1:
        Fo += orc.field_force(op, d["pos"], d["type"], Go)
    if which & 2:
        Fo += orc.bond_force(op, d["pos"], d["bonds"])
    F = s.forces(which)
    ok, worst = force_ok(F, Fo)
    assert ok, worst


def species_workload(S):
    """Chains of 10 beads cycling through S species; a seeded symmetric chi."""
    rng = np.random.default_rng(100 + S)
    chi = rng.uniform(0.2, 1.5, (S, S))
    chi = np.triu(chi, 1)
    chi = (chi + chi.T).tolist()
    return W.Workload(f"species{S}", [(90, [k % S for k in range(10)])], 7.9, 8, S, chi, 0.1,
                      field_every=3, steps=10)


@pytest.mark.parametrize("S", [1, 5, 8])
def test_species_counts_outside_the_tiled_range(hpf_gpu, orc, S):
    """One species and more than four take other paths (the untiled stencil,
    the node sums in a launch of their own, per-S instantiations): the mesh
    is exact, the field, forces and observables match the oracle at the
    usual bars, and so does a 10-step trajectory."""
    w = species_workload(S)
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)))
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    np.testing.assert_array_equal(s.scatter_density(), Do)
    Vo, Go = orc.field(op, Do)
    Fm = s.field(D_in=Do)
    scale = np.max(np.abs(Go)) + 1e-30
    np.testing.assert_allclose(Fm[..., :3], Go, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(Fm[..., 3], Vo, rtol=1e-5, atol=1e-6 * (np.max(np.abs(Vo)) + 1))
    Fo = orc.field_force(op, d["pos"], d["type"], Go) + orc.bond_force(op, d["pos"], d["bonds"])
    ok, worst = force_ok(s.forces(3), Fo)
    assert ok, worst
    s.close()
    s, d, pp = make(hpf_gpu, w, data=d)
    E = s.energy()
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    assert E[1] == pytest.approx(Eo[1], rel=1e-12, abs=1e-12)
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)
    s.step(10)
    pos, vel, _ = s.get_state()
    po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4
    s.close()


def test_uniform_lattice_gives_exactly_zero_field_force(hpf_gpu):
    M = 6
    g = np.stack(np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij"), -1)
    pos = np.repeat(g.reshape(-1, 3)[:, ::-1].astype(np.float32), 3, axis=0)
    n = len(pos)
    types = np.tile(np.array([0, 0, 1], np.int32), n // 3)
    p = W.diblock(1, 1, 1, float(M), M, 1.3).params()
    p["n_beads"] = n
    s = hpf_gpu.System(hpf_gpu.make_params(**p))
    s.set_state(pos, np.zeros_like(pos), types, np.zeros((0, 2), np.int32))
    assert np.all(s.forces(1) == 0.0)


def run_both(hpf, orc, w, n_steps, chunks=None, **over):
    s, d, pp = make(hpf, w, **over)
    for c in (chunks or [n_steps]):
        s.step(c)
    pos, vel, step = s.get_state()
    po, vo, _ = orc.run(oparams(orc, pp), d["pos"], d["vel"], d["type"], d["bonds"],
                        over.get("step", 0), n_steps)
    assert step == over.get("step", 0) + n_steps
    return pos, vel, po, vo


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_ten_step_trajectory(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("fe,step0,chunks", [(3, 7, [10]), (20, 0, [40]), (7, 5, [1, 2, 3, 4]),
                                             (1, 0, [10]), (10, 3, [10])])
def test_field_schedule_and_chunking(hpf_gpu, orc, fe, step0, chunks):
    w = W.diblock(80, 5, 5, 8.0, 8, 1.0)
    n = sum(chunks)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, n, chunks=chunks, field_every=fe, step=step0)
    tol = 1e-4 if n <= 10 else 5e-4   # 40-step case: FP32 rounding grows with the steps
    assert np.max(np.abs(pos - po)) <= tol
    assert np.max(np.abs(vel - vo)) <= tol


@pytest.mark.parametrize("fe,steps", [(10, 10), (5, 15), (20, 40), (3, 7)])
def test_mesh_deposited_by_the_step_kernel_is_exact(hpf_gpu, orc, fe, steps):
    """A launch that ends on a refresh step deposits its final positions into
    the next mesh; that mesh must be the exact scatter of those positions."""
    w = W.diblock(200, 6, 4, 9.0, 9, 1.0, field_every=fe)
    s, d, pp = make(hpf_gpu, w)
    op = oparams(orc, pp)
    s.step(steps)
    pos, vel, st = s.get_state()
    D = s.scatter_density()
    Do = orc.scatter(op, pos, d["type"])
    np.testing.assert_array_equal(D, Do)
    E = s.energy()
    assert E[2] == pytest.approx(orc.field_energy(op, Do), rel=1e-12)


def test_observed_steps_deposit_their_final_positions(hpf_gpu, orc):
    """Once hpf_step calls are followed by the observables of their final
    state, each call's last launch deposits its final positions, and a state
    upload deposits the new positions in its permutation pass.  The mesh the
    observables then use must be the exact scatter of the positions, at
    refresh and other steps, with no standalone scatter after the first
    observed call; when calls stop being observed the deposits stop, and the
    observables stay exact."""
    w = W.diblock(200, 6, 4, 9.0, 9, 1.0, field_every=4)
    s, d, pp = make(hpf_gpu, w)
    op = oparams(orc, pp)

    def check():
        E = s.energy()
        pos, _, _ = s.get_state()
        D = s.scatter_density()
        Do = orc.scatter(op, pos, d["type"])
        np.testing.assert_array_equal(D, Do)
        assert E[2] == pytest.approx(orc.field_energy(op, Do), rel=1e-12)
        return pos

    s.profile(True)
    s.profile_read()
    for _ in range(9):      # across two refreshes (steps 4 and 8)
        s.step(1)
        check()
    # the field refresh at step 0 and the first observed call's own scatter
    assert s.profile_read()["scatter"][1] == 2
    s.step(1)
    s.step(1)               # the first call's end deposit went unread
    s.step(2)
    pos = check()
    rng = np.random.default_rng(11)
    pos2 = (pos + rng.normal(0.0, 0.05, pos.shape)).astype(np.float32)
    vel2 = rng.normal(0.0, 1.0, pos.shape).astype(np.float32)
    s.profile_read()
    s.update_state(pos2, vel2, 6)
    np.testing.assert_array_equal(check(), pos2)
    s.step(3)
    check()
    assert s.profile_read()["scatter"][1] == 0
    s.close()


@pytest.mark.parametrize("therm", [dict(thermostat=1, nh_tau=0.3),
                                   dict(thermostat=2, andersen_nu=1.0)], ids=["nh", "andersen"])
def test_observed_steps_deposit_under_the_other_thermostats(hpf_gpu, orc, therm):
    """Nose-Hoover (its own launch sequence) and Andersen (no fused
    observables) also deposit the final positions of observed calls: the mesh
    the observables use is the exact scatter of the positions at every step,
    and no standalone scatter runs after the first observed call."""
    w = W.diblock(200, 6, 4, 9.0, 9, 1.0, field_every=4)
    s, d, pp = make(hpf_gpu, w, **therm)
    op = oparams(orc, pp)
    s.profile(True)
    s.profile_read()
    for _ in range(7):
        s.step(1)
        E = s.energy()
        pos, _, _ = s.get_state()
        D = s.scatter_density()
        Do = orc.scatter(op, pos, d["type"])
        np.testing.assert_array_equal(D, Do)
        assert E[2] == pytest.approx(orc.field_energy(op, Do), rel=1e-12)
    assert s.profile_read()["scatter"][1] == 2
    s.close()


def test_observed_steps_form_the_observables_in_the_step_launch(hpf_gpu, orc):
    """An observed hpf_step call whose launch does not end on a refresh step
    forms the observables' bead terms (F_n on the field in force, the on-step
    velocity, |v_n|^2, momentum, bond energies) in that launch; hpf_energy
    then runs only the node sums and the combination (two launches where the
    full pass takes three with four species).  At every step the observables
    must match the oracle (given the field of the last refresh) at the usual
    bars, and the full pass of a batch member on the same trajectory (a
    batch's steps never form them) to its summation order."""
    chi = [[0.0, 0.8, 0.3, 0.5], [0.8, 0.0, 0.6, 0.2], [0.3, 0.6, 0.0, 0.9],
           [0.5, 0.2, 0.9, 0.0]]
    w = W.Workload("abcd", [(136, [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4)], 9.0, 9, 4, chi, 0.1,
                   field_every=4, steps=10)
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)))
    bt = hpf_gpu.Batch([hpf_gpu.make_params(**pp)])
    rep = bt.replica(0)
    rep.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    op = oparams(orc, pp)
    s.profile(True)
    s.profile_read()
    ref = d["pos"]  # positions the field in force was formed from
    for k in range(7):
        s.step(1)
        bt.step(1)
        E = s.energy()
        launches = s.profile_read()["energy"][1]
        pos, vel, st = s.get_state()
        if st % w.field_every == 0:
            ref = pos
        Vr, Gr = orc.field(op, orc.scatter(op, ref, d["type"]))
        Eo = orc.energy(op, pos, vel, d["type"], d["bonds"], Vr, Gr, st)
        assert E[1] == pytest.approx(Eo[1], rel=1e-12, abs=1e-12)
        assert E[2] == pytest.approx(Eo[2], rel=1e-12)
        assert E[0] == pytest.approx(Eo[0], rel=1e-7)
        assert E[3] == pytest.approx(Eo[3], rel=1e-7)
        assert E[4] == pytest.approx(Eo[4], rel=1e-4, abs=1e-6 * w.n_beads)
        assert E[5] == pytest.approx(Eo[5], rel=1e-7)
        # the first observed call and refresh steps take the full pass
        fused = k > 0 and st % w.field_every != 0
        assert launches == (2 if fused else 3)
        pb, vb, sb = rep.get_state()
        assert sb == st
        np.testing.assert_array_equal(pb, pos)
        np.testing.assert_array_equal(vb, vel)
        Eb = rep.energy()
        assert Eb[1] == pytest.approx(E[1], rel=1e-12)
        assert Eb[2] == E[2]
        assert Eb[0] == pytest.approx(E[0], rel=1e-9)
        assert Eb[4] == pytest.approx(E[4], rel=1e-6, abs=1e-9 * w.n_beads)
    # a step whose terms were formed in the launch, then another field put in
    # force (an injected mesh): the observables take the full pass on it
    s.step(2)
    pos, vel, st = s.get_state()
    assert st % w.field_every != 0
    Dj = orc.scatter(op, d["pos"], d["type"])
    s.field(D_in=Dj)
    s.profile_read()
    E = s.energy()
    assert s.profile_read()["energy"][1] == 3
    Vj, Gj = orc.field(op, Dj)
    Eo = orc.energy(op, pos, vel, d["type"], d["bonds"], Vj, Gj, st)
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)
    s.close()
    bt.close()


def test_long_chains_take_the_halo_kernel(hpf_gpu, orc):
    """Chains longer than 64 beads cannot be packed into warp segments; the
    CTA kernel with recomputed halos advances them."""
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=5)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_long_field_period_in_warp_launches(hpf_gpu, orc):
    """field_every = 50: whole 50-step periods in one warp launch each."""
    w = W.diblock(120, 8, 12, 9.0, 9, 1.0, field_every=50)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 100)
    # 100 steps of FP32 rounding against the FP64 oracle
    assert np.max(np.abs(pos - po)) <= 1e-3
    assert np.max(np.abs(vel - vo)) <= 1e-3


def test_nve_trajectory_without_thermostat(hpf_gpu, orc):
    w = W.a5b5_10k()
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, gamma=0.0)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_energy_matches_oracle(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w)
    op = oparams(orc, pp)
    E = s.energy()
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    assert E[1] == pytest.approx(Eo[1], rel=1e-12, abs=1e-12)   # bond: same bits in
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)              # field: exact integers in
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)               # kinetic: FP32 force enters
    assert E[3] == pytest.approx(Eo[3], rel=1e-7)
    assert E[4] == pytest.approx(Eo[4], rel=1e-4, abs=1e-6 * w.n_beads)
    assert E[5] == pytest.approx(Eo[5], rel=1e-7)


def test_kT_other_than_one_follows_the_oracle(hpf_gpu, orc):
    """At kT = 2.5 (chi in kT units, 1/kappa in energy units, so only the chi
    terms scale) the field forces, the field energy and a 10-step trajectory
    follow the oracle at the usual bars."""
    w = SMALL[2]
    d = thermal(W.generate(w))
    s, d, pp = make(hpf_gpu, w, data=d, kT=2.5)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    ok, worst = force_ok(s.forces(1), orc.field_force(op, d["pos"], d["type"], Go))
    assert ok, worst
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    assert s.energy()[2] == pytest.approx(Eo[2], rel=1e-12)
    s.step(10)
    pos, vel, _ = s.get_state()
    po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_resume_is_bit_identical(hpf_gpu):
    w = W.diblock(100, 4, 4, 8.0, 8, 1.0, field_every=5)
    a, d, pp = make(hpf_gpu, w)
    a.step(20)
    pa, va, _ = a.get_state()
    b, _, _ = make(hpf_gpu, w, data=d)
    b.step(10)
    p1, v1, st = b.get_state()
    c = hpf_gpu.System(hpf_gpu.make_params(**pp))
    c.set_state(p1, v1, d["type"], d["bonds"], st)
    c.step(10)
    pc, vc, _ = c.get_state()
    np.testing.assert_array_equal(pa, pc)
    np.testing.assert_array_equal(va, vc)


def test_update_state_equals_a_fresh_load(hpf_gpu):
    """hpf_update_state (new coordinates, same topology, old bead order) then
    steps gives the same bits as loading the coordinates into a new context."""
    w = W.diblock(100, 4, 4, 8.0, 8, 1.0, field_every=5)
    a, d, pp = make(hpf_gpu, w, sort_every=6)
    a.step(20)  # re-sorted along the way
    p1, v1, st = a.get_state()
    b, _, _ = make(hpf_gpu, w, data=d, sort_every=6)
    b.step(10)  # a refresh step: the frozen field of b is that of these positions
    p2, v2, _ = b.get_state()
    a.update_state(p2, v2, 10)  # rewind a to b's state
    a.step(10)
    b.step(10)
    pa, va, sa = a.get_state()
    pb, vb, sb = b.get_state()
    assert sa == sb == 20
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(a.energy(), b.energy())
    bad = p2.copy()
    bad[3, 1] = np.nan
    a.update_state(bad, v2, 10)
    with pytest.raises(hpf_gpu.HPFError) as e:
        a.energy()
    assert e.value.status == 5


def expected_order(orc, op, pos, n_chain_beads):
    """Chain order by (brick-major cell key of the first bead, first tag), from the oracle."""
    firsts = np.concatenate([[0], np.cumsum(n_chain_beads)[:-1]])
    order = orc.chain_order(op, pos, firsts, 8)
    return np.concatenate([np.arange(firsts[c], firsts[c] + n_chain_beads[c]) for c in order])


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_sort_order_matches_definition(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w)
    lens = np.concatenate([[len(seq)] * n for n, seq in w.blocks])
    np.testing.assert_array_equal(s.order(), expected_order(orc, oparams(orc, pp), d["pos"], lens))
    # the state comes back in tag order, bit for bit
    pos, vel, _ = s.get_state()
    np.testing.assert_array_equal(pos, d["pos"])
    np.testing.assert_array_equal(vel, d["vel"])
    # after moving, a reload sorts by the new positions
    s.step(7)
    pos, vel, st = s.get_state()
    s.set_state(pos, vel, d["type"], d["bonds"], st)
    np.testing.assert_array_equal(s.order(), expected_order(orc, oparams(orc, pp), pos, lens))


def test_results_do_not_depend_on_sorting(hpf_gpu, orc):
    """Re-sorting at every launch gives the oracle trajectory."""
    w = W.diblock(150, 5, 5, 8.0, 8, 1.0, field_every=2)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, chunks=[3, 3, 4], sort_every=1)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_host_and_device_pointers_agree(hpf_gpu):
    import torch
    w = W.diblock(50, 5, 5, 6.0, 6, 1.0)
    a, d, pp = make(hpf_gpu, w)
    b = hpf_gpu.System(hpf_gpu.make_params(**pp))
    dev = {k: torch.from_numpy(v).cuda() for k, v in d.items()}
    b.set_state(dev["pos"], dev["vel"], dev["type"], dev["bonds"])
    Fa = a.forces()
    Fb = torch.empty((w.n_beads, 3), dtype=torch.float32, device="cuda")
    b.forces(out=Fb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Fa, Fb.cpu().numpy())


def test_empty_system(hpf_gpu, orc):
    w = W.diblock(1, 1, 1, 5.0, 5, 1.0)
    pp = w.params()
    pp["n_beads"] = 0
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    e = np.zeros((0, 3), np.float32)
    s.set_state(e, e, np.zeros(0, np.int32), np.zeros((0, 2), np.int32))
    s.step(5)
    assert np.all(s.scatter_density() == 0)
    E = s.energy()
    op = oparams(orc, pp)
    assert E[2] == pytest.approx(orc.field_energy(op, np.zeros((2, 5, 5, 5), np.int64)), rel=1e-12)
    assert E[0] == 0.0 and E[1] == 0.0


def test_invalid_state_is_rejected(hpf_gpu):
    w = W.diblock(3, 2, 2, 5.0, 5, 1.0)
    s, d, pp = make(hpf_gpu, w)
    HPFError = hpf_gpu.HPFError
    bad = d["type"].copy()
    bad[2] = 2
    with pytest.raises(HPFError, match="INVALID"):
        s.set_state(d["pos"], d["vel"], bad, d["bonds"])
    with pytest.raises(HPFError, match="INVALID"):
        s.set_state(d["pos"], d["vel"], d["type"], np.array([[0, 2]], np.int32))
    with pytest.raises(HPFError, match="INVALID"):
        s.set_state(d["pos"], d["vel"], d["type"], np.array([[0, 1], [1, 0]], np.int32))
    p = d["pos"].copy()
    p[4, 1] = np.nan
    with pytest.raises(HPFError, match="NONFINITE"):
        s.set_state(p, d["vel"], d["type"], d["bonds"])
    with pytest.raises(HPFError, match="STATE"):
        s.step(1)
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    s.step(1)


# ---------------------------------------------------------------- full sizes

@pytest.mark.parametrize("factory", [W.a10b10_1m], ids=["a10b10_1m"])
def test_full_size_melt_parity(hpf_gpu, orc, factory):
    """The 1M-bead melt in the benchmark's configuration: exact mesh, forces of
    every bead, and a whole 10-step field period against the oracle."""
    w = factory()
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), sort_every=500)
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    np.testing.assert_array_equal(s.scatter_density(), Do)
    Vo, Go = orc.field(op, Do)
    Fo = orc.field_force(op, d["pos"], d["type"], Go) + orc.bond_force(op, d["pos"], d["bonds"])
    ok, worst = force_ok(s.forces(), Fo)
    assert ok, worst
    s.step(10)
    pos, vel, _ = s.get_state()
    po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_full_size_ternary_blend(hpf_gpu, orc):
    """8.1M beads, 3 species: exact mesh and forces of every bead."""
    w = W.ternary_8m()
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)))
    op = oparams(orc, pp)
    Do = orc.scatter(op, d["pos"], d["type"])
    np.testing.assert_array_equal(s.scatter_density(), Do)
    for k in range(3):
        assert int(Do[k].sum()) == int((d["type"] == k).sum()) * BEAD
    Vo, Go = orc.field(op, Do)
    Fo = orc.field_force(op, d["pos"], d["type"], Go) + orc.bond_force(op, d["pos"], d["bonds"])
    ok, worst = force_ok(s.forces(), Fo)
    assert ok, worst


def test_bounded_wait_gives_up_and_the_context_survives(hpf_gpu, orc):
    """Failure detection without a fault: a device wait that nothing completes
    gives up within its limit, the host reads HPF_ERR_TIMEOUT, and the same
    context then steps and matches the oracle."""
    w = W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600")
    s, d, pp = make(hpf_gpu, w)
    status, seconds = s.selftest_timeout()
    assert status == 6  # HPF_ERR_TIMEOUT
    assert 0.1 <= seconds < 2.0
    s.step(10)
    pos, vel, step = s.get_state()  # no stale timeout reported
    po, vo, _ = orc.run(oparams(orc, pp), d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    assert step == 10
    assert np.max(np.abs(pos - po)) <= 1e-4 and np.max(np.abs(vel - vo)) <= 1e-4
