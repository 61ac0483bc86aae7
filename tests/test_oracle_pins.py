"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form, an
invariant, a hand computation, an independent library routine, or a
finite-difference derivative of an energy.  Each is chosen so that a plausible
slip (a dropped term, a wrong sign, index or axis, a missing factor 2 or 1/2)
fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

ONE = 1 << 13          # fixed-point weight of one axis
BEAD = 1 << 39         # fixed-point mass of one bead


def unit_params(orc, S=2, mesh=(8, 8, 8), **kw):
    """Box with h = 1 on every axis, so the mesh coordinate equals the position."""
    box = tuple(float(m) for m in mesh)
    return orc.make_params(S, mesh, box, **kw)


# ------------------------------------------------------------------ scatter (A2)

def test_scatter_bead_on_node(orc):
    p = unit_params(orc, mesh=(6, 7, 8))
    D = orc.scatter(p, [[3.0, 4.0, 5.0]], [1])
    assert D.dtype == np.int64 and D.shape == (2, 8, 7, 6)
    assert D[1, 5, 4, 3] == BEAD           # [species][z][y][x]
    assert D.sum() == BEAD and D[0].sum() == 0


def test_scatter_bead_at_cell_centre(orc):
    p = unit_params(orc)
    D = orc.scatter(p, [[3.5, 4.5, 5.5]], [0])
    for z in (5, 6):
        for y in (4, 5):
            for x in (3, 4):
                assert D[0, z, y, x] == 1 << 36
    assert D.sum() == BEAD


def test_scatter_hand_computed_weights(orc):
    # x = 3.25 -> q = 2048; y = 4.75 -> q = 6144; z = 5.125 -> q = 1024
    p = unit_params(orc)
    D = orc.scatter(p, [[3.25, 4.75, 5.125]], [0])
    wx = {3: 6144, 4: 2048}
    wy = {4: 2048, 5: 6144}
    wz = {5: 7168, 6: 1024}
    for z, a in wz.items():
        for y, b in wy.items():
            for x, c in wx.items():
                assert D[0, z, y, x] == a * b * c
    assert np.count_nonzero(D) == 8


def test_scatter_periodic_wrap_and_negative_coordinates(orc):
    p = unit_params(orc)  # M = 8
    # x = -0.25 lies in cell -1 == 7 with q = 6144; y = 7.5 straddles 7 and 0; z = 16.0 is node 0
    D = orc.scatter(p, [[-0.25, 7.5, 16.0]], [0])
    assert D[0, 0, 7, 7] == 2048 * 4096 * ONE
    assert D[0, 0, 7, 0] == 6144 * 4096 * ONE
    assert D[0, 0, 0, 7] == 2048 * 4096 * ONE
    assert D[0, 0, 0, 0] == 6144 * 4096 * ONE
    assert D.sum() == BEAD


def test_scatter_tiny_negative_coordinate(orc):
    # s = -1e-30 lies in cell -1 with frac(s) = 1 - 1e-30, so q = floor(8192 (1 - 1e-30)) = 8191:
    # the lower node keeps one quantum per axis (1 * 8192 * 8192 from the x axis alone)
    p = unit_params(orc)
    D = orc.scatter(p, [[-1e-30, 0.0, 0.0]], [0])
    assert D[0, 0, 0, 7] == 1 * ONE * ONE
    assert D[0, 0, 0, 0] == 8191 * ONE * ONE
    assert D.sum() == BEAD


def test_scatter_mass_conservation_random(orc):
    rng = np.random.default_rng(1)
    p = orc.make_params(3, (9, 10, 11), (8.7, 10.3, 12.9))
    n = 5000
    pos = rng.uniform(-30, 40, size=(n, 3)).astype(np.float32)
    types = rng.integers(0, 3, size=n)
    D = orc.scatter(p, pos, types)
    for k in range(3):
        assert int(D[k].sum()) == int((types == k).sum()) * BEAD
    assert D.min() >= 0


def test_scatter_matches_float_cic_within_quantisation(orc):
    # |D 2^-39 - CIC| <= 3 * 2^-13 per bead touching the node (textbook CIC in fp64)
    rng = np.random.default_rng(2)
    p = unit_params(orc, S=1, mesh=(5, 5, 5))
    pos = rng.uniform(0, 5, size=(40, 3)).astype(np.float32)
    D = orc.scatter(p, pos, np.zeros(40, dtype=np.int32))
    ref = np.zeros((5, 5, 5))
    for x in pos.astype(np.float64):
        i = np.floor(x).astype(int)
        f = x - i
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) *
                         (f[2] if dz else 1 - f[2]))
                    ref[(i[2] + dz) % 5, (i[1] + dy) % 5, (i[0] + dx) % 5] += w
    assert np.max(np.abs(D[0] / BEAD - ref)) <= 3 * 2.0 ** -13 * 40


# ------------------------------------------------------------------ field (A3)

def lattice_melt(mesh, per_node_types):
    """Beads exactly on every node (h = 1): identical integer density everywhere."""
    pos, types = [], []
    for z in range(mesh[2]):
        for y in range(mesh[1]):
            for x in range(mesh[0]):
                for t in per_node_types:
                    pos.append((x, y, z))
                    types.append(t)
    return np.array(pos, dtype=np.float32), np.array(types, dtype=np.int32)


def test_uniform_melt_has_exactly_zero_field_force(orc):
    mesh = (6, 5, 4)
    p = unit_params(orc, mesh=mesh, chi=[[0, 1.3], [1.3, 0]], inv_kappa=0.1)
    pos, types = lattice_melt(mesh, [0, 0, 1])
    D = orc.scatter(p, pos, types)
    V, G = orc.field(p, D)
    assert np.all(G == 0.0)
    rng = np.random.default_rng(3)
    probe = rng.uniform(-10, 10, size=(100, 3))
    F = orc.field_force(p, probe, rng.integers(0, 2, 100), G)
    assert np.all(F == 0.0)
    # phi_A = 2/3, phi_B = 1/3 with rho0 = 3, h = 1: V_A = chi_AB phi_B, V_B = chi_AB phi_A
    assert V[0, 0, 0, 0] == pytest.approx(1.3 / 3.0, rel=1e-14)
    assert V[1, 0, 0, 0] == pytest.approx(1.3 * 2.0 / 3.0, rel=1e-14)


def test_potential_closed_form_at_a_node(orc):
    # h = (2, 1, 0.5) -> cell volume 1; rho0 = 2; 3 A beads and 1 B bead worth at the node
    p = orc.make_params(2, (4, 4, 4), (8.0, 4.0, 2.0), rho0=2.0, kT=1.5, inv_kappa=0.25,
                        chi=[[0.2, 0.7], [0.7, 0.0]])
    D = np.zeros((2, 4, 4, 4), dtype=np.int64)
    D[0, 1, 2, 3] = 3 * BEAD
    D[1, 1, 2, 3] = 1 * BEAD
    V, _ = orc.field(p, D)
    phiA, phiB = 3 / 2.0, 1 / 2.0
    assert V[0, 1, 2, 3] == pytest.approx(1.5 * (0.2 * phiA + 0.7 * phiB) + 0.25 * (phiA + phiB - 1))
    assert V[1, 1, 2, 3] == pytest.approx(1.5 * (0.7 * phiA) + 0.25 * (phiA + phiB - 1))
    assert V[0, 0, 0, 0] == pytest.approx(-0.25)   # empty node: only the compressibility term


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gradient_of_sinusoid_closed_form(orc, axis):
    mesh = [12, 10, 8]
    box = [9.0, 11.0, 6.5]
    p = orc.make_params(2, mesh, box, kT=1.0, inv_kappa=0.3, chi=[[0.0, 0.9], [0.9, 0.0]])
    M = mesh[axis]
    h = box[axis] / M
    k = 2 * math.pi * 2 / box[axis]
    n = np.arange(M)
    A0, A1 = 3.0 * BEAD, 1.0 * BEAD
    prof = np.rint(A0 + A1 * np.sin(k * n * h)).astype(np.int64)
    D = np.zeros((2, mesh[2], mesh[1], mesh[0]), dtype=np.int64)
    shape = [1, 1, 1]
    shape[2 - axis] = M
    D[0] = np.broadcast_to(prof.reshape(shape), D[0].shape)
    _, G = orc.field(p, D)
    c = 1.0 / (3.0 * (9.0 / 12) * (11.0 / 10) * (6.5 / 8))  # phi per bead at a node
    dphi = c * 1.0 * np.cos(k * n * h) * np.sin(k * h) / h  # exact central difference
    exp_A = 0.3 * dphi                  # V_A = 0.3 (phi_A - 1): chi_AA = 0
    exp_B = (0.9 + 0.3) * dphi          # V_B = 0.9 phi_A + 0.3 (phi_A - 1)
    idx = [0, 0, 0]
    for i in range(M):
        idx[axis] = i
        gA = G[0, idx[2], idx[1], idx[0]]
        gB = G[1, idx[2], idx[1], idx[0]]
        assert gA[axis] == pytest.approx(exp_A[i], abs=1e-9)
        assert gB[axis] == pytest.approx(exp_B[i], abs=1e-9)
        for other in range(3):
            if other != axis:
                assert gA[other] == 0.0 and gB[other] == 0.0


def test_field_is_linear_in_the_interaction_matrix(orc):
    rng = np.random.default_rng(4)
    D = rng.integers(0, 5 * BEAD, size=(2, 5, 6, 7))
    base = dict(kT=1.0, inv_kappa=0.0)
    p1 = orc.make_params(2, (7, 6, 5), (7.0, 6.0, 5.0), chi=[[0, 1.0], [1.0, 0]], **base)
    p2 = orc.make_params(2, (7, 6, 5), (7.0, 6.0, 5.0), chi=[[0, 2.5], [2.5, 0]], **base)
    V1, G1 = orc.field(p1, D)
    V2, G2 = orc.field(p2, D)
    np.testing.assert_allclose(V2, 2.5 * V1, rtol=1e-13)
    np.testing.assert_allclose(G2, 2.5 * G1, rtol=1e-12, atol=1e-12)
    # swapping species labels swaps the potentials
    V3, _ = orc.field(p1, D[::-1].copy())
    np.testing.assert_allclose(V3, V1[::-1], rtol=1e-13)


# ------------------------------------------------------------------ gather (A4)

def test_gather_of_constant_gradient_is_exact(orc):
    p = orc.make_params(2, (5, 6, 7), (4.1, 5.3, 6.7))
    G = np.zeros((2, 7, 6, 5, 3))
    G[0, ..., :] = (0.3, -1.7, 2.2)
    G[1, ..., :] = (-5.0, 0.5, 0.25)
    rng = np.random.default_rng(5)
    pos = rng.uniform(-20, 20, size=(200, 3))
    types = rng.integers(0, 2, size=200)
    F = orc.field_force(p, pos, types, G)
    exp = np.where(types[:, None] == 0, -np.array([0.3, -1.7, 2.2]), -np.array([-5.0, 0.5, 0.25]))
    np.testing.assert_allclose(F, exp, rtol=1e-14, atol=1e-14)


def test_gather_reproduces_linear_field_and_node_values(orc):
    p = unit_params(orc, S=1, mesh=(10, 10, 10))
    z, y, x = np.meshgrid(np.arange(10), np.arange(10), np.arange(10), indexing="ij")
    G = np.zeros((1, 10, 10, 10, 3))
    G[0, ..., 0] = 1.0 + 0.5 * x - 0.25 * y
    G[0, ..., 1] = -2.0 + 0.125 * z
    G[0, ..., 2] = 0.75 * x + 0.5 * y - 0.5 * z
    rng = np.random.default_rng(6)
    pos = rng.uniform(1, 8.9, size=(100, 3)).astype(np.float32).astype(np.float64)
    F = orc.field_force(p, pos, np.zeros(100, dtype=np.int32), G)
    X, Y, Z = pos[:, 0], pos[:, 1], pos[:, 2]
    exp = -np.stack([1.0 + 0.5 * X - 0.25 * Y, -2.0 + 0.125 * Z, 0.75 * X + 0.5 * Y - 0.5 * Z], 1)
    np.testing.assert_allclose(F, exp, rtol=1e-12, atol=1e-12)
    Fn = orc.field_force(p, [[3.0, 4.0, 5.0]], [0], G)
    np.testing.assert_array_equal(Fn[0], -G[0, 5, 4, 3])


def _interp_energy(pos, types, V, inv_h):
    """Energy of beads in a frozen nodal potential, trilinear in the nodes (numpy)."""
    S, Mz, My, Mx = V.shape
    e = 0.0
    for x, t in zip(pos, types):
        s = (np.float32(x) * np.float32(inv_h)).astype(np.float64)
        i = np.floor(s).astype(int)
        f = s - i
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) *
                         (f[2] if dz else 1 - f[2]))
                    e += w * V[t, (i[2] + dz) % Mz, (i[1] + dy) % My, (i[0] + dx) % Mx]
    return e


def test_force_is_minus_energy_derivative_two_chains(orc):
    """Two 5-bead chains in a frozen potential that is linear in each node index:
    central differences and trilinear interpolation are then exact, so the
    oracle's field + bond force must equal minus the numerical derivative of
    U_bond + (potential energy of the beads in the nodal field)."""
    mesh = (16, 16, 16)
    p = unit_params(orc, mesh=mesh, chi=[[0.0, 1.1], [1.1, 0.0]], inv_kappa=0.2)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    D = np.zeros((2, 16, 16, 16), dtype=np.int64)
    D[0] = (3 * BEAD + (BEAD // 8) * (2 * x - y + 3 * z)).astype(np.int64)
    D[1] = (2 * BEAD + (BEAD // 16) * (x + 4 * y - 2 * z)).astype(np.int64)
    V, G = orc.field(p, D)
    rng = np.random.default_rng(7)
    pos = np.zeros((10, 3))
    for c in range(2):
        pos[5 * c] = rng.uniform(6, 9, size=3)
        for b in range(1, 5):
            d = rng.normal(size=3)
            pos[5 * c + b] = pos[5 * c + b - 1] + 0.75 * d / np.linalg.norm(d)
    pos = pos.astype(np.float32).astype(np.float64)
    types = np.array([0, 0, 1, 1, 1, 0, 1, 0, 1, 0], dtype=np.int32)
    bonds = [(0, 1), (1, 2), (2, 3), (3, 4), (5, 6), (6, 7), (7, 8), (8, 9)]
    F = orc.field_force(p, pos, types, G) + orc.bond_force(p, pos, bonds)
    inv_h = 1.0

    def energy(q):
        return orc.bond_energy(p, q, bonds) + _interp_energy(q, types, V, inv_h)

    d = 2.0 ** -12  # a float32-exact step, small enough to stay inside each cell
    for i in range(10):
        for a in range(3):
            qp, qm = pos.copy(), pos.copy()
            qp[i, a] += d
            qm[i, a] -= d
            fd = -(energy(qp) - energy(qm)) / (2 * d)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


# ------------------------------------------------------------------ bonds (A5)

def test_two_bead_bond_closed_form(orc):
    p = orc.make_params(1, 4, 4.0, bond_k=4.0, bond_r0=0.7)
    pos = np.array([[1.0, 2.0, 3.0], [1.6, 2.8, 3.0]])  # r = 1.0
    F = orc.bond_force(p, pos, [(0, 1)])
    # U = k (r - r0)^2 = 4 * 0.09; F_0 = -2 k (r - r0) (x0 - x1) / r = +2.4 * (0.6, 0.8, 0)
    assert orc.bond_energy(p, pos, [(0, 1)]) == pytest.approx(0.36, rel=1e-14)
    np.testing.assert_allclose(F[0], [1.44, 1.92, 0.0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(F[1], -F[0], rtol=1e-14)


def test_bond_forces_sum_to_zero_and_match_derivative(orc):
    rng = np.random.default_rng(8)
    p = orc.make_params(1, 4, 4.0, bond_k=3.0, bond_r0=0.9)
    pos = np.cumsum(rng.normal(scale=0.6, size=(12, 3)), axis=0)
    bonds = [(i, i + 1) for i in range(11)] + [(2, 9)]
    F = orc.bond_force(p, pos, bonds)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)
    d = 1e-6
    for i in range(12):
        for a in range(3):
            qp, qm = pos.copy(), pos.copy()
            qp[i, a] += d
            qm[i, a] -= d
            fd = -(orc.bond_energy(p, qp, bonds) - orc.bond_energy(p, qm, bonds)) / (2 * d)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-7)


# ------------------------------------------------------------------ energies (A7)

def test_field_energy_derivative_is_the_potential(orc):
    """W is quadratic in the counts, so a central difference in the count of
    one species at one node is exact and must equal V_K at that node."""
    rng = np.random.default_rng(9)
    p = orc.make_params(3, (4, 5, 6), (4.4, 5.0, 5.4), kT=1.3, inv_kappa=0.07,
                        chi=[[0, 1.2, 0.3], [1.2, 0, 0.8], [0.3, 0.8, 0]])
    D = rng.integers(0, 6 * BEAD, size=(3, 6, 5, 4))
    V, _ = orc.field(p, D)
    for (k, z, y, x) in [(0, 1, 2, 3), (1, 5, 0, 0), (2, 3, 4, 1)]:
        Dp, Dm = D.copy(), D.copy()
        Dp[k, z, y, x] += BEAD
        Dm[k, z, y, x] -= BEAD
        dW = (orc.field_energy(p, Dp) - orc.field_energy(p, Dm)) / 2.0
        assert dW == pytest.approx(V[k, z, y, x], rel=1e-9, abs=1e-9)


def test_field_energy_closed_form_uniform_mix(orc):
    # phi_A = phi_B = 1/2 everywhere: W = rho0 * volume * chi_AB / 4
    p = unit_params(orc, mesh=(4, 4, 4), chi=[[0, 1.6], [1.6, 0]], inv_kappa=0.5, rho0=2.0)
    D = np.full((2, 4, 4, 4), BEAD, dtype=np.int64)   # one bead of each per unit cell
    assert orc.field_energy(p, D) == pytest.approx(2.0 * 64 * 1.6 / 4, rel=1e-14)


def test_field_energy_and_potential_at_kT_2_scale_only_the_chi_terms(orc):
    """Reading of the MD-SCF potential V_K = kT sum chi phi + (1/kappa)(sum phi - 1)
    with chi in kT units and 1/kappa in energy units: at kT = 2.5 only the chi
    terms scale.  Uniform phi_A = phi_B = 0.6 (1.2 beads of each per unit cell),
    chi_AB = 0.5, 1/kappa = 1.5: W = rho0 vol [kT chi phiA phiB + (1/kappa)/2
    (phiA + phiB - 1)^2] = 128 (0.45 + 0.03) and V_A = kT chi phiB + (1/kappa)
    (phiA + phiB - 1) = 0.75 + 0.3; kT multiplying 1/kappa too would give
    W = 128 (0.45 + 0.075) and V_A = 1.5."""
    p = unit_params(orc, mesh=(4, 4, 4), chi=[[0, 0.5], [0.5, 0]], inv_kappa=1.5, rho0=2.0,
                    kT=2.5)
    D = np.full((2, 4, 4, 4), 12 * BEAD // 10, dtype=np.int64)
    phi = (12 * BEAD // 10) / BEAD / 2.0
    W = 2.0 * 64 * (2.5 * 0.5 * phi * phi + 0.5 * 1.5 * (2 * phi - 1) ** 2)
    assert orc.field_energy(p, D) == pytest.approx(W, rel=1e-12)
    assert W == pytest.approx(128 * 0.48, rel=1e-9)
    V, _ = orc.field(p, D)
    assert V[0, 2, 1, 3] == pytest.approx(2.5 * 0.5 * phi + 1.5 * (2 * phi - 1), rel=1e-12)
    assert V[1, 0, 3, 2] == pytest.approx(1.05, rel=1e-9)


def test_energy_observables_of_known_state(orc):
    # no field, no friction, no noise: v_n = v_{n-1/2} + dt/(2m) F_bond with the
    # two-bead closed form F_0 = -2k(r-r0)(x0-x1)/r = (1.44, 1.92, 0) = -F_1
    p = unit_params(orc, S=1, mesh=(4, 4, 4), chi=[[0.0]], inv_kappa=0.0, gamma=0.0, mass=2.0)
    pos = np.array([[1.0, 1.0, 1.0], [1.6, 1.8, 1.0], [3.0, 3.0, 3.0]])
    vel = np.array([[1.0, 2.0, 3.0], [-1.0, 0.0, 0.5], [0.0, 0.0, 0.0]])
    V, G = orc.field(p, orc.scatter(p, pos, [0, 0, 0]))
    E = orc.energy(p, pos, vel, [0, 0, 0], [(0, 1)], V, G, 0)
    kick = 0.01 / (2 * 2.0) * np.array([1.44, 1.92, 0.0])
    vn = vel + np.array([kick, -kick, np.zeros(3)])
    ke = 0.5 * 2.0 * float((vn ** 2).sum())
    assert E[0] == pytest.approx(ke, rel=1e-14)
    assert E[1] == pytest.approx(4.0 * 0.09, rel=1e-12)
    assert E[2] == 0.0
    assert E[3] == pytest.approx(ke + 0.36, rel=1e-12)
    assert E[4] == pytest.approx(2.0 * np.linalg.norm([0.0, 2.0, 3.5]), rel=1e-14)
    assert E[5] == pytest.approx(2 * ke / 9.0, rel=1e-14)


# ------------------------------------------------------------------ integrator (A6)

def test_harmonic_dimer_matches_discrete_closed_form(orc):
    """r0 = 0 makes the bond a linear spring 2k; the relative coordinate then
    obeys d_{n+1} - 2 d_n + d_{n-1} = -w^2 dt^2 d_n with w^2 = 4k/m, whose
    solution from d_{-1} = d_0 is d_n = d_0 cos((n+1/2) th) / cos(th/2) with
    cos th = 1 - w^2 dt^2 / 2."""
    k, m, dt = 4.0, 1.0, 0.01
    p = unit_params(orc, S=1, mesh=(8, 8, 8), chi=[[0.0]], inv_kappa=0.0, gamma=0.0,
                    bond_k=k, bond_r0=0.0, mass=m, dt=dt)
    pos0 = np.array([[4.5, 4.0, 4.0], [3.5, 4.0, 4.0]])
    vel0 = np.zeros((2, 3))
    th = math.acos(1 - 4 * k / m * dt * dt / 2)
    for n in (1, 10, 250, 1000):
        pos, vel, _ = orc.run(p, pos0, vel0, [0, 0], [(0, 1)], 0, n)
        d = pos[0, 0] - pos[1, 0]
        assert d == pytest.approx(math.cos((n + 0.5) * th) / math.cos(th / 2), abs=1e-10)
        assert pos[0, 0] + pos[1, 0] == pytest.approx(8.0, abs=1e-12)  # centre of mass fixed
        assert np.all(pos[:, 1:] == 4.0)


def test_friction_without_noise_decays_geometrically(orc):
    # kT = 0: no noise; a free bead's half-step velocity is multiplied by (1 - gamma dt)
    p = unit_params(orc, S=1, mesh=(4, 4, 4), chi=[[0.0]], inv_kappa=0.0, kT=0.0, gamma=2.0,
                    dt=0.01)
    v0 = np.array([[1.0, -2.0, 0.5]])
    x0 = np.array([[1.0, 1.0, 1.0]])
    n = 37
    pos, vel, _ = orc.run(p, x0, v0, [0], [], 0, n)
    a = 1 - 2.0 * 0.01
    np.testing.assert_allclose(vel, v0 * a ** n, rtol=1e-12)
    np.testing.assert_allclose(pos, x0 + 0.01 * v0 * a * (1 - a ** n) / (1 - a), rtol=1e-12)


def test_langevin_stationary_velocity_variance(orc):
    """Free beads: v <- (1 - g dt) v + sqrt(2 g kT dt / m) xi is AR(1) with
    stationary variance kT / (m (1 - g dt / 2)) per component."""
    kT, g, dt, m = 1.5, 1.0, 0.01, 2.0
    p = unit_params(orc, S=1, mesh=(4, 4, 4), chi=[[0.0]], inv_kappa=0.0, kT=kT, gamma=g,
                    dt=dt, mass=m, field_every=1 << 30)
    n = 4000
    rng = np.random.default_rng(10)
    x0 = rng.uniform(0, 4, size=(n, 3))
    v0 = rng.normal(scale=math.sqrt(kT / m), size=(n, 3))
    pos, vel, _ = orc.run(p, x0, v0, np.zeros(n, dtype=np.int32), [], 0, 600)
    samples = [vel.copy()]
    for s in range(1, 8):   # well-separated windows (correlation time 100 steps)
        pos, vel, _ = orc.run(p, pos, vel, np.zeros(n, dtype=np.int32), [], 600 + 300 * (s - 1),
                              300)
        samples.append(vel.copy())
    var = np.var(np.concatenate(samples))
    assert var == pytest.approx(kT / (m * (1 - g * dt / 2)), rel=0.02)


def test_nve_energy_conservation_bonds_only(orc):
    """Config-1 melt, no field, no thermostat: |E(1000) - E(0)| / N < 1e-4 kT."""
    w = W.a5b5_10k()
    d = W.generate(w)
    pp = w.params()
    pp.update(gamma=0.0, chi=np.zeros((8, 8)), inv_kappa=0.0)
    p = orc.make_params(**pp)
    _, _, E = orc.run(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 1000, energies=True)
    assert abs(E[-1, 3] - E[0, 3]) / w.n_beads < 1e-4
    assert np.max(np.abs(E[:, 3] - E[0, 3])) / w.n_beads < 2e-4


def test_nve_energy_conservation_exact_gradient_field(orc):
    """Config-1 melt with the field force taken as the exact derivative of the
    CIC field energy, field refreshed every step, at dt = 0.005 (the CIC force
    jumps at cell faces, so the error per crossing is first order in dt)."""
    w = W.a5b5_10k()
    d = W.generate(w)
    pp = w.params()
    pp.update(gamma=0.0, dt=0.005, force_mode=1)
    p = orc.make_params(**pp)
    _, _, E = orc.run(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 1000, energies=True)
    assert abs(E[-1, 3] - E[0, 3]) / w.n_beads < 1e-4
    assert E[0, 2] > 0 and E[0, 1] >= 0


# ------------------------------------------------------------------ Philox / noise

def test_philox_matches_independent_implementation(orc):
    """Triton ships its own Philox4x32-10; run it in the CPU interpreter."""
    import os
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    import torch

    @triton.jit
    def kern(out_ptr, c_ptr, seed, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a.to(tl.int64))
        tl.store(out_ptr + 4 * i + 1, b.to(tl.int64))
        tl.store(out_ptr + 4 * i + 2, c.to(tl.int64))
        tl.store(out_ptr + 4 * i + 3, d.to(tl.int64))

    rng = np.random.default_rng(11)
    for seed in (0, 42, 0x1234567890ABCDEF & 0x7FFFFFFFFFFFFFFF):
        ctr = rng.integers(0, 2 ** 32, size=(8, 4), dtype=np.uint64)
        ctr[0] = 0
        ctr[1] = 2 ** 32 - 1
        out = torch.zeros(32, dtype=torch.int64)
        kern[(1,)](out, torch.from_numpy(ctr.astype(np.int64).reshape(-1)), seed, 8)
        ref = out.numpy().reshape(8, 4) & 0xFFFFFFFF
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for j in range(8):
            assert list(orc.philox(ctr[j], key)) == list(ref[j])


def test_gaussian_noise_moments():
    import oracle
    n = 60000
    xi = np.array([oracle.gauss3(42, t % 5000, t // 5000) for t in range(n)])
    assert np.all(np.abs(xi.mean(axis=0)) < 4.5 / math.sqrt(n))
    assert np.all(np.abs(xi.var(axis=0) - 1) < 4.5 * math.sqrt(2.0 / n))
    kurt = (xi ** 4).mean(axis=0) / xi.var(axis=0) ** 2
    assert np.all(np.abs(kurt - 3) < 0.1)
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c - np.eye(3)) < 4.5 / math.sqrt(n))
    # counter independence: neighbouring tags and steps are uncorrelated
    assert abs(np.corrcoef(xi[:-1, 0], xi[1:, 0])[0, 1]) < 4.5 / math.sqrt(n)


# ------------------------------------------------------------------ order (A1)

def test_cell_key_brick_major(orc):
    p = unit_params(orc, mesh=(20, 20, 20))
    # cell (9, 2, 17): brick (1, 0, 2) of 3x3x3 bricks -> 19; inside (1, 2, 1) -> 81
    assert orc.cell_key(p, [9.5, 2.5, 17.5], 8) == 19 * 512 + 81
    assert orc.cell_key(p, [-0.5, 0.5, 0.5], 8) == (2 * 512) + 3   # cell 19 wraps in x
