"""Pins of the oracle's literal Algorithm 1 field force (force_mode 2).

Kernels 3-4 of Algorithm 1 blend, per axis, the backward and forward
differences of the field at the bead's vertex with two fraction ratios.  Read
as the linear weights between the two half-points around the nearest vertex,
the force component is minus the derivative of the 1-D quadratic through
V(c - 1), V(c), V(c + 1) on that vertex's grid line, evaluated at the bead.
Pins that fix this: the scheme is exact for quadratic fields along each axis
(with an anisotropic box, so no axis or spacing can be swapped); on a vertex
it is the central difference; it is continuous where the nearest vertex
changes (half-way between vertices); on a sinusoid it gives the closed form
-sin(kh) cos(k x_node) / h at the nodes; it wraps periodically; and each bead
reads its own species' potential.
"""
import numpy as np
import pytest

MESH = (16, 12, 10)
BOX = (11.0, 9.5, 13.0)


def params(orc, S=1):
    return orc.make_params(S, MESH, BOX, chi=np.zeros((S, S)), force_mode=2)


def node_grid(axis):
    """Node index along `axis` for every node of the [Mz][My][Mx] mesh."""
    z, y, x = np.meshgrid(np.arange(MESH[2]), np.arange(MESH[1]), np.arange(MESH[0]),
                          indexing="ij")
    return (x, y, z)[axis].astype(np.float64)


def place(orc, p, s):
    """Positions whose FP32 mesh coordinates are s, or the nearest the FP32
    product reaches (the tests use the returned coordinates)."""
    pos = np.zeros((len(s), 3))
    got = np.zeros((len(s), 3))
    for a in range(3):
        ih = np.float32(orc.inv_h(p, a))
        x = (np.asarray(s[:, a], np.float32) / ih).astype(np.float32)
        for k in range(len(x)):
            while np.float32(x[k] * ih) < np.float32(s[k, a]):
                x[k] = np.nextafter(x[k], np.float32(np.inf))
            got[k, a] = np.float32(x[k] * ih)
        pos[:, a] = x
    return pos, got


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quadratic_field_is_exact(orc, axis):
    p = params(orc)
    i = node_grid(axis)
    a0, b, c = 0.3, -0.7, 0.05
    V = (a0 + b * i + c * i * i)[None]
    rng = np.random.default_rng(axis)
    s = rng.uniform(2.6, np.array(MESH) - 3.6, size=(200, 3)).astype(np.float32).astype(np.float64)
    pos, s = place(orc, p, s)
    F = orc.field_force_staggered(p, pos, np.zeros(len(s), np.int32), V)
    ih = MESH[axis] / BOX[axis]  # the force scale 1/h (the coordinate uses fl32 of it)
    np.testing.assert_allclose(F[:, axis], -ih * (b + 2 * c * s[:, axis]), rtol=1e-12, atol=1e-12)
    for other in {0, 1, 2} - {axis}:
        assert np.all(F[:, other] == 0.0)


def test_on_a_vertex_it_is_the_central_difference(orc):
    p = params(orc)
    rng = np.random.default_rng(1)
    V = rng.normal(size=(1,) + MESH[::-1])
    s = np.array([[3, 4, 5], [7, 2, 8], [15, 11, 9], [0, 0, 0]], dtype=np.float64)
    pos, got = place(orc, p, s)
    assert np.array_equal(got, s)  # integers are reached exactly
    F = orc.field_force_staggered(p, pos, np.zeros(4, np.int32), V)
    for k, (x, y, z) in enumerate(s.astype(int)):
        for a, (lo, hi) in enumerate([
                (V[0, z, y, (x - 1) % 16], V[0, z, y, (x + 1) % 16]),
                (V[0, z, (y - 1) % 12, x], V[0, z, (y + 1) % 12, x]),
                (V[0, (z - 1) % 10, y, x], V[0, (z + 1) % 10, y, x])]):
            assert F[k, a] == pytest.approx(-MESH[a] / BOX[a] * (hi - lo) / 2, rel=1e-12)


def test_continuous_where_the_nearest_vertex_changes(orc):
    """Half-way between vertices k and k + 1 both sides give the one-sided
    difference V(k + 1) - V(k)."""
    p = params(orc)
    rng = np.random.default_rng(2)
    V = rng.normal(size=(1,) + MESH[::-1])
    eps = 2.0 ** -18
    s = np.array([[6.5 - eps, 3, 4], [6.5 + eps, 3, 4], [6.5, 3, 4]])
    pos, got = place(orc, p, s)
    assert got[0, 0] < 6.5 < got[1, 0] and got[2, 0] == 6.5
    F = orc.field_force_staggered(p, pos, np.zeros(3, np.int32), V)
    one_sided = -MESH[0] / BOX[0] * (V[0, 4, 3, 7] - V[0, 4, 3, 6])
    assert F[2, 0] == pytest.approx(one_sided, rel=1e-12)
    scale = np.abs(V).max() * MESH[0] / BOX[0]
    assert abs(F[0, 0] - one_sided) < 4 * eps * scale
    assert abs(F[1, 0] - one_sided) < 4 * eps * scale


def test_sinusoid_closed_form_and_periodic_wrap(orc):
    p = params(orc)
    M = MESH[0]
    k = 2 * np.pi * 3 / M
    V = np.sin(k * node_grid(0))[None]
    ih = MESH[0] / BOX[0]
    # on the nodes, including node 0 (whose lower neighbour wraps to M - 1)
    s = np.array([[x, 5, 5] for x in range(M)], dtype=np.float64)
    F = orc.field_force_staggered(p, place(orc, p, s)[0], np.zeros(M, np.int32), V)
    np.testing.assert_allclose(F[:, 0], -ih * np.sin(k) * np.cos(k * np.arange(M)), atol=1e-12)
    # a bead just below the box end has node 0 as its nearest vertex
    s2 = np.array([[M - 0.25, 5, 5], [-0.25, 5, 5]])
    F2 = orc.field_force_staggered(p, place(orc, p, s2)[0], np.zeros(2, np.int32), V)
    assert F2[0, 0] == pytest.approx(F2[1, 0], rel=1e-6)


def test_each_bead_reads_its_species(orc):
    p = params(orc, S=2)
    i = node_grid(1)
    V = np.stack([0.4 * i, -1.3 * i])
    s = np.array([[5.2, 4.3, 6.1], [5.2, 4.3, 6.1]])
    F = orc.field_force_staggered(p, place(orc, p, s)[0], np.array([0, 1], np.int32), V)
    ih = MESH[1] / BOX[1]
    assert F[0, 1] == pytest.approx(-0.4 * ih, rel=1e-12)
    assert F[1, 1] == pytest.approx(1.3 * ih, rel=1e-12)


def test_continuous_across_a_vertex(orc):
    """The vertex is the nearest one: just below and just above vertex 7 the
    force tends to the central difference there (a cell's lower vertex would
    extrapolate on one side and jump)."""
    p = params(orc)
    rng = np.random.default_rng(4)
    V = rng.normal(size=(1,) + MESH[::-1])
    eps = 2.0 ** -18
    pos, got = place(orc, p, np.array([[7 - eps, 3, 4], [7 + eps, 3, 4]]))
    assert got[0, 0] < 7 < got[1, 0]
    F = orc.field_force_staggered(p, pos, np.zeros(2, np.int32), V)
    central = -MESH[0] / BOX[0] * (V[0, 4, 3, 8] - V[0, 4, 3, 6]) / 2
    scale = np.abs(V).max() * MESH[0] / BOX[0]
    assert abs(F[0, 0] - central) < 8 * eps * scale
    assert abs(F[1, 0] - central) < 8 * eps * scale
