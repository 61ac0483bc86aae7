"""The oracle against hand-computed fixtures in tests/golden/.

The paper prints no worked numerical example of the method (its tables are
performance figures), so the stored values here are worked out by hand from
the definitions each fixture cites (MD-SCF section: the CIC scheme on the
cell's vertices and the two-component external potential; Algorithm 1,
kernels 2-3) and the arithmetic is shown in the fixture's header.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read(name):
    meta, rows = {}, []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line:
            continue
        if line.startswith("#"):
            if ":" in line:
                k, v = line[1:].split(":", 1)
                meta[k.strip()] = v.strip()
            continue
        rows.append(line.split())
    return meta, rows


def test_single_bead_cic_counts(orc):
    meta, rows = read("cic_single_bead.txt")
    mesh = tuple(int(v) for v in meta["mesh"].split())
    box = tuple(float(v) for v in meta["box"].split())
    b = meta["bead"].split()
    p = orc.make_params(1, mesh, box, chi=np.zeros((1, 1)))
    D = orc.scatter(p, np.array([[float(b[1]), float(b[2]), float(b[3])]]),
                    np.array([int(b[0])], np.int32))
    want = np.zeros_like(D)
    for k, ix, iy, iz, count in rows:
        want[int(k), int(iz), int(iy), int(ix)] = int(count)
    assert int(want.sum()) == 1 << 39
    assert np.array_equal(D, want)


def test_two_species_potential_and_gradient(orc):
    meta, rows = read("potential_two_species.txt")
    mesh = tuple(int(v) for v in meta["mesh"].split())
    box = tuple(float(v) for v in meta["box"].split())
    chi = float(meta["chi_ab"])
    p = orc.make_params(2, mesh, box, kT=float(meta["kT"]), rho0=float(meta["rho0"]),
                        inv_kappa=float(meta["inv_kappa"]), chi=[[0.0, chi], [chi, 0.0]])
    beads = [b.split() for b in meta["beads"].split("(")[0].split("/")]
    pos = np.array([[float(v) for v in b[1:4]] for b in beads])
    types = np.array([int(b[0]) for b in beads], np.int32)
    V, G = orc.field(p, orc.scatter(p, pos, types))
    axis = {"dVdx": 0, "dVdy": 1, "dVdz": 2}
    checked = 0
    for q, k, ix, iy, iz, val in rows:
        k, ix, iy, iz, val = int(k), int(ix), int(iy), int(iz), float(val)
        got = V[k, iz, iy, ix] if q == "V" else G[k, iz, iy, ix, axis[q]]
        assert got == pytest.approx(val, abs=1e-12), (q, k, ix, iy, iz)
        checked += 1
    assert checked == len(rows) == 13
