"""Pins of the synthetic mesh generators (inputs shared by oracle and GPU).

Table 1 of the paper (Sec. 4.1) lists the cell and face counts of the
structured cavity meshes and of the tp1M channel; the generators must
reproduce them exactly.  Geometric invariants (closed cells, total volume,
outward orientation) pin the face area vectors and volumes."""
import os

import numpy as np
import pytest

import meshgen as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_meshes.txt")


def _table1():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, cells, faces, _ = line.split()
        rows[name] = (int(cells), int(faces))
    return rows


def _closure(m):
    s = np.zeros((3, m.n_cells))
    F = m.n_internal_faces
    for d in range(3):
        np.add.at(s[d], m.owner, m.Sf[d])
        np.add.at(s[d], m.neighbour, -m.Sf[d, :F])
    return np.abs(s).max()


@pytest.mark.parametrize("n", [10, 47])
def test_table1_cube_generated(n):
    cells, faces = _table1()[f"cav{n}^3"]
    m = mg.cavity3d(n)
    assert m.n_cells == cells
    assert m.n_internal_faces + m.n_boundary_faces == faces


@pytest.mark.parametrize("n", [100, 181, 223])
def test_table1_cube_counts(n):
    # the large cubes are checked through the generator's own counting rule,
    # itself verified on the small cubes above
    cells, faces = _table1()[f"cav{n}^3"]
    assert n ** 3 == cells
    assert mg.table1_face_count(n) == faces
    m = mg.cavity3d(6)
    assert m.n_internal_faces + m.n_boundary_faces == mg.table1_face_count(6)


def test_table1_tp1m():
    cells, faces = _table1()["tp1M"]
    m = mg.channel2d(3200, 300, 0.16, 0.02)
    assert m.n_cells == cells
    assert m.n_internal_faces + m.n_boundary_faces == faces


@pytest.mark.parametrize("maker", [lambda: mg.cavity3d(5), lambda: mg.cavity2d(7, 4),
                                   lambda: mg.tet_box(3, 4, 2, (1.0, 2.0, 0.5), 0.1, 5),
                                   lambda: mg.duct_tets(4, 8)])
def test_cells_closed_and_volume(maker):
    m = maker()
    assert _closure(m) < 1e-14
    lo = np.min(m.Cf, axis=1); hi = np.max(m.Cf, axis=1)
    assert m.V.sum() == pytest.approx(np.prod(hi - lo), rel=1e-12)
    F = m.n_internal_faces
    # internal S points from owner to neighbour, boundary S out of the domain
    assert (np.einsum("ij,ij->j", m.Sf[:, :F], m.C[:, m.neighbour] - m.C[:, m.owner[:F]]) > 0).all()
    assert (np.einsum("ij,ij->j", m.Sf[:, F:], m.Cf[:, F:] - m.C[:, m.owner[F:]]) > 0).all()
    # patches tile the boundary
    assert sum(p.size for p in m.patches) == m.n_boundary_faces
    assert [p.start for p in m.patches] == list(np.cumsum([0] + [p.size for p in m.patches])[:-1])


def test_kuhn_counts():
    n, L = 4, 6
    m = mg.tet_box(n, n, L, jitter=0.1)
    assert m.n_cells == 6 * n * n * L
    assert m.n_boundary_faces == 2 * (2 * n * n + 4 * n * L)
    assert 2 * m.n_internal_faces + m.n_boundary_faces == 4 * m.n_cells
    # channel of the SIMPLE workload: 48x48x192 -> 2,654,208 tets
    assert 6 * 48 * 48 * 192 == 2654208


def test_jitter_moves_interior_only():
    a = mg.tet_box(3, 3, 3, jitter=0.0)
    b = mg.tet_box(3, 3, 3, jitter=0.1, seed=1)
    # same connectivity, boundary nodes fixed: boundary faces are unchanged
    assert np.array_equal(a.owner, b.owner)
    assert np.allclose(a.Cf[:, a.n_internal_faces:], b.Cf[:, b.n_internal_faces:], atol=1e-15)
    assert not np.allclose(a.C, b.C)
    assert a.V.sum() == pytest.approx(b.V.sum(), rel=1e-12)


def test_permutation_relabels():
    m = mg.cavity3d(4)
    perm = mg.random_permutation(m.n_cells, 1234)
    p = mg.permute_cells(m, perm)
    assert np.array_equal(p.owner, perm[m.owner])
    assert np.allclose(p.C[:, perm], m.C)
    assert p.corner_cell == perm[0]
    assert _closure(p) < 1e-14


def test_batch_sampler():
    cases = mg.batch_cases()
    assert len(cases) == 256
    ns = np.array([c[0] for c in cases]); re = 1.0 / np.array([c[1] for c in cases])
    assert ns.min() >= 32 and ns.max() <= 128
    assert re.min() >= 10.0 and re.max() <= 1000.0
    assert cases == mg.batch_cases()


def test_graded_box_reduces_to_uniform_box():
    # equal spacing gives the uniform generator's mesh (same numbering,
    # same faces, geometry to rounding)
    u = mg.hex_box(5, 4, 3, (1.0, 2.0, 0.6))
    g = mg.graded_box(mg.geometric_nodes(5, 1.0, 1.0), mg.geometric_nodes(4, 2.0, 1.0),
                      mg.geometric_nodes(3, 0.6, 1.0))
    assert np.array_equal(u.owner, g.owner) and np.array_equal(u.neighbour, g.neighbour)
    for a in ("Sf", "Cf", "C", "V"):
        assert np.allclose(getattr(u, a), getattr(g, a), rtol=0, atol=1e-15), a
    x = mg.geometric_nodes(6, 2.0, 1.3)
    h = np.diff(x)
    assert x[0] == 0.0 and x[-1] == 2.0 and np.allclose(h[1:] / h[:-1], 1.3, rtol=1e-13)
