"""Pins of the oracle's mesh addressing and geometry.

Reverse Cuthill-McKee order and face order are checked on a small box
computed by hand; the geometric quantities (interpolation weight, delta
coefficient, non-orthogonal vector) against their closed forms on uniform
hexahedra."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def test_rcm_hand_example_3x2():
    # 3x2x1 box, cells i + 3 j:      0 1 2
    #                                3 4 5
    # degrees 2,3,2,2,3,2.  Start = lowest-index minimum-degree cell 0;
    # BFS with neighbours in (degree, index) order: 0 | 3 1 | 4 | 2 | 5
    # -> [0, 3, 1, 4, 2, 5], reversed -> [5, 2, 4, 1, 3, 0].
    m = mg.hex_box(3, 2, 1)
    om = O.Mesh(m, renumber=True)
    cell, face, flipped = om.orders()
    assert cell.tolist() == [5, 3, 1, 4, 2, 0]
    # internal faces of the generator: (0,1) (3,4) (1,2) (4,5) (0,3) (1,4) (2,5)
    # renumbered:  (3,5) (2,4) (1,3) (0,2) (4,5) (2,3) (0,1), all flipped;
    # sorted by (owner, neighbour): (0,1) (0,2) (1,3) (2,3) (2,4) (3,5) (4,5)
    assert [tuple(x) for x in zip(m.owner[:7], m.neighbour)] == [(0, 1), (3, 4), (1, 2), (4, 5),
                                                                 (0, 3), (1, 4), (2, 5)]
    assert face[:7].tolist() == [5, 4, 2, 1, 6, 3, 0]
    assert flipped[:7].tolist() == [1] * 7
    own, nei = om.addressing()
    assert list(zip(own[:7].tolist(), nei.tolist())) == [(0, 1), (0, 2), (1, 3), (2, 3), (2, 4),
                                                           (3, 5), (4, 5)]


def test_rcm_hand_example_2x2():
    # four cells of equal degree: BFS 0 1 2 3, reversed -> new_of_old 3 2 1 0
    om = O.Mesh(mg.hex_box(2, 2, 1), renumber=True)
    assert om.orders()[0].tolist() == [3, 2, 1, 0]


def test_identity_order_keeps_cells():
    m = mg.cavity3d(4)
    om = O.Mesh(m, renumber=False)
    cell, face, flipped = om.orders()
    assert np.array_equal(cell, np.arange(m.n_cells))
    assert not flipped.any()


def _bandwidth(own, nei):
    return int(np.max(np.abs(nei.astype(np.int64) - own[:len(nei)])))


def test_rcm_permutation_and_bandwidth():
    m = mg.cavity3d(9)
    perm = mg.random_permutation(m.n_cells, 1234)
    mp = mg.permute_cells(m, perm)
    om = O.Mesh(mp, renumber=True)
    cell, face, flipped = om.orders()
    assert np.array_equal(np.sort(cell), np.arange(m.n_cells))
    assert np.array_equal(np.sort(face), np.arange(m.n_faces))
    own, nei = om.addressing()
    F = m.n_internal_faces
    # banded after RCM: no worse than the natural lexicographic order + margin
    natural = _bandwidth(m.owner, m.neighbour)
    assert _bandwidth(own, nei) <= natural + 2 * 9
    assert _bandwidth(mp.owner, mp.neighbour) > 5 * natural
    # orientation owner < neighbour; faces sorted by (owner, neighbour)
    assert (own[:F] < nei).all()
    key = own[:F].astype(np.int64) * m.n_cells + nei
    assert (np.diff(key) > 0).all()
    # re-oriented faces: own/nei are the relabelled endpoints, flipped iff swapped
    a, b = cell[mp.owner[:F]], cell[mp.neighbour]
    pos = face[:F]
    assert np.array_equal(own[pos], np.minimum(a, b))
    assert np.array_equal(nei[pos], np.maximum(a, b))
    assert np.array_equal(flipped[:F].astype(bool), a > b)
    # boundary faces: sorted by (patch, new owner, original index) and kept in patch
    Bpos = face[F:] - F
    patch_of = np.concatenate([np.full(p.size, q) for q, p in enumerate(mp.patches)])
    order = np.lexsort((np.arange(m.n_boundary_faces), cell[mp.owner[F:]], patch_of))
    assert np.array_equal(Bpos[order], np.arange(m.n_boundary_faces))
    # area vectors follow the flips
    g = om.geometry()
    sgn = np.where(flipped[:F] == 1, -1.0, 1.0)
    assert np.array_equal(g["Sf"][:, pos], mp.Sf[:, :F] * sgn)


def test_uniform_hex_geometry():
    m = mg.hex_box(4, 3, 5, (2.0, 1.5, 1.0))
    om = O.Mesh(m, renumber=False)
    g = om.geometry()
    F = m.n_internal_faces
    assert np.allclose(g["w"], 0.5, atol=1e-15)
    h = np.array([0.5, 0.5, 0.2])
    axis = np.argmax(np.abs(g["Sf"][:, :F]), axis=0)
    assert np.allclose(g["delta"][:F], 1.0 / h[axis], rtol=1e-14)
    assert np.abs(g["kv"]).max() < 1e-12
    # boundary delta = 1 / (half cell width)
    axb = np.argmax(np.abs(g["Sf"][:, F:]), axis=0)
    assert np.allclose(g["delta"][F:], 2.0 / h[axb], rtol=1e-14)
    assert np.allclose(g["magSf"], np.linalg.norm(g["Sf"], axis=0), rtol=1e-15)
    assert not om.nonorth


def test_tet_geometry_is_nonorthogonal():
    m = mg.tet_box(3, 3, 3, jitter=0.1)
    om = O.Mesh(m, renumber=True)
    g = om.geometry()
    assert om.nonorth
    assert ((g["w"] > 0.0) & (g["w"] < 1.0)).all()
    # over-relaxed split: S = |S| delta d + |S| k  ->  n = delta d + k
    own, nei = om.addressing()
    F = m.n_internal_faces
    # recover cell centres in internal order
    cell = om.orders()[0]
    C = np.empty_like(m.C); C[:, cell] = m.C
    d = C[:, nei] - C[:, own[:F]]
    n = g["Sf"][:, :F] / g["magSf"][:F]
    assert np.allclose(n, g["delta"][:F] * d + g["kv"], atol=1e-14)
    # k is orthogonal-free: n.d delta = 1 whenever the max() guard is inactive
    assert np.allclose(np.einsum("ij,ij->j", n, d) * g["delta"][:F], 1.0, atol=1e-12)
