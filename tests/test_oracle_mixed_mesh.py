"""Pins of the oracle on mixed-element meshes (hexahedra, triangular prisms
and pyramids; meshgen.mixed_box), the unstructured non-orthogonal meshes the
paper's artery case stands for (Sec. 4.1, Table 1 lca0.5M; Sec. 4.3.3 and
Sec. 5 on the cost of the non-orthogonal Laplacian).

* geometry: every cell closed (sum of outward area vectors zero), the cell
  volumes and first moments add up to the box's;
* Gauss gradient of a linear field exact in the hexahedra whose neighbours
  are hexahedra or pyramids (their face centres lie on the centroid
  segments; across a hexahedron-pyramid face the weight is 0.8 / 0.2);
* with the exact gradient in the explicit non-orthogonal term, a linear
  field satisfies the assembled Laplacian in every interior cell of a
  jittered mixed mesh (the over-relaxed split S = |S| delta d + |S| k);
* the manufactured-solution error falls with refinement, and the
  non-orthogonal correction lowers it (by more than 2x once the mesh
  resolves the solution); as on skewed tetrahedra, the Gauss gradient with
  linear interpolation is not consistent on skewed cells, so no order of
  convergence is claimed;
* PISO steps with non-orthogonal correctors keep the continuity identity of
  the flux correction and the zero net flux of the closed cavity."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def _internal(om, m):
    cell, face, flipped = om.orders()
    C = np.empty_like(m.C); C[:, cell] = m.C
    Cf = np.empty_like(m.Cf); Cf[:, face] = m.Cf
    return C, Cf


@pytest.mark.parametrize("jitter", [0.0, 0.15])
def test_mixed_mesh_geometry_closes(jitter):
    m = mg.mixed_box(6, 5, 4, (1.2, 1.0, 0.8), jitter=jitter, seed=3)
    F, N = m.n_internal_faces, m.n_cells
    net = np.zeros((3, N))
    np.add.at(net.T, m.owner, m.Sf.T)
    np.add.at(net.T, m.neighbour, -m.Sf[:, :F].T)
    assert np.abs(net).max() < 1e-15
    vol = 1.2 * 1.0 * 0.8
    assert abs(m.V.sum() - vol) < 1e-14 and m.V.min() > 0
    assert np.allclose((m.V * m.C).sum(axis=1), vol * np.array([0.6, 0.5, 0.4]), rtol=0, atol=1e-14)
    # the three element kinds are all there (volumes h^3, h^3/2, h^3/6 before jitter)
    if jitter == 0.0:
        h3 = 0.2 * 0.2 * 0.2
        kinds = {round(v / h3 * 6) for v in m.V}
        assert kinds == {6, 3, 1}
    # face centres of the boundary lie on the box (boundary nodes are fixed)
    om = O.Mesh(m, renumber=True)
    assert om.nonorth


def test_gauss_gradient_exact_in_hexes_next_to_hexes_and_pyramids():
    # prism columns every fifth diagonal, so some hexahedra have none as neighbour
    m = mg.mixed_box(6, 6, 6, jitter=0.0, prism_every=5)
    h3 = (1.0 / 6) ** 3
    kind = np.rint(m.V / h3 * 6).astype(int)          # 6 hex, 3 prism, 1 pyramid
    F = m.n_internal_faces
    ok = kind == 6
    bad_nb = np.zeros(m.n_cells, bool)
    for a, b in ((m.owner[:F], m.neighbour), (m.neighbour, m.owner[:F])):
        bad_nb[a[kind[b] == 3]] = True
    sel = ok & ~bad_nb
    assert sel.sum() >= 20
    om = O.Mesh(m, renumber=True)
    cell = om.orders()[0]
    C, Cf = _internal(om, m)
    a = np.array([0.3, -1.7, 2.5])
    f = lambda X: a @ X + 0.25
    g = om.gauss_grad(f(C), f(Cf[:, F:]))
    sel_int = np.zeros(m.n_cells, bool); sel_int[cell[sel]] = True
    assert np.abs(g[:, sel_int] - a[:, None]).max() < 1e-12
    # the weights across hexahedron-pyramid faces are 0.8 / 0.2
    w = om.geometry()["w"]
    assert np.isclose(w, 0.8).any() and np.isclose(w, 0.2).any()
    # and the mesh is not exact everywhere (prisms are off the segments)
    assert np.abs(g - a[:, None]).max() > 1e-3


def test_nonorthogonal_correction_exact_for_linear_field_mixed():
    m = mg.mixed_box(5, 5, 5, jitter=0.15, seed=7)
    om = O.Mesh(m, renumber=True)
    C, Cf = _internal(om, m)
    F = m.n_internal_faces
    a = np.array([0.7, -0.4, 1.3])
    xe = a @ C + 0.5
    xb = a @ Cf[:, F:] + 0.5
    own, nei = om.addressing()
    interior = np.ones(m.n_cells, bool)
    interior[own[F:]] = False
    assert interior.sum() > 100
    grad = np.repeat(a[:, None], m.n_cells, axis=1)
    d, up, b = om.laplacian_system(xb, grad)
    res = b - O.ldu_matvec(own, nei, d, up, up, xe)
    scale = np.abs(d * xe).max()
    assert np.abs(res[interior]).max() < 1e-12 * scale
    d0, up0, b0 = om.laplacian_system(xb, None)
    res0 = b0 - O.ldu_matvec(own, nei, d0, up0, up0, xe)
    assert np.abs(res0[interior]).max() > 1e-3 * scale


def _mms(m, iters_nonorth):
    om = O.Mesh(m, renumber=True)
    C, Cf = _internal(om, m)
    F = m.n_internal_faces
    s = lambda X: np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])
    exact, fb = s(C), s(Cf[:, F:])
    V = om.geometry()["V"]
    own, nei = om.addressing()
    x, gradx = np.zeros(m.n_cells), None
    for _ in range(max(1, iters_nonorth)):
        d, up, b = om.laplacian_system(fb, gradx)
        b = b + 3 * np.pi ** 2 * exact * V
        x, it, r0, r1, st = O.pcg(own, nei, d, up, b, x, tol=1e-13, maxit=20000)
        assert st == 0
        if iters_nonorth:
            gradx = om.gauss_grad(x, fb)
    return np.sqrt(np.sum((x - exact) ** 2 * V))


def test_mms_error_falls_with_refinement_mixed():
    e = {}
    for n in (4, 8, 16):
        m = mg.mixed_box(n, n, n, jitter=0.1, seed=5)
        e[n] = (_mms(m, 10), _mms(m, 0))
        assert e[n][0] < e[n][1], (n, e[n])
    assert e[4][0] > e[8][0] > e[16][0], e
    assert e[8][0] < 0.5 * e[8][1] and e[16][0] < 0.5 * e[16][1], e


@pytest.mark.parametrize("nn", [0, 2])
def test_piso_on_mixed_cavity_keeps_continuity(nn):
    m = mg.mixed_cavity3d(6, jitter=0.12, seed=9)
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.05)
    for _ in range(4):
        s = oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        assert s["status"] == 0 and s["cont_err"] < 1e-12, s
    u, p, phi = oc.get_fields()
    F = m.n_internal_faces
    assert abs(phi[F:].sum()) < 1e-12 * np.abs(phi).max()
    assert np.isfinite(u).all() and np.abs(u).max() < 2.0
