"""Pins of the oracle's finite-volume operators (Sec. 4.3.3: gradient,
divergence, Laplacian): exactness for linear fields on orthogonal meshes and
second-order convergence of a manufactured-solution Laplacian, including the
explicit non-orthogonal correction on jittered tetrahedra."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def _internal(om, m):
    cell, face, flipped = om.orders()
    C = np.empty_like(m.C); C[:, cell] = m.C
    Cf = np.empty_like(m.Cf); Cf[:, face] = m.Cf
    return C, Cf


@pytest.mark.parametrize("renumber", [False, True])
def test_gauss_gradient_exact_for_linear_field(renumber):
    m = mg.hex_box(5, 4, 3, (1.0, 2.0, 0.7))
    if renumber:
        m = mg.permute_cells(m, mg.random_permutation(m.n_cells, 9))
    om = O.Mesh(m, renumber=renumber)
    C, Cf = _internal(om, m)
    a = np.array([0.3, -1.7, 2.5])
    f = lambda X: a @ X + 0.25
    g = om.gauss_grad(f(C), f(Cf[:, m.n_internal_faces:]))
    assert np.allclose(g, a[:, None], rtol=0, atol=1e-12)


def test_gauss_gradient_of_constant_vanishes_on_tets():
    # closed cells (sum of outward S = 0): the Gauss gradient of a constant is
    # zero on any mesh; the Gauss gradient with linear interpolation is not
    # consistent on skewed tetrahedra, so no convergence claim is made there
    m = mg.tet_box(4, 4, 4, jitter=0.1, seed=11)
    om = O.Mesh(m, renumber=True)
    g = om.gauss_grad(np.full(m.n_cells, 3.25), np.full(m.n_boundary_faces, 3.25))
    assert np.abs(g).max() < 1e-11


def _mms_error(m, om, iters_nonorth, norm="max"):
    """-lap(phi) = 3 pi^2 phi, phi = sin(pi x) sin(pi y) sin(pi z) on the unit
    cube, phi = 0 on the walls; returns the max (or volume-weighted L2)
    error at the cell centres."""
    C, Cf = _internal(om, m)
    F = m.n_internal_faces
    exact = np.sin(np.pi * C[0]) * np.sin(np.pi * C[1]) * np.sin(np.pi * C[2])
    fb = np.sin(np.pi * Cf[0, F:]) * np.sin(np.pi * Cf[1, F:]) * np.sin(np.pi * Cf[2, F:])
    V = om.geometry()["V"]
    own, nei = om.addressing()
    x = np.zeros(m.n_cells)
    gradx = None
    for _ in range(max(1, iters_nonorth)):
        d, up, b = om.laplacian_system(fb, gradx)
        b = b + 3 * np.pi ** 2 * exact * V
        x, it, r0, r1, st = O.pcg(own, nei, d, up, b, x, tol=1e-13, maxit=20000)
        assert st == 0
        if iters_nonorth:
            gradx = om.gauss_grad(x, fb)
    if norm == "l2":
        return np.sqrt(np.sum((x - exact) ** 2 * V))
    return np.abs(x - exact).max()


def test_laplacian_mms_second_order_hex():
    errs = []
    for n in (8, 16, 32):
        m = mg.hex_box(n, n, n)
        om = O.Mesh(m, renumber=True)
        errs.append(_mms_error(m, om, 0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 >= 3.5 and r2 >= 3.5, errs


def test_nonorthogonal_correction_exact_for_linear_field_tets():
    # over-relaxed split n = delta d + k: with the exact gradient in the
    # explicit term, the face flux |S| delta (x_N - x_P) + |S| k.grad x equals
    # S.grad x for a linear field, so the exact field satisfies the assembled
    # system in every cell without boundary faces (no correction is applied
    # on boundary faces)
    m = mg.tet_box(5, 5, 5, jitter=0.1, seed=5)
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


def test_nonorthogonal_correction_reduces_mms_error_tets():
    # the Gauss gradient with linear interpolation is not consistent on skewed
    # tetrahedra, so the lagged correction does not restore second order; it
    # must still cut the error clearly on every mesh
    for n in (4, 8):
        m = mg.tet_box(n, n, n, jitter=0.1, seed=5)
        om = O.Mesh(m, renumber=True)
        assert om.nonorth
        e1, e0 = _mms_error(m, om, 12, "l2"), _mms_error(m, om, 0, "l2")
        assert e1 < 0.5 * e0, (n, e1, e0)
