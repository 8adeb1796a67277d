"""Pins of the face-interpolation weight w on graded (non-uniform) orthogonal
hexahedral meshes.

On a uniform mesh every face lies half-way between the two cell centroids,
so w = 1/2 and the convention "x_f = w x_P + (1 - w) x_N" cannot be told
apart from its mirror "x_f = (1 - w) x_P + w x_N".  On a graded mesh it can:
linear interpolation to the face centre reproduces a linear field exactly
only with the right weight.  Each test below holds a closed-form fact of
the textbook finite-volume method (the discretisation the paper's Sec. 3
says it follows) that fails when w and 1 - w are exchanged in the oracle:

* the Gauss gradient of a linear field is exact (face values of a linear
  field are exact at face centres lying on the centroid segment);
* the central-convection operator of the momentum matrix applied to the
  linear stagnation-point flow u = (x, -y, 0) with its exact face fluxes
  equals the exact cell integral of div(u u) = (x, y, 0), V times its value
  at the centroid (diffusion of a linear field cancels exactly on
  orthogonal meshes).

The Laplacian manufactured solution and plane Couette flow do not involve w
on orthogonal meshes; they are kept here as graded-mesh consistency checks
(second-order convergence, exact linear state)."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def _internal(om, m):
    cell, face, flipped = om.orders()
    C = np.empty_like(m.C); C[:, cell] = m.C
    Cf = np.empty_like(m.Cf); Cf[:, face] = m.Cf
    return C, Cf


def _box(nx, ny, nz, rx, ry, rz, L=(1.0, 1.3, 0.8), **kw):
    return mg.graded_box(mg.geometric_nodes(nx, L[0], rx), mg.geometric_nodes(ny, L[1], ry),
                         mg.geometric_nodes(nz, L[2], rz), **kw)


def test_graded_box_is_closed_and_orthogonal():
    m = _box(7, 5, 4, 1.3, 0.75, 1.2)
    F = m.n_internal_faces
    net = np.zeros((3, m.n_cells))
    np.add.at(net.T, m.owner, m.Sf.T)
    np.add.at(net.T, m.neighbour, -m.Sf[:, :F].T)
    assert np.abs(net).max() < 1e-15
    assert abs(m.V.sum() - 1.0 * 1.3 * 0.8) < 1e-14
    om = O.Mesh(m, renumber=True)
    assert not om.nonorth
    g = om.geometry()
    # the weights really differ from 1/2 on both sides
    assert g["w"].min() < 0.45 and g["w"].max() > 0.55


@pytest.mark.parametrize("renumber", [False, True])
def test_gauss_gradient_exact_for_linear_field_graded(renumber):
    m = _box(7, 5, 4, 1.3, 0.75, 1.2)
    if renumber:
        m = mg.permute_cells(m, mg.random_permutation(m.n_cells, 21))
    om = O.Mesh(m, renumber=renumber)
    C, Cf = _internal(om, m)
    a = np.array([0.3, -1.7, 2.5])
    f = lambda X: a @ X + 0.25
    g = om.gauss_grad(f(C), f(Cf[:, m.n_internal_faces:]))
    assert np.allclose(g, a[:, None], rtol=0, atol=1e-12)


def test_central_convection_exact_for_stagnation_flow_graded():
    # all six sides carry fixed (face-wise) velocities: the exact values
    specs = {"walls": (mg.INLET, (0.0, 0.0, 0.0), 0.0)}
    m = _box(8, 6, 5, 1.25, 0.8, 1.15, L=(1.0, 1.0, 1.0), patch_specs=specs)
    m = mg.permute_cells(m, mg.random_permutation(m.n_cells, 5))
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.3)
    U = lambda X: np.stack([X[0], -X[1], 0.0 * X[2]])
    cs.set_patch_faces(0, U(m.Cf[:, m.n_internal_faces:]))
    phi = np.einsum("ij,ij->j", U(m.Cf), m.Sf)       # exact face fluxes
    cs.set_fields(U(m.C), np.zeros(m.n_cells), phi)
    d, up, lo, src = cs.momentum_system(transient=False, alpha_u=1.0)
    C, _ = _internal(om, m)
    V = om.geometry()["V"]
    own, nei = om.addressing()
    F = m.n_internal_faces
    u = U(C)
    for c, exact in enumerate((C[0], C[1], 0.0 * C[2])):
        Mu = d * u[c]
        np.add.at(Mu, own[:F], up * u[c][nei])
        np.add.at(Mu, nei, lo * u[c][own[:F]])
        lhs = Mu - src[c]
        scale = np.abs(d * u[c]).max() + np.abs(V).max()
        assert np.abs(lhs - V * exact).max() < 1e-12 * scale, c


def _mms_error(m, om):
    C, Cf = _internal(om, m)
    F = m.n_internal_faces
    s = lambda X: np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])
    exact, fb = s(C), s(Cf[:, F:])
    V = om.geometry()["V"]
    own, nei = om.addressing()
    d, up, b = om.laplacian_system(fb, None)
    b = b + 3 * np.pi ** 2 * exact * V
    x, it, r0, r1, st = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-13, maxit=20000)
    assert st == 0
    return np.sqrt(np.sum((x - exact) ** 2 * V))


def test_laplacian_mms_second_order_graded():
    # a fixed total expansion (largest / smallest cell = 4 along each axis),
    # so that refinement halves every cell of a smooth mapping
    errs = []
    for n in (8, 16, 32):
        r = 4.0 ** (1.0 / (n - 1))
        m = _box(n, n, n, r, 1.0 / r, r, L=(1.0, 1.0, 1.0))
        errs.append(_mms_error(m, O.Mesh(m, renumber=True)))
    assert errs[0] / errs[1] >= 3.5 and errs[1] / errs[2] >= 3.5, errs


def test_couette_exact_state_is_preserved_graded():
    ys = mg.geometric_nodes(8, 1.0, 1.3)
    xs = mg.geometric_nodes(12, 2.0, 0.85)
    sp = {"xmin": "inlet", "xmax": "outlet", "ymin": "bottom", "ymax": "top",
          "zmin": "frontAndBack", "zmax": "frontAndBack"}
    specs = {"inlet": (mg.INLET, (0.0, 0.0, 0.0), 0.0), "outlet": (mg.OUTLET, (0.0, 0.0, 0.0), 0.0),
             "bottom": (mg.WALL, (0.0, 0.0, 0.0), 0.0), "top": (mg.WALL, (1.0, 0.0, 0.0), 0.0),
             "frontAndBack": (mg.EMPTY, (0.0, 0.0, 0.0), 0.0)}
    m = mg.graded_box(xs, ys, [0.0, 0.05], sp, specs)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.1)
    q = m.patch("inlet")
    p = m.patches[q]
    y = m.Cf[1, m.n_internal_faces + p.start:m.n_internal_faces + p.start + p.size]
    cs.set_patch_faces(q, np.stack([y, 0 * y, 0 * y]))
    u = np.zeros((3, m.n_cells)); u[0] = m.C[1]
    phi = m.Cf[1] * m.Sf[0]
    cs.set_fields(u, np.zeros(m.n_cells), phi)
    for _ in range(3):
        assert cs.piso_step(0.01, 2)["status"] == 0
    u2, p2, phi2 = cs.get_fields()
    assert np.abs(u2[0] - m.C[1]).max() < 1e-12
    assert np.abs(u2[1]).max() < 1e-12
    assert np.abs(p2).max() < 1e-12
    assert np.abs(phi2 - phi).max() < 1e-12
