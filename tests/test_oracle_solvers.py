"""Pins of the oracle's linear algebra: the LDU product (the paper's SMVP),
Jacobi-PCG and Jacobi-BiCGStab (Sec. 3) against dense direct solves on tiny
meshes -- the oracle's own Gaussian elimination, cross-checked by
``numpy.linalg.solve``."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def dense_from_ldu(own, nei, diag, upper, lower):
    N = len(diag)
    A = np.diag(diag).astype(float)
    # LDU convention: upper_f = coefficient of the neighbour in the owner's row
    A[own[:len(upper)], nei] += upper
    A[nei, own[:len(upper)]] += lower
    return A


def _stepped_case(mesh_desc, nu, dt, steps, renumber=True):
    om = O.Mesh(mesh_desc, renumber=renumber)
    cs = O.Case(om, nu)
    for _ in range(steps):
        st = cs.piso_step(dt, 2, p_ref_cell=mesh_desc.corner_cell)
        assert st["status"] == 0
    return om, cs


@pytest.mark.parametrize("maker", [lambda: mg.cavity2d(4), lambda: mg.cavity3d(4),
                                   lambda: mg.tet_box(2, 2, 2, jitter=0.1)])
def test_matvec_matches_dense(maker):
    m = maker()
    om = O.Mesh(m, renumber=True)
    own, nei = om.addressing()
    rng = np.random.default_rng(3)
    F = m.n_internal_faces
    d, u, l, x = rng.random(m.n_cells) + 4, rng.standard_normal(F), rng.standard_normal(F), \
        rng.standard_normal(m.n_cells)
    A = dense_from_ldu(own, nei, d, u, l)
    assert np.allclose(O.ldu_matvec(own, nei, d, u, l, x), A @ x, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("which", ["2d", "3d", "tet"])
def test_pcg_matches_dense_on_pressure_systems(which):
    if which == "2d":
        m = mg.cavity2d(4); nu, dt = 0.1, 0.005
    elif which == "3d":
        m = mg.cavity3d(4); nu, dt = 0.01, 0.02
    else:
        m = mg.tet_box(2, 2, 2, jitter=0.1); nu, dt = 0.05, 0.02
        m.patches[0].u = (0.3, 0.0, 0.1)
    om, cs = _stepped_case(m, nu, dt, 3)
    d, up, b = cs.pressure_system(dt, p_ref_cell=m.corner_cell)
    own, nei = om.addressing()
    A = dense_from_ldu(own, nei, d, up, up)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0
    x_ge = O.dense_solve(A, b)
    x_np = np.linalg.solve(A, b)
    assert np.allclose(x_ge, x_np, rtol=1e-11, atol=1e-13 * np.abs(x_np).max())
    x, it, r0, r1, st = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-14, maxit=1000)
    assert st == 0
    assert r1 <= 1e-14
    assert np.linalg.norm(x - x_np) <= 1e-11 * np.linalg.norm(x_np)
    # in exact arithmetic CG terminates in at most N steps
    assert it <= m.n_cells + 5
    # reported residual is the true one (up to rounding)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-13


def test_pcg_stopping_rule_and_warm_start():
    m = mg.cavity3d(4)
    om, cs = _stepped_case(m, 0.01, 0.02, 2)
    d, up, b = cs.pressure_system(0.02, p_ref_cell=m.corner_cell)
    own, nei = om.addressing()
    A = dense_from_ldu(own, nei, d, up, up)
    xs = np.linalg.solve(A, b)
    for tol in (1e-3, 1e-6, 1e-9):
        x, it, r0, r1, st = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=tol)
        assert st == 0 and r1 <= tol
        # one iteration fewer would not have met the tolerance
        x2, it2, _, r2, st2 = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=tol,
                                    maxit=it - 1)
        assert st2 == -1 and r2 > tol
    # exact start: zero iterations
    x, it, r0, r1, st = O.pcg(own, nei, d, up, b, xs, tol=1e-8)
    assert it == 0 and st == 0
    # zero right-hand side: x = 0, no iterations
    x, it, r0, r1, st = O.pcg(own, nei, d, up, 0 * b, xs, tol=1e-8)
    assert it == 0 and not x.any()
    # relative-to-initial tolerance
    x, it, r0, r1, st = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=0.0, reltol=1e-2)
    assert r1 <= 1e-2 * r0


@pytest.mark.parametrize("which", ["2d", "3d", "tet"])
def test_bicgstab_matches_dense_on_momentum_systems(which):
    if which == "2d":
        m = mg.cavity2d(4); nu, dt = 0.02, 0.05
    elif which == "3d":
        m = mg.cavity3d(4); nu, dt = 0.01, 0.05
    else:
        m = mg.tet_box(2, 2, 2, jitter=0.1); nu, dt = 0.02, 0.05
        m.patches[0].u = (1.0, 0.0, 0.5)
        m.corner_cell = 0
    om, cs = _stepped_case(m, nu, dt, 3)
    d, up, lo, src = cs.momentum_system(True, dt)
    own, nei = om.addressing()
    A = dense_from_ldu(own, nei, d, up, lo)
    assert not np.allclose(up, lo)         # convection makes M non-symmetric
    b = src[0]
    xs = np.linalg.solve(A, b)
    assert np.allclose(O.dense_solve(A, b), xs, rtol=1e-11, atol=1e-14)
    x, it, r0, r1, st = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=1e-14,
                                   maxit=500)
    assert st == 0 and r1 <= 1e-14
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
    # zero rhs and zero start: returns at once (keeps u_z = 0 in 2-D)
    x, it, *_ = O.bicgstab(own, nei, d, up, lo, 0 * b, np.zeros(m.n_cells))
    assert it == 0 and not x.any()


def test_bicgstab_stopping_rule_and_warm_start():
    """The rules both BiCGStab implementations share: stop once the updated
    residual meets max(tol ||b||, reltol ||r0||) (it equals the true residual
    b - A x to rounding), status -1 when the iteration limit comes first,
    no iteration from an exact start, x = 0 for a zero right-hand side."""
    m = mg.cavity3d(5)
    om, cs = _stepped_case(m, 0.01, 0.05, 3)
    d, up, lo, src = cs.momentum_system(True, 0.05)
    own, nei = om.addressing()
    A = dense_from_ldu(own, nei, d, up, lo)
    b = src[0]
    nb = np.linalg.norm(b)
    xs = np.linalg.solve(A, b)
    for tol in (1e-3, 1e-6, 1e-9):
        x, it, r0, r1, st = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=tol)
        assert st == 0 and r1 <= tol and it >= 1
        assert abs(np.linalg.norm(b - A @ x) / nb - r1) <= 1e-6 * r1 + 1e-15
        # one iteration fewer would not have met the tolerance
        x2, it2, _, r2, st2 = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=tol,
                                         maxit=it - 1)
        assert st2 == -1 and r2 > tol and it2 == it - 1
    # exact start: zero iterations
    x, it, r0, r1, st = O.bicgstab(own, nei, d, up, lo, b, xs, tol=1e-8)
    assert it == 0 and st == 0
    # zero right-hand side: x = 0, no iterations, whatever the start
    x, it, r0, r1, st = O.bicgstab(own, nei, d, up, lo, 0 * b, xs, tol=1e-8)
    assert it == 0 and st == 0 and not x.any()
    # relative-to-initial tolerance
    x, it, r0, r1, st = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=0.0,
                                   reltol=1e-2)
    assert st == 0 and r1 <= 1e-2 * r0


def test_dense_solve_pivoting():
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([3.0, 2.0, 4.0])
    assert np.allclose(O.dense_solve(A, b), [1.0, 1.0, 1.0], rtol=1e-15)


def test_piso_replay_with_own_iteration_counts_is_bit_identical():
    """The pressure-solve schedule (used to replay another run's stopping
    decisions) changes no arithmetic: replaying a run with its own counts
    gives the same bits, and a count one lower gives a different state."""
    import meshgen as mg
    m = mg.cavity2d(16)
    a = O.Case(O.Mesh(m, renumber=True), 0.05)
    b = O.Case(O.Mesh(m, renumber=True), 0.05)
    c = O.Case(O.Mesh(m, renumber=True), 0.05)
    for _ in range(5):
        sa = a.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
        sb = b.piso_step(0.005, 2, p_ref_cell=m.corner_cell, p_iters=sa["iters"][3:])
        assert np.array_equal(sa["iters"], sb["iters"])
        c.piso_step(0.005, 2, p_ref_cell=m.corner_cell, p_iters=np.maximum(sa["iters"][3:] - 1, 0))
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.get_fields()[1], c.get_fields()[1])
