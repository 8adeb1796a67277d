"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Bar: mesh addressing bit-exact; FP64 fields within 1e-9 relative L2; Krylov
iteration counts within +-1 (the tolerance of the FP64 path); plus the
degenerate cases (one cell, zero right-hand side, iteration limit, barrier
time-out) and determinism."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O
from parity_util import oracle_envelope, assert_in_envelope, assert_iters_where_well_conditioned

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1571_gb300 import build as B
    B.build()
    import paper_1207_1571_gb300 as P
    P.load()
    return P


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def t64(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def both(P, m, nu, renumber=True, precision=0):
    mesh = P.Mesh(m, renumber=renumber)
    case = P.Case(mesh, nu, precision)
    om = O.Mesh(m, renumber=renumber)
    oc = O.Case(om, nu)
    return mesh, case, om, oc


def assert_fields(case, oc, tol=TOL):
    u, p, phi = case.get_fields_host()
    uo, po, phio = oc.get_fields()
    assert rel(u, uo) <= tol, ("u", rel(u, uo))
    assert rel(p, po) <= tol, ("p", rel(p, po))
    assert rel(phi, phio) <= tol, ("phi", rel(phi, phio))


def assert_iters(s, so):
    gi, oi = np.array(s["iters"]), np.array(so["iters"])
    assert np.abs(gi - oi).max() <= 1, (gi, oi)


# ------------------------------------------------------------ addressing --

@pytest.mark.parametrize("maker", [
    lambda: mg.permute_cells(mg.cavity3d(10), mg.random_permutation(1000, 1234)),
    lambda: mg.tet_box(3, 3, 5, jitter=0.1),
    lambda: mg.mixed_box(4, 5, 3, jitter=0.15),
    lambda: mg.cavity2d(20)])
def test_mesh_addressing_bit_exact(P, maker):
    m = maker()
    mesh = P.Mesh(m, renumber=True)
    om = O.Mesh(m, renumber=True)
    c, f, fl = om.orders()
    assert np.array_equal(mesh.cell_order(), c)
    gf, gfl = mesh.face_order()
    assert np.array_equal(gf, f) and np.array_equal(gfl, fl)
    own, nei = mesh.addressing()
    oown, onei = om.addressing()
    assert np.array_equal(own.cpu().numpy(), oown) and np.array_equal(nei.cpu().numpy(), onei)
    assert mesh.info()["nonorth"] == om.nonorth


def test_gauss_grad_and_matvec(P):
    m = mg.tet_box(4, 3, 5, jitter=0.1)
    mesh = P.Mesh(m, renumber=True)
    om = O.Mesh(m, renumber=True)
    rng = np.random.default_rng(0)
    x, xb = rng.standard_normal(m.n_cells), rng.standard_normal(m.n_boundary_faces)
    g = mesh.gauss_grad(t64(x), t64(xb)).cpu().numpy()
    assert rel(g, om.gauss_grad(x, xb)) <= 1e-13
    own, nei = om.addressing()
    F = m.n_internal_faces
    d, up, lo = rng.random(m.n_cells) + 5, rng.standard_normal(F), rng.standard_normal(F)
    y = mesh.ldu_matvec(t64(d), t64(up), t64(lo), t64(x)).cpu().numpy()
    assert rel(y, O.ldu_matvec(own, nei, d, up, lo, x)) <= 1e-14


# --------------------------------------------------------------- solvers --

def _pressure_system(m, nu, dt, steps, ref):
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, nu)
    for _ in range(steps):
        oc.piso_step(dt, 2, p_ref_cell=ref)
    return om, oc, oc.pressure_system(dt, p_ref_cell=ref)


@pytest.mark.parametrize("which", ["2d", "3d", "tet", "3d_big"])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_pcg_matches_oracle(P, which, tol):
    if which == "2d":
        m, nu, dt = mg.cavity2d(20), 0.1, 0.005
    elif which == "3d":
        m, nu, dt = mg.permute_cells(mg.cavity3d(12), mg.random_permutation(1728, 7)), 0.01, 0.01
    elif which == "3d_big":
        m, nu, dt = mg.cavity3d(24), 0.01, 0.01          # several blocks, grid barrier
    else:
        m, nu, dt = mg.tet_box(4, 4, 4, jitter=0.1), 0.05, 0.02
        m.patches[0].u = (0.5, 0.0, 0.2)
    om, oc, (d, up, b) = _pressure_system(m, nu, dt, 2, m.corner_cell)
    own, nei = om.addressing()
    x0 = np.random.default_rng(1).standard_normal(m.n_cells) * 1e-3
    xo, ito, r0o, r1o, sto = O.pcg(own, nei, d, up, b, x0, tol=tol)
    mesh = P.Mesh(m, renumber=True)
    x = t64(x0)
    s = mesh.pcg_solve(t64(d), t64(up), t64(b), x, tol=tol)
    assert s["status"] == 0 and sto == 0
    assert abs(s["iters"] - ito) <= 1, (s["iters"], ito)
    assert rel(x.cpu().numpy(), xo) <= TOL
    assert s["res"] <= tol and abs(s["res0"] - r0o) <= 1e-12 * r0o


def test_pcg_degenerate_cases(P):
    m = mg.cavity3d(6)
    om, oc, (d, up, b) = _pressure_system(m, 0.01, 0.02, 1, 0)
    mesh = P.Mesh(m, renumber=True)
    # zero right-hand side: x = 0 without iterating
    x = t64(np.ones(m.n_cells))
    s = mesh.pcg_solve(t64(d), t64(up), t64(0 * b), x)
    assert s["iters"] == 0 and s["status"] == 0 and not x.cpu().numpy().any()
    # exact start: no iteration
    own, nei = om.addressing()
    xs = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-14)[0]
    x = t64(xs)
    s = mesh.pcg_solve(t64(d), t64(up), t64(b), x, tol=1e-8)
    assert s["iters"] == 0
    # iteration limit reached: status NOT_CONVERGED, same iterate as the oracle
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve(t64(d), t64(up), t64(b), x, tol=1e-12, maxit=5)
    xo, ito, _, _, sto = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-12, maxit=5)
    assert s["status"] == 4 and sto == -1 and s["iters"] == ito == 5
    assert rel(x.cpu().numpy(), xo) <= TOL


@pytest.mark.parametrize("which", ["2d", "tet", "3d_big"])
def test_bicgstab_matches_oracle(P, which):
    if which == "2d":
        m, nu, dt = mg.cavity2d(16), 0.02, 0.05
    elif which == "3d_big":
        m, nu, dt = mg.cavity3d(24), 0.01, 0.01          # several blocks, grid sums
    else:
        m, nu, dt = mg.tet_box(3, 3, 3, jitter=0.1), 0.02, 0.05
        m.patches[0].u = (1.0, 0.0, 0.5)
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, nu)
    for _ in range(3):
        oc.piso_step(dt, 2, p_ref_cell=m.corner_cell)
    d, up, lo, src = oc.momentum_system(True, dt)
    own, nei = om.addressing()
    x0 = np.zeros(m.n_cells)
    for tol in (1e-6, 1e-12):
        xo, ito, r0o, r1o, sto = O.bicgstab(own, nei, d, up, lo, src[0], x0, tol=tol)
        mesh = P.Mesh(m, renumber=True)
        x = t64(x0)
        s = mesh.bicgstab_solve(t64(d), t64(up), t64(lo), t64(src[0]), x, tol=tol)
        assert s["status"] == 0 and abs(s["iters"] - ito) <= 1, (s, ito)
        assert rel(x.cpu().numpy(), xo) <= TOL


def test_bicgstab_degenerate_cases(P):
    """Zero right-hand side, an exact start and the iteration limit, on a
    momentum system large enough for several blocks (grid sums)."""
    m = mg.cavity3d(12)
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.01)
    oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    d, up, lo, src = oc.momentum_system(True, 0.01)
    own, nei = om.addressing()
    mesh = P.Mesh(m, renumber=True)
    b = src[0]
    # zero right-hand side: x = 0 without iterating
    x = t64(np.ones(m.n_cells))
    s = mesh.bicgstab_solve(t64(d), t64(up), t64(lo), t64(0 * b), x)
    assert s["iters"] == 0 and s["status"] == 0 and not x.cpu().numpy().any()
    # exact start: no iteration
    xs = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=1e-15, maxit=200)[0]
    x = t64(xs)
    s = mesh.bicgstab_solve(t64(d), t64(up), t64(lo), t64(b), x, tol=1e-8)
    assert s["iters"] == 0 and s["status"] == 0
    # iteration limit: NOT_CONVERGED after exactly maxit iterations, the
    # oracle's iterate and residual
    x = t64(np.zeros(m.n_cells))
    s = mesh.bicgstab_solve(t64(d), t64(up), t64(lo), t64(b), x, tol=1e-15, maxit=3)
    xo, ito, r0o, r1o, sto = O.bicgstab(own, nei, d, up, lo, b, np.zeros(m.n_cells), tol=1e-15,
                                        maxit=3)
    assert s["status"] == 4 and sto == -1 and s["iters"] == ito == 3
    assert rel(x.cpu().numpy(), xo) <= TOL
    assert abs(s["res"] - r1o) <= 1e-9 * r1o and abs(s["res0"] - r0o) <= 1e-12 * r0o


# -------------------------------------------------------------- PISO step --

def test_piso_2d_cavity_40_steps_strict(P):
    """The 2-D lid-driven cavity workload (20x20, nu 0.1, dt 0.005, 2
    correctors, CG to 1e-6), 40 steps in lockstep with the oracle: iteration
    counts within 1, fields within 1e-9."""
    m = mg.cavity2d(20)
    mesh, case, om, oc = both(P, m, 0.1)
    for step in range(40):
        s = case.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
        so = oc.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
        assert s["status"] == 0
        assert_iters(s, so)
    assert_fields(case, oc)


def test_piso_2d_cavity_100_steps(P):
    """All 100 steps of the 2-D cavity workload.  Past about step 40 the
    tolerance-truncated CG amplifies rounding-sized differences (the oracle
    perturbed by 1e-15 drifts by ~1e-8 by step 80), and from about step 83
    the CG stopping iteration itself is decided by rounding; the GPU must
    stay within 10x the oracle's own spread, with iteration counts within 1
    wherever the perturbed oracle runs agree on them."""
    m = mg.cavity2d(20)
    step = lambda c, n: c.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
    base, its0, its_p, spread = oracle_envelope(m, 0.1, 100, step)
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.1)
    gpu_its = [case.piso_step(0.005, 2, p_ref_cell=m.corner_cell)["iters"] for _ in range(100)]
    stable = assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    assert stable[1:70].all()
    assert_in_envelope(case, base, spread)


def test_piso_2d_cavity_100_steps_fixed_iterations(P):
    """All 100 steps with the pressure CG fixed at 60 iterations per solve
    (tolerance 0) on both sides: no stopping decision at all."""
    m = mg.cavity2d(20)
    step = lambda c, n: c.piso_step(0.005, 2, p_ref_cell=m.corner_cell, p_tol=0.0, p_maxit=60)
    base, its0, its_p, spread = oracle_envelope(m, 0.1, 100, step)
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.1)
    for _ in range(100):
        s = case.piso_step(0.005, 2, p_ref_cell=m.corner_cell, p_tol=0.0, p_maxit=60)
        assert s["p"][0]["status"] == 4 and s["p"][0]["iters"] == 60
    assert_in_envelope(case, base, spread)


def test_piso_3d_cavity_permuted(P):
    n = 14
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    mesh, case, om, oc = both(P, m, 0.01)
    for step in range(8):
        s = case.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
        so = oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
        assert s["status"] == 0
        assert_iters(s, so)
    assert_fields(case, oc)


def _cavity_patches():
    sides = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
    sp = {k: "fixedWalls" for k in sides}
    sp["ymax"] = "movingWall"
    return sp, {"movingWall": (mg.WALL, (1.0, 0.0, 0.0), 0.0),
                "fixedWalls": (mg.WALL, (0.0, 0.0, 0.0), 0.0)}


def test_piso_graded_cavity(P):
    """The 3-D cavity on a graded mesh (cell sizes growing by 1.15 from cell
    to cell along x and z and shrinking by the same factor along y, so the
    face interpolation weights are 0.465 or 0.535 instead of 1/2), cells
    permuted: 8 PISO steps in lockstep with the oracle, whose weight
    convention the graded-mesh pins fix."""
    n = 14
    up, down = mg.geometric_nodes(n, 1.0, 1.15), mg.geometric_nodes(n, 1.0, 1.0 / 1.15)
    m = mg.graded_box(up, down, up, *_cavity_patches())
    m = mg.permute_cells(m, mg.random_permutation(n ** 3, 77))
    mesh, case, om, oc = both(P, m, 0.01)
    g = om.geometry()
    assert np.abs(g["w"] - 0.5).min() > 0.03
    for step in range(8):
        s = case.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
        so = oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
        assert s["status"] == 0
        assert_iters(s, so)
    assert_fields(case, oc)
    # the Gauss gradient of a linear field is exact on this mesh (to rounding)
    cell, face, _ = om.orders()
    C = np.empty_like(m.C); C[:, cell] = m.C
    Cf = np.empty_like(m.Cf); Cf[:, face] = m.Cf
    a = np.array([0.3, -1.7, 2.5])
    gr = mesh.gauss_grad(t64(a @ C), t64(a @ Cf[:, m.n_internal_faces:])).cpu().numpy()
    assert np.abs(gr - a[:, None]).max() < 1e-11


def test_piso_tets_nonorthogonal(P):
    m = mg.tet_box(4, 4, 4, jitter=0.1)
    m.patches[0].u = (1.0, 0.0, 0.0)
    mesh, case, om, oc = both(P, m, 0.05)
    assert mesh.info()["nonorth"]
    for step in range(5):
        s = case.piso_step(0.01, 2, p_ref_cell=0)
        so = oc.piso_step(0.01, 2, p_ref_cell=0)
        assert_iters(s, so)
    assert_fields(case, oc)


@pytest.mark.parametrize("nn", [1, 3])
def test_piso_tets_nonorth_correctors(P, nn):
    """Non-orthogonal correctors (1 + nn pressure solves per corrector, the
    explicit term re-evaluated from the newest pressure) on skewed tets."""
    m = mg.tet_box(5, 5, 5, jitter=0.15, seed=3)
    m.patches[0].u = (1.0, 0.0, 0.3)
    mesh, case, om, oc = both(P, m, 0.05)
    for step in range(4):
        s = case.piso_step(0.02, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        so = oc.piso_step(0.02, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        assert s["status"] == 0 and len(s["p"]) == 2 * (1 + nn)
        assert_iters(s, so)
    assert_fields(case, oc)
    # the same steps replayed from a CUDA graph
    case.set_fields_host(np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_faces))
    case.run_graph(4, 0.02, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
    assert_fields(case, oc)


@pytest.mark.parametrize("nn", [0, 1])
def test_piso_mixed_element_cavity(P, nn):
    """The lid-driven cavity on a jittered mixed mesh of hexahedra, prisms and
    pyramids (non-planar faces, non-orthogonal everywhere), with and without
    a non-orthogonal corrector: 5 PISO steps in lockstep with the oracle."""
    m = mg.mixed_cavity3d(8, jitter=0.12, seed=9)
    mesh, case, om, oc = both(P, m, 0.02)
    assert mesh.info()["nonorth"]
    for step in range(5):
        s = case.piso_step(0.01, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        so = oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        assert s["status"] == 0
        assert_iters(s, so)
    assert_fields(case, oc)


def test_simple_mixed_element_duct(P):
    """SIMPLE on a jittered mixed-element duct with an inlet profile and an
    outlet, one non-orthogonal corrector per iteration."""
    m = mg.mixed_duct(4, 8, jitter=0.1, seed=4)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    xy = m.Cf[:2, F + inl.start:F + inl.start + inl.size]
    prof = mg.duct_inlet_profile(xy)
    mesh, case, om, oc = both(P, m, 0.05)
    for c in (case, oc):
        c.set_patch_faces(m.patch("inlet"), np.stack([0 * prof, 0 * prof, prof]))
    for it in range(10):
        s = case.simple_iter(0.7, 0.3, n_nonorth=1)
        so = oc.simple_iter(0.7, 0.3, n_nonorth=1)
        assert_iters(s, so)
    assert_fields(case, oc)


def test_simple_tets_nonorth_correctors(P):
    m = mg.duct_tets(3, 6)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    xy = m.Cf[:2, F + inl.start:F + inl.start + inl.size]
    prof = mg.duct_inlet_profile(xy)
    mesh, case, om, oc = both(P, m, 0.05)
    for c in (case, oc):
        c.set_patch_faces(m.patch("inlet"), np.stack([0 * prof, 0 * prof, prof]))
    for it in range(10):
        s = case.simple_iter(0.7, 0.3, n_nonorth=2)
        so = oc.simple_iter(0.7, 0.3, n_nonorth=2)
        assert len(s["p"]) == 3
        assert_iters(s, so)
        assert s["init_res_max"] == pytest.approx(so["init_res_max"], rel=1e-6)
    assert_fields(case, oc)


def test_nonorth_corrector_limits(P):
    m = mg.cavity2d(4)
    case = P.Case(P.Mesh(m), 0.1)
    with pytest.raises(P.FvError):
        case.piso_step(0.01, 2, p_ref_cell=0, n_nonorth=4)      # 2 x 5 > 8 solves
    with pytest.raises(P.FvError):
        case.piso_step(0.01, 2, p_ref_cell=0, n_nonorth=-1)
    with pytest.raises(P.FvError):
        case.simple_iter(p_ref_cell=0, n_nonorth=8)
    s = case.piso_step(0.01, 4, p_ref_cell=0, n_nonorth=1)
    assert len(s["p"]) == 8


def test_piso_time_dependent_boundary_values(P):
    """Taylor-Green-like walls whose face values change every step."""
    n = 12
    L = np.pi
    sp = {"xmin": "walls", "xmax": "walls", "ymin": "walls", "ymax": "walls",
          "zmin": "fb", "zmax": "fb"}
    specs = {"walls": (mg.WALL, (0, 0, 0), 0.0), "fb": (mg.EMPTY, (0, 0, 0), 0.0)}
    m = mg.permute_cells(mg.hex_box(n, n, 1, (L, L, L / n), sp, specs),
                         mg.random_permutation(n * n, 5))
    mesh, case, om, oc = both(P, m, 0.01)
    F = m.n_internal_faces
    w = m.patches[0]
    Cw = m.Cf[:, F + w.start:F + w.start + w.size]
    u0 = np.stack([np.sin(m.C[0]) * np.cos(m.C[1]), -np.cos(m.C[0]) * np.sin(m.C[1]), 0 * m.C[0]])
    case.set_fields_host(u0, np.zeros(m.n_cells), np.zeros(m.n_faces))
    oc.set_fields(u0, np.zeros(m.n_cells), np.zeros(m.n_faces))
    for k in range(6):
        t = 0.05 * (k + 1)
        f = np.exp(-0.02 * t)
        ub = np.stack([np.sin(Cw[0]) * np.cos(Cw[1]) * f, -np.cos(Cw[0]) * np.sin(Cw[1]) * f,
                       0 * Cw[0]])
        case.set_patch_faces(0, ub)
        oc.set_patch_faces(0, ub)
        s = case.piso_step(0.05, 2, p_ref_cell=0)
        so = oc.piso_step(0.05, 2, p_ref_cell=0)
        assert_iters(s, so)
    assert_fields(case, oc)


def test_piso_single_cell(P):
    m = mg.cavity3d(1)
    mesh, case, om, oc = both(P, m, 0.01)
    for _ in range(3):
        s = case.piso_step(0.01, 2, p_ref_cell=0)
        so = oc.piso_step(0.01, 2, p_ref_cell=0)
        assert_iters(s, so)
    assert_fields(case, oc, tol=1e-12)


def test_piso_iteration_limit_status(P):
    m = mg.cavity2d(12)
    mesh, case, om, oc = both(P, m, 0.1)
    s = case.piso_step(0.005, 2, p_ref_cell=0, p_maxit=4)
    so = oc.piso_step(0.005, 2, p_ref_cell=0, p_maxit=4)
    assert s["status"] == 4 and s["p"][0]["status"] == 4
    assert so["status"] == -1
    assert_iters(s, so)
    assert_fields(case, oc)


def test_graph_replay_and_determinism(P):
    m = mg.permute_cells(mg.cavity3d(10), mg.random_permutation(1000, 2))
    mesh = P.Mesh(m, renumber=True)
    a, b = P.Case(mesh, 0.01), P.Case(mesh, 0.01)
    for _ in range(4):
        a.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    sb = b.run_graph(4, 0.01, 2, p_ref_cell=m.corner_cell)
    ua, pa, fa = a.get_fields_host()
    ub, pb, fb = b.get_fields_host()
    # same kernels, same order, fixed reduction order: identical bits
    assert np.array_equal(ua, ub) and np.array_equal(pa, pb) and np.array_equal(fa, fb)
    assert sb["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_classic"])
def test_cg_resident_and_global_forms_identical(P, monkeypatch, precision):
    """The CG keeps its row-local vectors (FP64: r^, q, y; mixed precision:
    the FP32 r^, q, e, w, v of the textbook order, p, s, e, w of the
    Chronopoulos-Gear order) in shared memory when a block's rows fit (meshes up to
    about 1.2M cells on GB300) and in global memory otherwise.  The FP64 CG
    and the Chronopoulos-Gear order do the same arithmetic in the same order
    in both forms, so a mesh created with FVGB_CG_RESIDENT=0 (global forms
    only) gives the same bits.  The textbook order's global form takes two
    rows per thread in its inner passes (8-byte loads), which groups the FP32
    per-thread sums differently: the same iteration counts and fields within
    the solver tolerance's reach."""
    m = mg.permute_cells(mg.cavity3d(24), mg.random_permutation(24 ** 3, 5))
    prec = P.FV_PREC_FP64 if precision == "fp64" else P.FV_PREC_MIXED
    monkeypatch.setenv("FVGB_MIXED_CG", "classic" if precision == "mixed_classic" else "cgcg")
    out = []
    for env in ("1", "0"):
        monkeypatch.setenv("FVGB_CG_RESIDENT", env)
        mesh = P.Mesh(m, renumber=True)
        case = P.Case(mesh, 0.01, prec)
        its = []
        for _ in range(3):
            s = case.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
            assert s["status"] == 0
            its.append([int(k) for k in s["iters"]])
        out.append((case.get_fields_host(), its))
    (fa, ia), (fb, ib) = out
    if precision == "mixed_classic":
        assert np.abs(np.array(ia) - np.array(ib)).max() <= 2, (ia, ib)
        for x, y, bar in zip(fa, fb, (1e-6, 1e-4, 1e-6)):
            if bar == 1e-4:
                x, y = x - x.mean(), y - y.mean()
            assert rel(x, y) <= bar, rel(x, y)
        return
    assert ia == ib
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


def test_fields_roundtrip(P):
    m = mg.permute_cells(mg.cavity3d(5), mg.random_permutation(125, 9))
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.01)
    rng = np.random.default_rng(3)
    u, p, phi = rng.standard_normal((3, 125)), rng.standard_normal(125), rng.standard_normal(m.n_faces)
    case.set_fields(t64(u), t64(p), t64(phi))
    gu, gp, gphi = case.get_fields()
    assert np.array_equal(gu.cpu().numpy(), u) and np.array_equal(gp.cpu().numpy(), p)
    assert np.array_equal(gphi.cpu().numpy(), phi)
    hu, hp, hphi = case.get_fields_host()
    assert np.array_equal(hu, u) and np.array_equal(hphi, phi)
    # internal order equals the oracle's internal order
    om = O.Mesh(m, renumber=True); oc = O.Case(om, 0.01); oc.set_fields(u, p, phi)
    iu, ip, iphi = case.get_fields(original_order=False)
    ou, op, ophi = oc.state()
    assert np.array_equal(iu.cpu().numpy(), ou) and np.array_equal(iphi.cpu().numpy(), ophi)


@pytest.mark.parametrize("staging", ["0", "1"])
def test_host_field_exchange(P, monkeypatch, staging):
    """Host-buffer set/get, with the kernels reading and writing the caller's
    pageable memory directly (where the device supports it) and through the
    pinned staging buffer (FVGB_HOST_STAGING=1): the values round-trip bit for
    bit in both orders and agree with the device-buffer exchange."""
    monkeypatch.setenv("FVGB_HOST_STAGING", staging)
    m = mg.permute_cells(mg.cavity3d(7), mg.random_permutation(343, 4))
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.01)
    rng = np.random.default_rng(8)
    u, p, phi = rng.standard_normal((3, 343)), rng.standard_normal(343), rng.standard_normal(m.n_faces)
    case.set_fields_host(u, p, phi)
    hu, hp, hphi = case.get_fields_host()
    assert np.array_equal(hu, u) and np.array_equal(hp, p) and np.array_equal(hphi, phi)
    gu, gp, gphi = case.get_fields()
    assert np.array_equal(gu.cpu().numpy(), u) and np.array_equal(gphi.cpu().numpy(), phi)
    iu, ip, iphi = case.get_fields_host(original_order=False)
    du, dp, dphi = case.get_fields(original_order=False)
    assert np.array_equal(iu, du.cpu().numpy()) and np.array_equal(ip, dp.cpu().numpy())
    assert np.array_equal(iphi, dphi.cpu().numpy())
    case.set_fields_host(2.0 * iu, -ip, 0.5 * iphi, original_order=False)
    hu2, hp2, hphi2 = case.get_fields_host()
    assert np.array_equal(hu2, 2.0 * u) and np.array_equal(hp2, -p) and np.array_equal(hphi2, 0.5 * phi)


# ------------------------------------------------------------ SIMPLE step --

def test_simple_channel_outlet(P):
    """30 SIMPLE iterations of a plane channel with an outlet (fixed-pressure
    boundary).  The loose inner solves (0.01 / 0.1 relative) make the run
    sensitive to rounding; compare within the oracle's own envelope."""
    m = mg.channel2d(24, 8, 2.0, 1.0)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    y = m.Cf[1, F + inl.start:F + inl.start + inl.size]
    prof = np.stack([6 * y * (1 - y), 0 * y, 0 * y])

    def step(c, n):
        if n == 0:
            c.set_patch_faces(m.patch("inlet"), prof)
        return c.simple_iter(0.7, 0.3)
    base, its0, its_p, spread = oracle_envelope(m, 0.1, 30, step)
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.1)
    case.set_patch_faces(m.patch("inlet"), prof)
    gpu = [case.simple_iter(0.7, 0.3) for _ in range(30)]
    assert_iters_where_well_conditioned([g["iters"] for g in gpu], its0, its_p)
    assert_in_envelope(case, base, spread)
    assert gpu[-1]["status"] == 0


def test_simple_duct_tets(P):
    m = mg.duct_tets(4, 8)
    mesh, case, om, oc = both(P, m, 0.05)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    xy = m.Cf[:2, F + inl.start:F + inl.start + inl.size]
    prof = mg.duct_inlet_profile(xy)
    ub = np.stack([0 * prof, 0 * prof, prof])
    case.set_patch_faces(m.patch("inlet"), ub)
    oc.set_patch_faces(m.patch("inlet"), ub)
    for it in range(10):
        s = case.simple_iter(0.7, 0.3)
        so = oc.simple_iter(0.7, 0.3)
        assert_iters(s, so)
    assert_fields(case, oc)
    assert s["init_res_max"] == pytest.approx(so["init_res_max"], rel=1e-7)


# --------------------------------------------------------- failure paths --

def test_barrier_timeout_is_reported(P):
    """A device-side wait that runs out returns FV_E_TIMEOUT; the context
    stays usable.  The wait limit is shrunk on the host to force it."""
    from paper_1207_1571_gb300 import _capi
    m = mg.cavity3d(40)
    om, oc, (d, up, b) = _pressure_system(m, 0.01, 0.01, 1, 0)
    mesh = P.Mesh(m, renumber=True)
    L = P.load()
    assert L.fv_set_barrier_spin_limit(1) == 0
    try:
        x = t64(np.zeros(m.n_cells))
        import ctypes as C
        prm = _capi.fv_pcg_params(1e-6, 0.0, 10000, 0)
        st = _capi.fv_solve_stats()
        rc = L.fv_pcg_solve(mesh.h, t64(d).data_ptr(), t64(up).data_ptr(), t64(b).data_ptr(),
                            x.data_ptr(), C.byref(prm), C.byref(st))
        assert rc == 6 and st.status == 6
    finally:
        L.fv_set_barrier_spin_limit(0)
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve(t64(d), t64(up), t64(b), x)
    assert s["status"] == 0


def test_closed_domain_needs_reference(P):
    m = mg.cavity2d(4)
    mesh = P.Mesh(m)
    case = P.Case(mesh, 0.1)
    with pytest.raises(P.FvError) as e:
        case.piso_step(0.01, 2, p_ref_cell=-1)
    assert e.value.status == 1


# --------------------------------------------------- full-size workload --

def test_full_size_cavity_100_cubed_first_step(P):
    """The 1M-cell cavity (100^3, permuted with seed 1234, RCM), one PISO step
    from rest at the launch configuration of the benchmark, against the
    oracle (about half a minute of CPU)."""
    n = 100
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    mesh, case, om, oc = both(P, m, 0.01)
    assert np.array_equal(mesh.cell_order(), om.orders()[0])
    s = case.piso_step(0.002, 2, p_ref_cell=m.corner_cell)
    so = oc.piso_step(0.002, 2, p_ref_cell=m.corner_cell)
    assert s["status"] == 0
    assert_iters(s, so)
    assert_fields(case, oc)
