"""Mixed-precision pressure solve (FP32 inner Jacobi-CG inside FP64 defect
correction) against the FP64 oracle, with the inner iterations in both
orders: Chronopoulos-Gear (two synchronisations per iteration, the
default) and textbook (FVGB_MIXED_CG=classic, read when a mesh is
created).

The gate is the true FP64 residual: ||b - A x|| <= tol ||b||, evaluated here
with the oracle's own LDU product.  The error of every field against the
FP64 oracle is reported and bounded."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O

pytestmark = pytest.mark.gpu


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


@pytest.fixture(autouse=True, params=["cgcg", "classic"])
def form(request, monkeypatch):
    monkeypatch.setenv("FVGB_MIXED_CG", request.param)
    return request.param


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def t64(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _system(m, nu, dt, steps, ref):
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, nu)
    for _ in range(steps):
        oc.piso_step(dt, 2, p_ref_cell=ref)
    d, up, b = oc.pressure_system(dt, p_ref_cell=ref)
    return om, d, up, b


@pytest.mark.parametrize("which", ["2d", "3d", "tet"])
@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_mixed_solve_meets_fp64_residual(P, which, tol):
    if which == "2d":
        m, nu, dt = mg.cavity2d(32), 0.01, 0.005
    elif which == "3d":
        m, nu, dt = mg.permute_cells(mg.cavity3d(24), mg.random_permutation(24 ** 3, 3)), 0.01, 0.01
    else:
        m, nu, dt = mg.tet_box(5, 5, 5, jitter=0.1), 0.05, 0.02
        m.patches[0].u = (0.5, 0.0, 0.2)
    om, d, up, b = _system(m, nu, dt, 2, m.corner_cell)
    own, nei = om.addressing()
    xs = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-13)[0]
    mesh = P.Mesh(m, renumber=True)
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve_mixed(t64(d), t64(up), t64(b), x, tol=tol)
    xg = x.cpu().numpy()
    assert s["status"] == 0 and s["outer"] >= 1
    # the true residual, computed by the oracle's product, meets the tolerance
    r = b - O.ldu_matvec(own, nei, d, up, up, xg)
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * (1 + 1e-9)
    assert s["res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-6)
    # and the solution is as close to the exact one as the FP64 CG's
    x64 = t64(np.zeros(m.n_cells))
    mesh.pcg_solve(t64(d), t64(up), t64(b), x64, tol=tol)
    e_mixed, e_fp64 = rel(xg, xs), rel(x64.cpu().numpy(), xs)
    assert e_mixed <= max(10 * e_fp64, 1e3 * tol), (e_mixed, e_fp64)


def test_mixed_iteration_budget(P):
    m = mg.cavity3d(16)
    om, d, up, b = _system(m, 0.01, 0.01, 1, 0)
    mesh = P.Mesh(m, renumber=True)
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve_mixed(t64(d), t64(up), t64(b), x, tol=1e-12, maxit=7)
    assert s["status"] == 4 and s["iters"] == 7
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve_mixed(t64(d), t64(up), t64(0 * b), x)
    assert s["status"] == 0 and s["iters"] == 0 and not x.cpu().numpy().any()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_mixed_piso_against_fp64_oracle(P, which):
    """PISO steps with the mixed-precision pressure solve; every solve meets
    the FP64 tolerance and the fields stay close to the FP64 oracle (errors
    of the order of the 1e-6 solver tolerance)."""
    if which == "2d":
        m, nu, dt, steps = mg.cavity2d(32), 0.01, 0.005, 20
    else:
        n = 16
        m, nu, dt, steps = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1)), 0.01, 0.01, 10
    import paper_1207_1571_gb300 as PP
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, nu, PP.FV_PREC_MIXED)
    oc = O.Case(O.Mesh(m, renumber=True), nu)
    for _ in range(steps):
        s = case.piso_step(dt, 2, p_ref_cell=m.corner_cell)
        oc.piso_step(dt, 2, p_ref_cell=m.corner_cell)
        assert s["status"] == 0
        assert all(sp["res"] <= 1e-6 for sp in s["p"])
    u, p, phi = case.get_fields_host()
    uo, po, phio = oc.get_fields()
    eu, ep, ephi = rel(u, uo), rel(p, po), rel(phi, phio)
    print(f"mixed vs FP64 oracle after {steps} steps: u {eu:.2e} p {ep:.2e} phi {ephi:.2e}")
    assert eu < 1e-4 and ep < 1e-3 and ephi < 1e-4
    # mass conservation holds to the FP64 tolerance (flux correction in FP64)
    F = m.n_internal_faces
    div = np.zeros(m.n_cells)
    np.add.at(div, m.owner, phi)
    np.add.at(div, m.neighbour, -phi[:F])
    assert np.abs(div).max() < 1e-4 * np.abs(phi).max()
