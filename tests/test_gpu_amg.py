"""The aggregation-multigrid preconditioned CG on the GPU against the
oracle's (same hierarchy, same V-cycle): stand-alone solves, PISO steps
and SIMPLE iterations with the multigrid pressure solver, graph replay, the
degenerate cases, and the full-size cavity and tp1M first steps."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O

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


def assert_close_modulo_mode(x, xo, pinned, tol=TOL):
    """Parity of a pressure-like vector.  On a closed domain pinned at one
    reference cell the constant vector is a near-null mode (eigenvalue of
    order 1/N); the multigrid cycle resolves it, and amplifies rounding in
    it: the oracle perturbed by 1e-15 moves the mean of x by ~1e-8 of |x| on
    the 40^3 cavity while the mean-free part moves by 4e-11.  So the
    mean-free part is held to `tol`, the mean to 1e-6 of |x|."""
    x, xo = np.asarray(x, float), np.asarray(xo, float)
    if not pinned:
        assert rel(x, xo) <= tol
        return
    assert rel(x - x.mean(), xo - xo.mean()) <= tol
    assert abs(x.mean() - xo.mean()) * np.sqrt(len(x)) <= 1e-6 * np.linalg.norm(xo)


def system(which):
    if which == "2d":
        m, nu, dt, ref = mg.cavity2d(40), 0.01, 0.005, True
    elif which == "3d":
        m, nu, dt, ref = mg.permute_cells(mg.cavity3d(16), mg.random_permutation(4096, 7)), 0.01, 0.01, True
    elif which == "3d_big":
        m, nu, dt, ref = mg.cavity3d(40), 0.01, 0.005, True          # several grid levels
    elif which == "tets":
        m, nu, dt, ref = mg.tet_box(6, 6, 6, jitter=0.1), 0.05, 0.02, True
        m.patches[0].u = (0.5, 0.0, 0.2)
    else:
        m, nu, dt, ref = mg.tp_channel(640, 60), 3.3e-6, 1e-4, False
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, nu)
    r = m.corner_cell if ref else -1
    for k in range(2):
        if which == "tp":
            oc.set_patch(m.patch("inlet"), mg.tp_inlet((k + 1) * dt), 0.0)
        oc.piso_step(dt, 2, p_ref_cell=r)
    if which == "tp":
        oc.set_patch(m.patch("inlet"), mg.tp_inlet(3 * dt), 0.0)
    d, up, b = oc.pressure_system(dt, p_ref_cell=r)
    return m, om, d, up, b


@pytest.mark.parametrize("which", ["2d", "3d", "3d_big", "tets", "tp"])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_amg_pcg_matches_oracle(P, which, tol):
    m, om, d, up, b = system(which)
    amg = O.Amg(om)
    mesh = P.Mesh(m, renumber=True)
    assert mesh.amg_levels() == list(amg.levels()[0])
    x0 = np.random.default_rng(1).standard_normal(m.n_cells) * 1e-3
    xo, ito, r0o, r1o, sto = amg.pcg(d, up, b, x0, tol=tol)
    x = t64(x0)
    s = mesh.pcg_solve_amg(t64(d), t64(up), t64(b), x, tol=tol)
    assert s["status"] == 0 and sto == 0
    assert abs(s["iters"] - ito) <= 1, (s["iters"], ito)
    assert_close_modulo_mode(x.cpu().numpy(), xo, which != "tp")
    assert s["res"] <= tol and abs(s["res0"] - r0o) <= 1e-12 * r0o
    # and far fewer iterations than Jacobi-CG
    own, nei = om.addressing()
    itj = O.pcg(own, nei, d, up, b, x0, tol=tol)[1]
    assert s["iters"] < 0.25 * itj, (s["iters"], itj)


def test_amg_pcg_degenerate_cases(P):
    m, om, d, up, b = system("3d")
    mesh = P.Mesh(m, renumber=True)
    x = t64(np.ones(m.n_cells))
    s = mesh.pcg_solve_amg(t64(d), t64(up), t64(0 * b), x)
    assert s["iters"] == 0 and s["status"] == 0 and not x.cpu().numpy().any()
    amg = O.Amg(om)
    xs = amg.pcg(d, up, b, np.zeros(m.n_cells), tol=1e-14)[0]
    x = t64(xs)
    s = mesh.pcg_solve_amg(t64(d), t64(up), t64(b), x, tol=1e-8)
    assert s["iters"] == 0
    x = t64(np.zeros(m.n_cells))
    s = mesh.pcg_solve_amg(t64(d), t64(up), t64(b), x, tol=1e-14, maxit=3)
    xo, ito, _, _, sto = amg.pcg(d, up, b, np.zeros(m.n_cells), tol=1e-14, maxit=3)
    assert s["status"] == 4 and sto == -1 and s["iters"] == ito == 3
    assert_close_modulo_mode(x.cpu().numpy(), xo, True)


def test_amg_single_level_mesh(P):
    """25 cells: the hierarchy is the coarsest level alone (a direct solve,
    one CG iteration)."""
    m = mg.cavity2d(5)
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.1)
    for _ in range(3):
        oc.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
    d, up, b = oc.pressure_system(0.005, p_ref_cell=m.corner_cell)
    mesh = P.Mesh(m, renumber=True)
    assert mesh.amg_levels() == [25]
    x = t64(np.zeros(25))
    s = mesh.pcg_solve_amg(t64(d), t64(up), t64(b), x, tol=1e-12)
    assert s["status"] == 0 and s["iters"] == 1
    xo = O.Amg(om).pcg(d, up, b, np.zeros(25), tol=1e-12)[0]
    assert rel(x.cpu().numpy(), xo) <= TOL


def split_p(p, pinned):
    """(mean-free part, mean) of a pressure field on a pinned closed domain;
    (p, 0) otherwise."""
    p = np.asarray(p, float)
    return (p - p.mean(), p.mean()) if pinned else (p, 0.0)


def oracle_runs(m, nu, steps, step, pinned, eps=1e-15, seeds=(1, 2)):
    """The oracle with the multigrid pressure solver from rest, and from rest
    plus eps-sized velocity perturbations: the unperturbed fields and counts,
    the perturbed counts, and the largest spread of u, phi, the mean-free
    pressure and the pressure mean (the oracle's own rounding sensitivity)."""
    def run(e, seed):
        oc = O.Case(O.Mesh(m, renumber=True), nu)
        oc.set_pressure_solver(1)
        if e > 0:
            u = np.zeros((3, m.n_cells))
            u[:2] = e * np.random.default_rng(seed).standard_normal((2, m.n_cells))
            oc.set_fields(u, np.zeros(m.n_cells), np.zeros(m.n_faces))
        its = np.array([np.array(step(oc, k)["iters"]) for k in range(steps)])
        return oc.get_fields(), its
    f0, its0 = run(0.0, 0)
    spread = dict(u=0.0, phi=0.0, p=0.0, mean=0.0)
    its_p = []
    for sd in seeds:
        f, its = run(eps, sd)
        its_p.append(its)
        spread["u"] = max(spread["u"], rel(f[0], f0[0]))
        spread["phi"] = max(spread["phi"], rel(f[2], f0[2]))
        (a, ma), (b, mb) = split_p(f[1], pinned), split_p(f0[1], pinned)
        spread["p"] = max(spread["p"], rel(a, b))
        spread["mean"] = max(spread["mean"], abs(ma - mb))
    return f0, its0, its_p, spread


def lockstep(P, m, nu, steps, step_gpu, step_orc, pinned=True):
    """GPU multigrid-CG steps against the oracle's: fields within
    max(1e-9, 10x the oracle's own spread under 1e-15 perturbations) (the
    pressure of a pinned domain split into its mean-free part and its mean),
    iteration counts within 1 wherever the perturbed oracle runs agree."""
    from parity_util import assert_iters_where_well_conditioned
    f0, its0, its_p, spread = oracle_runs(m, nu, steps, step_orc, pinned)
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, nu)
    case.set_pressure_solver(P.FV_PSOLVER_AMG)
    gpu_its = []
    for k in range(steps):
        s = step_gpu(case, k)
        assert s["status"] == 0
        gpu_its.append(s["iters"])
    assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    u, p, phi = case.get_fields_host()
    assert rel(u, f0[0]) <= max(TOL, 10 * spread["u"]), (rel(u, f0[0]), spread)
    assert rel(phi, f0[2]) <= max(TOL, 10 * spread["phi"]), (rel(phi, f0[2]), spread)
    (a, ma), (b, mb) = split_p(p, pinned), split_p(f0[1], pinned)
    assert rel(a, b) <= max(TOL, 10 * spread["p"]), (rel(a, b), spread)
    assert abs(ma - mb) <= max(1e-6 * np.linalg.norm(b) / np.sqrt(len(b)), 10 * spread["mean"])
    return case


@pytest.mark.parametrize("which", ["2d", "3d", "tets_nonorth"])
def test_piso_with_amg_matches_oracle(P, which):
    if which == "2d":
        m, nu, dt, nn = mg.cavity2d(20), 0.1, 0.005, 0
    elif which == "3d":
        m, nu, dt, nn = mg.permute_cells(mg.cavity3d(14), mg.random_permutation(14 ** 3, 2)), 0.01, 0.01, 0
    else:
        m, nu, dt, nn = mg.tet_box(5, 5, 5, jitter=0.15, seed=3), 0.05, 0.02, 1
        m.patches[0].u = (1.0, 0.0, 0.3)
    ref = m.corner_cell
    step = lambda c, k: c.piso_step(dt, 2, p_ref_cell=ref, n_nonorth=nn)
    lockstep(P, m, nu, 20 if which == "2d" else 8, step, step)


def test_piso_with_amg_graph_replay(P):
    m = mg.permute_cells(mg.cavity3d(12), mg.random_permutation(1728, 5))
    mesh = P.Mesh(m, renumber=True)
    a, b = P.Case(mesh, 0.01), P.Case(mesh, 0.01)
    for c in (a, b):
        c.set_pressure_solver(P.FV_PSOLVER_AMG)
    for _ in range(6):
        a.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    b.run_graph(6, 0.01, 2, p_ref_cell=m.corner_cell)
    for x, y in zip(a.get_fields_host(), b.get_fields_host()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_amg_shared_memory_levels_identical(P, monkeypatch, precision):
    """Block 0 runs the levels of up to 256 rows from a shared-memory copy
    (FVGB_AMG_SHADOW=0 keeps them in global memory); the arithmetic and its
    order are the same, so the results are the same bits, for the FP64 and
    the FP32 cycle."""
    m = mg.permute_cells(mg.cavity3d(40), mg.random_permutation(40 ** 3, 3))
    prec = P.FV_PREC_FP64 if precision == "fp64" else P.FV_PREC_MIXED
    out = []
    for env in ("1", "0"):
        monkeypatch.setenv("FVGB_AMG_SHADOW", env)
        mesh = P.Mesh(m, renumber=True)
        case = P.Case(mesh, 0.01, prec)
        case.set_pressure_solver(P.FV_PSOLVER_AMG)
        its = []
        for _ in range(3):
            s = case.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
            assert s["status"] == 0
            its.append([int(k) for k in s["iters"]])
        out.append((case.get_fields_host(), its))
    (fa, ia), (fb, ib) = out
    assert ia == ib
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


def test_tp_reduced_with_amg(P):
    m = mg.tp_channel(320, 30)
    dt = 1e-4

    def step(c, k):
        c.set_patch(m.patch("inlet"), mg.tp_inlet((k + 1) * dt), 0.0)
        return c.piso_step(dt, 2)
    lockstep(P, m, 3.3e-6, 20, step, step, pinned=False)


def test_simple_with_amg(P):
    m = mg.duct_tets(4, 8)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    prof = mg.duct_inlet_profile(m.Cf[:2, F + inl.start:F + inl.start + inl.size])
    u_in = np.stack([0 * prof, 0 * prof, prof])

    def step(c, k):
        if k == 0:
            c.set_patch_faces(m.patch("inlet"), u_in)
        return c.simple_iter(0.7, 0.3, n_nonorth=1)
    lockstep(P, m, 0.05, 15, step, step, pinned=False)


def test_amg_pressure_solver_rules(P):
    m = mg.cavity2d(8)
    mesh = P.Mesh(m)
    P.Case(mesh, 0.1, P.FV_PREC_MIXED).set_pressure_solver(P.FV_PSOLVER_AMG)
    with pytest.raises(P.FvError):
        P.Case(mesh, 0.1).set_pressure_solver(7)


@pytest.mark.parametrize("which", ["3d", "3d_big", "tp"])
def test_amg_mixed_solve_meets_fp64_residual(P, which):
    """The V-cycle in FP32: the final FP64 residual (the oracle's product)
    meets the tolerance, the solution is as close to the FP64 multigrid
    solution as the tolerance allows, in about as many iterations."""
    m, om, d, up, b = system(which)
    own, nei = om.addressing()
    amg = O.Amg(om)
    mesh = P.Mesh(m, renumber=True)
    for tol in (1e-6, 1e-10):
        xo, ito, _, _, _ = amg.pcg(d, up, b, np.zeros(m.n_cells), tol=tol)
        x = t64(np.zeros(m.n_cells))
        s = mesh.pcg_solve_amg_mixed(t64(d), t64(up), t64(b), x, tol=tol)
        xg = x.cpu().numpy()
        assert s["status"] == 0
        r = b - O.ldu_matvec(own, nei, d, up, up, xg)
        assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * (1 + 1e-6)
        assert s["iters"] <= ito + max(2, ito // 4), (s["iters"], ito)
        pinned = which != "tp"
        a_, b_ = (xg - xg.mean(), xo - xo.mean()) if pinned else (xg, xo)
        assert rel(a_, b_) <= 1e3 * tol, rel(a_, b_)


@pytest.mark.parametrize("which", ["3d", "tp"])
def test_piso_with_mixed_amg_against_fp64_oracle(P, which):
    """PISO steps of a mixed-precision case with the multigrid pressure
    solver (FP32 V-cycle) against the FP64 oracle with the FP64 multigrid
    solver: every pressure solve meets the FP64 tolerance; fields agree to
    about the solver tolerance."""
    if which == "3d":
        m, nu, dt, steps = mg.permute_cells(mg.cavity3d(14), mg.random_permutation(14 ** 3, 2)), 0.01, 0.01, 8
        ref = m.corner_cell
    else:
        m, nu, dt, steps = mg.tp_channel(320, 30), 3.3e-6, 1e-4, 10
        ref = -1
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, nu, P.FV_PREC_MIXED)
    case.set_pressure_solver(P.FV_PSOLVER_AMG)
    oc = O.Case(O.Mesh(m, renumber=True), nu)
    oc.set_pressure_solver(1)
    for k in range(steps):
        for c in (case, oc):
            if which == "tp":
                c.set_patch(m.patch("inlet"), mg.tp_inlet((k + 1) * dt), 0.0)
        s = case.piso_step(dt, 2, p_ref_cell=ref)
        oc.piso_step(dt, 2, p_ref_cell=ref)
        assert s["status"] == 0 and all(x["res"] <= 1e-6 for x in s["p"]), s["p"]
    (u, p, phi), (uo, po, phio) = case.get_fields_host(), oc.get_fields()
    if ref >= 0:
        p, po = p - p.mean(), po - po.mean()
    eu, ep, ef = rel(u, uo), rel(p, po), rel(phi, phio)
    print(f"mixed multigrid vs FP64 oracle after {steps} steps: u {eu:.2e} p {ep:.2e} phi {ef:.2e}")
    assert eu < 1e-4 and ep < 1e-3 and ef < 1e-4


def test_full_size_cavity_first_step_with_amg(P):
    m = mg.permute_cells(mg.cavity3d(100), mg.random_permutation(10 ** 6, 1234))
    step = lambda c, k: c.piso_step(0.002, 2, p_ref_cell=m.corner_cell)
    lockstep(P, m, 0.01, 1, step, step)


def test_full_size_tp1m_first_steps_with_amg(P):
    m = mg.tp_channel()
    dt = 1e-4

    def step(c, k):
        c.set_patch(m.patch("inlet"), mg.tp_inlet((k + 1) * dt), 0.0)
        return c.piso_step(dt, 2)
    lockstep(P, m, 3.3e-6, 2, step, step, pinned=False)
