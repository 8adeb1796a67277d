"""The transient Poiseuille workload (the paper's tp1M case, Sec. 4.1): a
2-D pipe 0.16 m x 0.02 m, nu 3.3e-6, uniform inlet velocity
0.01 sin(pi t) set before every PISO step of 0.1 ms through the
stream-ordered boundary-value call, p = 0 at the outlet.

* 320 x 30 cells, 50 steps, in lockstep with the oracle (within 10x the
  oracle's own spread under 1e-15 input perturbations, floor 1e-9);
* the full 3200 x 300 mesh: the first step against the oracle at 1e-9, and
  100 steps against the exact start-up solution (parallel flow far from
  both ends) with the inlet/outlet flux balance."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O
from parity_util import TOL, rel, oracle_envelope, assert_in_envelope, \
    assert_iters_where_well_conditioned

pytestmark = pytest.mark.gpu

TP = mg.TP1M


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


def tp_step(c, m, n, stats=True):
    """Inlet value at the new time level, then one PISO step (2 correctors)."""
    c.set_patch(m.patch("inlet"), mg.tp_inlet((n + 1) * TP["dt"], TP["u0"], TP["f"]), 0.0)
    if stats:
        return c.piso_step(TP["dt"], 2)
    return c.piso_step(TP["dt"], 2, stats=False)


def test_tp_reduced_in_lockstep_with_oracle(P):
    m = mg.tp_channel(320, 30)
    base, its0, its_p, spread = oracle_envelope(m, TP["nu"], 50, lambda c, n: tp_step(c, m, n))
    case = P.Case(P.Mesh(m, renumber=True), TP["nu"])
    gpu_its = []
    for n in range(50):
        s = tp_step(case, m, n)
        assert s["status"] == 0
        gpu_its.append(s["iters"])
    stable = assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    assert stable[:, 3].all()           # the first corrector's count is never rounding-decided
    assert_in_envelope(case, base, spread)


@pytest.fixture(scope="module")
def full_mesh():
    return mg.tp_channel()


def test_tp_full_size_first_step(P, full_mesh):
    m = full_mesh
    assert m.n_cells == 960000
    case = P.Case(P.Mesh(m, renumber=True), TP["nu"])
    oc = O.Case(O.Mesh(m, renumber=True), TP["nu"])
    s = tp_step(case, m, 0)
    so = tp_step(oc, m, 0)
    assert s["status"] == 0
    assert np.abs(np.array(s["iters"]) - so["iters"]).max() <= 1, (s["iters"], so["iters"])
    for a, b in zip(case.get_fields_host(), oc.get_fields()):
        assert rel(a, b) <= TOL


def test_tp_full_size_startup_profile(P, full_mesh):
    """After 100 steps (t = 10 ms) the flow in the middle of the pipe is the
    exact start-up solution: Stokes layers 0.18 mm (2.7 cells) thick on a
    plug core."""
    from womersley import StartupChannel
    m = full_mesh
    case = P.Case(P.Mesh(m, renumber=True), TP["nu"])
    steps = 100
    for n in range(steps):
        tp_step(case, m, n, stats=False)
    st = case.last_stats()
    assert st["status"] == 0
    u, p, phi = case.get_fields_host()
    T = steps * TP["dt"]
    S = StartupChannel(TP["H"], TP["nu"], TP["u0"], 2 * np.pi * TP["f"])
    nx, h = TP["nx"], TP["L"] / TP["nx"]
    i = np.arange(m.n_cells) % nx
    for a in (nx // 4, nx // 2 - 1, 3 * nx // 4):
        y = m.C[1][i == a]
        ue = S.u(y, T)
        err = rel(u[0][i == a], ue)
        print(f"column {a}: profile rel L2 error {err:.2e}")
        # the oracle on a 400 x 300 stretch of the same pipe: 1.5e-3 to 1.8e-3
        assert err < 3e-3
        assert np.abs(u[1][i == a]).max() < 1e-4 * TP["u0"]
    a, b = nx // 2 - 1, nx // 2
    G = -(p[i == b] - p[i == a]).mean() / h
    assert G == pytest.approx(S.G(T), rel=1e-2)     # oracle stretch: 2e-4
    F = m.n_internal_faces
    inl, out = m.patches[m.patch("inlet")], m.patches[m.patch("outlet")]
    fin = phi[F + inl.start:F + inl.start + inl.size].sum()
    fout = phi[F + out.start:F + out.start + out.size].sum()
    dz = m.V[0] / (h * TP["H"] / TP["ny"])
    assert -fin / dz == pytest.approx(S.Q(T), rel=1e-12)
    assert fout == pytest.approx(-fin, rel=1e-5)


def test_tp1m_all_5000_steps_with_multigrid(P, full_mesh):
    """The paper's whole tp1M run: 5000 PISO steps of 0.1 ms (to t = 0.5 s,
    a quarter period of the inlet), pressure by the multigrid CG with the
    FP32 V-cycle.  At the end the flow in the middle of the pipe is the
    exact start-up solution (Stokes layers 1.3 mm = 19 cells thick by
    then), the pressure gradient matches, and the pipe passes the inlet's
    flow rate."""
    import time
    import torch
    from womersley import StartupChannel
    m = full_mesh
    case = P.Case(P.Mesh(m, renumber=True), TP["nu"], P.FV_PREC_MIXED)
    case.set_pressure_solver(P.FV_PSOLVER_AMG)
    steps = TP["steps"]
    its = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(steps):
        tp_step(case, m, n, stats=False)
        if n % 250 == 249:
            st = case.last_stats()
            assert st["status"] == 0, (n, st)
            its += sum(st["iters"][3:])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    u, p, phi = case.get_fields_host()
    T = steps * TP["dt"]
    S = StartupChannel(TP["H"], TP["nu"], TP["u0"], 2 * np.pi * TP["f"])
    nx, h = TP["nx"], TP["L"] / TP["nx"]
    i = np.arange(m.n_cells) % nx
    errs = []
    for a in (nx // 4, nx // 2 - 1, 3 * nx // 4):
        y = m.C[1][i == a]
        errs.append(rel(u[0][i == a], S.u(y, T)))
    a, b = nx // 2 - 1, nx // 2
    G = -(p[i == b] - p[i == a]).mean() / h
    print(f"tp1M 5000 steps in {wall:.1f} s wall; CG iterations of every 250th step: {its}; "
          f"profile errors {['%.2e' % e for e in errs]}; dp/dx error {abs(G / S.G(T) - 1):.2e}")
    assert max(errs) < 5e-4          # measured 6.7e-5
    assert G == pytest.approx(S.G(T), rel=1e-2)     # measured 2.6e-3
    F = m.n_internal_faces
    inl, out = m.patches[m.patch("inlet")], m.patches[m.patch("outlet")]
    fin = phi[F + inl.start:F + inl.start + inl.size].sum()
    fout = phi[F + out.start:F + out.start + out.size].sum()
    dz = m.V[0] / (h * TP["H"] / TP["ny"])
    assert -fin / dz == pytest.approx(S.Q(T), rel=1e-12)
    assert fout == pytest.approx(-fin, rel=1e-5)
