"""Pins of the oracle's PISO step and SIMPLE iteration (paper Sec. 3) against
closed-form flows and exact identities: mass conservation after every
pressure correction, plane Couette flow (reproduced exactly by central
differencing), plane Poiseuille flow (second-order convergence to the
parabola), Taylor-Green vortex decay with time-dependent boundary values
(Sec. 1/6: time-dependent boundary conditions), transient Poiseuille flow
started by a sinusoidal inlet (exact start-up solution), the rectangular-duct series
solution, and the mirror symmetry of the 3-D lid-driven cavity."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def divergence(m, phi):
    """Net outflow of every cell from face fluxes in the generator's order."""
    F = m.n_internal_faces
    div = np.zeros(m.n_cells)
    np.add.at(div, m.owner, phi)
    np.add.at(div, m.neighbour, -phi[:F])
    return div


def patch_face_centres(m, name):
    p = m.patches[m.patch(name)]
    F = m.n_internal_faces
    return m.Cf[:, F + p.start:F + p.start + p.size]


# ---------------------------------------------------------------------------
# mass conservation
# ---------------------------------------------------------------------------

def test_piso_continuity_identity_2d_cavity():
    m = mg.cavity2d(20)
    om = O.Mesh(m)
    cs = O.Case(om, 0.1)
    for step in range(20):
        st = cs.piso_step(0.005, 2, p_ref_cell=m.corner_cell)
        assert st["status"] == 0
        # flux correction identity: sum_out phi = -(b - A p) in every cell
        assert st["cont_err"] < 1e-12
        u, p, phi = cs.get_fields()
        div = divergence(m, phi)
        # cells are conservative to the pressure-solver tolerance
        assert np.abs(div).max() < 1e-4 * np.abs(phi).max()
        # closed cavity: no net flux through the boundary
        assert abs(phi[m.n_internal_faces:].sum()) < 1e-15
        assert np.abs(u[2]).max() == 0.0   # 2-D: the z velocity stays exactly zero
    # the pressure-solver iteration counts settle as the flow develops
    assert st["iters"][3] < 150


def test_simple_continuity_identity_tets():
    m = mg.duct_tets(3, 6)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.05)
    xy = patch_face_centres(m, "inlet")[:2]
    prof = mg.duct_inlet_profile(xy)
    cs.set_patch_faces(m.patch("inlet"), np.stack([0 * prof, 0 * prof, prof]))
    for _ in range(5):
        st = cs.simple_iter(0.7, 0.3)
        assert st["status"] == 0 and st["cont_err"] < 1e-12


def test_cavity2d_cg_stop_is_rounding_sensitive_late():
    """Property of the 2-D cavity workload (20x20, nu 0.1, dt 0.005, CG to
    1e-6) that bounds any parity claim: its pressure-CG residual is not
    monotone, and from about step 83 on it dips to the threshold and climbs
    again inside a solve.  A 1e-16 perturbation of the initial velocity then
    changes the oracle's own iteration counts by more than one and its final
    pressure by far more than 1e-9, while the first 80 steps are unaffected."""
    m = mg.cavity2d(20)

    def run(eps, seed):
        oc = O.Case(O.Mesh(m, renumber=True), 0.1)
        u = np.zeros((3, m.n_cells))
        u[:2] = eps * np.random.default_rng(seed).standard_normal((2, m.n_cells))
        oc.set_fields(u, np.zeros(m.n_cells), np.zeros(m.n_faces))
        its = [oc.piso_step(0.005, 2, p_ref_cell=m.corner_cell)["iters"][3:].copy()
               for _ in range(100)]
        return np.array(its), oc.get_fields()[1]

    base, p0 = run(0.0, 0)
    pert, p1 = run(1e-16, 0)
    diff = np.abs(base - pert).max(axis=1)
    assert diff[1:80].max() <= 1
    assert diff[80:].max() > 1
    assert np.linalg.norm(p1 - p0) > 1e-6 * np.linalg.norm(p0)


# ---------------------------------------------------------------------------
# plane Couette flow: u = U y/H is reproduced to rounding
# ---------------------------------------------------------------------------

def _couette(nx, ny, U=1.0, H=1.0, Lx=2.0):
    m = mg.channel2d(nx, ny, Lx, H, top_u=(U, 0.0, 0.0))
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.1)
    y = patch_face_centres(m, "inlet")[1]
    cs.set_patch_faces(m.patch("inlet"), np.stack([U * y / H, 0 * y, 0 * y]))
    return m, om, cs


def test_couette_exact_state_is_preserved():
    m, om, cs = _couette(12, 8)
    F = m.n_internal_faces
    u = np.zeros((3, m.n_cells)); u[0] = m.C[1]
    phi = np.zeros(m.n_faces)
    uf = m.Cf[1]                        # exact u_x at the face centres
    phi[:] = uf * m.Sf[0]
    cs.set_fields(u, np.zeros(m.n_cells), phi)
    for _ in range(3):
        st = cs.piso_step(0.01, 2)
        assert st["status"] == 0
    u2, p2, phi2 = cs.get_fields()
    assert np.abs(u2[0] - m.C[1]).max() < 1e-12
    assert np.abs(u2[1]).max() < 1e-12
    assert np.abs(p2).max() < 1e-12
    assert np.abs(phi2 - phi).max() < 1e-12


def test_couette_simple_converges_to_linear_profile():
    m, om, cs = _couette(16, 8)
    for it in range(3000):
        st = cs.simple_iter(0.7, 0.3)
        assert st["status"] == 0
        if st["init_res_max"] < 1e-9:
            break
    assert st["init_res_max"] < 1e-9
    u, p, phi = cs.get_fields()
    assert np.abs(u[0] - m.C[1]).max() < 1e-7
    assert np.abs(p).max() < 1e-7


# ---------------------------------------------------------------------------
# plane Poiseuille flow: second-order convergence to the parabola
# ---------------------------------------------------------------------------

def _poiseuille_error(ny, nu=0.1, Ubar=1.0, H=1.0):
    m = mg.channel2d(2 * ny, ny, 2.0 * H, H)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, nu)
    y = patch_face_centres(m, "inlet")[1]
    prof = 6.0 * Ubar * (y / H) * (1.0 - y / H)
    cs.set_patch_faces(m.patch("inlet"), np.stack([prof, 0 * y, 0 * y]))
    for it in range(5000):
        st = cs.simple_iter(0.7, 0.3)
        assert st["status"] == 0
        if st["init_res_max"] < 1e-9:
            break
    u, p, phi = cs.get_fields()
    yc = m.C[1]
    exact = 6.0 * Ubar * (yc / H) * (1.0 - yc / H)
    last = m.C[0] > 2.0 * H - 2.0 * H / (2 * ny)       # outlet column
    err = np.linalg.norm(u[0][last] - exact[last]) / np.linalg.norm(exact[last])
    # pressure gradient of the fully developed flow: dp/dx = -12 nu Ubar / H^2
    mid = (m.C[0] > 0.5) & (m.C[0] < 1.5)
    slope = np.polyfit(m.C[0][mid], p[mid], 1)[0]
    return err, slope


def test_poiseuille_second_order():
    e = [_poiseuille_error(n) for n in (6, 12, 24)]
    errs = [x[0] for x in e]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 2e-3
    assert e[2][1] == pytest.approx(-12 * 0.1, rel=2e-2)


# ---------------------------------------------------------------------------
# Taylor-Green vortex decay with time-dependent wall values
# ---------------------------------------------------------------------------

def _tg_u(X, t, nu):
    x, y = X[0], X[1]
    f = np.exp(-2 * nu * t)
    return np.stack([np.sin(x) * np.cos(y) * f, -np.cos(x) * np.sin(y) * f, 0 * x])


def _taylor_green(n, nu=0.01, dt=0.01, t_end=1.0):
    L = np.pi
    sp = {"xmin": "walls", "xmax": "walls", "ymin": "walls", "ymax": "walls",
          "zmin": "frontAndBack", "zmax": "frontAndBack"}
    specs = {"walls": (mg.WALL, (0, 0, 0), 0.0), "frontAndBack": (mg.EMPTY, (0, 0, 0), 0.0)}
    m = mg.hex_box(n, n, 1, (L, L, L / n), sp, specs)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, nu)
    F = m.n_internal_faces
    u0 = _tg_u(m.C, 0.0, nu)
    # pressure of this velocity field: p = (cos 2x + cos 2y)/4 e^{-4 nu t}
    p0 = 0.25 * (np.cos(2 * m.C[0]) + np.cos(2 * m.C[1]))
    phi0 = np.einsum("ij,ij->j", _tg_u(m.Cf, 0.0, nu), m.Sf)
    cs.set_fields(u0, p0, phi0)
    Cw = patch_face_centres(m, "walls")
    V = m.V
    ke0 = 0.5 * np.sum(V * (u0 ** 2).sum(0))
    t = 0.0
    for _ in range(int(round(t_end / dt))):
        t += dt
        cs.set_patch_faces(m.patch("walls"), _tg_u(Cw, t, nu))
        st = cs.piso_step(dt, 2, p_ref_cell=0, p_tol=1e-10)
        assert st["status"] == 0
    u, p, phi = cs.get_fields()
    ue = _tg_u(m.C, t, nu)
    err = np.sqrt(np.sum(V * ((u - ue) ** 2).sum(0)) / np.sum(V * (ue ** 2).sum(0)))
    pe = 0.25 * (np.cos(2 * m.C[0]) + np.cos(2 * m.C[1])) * np.exp(-4 * nu * t)
    perr = np.sqrt(np.sum(V * ((p - p.mean()) - (pe - pe.mean())) ** 2) /
                   np.sum(V * (pe - pe.mean()) ** 2))
    ke = 0.5 * np.sum(V * (u ** 2).sum(0))
    return err, perr, ke / ke0, np.exp(-4 * nu * t)


def test_taylor_green_decay():
    e16, e32, e64 = _taylor_green(16), _taylor_green(32), _taylor_green(64)
    # velocity and pressure errors fall at (asymptotically) second order
    assert e16[0] / e32[0] > 2.5 and e32[0] / e64[0] > 3.3, (e16, e32, e64)
    assert e16[1] / e32[1] > 3.0 and e32[1] / e64[1] > 3.0, (e16, e32, e64)
    # kinetic energy decays as exp(-4 nu t)
    assert e64[2] == pytest.approx(e64[3], rel=1e-3)
    assert e32[2] == pytest.approx(e32[3], rel=1e-2)
    assert e64[0] < 2e-4


# ---------------------------------------------------------------------------
# non-orthogonal correctors: the pressure equation re-solved with the
# explicit non-orthogonal term evaluated from the newest pressure
# ---------------------------------------------------------------------------

def test_nonorth_correctors_contract_on_skewed_tets():
    """Each extra loop starts from the defect left by re-evaluating the
    explicit term at the new pressure; the loops are a contraction, so
    those initial residuals fall geometrically, and the flux correction
    (made with the last loop's term) satisfies the continuity identity."""
    m = mg.tet_box(5, 5, 5, jitter=0.15, seed=3)
    m.patches[0].u = (1.0, 0.0, 0.3)
    cs = O.Case(O.Mesh(m, renumber=True), 0.05)
    nn = 4
    for _ in range(3):
        st = cs.piso_step(0.02, 2, p_ref_cell=m.corner_cell, n_nonorth=nn, p_tol=1e-10)
        assert st["status"] == 0 and st["cont_err"] < 1e-12
        assert len(st["iters"]) == 3 + 2 * (nn + 1)
        r0 = st["res0"][3:].reshape(2, nn + 1)
        for k in range(2):
            assert (r0[k, 2:] < 0.6 * r0[k, 1:-1]).all(), r0


def test_nonorth_correctors_are_no_ops_on_orthogonal_meshes():
    m = mg.cavity2d(20)
    out = {}
    for nn in (0, 2):
        cs = O.Case(O.Mesh(m), 0.1)
        for _ in range(10):
            st = cs.piso_step(0.005, 2, p_ref_cell=m.corner_cell, n_nonorth=nn)
        if nn:
            assert (st["iters"][3:].reshape(2, 3)[:, 1:] == 0).all()
        out[nn] = cs.get_fields()
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a, b)


def test_nonorth_correctors_keep_the_simple_fixed_point():
    """At the converged SIMPLE state the pressure already satisfies the
    equation with its own explicit term, so the steady solution does not
    depend on the number of non-orthogonal correctors."""
    m = mg.duct_tets(3, 6)
    xy = patch_face_centres(m, "inlet")[:2]
    prof = mg.duct_inlet_profile(xy)
    out = {}
    for nn in (0, 2):
        cs = O.Case(O.Mesh(m, renumber=True), 0.05)
        cs.set_patch_faces(m.patch("inlet"), np.stack([0 * prof, 0 * prof, prof]))
        for it in range(3000):
            st = cs.simple_iter(0.7, 0.3, n_nonorth=nn, p_tol=1e-12, p_reltol=0.01)
            assert len(st["iters"]) == 4 + nn
            if st["init_res_max"] < 1e-10:
                break
        assert st["init_res_max"] < 1e-10
        out[nn] = cs.get_fields()
    for a, b in zip(out[0], out[2]):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)


# ---------------------------------------------------------------------------
# transient Poiseuille flow (the paper's tp1M case, Sec. 4.1): a channel
# started from rest by a sinusoidal uniform inlet velocity
# ---------------------------------------------------------------------------

def _startup_channel(ny, nsteps, T=0.5, H=1.0, L=8.0, nu=0.05, u0=1.0, w=np.pi):
    """Oracle PISO run with the inlet value set to u0 sin(w t_{n+1}) before
    every step; returns the mid-channel profile error against the exact
    start-up solution, the pressure-gradient error, and max |v|."""
    from womersley import StartupChannel
    nx = int(L / H * ny / 2)
    m = mg.channel2d(nx, ny, L, H, inlet_u=(0.0, 0.0, 0.0))
    cs = O.Case(O.Mesh(m), nu)
    q = m.patch("inlet")
    dt = T / nsteps
    for n in range(nsteps):
        cs.set_patch(q, (u0 * np.sin(w * (n + 1) * dt), 0.0, 0.0), 0.0)
        st = cs.piso_step(dt, 2)
        assert st["status"] == 0 and st["cont_err"] < 1e-12
    u, p, phi = cs.get_fields()
    S = StartupChannel(H, nu, u0, w)
    i = np.arange(m.n_cells) % nx
    a, b = nx // 2 - 1, nx // 2
    y = m.C[1][i == a]
    ue = S.u(y, T)
    eu = np.linalg.norm(u[0][i == a] - ue) / np.linalg.norm(ue)
    G = -(p[i == b] - p[i == a]).mean() / (L / nx)
    eg = abs(G - S.G(T)) / abs(S.G(T))
    # the inlet delivers Q(T) and the outlet takes it out
    F = m.n_internal_faces
    inl, out = m.patches[q], m.patches[m.patch("outlet")]
    dz = m.V[0] / (L / nx * H / ny)
    qin = -phi[F + inl.start:F + inl.start + inl.size].sum() / dz
    qout = phi[F + out.start:F + out.start + out.size].sum() / dz
    assert qin == pytest.approx(S.Q(T), rel=1e-12)
    assert qout == pytest.approx(qin, rel=1e-5)
    return eu, eg, np.abs(u[1][i == a]).max()


def test_transient_poiseuille_startup_converges():
    """Womersley number 4 (H = 1, nu = 0.05, w = pi) to a quarter period:
    the velocity profile far from both ends converges at second order to
    the exact start-up solution; the pressure gradient at first order (the
    wall shear from the half-cell distance is first order); the flow there
    is parallel."""
    e8, e16, e32 = _startup_channel(8, 25), _startup_channel(16, 50), _startup_channel(32, 100)
    assert e8[0] / e16[0] > 3.5 and e16[0] / e32[0] > 3.5, (e8, e16, e32)
    assert e32[0] < 3e-3
    assert e8[1] / e16[1] > 1.7 and e16[1] / e32[1] > 1.7, (e8, e16, e32)
    assert e32[1] < 0.05
    assert max(e8[2], e16[2], e32[2]) < 1e-6


# ---------------------------------------------------------------------------
# rectangular-duct Poiseuille series (the channel workload's analytic check)
# ---------------------------------------------------------------------------

def duct_series(x, y, terms=99):
    """Fully developed laminar flow in the unit square duct, normalised to
    mean 1: -lap u = k, u = 0 on the walls, by the double sine series."""
    u = np.zeros_like(x)
    mean = 0.0
    for a in range(1, terms + 1, 2):
        for b in range(1, terms + 1, 2):
            c = 16.0 / (np.pi ** 4 * a * b * (a * a + b * b))
            u += c * np.sin(a * np.pi * x) * np.sin(b * np.pi * y)
            mean += c * 4.0 / (a * b * np.pi ** 2)
    return u / mean


def test_duct_series_is_normalised():
    g = (np.arange(200) + 0.5) / 200
    X, Y = np.meshgrid(g, g)
    u = duct_series(X, Y, terms=39)
    assert u.mean() == pytest.approx(1.0, rel=1e-4)
    assert np.abs(u[0]).max() < 0.1 * u.max()          # vanishes towards the walls
    assert u.max() == pytest.approx(u[100, 100], rel=1e-3)  # peak on the axis


def _duct_error(n, length):
    m = mg.duct_hex(n, length)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.05)
    xy = patch_face_centres(m, "inlet")[:2]
    prof = duct_series(xy[0], xy[1])
    cs.set_patch_faces(m.patch("inlet"), np.stack([0 * prof, 0 * prof, prof]))
    for it in range(4000):
        st = cs.simple_iter(0.7, 0.3)
        assert st["status"] == 0
        if st["init_res_max"] < 1e-8:
            break
    u, p, phi = cs.get_fields()
    Lz = length / n
    last = m.C[2] > Lz - 1.0 / n
    exact = duct_series(m.C[0][last], m.C[1][last])
    return np.linalg.norm(u[2][last] - exact) / np.linalg.norm(exact)


def test_duct_outlet_profile_second_order():
    e = [_duct_error(n, 2 * n) for n in (4, 8, 16)]
    # second order once the 4x4 section is out of the way (pre-asymptotic)
    assert e[0] / e[1] > 2.2 and e[1] / e[2] > 3.2, e
    assert e[2] < 1e-2


# ---------------------------------------------------------------------------
# 3-D cavity: mirror symmetry about z = 1/2
# ---------------------------------------------------------------------------

def test_cavity3d_mirror_symmetry():
    n = 8
    m0 = mg.cavity3d(n)
    perm = mg.random_permutation(m0.n_cells, 1234)
    m = mg.permute_cells(m0, perm)
    om = O.Mesh(m, renumber=True)
    cs = O.Case(om, 0.01)
    # tight solver tolerances: the corner reference cell has no mirror image,
    # so the solution is symmetric only up to the pressure-solver error
    for _ in range(5):
        assert cs.piso_step(0.02, 2, p_ref_cell=m.corner_cell, p_tol=1e-13,
                            u_tol=1e-14)["status"] == 0
    u, p, phi = cs.get_fields()
    # mirror partner of each cell: same (x, y), z -> 1 - z
    key = lambda X: np.round(X * 2 * n).astype(np.int64)
    kk = key(m.C)
    idx = {tuple(k): i for i, k in enumerate(kk.T)}
    mirror = np.array([idx[(a, b, 2 * n - c)] for a, b, c in kk.T])
    s = np.abs(u).max()
    assert np.abs(u[0] - u[0][mirror]).max() < 1e-10 * s
    assert np.abs(u[1] - u[1][mirror]).max() < 1e-10 * s
    assert np.abs(u[2] + u[2][mirror]).max() < 1e-10 * s
    assert np.abs(u[2]).max() > 1e-3 * s          # a genuinely 3-D flow
    # the pinned reference cell keeps p there at the reference value
    assert abs(p[m.corner_cell]) < 1e-4 * np.abs(p).max()
