"""The SIMPLE channel workload at full size: a 48x48x192 hex box split into
2,654,208 jittered Kuhn tetrahedra (seed 2024), parabolic inlet with mean 1,
nu 0.05, relaxation 0.7 / 0.3.

* the first SIMPLE iteration against the FP64 oracle (same inputs);
* iterated to an outer residual of 1e-6, the outlet profile against the
  fully developed square-duct (Poiseuille) series solution."""
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


@pytest.fixture(scope="module")
def duct():
    m = mg.duct_tets(48, 192, jitter=0.1, seed=2024)
    F = m.n_internal_faces
    inl = m.patches[m.patch("inlet")]
    xy = m.Cf[:2, F + inl.start:F + inl.start + inl.size]
    prof = mg.duct_inlet_profile(xy)
    return m, np.stack([0 * prof, 0 * prof, prof])


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def duct_series(x, y, terms=99):
    u = np.zeros_like(x)
    mean = 0.0
    for a in range(1, terms + 1, 2):
        for b in range(1, terms + 1, 2):
            c = 16.0 / (np.pi ** 4 * a * b * (a * a + b * b))
            u += c * np.sin(a * np.pi * x) * np.sin(b * np.pi * y)
            mean += c * 4.0 / (a * b * np.pi ** 2)
    return u / mean


def test_channel_first_iteration_matches_oracle(P, duct):
    m, inlet = duct
    assert m.n_cells == 2654208 and m.n_internal_faces == 5266944 and m.n_boundary_faces == 82944
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.05)
    q = m.patch("inlet")
    case.set_patch_faces(q, inlet)
    om = O.Mesh(m, renumber=True)
    assert np.array_equal(mesh.cell_order(), om.orders()[0])
    oc = O.Case(om, 0.05)
    oc.set_patch_faces(q, inlet)
    s = case.simple_iter(0.7, 0.3)
    so = oc.simple_iter(0.7, 0.3)
    assert np.abs(np.array(s["iters"]) - so["iters"]).max() <= 1, (s["iters"], so["iters"])
    for a, b in zip(case.get_fields_host(), oc.get_fields()):
        assert rel(a, b) <= 1e-9
    assert s["init_res_max"] == pytest.approx(so["init_res_max"], rel=1e-6)


def test_channel_converges_to_duct_profile(P, duct):
    m, inlet = duct
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, 0.05)
    case.set_patch_faces(m.patch("inlet"), inlet)
    res = None
    for it in range(6000):
        st = case.simple_iter(0.7, 0.3, stats=(it % 25 == 0))
        if st is not None:
            res = st["init_res_max"]
            assert st["status"] in (0, 4)
            if res < 1e-6:
                break
    st = case.simple_iter(0.7, 0.3)
    assert st["init_res_max"] < 1e-6, st["init_res_max"]
    u, p, phi = case.get_fields_host()
    # outlet profile: cells of the last hex layer (z > Lz - h)
    h = 1.0 / 48
    Lz = 4.0
    last = m.C[2] > Lz - h
    exact = duct_series(m.C[0][last], m.C[1][last])
    err = rel(u[2][last], exact)
    print(f"SIMPLE iterations {it + 1}, outlet profile rel L2 error {err:.4f}")
    # Jittered tetrahedra: the Gauss gradient with linear interpolation is
    # not consistent on skewed cells (pinned on the oracle in
    # test_oracle_operators), so the developed profile keeps a skewness error
    # of a few percent at this resolution (2.5 % measured); on hexahedra the
    # same solver converges at second order (test_oracle_flows).
    assert err < 0.03
    # mass balance: inflow = outflow
    F = m.n_internal_faces
    inl, out = m.patches[m.patch("inlet")], m.patches[m.patch("outlet")]
    fin = phi[F + inl.start:F + inl.start + inl.size].sum()
    fout = phi[F + out.start:F + out.start + out.size].sum()
    assert fin == pytest.approx(-1.0, rel=1e-3)
    assert fout == pytest.approx(-fin, rel=1e-5)
