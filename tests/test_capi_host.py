"""Host-side checks of the C ABI (no GPU): the library loads and exports every
function ``include/fvgb.h`` declares; the host addressing step
(``fv_mesh_plan``: reverse Cuthill-McKee order, face orientation and order)
matches the oracle bit for bit; malformed meshes are rejected with
FV_E_INVALID."""
import os
import re

import numpy as np
import pytest

import meshgen as mg
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1207_1571_gb300 import build as B
    B.build()
    import paper_1207_1571_gb300 as P
    P.load()
    return P


def declared():
    src = open(os.path.join(ROOT, "include", "fvgb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:fv_status|const char \*)\s*(fv_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(P):
    from paper_1207_1571_gb300 import _capi
    L = P.load()
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(_capi.EXPORTS) == names


def test_struct_sizes_match_header(P):
    from paper_1207_1571_gb300 import _capi
    import ctypes as C
    assert C.sizeof(_capi.fv_patch) == 48
    assert C.sizeof(_capi.fv_mesh_desc) == 80
    assert C.sizeof(_capi.fv_solve_stats) == 32
    assert C.sizeof(_capi.fv_step_stats) == 32 * 11 + 16
    assert C.sizeof(_capi.fv_piso_params) == 56
    assert C.sizeof(_capi.fv_simple_params) == 72
    assert C.sizeof(_capi.fv_pcg_params) == 24


def test_struct_layout_matches_header(tmp_path):
    """Every ctypes field sits at the offset a C compiler gives it from the
    header, and every struct has the header's size."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_1207_1571_gb300 import _capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_capi.fv_patch, _capi.fv_mesh_desc, _capi.fv_solve_stats, _capi.fv_step_stats,
               _capi.fv_piso_params, _capi.fv_simple_params, _capi.fv_pcg_params]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fvgb.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f in st._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        n = st.__name__
        assert got[(n, "sizeof")] == C.sizeof(st), n
        for f in st._fields_:
            assert got[(n, f[0])] == getattr(st, f[0]).offset, (n, f[0])


MESHES = {
    "cube_perm": lambda: mg.permute_cells(mg.cavity3d(7), mg.random_permutation(343, 1234)),
    "cavity2d": lambda: mg.cavity2d(9, 5),
    "tets": lambda: mg.permute_cells(mg.tet_box(3, 3, 4, jitter=0.1), mg.random_permutation(216, 3)),
    "duct": lambda: mg.duct_tets(3, 5),
    "hex_box_3x2": lambda: mg.hex_box(3, 2, 1),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("renumber", [False, True])
def test_plan_matches_oracle_bit_exact(P, name, renumber):
    m = MESHES[name]()
    c, f, fl = P.mesh_plan(m, renumber)
    oc, of, ofl = O.Mesh(m, renumber=renumber).orders()
    assert np.array_equal(c, oc)
    assert np.array_equal(f, of)
    assert np.array_equal(fl, ofl)


def _bad(P, mutate):
    from paper_1207_1571_gb300 import FvError
    m = mg.cavity3d(3)
    mutate(m)
    with pytest.raises(FvError) as e:
        P.mesh_plan(m, True)
    assert e.value.status == 1  # FV_E_INVALID
    return str(e.value)


def test_rejects_neighbour_out_of_range(P):
    def f(m):
        m.neighbour = m.neighbour.copy(); m.neighbour[5] = m.n_cells
    assert "out of range" in _bad(P, f)


def test_rejects_owner_equal_neighbour(P):
    def f(m):
        m.neighbour = m.neighbour.copy(); m.neighbour[2] = m.owner[2]
    assert "owner == neighbour" in _bad(P, f)


def test_rejects_duplicate_face(P):
    def f(m):
        m.owner = m.owner.copy(); m.neighbour = m.neighbour.copy()
        m.owner[1], m.neighbour[1] = m.neighbour[0], m.owner[0]
    assert "same two cells" in _bad(P, f)


def test_rejects_bad_volume(P):
    def f(m):
        m.V = m.V.copy(); m.V[3] = 0.0
    assert "volume" in _bad(P, f)


def test_rejects_patches_not_tiling(P):
    def f(m):
        m.patches[-1].size -= 1
    assert "patches" in _bad(P, f)


# ------------------------------------------- hybrid ELL + J (paper Sec. 3.1) --

def _ellj_equal(a, b):
    for k in ("I", "J", "crs_ptr", "crs_col", "crs_tr"):
        assert np.array_equal(a[k], b[k]), k


def test_ellj_builder_worked_example(P):
    from test_oracle_ellj import golden, example_pattern
    I, J = golden()
    rp, col = example_pattern()
    e = P.ellj_build_host(rp, col, 3)
    assert np.array_equal(e["I"], I) and np.array_equal(e["J"], J)


@pytest.mark.parametrize("K", [2, 4, 5, 7, 8])
@pytest.mark.parametrize("name", ["cube_perm", "tets", "cavity2d"])
def test_ellj_builder_matches_oracle(P, name, K):
    m = MESHES[name]()
    om = O.Mesh(m, renumber=True)
    own, nei = om.addressing()
    rp, col = O.pattern_rows(m.n_cells, own, nei)
    _ellj_equal(P.ellj_build_host(rp, col, K), O.ellj_build(rp, col, K))


def test_ellj_builder_rejects_bad_patterns(P):
    with pytest.raises(P.FvError):
        P.ellj_build_host(np.array([0, 2, 3]), np.array([0, 1, 1]), 2)   # no transpose
    with pytest.raises(P.FvError):
        P.ellj_build_host(np.array([0, 2, 3]), np.array([1, 0, 1]), 2)   # unsorted row
    with pytest.raises(P.FvError):
        P.ellj_build_host(np.array([0, 1]), np.array([0]), 0)            # K = 0


# ------------------------------------------ multigrid hierarchy (host side) --

@pytest.mark.parametrize("name", ["cube_perm", "tets", "cavity2d", "duct"])
def test_amg_coarsening_matches_oracle(P, name):
    """The library's coarsening, applied level by level to the level-0 graph
    weighted by |S_f| Delta_f (the oracle's geometry, which the device
    geometry reproduces bit for bit), gives the oracle's aggregates, edge
    maps and coarse graphs exactly."""
    m = MESHES[name]()
    om = O.Mesh(m, renumber=True)
    geo = om.geometry()
    own, nei = om.addressing()
    F = m.n_internal_faces
    a, b, w = own[:F], nei, geo["magSf"][:F] * geo["delta"][:F]
    amg = O.Amg(om)
    n, ne = amg.levels()
    cur_n = m.n_cells
    for l in range(len(n) - 1):
        lvl = P.amg_coarsen_host(cur_n, a, b, w)
        agg, emap = amg.maps(l)
        assert np.array_equal(lvl["agg"], agg) and np.array_equal(lvl["emap"], emap)
        ea, eb = amg.edges(l + 1)
        assert lvl["n"] == n[l + 1]
        assert np.array_equal(lvl["a"], ea) and np.array_equal(lvl["b"], eb)
        a, b, w, cur_n = lvl["a"], lvl["b"], lvl["w"], lvl["n"]


def test_amg_coarsening_rejects_bad_graphs(P):
    with pytest.raises(P.FvError):
        P.amg_coarsen_host(3, [1], [0], [1.0])          # not (lower, higher)
    with pytest.raises(P.FvError):
        P.amg_coarsen_host(3, [0, 0], [2, 1], [1.0, 1.0])  # not ordered
    with pytest.raises(P.FvError):
        P.amg_coarsen_host(3, [0], [1], [0.0])          # weight not positive
