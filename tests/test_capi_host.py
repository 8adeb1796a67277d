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
    assert C.sizeof(_capi.fv_piso_params) == 48
    assert C.sizeof(_capi.fv_simple_params) == 72
    assert C.sizeof(_capi.fv_pcg_params) == 24


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
