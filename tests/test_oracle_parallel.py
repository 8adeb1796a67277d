"""Pins of the oracle's OpenMP build (liborc_omp.so) against its sequential
build: the two differ only in how dot products are summed (fixed blocks of
4096 terms, block sums added pairwise), so solver iteration counts agree,
fields agree to rounding, and the parallel results do not depend on the
number of threads (bit for bit)."""
import numpy as np
import pytest

import meshgen as mg
import oracle as O


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(autouse=True)
def _restore_threads():
    n = O.threads()
    yield
    O.set_threads(n)


def _cavity(n, seed=1234):
    return mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, seed))


def test_parallel_build_flags():
    assert O.lib(True).orc_parallel_build() == 1
    assert O.lib(False).orc_parallel_build() == 0


def test_pcg_parallel_matches_sequential():
    m = _cavity(26)          # 17576 cells: five dot-product blocks
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.01)
    oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    d, up, b = oc.pressure_system(0.01, p_ref_cell=m.corner_cell)
    own, nei = om.addressing()
    xs, its, _, rs, sts = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-10)
    xp, itp, _, rp, stp = O.pcg(own, nei, d, up, b, np.zeros(m.n_cells), tol=1e-10, parallel=True)
    assert sts == stp == 0 and abs(its - itp) <= 1
    assert rel(xp, xs) < 1e-11
    # a face order that is not sorted by (owner, neighbour): the parallel
    # build keeps the face-loop product there and still agrees
    perm = np.random.default_rng(3).permutation(len(up))
    xq, itq, _, _, stq = O.pcg(own[:len(up)][perm], nei[perm], d, up[perm], b,
                               np.zeros(m.n_cells), tol=1e-10, parallel=True)
    assert stq == 0 and abs(itq - its) <= 1 and rel(xq, xs) < 1e-11


def test_bicgstab_parallel_matches_sequential():
    m = mg.tet_box(5, 5, 5, jitter=0.1, seed=2)
    m.patches[0].u = (1.0, 0.2, 0.0)
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.02)
    oc.piso_step(0.02, 2, p_ref_cell=0)
    d, up, lo, src = oc.momentum_system(True, 0.02)
    own, nei = om.addressing()
    for c in range(2):
        xs, its, _, _, sts = O.bicgstab(own, nei, d, up, lo, src[c], np.zeros(m.n_cells))
        xp, itp, _, _, stp = O.bicgstab(own, nei, d, up, lo, src[c], np.zeros(m.n_cells),
                                        parallel=True)
        assert sts == stp == 0 and abs(its - itp) <= 1
        assert rel(xp, xs) < 1e-11


def test_piso_parallel_matches_sequential_and_is_thread_count_independent():
    m = _cavity(25)          # 15625 cells: four blocks
    runs = {}
    for key, par, nt in (("seq", False, 1), ("par1", True, 1), ("par3", True, 3)):
        if par:
            O.set_threads(nt)
        oc = O.Case(O.Mesh(m, renumber=True, parallel=par), 0.01)
        its = [oc.piso_step(0.002, 2, p_ref_cell=m.corner_cell)["iters"] for _ in range(3)]
        runs[key] = (np.array(its), oc.get_fields())
    its_s, f_s = runs["seq"]
    its_1, f_1 = runs["par1"]
    its_3, f_3 = runs["par3"]
    assert np.array_equal(its_1, its_3)
    for a, b in zip(f_1, f_3):
        assert np.array_equal(a, b)
    assert np.abs(its_1 - its_s).max() <= 1
    for a, b in zip(f_1, f_s):
        assert rel(a, b) < 1e-10
