"""Pins of the oracle's hybrid ELL + J (+ CRS overflow) builder (paper
Sec. 3.1) against the paper's worked example and the defining property of
J (the transposed entry of slot (i, k) sits in row I[i][k], slot J[i][k]),
including rows longer than K whose tails go to the CRS part."""
import os

import numpy as np
import pytest

import meshgen as mg
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ellj_example.txt")


def golden():
    sec, out = None, {"I": [], "J": []}
    for line in open(GOLDEN):
        line = line.strip()
        if line.startswith("# section"):
            sec = line.split()[-1]
        elif line and not line.startswith("#"):
            out[sec].append([int(v) for v in line.split()])
    return np.array(out["I"]), np.array(out["J"])


def example_pattern():
    rows = [[0, 1, 3], [0, 1, 2], [1, 2, 3], [0, 2, 3]]
    return np.cumsum([0] + [len(r) for r in rows]), np.concatenate(rows)


def test_paper_worked_example():
    I, J = golden()
    rp, col = example_pattern()
    e = O.ellj_build(rp, col, 3)
    assert np.array_equal(e["I"], I)
    assert np.array_equal(e["J"], J)
    assert len(e["crs_col"]) == 0
    assert e["J"][1, 2] == 0                      # the entry the paper works by hand


def check_transpose_property(rp, col, K, e):
    n = len(rp) - 1
    I, J = e["I"], e["J"]
    crs_ptr, crs_col, crs_tr = e["crs_ptr"], e["crs_col"], e["crs_tr"]

    def entry_col(j, loc):
        return I[j, loc] if loc >= 0 else crs_col[-2 - loc]

    def row_of_crs(p):
        return int(np.searchsorted(crs_ptr, p, side="right") - 1)

    for i in range(n):
        cols = list(col[rp[i]:rp[i + 1]])
        got = [c for c in I[i] if c >= 0] + list(crs_col[crs_ptr[i]:crs_ptr[i + 1]])
        assert got == cols                         # the row, in order, ELL first
        for k in range(K):
            if I[i, k] < 0:
                assert J[i, k] == -1 and k >= len(cols)
                continue
            j = I[i, k]
            loc = J[i, k]
            assert entry_col(j, loc) == i          # the transposed entry
            if loc < -1:
                assert row_of_crs(-2 - loc) == j
        for p in range(crs_ptr[i], crs_ptr[i + 1]):
            j, loc = crs_col[p], crs_tr[p]
            assert entry_col(j, loc) == i
            if loc < -1:
                assert row_of_crs(-2 - loc) == j


@pytest.mark.parametrize("K", [3, 4, 7, 9])
def test_transpose_index_on_meshes(K):
    for m in (mg.cavity3d(4), mg.tet_box(2, 3, 2, jitter=0.1)):
        om = O.Mesh(m, renumber=True)
        own, nei = om.addressing()
        rp, col = O.pattern_rows(m.n_cells, own, nei)
        e = O.ellj_build(rp, col, K)
        lens = np.diff(rp)
        assert len(e["crs_col"]) == np.maximum(lens - K, 0).sum()
        check_transpose_property(rp, col, K, e)


def test_hex_interior_rows_fill_seven_slots():
    m = mg.cavity3d(5)
    om = O.Mesh(m, renumber=True)
    own, nei = om.addressing()
    rp, col = O.pattern_rows(m.n_cells, own, nei)
    lens = np.diff(rp)
    assert lens.max() == 7 and (lens == 7).sum() == 27      # 3^3 interior cells
    e = O.ellj_build(rp, col, 7)
    assert len(e["crs_col"]) == 0                            # C vanishes on structured meshes


def test_unsymmetric_pattern_is_rejected():
    rp, col = np.array([0, 2, 3]), np.array([0, 1, 1])      # (0,1) without (1,0)
    with pytest.raises(ValueError):
        O.ellj_build(rp, col, 2)


def test_q_encoding_round_trip():
    """I and J packed in one integer, Q = K I + J (J < K), decoded by
    integer division and remainder."""
    I, J = golden()
    K = 3
    Q = K * I + J
    assert np.array_equal(Q // K, I) and np.array_equal(Q % K, J)
