"""The paper's hybrid ELL + J (+ CRS) storage on the GPU (Sec. 3.1): the
matrix scattered from LDU coefficients, the row product A x and the column
product A^T x (through J, and through the packed Q) against the oracle's
LDU product (A^T swaps the upper and lower coefficients)."""
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


def t64(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


MESHES = {
    "cube": lambda: mg.permute_cells(mg.cavity3d(12), mg.random_permutation(1728, 1234)),
    "tets": lambda: mg.tet_box(4, 5, 3, jitter=0.1),
    "cavity2d": lambda: mg.cavity2d(20),
}


@pytest.mark.parametrize("K", [0, 3, 9])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_ellj_products_match_oracle(P, name, K):
    m = MESHES[name]()
    mesh = P.Mesh(m, renumber=True)
    om = O.Mesh(m, renumber=True)
    own, nei = om.addressing()
    rng = np.random.default_rng(11)
    N, F = m.n_cells, m.n_internal_faces
    d, up, lo, x = rng.random(N) + 4, rng.standard_normal(F), rng.standard_normal(F), rng.standard_normal(N)
    e = P.Ellj(mesh, K)
    lens = np.diff(O.pattern_rows(N, own, nei)[0])
    if K == 0:
        vals, counts = np.unique(lens, return_counts=True)
        assert e.K == vals[counts == counts.max()].max()
    assert e.n_crs == np.maximum(lens - e.K, 0).sum()
    V, Cv = e.from_ldu(t64(d), t64(up), t64(lo))
    Ax = O.ldu_matvec(own, nei, d, up, lo, x)
    ATx = O.ldu_matvec(own, nei, d, lo, up, x)
    assert rel(e.spmv(V, Cv, t64(x), 0).cpu().numpy(), Ax) <= 1e-14
    assert rel(e.spmv(V, Cv, t64(x), 1).cpu().numpy(), ATx) <= 1e-14
    if e.n_crs == 0:
        assert rel(e.spmv(V, Cv, t64(x), 2).cpu().numpy(), ATx) <= 1e-14
    else:
        with pytest.raises(P.FvError):
            e.spmv(V, Cv, t64(x), 2)
    e.close()


def test_ellj_full_size_cavity(P):
    """The 100^3 cavity (seed-1234 permutation + RCM): K = 7, no CRS part;
    both products against the oracle's LDU product over the whole mesh."""
    m = mg.permute_cells(mg.cavity3d(100), mg.random_permutation(10 ** 6, 1234))
    mesh = P.Mesh(m, renumber=True)
    own, nei = mesh.addressing()
    own, nei = own.cpu().numpy(), nei.cpu().numpy()
    rng = np.random.default_rng(5)
    N, F = m.n_cells, m.n_internal_faces
    d, up, lo, x = rng.random(N) + 4, rng.standard_normal(F), rng.standard_normal(F), rng.standard_normal(N)
    e = P.Ellj(mesh)
    assert e.K == 7 and e.n_crs == 0
    V, Cv = e.from_ldu(t64(d), t64(up), t64(lo))
    y = [e.spmv(V, Cv, t64(x), k).cpu().numpy() for k in (0, 1, 2)]
    assert rel(y[0], O.ldu_matvec(own, nei, d, up, lo, x)) <= 1e-14
    assert rel(y[1], O.ldu_matvec(own, nei, d, lo, up, x)) <= 1e-14
    assert np.array_equal(y[2], y[1])
