"""fv_pcg_solve_noalloc: the pressure CG solve for callers that cannot let the
library allocate device memory when they solve (their memory is all handed
out by their own allocator, or a global-mode stream capture is active in the
process).  It must give the same answer as fv_pcg_solve, call after call,
while using only the library's static scratch array.

This file is collected last on purpose; it works alone in a fresh process
and after the other tests."""
import ctypes as C

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


def t64(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _system(m, steps=2):
    # a pressure system of the lid-driven cavity, assembled by the oracle
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.01)
    for _ in range(steps):
        oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    return oc.pressure_system(0.01, p_ref_cell=m.corner_cell)


def _solve(P, mesh, fn, d, up, b, x0, tol):
    from paper_1207_1571_gb300 import _capi
    import torch
    prm = _capi.fv_pcg_params(tol, 0.0, 10000, 0)
    st = _capi.fv_solve_stats()
    x = t64(x0)
    dd, uu, bb = t64(d), t64(up), t64(b)
    torch.cuda.synchronize()
    rc = fn(mesh.h, dd.data_ptr(), uu.data_ptr(), bb.data_ptr(), x.data_ptr(), C.byref(prm),
            C.byref(st))
    return rc, st, x.cpu().numpy()


@pytest.mark.parametrize("n", [12, 40])
def test_noalloc_solve_matches_allocating_solve_twice(P, n):
    L = P.load()
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    d, up, b = _system(m)
    mesh = P.Mesh(m, renumber=True)
    x0 = np.zeros(m.n_cells)
    rc_ref, st_ref, x_ref = _solve(P, mesh, L.fv_pcg_solve, d, up, b, x0, 1e-8)
    assert rc_ref == 0 and st_ref.status == 0
    for call in range(2):
        rc, st, x = _solve(P, mesh, L.fv_pcg_solve_noalloc, d, up, b, x0, 1e-8)
        assert rc == 0 and st.status == 0
        assert abs(st.iters - st_ref.iters) <= 1
        assert np.linalg.norm(x - x_ref) <= TOL * np.linalg.norm(x_ref)
    # a different right-hand side right after: the kept array contents must
    # not leak into the next solve
    rc, st, x = _solve(P, mesh, L.fv_pcg_solve_noalloc, d, up, 2.0 * b, x0, 1e-8)
    rc2, st2, x2 = _solve(P, mesh, L.fv_pcg_solve, d, up, 2.0 * b, x0, 1e-8)
    assert rc == 0 and np.linalg.norm(x - x2) <= TOL * np.linalg.norm(x2)


def test_noalloc_rejects_meshes_beyond_its_limit(P):
    L = P.load()
    m = mg.cavity3d(51)          # 132651 cells > 131072
    mesh = P.Mesh(m, renumber=False)
    rc, st, x = _solve(P, mesh, L.fv_pcg_solve_noalloc, np.ones(m.n_cells),
                       np.zeros(m.n_internal_faces), np.ones(m.n_cells), np.zeros(m.n_cells), 1e-6)
    assert rc == 1  # FV_E_INVALID
    assert b"at most 131072 cells" in L.fv_last_error()
