"""fv_pcg_solve_noalloc: the pressure CG solve for callers that cannot let the
library allocate device memory when they solve (their memory is all handed
out by their own allocator, or a global-mode stream capture is active in the
process).  It must give the same answer as fv_pcg_solve and as the FP64
oracle's Jacobi-CG, call after call, while using only the library's static
scratch array -- no device memory may change hands during a call.

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
    # a pressure system of the lid-driven cavity, assembled by the oracle, in
    # the oracle's internal (renumbered) order, with that order's addressing
    om = O.Mesh(m, renumber=True)
    oc = O.Case(om, 0.01)
    for _ in range(steps):
        oc.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    d, up, b = oc.pressure_system(0.01, p_ref_cell=m.corner_cell)
    own, nei = om.addressing()
    return d, up, b, own, nei


class _Solver:
    """Device copies of one system made up front, so that a call moves no
    memory through torch's allocator either."""

    def __init__(self, P, mesh, d, up, b, x0, tol):
        from paper_1207_1571_gb300 import _capi
        import torch
        self.mesh = mesh
        self.prm = _capi.fv_pcg_params(tol, 0.0, 10000, 0)
        self.st = _capi.fv_solve_stats()
        self.dd, self.uu, self.bb = t64(d), t64(up), t64(b)
        self.x0 = t64(x0)
        self.x = self.x0.clone()
        torch.cuda.synchronize()

    def __call__(self, fn):
        import torch
        self.x.copy_(self.x0)
        torch.cuda.synchronize()
        rc = fn(self.mesh.h, self.dd.data_ptr(), self.uu.data_ptr(), self.bb.data_ptr(),
                self.x.data_ptr(), C.byref(self.prm), C.byref(self.st))
        torch.cuda.synchronize()
        return rc, self.st.status, self.st.iters

    def solution(self):
        return self.x.cpu().numpy()


@pytest.mark.parametrize("n", [12, 40])
def test_noalloc_solve_matches_oracle_and_allocating_solve_twice(P, n):
    L = P.load()
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    d, up, b, own, nei = _system(m)
    x0 = np.zeros(m.n_cells)
    x_or, it_or, _, _, st_or = O.pcg(own, nei, d, up, b, x0, tol=1e-8)
    assert st_or == 0
    mesh = P.Mesh(m, renumber=True)
    s = _Solver(P, mesh, d, up, b, x0, 1e-8)
    rc_ref, st_ref, it_ref = s(L.fv_pcg_solve)
    assert rc_ref == 0 and st_ref == 0
    x_ref = s.solution()
    for call in range(2):
        rc, st, it = s(L.fv_pcg_solve_noalloc)
        assert rc == 0 and st == 0
        x = s.solution()
        # against the oracle (Jacobi-CG of the paper, FP64, same stopping rule)
        assert abs(it - it_or) <= 1, (call, it, it_or)
        assert np.linalg.norm(x - x_or) <= TOL * np.linalg.norm(x_or)
        # and against the allocating entry point
        assert abs(it - it_ref) <= 1
        assert np.linalg.norm(x - x_ref) <= TOL * np.linalg.norm(x_ref)
    # a different right-hand side right after: the kept array contents must
    # not leak into the next solve
    x2_or, it2_or, _, _, _ = O.pcg(own, nei, d, up, 2.0 * b, x0, tol=1e-8)
    s2 = _Solver(P, mesh, d, up, 2.0 * b, x0, 1e-8)
    rc, st, it = s2(L.fv_pcg_solve_noalloc)
    assert rc == 0 and abs(it - it2_or) <= 1
    x2 = s2.solution()
    assert np.linalg.norm(x2 - x2_or) <= TOL * np.linalg.norm(x2_or)


def test_noalloc_calls_take_no_device_memory(P):
    """The defining property: after a first call has loaded the kernels,
    further calls -- also on a mesh never solved on before -- leave the
    device's free memory and the library's own allocations unchanged."""
    import torch
    L = P.load()
    ma = mg.permute_cells(mg.cavity3d(16), mg.random_permutation(16 ** 3, 1234))
    mb = mg.cavity3d(24)
    da, ua, ba, _, _ = _system(ma, steps=1)
    db, ub, bb, _, _ = _system(mb, steps=1)
    mesh_a = P.Mesh(ma, renumber=True)
    mesh_b = P.Mesh(mb, renumber=True)
    case_b = P.Case(mesh_b, 0.01)          # reports the mesh's arena bytes too
    sa = _Solver(P, mesh_a, da, ua, ba, np.zeros(ma.n_cells), 1e-8)
    sb = _Solver(P, mesh_b, db, ub, bb, np.zeros(mb.n_cells), 1e-8)
    assert sa(L.fv_pcg_solve_noalloc)[0] == 0          # warm-up: kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    arena0 = case_b.memory_bytes()
    for _ in range(2):
        assert sa(L.fv_pcg_solve_noalloc)[0] == 0
        assert sb(L.fv_pcg_solve_noalloc)[0] == 0      # first solve on mesh_b
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert case_b.memory_bytes() == arena0
    case_b.close()


def test_noalloc_rejects_meshes_beyond_its_limit(P):
    L = P.load()
    m = mg.cavity3d(51)          # 132651 cells > 131072
    mesh = P.Mesh(m, renumber=False)
    s = _Solver(P, mesh, np.ones(m.n_cells), np.zeros(m.n_internal_faces), np.ones(m.n_cells),
                np.zeros(m.n_cells), 1e-6)
    rc, _, _ = s(L.fv_pcg_solve_noalloc)
    assert rc == 1  # FV_E_INVALID
    assert b"at most 131072 cells" in L.fv_last_error()
