"""The 8M-cell cavity (200^3 hex cells, permuted with seed 1234, RCM: the mesh
of the mixed-precision configuration; nu 0.01, dt 0.001, 2 correctors, CG to
1e-6) at full size, in the launch configuration the benchmark times (152
blocks, the CG row vectors in global memory because a block's rows do not
fit in shared memory).

* The first two PISO steps from rest, FP64, in lockstep with the oracle (its
  OpenMP build on all host cores): iteration counts within 1, fields within
  1e-9; the same two steps with the mixed-precision pressure solve, whose
  per-field error against the FP64 oracle is reported (u, phi, mean-free p,
  mean of p; ``-rA`` shows it) and bounded.
* Properties that hold at any size, checked with an independent sparse
  matrix-vector product (SciPy): the FP64 and the mixed-precision pressure
  solves of a pinned Laplacian meet ||b - A x||_2 <= 1e-6 ||b||_2 (the FP64
  one up to the drift of its recursively updated residual)."""
import os
import time

import numpy as np
import pytest

import meshgen as mg
import oracle as O
from parity_util import field_errors, assert_errors_within

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


def test_full_size_200_cubed_two_piso_steps_fp64_and_mixed(P):
    n = 200
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    O.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    om = O.Mesh(m, renumber=True, parallel=True)
    oc = O.Case(om, 0.01)
    t_mesh = time.perf_counter() - t0
    mesh = P.Mesh(m, renumber=True)
    assert np.array_equal(mesh.cell_order(), om.orders()[0])
    c64 = P.Case(mesh, 0.01)
    cmx = P.Case(mesh, 0.01, P.FV_PREC_MIXED)
    t_step = []
    for step in range(2):
        s = c64.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
        sm = cmx.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
        t0 = time.perf_counter()
        so = oc.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
        t_step.append(time.perf_counter() - t0)
        assert s["status"] == 0 and sm["status"] == 0, (s, sm)
        gi, oi = np.array(s["iters"]), so["iters"]
        assert np.abs(gi - oi).max() <= 1, (step, gi, oi)
        assert all(x["res"] <= 1e-6 for x in sm["p"]), sm
        ref = oc.get_fields()
        e64 = field_errors(c64.get_fields_host(), ref)
        emx = field_errors(cmx.get_fields_host(), ref)
        print(f"\n200^3 cavity step {step + 1}: FP64 vs oracle {e64}\n mixed vs FP64 oracle {emx}"
              f"\n iterations GPU {gi.tolist()} oracle {oi.tolist()} mixed {sm['iters']}")
        assert_errors_within(e64)
        # mixed precision: the FP32 inner solve changes the iterates at the
        # level of the 1e-6 stopping tolerance, not of rounding
        assert emx["u"] < 1e-5 and emx["phi"] < 1e-5 and emx["p_meanfree"] < 1e-4, emx
    print(f" oracle on {O.threads()} threads: mesh {t_mesh:.1f} s, steps "
          f"{', '.join(f'{t:.1f}' for t in t_step)} s")


def test_full_size_200_cubed_pressure_solves(P):
    sparse = pytest.importorskip("scipy.sparse")
    n = 200
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    mesh = P.Mesh(m, renumber=True)
    own_t, nei_t = mesh.addressing()
    F, N = m.n_internal_faces, m.n_cells
    own = own_t.cpu().numpy()[:F].astype(np.int64)
    nei = nei_t.cpu().numpy().astype(np.int64)
    assert (own < nei).all()
    # the pressure Laplacian of the uniform cube (a_f = |S| Delta = h, walls
    # zero-gradient) pinned at internal cell 0, as the reference-cell rule does
    h = 1.0 / n
    a = np.full(F, h)
    d = np.bincount(own, weights=a, minlength=N) + np.bincount(nei, weights=a, minlength=N)
    d[0] *= 2.0
    up = -a
    A = sparse.csr_matrix((np.concatenate([d, up, up]),
                           (np.concatenate([np.arange(N), own, nei]),
                            np.concatenate([np.arange(N), nei, own]))), shape=(N, N))
    # a mean-free right-hand side (about 1,600 Jacobi-CG iterations, like the
    # cavity's own pressure solves at this size)
    b = np.random.default_rng(11).standard_normal(N) * h ** 3
    b -= b.mean()
    nb = np.linalg.norm(b)
    for solve in (mesh.pcg_solve, mesh.pcg_solve_mixed):
        x = t64(np.zeros(N))
        s = solve(t64(d), t64(up), t64(b), x, tol=1e-6)
        assert s["status"] == 0, s
        xh = x.cpu().numpy()
        res = np.linalg.norm(b - A @ xh) / nb
        # FP64: the recursively updated residual meets 1e-6, the true one to
        # within its drift; mixed: the stop is on the FP64 true residual
        assert res <= 1.5e-6, (solve.__name__, res, s)
        assert s["res"] <= 1e-6 * (1 + 1e-9)
