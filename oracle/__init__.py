"""FP64 CPU oracle of the PISO / SIMPLE hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library neither imports,
links nor calls it, and this package imports nothing from the product.

``fv_oracle.c`` is a plain sequential C implementation (``-O2
-ffp-contract=off``) of the collocated finite-volume PISO time step and SIMPLE
iteration that the paper ("Complete PISO and SIMPLE solvers on GPUs", Sec. 3)
says it follows, with Jacobi-preconditioned CG for pressure and
Jacobi-preconditioned BiCGStab for momentum.  This module builds it with gcc
and binds it with ctypes.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and dense direct solves; see the pin table in the design notes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liborc_omp.so")
_lock = threading.Lock()
_libs = {}

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile ``fv_oracle.c`` into ``oracle/_build/liborc.so`` (gcc, FP64,
    no FMA contraction, no fast-math).  ``parallel=True`` builds the OpenMP
    variant ``liborc_omp.so`` (``-fopenmp -DORC_PARALLEL``: fixed-block dot
    products, Krylov loops over threads; see the source header)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if parallel else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    if parallel:
        cmd[1:1] = ["-fopenmp", "-DORC_PARALLEL"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def lib(parallel: bool = False):
    """The sequential oracle, or with ``parallel=True`` its OpenMP build."""
    parallel = bool(parallel)
    with _lock:
        if parallel not in _libs:
            L = C.CDLL(build(parallel=parallel))
            vp = C.c_void_p
            L.orc_mesh_new.restype = vp
            L.orc_mesh_new.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, _f64p, _f64p,
                                       _f64p, _f64p, C.c_int, _i32p, _i32p, _i32p, C.c_int]
            L.orc_mesh_free.argtypes = [vp]
            L.orc_mesh_orders.argtypes = [vp, _i32p, _i32p, _i8p]
            L.orc_mesh_addressing.argtypes = [vp, _i32p, _i32p]
            L.orc_mesh_geometry.argtypes = [vp, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_mesh_nonorth.argtypes = [vp]
            L.orc_mesh_nonorth.restype = C.c_int
            L.orc_ldu_matvec.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p,
                                         _f64p, _f64p]
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.orc_pcg.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                  C.c_double, C.c_double, C.c_int, dp, dp, ip]
            L.orc_pcg.restype = C.c_int
            L.orc_bicgstab.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p,
                                       _f64p, _f64p, C.c_double, C.c_double, C.c_int, dp, dp, ip]
            L.orc_bicgstab.restype = C.c_int
            L.orc_dense_solve.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_dense_solve.restype = C.c_int
            L.orc_case_new.restype = vp
            L.orc_case_new.argtypes = [vp, C.c_double]
            L.orc_case_free.argtypes = [vp]
            L.orc_case_set_fields.argtypes = [vp, _f64p, _f64p, _f64p, C.c_int]
            L.orc_case_get_fields.argtypes = [vp, _f64p, _f64p, _f64p, C.c_int]
            L.orc_case_state.argtypes = [vp, _f64p, _f64p, _f64p]
            L.orc_patch_set_value.argtypes = [vp, C.c_int, _f64p, C.c_double]
            L.orc_patch_set_face_values.argtypes = [vp, C.c_int, _f64p, vp]
            L.orc_piso_step.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int,
                                        C.c_double, C.c_int, C.c_int, C.c_double, _i32p, _f64p,
                                        dp]
            L.orc_piso_step.restype = C.c_int
            L.orc_piso_step_sched.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.c_double,
                                              C.c_int, C.c_int, C.c_double, _i32p, _i32p, _f64p,
                                              dp]
            L.orc_piso_step_sched.restype = C.c_int
            L.orc_simple_iter.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_double,
                                          C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                          C.c_int, C.c_double, _i32p, _f64p, dp, dp]
            L.orc_simple_iter.restype = C.c_int
            L.orc_case_momentum_system.argtypes = [vp, C.c_int, C.c_double, C.c_double, _f64p,
                                                   _f64p, _f64p, _f64p]
            L.orc_case_pressure_system.argtypes = [vp, C.c_double, C.c_int, C.c_double, _f64p,
                                                   _f64p, _f64p]
            L.orc_case_grad_p.argtypes = [vp, _f64p]
            L.orc_laplacian_system.argtypes = [vp, _f64p, vp, _f64p, _f64p, _f64p]
            L.orc_ellj_build.argtypes = [C.c_int, _i32p, _i32p, C.c_int, vp, vp, _i32p, vp, vp]
            L.orc_ellj_build.restype = C.c_int
            L.orc_case_set_pressure_solver.argtypes = [vp, C.c_int]
            L.orc_case_set_pressure_solver.restype = C.c_int
            L.orc_amg_new.restype = vp
            L.orc_amg_new.argtypes = [vp]
            L.orc_amg_free.argtypes = [vp]
            L.orc_amg_levels.argtypes = [vp, _i32p, _i32p]
            L.orc_amg_levels.restype = C.c_int
            L.orc_amg_maps.argtypes = [vp, C.c_int, _i32p, _i32p]
            L.orc_amg_matrix.argtypes = [vp, C.c_int, _f64p, _f64p]
            L.orc_amg_edges.argtypes = [vp, C.c_int, _i32p, _i32p]
            L.orc_amg_vcycle.argtypes = [vp, _f64p, _f64p, _f64p, _f64p]
            L.orc_amg_vcycle.restype = C.c_int
            L.orc_amg_pcg.argtypes = [vp, _f64p, _f64p, _f64p, _f64p, C.c_double, C.c_double,
                                      C.c_int, dp, dp, ip]
            L.orc_amg_pcg.restype = C.c_int
            L.orc_gauss_grad.argtypes = [vp, _f64p, _f64p, _f64p]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_threads.restype = C.c_int
            L.orc_parallel_build.restype = C.c_int
            _libs[parallel] = L
    return _libs[parallel]


def set_threads(n: int) -> None:
    """Thread count of the OpenMP build (results do not depend on it)."""
    lib(True).orc_set_threads(int(n))


def threads() -> int:
    return int(lib(True).orc_threads())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# Stand-alone solvers on LDU arrays
# ---------------------------------------------------------------------------

def pcg(own, nei, diag, upper, b, x0, tol=1e-6, reltol=0.0, maxit=10000, parallel=False):
    """Jacobi-PCG on the symmetric LDU matrix (diag, upper); returns
    ``(x, iters, res0, res, status)`` with normalised residuals."""
    N, F = len(diag), len(upper)
    x = _c(x0, np.float64).copy()
    r0, r1, it = C.c_double(), C.c_double(), C.c_int()
    st = lib(parallel).orc_pcg(N, F, _c(own[:F], np.int32), _c(nei, np.int32), _c(diag, np.float64),
                       _c(upper, np.float64), _c(b, np.float64), x, tol, reltol, maxit,
                       C.byref(r0), C.byref(r1), C.byref(it))
    return x, it.value, r0.value, r1.value, st


def bicgstab(own, nei, diag, upper, lower, b, x0, tol=1e-10, reltol=0.0, maxit=1000,
             parallel=False):
    N, F = len(diag), len(upper)
    x = _c(x0, np.float64).copy()
    r0, r1, it = C.c_double(), C.c_double(), C.c_int()
    st = lib(parallel).orc_bicgstab(N, F, _c(own[:F], np.int32), _c(nei, np.int32),
                            _c(diag, np.float64), _c(upper, np.float64), _c(lower, np.float64),
                            _c(b, np.float64), x, tol, reltol, maxit, C.byref(r0), C.byref(r1),
                            C.byref(it))
    return x, it.value, r0.value, r1.value, st


def ldu_matvec(own, nei, diag, upper, lower, x):
    N, F = len(diag), len(upper)
    y = np.zeros(N)
    lib().orc_ldu_matvec(N, F, _c(own[:F], np.int32), _c(nei, np.int32), _c(diag, np.float64),
                         _c(upper, np.float64), _c(lower, np.float64), _c(x, np.float64), y)
    return y


def dense_solve(A, b):
    """Gaussian elimination with partial pivoting (the oracle's own)."""
    A = _c(A, np.float64).copy()
    x = _c(b, np.float64).copy()
    if lib().orc_dense_solve(len(x), A, x) != 0:
        raise np.linalg.LinAlgError("singular")
    return x


# ---------------------------------------------------------------------------
# Mesh and case objects
# ---------------------------------------------------------------------------

class Mesh:
    """Oracle mesh built from a :class:`meshgen.Mesh`-like description."""

    def __init__(self, m, renumber: bool = False, parallel: bool = False):
        """``parallel=True``: run on the OpenMP build of the oracle."""
        L = self.L = lib(parallel)
        self.parallel = bool(parallel)
        self.desc = m
        self.N, self.F, self.B = m.n_cells, m.n_internal_faces, m.n_boundary_faces
        self.np = len(m.patches)
        pt = np.array([p.type for p in m.patches], np.int32)
        ps = np.array([p.start for p in m.patches], np.int32)
        pz = np.array([p.size for p in m.patches], np.int32)
        self.h = L.orc_mesh_new(self.N, self.F, self.B, _c(m.owner, np.int32),
                                _c(m.neighbour, np.int32) if self.F else np.zeros(1, np.int32),
                                _c(m.Sf, np.float64), _c(m.Cf, np.float64),
                                _c(m.C, np.float64), _c(m.V, np.float64), self.np, pt, ps, pz,
                                1 if renumber else 0)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_mesh_free(self.h)
            self.h = None

    def orders(self):
        M = self.F + self.B
        c = np.zeros(self.N, np.int32); f = np.zeros(M, np.int32); fl = np.zeros(M, np.int8)
        self.L.orc_mesh_orders(self.h, c, f, fl)
        return c, f, fl

    def addressing(self):
        own = np.zeros(self.F + self.B, np.int32); nei = np.zeros(max(self.F, 1), np.int32)
        self.L.orc_mesh_addressing(self.h, own, nei)
        return own, nei[:self.F]

    def geometry(self):
        M = self.F + self.B
        magSf, w, delta = np.zeros(M), np.zeros(max(self.F, 1)), np.zeros(M)
        kv, Sf, V = np.zeros(3 * max(self.F, 1)), np.zeros(3 * M), np.zeros(self.N)
        self.L.orc_mesh_geometry(self.h, magSf, w, delta, kv, Sf, V)
        return dict(magSf=magSf, w=w[:self.F], delta=delta, kv=kv[:3 * self.F].reshape(3, self.F),
                    Sf=Sf.reshape(3, M), V=V)

    @property
    def nonorth(self) -> bool:
        return bool(self.L.orc_mesh_nonorth(self.h))

    def gauss_grad(self, x, xb):
        g = np.zeros(3 * self.N)
        self.L.orc_gauss_grad(self.h, _c(x, np.float64), _c(xb, np.float64), g)
        return g.reshape(3, self.N)

    def laplacian_system(self, xb, gradx=None):
        d, u, b = np.zeros(self.N), np.zeros(max(self.F, 1)), np.zeros(self.N)
        g = None if gradx is None else _c(gradx, np.float64).ravel()
        self.L.orc_laplacian_system(self.h, _c(xb, np.float64),
                                   None if g is None else g.ctypes.data, d, u, b)
        return d, u[:self.F], b


class Case:
    """Oracle case: fields (u, p, phi) and boundary values on a mesh."""

    def __init__(self, mesh: Mesh, nu: float):
        self.mesh = mesh
        self.nu = nu
        self.L = mesh.L
        self.h = self.L.orc_case_new(mesh.h, nu)
        for q, p in enumerate(mesh.desc.patches):
            self.set_patch(q, p.u, p.p)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_case_free(self.h)
            self.h = None

    def set_patch(self, q: int, u, p: float = 0.0):
        self.L.orc_patch_set_value(self.h, q, _c(u, np.float64), float(p))

    def set_patch_faces(self, q: int, u, p=None):
        u = _c(u, np.float64)
        pp = None if p is None else _c(p, np.float64)
        self.L.orc_patch_set_face_values(self.h, q, u, None if pp is None else pp.ctypes.data)

    def set_fields(self, u, p, phi, original_order=True):
        self.L.orc_case_set_fields(self.h, _c(u, np.float64).ravel(), _c(p, np.float64),
                                  _c(phi, np.float64), 1 if original_order else 0)

    def get_fields(self, original_order=True):
        m = self.mesh
        u, p, phi = np.zeros(3 * m.N), np.zeros(m.N), np.zeros(m.F + m.B)
        self.L.orc_case_get_fields(self.h, u, p, phi, 1 if original_order else 0)
        return u.reshape(3, m.N), p, phi

    def state(self):
        return self.get_fields(original_order=False)

    def piso_step(self, dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10, u_maxit=1000,
                  p_ref_cell=-1, p_ref=0.0, n_nonorth=0, p_iters=None):
        """One PISO step.  p_iters (optional): the iteration count of each
        pressure solve, to replay another run's stopping decisions."""
        ns = 3 + n_corr * (n_nonorth + 1)
        its = np.zeros(ns, np.int32); res = np.zeros(2 * ns); ce = C.c_double()
        if p_iters is not None:
            sched = _c(p_iters, np.int32)
            assert sched.size == ns - 3
            st = self.L.orc_piso_step_sched(self.h, dt, n_corr, n_nonorth, u_tol, u_maxit,
                                            p_ref_cell, p_ref, sched, its, res, C.byref(ce))
        else:
            st = self.L.orc_piso_step(self.h, dt, n_corr, n_nonorth, p_tol, p_maxit, u_tol,
                                      u_maxit, p_ref_cell, p_ref, its, res, C.byref(ce))
        return dict(status=st, iters=its, res0=res[0::2], res=res[1::2], cont_err=ce.value)

    def simple_iter(self, alpha_u=0.7, alpha_p=0.3, p_tol=1e-10, p_reltol=0.01, p_maxit=10000,
                    u_tol=1e-10, u_reltol=0.1, u_maxit=1000, p_ref_cell=-1, p_ref=0.0,
                    n_nonorth=0):
        ns = 4 + n_nonorth
        its = np.zeros(ns, np.int32); res = np.zeros(2 * ns); ce = C.c_double()
        irm = C.c_double()
        st = self.L.orc_simple_iter(self.h, alpha_u, alpha_p, n_nonorth, p_tol, p_reltol, p_maxit,
                                   u_tol, u_reltol, u_maxit, p_ref_cell, p_ref, its, res,
                                   C.byref(ce), C.byref(irm))
        return dict(status=st, iters=its, res0=res[0::2], res=res[1::2], cont_err=ce.value,
                    init_res_max=irm.value)

    def set_pressure_solver(self, solver):
        """0: Jacobi-CG (default), 1: aggregation-multigrid preconditioned CG."""
        if self.L.orc_case_set_pressure_solver(self.h, solver) != 0:
            raise ValueError(f"unknown pressure solver {solver}")

    def momentum_system(self, transient=True, dt=1.0, alpha_u=1.0):
        m = self.mesh
        d, u, l, s = np.zeros(m.N), np.zeros(max(m.F, 1)), np.zeros(max(m.F, 1)), np.zeros(3 * m.N)
        self.L.orc_case_momentum_system(self.h, 1 if transient else 0, dt, alpha_u, d, u, l, s)
        return d, u[:m.F], l[:m.F], s.reshape(3, m.N)

    def pressure_system(self, dt, p_ref_cell=-1, p_ref=0.0):
        m = self.mesh
        d, u, b = np.zeros(m.N), np.zeros(max(m.F, 1)), np.zeros(m.N)
        self.L.orc_case_pressure_system(self.h, dt, p_ref_cell, p_ref, d, u, b)
        return d, u[:m.F], b

    def grad_p(self):
        g = np.zeros(3 * self.mesh.N)
        self.L.orc_case_grad_p(self.h, g)
        return g.reshape(3, self.mesh.N)


def ellj_build(row_ptr, col, K):
    """Hybrid ELL + J + CRS arrays of a structurally symmetric pattern (paper
    Sec. 3.1): returns dict(I, J) as N x K arrays, crs_ptr, crs_col, crs_tr."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(row_ptr) - 1
    crs_ptr = np.zeros(n + 1, np.int32)
    ncrs = lib().orc_ellj_build(n, row_ptr, col, K, None, None, crs_ptr, None, None)
    I = np.zeros((n, K), np.int32)
    J = np.zeros((n, K), np.int32)
    crs_col = np.zeros(max(ncrs, 1), np.int32)
    crs_tr = np.zeros(max(ncrs, 1), np.int32)
    rc = lib().orc_ellj_build(n, row_ptr, col, K, I.ctypes.data, J.ctypes.data, crs_ptr,
                              crs_col.ctypes.data, crs_tr.ctypes.data)
    if rc < 0:
        raise ValueError("sparsity pattern is not structurally symmetric")
    return dict(I=I, J=J, crs_ptr=crs_ptr, crs_col=crs_col[:ncrs], crs_tr=crs_tr[:ncrs])


def pattern_rows(n, own, nei):
    """Row structure of an LDU matrix (diagonal plus both sides of every
    internal face), columns ascending: (row_ptr, col)."""
    own = np.asarray(own[:len(nei)], dtype=np.int64)
    nei = np.asarray(nei, dtype=np.int64)
    r = np.concatenate([np.arange(n), own, nei])
    c = np.concatenate([np.arange(n), nei, own])
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, r + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), c.astype(np.int32)


class Amg:
    """Aggregation multigrid hierarchy of a mesh (orc_amg_new) and the
    V-cycle preconditioned CG for symmetric LDU matrices in the mesh's
    internal order."""

    def __init__(self, mesh: "Mesh"):
        self._mesh = mesh
        self.L = mesh.L
        self.h = self.L.orc_amg_new(mesh.h)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_amg_free(self.h)
            self.h = None

    def levels(self):
        n = np.zeros(32, np.int32); ne = np.zeros(32, np.int32)
        k = self.L.orc_amg_levels(self.h, n, ne)
        return n[:k].copy(), ne[:k].copy()

    def maps(self, l):
        n, ne = self.levels()
        agg = np.zeros(max(n[l], 1), np.int32); emap = np.zeros(max(ne[l], 1), np.int32)
        self.L.orc_amg_maps(self.h, l, agg, emap)
        return agg[:n[l]], emap[:ne[l]]

    def matrix(self, l):
        """Level-l (diag, off) of the matrix of the last V-cycle or solve."""
        n, ne = self.levels()
        d = np.zeros(max(n[l], 1)); o = np.zeros(max(ne[l], 1))
        self.L.orc_amg_matrix(self.h, l, d, o)
        return d[:n[l]], o[:ne[l]]

    def edges(self, l):
        n, ne = self.levels()
        a = np.zeros(max(ne[l], 1), np.int32); b = np.zeros(max(ne[l], 1), np.int32)
        self.L.orc_amg_edges(self.h, l, a, b)
        return a[:ne[l]], b[:ne[l]]

    def vcycle(self, diag, upper, r):
        z = np.zeros(len(diag))
        if self.L.orc_amg_vcycle(self.h, _c(diag, np.float64), _c(upper, np.float64),
                                _c(r, np.float64), z) != 0:
            raise ValueError("coarsest matrix is not positive definite")
        return z

    def pcg(self, diag, upper, b, x0, tol=1e-6, reltol=0.0, maxit=10000):
        x = np.array(x0, dtype=np.float64, copy=True)
        r0, r1, it = C.c_double(), C.c_double(), C.c_int()
        st = self.L.orc_amg_pcg(self.h, _c(diag, np.float64), _c(upper, np.float64),
                               _c(b, np.float64), x, tol, reltol, maxit, C.byref(r0),
                               C.byref(r1), C.byref(it))
        return x, it.value, r0.value, r1.value, st

