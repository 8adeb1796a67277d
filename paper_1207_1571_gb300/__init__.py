"""GB300-native PISO / SIMPLE finite-volume solver core.

Python binding of ``libfvgb`` (C ABI in ``include/fvgb.h``): the functions
keep the C names in :mod:`._capi`; the classes below only marshal arguments
(numpy arrays for host data, CUDA ``torch`` tensors for device data, a CUDA
stream for ordering).  Every step of the solver runs in the library's CUDA
kernels; there is no CPU or PyTorch fallback -- importing works without a
GPU, but any call that needs the library raises if it is missing.

Method: Tomczak et al., "Complete PISO and SIMPLE solvers on Graphics
Processing Units" (Sec. 3: PISO/SIMPLE with Jacobi-preconditioned CG and
BiCGStab; Sec. 3.1: face-addressed mesh, row access to the sparse matrix).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _capi
from ._capi import (FV_PREC_FP64, FV_PREC_MIXED, FV_PSOLVER_JACOBI, FV_PSOLVER_AMG, FV_E_NOT_CONVERGED, FV_OK, FvError,  # noqa
                    check, load)

__all__ = ["Mesh", "Case", "Batch", "Ellj", "mesh_plan", "ellj_build_host", "amg_coarsen_host", "load", "FvError", "FV_PREC_FP64",
           "FV_PREC_MIXED"]


def _desc(m, renumber: bool):
    """fv_mesh_desc from a mesh description with numpy arrays; returns the
    struct and the arrays it points into (kept alive by the caller)."""
    keep = dict(
        owner=np.ascontiguousarray(m.owner, dtype=np.int32),
        neighbour=np.ascontiguousarray(m.neighbour, dtype=np.int32),
        Sf=np.ascontiguousarray(m.Sf, dtype=np.float64),
        Cf=np.ascontiguousarray(m.Cf, dtype=np.float64),
        C=np.ascontiguousarray(m.C, dtype=np.float64),
        V=np.ascontiguousarray(m.V, dtype=np.float64),
    )
    pts = (_capi.fv_patch * max(1, len(m.patches)))()
    for q, p in enumerate(m.patches):
        pts[q].type, pts[q].start, pts[q].size = p.type, p.start, p.size
        for c in range(3):
            pts[q].u[c] = p.u[c]
        pts[q].p = p.p
    d = _capi.fv_mesh_desc()
    d.n_cells, d.n_internal_faces = m.n_cells, m.n_internal_faces
    d.n_boundary_faces, d.n_patches = m.n_boundary_faces, len(m.patches)
    for k in ("owner", "neighbour", "Sf", "Cf", "C", "V"):
        setattr(d, k, keep[k].ctypes.data)
    d.patches = pts
    d.renumber = 1 if renumber else 0
    keep["patches"] = pts
    return d, keep


def mesh_plan(m, renumber: bool = True):
    """Host-only addressing of fv_mesh_create: (cell new_of_old, face
    new_of_old, flipped) as numpy arrays.  Touches no GPU."""
    L = load()
    d, keep = _desc(m, renumber)
    M = m.n_internal_faces + m.n_boundary_faces
    c = np.zeros(m.n_cells, np.int32); f = np.zeros(M, np.int32); fl = np.zeros(M, np.int8)
    check(L.fv_mesh_plan(C.byref(d), c.ctypes.data, f.ctypes.data, fl.ctypes.data), "fv_mesh_plan")
    return c, f, fl


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _solve_dict(s) -> dict:
    return dict(iters=s.iters, status=s.status, res0=s.res0, res=s.res, outer=s.outer)


def _step_dict(s: _capi.fv_step_stats) -> dict:
    return dict(status=s.status, u=[_solve_dict(s.u[k]) for k in range(3)],
                p=[_solve_dict(s.p[k]) for k in range(s.n_p)],
                iters=[s.u[k].iters for k in range(3)] + [s.p[k].iters for k in range(s.n_p)],
                init_res_max=s.init_res_max)


class Mesh:
    """A mesh on the current CUDA device (``fv_mesh_create``)."""

    def __init__(self, m, renumber: bool = True, stream=None):
        import torch
        self._torch = torch
        self.L = load()
        self.desc = m
        self.N, self.F, self.B = m.n_cells, m.n_internal_faces, m.n_boundary_faces
        self.M = self.F + self.B
        self.stream = stream if stream is not None else torch.cuda.Stream()
        d, keep = _desc(m, renumber)
        h = C.c_void_p()
        check(self.L.fv_mesh_create(C.byref(d), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
              "fv_mesh_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fv_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # stream ordering between torch's current stream and the library stream
    def _enter(self, *tensors):
        cur = self._torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        for t in tensors:
            if t is not None:
                t.record_stream(self.stream)

    def _leave(self):
        self._torch.cuda.current_stream().wait_stream(self.stream)

    def _new(self, *shape, dtype=None):
        t = self._torch
        return t.zeros(*shape, dtype=dtype or t.float64, device="cuda")

    def info(self) -> dict:
        a = np.zeros(4, np.int32)
        check(self.L.fv_mesh_info(self.h, a.ctypes.data), "fv_mesh_info")
        return dict(n_cells=int(a[0]), n_internal_faces=int(a[1]), n_boundary_faces=int(a[2]),
                    nonorth=bool(a[3]))

    def cell_order(self) -> np.ndarray:
        a = np.zeros(self.N, np.int32)
        check(self.L.fv_mesh_cell_order(self.h, a.ctypes.data), "fv_mesh_cell_order")
        return a

    def face_order(self):
        a = np.zeros(self.M, np.int32); fl = np.zeros(self.M, np.int8)
        check(self.L.fv_mesh_face_order(self.h, a.ctypes.data, fl.ctypes.data), "fv_mesh_face_order")
        return a, fl

    def addressing(self):
        t = self._torch
        own = t.zeros(self.M, dtype=t.int32, device="cuda")
        nei = t.zeros(max(self.F, 1), dtype=t.int32, device="cuda")
        self._enter(own, nei)
        check(self.L.fv_mesh_addressing(self.h, own.data_ptr(), nei.data_ptr()), "fv_mesh_addressing")
        self._leave()
        return own, nei[:self.F]

    def pcg_solve(self, diag, upper, b, x, tol=1e-6, reltol=0.0, maxit=10000) -> dict:
        """Jacobi-PCG (fv_pcg_solve); x is updated in place."""
        prm = _capi.fv_pcg_params(tol, reltol, maxit, 0)
        st = _capi.fv_solve_stats()
        self._enter(diag, upper, b, x)
        rc = self.L.fv_pcg_solve(self.h, diag.data_ptr(), _ptr(upper), b.data_ptr(), x.data_ptr(),
                                 C.byref(prm), C.byref(st))
        self._leave()
        check(rc, "fv_pcg_solve", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _solve_dict(st)

    def pcg_solve_mixed(self, diag, upper, b, x, tol=1e-6, reltol=0.0, maxit=10000) -> dict:
        """FP32-inside-FP64 defect-correction CG (fv_pcg_solve_mixed)."""
        prm = _capi.fv_pcg_params(tol, reltol, maxit, 0)
        st = _capi.fv_solve_stats()
        self._enter(diag, upper, b, x)
        rc = self.L.fv_pcg_solve_mixed(self.h, diag.data_ptr(), _ptr(upper), b.data_ptr(),
                                       x.data_ptr(), C.byref(prm), C.byref(st))
        self._leave()
        check(rc, "fv_pcg_solve_mixed", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _solve_dict(st)

    def pcg_solve_amg(self, diag, upper, b, x, tol=1e-6, reltol=0.0, maxit=10000) -> dict:
        """Aggregation-multigrid preconditioned CG (fv_pcg_solve_amg)."""
        prm = _capi.fv_pcg_params(tol, reltol, maxit, 0)
        st = _capi.fv_solve_stats()
        self._enter(diag, upper, b, x)
        rc = self.L.fv_pcg_solve_amg(self.h, diag.data_ptr(), _ptr(upper), b.data_ptr(),
                                     x.data_ptr(), C.byref(prm), C.byref(st))
        self._leave()
        check(rc, "fv_pcg_solve_amg", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _solve_dict(st)

    def pcg_solve_amg_mixed(self, diag, upper, b, x, tol=1e-6, reltol=0.0, maxit=10000) -> dict:
        """Multigrid-preconditioned CG with the V-cycle in FP32 (fv_pcg_solve_amg_mixed)."""
        prm = _capi.fv_pcg_params(tol, reltol, maxit, 0)
        st = _capi.fv_solve_stats()
        self._enter(diag, upper, b, x)
        rc = self.L.fv_pcg_solve_amg_mixed(self.h, diag.data_ptr(), _ptr(upper), b.data_ptr(),
                                           x.data_ptr(), C.byref(prm), C.byref(st))
        self._leave()
        check(rc, "fv_pcg_solve_amg_mixed", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _solve_dict(st)

    def amg_levels(self) -> list:
        """Node count of every level of the multigrid hierarchy."""
        n = C.c_int32()
        sizes = np.zeros(32, np.int32)
        check(self.L.fv_amg_info(self.h, C.byref(n), sizes.ctypes.data), "fv_amg_info")
        return [int(v) for v in sizes[:n.value]]

    def bicgstab_solve(self, diag, upper, lower, b, x, tol=1e-10, reltol=0.0, maxit=1000) -> dict:
        prm = _capi.fv_pcg_params(tol, reltol, maxit, 0)
        st = _capi.fv_solve_stats()
        self._enter(diag, upper, lower, b, x)
        rc = self.L.fv_bicgstab_solve(self.h, diag.data_ptr(), _ptr(upper), _ptr(lower),
                                      b.data_ptr(), x.data_ptr(), C.byref(prm), C.byref(st))
        self._leave()
        check(rc, "fv_bicgstab_solve", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _solve_dict(st)

    def gauss_grad(self, x, xb):
        g = self._new(3, self.N)
        self._enter(x, xb, g)
        check(self.L.fv_gauss_grad(self.h, x.data_ptr(), _ptr(xb), g.data_ptr()), "fv_gauss_grad")
        self._leave()
        return g

    def ldu_matvec(self, diag, upper, lower, x):
        y = self._new(self.N)
        self._enter(diag, upper, lower, x, y)
        check(self.L.fv_ldu_matvec(self.h, diag.data_ptr(), _ptr(upper), _ptr(lower), x.data_ptr(),
                                   y.data_ptr()), "fv_ldu_matvec")
        self._leave()
        return y


def ellj_build_host(row_ptr, col, K: int) -> dict:
    """Host-only hybrid ELL + J + CRS arrays of a structurally symmetric
    pattern (``fv_ellj_build_host``): I, J as n x K arrays, crs_ptr,
    crs_col, crs_tr.  Touches no GPU."""
    L = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(row_ptr) - 1
    crs_ptr = np.zeros(n + 1, np.int32)
    ncrs = C.c_int32()
    check(L.fv_ellj_build_host(n, row_ptr.ctypes.data, col.ctypes.data, K, None, None,
                               crs_ptr.ctypes.data, None, None, C.byref(ncrs)), "fv_ellj_build_host")
    I = np.zeros((n, K), np.int32)
    J = np.zeros((n, K), np.int32)
    crs_col = np.zeros(max(ncrs.value, 1), np.int32)
    crs_tr = np.zeros(max(ncrs.value, 1), np.int32)
    check(L.fv_ellj_build_host(n, row_ptr.ctypes.data, col.ctypes.data, K, I.ctypes.data,
                               J.ctypes.data, crs_ptr.ctypes.data, crs_col.ctypes.data,
                               crs_tr.ctypes.data, C.byref(ncrs)), "fv_ellj_build_host")
    return dict(I=I, J=J, crs_ptr=crs_ptr, crs_col=crs_col[:ncrs.value], crs_tr=crs_tr[:ncrs.value])


def amg_coarsen_host(n, ea, eb, ew) -> dict:
    """Host-only multigrid coarsening level (``fv_amg_coarsen_host``):
    agg, emap and the coarse graph (n, a, b, w).  Touches no GPU."""
    L = load()
    ea = np.ascontiguousarray(ea, dtype=np.int32)
    eb = np.ascontiguousarray(eb, dtype=np.int32)
    ew = np.ascontiguousarray(ew, dtype=np.float64)
    ne = len(ea)
    agg = np.zeros(max(n, 1), np.int32)
    emap = np.zeros(max(ne, 1), np.int32)
    cea = np.zeros(max(ne, 1), np.int32); ceb = np.zeros(max(ne, 1), np.int32)
    cew = np.zeros(max(ne, 1))
    nc, nec = C.c_int32(), C.c_int32()
    check(L.fv_amg_coarsen_host(n, ne, ea.ctypes.data, eb.ctypes.data, ew.ctypes.data,
                                agg.ctypes.data, emap.ctypes.data, C.byref(nc), C.byref(nec),
                                cea.ctypes.data, ceb.ctypes.data, cew.ctypes.data),
          "fv_amg_coarsen_host")
    k = nec.value
    return dict(agg=agg[:n], emap=emap[:ne], n=nc.value, a=cea[:k], b=ceb[:k], w=cew[:k])


class Ellj:
    """The paper's hybrid ELL + J (+ CRS) storage of a mesh's LDU pattern
    (``fv_ellj_create``), with assembly from LDU coefficients and the row
    and column products."""

    def __init__(self, mesh: Mesh, K: int = 0):
        self.mesh, self.L = mesh, mesh.L
        h = C.c_void_p()
        check(self.L.fv_ellj_create(mesh.h, K, C.byref(h)), "fv_ellj_create")
        self.h = h
        k, n = C.c_int32(), C.c_int32()
        check(self.L.fv_ellj_info(self.h, C.byref(k), C.byref(n)), "fv_ellj_info")
        self.K, self.n_crs = k.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self.L.fv_ellj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def from_ldu(self, diag, upper, lower):
        """(V [K*N], C [n_crs]) device tensors holding the LDU matrix."""
        V = self.mesh._new(self.K * self.mesh.N)
        Cv = self.mesh._new(max(self.n_crs, 1))
        self.mesh._enter(diag, upper, lower, V, Cv)
        check(self.L.fv_ellj_from_ldu(self.h, diag.data_ptr(), _ptr(upper), _ptr(lower),
                                      V.data_ptr(), Cv.data_ptr()), "fv_ellj_from_ldu")
        self.mesh._leave()
        return V, Cv

    def spmv(self, V, Cv, x, mode: int = 0, y=None):
        """mode 0: A x; 1: A^T x through I and J; 2: A^T x through Q."""
        y = self.mesh._new(self.mesh.N) if y is None else y
        self.mesh._enter(V, Cv, x, y)
        check(self.L.fv_ellj_spmv(self.h, V.data_ptr(), Cv.data_ptr(), x.data_ptr(), y.data_ptr(),
                                  mode), "fv_ellj_spmv")
        self.mesh._leave()
        return y


class Case:
    """A flow case (``fv_case_create``): fields u, p, phi and boundary values."""

    def __init__(self, mesh: Mesh, nu: float, precision: int = FV_PREC_FP64):
        self.mesh = mesh
        self.L = mesh.L
        self.nu = nu
        h = C.c_void_p()
        check(self.L.fv_case_create(mesh.h, nu, precision, C.byref(h)), "fv_case_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fv_case_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory_bytes(self) -> int:
        v = C.c_int64()
        check(self.L.fv_case_memory(self.h, C.byref(v)), "fv_case_memory")
        return v.value

    def set_fields(self, u=None, p=None, phi=None, original_order=True):
        m = self.mesh
        m._enter(u, p, phi)
        check(self.L.fv_case_set_fields(self.h, _ptr(u), _ptr(p), _ptr(phi),
                                        1 if original_order else 0), "fv_case_set_fields")
        m._leave()

    def get_fields(self, original_order=True):
        m = self.mesh
        u, p, phi = m._new(3, m.N), m._new(m.N), m._new(m.M)
        m._enter(u, p, phi)
        check(self.L.fv_case_get_fields(self.h, u.data_ptr(), p.data_ptr(), phi.data_ptr(),
                                        1 if original_order else 0), "fv_case_get_fields")
        m._leave()
        return u, p, phi

    def set_fields_host(self, u=None, p=None, phi=None, original_order=True):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (u, p, phi)]
        check(self.L.fv_case_set_fields_host(self.h, *[None if a is None else a.ctypes.data
                                                       for a in arrs],
                                             1 if original_order else 0), "fv_case_set_fields_host")

    def get_fields_host(self, original_order=True):
        m = self.mesh
        u, p, phi = np.zeros((3, m.N)), np.zeros(m.N), np.zeros(m.M)
        check(self.L.fv_case_get_fields_host(self.h, u.ctypes.data, p.ctypes.data, phi.ctypes.data,
                                             1 if original_order else 0), "fv_case_get_fields_host")
        return u, p, phi

    def save(self, path: str, **extra):
        """Checkpoint: fields in the caller's numbering, as a .npz file."""
        u, p, phi = self.get_fields_host()
        np.savez(path, u=u, p=p, phi=phi, nu=self.nu, **extra)

    def load(self, path: str) -> dict:
        """Restore fields saved by :meth:`save`; returns the extra entries."""
        d = np.load(path)
        self.set_fields_host(d["u"], d["p"], d["phi"])
        return {k: d[k] for k in d.files if k not in ("u", "p", "phi", "nu")}

    def set_pressure_solver(self, solver: int):
        """FV_PSOLVER_JACOBI (default) or FV_PSOLVER_AMG."""
        check(self.L.fv_case_set_pressure_solver(self.h, solver), "fv_case_set_pressure_solver")

    def set_patch(self, q: int, u=(0.0, 0.0, 0.0), p: float = 0.0):
        uu = np.ascontiguousarray(u, dtype=np.float64)
        check(self.L.fv_patch_set_value(self.h, q, uu.ctypes.data, float(p)), "fv_patch_set_value")

    def set_patch_faces(self, q: int, u=None, p=None):
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        pp = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
        check(self.L.fv_patch_set_face_values(self.h, q, None if uu is None else uu.ctypes.data,
                                              None if pp is None else pp.ctypes.data),
              "fv_patch_set_face_values")

    def last_stats(self) -> dict:
        """Statistics of the last step (synchronises the library stream)."""
        s = _capi.fv_step_stats()
        rc = self.L.fv_case_last_stats(self.h, C.byref(s))
        check(rc, "fv_case_last_stats", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _step_dict(s)

    @staticmethod
    def piso_params(dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10, u_maxit=1000,
                    p_ref_cell=-1, p_ref=0.0, n_nonorth=0):
        return _capi.fv_piso_params(dt, n_corr, p_maxit, p_tol, u_tol, u_maxit, p_ref_cell, p_ref,
                                    n_nonorth, 0)

    def piso_step(self, dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10, u_maxit=1000,
                  p_ref_cell=-1, p_ref=0.0, stats=True, n_nonorth=0):
        prm = self.piso_params(dt, n_corr, p_tol, p_maxit, u_tol, u_maxit, p_ref_cell, p_ref,
                               n_nonorth)
        self.mesh._enter()
        if not stats:
            check(self.L.fv_piso_step(self.h, C.byref(prm), None), "fv_piso_step")
            return None
        s = _capi.fv_step_stats()
        rc = self.L.fv_piso_step(self.h, C.byref(prm), C.byref(s))
        check(rc, "fv_piso_step", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _step_dict(s)

    def run_graph(self, n_steps, dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10,
                  u_maxit=1000, p_ref_cell=-1, p_ref=0.0, stats=True, n_nonorth=0):
        prm = self.piso_params(dt, n_corr, p_tol, p_maxit, u_tol, u_maxit, p_ref_cell, p_ref,
                               n_nonorth)
        self.mesh._enter()
        s = _capi.fv_step_stats() if stats else None
        rc = self.L.fv_piso_run_graph(self.h, C.byref(prm), n_steps, C.byref(s) if stats else None)
        check(rc, "fv_piso_run_graph", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _step_dict(s) if stats else None

    def simple_iter(self, alpha_u=0.7, alpha_p=0.3, p_tol=1e-10, p_reltol=0.01, p_maxit=10000,
                    u_tol=1e-10, u_reltol=0.1, u_maxit=1000, p_ref_cell=-1, p_ref=0.0, stats=True,
                    n_nonorth=0):
        prm = _capi.fv_simple_params(alpha_u, alpha_p, p_tol, p_reltol, u_tol, u_reltol, p_maxit,
                                     u_maxit, p_ref_cell, n_nonorth, p_ref)
        self.mesh._enter()
        if not stats:
            check(self.L.fv_simple_iter(self.h, C.byref(prm), None), "fv_simple_iter")
            return None
        s = _capi.fv_step_stats()
        rc = self.L.fv_simple_iter(self.h, C.byref(prm), C.byref(s))
        check(rc, "fv_simple_iter", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return _step_dict(s)


class Batch:
    """Many independent cases advanced together (``fv_batch_create``)."""

    def __init__(self, meshes, nu, p_ref_cells=None, precision: int = FV_PREC_FP64, stream=None):
        import torch
        self.L = load()
        self.n = len(meshes)
        self.meshes = meshes
        self.stream = stream if stream is not None else torch.cuda.Stream()
        descs = (_capi.fv_mesh_desc * self.n)()
        self._keep = []
        for k, m in enumerate(meshes):
            d, keep = _desc(m, True)
            descs[k] = d
            self._keep.append(keep)
        nu_a = np.ascontiguousarray(nu, dtype=np.float64)
        ref = None if p_ref_cells is None else np.ascontiguousarray(p_ref_cells, dtype=np.int32)
        h = C.c_void_p()
        check(self.L.fv_batch_create(descs, self.n, nu_a.ctypes.data,
                                     None if ref is None else ref.ctypes.data, precision,
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h)),
              "fv_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stats(self, arr):
        return [_step_dict(arr[k]) for k in range(self.n)]

    def piso_step(self, dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10, u_maxit=1000,
                  stats=True, n_nonorth=0):
        prm = Case.piso_params(dt, n_corr, p_tol, p_maxit, u_tol, u_maxit, -1, 0.0, n_nonorth)
        arr = (_capi.fv_step_stats * self.n)() if stats else None
        self._torch_wait()
        rc = self.L.fv_batch_piso_step(self.h, C.byref(prm), arr)
        check(rc, "fv_batch_piso_step", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return self._stats(arr) if stats else None

    def run_graph(self, n_steps, dt, n_corr=2, p_tol=1e-6, p_maxit=10000, u_tol=1e-10,
                  u_maxit=1000, stats=True, n_nonorth=0):
        prm = Case.piso_params(dt, n_corr, p_tol, p_maxit, u_tol, u_maxit, -1, 0.0, n_nonorth)
        arr = (_capi.fv_step_stats * self.n)() if stats else None
        self._torch_wait()
        rc = self.L.fv_batch_run_graph(self.h, C.byref(prm), n_steps, arr)
        check(rc, "fv_batch_run_graph", allow=(FV_E_NOT_CONVERGED, _capi.FV_E_DIVERGED))
        return self._stats(arr) if stats else None

    def _torch_wait(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def get_fields(self, c):
        m = self.meshes[c]
        u, p, phi = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_faces)
        check(self.L.fv_batch_get_fields(self.h, c, u.ctypes.data, p.ctypes.data, phi.ctypes.data),
              "fv_batch_get_fields")
        return u, p, phi

    @staticmethod
    def schedules():
        L = load()
        a = np.zeros(5, np.int32)
        check(L.fv_batch_schedule_info(0, a.ctypes.data), "fv_batch_schedule_info")
        out = []
        for k in range(int(a[3])):
            check(L.fv_batch_schedule_info(k, a.ctypes.data), "fv_batch_schedule_info")
            out.append(dict(block=int(a[0]), rows_per_trip=int(a[1]), reduction=int(a[2]),
                            blocks_per_case=int(a[4])))
        return out

    def set_schedule(self, k: int):
        check(self.L.fv_batch_set_schedule(self.h, k), "fv_batch_set_schedule")

    def autotune(self, dt, n_corr=2, p_tol=1e-6, cache_path=None, key=None) -> dict:
        """Pick the fastest schedule (fv_batch_autotune); with cache_path, the
        choice is stored in / reused from a JSON file under key."""
        import json
        import os
        if cache_path and key and os.path.exists(cache_path):
            try:
                cache = json.load(open(cache_path))
                if key in cache:
                    self.set_schedule(int(cache[key]["schedule"]))
                    return dict(cache[key], cached=True)
            except Exception:
                pass
        prm = Case.piso_params(dt, n_corr, p_tol)
        ns = len(self.schedules())
        best = C.c_int32()
        ms = (C.c_double * ns)()
        self._torch_wait()
        check(self.L.fv_batch_autotune(self.h, C.byref(prm), C.byref(best), ms), "fv_batch_autotune")
        res = dict(schedule=best.value, ms=[ms[k] for k in range(ns)],
                   **self.schedules()[best.value])
        if cache_path and key:
            try:
                cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
            except Exception:
                cache = {}
            cache[key] = res
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            json.dump(cache, open(cache_path, "w"), indent=1)
        return dict(res, cached=False)
