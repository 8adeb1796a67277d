"""Seeded synthetic finite-volume meshes and case descriptions.

This module produces the *inputs* that both the CUDA library and the CPU
oracle consume: face-addressed polyhedral meshes (owner/neighbour lists,
face area vectors, face centres, cell centroids and volumes, boundary
patches), cell permutations, and the parameter sets of the lid-driven
cavity, duct and batch workloads.  It contains geometry of the meshes only;
none of the finite-volume discretisation, the pressure/velocity coupling or
the linear solvers lives here.

Mesh conventions (the paper's mesh model, Sec. 3.1: every face belongs to
exactly two cells or is a boundary face):

* ``owner[f]`` for all ``F + B`` faces, ``neighbour[f]`` for the ``F``
  internal faces, which come first; boundary faces follow, grouped by patch.
* ``Sf`` is the face area vector, shape ``(3, F + B)``, pointing out of the
  owner cell (towards the neighbour for internal faces).
* ``Cf`` face centres ``(3, F + B)``; ``C`` cell centroids ``(3, N)``; ``V``
  cell volumes ``(N,)``.
* Patch types: 0 wall (fixed velocity, zero-gradient pressure), 1 inlet
  (fixed velocity, zero-gradient pressure), 2 outlet (zero-gradient velocity,
  fixed pressure), 3 empty (front/back of a 2-D mesh; ignored).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

WALL, INLET, OUTLET, EMPTY = 0, 1, 2, 3


@dataclasses.dataclass
class Patch:
    name: str
    type: int
    start: int          # offset into the boundary faces (0 .. B-1)
    size: int
    u: tuple = (0.0, 0.0, 0.0)
    p: float = 0.0


@dataclasses.dataclass
class Mesh:
    n_cells: int
    n_internal_faces: int
    n_boundary_faces: int
    owner: np.ndarray       # int32 [F+B]
    neighbour: np.ndarray   # int32 [F]
    Sf: np.ndarray          # float64 [3, F+B]
    Cf: np.ndarray          # float64 [3, F+B]
    C: np.ndarray           # float64 [3, N]
    V: np.ndarray           # float64 [N]
    patches: List[Patch]
    # index (in this mesh's cell numbering) of the cell at the domain origin
    # corner; used as the pressure reference cell of closed cavities
    corner_cell: int = 0

    @property
    def n_faces(self) -> int:
        return self.n_internal_faces + self.n_boundary_faces

    def patch(self, name: str) -> int:
        for i, p in enumerate(self.patches):
            if p.name == name:
                return i
        raise KeyError(name)

    def copy(self) -> "Mesh":
        return dataclasses.replace(
            self, owner=self.owner.copy(), neighbour=self.neighbour.copy(),
            Sf=self.Sf.copy(), Cf=self.Cf.copy(), C=self.C.copy(), V=self.V.copy(),
            patches=[dataclasses.replace(p) for p in self.patches])


# ---------------------------------------------------------------------------
# Structured hexahedral boxes stored as unstructured face lists
# ---------------------------------------------------------------------------

_SIDES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")


def hex_box(nx: int, ny: int, nz: int, L=(1.0, 1.0, 1.0), side_patch=None,
            patch_specs=None) -> Mesh:
    """Uniform ``nx*ny*nz`` hexahedral mesh of the box ``[0,Lx]x[0,Ly]x[0,Lz]``.

    ``side_patch`` maps each of the six sides (``xmin`` ... ``zmax``) to a patch
    name; ``patch_specs`` maps each patch name to ``(type, u, p)``.  Patches are
    emitted in the order of first appearance in ``patch_specs``.  Cell
    ``(i, j, k)`` gets index ``i + nx*(j + ny*k)``.
    """
    Lx, Ly, Lz = (float(v) for v in L)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    N = nx * ny * nz
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cid = lambda i, j, k: (i + nx * (j + ny * k)).astype(np.int64)

    C = np.zeros((3, N))
    idx = cid(ii, jj, kk).ravel()
    C[0, idx] = (ii.ravel() + 0.5) * hx
    C[1, idx] = (jj.ravel() + 0.5) * hy
    C[2, idx] = (kk.ravel() + 0.5) * hz
    V = np.full(N, hx * hy * hz)

    own, nei, S, Cf = [], [], [], []
    # internal x-faces
    i, j, k = np.meshgrid(np.arange(nx - 1), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    own.append(cid(i, j, k)); nei.append(cid(i + 1, j, k))
    S.append(np.stack([np.full(i.size, hy * hz), np.zeros(i.size), np.zeros(i.size)]))
    Cf.append(np.stack([(i + 1) * hx, (j + 0.5) * hy, (k + 0.5) * hz]))
    # internal y-faces
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny - 1), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    own.append(cid(i, j, k)); nei.append(cid(i, j + 1, k))
    S.append(np.stack([np.zeros(i.size), np.full(i.size, hx * hz), np.zeros(i.size)]))
    Cf.append(np.stack([(i + 0.5) * hx, (j + 1) * hy, (k + 0.5) * hz]))
    # internal z-faces
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz - 1), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    own.append(cid(i, j, k)); nei.append(cid(i, j, k + 1))
    S.append(np.stack([np.zeros(i.size), np.zeros(i.size), np.full(i.size, hx * hy)]))
    Cf.append(np.stack([(i + 0.5) * hx, (j + 0.5) * hy, (k + 1) * hz]))
    F = sum(a.size for a in own)

    # boundary faces of each side
    def side_faces(side):
        if side in ("xmin", "xmax"):
            j, k = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
            j, k = j.ravel(), k.ravel()
            i = np.zeros_like(j) if side == "xmin" else np.full_like(j, nx - 1)
            s = -1.0 if side == "xmin" else 1.0
            xf = 0.0 if side == "xmin" else Lx
            area = np.stack([np.full(j.size, s * hy * hz), np.zeros(j.size), np.zeros(j.size)])
            cf = np.stack([np.full(j.size, xf), (j + 0.5) * hy, (k + 0.5) * hz])
        elif side in ("ymin", "ymax"):
            i, k = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
            i, k = i.ravel(), k.ravel()
            j = np.zeros_like(i) if side == "ymin" else np.full_like(i, ny - 1)
            s = -1.0 if side == "ymin" else 1.0
            yf = 0.0 if side == "ymin" else Ly
            area = np.stack([np.zeros(i.size), np.full(i.size, s * hx * hz), np.zeros(i.size)])
            cf = np.stack([(i + 0.5) * hx, np.full(i.size, yf), (k + 0.5) * hz])
        else:
            i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
            i, j = i.ravel(), j.ravel()
            k = np.zeros_like(i) if side == "zmin" else np.full_like(i, nz - 1)
            s = -1.0 if side == "zmin" else 1.0
            zf = 0.0 if side == "zmin" else Lz
            area = np.stack([np.zeros(i.size), np.zeros(i.size), np.full(i.size, s * hx * hy)])
            cf = np.stack([(i + 0.5) * hx, (j + 0.5) * hy, np.full(i.size, zf)])
        return cid(i, j, k), area, cf

    if side_patch is None:
        side_patch = {s: "walls" for s in _SIDES}
    if patch_specs is None:
        patch_specs = {"walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    patches = []
    start = 0
    for pname, (ptype, pu, pp) in patch_specs.items():
        size = 0
        for side in _SIDES:
            if side_patch[side] != pname:
                continue
            o, a, cf = side_faces(side)
            own.append(o); S.append(a); Cf.append(cf)
            size += o.size
        patches.append(Patch(pname, int(ptype), start, size, tuple(float(x) for x in pu), float(pp)))
        start += size
    B = start
    owner = np.concatenate(own).astype(np.int32)
    neighbour = np.concatenate(nei).astype(np.int32)
    assert owner.size == F + B and neighbour.size == F
    return Mesh(N, F, B, owner, neighbour, np.concatenate(S, axis=1),
                np.concatenate(Cf, axis=1), C, V, patches, corner_cell=0)


def geometric_nodes(n: int, L: float = 1.0, ratio: float = 1.0) -> np.ndarray:
    """``n + 1`` node coordinates on ``[0, L]`` whose spacings grow by
    ``ratio`` from one cell to the next (``h_{i+1} = ratio * h_i``)."""
    h = ratio ** np.arange(n, dtype=np.float64)
    x = np.concatenate([[0.0], np.cumsum(h)])
    x *= L / x[-1]
    x[-1] = L
    return x


def graded_box(xs, ys, zs, side_patch=None, patch_specs=None) -> Mesh:
    """Orthogonal hexahedral mesh on the tensor grid of node coordinates
    ``xs``, ``ys``, ``zs`` (strictly increasing; cell sizes may differ from
    cell to cell).  Cell ``(i, j, k)`` gets index ``i + nx*(j + ny*k)``; its
    centroid is the midpoint of its node intervals, face centres are the
    midpoints of the faces.  On such a mesh the face between two cells is
    generally not half-way between their centroids, which is what makes the
    interpolation weight of a face differ from 1/2.  Patch arguments as
    :func:`hex_box`."""
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    for a in (xs, ys, zs):
        assert a.ndim == 1 and a.size >= 2 and (np.diff(a) > 0).all()
    nx, ny, nz = xs.size - 1, ys.size - 1, zs.size - 1
    hx, hy, hz = np.diff(xs), np.diff(ys), np.diff(zs)
    cx, cy, cz = 0.5 * (xs[:-1] + xs[1:]), 0.5 * (ys[:-1] + ys[1:]), 0.5 * (zs[:-1] + zs[1:])
    N = nx * ny * nz
    cid = lambda i, j, k: (i + nx * (j + ny * k)).astype(np.int64)
    ii, jj, kk = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                                                  indexing="ij"))
    idx = cid(ii, jj, kk)
    C = np.zeros((3, N))
    C[0, idx], C[1, idx], C[2, idx] = cx[ii], cy[jj], cz[kk]
    V = np.zeros(N)
    V[idx] = hx[ii] * hy[jj] * hz[kk]

    own, nei, S, Cf = [], [], [], []
    z0 = lambda n: np.zeros(n)
    i, j, k = (a.ravel() for a in np.meshgrid(np.arange(nx - 1), np.arange(ny), np.arange(nz),
                                               indexing="ij"))
    own.append(cid(i, j, k)); nei.append(cid(i + 1, j, k))
    S.append(np.stack([hy[j] * hz[k], z0(i.size), z0(i.size)]))
    Cf.append(np.stack([xs[i + 1], cy[j], cz[k]]))
    i, j, k = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(ny - 1), np.arange(nz),
                                               indexing="ij"))
    own.append(cid(i, j, k)); nei.append(cid(i, j + 1, k))
    S.append(np.stack([z0(i.size), hx[i] * hz[k], z0(i.size)]))
    Cf.append(np.stack([cx[i], ys[j + 1], cz[k]]))
    i, j, k = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz - 1),
                                               indexing="ij"))
    own.append(cid(i, j, k)); nei.append(cid(i, j, k + 1))
    S.append(np.stack([z0(i.size), z0(i.size), hx[i] * hy[j]]))
    Cf.append(np.stack([cx[i], cy[j], zs[k + 1]]))
    F = sum(a.size for a in own)

    def side_faces(side):
        if side in ("xmin", "xmax"):
            j, k = (a.ravel() for a in np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij"))
            lo = side == "xmin"
            i = np.full_like(j, 0 if lo else nx - 1)
            area = np.stack([(-1.0 if lo else 1.0) * hy[j] * hz[k], z0(j.size), z0(j.size)])
            cf = np.stack([np.full(j.size, xs[0] if lo else xs[-1]), cy[j], cz[k]])
        elif side in ("ymin", "ymax"):
            i, k = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij"))
            lo = side == "ymin"
            j = np.full_like(i, 0 if lo else ny - 1)
            area = np.stack([z0(i.size), (-1.0 if lo else 1.0) * hx[i] * hz[k], z0(i.size)])
            cf = np.stack([cx[i], np.full(i.size, ys[0] if lo else ys[-1]), cz[k]])
        else:
            i, j = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij"))
            lo = side == "zmin"
            k = np.full_like(i, 0 if lo else nz - 1)
            area = np.stack([z0(i.size), z0(i.size), (-1.0 if lo else 1.0) * hx[i] * hy[j]])
            cf = np.stack([cx[i], cy[j], np.full(i.size, zs[0] if lo else zs[-1])])
        return cid(i, j, k), area, cf

    if side_patch is None:
        side_patch = {s: "walls" for s in _SIDES}
    if patch_specs is None:
        patch_specs = {"walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    patches, start = [], 0
    for pname, (ptype, pu, pp) in patch_specs.items():
        size = 0
        for side in _SIDES:
            if side_patch[side] != pname:
                continue
            o, a, cf = side_faces(side)
            own.append(o); S.append(a); Cf.append(cf)
            size += o.size
        patches.append(Patch(pname, int(ptype), start, size, tuple(float(x) for x in pu), float(pp)))
        start += size
    owner = np.concatenate(own).astype(np.int32)
    neighbour = np.concatenate(nei).astype(np.int32)
    assert owner.size == F + start and neighbour.size == F
    return Mesh(N, F, start, owner, neighbour, np.concatenate(S, axis=1),
                np.concatenate(Cf, axis=1), C, V, patches, corner_cell=0)


def graded_cavity3d(n: int, ratio: float = 1.3, u_lid: float = 1.0, L: float = 1.0) -> Mesh:
    """The 3-D lid-driven cavity of :func:`cavity3d` on a graded mesh: the
    cell sizes grow by ``ratio`` from cell to cell along every axis."""
    x = geometric_nodes(n, L, ratio)
    sp = {s: "fixedWalls" for s in _SIDES}
    sp["ymax"] = "movingWall"
    specs = {"movingWall": (WALL, (u_lid, 0.0, 0.0), 0.0),
             "fixedWalls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return graded_box(x, x, x, sp, specs)


def cavity3d(n: int, u_lid: float = 1.0, L: float = 1.0) -> Mesh:
    """3-D lid-driven cavity on the cube ``[0,L]^3`` with ``n^3`` hexahedra.

    The lid is the ``y = L`` side moving with ``(u_lid, 0, 0)``; the five other
    sides are fixed no-slip walls (the cavity of the paper's Sec. 4.1)."""
    sp = {s: "fixedWalls" for s in _SIDES}
    sp["ymax"] = "movingWall"
    specs = {"movingWall": (WALL, (u_lid, 0.0, 0.0), 0.0),
             "fixedWalls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return hex_box(n, n, n, (L, L, L), sp, specs)


def cavity2d(nx: int, ny: int = None, u_lid: float = 1.0, L: float = 1.0) -> Mesh:
    """2-D lid-driven cavity: ``nx*ny*1`` hexahedra with empty front/back."""
    ny = nx if ny is None else ny
    sp = {"xmin": "fixedWalls", "xmax": "fixedWalls", "ymin": "fixedWalls",
          "ymax": "movingWall", "zmin": "frontAndBack", "zmax": "frontAndBack"}
    specs = {"movingWall": (WALL, (u_lid, 0.0, 0.0), 0.0),
             "fixedWalls": (WALL, (0.0, 0.0, 0.0), 0.0),
             "frontAndBack": (EMPTY, (0.0, 0.0, 0.0), 0.0)}
    return hex_box(nx, ny, 1, (L, L * ny / nx, L / nx), sp, specs)


def channel2d(nx: int, ny: int, Lx: float, Ly: float, inlet_u=(1.0, 0.0, 0.0),
              top_u=(0.0, 0.0, 0.0)) -> Mesh:
    """2-D channel ``[0,Lx]x[0,Ly]``: inlet at ``x=0``, outlet (p = 0) at
    ``x=Lx``, no-slip bottom wall, top wall moving with ``top_u``."""
    sp = {"xmin": "inlet", "xmax": "outlet", "ymin": "bottom", "ymax": "top",
          "zmin": "frontAndBack", "zmax": "frontAndBack"}
    specs = {"inlet": (INLET, inlet_u, 0.0), "outlet": (OUTLET, (0.0, 0.0, 0.0), 0.0),
             "bottom": (WALL, (0.0, 0.0, 0.0), 0.0), "top": (WALL, top_u, 0.0),
             "frontAndBack": (EMPTY, (0.0, 0.0, 0.0), 0.0)}
    return hex_box(nx, ny, 1, (Lx, Ly, min(Lx / nx, Ly / ny)), sp, specs)


# Transient Poiseuille flow (the paper's "tp1M" case, Sec. 4.1): a 2-D pipe
# 0.16 m long and 0.02 m high, 3200 x 300 cells, nu = 3.3e-6 m^2/s, uniform
# inlet velocity u0 sin(2 pi f t) with u0 = 0.01 m/s and f = 0.5 1/s, p = 0
# at the outlet, 5000 PISO steps of 0.1 ms.
TP1M = {"L": 0.16, "H": 0.02, "nx": 3200, "ny": 300, "nu": 3.3e-6, "u0": 0.01, "f": 0.5,
        "dt": 1e-4, "steps": 5000}


def tp_channel(nx: int = 3200, ny: int = 300, L: float = 0.16, H: float = 0.02) -> Mesh:
    """The transient-Poiseuille pipe (inlet at x = 0, outlet at x = L, no-slip
    walls at y = 0 and y = H); the inlet starts at rest."""
    return channel2d(nx, ny, L, H, inlet_u=(0.0, 0.0, 0.0))


def tp_inlet(t: float, u0: float = 0.01, f: float = 0.5) -> tuple:
    """Inlet velocity of the transient-Poiseuille case at time t."""
    return (u0 * float(np.sin(2.0 * np.pi * f * t)), 0.0, 0.0)


# ---------------------------------------------------------------------------
# Cell relabelling
# ---------------------------------------------------------------------------

def permute_cells(mesh: Mesh, new_of_old: np.ndarray) -> Mesh:
    """Relabel cells: old cell ``c`` becomes ``new_of_old[c]``.  Faces keep
    their order and orientation (so owner may exceed neighbour afterwards)."""
    new_of_old = np.asarray(new_of_old, dtype=np.int64)
    N = mesh.n_cells
    assert new_of_old.shape == (N,) and np.array_equal(np.sort(new_of_old), np.arange(N))
    m = mesh.copy()
    m.owner = new_of_old[mesh.owner].astype(np.int32)
    m.neighbour = new_of_old[mesh.neighbour].astype(np.int32)
    m.C = np.empty_like(mesh.C)
    m.C[:, new_of_old] = mesh.C
    m.V = np.empty_like(mesh.V)
    m.V[new_of_old] = mesh.V
    m.corner_cell = int(new_of_old[mesh.corner_cell])
    return m


def random_permutation(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).permutation(n)


# ---------------------------------------------------------------------------
# Kuhn (Freudenthal) tetrahedral split of a hex box, with node jitter
# ---------------------------------------------------------------------------

def _tri_area_vec(a, b, c):
    return 0.5 * np.cross(b - a, c - a, axis=0)


def tet_box(nx: int, ny: int, nz: int, L=(1.0, 1.0, 1.0), jitter: float = 0.0,
            seed: int = 2024, side_patch=None, patch_specs=None) -> Mesh:
    """Split every hexahedron of an ``nx*ny*nz`` box into the six Kuhn
    tetrahedra along its ``(0,0,0)->(1,1,1)`` diagonal (conforming).  Interior
    nodes are moved by ``U(-jitter*h, +jitter*h)`` per coordinate
    (``numpy.random.default_rng(seed)``); boundary nodes stay, so boundary
    faces remain planar.  Tet centroid = vertex mean, face centre = triangle
    centroid, ``S = (b-a)x(c-a)/2`` oriented out of the owner."""
    Lx, Ly, Lz = (float(v) for v in L)
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    I, J, K = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    nid = lambda i, j, k: i + NX * (j + NY * k)
    X = np.zeros((3, NX * NY * NZ))
    X[0, nid(I, J, K)] = I * h[0]
    X[1, nid(I, J, K)] = J * h[1]
    X[2, nid(I, J, K)] = K * h[2]
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=(3, X.shape[1])) * h[:, None]
        interior = (I > 0) & (I < nx) & (J > 0) & (J < ny) & (K > 0) & (K < nz)
        X[:, nid(I, J, K)[interior]] += d[:, nid(I, J, K)[interior]]

    # hexes
    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    nhex = hi.size
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = np.empty((nhex * 6, 4), dtype=np.int64)
    for t, pm in enumerate(perms):
        off = [np.zeros(nhex, np.int64)] * 3
        cur = [hi.copy(), hj.copy(), hk.copy()]
        verts = [nid(*cur)]
        for ax in pm:
            cur[ax] = cur[ax] + 1
            verts.append(nid(*cur))
        tets[t::6] = np.stack(verts, axis=1)      # hex h -> tets 6h .. 6h+5
    N = tets.shape[0]
    C = X[:, tets].mean(axis=2)
    a, b, c, d = (X[:, tets[:, m]] for m in range(4))
    V = np.abs(np.einsum("ij,ij->j", b - a, np.cross(c - a, d - a, axis=0))) / 6.0

    # faces: (sorted node triple) -> cells
    faces_nodes = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                                  tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0)
    faces_cell = np.concatenate([np.arange(N)] * 4)
    fs = np.sort(faces_nodes, axis=1)
    nn = X.shape[1]
    key = (fs[:, 0] * nn + fs[:, 1]) * nn + fs[:, 2]
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    same = np.zeros(key_s.size, bool)
    same[1:] = key_s[1:] == key_s[:-1]
    # internal faces: positions where same[i] is True -> (order[i-1], order[i])
    pos = np.nonzero(same)[0]
    a_idx, b_idx = order[pos - 1], order[pos]
    own_i = faces_cell[a_idx]; nei_i = faces_cell[b_idx]
    tri_i = fs[a_idx]
    single = np.ones(key_s.size, bool)
    single[pos] = False; single[pos - 1] = False
    bidx = order[single]
    own_b = faces_cell[bidx]; tri_b = fs[bidx]

    def geom(tri, ocell):
        pa, pb, pc = X[:, tri[:, 0]], X[:, tri[:, 1]], X[:, tri[:, 2]]
        S = _tri_area_vec(pa, pb, pc)
        cf = (pa + pb + pc) / 3.0
        sgn = np.sign(np.einsum("ij,ij->j", S, cf - C[:, ocell]))
        return S * sgn, cf

    Si, Cfi = geom(tri_i, own_i)
    Sb, Cfb = geom(tri_b, own_b)
    # classify boundary faces by side
    tol = 1e-9 * max(Lx, Ly, Lz)
    side = np.full(own_b.size, -1)
    for s_id, (ax, val) in enumerate([(0, 0.0), (0, Lx), (1, 0.0), (1, Ly), (2, 0.0), (2, Lz)]):
        side[np.abs(Cfb[ax] - val) < tol] = s_id
    assert (side >= 0).all()
    if side_patch is None:
        side_patch = {s: "walls" for s in _SIDES}
    if patch_specs is None:
        patch_specs = {"walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    b_order, patches, start = [], [], 0
    for pname, (ptype, pu, pp) in patch_specs.items():
        sel = np.concatenate([np.nonzero(side == s_id)[0] for s_id, s in enumerate(_SIDES)
                              if side_patch[s] == pname])
        b_order.append(sel)
        patches.append(Patch(pname, int(ptype), start, sel.size, tuple(float(x) for x in pu), float(pp)))
        start += sel.size
    b_order = np.concatenate(b_order)
    owner = np.concatenate([own_i, own_b[b_order]]).astype(np.int32)
    Sf = np.concatenate([Si, Sb[:, b_order]], axis=1)
    Cf = np.concatenate([Cfi, Cfb[:, b_order]], axis=1)
    return Mesh(N, own_i.size, b_order.size, owner, nei_i.astype(np.int32), Sf, Cf, C, V,
                patches, corner_cell=0)


def duct_tets(n: int = 48, length_cells: int = 192, jitter: float = 0.1, seed: int = 2024) -> Mesh:
    """Square duct ``[0,1]^2 x [0, length_cells/n]`` of jittered Kuhn tets,
    flow along ``+z``: inlet ``z = 0`` (fixed velocity, its profile set per
    face by :func:`duct_inlet_profile`), outlet ``z = Lz`` (``p = 0``), four
    no-slip walls."""
    Lz = length_cells / n
    sp = {"xmin": "walls", "xmax": "walls", "ymin": "walls", "ymax": "walls",
          "zmin": "inlet", "zmax": "outlet"}
    specs = {"inlet": (INLET, (0.0, 0.0, 1.0), 0.0), "outlet": (OUTLET, (0.0, 0.0, 0.0), 0.0),
             "walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return tet_box(n, n, length_cells, (1.0, 1.0, Lz), jitter, seed, sp, specs)


def duct_hex(n: int, length_cells: int) -> Mesh:
    """Hexahedral version of :func:`duct_tets` (orthogonal)."""
    Lz = length_cells / n
    sp = {"xmin": "walls", "xmax": "walls", "ymin": "walls", "ymax": "walls",
          "zmin": "inlet", "zmax": "outlet"}
    specs = {"inlet": (INLET, (0.0, 0.0, 1.0), 0.0), "outlet": (OUTLET, (0.0, 0.0, 0.0), 0.0),
             "walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return hex_box(n, n, length_cells, (1.0, 1.0, Lz), sp, specs)


def duct_inlet_profile(Cf_xy: np.ndarray) -> np.ndarray:
    """Parabolic inlet ``u_z = 36 x(1-x) y(1-y)`` (mean 1 over the unit
    square) evaluated at face centres ``(2, n)``."""
    x, y = Cf_xy
    return 36.0 * x * (1.0 - x) * y * (1.0 - y)


# ---------------------------------------------------------------------------
# Mixed-element meshes: hexahedra, triangular prisms and pyramids
# ---------------------------------------------------------------------------

def polyhedral_mesh(X, cells, L, side_patch=None, patch_specs=None) -> Mesh:
    """Face-addressed mesh of polyhedral cells.  ``X`` (3, n_nodes) node
    coordinates; ``cells`` a list of cells, each a list of faces, each face a
    list of node indices in cyclic order (either orientation).  Faces shared
    by two cells become internal faces (owner = the cell listed first),
    the others boundary faces, assigned to the box sides of ``[0,L]``
    (``hex_box`` patch arguments).

    Geometry of possibly non-planar faces and of the cells, by the usual
    decomposition: a face is split into triangles around the mean of its
    nodes; its area vector is the sum of theirs and its centre their
    area-weighted centroid.  A cell is split into the tetrahedra spanned by
    the mean of its nodes and those face triangles; its volume and centroid
    are theirs summed and volume-averaged.  Area vectors point out of the
    owner."""
    X = np.asarray(X, dtype=np.float64)
    Lx, Ly, Lz = (float(v) for v in L)

    def face_geom(nodes):
        P = X[:, nodes]
        xc = P.mean(axis=1)
        Pn = np.roll(P, -1, axis=1)
        s = 0.5 * np.cross(Pn - P, xc[:, None] - P, axis=0)
        c = (P + Pn + xc[:, None]) / 3.0
        a = np.linalg.norm(s, axis=0)
        return s.sum(axis=1), (c * a).sum(axis=1) / a.sum(), s, c

    keys = {}
    faces = []          # [nodes, owner, neighbour]
    for ci, cf in enumerate(cells):
        for nodes in cf:
            k = tuple(sorted(nodes))
            if k in keys:
                f = faces[keys[k]]
                assert f[2] < 0, "a face shared by more than two cells"
                f[2] = ci
            else:
                keys[k] = len(faces)
                faces.append([list(nodes), ci, -1])
    geo = [face_geom(f[0]) for f in faces]
    N = len(cells)
    C = np.zeros((3, N))
    V = np.zeros(N)
    for ci, cf in enumerate(cells):
        x0 = X[:, sorted({n for nodes in cf for n in nodes})].mean(axis=1)
        vol, mom = 0.0, np.zeros(3)
        for nodes in cf:
            S, Cf, s, c = geo[keys[tuple(sorted(nodes))]]
            sgn = 1.0 if S @ (Cf - x0) > 0 else -1.0
            v = sgn * np.einsum("ij,ij->j", s, c - x0[:, None]) / 3.0
            vol += v.sum()
            mom += ((0.25 * x0[:, None] + 0.75 * c) * v).sum(axis=1)
        V[ci] = vol
        C[:, ci] = mom / vol
    internal = [f for f in range(len(faces)) if faces[f][2] >= 0]
    bnd = [f for f in range(len(faces)) if faces[f][2] < 0]

    def oriented(f):
        S, Cf = geo[f][0], geo[f][1]
        o = faces[f][1]
        return (S if S @ (Cf - C[:, o]) > 0 else -S), Cf

    Si = np.array([oriented(f)[0] for f in internal]).T.reshape(3, -1)
    Cfi = np.array([geo[f][1] for f in internal]).T.reshape(3, -1)
    own_i = np.array([faces[f][1] for f in internal], np.int32)
    nei_i = np.array([faces[f][2] for f in internal], np.int32)
    Sb = np.array([oriented(f)[0] for f in bnd]).T.reshape(3, -1)
    Cfb = np.array([geo[f][1] for f in bnd]).T.reshape(3, -1)
    own_b = np.array([faces[f][1] for f in bnd], np.int32)
    tol = 1e-9 * max(Lx, Ly, Lz)
    side = np.full(len(bnd), -1)
    for s_id, (ax, val) in enumerate([(0, 0.0), (0, Lx), (1, 0.0), (1, Ly), (2, 0.0), (2, Lz)]):
        side[np.abs(Cfb[ax] - val) < tol] = s_id
    assert (side >= 0).all()
    if side_patch is None:
        side_patch = {s: "walls" for s in _SIDES}
    if patch_specs is None:
        patch_specs = {"walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    b_order, patches, start = [], [], 0
    for pname, (ptype, pu, pp) in patch_specs.items():
        sel = np.concatenate([np.nonzero(side == s_id)[0] for s_id, s in enumerate(_SIDES)
                              if side_patch[s] == pname]).astype(np.int64)
        b_order.append(sel)
        patches.append(Patch(pname, int(ptype), start, sel.size, tuple(float(x) for x in pu), float(pp)))
        start += sel.size
    b_order = np.concatenate(b_order)
    owner = np.concatenate([own_i, own_b[b_order]]).astype(np.int32)
    Sf = np.concatenate([Si, Sb[:, b_order]], axis=1)
    Cf = np.concatenate([Cfi, Cfb[:, b_order]], axis=1)
    return Mesh(N, own_i.size, b_order.size, owner, nei_i, Sf, Cf, C, V, patches, corner_cell=0)


def mixed_box(nx: int, ny: int, nz: int, L=(1.0, 1.0, 1.0), jitter: float = 0.0,
              seed: int = 2024, prism_every: int = 3, pyramid_every: int = 4,
              side_patch=None, patch_specs=None) -> Mesh:
    """A conforming mixed-element mesh of the box ``[0,L]``: an ``nx*ny*nz``
    hexahedral grid in which

    * every hexahedron of the columns with ``(i + j) % prism_every == 0`` is
      split into two triangular prisms by the vertical plane through its
      (i, j) -> (i+1, j+1) diagonal (the whole column the same way, so the
      prism caps match);
    * outside those columns, every hexahedron with
      ``(i + j + k) % pyramid_every == 1`` is split into six pyramids, one
      on each of its faces, with their apex at a node added at its centre;
    * the other cells stay hexahedra.

    Interior nodes (grid nodes off the boundary and the added centre nodes)
    are moved by ``U(-jitter*h, +jitter*h)`` per coordinate
    (``numpy.random.default_rng(seed)``), so faces become non-planar and
    the mesh non-orthogonal; boundary nodes stay, so the boundary stays
    planar.  Cell (i, j, k)'s pieces are numbered in grid order."""
    Lx, Ly, Lz = (float(v) for v in L)
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    nid = lambda i, j, k: i + NX * (j + NY * k)
    I, J, K = (a.ravel() for a in np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ),
                                               indexing="ij"))
    ng = NX * NY * NZ
    Xg = np.zeros((3, ng))
    Xg[0, nid(I, J, K)] = I * h[0]
    Xg[1, nid(I, J, K)] = J * h[1]
    Xg[2, nid(I, J, K)] = K * h[2]
    interior = np.zeros(ng, bool)
    interior[nid(I, J, K)] = (I > 0) & (I < nx) & (J > 0) & (J < ny) & (K > 0) & (K < nz)
    pyr = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if (i + j) % prism_every != 0 and (i + j + k) % pyramid_every == 1:
                    pyr.append((i, j, k))
    centre = {c: ng + q for q, c in enumerate(pyr)}
    X = np.zeros((3, ng + len(pyr)))
    X[:, :ng] = Xg
    for (i, j, k), q in centre.items():
        X[:, q] = (np.array([i, j, k]) + 0.5) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=X.shape) * h[:, None]
        movable = np.concatenate([interior, np.ones(len(pyr), bool)])
        X[:, movable] += d[:, movable]

    cells = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                n = {(a, b, c): nid(i + a, j + b, k + c) for a in (0, 1) for b in (0, 1)
                     for c in (0, 1)}
                quads = [[n[0, 0, 0], n[0, 1, 0], n[0, 1, 1], n[0, 0, 1]],
                         [n[1, 0, 0], n[1, 0, 1], n[1, 1, 1], n[1, 1, 0]],
                         [n[0, 0, 0], n[0, 0, 1], n[1, 0, 1], n[1, 0, 0]],
                         [n[0, 1, 0], n[1, 1, 0], n[1, 1, 1], n[0, 1, 1]],
                         [n[0, 0, 0], n[1, 0, 0], n[1, 1, 0], n[0, 1, 0]],
                         [n[0, 0, 1], n[0, 1, 1], n[1, 1, 1], n[1, 0, 1]]]
                if (i + j) % prism_every == 0:
                    diag = [n[0, 0, 0], n[1, 1, 0], n[1, 1, 1], n[0, 0, 1]]
                    cells.append([[n[0, 0, 0], n[1, 0, 0], n[1, 1, 0]],
                                  [n[0, 0, 1], n[1, 0, 1], n[1, 1, 1]], quads[2], quads[1], diag])
                    cells.append([[n[0, 0, 0], n[1, 1, 0], n[0, 1, 0]],
                                  [n[0, 0, 1], n[1, 1, 1], n[0, 1, 1]], quads[0], quads[3], diag])
                elif (i, j, k) in centre:
                    c = centre[(i, j, k)]
                    for q in quads:
                        cells.append([q] + [[q[t], q[(t + 1) % 4], c] for t in range(4)])
                else:
                    cells.append(quads)
    return polyhedral_mesh(X, cells, (Lx, Ly, Lz), side_patch, patch_specs)


def mixed_cavity3d(n: int, jitter: float = 0.0, seed: int = 2024) -> Mesh:
    """The 3-D lid-driven cavity of :func:`cavity3d` on a :func:`mixed_box`
    mesh of the unit cube."""
    sp = {s: "fixedWalls" for s in _SIDES}
    sp["ymax"] = "movingWall"
    specs = {"movingWall": (WALL, (1.0, 0.0, 0.0), 0.0),
             "fixedWalls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return mixed_box(n, n, n, (1.0, 1.0, 1.0), jitter, seed, side_patch=sp, patch_specs=specs)


def mixed_duct(n: int, length_cells: int, jitter: float = 0.0, seed: int = 2024) -> Mesh:
    """The square duct of :func:`duct_hex` on a :func:`mixed_box` mesh: inlet
    ``z = 0``, outlet ``z = Lz`` (p = 0), four no-slip walls."""
    Lz = length_cells / n
    sp = {"xmin": "walls", "xmax": "walls", "ymin": "walls", "ymax": "walls",
          "zmin": "inlet", "zmax": "outlet"}
    specs = {"inlet": (INLET, (0.0, 0.0, 1.0), 0.0), "outlet": (OUTLET, (0.0, 0.0, 0.0), 0.0),
             "walls": (WALL, (0.0, 0.0, 0.0), 0.0)}
    return mixed_box(n, n, length_cells, (1.0, 1.0, Lz), jitter, seed, side_patch=sp,
                     patch_specs=specs)


# ---------------------------------------------------------------------------
# Batch sampler (256 uneven 2-D cavities)
# ---------------------------------------------------------------------------

def batch_cases(n_cases: int = 256, seed: int = 7, n_lo: int = 32, n_hi: int = 128,
                re_lo: float = 10.0, re_hi: float = 1000.0):
    """``n_i ~ integers(n_lo, n_hi+1)`` and ``Re_i ~ exp(U(ln re_lo, ln re_hi))``
    drawn from ``numpy.random.default_rng(seed)``; returns ``[(n_i, nu_i)]``
    with ``nu_i = 1/Re_i`` (lid speed 1, unit square)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(n_lo, n_hi + 1, size=n_cases)
    re = np.exp(rng.uniform(math.log(re_lo), math.log(re_hi), size=n_cases))
    return [(int(a), float(1.0 / b)) for a, b in zip(n, re)]


# ---------------------------------------------------------------------------
# Small helpers shared by tests and the benchmark (no discretisation here)
# ---------------------------------------------------------------------------

def table1_face_count(n: int) -> int:
    """Faces of a structured n^3 cube including the boundary: 3 n^2 (n+1)."""
    return 3 * n * n * (n + 1)


def structured_seeded_field(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return scale * np.random.default_rng(seed).standard_normal(n)
