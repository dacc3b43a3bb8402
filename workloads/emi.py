"""Cell-by-cell (EMI) meshes: brick myocytes in an extracellular bath.

A voxel grid is labelled 0 (extracellular space) or c >= 1 (cell c).  Every
voxel is split into the six Kuhn tetrahedra; a tetrahedron belongs to its
voxel's subdomain.  Each grid vertex carries one dof per distinct label of the
voxels around it, so the potentials are discontinuous across membranes.

Membranes are the voxel faces between different labels.  A face of area h^2
gives each of its four vertices a quarter of its area, accumulated per pair of
dofs (the two sides of the membrane at that vertex): the lumped membrane
measure of the pair.  Cell-ECS pairs (kind 0) carry the Aliev-Panfilov
current and a gating variable; cell-cell pairs (kind 1) are gap junctions
with a linear current.  The pair is oriented (k, l) = (cell side, ECS side)
for kind 0 and (lower cell, higher cell) for kind 1, so v = u_k - u_l is the
transmembrane voltage.  Outer box faces give their vertices' dofs a lumped
boundary measure for the Robin term.

No arithmetic of the method is done here.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

from .configs import AP_BENCH, SEED_BASE
from .meshes import Mesh

_PERMS = list(permutations(range(3)))


@dataclass
class EmiWorkload:
    name: str
    mesh: Mesh                     # elements on the dof numbering, per-element tensors
    pair_k: np.ndarray
    pair_l: np.ndarray
    pair_area: np.ndarray
    pair_kind: np.ndarray          # 0 membrane (ionic + gating), 1 gap junction
    robin_area: np.ndarray         # per dof lumped boundary measure
    labels: np.ndarray             # per dof subdomain label
    ionic: dict
    M: int
    dt: float
    sweeps: int
    tol: float
    steps: int
    u0: np.ndarray
    w0: np.ndarray                 # per pair
    robin_eps: float = 0.0
    Cm: float = 1.0
    g_gap: float = 0.0
    sigma_i: float = 1.0
    sigma_e: float = 1.0
    cg_rtol: float = 1e-10
    alpha: float = 0.1
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.mesh.n_nodes

    @property
    def n_pairs(self) -> int:
        return int(self.pair_k.size)

    @property
    def robin(self) -> np.ndarray:
        return self.robin_eps * self.robin_area


def emi_from_labels(lab: np.ndarray, h: float, sigma_i: float, sigma_e: float):
    """Dofs, tetrahedra, membrane pairs and Robin areas of a labelled voxel grid."""
    nx, ny, nz = lab.shape
    vx, vy, vz = nx + 1, ny + 1, nz + 1

    def vid(i, j, k):
        return i + vx * (j + vy * k)

    nvert = vx * vy * vz
    # labels around each vertex
    vlabels = [set() for _ in range(nvert)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = int(lab[i, j, k])
                for dk in (0, 1):
                    for dj in (0, 1):
                        for di in (0, 1):
                            vlabels[vid(i + di, j + dj, k + dk)].add(c)
    dof = {}
    xyz, dlab = [], []
    for k in range(vz):
        for j in range(vy):
            for i in range(vx):
                v = vid(i, j, k)
                for c in sorted(vlabels[v]):
                    dof[(v, c)] = len(xyz)
                    xyz.append((i * h, j * h, k * h))
                    dlab.append(c)
    xyz = np.array(xyz, dtype=np.float64)
    dlab = np.array(dlab, dtype=np.int32)
    elems, esig = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = int(lab[i, j, k])
                s = sigma_e if c == 0 else sigma_i
                for perm in _PERMS:
                    off = [0, 0, 0]
                    vs = []
                    for step in range(4):
                        if step > 0:
                            off[perm[step - 1]] += 1
                        vs.append(dof[(vid(i + off[0], j + off[1], k + off[2]), c)])
                    elems.append(vs)
                    esig.append(s * np.eye(3))
    elems = np.array(elems, dtype=np.int32)
    esig = np.array(esig, dtype=np.float64)
    # membrane faces between voxels of different labels
    quarter = h * h / 4.0
    acc = {}

    def add_face(verts, ca, cb):
        if ca == cb:
            return
        if ca == 0 or cb == 0:
            cell, ecs = (ca, cb) if cb == 0 else (cb, ca)
            kind = 0
            first, second = cell, ecs
        else:
            kind = 1
            first, second = min(ca, cb), max(ca, cb)
        for v in verts:
            key = (dof[(v, first)], dof[(v, second)], kind)
            acc[key] = acc.get(key, 0.0) + quarter

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = int(lab[i, j, k])
                if i + 1 < nx:
                    add_face([vid(i + 1, j, k), vid(i + 1, j + 1, k), vid(i + 1, j, k + 1),
                              vid(i + 1, j + 1, k + 1)], c, int(lab[i + 1, j, k]))
                if j + 1 < ny:
                    add_face([vid(i, j + 1, k), vid(i + 1, j + 1, k), vid(i, j + 1, k + 1),
                              vid(i + 1, j + 1, k + 1)], c, int(lab[i, j + 1, k]))
                if k + 1 < nz:
                    add_face([vid(i, j, k + 1), vid(i + 1, j, k + 1), vid(i, j + 1, k + 1),
                              vid(i + 1, j + 1, k + 1)], c, int(lab[i, j, k + 1]))
    keys = sorted(acc)
    pk = np.array([key[0] for key in keys], dtype=np.int32)
    pl = np.array([key[1] for key in keys], dtype=np.int32)
    pkind = np.array([key[2] for key in keys], dtype=np.int32)
    parea = np.array([acc[key] for key in keys], dtype=np.float64)
    # outer box faces: Robin measure on the dofs of the boundary voxels' labels
    robin = np.zeros(len(xyz))

    def add_bface(verts, c):
        for v in verts:
            robin[dof[(v, c)]] += quarter

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = int(lab[i, j, k])
                if i == 0:
                    add_bface([vid(0, j, k), vid(0, j + 1, k), vid(0, j, k + 1), vid(0, j + 1, k + 1)], c)
                if i == nx - 1:
                    add_bface([vid(nx, j, k), vid(nx, j + 1, k), vid(nx, j, k + 1),
                               vid(nx, j + 1, k + 1)], c)
                if j == 0:
                    add_bface([vid(i, 0, k), vid(i + 1, 0, k), vid(i, 0, k + 1), vid(i + 1, 0, k + 1)], c)
                if j == ny - 1:
                    add_bface([vid(i, ny, k), vid(i + 1, ny, k), vid(i, ny, k + 1),
                               vid(i + 1, ny, k + 1)], c)
                if k == 0:
                    add_bface([vid(i, j, 0), vid(i + 1, j, 0), vid(i, j + 1, 0), vid(i + 1, j + 1, 0)], c)
                if k == nz - 1:
                    add_bface([vid(i, j, nz), vid(i + 1, j, nz), vid(i, j + 1, nz),
                               vid(i + 1, j + 1, nz)], c)
    mesh = Mesh(3, xyz, elems, elem_sigma=esig, meta={"h": h, "voxels": lab.shape})
    return mesh, pk, pl, parea, pkind, robin, dlab


def brick_labels(cells, cell_vox, gap_vox, margin):
    """Labels of an array of brick cells: cells = (cx, cy, cz) counts, each cell
    cell_vox = (lx, ly, lz) voxels; cells touch end to end along x, lateral
    neighbours are separated by gap_vox voxels of ECS, margin voxels of bath."""
    cx, cy, cz = cells
    lx, ly, lz = cell_vox
    nx = 2 * margin + cx * lx
    ny = 2 * margin + cy * ly + (cy - 1) * gap_vox
    nz = 2 * margin + cz * lz + (cz - 1) * gap_vox
    lab = np.zeros((nx, ny, nz), dtype=np.int32)
    cid = 0
    for kz in range(cz):
        for ky in range(cy):
            for kx in range(cx):
                cid += 1
                x0 = margin + kx * lx
                y0 = margin + ky * (ly + gap_vox)
                z0 = margin + kz * (lz + gap_vox)
                lab[x0:x0 + lx, y0:y0 + ly, z0:z0 + lz] = cid
    return lab


def emi_bricks(cells=(8, 4, 4), cell_um=(100.0, 20.0, 20.0), h=2.0, gap_vox=1, margin=5,
               name=None, dt=0.02, sweeps=4, tol=1e-5, steps=50, w_frozen=False) -> EmiWorkload:
    """Brick myocytes (cell_um each, h-um voxels) in a bath.  Units: um, ms,
    C_m = 1, conductivities divided by C_m: sigma_i = 3e4 um/ms (0.3 S/m),
    sigma_e = 2e5 um/ms (2.0 S/m); gap junctions 5 % of the face at
    1/(R_g C_m) = 222 /ms; Robin coefficient 1e-4 sigma_e / box length.
    The first cell (lowest x, y, z) starts excited (u = 1 inside)."""
    lx, ly, lz = (int(round(c / h)) for c in cell_um)
    lab = brick_labels(cells, (lx, ly, lz), gap_vox, margin)
    sigma_i, sigma_e = 3.0e4, 2.0e5
    mesh, pk, pl, parea, pkind, robin_area, dlab = emi_from_labels(lab, h, sigma_i, sigma_e)
    n = mesh.n_nodes
    u0 = np.where(dlab == 1, 1.0, 0.0)
    box = max(lab.shape) * h
    wl = EmiWorkload(name or "emi_%dx%dx%d_cells_%d_dofs" % (cells + (n,)), mesh, pk, pl, parea,
                     pkind, robin_area, dlab, dict(AP_BENCH), M=3, dt=dt, sweeps=sweeps, tol=tol,
                     steps=steps, u0=u0, w0=np.zeros(pk.size), robin_eps=1e-4 * sigma_e / box,
                     Cm=1.0, g_gap=0.05 * 222.0, sigma_i=sigma_i, sigma_e=sigma_e,
                     meta={"seed": SEED_BASE + 2, "w_frozen": w_frozen, "labels": lab.shape})
    return wl


def emi_tiny(kind="pair"):
    """Small EMI problems for exact checks."""
    if kind == "two_cells":
        return emi_bricks(cells=(2, 1, 1), cell_um=(8.0, 4.0, 4.0), h=2.0, gap_vox=1, margin=1,
                          name="emi_two_cells", dt=0.02, sweeps=4, tol=1e-4, steps=3)
    if kind == "grid":
        return emi_bricks(cells=(2, 2, 1), cell_um=(10.0, 4.0, 4.0), h=2.0, gap_vox=1, margin=2,
                          name="emi_2x2_cells", dt=0.02, sweeps=4, tol=1e-4, steps=3)
    raise ValueError(kind)
