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
    """Dofs, tetrahedra, membrane pairs and Robin areas of a labelled voxel grid.

    Numbering: vertices in x-fastest order, at each vertex one dof per label of
    its voxels in ascending label order.  Elements: voxels in x-fastest order,
    six Kuhn tetrahedra per voxel in the order of the axis permutations.  Pairs
    sorted by (first dof, second dof, kind); each membrane face adds a quarter
    of its area to the pair of every one of its four vertices."""
    lab = np.asarray(lab, dtype=np.int64)
    nx, ny, nz = lab.shape
    vx, vy, vz = nx + 1, ny + 1, nz + 1
    L = int(lab.max()) + 1
    I, J, Kz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # voxels in x-fastest order
    order = lambda a: np.ascontiguousarray(a.transpose(2, 1, 0)).reshape(-1)
    vi, vj, vk, vl = order(I), order(J), order(Kz), order(lab)

    def vid(i, j, k):
        return i + vx * (j + vy * k)

    # (vertex, label) keys of every voxel corner -> dof numbers
    corners = [vid(vi + di, vj + dj, vk + dk) * L + vl
               for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    keys = np.unique(np.concatenate(corners))
    vert = keys // L
    dlab = (keys % L).astype(np.int32)
    xyz = np.stack([vert % vx, (vert // vx) % vy, vert // (vx * vy)], axis=1).astype(np.float64) * h

    def dof(v, c):
        return np.searchsorted(keys, v * L + c).astype(np.int32)

    # six Kuhn tetrahedra per voxel
    tets = []
    for perm in _PERMS:
        off = np.zeros(3, np.int64)
        vs = []
        for step in range(4):
            if step > 0:
                off[perm[step - 1]] += 1
            vs.append(dof(vid(vi + off[0], vj + off[1], vk + off[2]), vl))
        tets.append(np.stack(vs, axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    sig = np.where(np.repeat(vl, 6) == 0, sigma_e, sigma_i)
    esig = sig[:, None, None] * np.eye(3)[None]
    # membrane faces: voxel pairs of different labels across each axis
    quarter = h * h / 4.0
    f_first, f_second, f_kind = [], [], []
    face_verts = {0: ((1, 0, 0), (1, 1, 0), (1, 0, 1), (1, 1, 1)),
                  1: ((0, 1, 0), (1, 1, 0), (0, 1, 1), (1, 1, 1)),
                  2: ((0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1))}
    for ax in range(3):
        nb = [0, 0, 0]
        nb[ax] = 1
        a = lab[:lab.shape[0] - nb[0], :lab.shape[1] - nb[1], :lab.shape[2] - nb[2]]
        b = lab[nb[0]:, nb[1]:, nb[2]:]
        ii, jj, kk = np.nonzero(a != b)
        ca, cb = a[ii, jj, kk], b[ii, jj, kk]
        ecs = (ca == 0) | (cb == 0)
        first = np.where(ecs, np.maximum(ca, cb), np.minimum(ca, cb))
        second = np.where(ecs, 0, np.maximum(ca, cb))
        for d in face_verts[ax]:
            v = vid(ii + d[0], jj + d[1], kk + d[2])
            f_first.append(dof(v, first))
            f_second.append(dof(v, second))
            f_kind.append(np.where(ecs, 0, 1))
    f_first = np.concatenate(f_first).astype(np.int64)
    f_second = np.concatenate(f_second).astype(np.int64)
    f_kind = np.concatenate(f_kind).astype(np.int64)
    n = keys.size
    pkey, counts = np.unique((f_first * n + f_second) * 2 + f_kind, return_counts=True)
    pk = (pkey // 2 // n).astype(np.int32)
    pl = (pkey // 2 % n).astype(np.int32)
    pkind = (pkey % 2).astype(np.int32)
    parea = counts * quarter
    # outer box faces: Robin measure on the dofs of the boundary voxels' labels
    b_dofs = []
    for ax in range(3):
        for side in (0, 1):
            sl = [slice(None)] * 3
            sl[ax] = 0 if side == 0 else lab.shape[ax] - 1
            sub = lab[tuple(sl)]
            g = np.meshgrid(*[np.arange(m) for m in sub.shape], indexing="ij")
            c = sub.reshape(-1)
            other = [g[0].reshape(-1), g[1].reshape(-1)]
            for d0 in (0, 1):
                for d1 in (0, 1):
                    idx = [None, None, None]
                    rest = [q for q in range(3) if q != ax]
                    idx[ax] = np.full(c.size, 0 if side == 0 else lab.shape[ax])
                    idx[rest[0]] = other[0] + d0
                    idx[rest[1]] = other[1] + d1
                    b_dofs.append(dof(vid(idx[0], idx[1], idx[2]), c))
    robin = np.bincount(np.concatenate(b_dofs), minlength=n) * quarter
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


def emi_from_labels_2d(lab: np.ndarray, h: float, sigma_i: float, sigma_e: float):
    """The 2D analogue of emi_from_labels on a labelled pixel grid.

    Numbering: vertices in x-fastest order, at each vertex one dof per label of
    its pixels in ascending label order.  Elements: pixels in x-fastest order,
    two right triangles per pixel split along the (i, j)-(i+1, j+1) diagonal.
    Membranes are the pixel edges between different labels: an edge of length
    h gives each of its two vertices half its length, accumulated per pair of
    dofs; outer box edges give their vertices' dofs half their length of Robin
    measure."""
    lab = np.asarray(lab, dtype=np.int64)
    nx, ny = lab.shape
    vx, vy = nx + 1, ny + 1
    L = int(lab.max()) + 1
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    order = lambda a: np.ascontiguousarray(a.T).reshape(-1)     # pixels in x-fastest order
    pi, pj, pl = order(I), order(J), order(lab)

    def vid(i, j):
        return i + vx * j

    corners = [vid(pi + di, pj + dj) * L + pl for dj in (0, 1) for di in (0, 1)]
    keys = np.unique(np.concatenate(corners))
    vert = keys // L
    dlab = (keys % L).astype(np.int32)
    xyz = np.stack([vert % vx, vert // vx], axis=1).astype(np.float64) * h

    def dof(v, c):
        return np.searchsorted(keys, v * L + c).astype(np.int32)

    a = dof(vid(pi, pj), pl)
    b = dof(vid(pi + 1, pj), pl)
    c = dof(vid(pi + 1, pj + 1), pl)
    d = dof(vid(pi, pj + 1), pl)
    elems = np.stack([np.stack([a, b, c], axis=1), np.stack([a, c, d], axis=1)],
                     axis=1).reshape(-1, 3).astype(np.int32)
    sig = np.where(np.repeat(pl, 2) == 0, sigma_e, sigma_i)
    esig = sig[:, None, None] * np.eye(3)[None]
    half = h / 2.0
    f_first, f_second, f_kind = [], [], []
    # the shared edge of pixels (i, j) and (i, j) + e_ax, as two vertex offsets
    edge_verts = {0: ((1, 0), (1, 1)), 1: ((0, 1), (1, 1))}
    for ax in range(2):
        nb = [0, 0]
        nb[ax] = 1
        p = lab[:nx - nb[0], :ny - nb[1]]
        q = lab[nb[0]:, nb[1]:]
        ii, jj = np.nonzero(p != q)
        ca, cb = p[ii, jj], q[ii, jj]
        ecs = (ca == 0) | (cb == 0)
        first = np.where(ecs, np.maximum(ca, cb), np.minimum(ca, cb))
        second = np.where(ecs, 0, np.maximum(ca, cb))
        for dv in edge_verts[ax]:
            v = vid(ii + dv[0], jj + dv[1])
            f_first.append(dof(v, first))
            f_second.append(dof(v, second))
            f_kind.append(np.where(ecs, 0, 1))
    f_first = np.concatenate(f_first).astype(np.int64)
    f_second = np.concatenate(f_second).astype(np.int64)
    f_kind = np.concatenate(f_kind).astype(np.int64)
    n = keys.size
    pkey, counts = np.unique((f_first * n + f_second) * 2 + f_kind, return_counts=True)
    pk = (pkey // 2 // n).astype(np.int32)
    plr = (pkey // 2 % n).astype(np.int32)
    pkind = (pkey % 2).astype(np.int32)
    parea = counts * half
    b_dofs = []
    for ax in range(2):
        for side in (0, 1):
            if ax == 0:
                i0 = 0 if side == 0 else nx - 1
                cl, jj = lab[i0, :], np.arange(ny)
                iv = np.full(ny, 0 if side == 0 else nx)
                b_dofs += [dof(vid(iv, jj), cl), dof(vid(iv, jj + 1), cl)]
            else:
                j0 = 0 if side == 0 else ny - 1
                cl, ii = lab[:, j0], np.arange(nx)
                jv = np.full(nx, 0 if side == 0 else ny)
                b_dofs += [dof(vid(ii, jv), cl), dof(vid(ii + 1, jv), cl)]
    robin = np.bincount(np.concatenate(b_dofs), minlength=n) * half
    mesh = Mesh(2, xyz, elems, elem_sigma=esig, meta={"h": h, "pixels": lab.shape})
    return mesh, pk, plr, parea, pkind, robin, dlab


def branched_labels_2d(h=1.25):
    """A branching arrangement of myocytes in a 700 x 240 um bath: a trunk of two
    cells splits through a connector cell into two rows of two cells, each of
    which splits again into two rows (17 cells, all 15 um thick); cells touch end
    to end (gap-junction edges).  Lengths in um on an h-um pixel grid."""
    px = lambda um: int(round(um / h))
    lab = np.zeros((px(700.0), px(240.0)), dtype=np.int32)
    cells = []
    t = 15.0

    def row(x0, x1, yc, parts=2):
        xs = np.linspace(x0, x1, parts + 1)
        for a, b in zip(xs[:-1], xs[1:]):
            cells.append((a, b, yc - t / 2, yc + t / 2))

    row(10.0, 230.0, 120.0)                          # trunk
    cells.append((230.0, 245.0, 52.5, 187.5))        # connector to level 1
    row(245.0, 465.0, 60.0)
    row(245.0, 465.0, 180.0)
    cells.append((465.0, 480.0, 22.5, 97.5))         # connectors to level 2
    cells.append((465.0, 480.0, 142.5, 217.5))
    for yc in (30.0, 90.0, 150.0, 210.0):
        row(480.0, 690.0, yc)
    for cid, (x0, x1, y0, y1) in enumerate(cells, start=1):
        lab[px(x0):px(x1), px(y0):px(y1)] = cid
    return lab


def emi_branched_2d(h=1.25, dt=0.02, sweeps=12, tol=1e-4, steps=125, name=None) -> EmiWorkload:
    """2D cell-by-cell workload in the shape of the paper's 2D EMI example
    (Sec. 5.1: branched myocytes in 700 x 240 um, leftmost cell excited, gating
    fixed at w = 0): branched_labels_2d on h-um pixels, same units and
    coefficients as emi_bricks (C_m = 1, sigma_i = 3e4, sigma_e = 2e5 um/ms,
    gap junctions 5 % of 1/(R_g C_m) per length, Robin 1e-4 sigma_e / box)."""
    lab = branched_labels_2d(h)
    sigma_i, sigma_e = 3.0e4, 2.0e5
    mesh, pk, pl, parea, pkind, robin_area, dlab = emi_from_labels_2d(lab, h, sigma_i, sigma_e)
    n = mesh.n_nodes
    u0 = np.where(dlab == 1, 1.0, 0.0)
    box = max(lab.shape) * h
    return EmiWorkload(name or "emi_branched_2d_%d_dofs" % n, mesh, pk, pl, parea, pkind,
                       robin_area, dlab, dict(AP_BENCH), M=3, dt=dt, sweeps=sweeps, tol=tol,
                       steps=steps, u0=u0, w0=np.zeros(pk.size), robin_eps=1e-4 * sigma_e / box,
                       Cm=1.0, g_gap=0.05 * 222.0, sigma_i=sigma_i, sigma_e=sigma_e,
                       meta={"seed": SEED_BASE + 2, "w_frozen": True, "labels": lab.shape})


def coarse_blocks(wl, split=(16, 4, 4), min_dofs=None) -> np.ndarray:
    """Blocks of the two-level preconditioner of the node solves: each subdomain (a
    cell) is one block, and each subdomain with more than `min_dofs` dofs (default:
    four times the median subdomain) is cut by a grid of split[0] x split[1] (x
    split[2]) boxes over its bounding box.  Returns consecutive labels 0 .. nb-1."""
    lab = np.asarray(wl.labels)
    xyz = wl.mesh.xyz
    dim = xyz.shape[1]
    sizes = np.bincount(lab)
    if min_dofs is None:
        min_dofs = 4 * int(np.median(sizes[sizes > 0]))
    key = lab.astype(np.int64) * 0
    big = np.nonzero(sizes > min_dofs)[0]
    for b in big:
        sel = lab == b
        lo, hi = xyz[sel].min(axis=0), xyz[sel].max(axis=0)
        cells = np.array(split[:dim], dtype=np.int64)
        ijk = np.floor((xyz[sel] - lo) / ((hi - lo) / cells + 1e-12)).astype(np.int64)
        ijk = np.minimum(ijk, cells - 1)
        flat = np.ravel_multi_index(tuple(ijk.T), tuple(cells))
        key[sel] = 1 + flat
    # consecutive labels in (subdomain, box) order
    _, out = np.unique(lab.astype(np.int64) * (1 << 32) + key, return_inverse=True)
    return out.astype(np.int32)


def renumber(wl, order) -> "EmiWorkload":
    """The same workload with its dofs renumbered: new dof k is old dof order[k]
    (mesh coordinates and elements, pair ends, Robin measures, labels, initial
    potentials; per-pair data unchanged)."""
    order = np.asarray(order, dtype=np.int64)
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    mesh = Mesh(wl.mesh.dim, wl.mesh.xyz[order], inv[wl.mesh.elems].astype(np.int32),
                wl.mesh.elem_sigma, dict(wl.mesh.meta))
    out = EmiWorkload(wl.name, mesh, inv[wl.pair_k].astype(np.int32),
                      inv[wl.pair_l].astype(np.int32), wl.pair_area, wl.pair_kind,
                      wl.robin_area[order], wl.labels[order], wl.ionic, M=wl.M, dt=wl.dt,
                      sweeps=wl.sweeps, tol=wl.tol, steps=wl.steps, u0=wl.u0[order], w0=wl.w0,
                      robin_eps=wl.robin_eps, Cm=wl.Cm, g_gap=wl.g_gap, sigma_i=wl.sigma_i,
                      sigma_e=wl.sigma_e, cg_rtol=wl.cg_rtol, alpha=wl.alpha,
                      meta=dict(wl.meta, renumbered=True))
    return out


def block_major(wl, blocks):
    """Dof order grouping each block's dofs (stable: the original order inside a
    block), and the blocks in that order: (order, blocks[order])."""
    order = np.argsort(np.asarray(blocks), kind="stable")
    return order, np.asarray(blocks)[order]


def emi_tiny(kind="pair"):
    """Small EMI problems for exact checks."""
    if kind == "two_cells":
        return emi_bricks(cells=(2, 1, 1), cell_um=(8.0, 4.0, 4.0), h=2.0, gap_vox=1, margin=1,
                          name="emi_two_cells", dt=0.02, sweeps=4, tol=1e-4, steps=3)
    if kind == "grid":
        return emi_bricks(cells=(2, 2, 1), cell_um=(10.0, 4.0, 4.0), h=2.0, gap_vox=1, margin=2,
                          name="emi_2x2_cells", dt=0.02, sweeps=4, tol=1e-4, steps=3)
    if kind == "branched_2d":
        return emi_branched_2d(h=10.0, sweeps=4, tol=1e-4, steps=3, name="emi_branched_2d_tiny")
    raise ValueError(kind)
