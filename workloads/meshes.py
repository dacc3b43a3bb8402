"""Structured simplex meshes with deterministic vertex numbering.

Vertex numbering is lexicographic with x fastest.  Every element is a P1
simplex given by its dim+1 vertex indices.  Nothing here evaluates any part of
the method; the arrays are inputs for both the CUDA library and the oracle.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np


@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray          # (n_nodes, dim) float64
    elems: np.ndarray        # (n_elems, dim + 1) int32
    elem_sigma: np.ndarray | None = None   # (n_elems, 3, 3) float64 or None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])


def grid2d(nx: int, ny: int, hx: float, hy: float | None = None) -> Mesh:
    """Right-triangle mesh of an nx-by-ny vertex grid.

    Each square [i, i+1] x [j, j+1] is cut along its (i, j)-(i+1, j+1)
    diagonal into {(i,j), (i+1,j), (i+1,j+1)} and {(i,j), (i+1,j+1), (i,j+1)}.
    """
    hy = hx if hy is None else hy
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xyz = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()

    def vid(i, j):
        return i + nx * j

    t1 = np.stack([vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1)], axis=1)
    t2 = np.stack([vid(ci, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)], axis=1)
    elems = np.empty((2 * ci.size, 3), dtype=np.int32)
    elems[0::2] = t1
    elems[1::2] = t2
    return Mesh(2, xyz, elems, meta={"nx": nx, "ny": ny, "h": (hx, hy)})


_KUHN_PERMS = list(permutations(range(3)))


def kuhn3d(nx: int, ny: int, nz: int, hx: float, hy: float | None = None,
           hz: float | None = None) -> Mesh:
    """Kuhn (Freudenthal) 6-tetrahedron split of an nx-by-ny-by-nz vertex grid.

    For the cube with lowest corner c, one tetrahedron per permutation p of the
    axes has vertices c, c+e_p0, c+e_p0+e_p1, c+e_p0+e_p1+e_p2.  The split is
    conforming because every cube uses the same six permutations.
    """
    hy = hx if hy is None else hy
    hz = hx if hz is None else hz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = np.stack([i.ravel() * hx, j.ravel() * hy, k.ravel() * hz], axis=1).astype(np.float64)
    ck, cj, ci = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    nc = ci.size
    elems = np.empty((6 * nc, 4), dtype=np.int32)
    for t, perm in enumerate(_KUHN_PERMS):
        off = np.zeros(3, dtype=np.int64)
        cols = []
        for step in range(4):
            if step > 0:
                off[perm[step - 1]] += 1
            cols.append((ci + off[0]) + nx * ((cj + off[1]) + ny * (ck + off[2])))
        elems[t::6] = np.stack(cols, axis=1)
    return Mesh(3, xyz, elems, meta={"nx": nx, "ny": ny, "nz": nz, "h": (hx, hy, hz)})


def ventricle_shell(h: float, seed: int, outer=(5.0, 5.0, 10.0), wall: float = 2.5,
                    d_long: float = 1.0, d_trans: float = 0.25) -> Mesh:
    """Synthetic left-ventricle-like shell carved out of a Kuhn grid.

    Truncated thick ellipsoidal shell: outer semi-axes ``outer`` (mm), wall
    thickness ``wall``, cut at the base plane z = 0 (apex at z = -outer[2]).
    Tetrahedra whose centroid lies inside the shell are kept, unused vertices
    dropped, and the vertex numbering is randomly permuted (seeded) so that the
    stored matrix rows have an irregular neighbour pattern.  Each element gets a
    full conductivity tensor d_trans*I + (d_long-d_trans)*f f^T whose fibre
    direction f rotates from -60 to +60 degrees through the wall.
    """
    ax, ay, az = outer
    bx, by, bz = ax - wall, ay - wall, az - wall
    nx = int(np.ceil(2 * ax / h)) + 1
    ny = int(np.ceil(2 * ay / h)) + 1
    nz = int(np.ceil(az / h)) + 1
    base = kuhn3d(nx, ny, nz, h)
    xyz = base.xyz + np.array([-ax, -ay, -az])
    cen = xyz[base.elems].mean(axis=1)
    ro = (cen[:, 0] / ax) ** 2 + (cen[:, 1] / ay) ** 2 + (cen[:, 2] / az) ** 2
    ri = (cen[:, 0] / bx) ** 2 + (cen[:, 1] / by) ** 2 + (cen[:, 2] / bz) ** 2
    keep = (ro <= 1.0) & (ri >= 1.0) & (cen[:, 2] <= 0.0)
    elems = base.elems[keep]
    used = np.unique(elems)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(used.size)
    newid = np.full(base.n_nodes, -1, dtype=np.int64)
    newid[used] = perm
    xyz_new = np.empty((used.size, 3))
    xyz_new[perm] = xyz[used]
    elems = newid[elems].astype(np.int32)
    # transmural depth in [0, 1]: 0 on the endocardium, 1 on the epicardium
    c = cen[keep]
    rad_o = np.sqrt((c[:, 0] / ax) ** 2 + (c[:, 1] / ay) ** 2 + (c[:, 2] / az) ** 2)
    rad_i = np.sqrt((c[:, 0] / bx) ** 2 + (c[:, 1] / by) ** 2 + (c[:, 2] / bz) ** 2)
    depth = np.clip((rad_i - 1.0) / np.maximum(rad_i - rad_o, 1e-12), 0.0, 1.0)
    angle = np.deg2rad(-60.0 + 120.0 * depth)
    # circumferential and longitudinal unit vectors
    phi = np.arctan2(c[:, 1], c[:, 0])
    e_circ = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    e_long = np.tile(np.array([0.0, 0.0, 1.0]), (c.shape[0], 1))
    f = np.cos(angle)[:, None] * e_circ + np.sin(angle)[:, None] * e_long
    sig = d_trans * np.eye(3)[None, :, :] + (d_long - d_trans) * f[:, :, None] * f[:, None, :]
    apex = np.array([0.0, 0.0, -az])
    return Mesh(3, xyz_new, elems, elem_sigma=sig,
                meta={"h": h, "apex": apex, "seed": seed})
