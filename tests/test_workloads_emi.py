"""The vectorised EMI voxel generator against a plain loop construction of
the same dofs, tetrahedra, membrane pairs and Robin measures (the loops
follow the definitions one voxel, face and vertex at a time)."""

from itertools import permutations

import numpy as np
import pytest

from workloads.emi import brick_labels, emi_from_labels, emi_tiny
from workloads.meshes import Mesh

_PERMS = list(permutations(range(3)))


def _loops(lab: np.ndarray, h: float, sigma_i: float, sigma_e: float):
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



@pytest.mark.parametrize("case", ["two_cells", "grid", "mixed"])
def test_vectorised_generator_matches_loops(case):
    if case == "two_cells":
        lab, h = brick_labels((2, 1, 1), (4, 2, 2), 1, 1), 2.0
    elif case == "grid":
        lab, h = brick_labels((2, 2, 1), (5, 2, 2), 1, 2), 2.0
    else:
        rng = np.random.default_rng(7)
        lab, h = rng.integers(0, 4, size=(5, 4, 3)).astype(np.int32), 1.5
    a = emi_from_labels(lab, h, 3.0, 20.0)
    b = _loops(lab, h, 3.0, 20.0)
    ma, mb = a[0], b[0]
    assert np.array_equal(ma.xyz, mb.xyz)
    assert np.array_equal(ma.elems, mb.elems)
    assert np.array_equal(ma.elem_sigma, mb.elem_sigma)
    for x, y in zip(a[1:], b[1:]):
        assert x.shape == y.shape
        np.testing.assert_allclose(x, y, rtol=1e-15, atol=0)
    # every membrane area is a whole number of quarter faces
    q = a[3] / (h * h / 4)
    assert np.array_equal(q, np.round(q))


def test_tiny_workloads_have_both_pair_kinds():
    wl = emi_tiny("grid")
    assert set(wl.pair_kind.tolist()) == {0, 1}
    assert np.all(wl.pair_k != wl.pair_l)
    # kind 0 is oriented cell -> bath
    assert np.all(wl.labels[wl.pair_k[wl.pair_kind == 0]] > 0)
    assert np.all(wl.labels[wl.pair_l[wl.pair_kind == 0]] == 0)
