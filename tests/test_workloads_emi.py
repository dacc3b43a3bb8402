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


def _loops_2d(lab: np.ndarray, h: float, sigma_i: float, sigma_e: float):
    """The 2D generator's definitions, one pixel, edge and vertex at a time."""
    nx, ny = lab.shape
    vx, vy = nx + 1, ny + 1

    def vid(i, j):
        return i + vx * j

    vlabels = [set() for _ in range(vx * vy)]
    for j in range(ny):
        for i in range(nx):
            for dj in (0, 1):
                for di in (0, 1):
                    vlabels[vid(i + di, j + dj)].add(int(lab[i, j]))
    dof, xyz, dlab = {}, [], []
    for j in range(vy):
        for i in range(vx):
            for c in sorted(vlabels[vid(i, j)]):
                dof[(vid(i, j), c)] = len(xyz)
                xyz.append((i * h, j * h))
                dlab.append(c)
    elems, esig = [], []
    for j in range(ny):
        for i in range(nx):
            c = int(lab[i, j])
            a, b = dof[(vid(i, j), c)], dof[(vid(i + 1, j), c)]
            cc, d = dof[(vid(i + 1, j + 1), c)], dof[(vid(i, j + 1), c)]
            for tri in ((a, b, cc), (a, cc, d)):
                elems.append(tri)
                esig.append((sigma_e if c == 0 else sigma_i) * np.eye(3))
    acc = {}

    def add_edge(verts, ca, cb):
        if ca == cb:
            return
        if ca == 0 or cb == 0:
            first, second, kind = max(ca, cb), 0, 0
        else:
            first, second, kind = min(ca, cb), max(ca, cb), 1
        for v in verts:
            key = (dof[(v, first)], dof[(v, second)], kind)
            acc[key] = acc.get(key, 0.0) + h / 2

    robin = np.zeros(len(xyz))
    for j in range(ny):
        for i in range(nx):
            c = int(lab[i, j])
            if i + 1 < nx:
                add_edge([vid(i + 1, j), vid(i + 1, j + 1)], c, int(lab[i + 1, j]))
            if j + 1 < ny:
                add_edge([vid(i, j + 1), vid(i + 1, j + 1)], c, int(lab[i, j + 1]))
            for on, verts in ((i == 0, [vid(0, j), vid(0, j + 1)]),
                              (i == nx - 1, [vid(nx, j), vid(nx, j + 1)]),
                              (j == 0, [vid(i, 0), vid(i + 1, 0)]),
                              (j == ny - 1, [vid(i, ny), vid(i + 1, ny)])):
                if on:
                    for v in verts:
                        robin[dof[(v, c)]] += h / 2
    keys = sorted(acc)
    mesh = Mesh(2, np.array(xyz), np.array(elems, np.int32), elem_sigma=np.array(esig))
    return (mesh, np.array([k[0] for k in keys], np.int32), np.array([k[1] for k in keys], np.int32),
            np.array([acc[k] for k in keys]), np.array([k[2] for k in keys], np.int32), robin,
            np.array(dlab, np.int32))


@pytest.mark.parametrize("case", ["cells", "mixed"])
def test_vectorised_2d_generator_matches_loops(case):
    from workloads.emi import emi_from_labels_2d
    if case == "cells":
        lab = np.zeros((9, 6), np.int32)
        lab[1:4, 1:3], lab[4:8, 1:3], lab[2:5, 4:5] = 1, 2, 3
        h = 2.0
    else:
        lab, h = np.random.default_rng(3).integers(0, 3, size=(6, 5)).astype(np.int32), 1.25
    a = emi_from_labels_2d(lab, h, 3.0, 20.0)
    b = _loops_2d(lab, h, 3.0, 20.0)
    assert np.array_equal(a[0].xyz, b[0].xyz) and np.array_equal(a[0].elems, b[0].elems)
    assert np.array_equal(a[0].elem_sigma, b[0].elem_sigma)
    for x, y in zip(a[1:], b[1:]):
        assert x.shape == y.shape
        np.testing.assert_allclose(x, y, rtol=1e-15, atol=0)


def test_branched_2d_layout_measures():
    """Membrane measure = the cells' perimeters less twice the shared (gap
    junction) edges; Robin measure = the box perimeter; every cell reachable
    from the first through gap junctions."""
    from workloads.emi import branched_labels_2d, emi_from_labels_2d
    h = 2.5
    lab = branched_labels_2d(h)
    mesh, pk, pl, pa, kind, robin, dlab = emi_from_labels_2d(lab, h, 3.0, 20.0)
    per = 0.0
    for c in range(1, lab.max() + 1):
        m = lab == c
        per += h * (np.abs(np.diff(np.pad(m, 1).astype(int), axis=0)).sum()
                    + np.abs(np.diff(np.pad(m, 1).astype(int), axis=1)).sum())
    gap = pa[kind == 1].sum()
    assert pa[kind == 0].sum() + 2 * gap == pytest.approx(per, rel=1e-14)
    assert robin.sum() == pytest.approx(2 * h * (lab.shape[0] + lab.shape[1]), rel=1e-14)
    adj = {}
    for k, l in zip(pk[kind == 1], pl[kind == 1]):
        adj.setdefault(dlab[k], set()).add(dlab[l])
        adj.setdefault(dlab[l], set()).add(dlab[k])
    seen, todo = {1}, [1]
    while todo:
        for nb in adj.get(todo.pop(), ()):
            if nb not in seen:
                seen.add(nb)
                todo.append(nb)
    assert seen == set(range(1, lab.max() + 1))
