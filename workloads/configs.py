"""Seeded synthetic workloads with the shapes of the paper's examples.

Names and sizes:
  w0_square  65x65-node right-triangle mesh of [0,20]^2 (2D monodomain)
  w1_slab    201x71x31-node Kuhn slab, 20x7x3 mm, h = 0.1 mm (3D monodomain)
  w1l_slab   401x141x61-node slab, same physics, larger than the GPU's L2
  w4_slab    101x36x16-node slab, h = 0.2 mm (differentiation workload)
  w5_tissue  ventricle-like shell with per-element fibre tensors
  tiny       3x3 / 5x5 / 2x2x2 meshes for exact-solve checks
  batch_instances  many 2D instances of log-uniform size

The voltage variable is v (transmembrane), the recovery variable is w.  Time
is in ms, lengths in mm, conductivities in mm^2/ms (dimensionless
Aliev-Panfilov kinetics with C_m = 1).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .meshes import Mesh, grid2d, kuhn3d, ventricle_shell

SEED_BASE = 2311_07206

# Aliev-Panfilov parameter sets (ga, gs, a, eps, mu1, mu2, cw).
# AP_BENCH: the standard 1996 form (k = 8, a = 0.15, eps0 = 0.002, mu1 = 0.2,
# mu2 = 0.3, no 1/4 prefactor).  AP_PAPER: the values listed in Sec. 5.1.1.
AP_BENCH = dict(ga=8.0, gs=8.0, a=0.15, eps=0.002, mu1=0.2, mu2=0.3, cw=1.0)
AP_PAPER = dict(ga=8.0, gs=8.0, a=0.1, eps=0.01, mu1=0.07, mu2=0.3, cw=0.25)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    sigma: np.ndarray                  # (3, 3) global conductivity tensor
    ionic: dict
    M: int
    dt: float
    sweeps: int
    tol: float                         # SDC tolerance; drop tolerance = alpha * tol
    steps: int
    v0: np.ndarray
    w0: np.ndarray
    stim_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    stim_amp: float = 0.0
    stim_t_on: float = 0.0
    stim_t_off: float = 0.0
    dof_scale: np.ndarray | None = None
    cg_rtol: float = 1e-10
    alpha: float = 0.1
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.mesh.n_nodes

    def stim_vector(self, t: float) -> np.ndarray:
        """Per-node stimulus current for a step starting at time t.

        The stimulus is on for whole steps: on iff t_on <= t < t_off.
        """
        s = np.zeros(self.n)
        if self.stim_nodes.size and self.stim_t_on <= t < self.stim_t_off:
            s[self.stim_nodes] = self.stim_amp
        return s


def _box_nodes(xyz: np.ndarray, upper) -> np.ndarray:
    mask = np.ones(xyz.shape[0], dtype=bool)
    for d, u in enumerate(upper):
        mask &= xyz[:, d] <= u + 1e-12
    return np.nonzero(mask)[0].astype(np.int32)


def w0_square(tol: float = 1e-4, n: int = 65, length: float = 20.0) -> Workload:
    """2D monodomain square: v = 1 on the [0,2]^2 corner block at t = 0."""
    h = length / (n - 1)
    mesh = grid2d(n, n, h)
    v0 = np.zeros(mesh.n_nodes)
    v0[_box_nodes(mesh.xyz, (2.0, 2.0))] = 1.0
    return Workload("w0_square_%dx%d" % (n, n), mesh, np.eye(3), dict(AP_BENCH), M=3,
                    dt=0.1, sweeps=4, tol=tol, steps=100, v0=v0, w0=np.zeros(mesh.n_nodes))


def _slab(name, nx, ny, nz, h, M, dt, sweeps, tol, steps) -> Workload:
    mesh = kuhn3d(nx, ny, nz, h)
    sigma = np.diag([1.0, 0.25, 0.25])
    stim = _box_nodes(mesh.xyz, (1.5, 1.5, 1.5))
    n = mesh.n_nodes
    return Workload(name, mesh, sigma, dict(AP_BENCH), M=M, dt=dt, sweeps=sweeps, tol=tol,
                    steps=steps, v0=np.zeros(n), w0=np.zeros(n), stim_nodes=stim,
                    stim_amp=2.0, stim_t_on=0.0, stim_t_off=1.0)


def w1_slab(tol: float = 1e-5) -> Workload:
    """3D slab 20x7x3 mm, 201x71x31 nodes, fibres along x (4:1), 1 ms corner stimulus."""
    return _slab("w1_slab_201x71x31", 201, 71, 31, 0.1, M=4, dt=0.05, sweeps=5, tol=tol,
                 steps=1000)


def w1l_slab(tol: float = 1e-5) -> Workload:
    """The slab scaled to 401x141x61 nodes (40x14x6 mm), same physics."""
    return _slab("w1l_slab_401x141x61", 401, 141, 61, 0.1, M=4, dt=0.05, sweeps=5, tol=tol,
                 steps=1000)


def w4_slab(seed_offset: int = 4) -> Workload:
    """Slab of 101x36x16 nodes (h = 0.2 mm) with a seeded per-node conductivity scale."""
    wl = _slab("w4_slab_101x36x16", 101, 36, 16, 0.2, M=3, dt=0.05, sweeps=4, tol=1e-5,
               steps=200)
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    wl.dof_scale = 1.0 + 0.1 * rng.standard_normal(wl.n)
    wl.meta["probes"] = np.sort(rng.choice(wl.n, size=256, replace=False)).astype(np.int32)
    return wl


def w5_tissue(h: float = 0.087, seed_offset: int = 5) -> Workload:
    """Ventricle-like shell with fibre rotation and randomly permuted vertices."""
    mesh = ventricle_shell(h, SEED_BASE + seed_offset)
    apex = mesh.meta["apex"]
    d = np.linalg.norm(mesh.xyz - apex[None, :], axis=1)
    stim = np.nonzero(d <= 1.5 + 1e-12)[0].astype(np.int32)
    n = mesh.n_nodes
    return Workload("w5_tissue_%d" % n, mesh, np.eye(3), dict(AP_BENCH), M=3, dt=0.05,
                    sweeps=5, tol=1e-4, steps=1000, v0=np.zeros(n), w0=np.zeros(n),
                    stim_nodes=stim, stim_amp=2.0, stim_t_on=0.0, stim_t_off=1.0)


def tiny(kind: str) -> Workload:
    """Tiny meshes for checks that need a dense direct solve."""
    if kind == "2d3":
        mesh = grid2d(3, 3, 0.5)
    elif kind == "2d5":
        mesh = grid2d(5, 5, 0.25)
    elif kind == "3d2":
        mesh = kuhn3d(2, 2, 2, 0.5)
    elif kind == "3d3":
        mesh = kuhn3d(3, 3, 3, 0.5)
    else:
        raise ValueError(kind)
    n = mesh.n_nodes
    v0 = np.zeros(n)
    v0[0] = 1.0
    v0[1] = 0.6
    w0 = np.zeros(n)
    w0[n - 1] = 0.3
    sigma = np.diag([1.0, 0.5, 0.25])
    return Workload("tiny_" + kind, mesh, sigma, dict(AP_BENCH), M=3, dt=0.05, sweeps=60,
                    tol=0.0, steps=1, v0=v0, w0=w0)


def batch_instances(count: int = 96, seed_offset: int = 3, h: float = 0.3125,
                    nmin: int = 64, nmax: int = 512):
    """Independent 2D instances: side n log-uniform in [nmin, nmax], D ~ U[0.5, 2],
    a 2x2 excited square at a uniformly drawn centre (clipped to the domain)."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    out = []
    for b in range(count):
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        D = float(rng.uniform(0.5, 2.0))
        L = (n - 1) * h
        cx, cy = rng.uniform(0.0, L, size=2)
        mesh = grid2d(n, n, h)
        x, y = mesh.xyz[:, 0], mesh.xyz[:, 1]
        v0 = np.where((np.abs(x - cx) <= 1.0 + 1e-12) & (np.abs(y - cy) <= 1.0 + 1e-12), 1.0, 0.0)
        out.append(Workload("batch_%d_n%d" % (b, n), mesh, D * np.eye(3), dict(AP_BENCH), M=3,
                            dt=0.1, sweeps=4, tol=1e-4, steps=100, v0=v0,
                            w0=np.zeros(mesh.n_nodes), meta={"D": D, "centre": (cx, cy)}))
    return out
