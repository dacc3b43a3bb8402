"""Pins of the oracle's cell-by-cell (EMI) step (Sec. 2.1, eq. cell-by-cell
model / abstract reaction diffusion / abstract gating; sweep of Sec. 3.2).

Expected values come from reductions of the EMI system that the mathematics
fixes: a single membrane with the Robin-grounded bath side reduces to the
point Aliev-Panfilov ODE C_m v' = -I_ion(v, w) (the bath potential stays 0);
a single gap junction between two Robin-grounded nodes reduces to the linear
ODE v' = -(g / C_m + eps / (2 A C_m)) v, whose converged Radau step is the
Pade(M-1, M) function; and on two cells, plain SDC swept to convergence equals
the collocation solution of the whole EMI system, solved densely by Newton
from its definition (numpy).
"""

import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.emi import EmiWorkload, emi_tiny


def _pair_system(kind, area, robin, Cm, g_gap, ionic, u0, w0, dt=0.05, M=3):
    S = oracle.System.from_matrix([0, 2, 4], [0, 1, 0, 1], [0.0, 0.0, 0.0, 0.0], [1.0, 1.0])
    mesh = W.Mesh(3, np.zeros((2, 3)), np.zeros((0, 4), np.int32))
    wl = EmiWorkload("pair", mesh, np.array([0], np.int32), np.array([1], np.int32),
                     np.array([area]), np.array([kind], np.int32), np.asarray(robin, float),
                     np.array([1, 0], np.int32), ionic, M=M, dt=dt, sweeps=60, tol=0.0, steps=1,
                     u0=np.asarray(u0, float), w0=np.asarray(w0, float), robin_eps=1.0, Cm=Cm,
                     g_gap=g_gap)
    return S, wl


@pytest.mark.parametrize("M", [2, 3])
def test_single_membrane_reduces_to_point_ionic_ode(M):
    # C_m = 1: the point model v' = -I_ion(v, w) is the one-dof monodomain
    # system (its lumped mass multiplies both v' and the ionic load); C_m enters
    # the gap-junction pin below
    p = dict(W.AP_PAPER)
    Cm, area = 1.0, 3.0
    S, wl = _pair_system(0, area, [0.0, 0.4], Cm, 0.0, p, [0.35, 0.0], [0.05], M=M)
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=60, cg_rtol=1e-15)
    assert r["status"] == 0
    S1 = oracle.System.from_matrix([0, 1], [0], [0.0], [0.7])
    s = S1.step(p, M, [0.35], [0.05], 0.05, 60, 0.0, cg_rtol=1e-15)
    assert abs(r["u"][1]) <= 1e-14
    assert r["u"][0] == pytest.approx(s["v"][0], abs=1e-13)
    assert r["w"][0] == pytest.approx(s["w"][0], abs=1e-13)
    assert abs(r["u"][0] - 0.35) > 1e-3


def _pade(M, z):
    f = math.factorial
    num = sum(f(2 * M - 1 - j) * f(M - 1) / (f(2 * M - 1) * f(j) * f(M - 1 - j)) * z ** j
              for j in range(M))
    den = sum(f(2 * M - 1 - j) * f(M) / (f(2 * M - 1) * f(j) * f(M - j)) * (-z) ** j
              for j in range(M + 1))
    return num / den


@pytest.mark.parametrize("M", [1, 3, 4])
def test_gap_junction_pair_is_a_linear_ode(M):
    Cm, area, g, eps = 1.3, 2.0, 5.0, 0.6
    S, wl = _pair_system(1, area, [eps, eps], Cm, g, dict(W.AP_BENCH), [0.3, -0.1], [0.0], M=M)
    dt = 0.05
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=60, cg_rtol=1e-15)
    assert r["status"] == 0
    # u_k + u_l -> 0 is algebraic; v = u_k - u_l decays with rate lam
    lam = g / Cm + eps / (2 * area * Cm)
    v0 = 0.3 - (-0.1)
    v = r["u"][0] - r["u"][1]
    assert abs(r["u"][0] + r["u"][1]) <= 1e-13
    assert v == pytest.approx(_pade(M, -lam * dt) * v0, rel=1e-12)


def test_emi_invariants_on_two_cells():
    wl = emi_tiny("two_cells")
    S = oracle.System.from_mesh(wl.mesh)
    plain = S.step_emi(wl, wl.u0, wl.w0, tol=0.0, want_log=True)
    a0 = S.step_emi(wl, wl.u0, wl.w0, tol=0.0)
    assert plain["status"] == 0 and np.array_equal(plain["u"], a0["u"])
    assert all(len(x) == wl.n for x in plain["active"])
    ad = S.step_emi(wl, wl.u0, wl.w0, tol=1e-2, want_log=True)
    assert ad["status"] == 0
    act = ad["active"]
    for k in range(len(act) - 1):
        assert set(act[k + 1].tolist()) <= set(act[k].tolist())
    assert len(act[1]) < wl.n
    # the excited cell pulls the bath and the neighbour: the state moved everywhere
    assert np.abs(ad["u"] - wl.u0).max() > 1e-3


def _emi_collocation_solve(wl, M, dt):
    """The Radau-IIA collocation system of the cell-by-cell model written out
    densely and solved by Newton (finite-difference Jacobian, numpy):
        B (U_m - u0) + dt sum_j Q_mj (A U_j + b(U_j, W_j)) = 0,
        W_m - w0 - dt sum_j Q_mj R(v_j, W_j) = 0  on the cell-bath pairs,
    with B = sum_p area_p Cm e_p e_p', A = K + diag(robin), b = sum_p area_p
    I_p(v_p, w_p) e_p, e_p = e_k - e_l, v_p = u_k - u_l, I_p the Aliev-Panfilov
    current (cell-bath) or g_gap v (gap junction); gap-junction w stays w0."""
    import scipy.sparse as sp
    S = oracle.System.from_mesh(wl.mesh)
    ptr, col, val, _ = S.matrix()
    n, npair = wl.n, wl.n_pairs
    A = sp.csr_matrix((val, col, ptr), shape=(n, n)) + sp.diags(wl.robin)
    E = sp.csr_matrix((np.concatenate([np.ones(npair), -np.ones(npair)]),
                       (np.concatenate([np.arange(npair)] * 2),
                        np.concatenate([wl.pair_k, wl.pair_l]))), shape=(npair, n))
    area = wl.pair_area
    memb = wl.pair_kind == 0
    p = wl.ionic
    _, Q, _ = oracle.collocation(M)
    u0, w0 = wl.u0, wl.w0
    B = E.T @ sp.diags(area * wl.Cm) @ E

    def I(v, w):
        return np.where(memb, p["ga"] * v * (v - p["a"]) * (v - 1.0) + v * w, wl.g_gap * v)

    def R(v, w):
        E_ = p["eps"] + p["mu1"] * w / (v + p["mu2"])
        G = -w - p["gs"] * v * (v - p["a"] - 1.0)
        return np.where(memb, p["cw"] * E_ * G, 0.0)

    def G(z):
        U = z[:M * n].reshape(M, n)
        Wp = z[M * n:].reshape(M, npair)
        F = np.array([A @ U[j] + E.T @ (area * I(E @ U[j], Wp[j])) for j in range(M)])
        Rv = np.array([R(E @ U[j], Wp[j]) for j in range(M)])
        gu = np.array([B @ (U[m] - u0) + dt * Q[m] @ F for m in range(M)])
        gw = np.array([Wp[m] - w0 - dt * Q[m] @ Rv for m in range(M)])
        return np.concatenate([gu.ravel(), gw.ravel()])

    z = np.concatenate([np.tile(u0, M), np.tile(w0, M)])
    for _ in range(20):
        g = G(z)
        if np.abs(g).max() < 1e-14:
            break
        h = 1e-7
        Jac = np.empty((z.size, z.size))
        for c in range(z.size):
            zc = z.copy()
            zc[c] += h
            Jac[:, c] = (G(zc) - g) / h
        z = z - np.linalg.solve(Jac, g)
    assert np.abs(G(z)).max() < 1e-12
    return z[(M - 1) * n:M * n], z[M * n + (M - 1) * npair:]


def test_converged_emi_sdc_equals_the_collocation_solve():
    """Sec. 3.1/3.2 on the cell-by-cell system: plain SDC swept to convergence
    reaches the fixed point, the Radau-IIA collocation solution of the EMI
    system, solved here densely from its definition."""
    wl = emi_tiny("two_cells")
    wl.u0 = np.where(wl.u0 > 0.5, 0.6, 0.0)
    wl.w0 = np.full(wl.n_pairs, 0.02)
    M, dt = 2, 0.02
    wl.M, wl.dt = M, dt
    S = oracle.System.from_mesh(wl.mesh)
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=60, tol=0.0, cg_rtol=1e-15)
    assert r["status"] == 0
    u_ref, w_ref = _emi_collocation_solve(wl, M, dt)
    assert np.abs(r["u"] - u_ref).max() <= 1e-11 * max(1.0, np.abs(u_ref).max())
    assert np.abs(r["w"] - w_ref).max() <= 1e-11
    assert np.abs(r["u"] - wl.u0).max() > 1e-3      # the step really moves
