"""Pins of the oracle's cell-by-cell (EMI) step (Sec. 2.1, eq. cell-by-cell
model / abstract reaction diffusion / abstract gating; sweep of Sec. 3.2).

Expected values come from reductions of the EMI system that the mathematics
fixes: a single membrane with the Robin-grounded bath side reduces to the
point Aliev-Panfilov ODE C_m v' = -I_ion(v, w) (the bath potential stays 0);
a single gap junction between two Robin-grounded nodes reduces to the linear
ODE v' = -(g / C_m + eps / (2 A C_m)) v, whose converged Radau step is the
Pade(M-1, M) function.
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
