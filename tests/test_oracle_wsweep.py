"""Pins of the oracle's pointwise gating sweep for M >= 2 (Sec. 3.2, w line of
eq. final-sdc in its Newton-consistent reading: with g_j = R(v_j, w_j) and
d_j = dR/dw(v_j, w_j),
    s_m   = w0 + dt sum_j Q_mj g_j - w_m,
    eps_m = (s_m + dt sum_{j<m} Qhat_mj d_j eps_j) / (1 - dt Qhat_mm d_m),
    w_m  += eps_m).

The fixed-point pins (dense collocation solve, Pade, observed order) cannot see
which lower-triangular Qhat couples the nodes, so these tests fix the coupling
itself.  The voltage is held at v = 0 exactly (v0 = 0, no stimulus, and
I_ion(0, w) = 0, so every residual and correction of v vanishes); then
R(0, w) = -cw (eps + mu1 w / mu2) w is a scalar ODE in w alone.

1. Stiff limit (mu1 = 0, R = lam w, z = dt lam -> -inf): the sweep's error
   propagator tends to E = I - Qhat^-1 Q = I - L^T, which is nilpotent for the
   LU trick (Q^T = L U, Qhat = U^T).  So the node values reach the collocation
   solution w0 (I - z Q)^-1 1 after exactly M sweeps, and not after M - 1.
2. Non-stiff, nonlinear (mu1 != 0): after the first sweep the node values
   differ, so d_j differs between nodes, and the second sweep's result is
   fixed by the lower-triangular system (I - dt Qhat diag(d)) eps = s, solved
   here by numpy's dense solver.

A sign error in the coupling, a loop bound j <= m, or d_m in place of d_j
fails one of them.  The same two checks run on the cell-by-cell step with one
cell-bath membrane pair whose bath side is grounded by its Robin term.
"""

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.emi import EmiWorkload


def _R(p, w):
    """R(0, w) and dR/dw(0, w) of the Aliev-Panfilov gating equation."""
    g = -p["cw"] * (p["eps"] + p["mu1"] * w / p["mu2"]) * w
    d = -p["cw"] * (p["eps"] + 2.0 * p["mu1"] * w / p["mu2"])
    return g, d


def _dense_sweeps(p, M, w0, dt, sweeps):
    """Node values of w after `sweeps` sweeps from the spread predictor, each
    sweep one dense solve of (I - dt Qhat diag(d)) eps = s."""
    tau, Q, Qh = oracle.collocation(M)
    Wn = np.full(M, float(w0))
    for _ in range(sweeps):
        g, d = _R(p, Wn)
        s = w0 + dt * Q @ g - Wn
        Wn = Wn + np.linalg.solve(np.eye(M) - dt * Qh @ np.diag(d), s)
    return Wn


def _collocation_linear(M, lam, dt, w0):
    _, Q, _ = oracle.collocation(M)
    return np.linalg.solve(np.eye(M) - dt * lam * Q, np.full(M, float(w0)))


def _mono_nodes(p, M, w0, dt, sweeps):
    S = oracle.System.from_matrix([0, 1], [0], [0.0], [0.7])
    r = S.step(p, M, [0.0], [w0], dt, sweeps, 0.0, cg_rtol=1e-15, want_nodes=True)
    assert r["status"] == 0
    assert np.all(r["V"] == 0.0)
    return r["W"][:, 0]


def _emi_last(p, M, w0, dt, sweeps):
    S = oracle.System.from_matrix([0, 2, 4], [0, 1, 0, 1], [0.0] * 4, [1.0, 1.0])
    mesh = W.Mesh(3, np.zeros((2, 3)), np.zeros((0, 4), np.int32))
    wl = EmiWorkload("pair", mesh, np.array([0], np.int32), np.array([1], np.int32),
                     np.array([2.0]), np.array([0], np.int32), np.array([0.0, 0.4]),
                     np.array([1, 0], np.int32), p, M=M, dt=dt, sweeps=sweeps, tol=0.0, steps=1,
                     u0=np.zeros(2), w0=np.array([w0]), robin_eps=1.0, Cm=1.0, g_gap=0.0)
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=sweeps, cg_rtol=1e-15)
    assert r["status"] == 0
    assert np.all(r["u"] == 0.0)
    return r["w"][0]


STIFF = dict(ga=8.0, gs=8.0, a=0.15, eps=1.0, mu1=0.0, mu2=0.3, cw=1.0)
NONLINEAR = dict(ga=8.0, gs=8.0, a=0.15, eps=0.8, mu1=1.5, mu2=0.3, cw=1.0)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_stiff_gating_sweep_reaches_collocation_in_exactly_M_sweeps(M):
    dt, w0 = 1e9, 0.6          # z = dt lam = -1e9
    lam = -STIFF["cw"] * STIFF["eps"]
    ref = _collocation_linear(M, lam, dt, w0)
    after_M = _mono_nodes(STIFF, M, w0, dt, M)
    after_Mm1 = _mono_nodes(STIFF, M, w0, dt, M - 1)
    # E(z) = I - L^T + O(1/z): E^M = O(1/z), E^(M-1) applied to ~w0 1 is O(1)
    assert np.abs(after_M - ref).max() <= 1e-6 * w0
    assert np.abs(after_Mm1 - ref).max() >= 1e-3 * w0
    # and the collocation solution itself is ~0 (L-stability): the check is on
    # the approach, not on a value the predictor already holds
    assert np.abs(ref).max() <= 1e-6 * w0


@pytest.mark.parametrize("M", [2, 3, 4])
def test_stiff_gating_sweep_cell_by_cell_pair(M):
    dt, w0 = 1e9, 0.6
    lam = -STIFF["cw"] * STIFF["eps"]
    ref = _collocation_linear(M, lam, dt, w0)[-1]
    # the last node's row of I - L^T is zero, so the last node is already at the
    # limit after one sweep when the coupling is the LU trick's
    for k in range(1, M + 1):
        assert abs(_emi_last(STIFF, M, w0, dt, k) - ref) <= 1e-6 * w0


@pytest.mark.parametrize("M", [2, 3, 4])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_nonlinear_gating_sweeps_match_dense_lower_triangular_solves(M, sweeps):
    dt, w0 = 0.4, 0.9
    ref = _dense_sweeps(NONLINEAR, M, w0, dt, sweeps)
    got = _mono_nodes(NONLINEAR, M, w0, dt, sweeps)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)
    if sweeps >= 2:
        # the nodes' Jacobians differ in the sweeps checked here, so the order
        # of d and Qhat in the coupling matters
        g, d = _R(NONLINEAR, _dense_sweeps(NONLINEAR, M, w0, dt, sweeps - 1))
        assert np.ptp(d) > 0.05


@pytest.mark.parametrize("M", [2, 3, 4])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_nonlinear_gating_sweeps_cell_by_cell_pair(M, sweeps):
    dt, w0 = 0.4, 0.9
    ref = _dense_sweeps(NONLINEAR, M, w0, dt, sweeps)[-1]
    assert _emi_last(NONLINEAR, M, w0, dt, sweeps) == pytest.approx(ref, abs=1e-14)
