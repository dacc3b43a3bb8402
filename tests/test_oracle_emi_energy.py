"""Pins of the energy-norm termination (Sec. 3.2) in the oracle's cell-by-cell
(EMI) step: the sweep energy is E_k = sum_m du_m' A~_m du_m with A~_m the node
system B + c_m (A + G_m) of the EMI operator, and the sweeps end once E_k is at
most ((1 - rho) / rho * TOL)^2.

Expected values come from the EMI matrices assembled densely here from the
pair list (membrane capacitance B, gap-junction conductance G, Robin term)
and a dense solve (numpy), and from the plain run for TOL = 0.
"""

import numpy as np
import pytest

import oracle
from workloads.emi import emi_tiny

ZERO_REACTION = dict(ga=0.0, gs=0.0, a=0.15, eps=0.002, mu1=0.2, mu2=50.0, cw=1.0)


def _pair_matrix(wl, weight):
    P = np.zeros((wl.n, wl.n))
    for k, l, a, wq in zip(wl.pair_k, wl.pair_l, wl.pair_area, weight):
        e = np.zeros(wl.n)
        e[k], e[l] = 1.0, -1.0
        P += a * wq * np.outer(e, e)
    return P


def test_first_sweep_energy_is_the_dense_emi_energy_norm():
    """M = 1, ionic current 0 (w = 0, g_a = 0), gap junctions of conductance g:
    sweep 0 solves (B + dt (A + G)) du = -dt (A + G) u0, so E_0 = b' A~^-1 b."""
    wl = emi_tiny("grid")
    wl.M, wl.ionic, wl.g_gap = 1, dict(ZERO_REACTION), 0.7
    wl.w0 = np.zeros(wl.n_pairs)
    assert (wl.pair_kind == 1).any() and wl.robin.max() > 0
    S = oracle.System.from_mesh(wl.mesh)
    K, _ = S.dense()
    A = K + np.diag(wl.robin)
    B = _pair_matrix(wl, np.full(wl.n_pairs, wl.Cm))
    G = _pair_matrix(wl, np.where(wl.pair_kind == 1, wl.g_gap, 0.0))
    dt = 0.05
    wl.dt = dt
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=1, tol=0.0, cg_rtol=1e-15)
    assert r["status"] == 0
    At = B + dt * (A + G)
    b = -dt * (A + G) @ wl.u0
    ref = b @ np.linalg.solve(At, b)
    assert ref > 0
    assert r["stats"].energy[0] == pytest.approx(ref, rel=1e-10)


def test_emi_tol_zero_never_stops_early_and_matches_plain_sdc():
    wl = emi_tiny("two_cells")
    S = oracle.System.from_mesh(wl.mesh)
    a = S.step_emi(wl, wl.u0, wl.w0, sweeps=6, tol=0.0, cg_rtol=1e-13)
    b = S.step_emi(wl, wl.u0, wl.w0, sweeps=6, tol=0.0, cg_rtol=1e-13, energy_stop=True, rho=0.3)
    assert b["stats"].sweeps_run == 6
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["w"], b["w"])
    e = [b["stats"].energy[k] for k in range(6)]
    assert all(x > 0 for x in e) and e[-1] < e[0]


def test_emi_huge_tolerance_stops_after_one_sweep_with_a_given_rho():
    """alpha = 0 keeps every dof active, so only the energy test ends the step;
    with an estimated rho the first sweep can never end it."""
    wl = emi_tiny("two_cells")
    S = oracle.System.from_mesh(wl.mesh)
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=6, tol=1e6, alpha=0.0, cg_rtol=1e-13,
                   energy_stop=True, rho=0.3)
    assert r["stats"].sweeps_run == 1
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=6, tol=1e6, alpha=0.0, cg_rtol=1e-13,
                   energy_stop=True, rho=0.0)
    assert r["stats"].sweeps_run == 2


def test_emi_stop_sweep_is_the_first_to_meet_the_bound():
    wl = emi_tiny("grid")
    S = oracle.System.from_mesh(wl.mesh)
    full = S.step_emi(wl, wl.u0, wl.w0, sweeps=12, tol=0.0, cg_rtol=1e-13)
    e = np.array([full["stats"].energy[k] for k in range(12)])
    rho, tol = 0.5, 1e-4
    lim2 = ((1 - rho) / rho * tol) ** 2
    first = int(np.argmax(e <= lim2))
    assert e[first] <= lim2 and 0 < first < 11
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=12, tol=tol, alpha=0.0, cg_rtol=1e-13,
                   energy_stop=True, rho=rho)
    assert r["stats"].sweeps_run == first + 1
    np.testing.assert_allclose([r["stats"].energy[k] for k in range(first + 1)], e[:first + 1],
                               rtol=1e-12)
