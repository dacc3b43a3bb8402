"""Pins of the oracle's energy-norm termination of the SDC sweeps (Sec. 3.2):
the sweeps end once E_k = sum_m dv_m' A~_m dv_m, with A~_m the node system
matrix, is at most ((1 - rho) / rho * TOL)^2.

Expected values come from: a dense solve (numpy) for the energy of a single
linear sweep, the collocation solution of the dense Newton solver for the
error bound the stop is meant to guarantee, and the plain run for TOL = 0.
"""

import numpy as np
import pytest

import oracle
import workloads as W

ZERO_REACTION = dict(ga=0.0, gs=0.0, a=0.15, eps=0.002, mu1=0.2, mu2=50.0, cw=1.0)


def _square(n=9, length=2.5):
    mesh = W.grid2d(n, n, length / (n - 1))
    v0 = np.exp(-((mesh.xyz[:, 0] - 0.8) ** 2 + (mesh.xyz[:, 1] - 1.1) ** 2) * 3.0)
    return mesh, v0


def test_first_sweep_energy_is_the_dense_energy_norm():
    """M = 1, no reaction: sweep 0 solves (diag(m) + dt K) dv = -dt K v0, so
    E_0 = b' A~^-1 b with b = -dt K v0."""
    mesh, v0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    K, mass = S.dense()
    dt = 0.3
    r = S.step(ZERO_REACTION, 1, v0, np.zeros_like(v0), dt, 1, 0.0, cg_rtol=1e-15)
    assert r["status"] == 0
    A = np.diag(mass) + dt * K
    b = -dt * K @ v0
    ref = b @ np.linalg.solve(A, b)
    assert ref > 0
    assert r["stats"].energy[0] == pytest.approx(ref, rel=1e-12)


def test_tol_zero_never_stops_early_and_matches_plain_sdc():
    mesh, v0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    w0 = np.zeros_like(v0)
    a = S.step(W.AP_BENCH, 3, v0, w0, 0.2, 6, 0.0, cg_rtol=1e-13)
    b = S.step(W.AP_BENCH, 3, v0, w0, 0.2, 6, 0.0, cg_rtol=1e-13, energy_stop=True, rho=0.3)
    assert b["stats"].sweeps_run == 6
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["w"], b["w"])
    e = [b["stats"].energy[k] for k in range(6)]
    assert all(x > 0 for x in e) and e[-1] < e[0]


def test_huge_tolerance_stops_after_one_sweep_with_a_given_rho():
    """alpha = 0 keeps every dof active, so only the energy test ends the step."""
    mesh, v0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    r = S.step(W.AP_BENCH, 3, v0, np.zeros_like(v0), 0.2, 6, 1e6, alpha=0.0, cg_rtol=1e-13,
               energy_stop=True, rho=0.3)
    assert r["stats"].sweeps_run == 1
    # with an estimated rho the first sweep can never end the step
    r = S.step(W.AP_BENCH, 3, v0, np.zeros_like(v0), 0.2, 6, 1e6, alpha=0.0, cg_rtol=1e-13,
               energy_stop=True, rho=0.0)
    assert r["stats"].sweeps_run == 2


@pytest.mark.parametrize("tol", [1e-5, 1e-7])
def test_stop_bounds_the_energy_norm_error_of_the_collocation_solution(tol):
    """Linear diffusion (SDC contracts linearly): with rho at least the
    observed contraction, the iterate the stop accepts is within TOL of the
    collocation solution in the norm sum_m e_m' A~_m e_m (the geometric-series
    argument of Sec. 3.2), and the stop saves sweeps."""
    mesh, v0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    K, mass = S.dense()
    M, dt = 3, 0.4
    w0 = np.zeros_like(v0)
    full = S.step(ZERO_REACTION, M, v0, w0, dt, 40, 0.0, cg_rtol=1e-15)
    e = np.array([full["stats"].energy[k] for k in range(40)])
    ratios = np.sqrt(e[1:12] / e[:11])
    rho = min(0.95, 1.1 * ratios.max())
    r = S.step(ZERO_REACTION, M, v0, w0, dt, 40, tol, alpha=0.0, cg_rtol=1e-15,
               energy_stop=True, rho=rho, want_nodes=True)
    assert r["status"] == 0 and r["stats"].sweeps_run < 40
    d = S.collocation_solve(ZERO_REACTION, M, v0, w0, dt)
    _, _, Qh = oracle.collocation(M)
    err2 = 0.0
    for m in range(M):
        A = np.diag(mass) + dt * Qh[m, m] * K
        em = r["V"][m] - d["V"][m]
        err2 += em @ A @ em
    assert np.sqrt(err2) <= tol
    # one sweep fewer would not have met the bound test
    k = r["stats"].sweeps_run - 1
    lim = (1 - rho) / rho * tol
    assert r["stats"].energy[k] <= lim ** 2
    assert k == 0 or r["stats"].energy[k - 1] > lim ** 2
