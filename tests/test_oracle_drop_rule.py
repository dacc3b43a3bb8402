"""Pins of the oracle's a priori drop tolerance (Sec. 4.1, Eq. drop-tolerance
with Theorems 1 and 2): TOL_drop = exp(-eta dt) (1 - rho) / (r + 1) TOL, with
c = ||dv^0||_inf from the first sweep, r the fewest sweeps with c rho^r <=
(1 - rho) TOL (Eq. r-condition), eta = max(0, -min dI/dv) / C_m.

Expected values come from: the first correction dv^0 read off a one-sweep run
(node values minus the spread start), r found by counting sweeps of the
geometric bound, and dI/dv by central differences of the Aliev-Panfilov
current I = g_a v (v - a)(v - 1) + v w (exact up to h^2 g_a for a cubic).
"""

import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.emi import emi_tiny


def _didv_fd(p, v, w, h=1e-5):
    cur = lambda x: p["ga"] * x * (x - p["a"]) * (x - 1.0) + x * w
    return (cur(v + h) - cur(v - h)) / (2 * h)


def _expected(c, neg_jmin, Cm, rho, tol, dt):
    r = 0
    while c * rho ** r > (1 - rho) * tol:
        r += 1
    return math.exp(-max(0.0, neg_jmin) / Cm * dt) * (1 - rho) / (r + 1) * tol, r


def _square():
    mesh = W.grid2d(17, 17, 0.3)
    x, y = mesh.xyz[:, 0], mesh.xyz[:, 1]
    v0 = np.exp(-((x - 1.5) ** 2 + (y - 2.0) ** 2) / 2.0)   # spans (0, 1]: dI/dv < 0 near 0.38
    w0 = np.full(mesh.n_nodes, 0.02)
    return mesh, v0, w0


@pytest.mark.parametrize("rho,tol", [(0.05, 1e-4), (0.3, 1e-6)])
def test_monodomain_drop_tolerance_is_the_a_priori_formula(rho, tol):
    mesh, v0, w0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    p, M, dt = W.AP_BENCH, 3, 0.1
    one = S.step(p, M, v0, w0, dt, 1, 0.0, cg_rtol=1e-13, want_nodes=True)
    c = np.abs(one["V"] - v0[None, :]).max()
    neg_jmin = max(0.0, -min(_didv_fd(p, v, w) for v, w in zip(v0, w0)))
    assert neg_jmin > 1.0                 # the exp(-eta dt) factor is exercised
    ref, r = _expected(c, neg_jmin, 1.0, rho, tol, dt)
    assert r >= 1
    out = S.step(p, M, v0, w0, dt, 4, tol, cg_rtol=1e-13, drop_rule=1, rho=rho)
    assert out["status"] == 0
    assert out["stats"].tol_drop == pytest.approx(ref, rel=1e-9)


def test_drop_rule_selects_like_alpha_tol_of_the_same_value():
    mesh, v0, w0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    p, M, dt, tol = W.AP_BENCH, 3, 0.1, 1e-4
    a = S.step(p, M, v0, w0, dt, 5, tol, cg_rtol=1e-13, drop_rule=1, rho=0.05, want_log=True)
    td = a["stats"].tol_drop
    assert 0 < td < tol and a["stats"].n_active[4] < mesh.n_nodes
    b = S.step(p, M, v0, w0, dt, 5, tol, alpha=td / tol, cg_rtol=1e-13, want_log=True)
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["w"], b["w"])
    for la, lb in zip(a["active"], b["active"]):
        assert np.array_equal(la, lb)


def test_drop_rule_special_cases():
    mesh, v0, w0 = _square()
    S = oracle.System.from_mesh(mesh, np.eye(3))
    p = W.AP_BENCH
    plain = S.step(p, 3, v0, w0, 0.1, 3, 0.0, cg_rtol=1e-13)
    r = S.step(p, 3, v0, w0, 0.1, 3, 0.0, cg_rtol=1e-13, drop_rule=1, rho=0.05)
    assert r["stats"].tol_drop == 0.0 and np.array_equal(r["v"], plain["v"])
    # a state at rest (v = w = 0, no stimulus) has c = 0: r = 0, eta from dI/dv(0, 0) = g_a a > 0
    z = np.zeros(mesh.n_nodes)
    r = S.step(p, 3, z, z, 0.1, 3, 1e-4, cg_rtol=1e-13, drop_rule=1, rho=0.05)
    assert r["stats"].tol_drop == pytest.approx(0.95e-4, rel=1e-15)
    # the rule needs a given contraction
    assert S.step(p, 3, v0, w0, 0.1, 3, 1e-4, drop_rule=1, rho=0.0)["status"] != 0


@pytest.mark.parametrize("Cm", [1.0, 2.5])
def test_emi_drop_tolerance_uses_the_membrane_jacobian_over_cm(Cm):
    """eta = max(0, -min over the pairs of dI_p/dv) / C_m: (1 - rho) TOL
    exp(-eta dt) / TOL_drop is the integer r + 1, and r is at least the count
    the step-end correction alone gives (c is the max over all nodes)."""
    wl = emi_tiny("two_cells")
    wl.Cm = Cm
    wl.u0 = np.where(wl.u0 > 0.5, 0.4, 0.0)   # membrane voltage 0.4: dI/dv < 0 there
    wl.w0 = np.full(wl.n_pairs, 0.01)
    S = oracle.System.from_mesh(wl.mesh)
    vpair = wl.u0[wl.pair_k] - wl.u0[wl.pair_l]
    J = [_didv_fd(wl.ionic, v, w) if kd == 0 else wl.g_gap
         for v, w, kd in zip(vpair, wl.w0, wl.pair_kind)]
    neg_jmin = max(0.0, -min(J))
    assert neg_jmin > 0.5
    rho, tol = 0.1, 1e-5
    r = S.step_emi(wl, wl.u0, wl.w0, sweeps=3, tol=tol, cg_rtol=1e-13, drop_rule=1, rho=rho)
    assert r["status"] == 0
    td = r["stats"].tol_drop
    q = (1 - rho) * tol * math.exp(-neg_jmin / Cm * wl.dt) / td
    assert abs(q - round(q)) <= 1e-9 * q and round(q) >= 1
    one = S.step_emi(wl, wl.u0, wl.w0, sweeps=1, tol=0.0, cg_rtol=1e-13)
    _, r_end = _expected(np.abs(one["u"] - wl.u0).max(), neg_jmin, Cm, rho, tol, wl.dt)
    assert round(q) - 1 >= r_end >= 1
    # the rule feeds the selection exactly like alpha TOL of the same value
    a = S.step_emi(wl, wl.u0, wl.w0, sweeps=4, tol=tol, cg_rtol=1e-13, drop_rule=1, rho=rho,
                   want_log=True)
    b = S.step_emi(wl, wl.u0, wl.w0, sweeps=4, tol=tol, cg_rtol=1e-13, alpha=td / tol,
                   want_log=True)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["w"], b["w"])
    assert [x.tolist() for x in a["active"]] == [x.tolist() for x in b["active"]]
