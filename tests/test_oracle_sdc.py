"""Pins of the oracle's SDC step (Sec. 3.1-3.2, eq. SDC and eq. final-sdc) and
of its nested active sets (Sec. 4.2).

Expected values come from: the dense Newton solve of the collocation system
(the SDC fixed point), the Pade(M-1, M) stability function of Radau-IIA, the
matrix exponential (scipy) for the semi-discrete diffusion problem, an RK4
reference for the pointwise ionic ODE, dense linear solves (numpy) for single
sweeps, conservation of sum(m v) and the set-nesting invariants.
"""

import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W

# no ionic current and no gating dynamics (w stays 0); mu2 large so that the
# gating rate has no pole in the voltage range of the linear tests
ZERO_REACTION = dict(ga=0.0, gs=0.0, a=0.15, eps=0.002, mu1=0.2, mu2=50.0, cw=1.0)


# ------------------------------------------------------------------ fixed point
@pytest.mark.parametrize("kind", ["2d3", "2d5", "3d2", "3d3"])
@pytest.mark.parametrize("M", [2, 3, 4])
def test_converged_sdc_equals_direct_collocation_solve(kind, M):
    wl = W.tiny(kind)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    istim = np.zeros(wl.n)
    istim[wl.n // 2] = 1.5
    r = S.step(wl.ionic, M, wl.v0, wl.w0, 0.05, 60, 0.0, cg_rtol=1e-14, istim=istim, want_nodes=True)
    d = S.collocation_solve(wl.ionic, M, wl.v0, wl.w0, 0.05, istim=istim)
    assert r["status"] == 0 and d["status"] == 0
    assert d["newton_iters"] < 20
    scale = max(1.0, np.abs(d["V"]).max())
    assert np.abs(r["V"] - d["V"]).max() <= 1e-12 * scale
    assert np.abs(r["W"] - d["W"]).max() <= 1e-12 * max(1.0, np.abs(d["W"]).max())
    # the converged state moved: the check is not trivially satisfied by v0
    assert np.abs(d["V"][-1] - wl.v0).max() > 1e-3


# ------------------------------------------------------------ scalar test problem
def _scalar_system(kappa):
    return oracle.System.from_matrix([0, 1], [0], [kappa], [1.0])


def _pade(M, z):
    f = math.factorial
    num = sum(f(2 * M - 1 - j) * f(M - 1) / (f(2 * M - 1) * f(j) * f(M - 1 - j)) * z ** j
              for j in range(M))
    den = sum(f(2 * M - 1 - j) * f(M) / (f(2 * M - 1) * f(j) * f(M - j)) * (-z) ** j
              for j in range(M + 1))
    return num / den


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("z", [-0.1, -1.0, -5.0, -40.0])
def test_scalar_stability_function_is_pade(M, z):
    # v' = -kappa v with m = 1: one step of converged SDC gives R(z) v0, z = -kappa dt
    dt = 0.1
    S = _scalar_system(-z / dt)
    r = S.step(ZERO_REACTION, M, [1.0], [0.0], dt, 60, 0.0, cg_rtol=1e-15)
    assert r["status"] == 0
    assert r["v"][0] == pytest.approx(_pade(M, z), rel=1e-12, abs=1e-15)
    assert r["w"][0] == 0.0


def test_scalar_pade_m3_closed_form():
    z = -2.5
    R = (1 + 2 * z / 5 + z * z / 20) / (1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60)
    assert _pade(3, z) == pytest.approx(R, rel=1e-15)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_stiff_limit_converges_in_M_sweeps(M):
    # LU trick: E = I - Qhat^{-1} Q is nilpotent, so a very stiff scalar problem
    # is solved after M sweeps up to O(1/|z|)
    dt = 0.1
    z = -1e9
    S = _scalar_system(-z / dt)
    r = S.step(ZERO_REACTION, M, [1.0], [0.0], dt, M, 0.0, cg_rtol=1e-15)
    assert abs(r["v"][0] - _pade(M, z)) < 1e-7


def test_sweeps_contract_towards_collocation():
    dt, z = 0.1, -2.0
    S = _scalar_system(-z / dt)
    errs = []
    for k in range(1, 9):
        r = S.step(ZERO_REACTION, 3, [1.0], [0.0], dt, k, 0.0, cg_rtol=1e-15)
        errs.append(abs(r["v"][0] - _pade(3, z)))
    assert all(errs[i + 1] < 0.7 * errs[i] for i in range(6))


# ----------------------------------------------------------------- time order
def _diffusion_setup():
    mesh = W.grid2d(9, 9, 0.125)
    S = oracle.System.from_mesh(mesh, 0.003 * np.eye(3))
    K, m = S.dense()
    x, y = mesh.xyz[:, 0], mesh.xyz[:, 1]
    v0 = np.cos(np.pi * x) * np.cos(np.pi * y) + 0.3 * x
    return S, K, m, v0


@pytest.mark.parametrize("M,sweeps,order", [(2, 40, 3), (3, 40, 5), (3, 2, 2)])
def test_observed_time_order_on_diffusion(M, sweeps, order):
    """v' = -m^{-1} K v, exact solution by the matrix exponential (non-stiff
    regime: dt * lambda_max < 1).  Converged SDC shows order 2M-1; with a fixed
    number of sweeps from the spread predictor it shows min(sweeps, 2M-1)."""
    S, K, m, v0 = _diffusion_setup()
    T = 1.6
    exact = scipy.linalg.expm(-T * (K / m[:, None])) @ v0
    lam = np.max(np.abs(np.linalg.eigvals(K / m[:, None])))
    errs = []
    dts = [0.4, 0.2, 0.1]
    for dt in dts:
        assert dt * lam < 1.5
        v, w = v0.copy(), np.zeros_like(v0)
        for _ in range(int(round(T / dt))):
            r = S.step(ZERO_REACTION, M, v, w, dt, sweeps, 0.0, cg_rtol=1e-15)
            assert r["status"] == 0
            v, w = r["v"], r["w"]
        errs.append(np.abs(v - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > order - 0.4, (errs, rates)
    assert max(rates) < order + 0.8, (errs, rates)


def _rk4_ap(p, v, w, T, n):
    def rhs(v, w):
        I = p["ga"] * v * (v - p["a"]) * (v - 1) + v * w
        R = p["cw"] * (p["eps"] + p["mu1"] * w / (v + p["mu2"])) * (-w - p["gs"] * v * (v - p["a"] - 1))
        return -I, R
    h = T / n
    for _ in range(n):
        k1 = rhs(v, w)
        k2 = rhs(v + h / 2 * k1[0], w + h / 2 * k1[1])
        k3 = rhs(v + h / 2 * k2[0], w + h / 2 * k2[1])
        k4 = rhs(v + h * k3[0], w + h * k3[1])
        v += h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        w += h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return v, w


def test_observed_time_order_on_ionic_ode():
    """One dof, no diffusion: v' = -I_ion(v, w), w' = R(v, w); RK4 reference."""
    p = dict(W.AP_PAPER)
    S = oracle.System.from_matrix([0, 1], [0], [0.0], [1.0])
    T = 0.8
    v_ref, w_ref = _rk4_ap(p, 0.4, 0.05, T, 64000)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        v, w = np.array([0.4]), np.array([0.05])
        for _ in range(int(round(T / dt))):
            r = S.step(p, 3, v, w, dt, 40, 0.0, cg_rtol=1e-15)
            assert r["status"] == 0
            v, w = r["v"], r["w"]
        errs.append(max(abs(v[0] - v_ref), abs(w[0] - w_ref)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4.3, (errs, rates)


# ----------------------------------------------------- single sweeps by dense algebra
def test_one_sweep_m1_is_linearised_implicit_euler():
    """M = 1, one sweep: (diag(m (1 + dt J)) + dt K) dv = dt f(v0)."""
    wl = W.tiny("2d5")
    p = wl.ionic
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    K, m = S.dense()
    rng = np.random.default_rng(1)
    v0 = rng.uniform(0, 1, wl.n)
    w0 = rng.uniform(0, 0.5, wl.n)
    ev = np.array([oracle.ionic_eval(p, a, b) for a, b in zip(v0, w0)])
    dt = 0.07
    f = -K @ v0 - m * ev[:, 0]
    A = np.diag(m * (1 + dt * ev[:, 1])) + dt * K
    dv = np.linalg.solve(A, dt * f)
    r = S.step(p, 1, v0, w0, dt, 1, 0.0, cg_rtol=1e-15)
    np.testing.assert_allclose(r["v"], v0 + dv, rtol=0, atol=1e-13)
    # w: one pointwise linearised implicit-Euler step with the new v
    v1 = v0 + dv
    ev1 = np.array([oracle.ionic_eval(p, a, b) for a, b in zip(v1, w0)])
    dw = dt * ev1[:, 3] / (1 - dt * ev1[:, 5])
    np.testing.assert_allclose(r["w"], w0 + dw, rtol=0, atol=1e-14)


def test_restricted_sweep_holds_inactive_dofs_fixed():
    """Second sweep on I_1: the restricted system has homogeneous Dirichlet
    values on the dropped dofs (Theorem 1), solved densely here."""
    wl = W.tiny("2d5")
    p = wl.ionic
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    K, m = S.dense()
    v0 = np.zeros(wl.n)
    v0[:3] = [1.0, 0.8, 0.5]
    w0 = np.zeros(wl.n)
    dt, tol, alpha = 0.05, 0.12, 0.1
    r1 = S.step(p, 1, v0, w0, dt, 1, 0.0, cg_rtol=1e-15)
    dv1 = r1["v"] - v0
    act = np.nonzero(np.abs(dv1) >= alpha * tol)[0]
    assert 0 < act.size < wl.n
    # residual at the one-sweep iterate, restricted dense solve on act
    v1, w1 = r1["v"], r1["w"]
    ev = np.array([oracle.ionic_eval(p, a, b) for a, b in zip(v1, w1)])
    f = -K @ v1 - m * ev[:, 0]
    res = m * v0 + dt * f - m * v1
    A = np.diag(m * (1 + dt * ev[:, 1])) + dt * K
    dv2 = np.zeros(wl.n)
    dv2[act] = np.linalg.solve(A[np.ix_(act, act)], res[act])
    r2 = S.step(p, 1, v0, w0, dt, 2, tol, alpha=alpha, cg_rtol=1e-15, want_log=True)
    assert r2["active"][1].tolist() == act.tolist()
    np.testing.assert_allclose(r2["v"], v1 + dv2, rtol=0, atol=1e-13)
    dropped = np.setdiff1d(np.arange(wl.n), act)
    assert np.array_equal(r2["v"][dropped], v1[dropped])
    assert np.array_equal(r2["w"][dropped], w1[dropped])


# --------------------------------------------------------- adaptivity invariants
@pytest.fixture(scope="module")
def w0sys():
    wl = W.w0_square()
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0, wl.w0
    for n in range(6):   # move into a propagating front
        r = S.step(wl.ionic, 3, v, w, wl.dt, 4, 0.0)
        v, w = r["v"], r["w"]
    return wl, S, v, w


def test_tol_zero_equals_plain(w0sys):
    wl, S, v, w = w0sys
    a = S.step(wl.ionic, 3, v, w, wl.dt, 4, 0.0, alpha=0.1, want_log=True)
    b = S.step(wl.ionic, 3, v, w, wl.dt, 4, 0.0, alpha=0.0)
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["w"], b["w"])
    assert all(len(x) == wl.n for x in a["active"])


def test_tol_infinite_equals_one_sweep(w0sys):
    wl, S, v, w = w0sys
    a = S.step(wl.ionic, 3, v, w, wl.dt, 4, 1e300)
    b = S.step(wl.ionic, 3, v, w, wl.dt, 1, 0.0)
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["w"], b["w"])
    assert list(a["stats"].n_active[:4]) == [wl.n, 0, 0, 0]


def test_nested_sets_and_frozen_rows(w0sys):
    wl, S, v, w = w0sys
    runs = [S.step(wl.ionic, 3, v, w, wl.dt, k, wl.tol, want_log=True, want_nodes=True)
            for k in range(1, 5)]
    act = runs[-1]["active"]
    assert act[0].tolist() == list(range(wl.n))
    for k in range(3):
        assert np.all(np.diff(act[k + 1]) > 0)
        assert set(act[k + 1].tolist()) <= set(act[k].tolist())
    assert len(act[1]) < wl.n // 2 and len(act[3]) <= len(act[2]) <= len(act[1])
    # dofs outside I_{k+1} are unchanged by sweep k+1 (all collocation nodes)
    for k in range(3):
        out = np.setdiff1d(np.arange(wl.n), act[k + 1])
        assert np.array_equal(runs[k + 1]["V"][:, out], runs[k]["V"][:, out])
        assert np.array_equal(runs[k + 1]["W"][:, out], runs[k]["W"][:, out])


def test_conservation_without_reaction():
    """No reaction, Neumann boundary: sum(m v) is invariant (K has zero row sums)."""
    wl = W.w0_square()
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    _, _, _, m = S.matrix()
    v, w = wl.v0.copy(), wl.w0.copy()
    tot0 = m @ v
    for _ in range(5):
        r = S.step(ZERO_REACTION, 3, v, w, wl.dt, 4, 0.0, cg_rtol=1e-13)
        assert r["status"] == 0
        v, w = r["v"], r["w"]
    assert abs(m @ v - tot0) <= 1e-10 * abs(tot0)


@pytest.mark.slow
def test_adaptive_accuracy_and_shrinking_sets():
    """Qualitative facts of Sec. 5.2 on the 2D square: sets shrink after the
    first sweep; the adaptive error stays below the SDC tolerance TOL
    (Theorem 2's requirement) and, with TOL small enough to sit on the sweet
    line, it is as accurate as plain SDC."""
    wl = W.w0_square()
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    steps = 30

    def run(sweeps, tol):
        v, w = wl.v0.copy(), wl.w0.copy()
        counts = np.zeros(sweeps)
        for _ in range(steps):
            r = S.step(wl.ionic, 3, v, w, wl.dt, sweeps, tol)
            assert r["status"] == 0
            v, w = r["v"], r["w"]
            counts += np.array(r["stats"].n_active[:sweeps])
        return v, counts / steps

    ref, _ = run(12, 0.0)
    plain, _ = run(4, 0.0)
    err_plain = np.abs(plain - ref).max()
    for tol in (1e-4, 1e-5):
        adapt, c = run(4, tol)
        err_adapt = np.abs(adapt - ref).max()
        assert err_adapt <= tol
        assert c[0] == wl.n and c[1] < 0.5 * wl.n and c[2] <= c[1] and c[3] <= c[2]
    assert err_adapt <= 1.1 * err_plain
