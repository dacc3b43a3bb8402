"""Pins of the implicit-Euler preconditioner of the sweeps (Sec. 3.1: the
right-looking rectangle rule, a bidiagonal S-hat; in cumulative form
Qhat_mj = tau_j - tau_{j-1} for j <= m).

Expected values: the dense Newton solve of the collocation system (any
lower-triangular Qhat has the collocation solution as its fixed point); the
M = 1 case, where both preconditioners are [[1]]; and the ordering of the
contraction on stiff diffusion that the LU trick is chosen for.
"""

import numpy as np
import pytest

import oracle
import workloads as W

ZERO_REACTION = dict(ga=0.0, gs=0.0, a=0.15, eps=0.002, mu1=0.2, mu2=50.0, cw=1.0)


@pytest.mark.parametrize("kind", ["2d3", "3d2"])
@pytest.mark.parametrize("M", [2, 3, 4])
def test_converged_implicit_euler_sdc_equals_collocation_solve(kind, M):
    wl = W.tiny(kind)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    istim = np.zeros(wl.n)
    istim[wl.n // 2] = 1.5
    r = S.step(wl.ionic, M, wl.v0, wl.w0, 0.05, 60, 0.0, cg_rtol=1e-14, istim=istim,
               want_nodes=True, qhat="ie")
    d = S.collocation_solve(wl.ionic, M, wl.v0, wl.w0, 0.05, istim=istim)
    assert r["status"] == 0 and d["status"] == 0
    assert np.abs(r["V"] - d["V"]).max() <= 1e-12 * max(1.0, np.abs(d["V"]).max())
    assert np.abs(r["W"] - d["W"]).max() <= 1e-12 * max(1.0, np.abs(d["W"]).max())


def test_one_node_preconditioners_coincide():
    wl = W.tiny("2d3")
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    a = S.step(wl.ionic, 1, wl.v0, wl.w0, 0.1, 3, 0.0, cg_rtol=1e-13, qhat="lu")
    b = S.step(wl.ionic, 1, wl.v0, wl.w0, 0.1, 3, 0.0, cg_rtol=1e-13, qhat="ie")
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["w"], b["w"])


def _sweeps_to(S, M, v0, dt, qhat, target, ref):
    for k in range(1, 60):
        r = S.step(ZERO_REACTION, M, v0, np.zeros_like(v0), dt, k, 0.0, cg_rtol=1e-15, qhat=qhat)
        if np.abs(r["v"] - ref).max() <= target:
            return k
    return 60


def test_lu_trick_contracts_faster_than_implicit_euler_on_stiff_diffusion():
    mesh = W.grid2d(11, 11, 0.25)
    S = oracle.System.from_mesh(mesh, np.eye(3))
    v0 = np.exp(-((mesh.xyz[:, 0] - 1.2) ** 2 + (mesh.xyz[:, 1] - 1.0) ** 2) * 4.0)
    M, dt = 3, 1.0          # dt D / h^2 = 16: stiff
    ref = S.collocation_solve(ZERO_REACTION, M, v0, np.zeros_like(v0), dt)["v"]
    k_lu = _sweeps_to(S, M, v0, dt, "lu", 1e-10, ref)
    k_ie = _sweeps_to(S, M, v0, dt, "ie", 1e-10, ref)
    assert k_lu < 60 and k_ie < 60
    assert k_lu < k_ie
