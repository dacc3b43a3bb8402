"""Pins of the oracle's tangent step (forward mode, dual numbers) used to check
the library's discrete adjoint: with the active sets given, it is the derivative
of ora_step_forced along a direction of the initial state, of the ionic
parameters and of the conductivity scale.

Expected values come from the primal oracle itself, through definitions that do
not share the tangent's arithmetic: second-order central differences of the
forced-set step, and linearity of the derivative in the direction.
"""

import numpy as np
import pytest

import oracle
import workloads as W


def _case():
    rng = np.random.default_rng(7)
    wl = W.w0_square(tol=1e-3, n=13, length=3.75)
    wl.sweeps, wl.dt = 4, 0.1
    scale = 1.0 + 0.1 * rng.standard_normal(wl.n)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, scale)
    # a state with a front and its adaptive sets
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(2):
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, cg_rtol=1e-14)
        v, w = r["v"], r["w"]
    r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, cg_rtol=1e-14, want_log=True)
    lists = [None] + [r["active"][k] for k in range(1, wl.sweeps)]
    assert 0 < len(lists[-1]) < wl.n          # the sets really shrink
    return wl, scale, S, v, w, lists, rng


def _fwd(wl, scale, v, w, lists, ionic=None):
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, scale)
    r = S.step_forced(ionic or wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, lists, cg_rtol=1e-14)
    assert r["status"] == 0
    return r["v"], r["w"]


def test_tangent_value_part_is_the_forced_step_bitwise():
    wl, scale, S, v, w, lists, rng = _case()
    t = S.step_tangent(wl.ionic, wl.M, v, rng.standard_normal(wl.n), w, np.zeros(wl.n), wl.dt,
                       wl.sweeps, lists, cg_rtol=1e-14)
    assert t["status"] == 0
    fv, fw = _fwd(wl, scale, v, w, lists)
    assert np.array_equal(t["v"], fv) and np.array_equal(t["w"], fw)


@pytest.mark.parametrize("what", ["v0", "w0", "scale", "k", "a"])
def test_tangent_matches_central_differences(what):
    wl, scale, S, v, w, lists, rng = _case()
    dv, dw, ds = np.zeros(wl.n), np.zeros(wl.n), None
    dion = None
    if what == "v0":
        dv = rng.standard_normal(wl.n) * 0.1
    elif what == "w0":
        dw = rng.standard_normal(wl.n) * 0.01
    elif what == "scale":
        ds = rng.standard_normal(wl.n)
    else:
        dion = {k: 0.0 for k in wl.ionic}
        if what == "k":
            dion["ga"] = dion["gs"] = 1.0
        else:
            dion["a"] = 1.0
    Sd = oracle.System.from_mesh(wl.mesh, wl.sigma, ds) if ds is not None else None
    t = S.step_tangent(wl.ionic, wl.M, v, dv, w, dw, wl.dt, wl.sweeps, lists, dionic=dion,
                       dscale_system=Sd, cg_rtol=1e-14)
    assert t["status"] == 0

    def at(h):
        ion = dict(wl.ionic)
        if dion is not None:
            for k in ion:
                ion[k] = ion[k] + h * dion[k]
        sc = scale + h * ds if ds is not None else scale
        return _fwd(wl, sc, v + h * dv, w + h * dw, lists, ion)

    h = 1e-5
    (vp, wp), (vm, wm) = at(h), at(-h)
    fdv, fdw = (vp - vm) / (2 * h), (wp - wm) / (2 * h)
    nv = max(np.abs(fdv).max(), 1e-12)
    assert np.abs(fdv).max() > 1e-6
    assert np.abs(t["dv"] - fdv).max() <= 1e-6 * nv
    assert np.abs(t["dw"] - fdw).max() <= 1e-6 * max(np.abs(fdw).max(), nv)


def test_tangent_is_linear_in_the_direction():
    wl, scale, S, v, w, lists, rng = _case()
    d1, d2 = rng.standard_normal(wl.n), rng.standard_normal(wl.n)
    z = np.zeros(wl.n)
    t1 = S.step_tangent(wl.ionic, wl.M, v, d1, w, z, wl.dt, wl.sweeps, lists, cg_rtol=1e-14)
    t2 = S.step_tangent(wl.ionic, wl.M, v, d2, w, z, wl.dt, wl.sweeps, lists, cg_rtol=1e-14)
    t3 = S.step_tangent(wl.ionic, wl.M, v, d1 + 2 * d2, w, z, wl.dt, wl.sweeps, lists,
                        cg_rtol=1e-14)
    ref = t1["dv"] + 2 * t2["dv"]
    assert np.abs(t3["dv"] - ref).max() <= 1e-9 * np.abs(ref).max()
