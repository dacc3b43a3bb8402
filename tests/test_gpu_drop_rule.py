"""GPU parity of the a priori drop tolerance (Sec. 4.1, Eq. drop-tolerance):
the library reduces c = max |dv| and max(0, -dI/dv) of the first sweep on the
device and forms TOL_drop there; the oracle does it on the host.  Same
TOL_drop (1e-13 relative: log/exp rounding), identical active sets, states
within 1e-10."""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_07206_gb300 import build as b
    b.build()
    return torch, torch.device("cuda:0")


def _relmax(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def _slab():
    mesh = W.kuhn3d(31, 11, 6, 0.1)
    stim = np.nonzero((mesh.xyz <= 0.5 + 1e-12).all(axis=1))[0].astype(np.int32)
    return W.Workload("slab_31x11x6", mesh, np.diag([1.0, 0.25, 0.25]), dict(W.AP_BENCH), M=4,
                      dt=0.05, sweeps=5, tol=1e-5, steps=10, v0=np.zeros(mesh.n_nodes),
                      w0=np.zeros(mesh.n_nodes), stim_nodes=stim, stim_amp=2.0, stim_t_on=0.0,
                      stim_t_off=1.0)


@pytest.mark.parametrize("case,rho,variant", [("square", 0.05, 0), ("slab", 0.2, 0),
                                              ("slab", 0.05, 1), ("slab", 0.05, 2)])
def test_drop_rule_parity(torch_dev, case, rho, variant):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Context, default_options
    wl = W.w0_square() if case == "square" else _slab()
    ctx = Context.from_workload(wl, options=default_options(drop_rule=1, sdc_rho=rho,
                                                            cg_variant=variant),
                                stream=torch.cuda.current_stream(dev).cuda_stream)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    shrank = False
    for n in range(8):
        t = n * wl.dt
        dv = torch.tensor(v, dtype=torch.float64, device=dev)
        dw = torch.tensor(w, dtype=torch.float64, device=dev)
        st = ctx.step(dv, dw, t, wl.dt, wl.sweeps, wl.tol)
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, cg_rtol=wl.cg_rtol,
                   istim=wl.stim_vector(t), want_log=True, drop_rule=1, rho=rho)
        assert r["status"] == 0
        assert st.tol_drop == pytest.approx(r["stats"].tol_drop, rel=1e-13), n
        assert 0 < st.tol_drop < wl.tol
        for k in range(wl.sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k]), (n, k)
        shrank |= st.n_active[wl.sweeps - 1] < wl.n
        assert _relmax(dv.cpu().numpy(), r["v"]) <= 1e-10
        assert _relmax(dw.cpu().numpy(), r["w"]) <= 1e-10
        v, w = r["v"], r["w"]
    assert shrank
    ctx.close()


def test_drop_rule_tol_zero_is_plain(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Context, default_options
    wl = W.w0_square(n=17, length=5.0)
    ctx = Context.from_workload(wl, options=default_options(drop_rule=1, sdc_rho=0.05),
                                stream=torch.cuda.current_stream(dev).cuda_stream)
    dv = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    dw = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    st = ctx.step(dv, dw, 0.0, wl.dt, wl.sweeps, 0.0)
    assert st.tol_drop == 0.0 and list(st.n_active[:wl.sweeps]) == [wl.n] * wl.sweeps
    ctx.close()


@pytest.mark.parametrize("kind", ["two_cells", "grid"])
def test_emi_drop_rule_parity(torch_dev, kind):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Context, default_options
    from workloads.emi import emi_tiny
    wl = emi_tiny(kind)
    opts = default_options(drop_rule=1, sdc_rho=0.1, alpha=wl.alpha, cg_rtol=wl.cg_rtol,
                           cg_maxit=100000)
    ctx = Context.from_emi(wl, options=opts, stream=torch.cuda.current_stream(dev).cuda_stream)
    S = oracle.System.from_mesh(wl.mesh)
    u, w = wl.u0.copy(), wl.w0.copy()
    for n in range(3):
        du = torch.tensor(u, dtype=torch.float64, device=dev)
        dw = torch.tensor(w, dtype=torch.float64, device=dev)
        st = ctx.step(du, dw, n * wl.dt, wl.dt, wl.sweeps, wl.tol)
        r = S.step_emi(wl, u, w, want_log=True, drop_rule=1, rho=0.1)
        assert r["status"] == 0
        assert st.tol_drop == pytest.approx(r["stats"].tol_drop, rel=1e-13), n
        for k in range(wl.sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k]), (n, k)
        assert _relmax(du.cpu().numpy(), r["u"]) <= 1e-10
        assert _relmax(dw.cpu().numpy(), r["w"]) <= 1e-10
        u, w = r["u"], r["w"]
    ctx.close()
