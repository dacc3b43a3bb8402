"""The reorder option: the library numbers the dofs internally in Morton order
and maps everything back at its boundary.  Parity with the oracle (in the
caller's numbering) at 1e-10, active lists identical, node values, the
assembled matrix and the conductivity scale in the caller's numbering."""

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


def _ctx(wl, torch, dev, **opts):
    from paper_2311_07206_gb300 import Context, default_options
    return Context.from_workload(wl, options=default_options(**opts),
                                 stream=torch.cuda.current_stream(dev).cuda_stream)


@pytest.mark.parametrize("case", ["square", "tissue"])
def test_reordered_step_parity(torch_dev, case):
    torch, dev = torch_dev
    wl = W.w0_square() if case == "square" else W.w5_tissue(h=0.5)
    ctx = _ctx(wl, torch, dev, reorder=1)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    shrank = False
    for n in range(6):
        t = n * wl.dt
        dv = torch.tensor(v, dtype=torch.float64, device=dev)
        dw = torch.tensor(w, dtype=torch.float64, device=dev)
        st = ctx.step(dv, dw, t, wl.dt, wl.sweeps, wl.tol)
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, alpha=wl.alpha,
                   cg_rtol=wl.cg_rtol, istim=wl.stim_vector(t), want_log=True, want_nodes=True)
        assert r["status"] == 0
        assert _relmax(dv.cpu().numpy(), r["v"]) <= 1e-10
        assert _relmax(dw.cpu().numpy(), r["w"]) <= 1e-10
        for k in range(wl.sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k]), (n, k)
        shrank |= r["stats"].n_active[wl.sweeps - 1] < wl.n
        V = torch.empty((wl.M, wl.n), dtype=torch.float64, device=dev)
        Wn = torch.empty_like(V)
        ctx.nodes(V, Wn)
        assert _relmax(V.cpu().numpy(), r["V"]) <= 1e-10
        v, w = r["v"], r["w"]
    assert shrank
    ctx.close()


def test_reordered_matrix_and_scale_in_callers_numbering(torch_dev):
    torch, dev = torch_dev
    wl = W.w4_slab()
    a = _ctx(wl, torch, dev, reorder=0)
    b = _ctx(wl, torch, dev, reorder=1)
    ra, rb = a.matrix(), b.matrix()
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    np.testing.assert_allclose(rb[2], ra[2], rtol=1e-14, atol=1e-14 * np.abs(ra[2]).max())
    np.testing.assert_allclose(rb[3], ra[3], rtol=1e-14)
    # a new conductivity scale, also in the caller's numbering
    rng = np.random.default_rng(5)
    s = 1.0 + 0.2 * rng.random(wl.n)
    a.set_dof_scale(s)
    b.set_dof_scale(s)
    ra, rb = a.matrix(), b.matrix()
    np.testing.assert_allclose(rb[2], ra[2], rtol=1e-14, atol=1e-14 * np.abs(ra[2]).max())
    a.close()
    b.close()


def test_reorder_rejects_tapes(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import SdcError
    wl = W.w0_square(n=17, length=5.0)
    ctx = _ctx(wl, torch, dev, reorder=1)
    v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    tp = ctx.new_tape(wl.sweeps, dev)
    with pytest.raises(SdcError):
        ctx.step_taped(v, w, 0.0, wl.dt, wl.sweeps, wl.tol, tp)
    ctx.close()


@pytest.mark.parametrize("scaled,pipe", [(1, -1), (0, 1), (1, 0)])
def test_options_together_against_the_oracle(torch_dev, scaled, pipe):
    """Internal Morton numbering, the energy-norm stop with a given rho, the a
    priori drop tolerance, each CG form and arrangement, and an autotuned launch
    shape at once, on the tissue mesh: the oracle (plain numbering, same
    options) gives the same sweeps, drop tolerance, active sets and states."""
    torch, dev = torch_dev
    wl = W.w5_tissue(h=0.5)
    ctx = _ctx(wl, torch, dev, reorder=1, energy_stop=1, sdc_rho=0.2, drop_rule=1,
               cg_scaled=scaled, cg_pipelined=pipe)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    dv = torch.tensor(v, dtype=torch.float64, device=dev)
    dw = torch.tensor(w, dtype=torch.float64, device=dev)
    rep = ctx.autotune(dv, dw, 0.0, wl.dt, 8, wl.tol, trial_steps=1)
    assert np.array_equal(dv.cpu().numpy(), v)
    assert rep["trials"] >= 8
    stopped = False
    for n in range(4):
        t = n * wl.dt
        st = ctx.step(dv, dw, t, wl.dt, 8, wl.tol)
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, 8, wl.tol, cg_rtol=wl.cg_rtol,
                   istim=wl.stim_vector(t), want_log=True, energy_stop=True, rho=0.2,
                   drop_rule=1)
        assert r["status"] == 0
        assert st.sweeps_run == r["stats"].sweeps_run, n
        stopped |= st.sweeps_run < 8
        assert st.tol_drop == pytest.approx(r["stats"].tol_drop, rel=1e-13)
        for k in range(st.sweeps_run):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k]), (n, k)
        assert _relmax(dv.cpu().numpy(), r["v"]) <= 1e-10
        assert _relmax(dw.cpu().numpy(), r["w"]) <= 1e-10
        v, w = r["v"], r["w"]
    assert stopped
    ctx.close()
