"""The launch-shape autotuner (sdc_autotune, sdc_batch_autotune): the caller's
state comes back bitwise, the chosen configuration is one of the candidates,
and steps under it still match the oracle (single context) and the
per-instance runs (batch) within the parity tolerance."""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_07206_gb300 import build as b
    b.build()
    return torch, torch.device("cuda:0")


def _slab():
    mesh = W.kuhn3d(41, 15, 9, 0.1)
    stim = np.nonzero((mesh.xyz <= 0.5 + 1e-12).all(axis=1))[0].astype(np.int32)
    return W.Workload("slab_41x15x9", mesh, np.diag([1.0, 0.25, 0.25]), dict(W.AP_BENCH), M=4,
                      dt=0.05, sweeps=5, tol=1e-5, steps=10, v0=np.zeros(mesh.n_nodes),
                      w0=np.zeros(mesh.n_nodes), stim_nodes=stim, stim_amp=2.0, stim_t_on=0.0,
                      stim_t_off=1.0)


def _relmax(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("case", ["square", "slab"])
def test_autotune_restores_state_and_keeps_parity(torch_dev, case):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Context, default_options
    wl = W.w0_square() if case == "square" else _slab()
    ctx = Context.from_workload(wl, options=default_options(),
                                stream=torch.cuda.current_stream(dev).cuda_stream)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    # a state with a front: a few plain steps of the oracle
    for n in range(3):
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, cg_rtol=wl.cg_rtol,
                   istim=wl.stim_vector(n * wl.dt))
        v, w = r["v"], r["w"]
    dv = torch.tensor(v, dtype=torch.float64, device=dev)
    dw = torch.tensor(w, dtype=torch.float64, device=dev)
    rep = ctx.autotune(dv, dw, 3 * wl.dt, wl.dt, wl.sweeps, wl.tol, trial_steps=2)
    assert np.array_equal(dv.cpu().numpy(), v) and np.array_equal(dw.cpu().numpy(), w)
    assert rep["trials"] >= 8 and 0 < rep["best_ms"] <= rep["base_ms"]
    assert rep["cg_pipelined"] in (0, 1) and rep["cg_scaled"] in (0, 1)
    assert rep["smem_block"] in (512, 1024) and rep["general_block"] in (256, 512, 1024)
    assert rep["big_rows"] in (0, 100000, 300000, 0x7fffffff)
    assert rep["cluster_rows"] in (0, 2000, 5000, 10000, 20000)
    for n in range(3, 5):
        t = n * wl.dt
        st = ctx.step(dv, dw, t, wl.dt, wl.sweeps, wl.tol)
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, cg_rtol=wl.cg_rtol,
                   istim=wl.stim_vector(t), want_log=True)
        assert _relmax(dv.cpu().numpy(), r["v"]) <= RTOL
        assert _relmax(dw.cpu().numpy(), r["w"]) <= RTOL
        for k in range(wl.sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k])
        v, w = r["v"], r["w"]
    ctx.close()


def test_batch_autotune_restores_state_and_matches_solo_runs(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Batch, Context
    insts = W.batch_instances(count=6, nmin=32, nmax=128)
    stream = torch.cuda.current_stream(dev).cuda_stream
    batch = Batch(insts, stream=stream)
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    v0 = np.concatenate([wl.v0 for wl in insts])
    w0 = np.concatenate([wl.w0 for wl in insts])
    bv, bw = t64(v0), t64(w0)
    wl0 = insts[0]
    rep = batch.autotune(bv, bw, 0.0, wl0.dt, wl0.sweeps, wl0.tol, trial_steps=2)
    assert np.array_equal(bv.cpu().numpy(), v0) and np.array_equal(bw.cpu().numpy(), w0)
    assert rep["trials"] >= 6 and 0 < rep["best_ms"] <= rep["base_ms"]
    assert rep["batch_block"] in (256, 512, 1024)
    assert rep["batch_rows_per_block"] in (256, 512, 1024, 2048, 4096)
    solos = [Context.from_workload(wl, stream=stream) for wl in insts]
    sv, sw = [t64(wl.v0) for wl in insts], [t64(wl.w0) for wl in insts]
    off = batch.offsets
    for n in range(3):
        t = n * wl0.dt
        batch.step(bv, bw, t, wl0.dt, wl0.sweeps, wl0.tol)
        gv = bv.cpu().numpy()
        for b, wl in enumerate(insts):
            solos[b].step(sv[b], sw[b], t, wl.dt, wl.sweeps, wl.tol)
            ref = sv[b].cpu().numpy()
            assert np.abs(gv[off[b]:off[b + 1]] - ref).max() <= RTOL * max(1.0, np.abs(ref).max())
    batch.close()
    for c in solos:
        c.close()


def test_emi_autotune_restores_state(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Context, default_options
    from workloads.emi import emi_tiny
    wl = emi_tiny("grid")
    ctx = Context.from_emi(wl, options=default_options(cg_maxit=100000),
                           stream=torch.cuda.current_stream(dev).cuda_stream)
    du = torch.tensor(wl.u0, dtype=torch.float64, device=dev)
    dw = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    rep = ctx.autotune(du, dw, 0.0, wl.dt, wl.sweeps, wl.tol, trial_steps=1)
    assert np.array_equal(du.cpu().numpy(), wl.u0) and np.array_equal(dw.cpu().numpy(), wl.w0)
    assert rep["trials"] >= 8
    S = oracle.System.from_mesh(wl.mesh)
    st = ctx.step(du, dw, 0.0, wl.dt, wl.sweeps, wl.tol)
    r = S.step_emi(wl, wl.u0, wl.w0)
    assert _relmax(du.cpu().numpy(), r["u"]) <= RTOL
    ctx.close()
