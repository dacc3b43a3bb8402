"""Batched step: instances of uneven size, conductivity and stimulus advanced
together must follow their solo runs (each instance's state within the parity
tolerance, its active sets identical, its CG iteration counts within one) and
the oracle."""

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


def _instances(count=7):
    insts = W.batch_instances(count=count, nmin=9, nmax=48)
    # two instances also get a stimulus current (one shared window)
    for b in (1, count - 2):
        wl = insts[b]
        wl.stim_nodes = np.arange(0, wl.n, 5, dtype=np.int32)
        wl.stim_amp = 1.5 + 0.25 * b
        wl.stim_t_on, wl.stim_t_off = 0.0, 0.25
    return insts


@pytest.mark.parametrize("max_blocks,scaled", [(0, 1), (3, 1), (0, 0)])
def test_batch_follows_solo_runs(torch_dev, max_blocks, scaled):
    """max_blocks = 3 forces several waves of the batched CG launch; scaled = 0
    runs the batched solves in the Jacobi form."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Batch, Context, default_options
    insts = _instances()
    stream = torch.cuda.current_stream(dev).cuda_stream
    batch = Batch(insts, options=default_options(cg_max_blocks=max_blocks, cg_scaled=scaled),
                  stream=stream)
    off = batch.offsets
    solos = [Context.from_workload(wl, stream=stream) for wl in insts]
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    bv = t64(np.concatenate([wl.v0 for wl in insts]))
    bw = t64(np.concatenate([wl.w0 for wl in insts]))
    sv = [t64(wl.v0) for wl in insts]
    sw = [t64(wl.w0) for wl in insts]
    wl0 = insts[0]
    for n in range(5):
        t = n * wl0.dt
        bst = batch.step(bv, bw, t, wl0.dt, wl0.sweeps, wl0.tol)
        per = [batch.instance_stats(k) for k in range(wl0.sweeps)]
        act = [batch.active(k) if bst.n_active[k] else np.zeros(0, np.int32)
               for k in range(wl0.sweeps)]
        gv, gw = bv.cpu().numpy(), bw.cpu().numpy()
        for b, wl in enumerate(insts):
            st = solos[b].step(sv[b], sw[b], t, wl.dt, wl.sweeps, wl.tol)
            a, z = off[b], off[b + 1]
            ref_v, ref_w = sv[b].cpu().numpy(), sw[b].cpu().numpy()
            assert np.abs(gv[a:z] - ref_v).max() <= RTOL * max(1.0, np.abs(ref_v).max())
            assert np.abs(gw[a:z] - ref_w).max() <= RTOL * max(1.0, np.abs(ref_w).max())
            for k in range(wl.sweeps):
                assert per[k][0][b] == st.n_active[k]
                mine = act[k][(act[k] >= a) & (act[k] < z)] - a
                if st.n_active[k]:
                    assert np.array_equal(mine, solos[b].active(k))
                else:
                    assert mine.size == 0
                for m in range(wl.M):
                    assert abs(int(per[k][1][m][b]) - st.cg_iters[k][m]) <= 1
    assert sum(bst.n_active[:wl0.sweeps]) > 0
    batch.close()
    for c in solos:
        c.close()


def test_batch_instances_match_oracle(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Batch
    insts = _instances(count=4)
    stream = torch.cuda.current_stream(dev).cuda_stream
    batch = Batch(insts, stream=stream)
    off = batch.offsets
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    bv = t64(np.concatenate([wl.v0 for wl in insts]))
    bw = t64(np.concatenate([wl.w0 for wl in insts]))
    states = [(wl.v0.copy(), wl.w0.copy()) for wl in insts]
    systems = [oracle.System.from_mesh(wl.mesh, wl.sigma) for wl in insts]
    wl0 = insts[0]
    for n in range(3):
        t = n * wl0.dt
        batch.step(bv, bw, t, wl0.dt, wl0.sweeps, wl0.tol)
        gv, gw = bv.cpu().numpy(), bw.cpu().numpy()
        for b, wl in enumerate(insts):
            r = systems[b].step(wl.ionic, wl.M, states[b][0], states[b][1], wl.dt, wl.sweeps,
                                wl.tol, cg_rtol=wl.cg_rtol, istim=wl.stim_vector(t))
            assert r["status"] == 0
            a, z = off[b], off[b + 1]
            assert np.abs(gv[a:z] - r["v"]).max() <= RTOL * max(1.0, np.abs(r["v"]).max())
            assert np.abs(gw[a:z] - r["w"]).max() <= RTOL * max(1.0, np.abs(r["w"]).max())
            states[b] = (r["v"], r["w"])
    batch.close()


def test_captured_batch_step_equals_host_driven_bitwise(torch_dev):
    """batch_graph = 1 (device-driven sweeps replayed as a CUDA graph) against
    host-driven sweeps: the same kernels and exact sums, so the states, active
    lists, per-instance set sizes and CG counts agree bitwise, across the end
    of the stimulus window (a second capture)."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import Batch, default_options
    insts = _instances()
    stream = torch.cuda.current_stream(dev).cuda_stream
    bg = Batch(insts, options=default_options(batch_graph=1), stream=stream)
    bh = Batch(insts, options=default_options(batch_graph=0), stream=stream)
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    v0 = np.concatenate([wl.v0 for wl in insts])
    w0 = np.concatenate([wl.w0 for wl in insts])
    gv, gw, hv, hw = t64(v0), t64(w0), t64(v0), t64(w0)
    wl0 = insts[0]
    for n in range(6):
        t = n * wl0.dt
        sg = bg.step(gv, gw, t, wl0.dt, wl0.sweeps, wl0.tol)
        sh = bh.step(hv, hw, t, wl0.dt, wl0.sweeps, wl0.tol)
        assert sg.captured == 1 and sh.captured == 0
        assert torch.equal(gv, hv) and torch.equal(gw, hw), n
        assert list(sg.n_active[:wl0.sweeps]) == list(sh.n_active[:wl0.sweeps])
        assert list(sg.nnz_active[:wl0.sweeps]) == list(sh.nnz_active[:wl0.sweeps])
        for k in range(wl0.sweeps):
            assert [sg.cg_iters[k][m] for m in range(wl0.M)] == \
                [sh.cg_iters[k][m] for m in range(wl0.M)]
            if sg.n_active[k]:
                assert np.array_equal(bg.active(k), bh.active(k))
            ng, ig = bg.instance_stats(k)
            nh, ih = bh.instance_stats(k)
            assert np.array_equal(ng, nh) and np.array_equal(ig, ih)
    assert sum(sg.n_active[:wl0.sweeps]) > 0
    bg.close()
    bh.close()
