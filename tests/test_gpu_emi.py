"""GPU parity of the cell-by-cell (EMI) step (Sec. 2.1 in the abstract form of
Sec. 3, sweep of Sec. 3.2, nested sets of Sec. 4.2) against the oracle's
EMI step, through the C ABI.

Each GPU step starts from the oracle's state.  Tolerance 1e-10 relative in
the max norm for the potentials and the per-pair gating, active index lists
identical, CG iteration counts within one.
"""

import numpy as np
import pytest

import oracle
from workloads.emi import emi_tiny

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


def _relmax(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def _ctx(wl, torch, dev, **opts):
    from paper_2311_07206_gb300 import Context, default_options
    return Context.from_emi(wl, options=default_options(**opts),
                            stream=torch.cuda.current_stream(dev).cuda_stream)


def _run(wl, torch, dev, steps, tol, sweeps=None, w_frozen=False, iters_rel=0.0, **opts):
    sweeps = wl.sweeps if sweeps is None else sweeps
    ctx = _ctx(wl, torch, dev, w_frozen=int(w_frozen), **opts)
    S = oracle.System.from_mesh(wl.mesh)
    u, w = wl.u0.copy(), wl.w0.copy()
    shrank = False
    for n in range(steps):
        du = torch.tensor(u, dtype=torch.float64, device=dev)
        dw = torch.tensor(w, dtype=torch.float64, device=dev)
        st = ctx.step(du, dw, n * wl.dt, wl.dt, sweeps, tol)
        r = S.step_emi(wl, u, w, sweeps=sweeps, tol=tol, w_frozen=w_frozen, want_log=True)
        assert r["status"] == 0
        gu, gw = du.cpu().numpy(), dw.cpu().numpy()
        assert _relmax(gu, r["u"]) <= RTOL, n
        assert _relmax(gw, r["w"]) <= RTOL, n
        assert list(st.n_active[:sweeps]) == list(r["stats"].n_active[:sweeps])
        for k in range(sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k]), "sweep %d" % k
            for m in range(wl.M):
                ref = r["stats"].cg_iters[k * 8 + m]
                assert abs(st.cg_iters[k][m] - ref) <= max(1, iters_rel * ref)
        assert st.cg_relres_max <= wl.cg_rtol
        shrank |= st.n_active[sweeps - 1] < wl.n
        # kind-1 (gap junction) pairs carry no gating: left as given
        gap = wl.pair_kind == 1
        assert np.array_equal(gw[gap], w[gap])
        u, w = r["u"], r["w"]
    ctx.close()
    return shrank


@pytest.mark.parametrize("kind", ["two_cells", "grid"])
@pytest.mark.parametrize("variant,cluster", [(0, 20000), (2, 0), (1, 0)])
def test_emi_step_parity_adaptive(torch_dev, kind, variant, cluster):
    torch, dev = torch_dev
    wl = emi_tiny(kind)
    shrank = _run(wl, torch, dev, 3, wl.tol, cg_variant=variant, cg_cluster_rows=cluster)
    assert shrank    # the nested sets really drop dofs here


@pytest.mark.parametrize("kind", ["two_cells", "grid"])
def test_emi_step_parity_plain_sdc(torch_dev, kind):
    torch, dev = torch_dev
    wl = emi_tiny(kind)
    _run(wl, torch, dev, 2, 0.0)


@pytest.mark.parametrize("M", [1, 2, 4])
def test_emi_parity_other_node_counts(torch_dev, M):
    torch, dev = torch_dev
    wl = emi_tiny("two_cells")
    wl.M = M
    _run(wl, torch, dev, 2, wl.tol, sweeps=M + 1)


def test_emi_parity_frozen_gating(torch_dev):
    torch, dev = torch_dev
    wl = emi_tiny("grid")
    wl.w0 = np.full(wl.n_pairs, 0.05)
    _run(wl, torch, dev, 2, wl.tol, w_frozen=True)


def test_emi_host_entry_and_nodes(torch_dev):
    torch, dev = torch_dev
    wl = emi_tiny("two_cells")
    ctx = _ctx(wl, torch, dev)
    du = torch.tensor(wl.u0, dtype=torch.float64, device=dev)
    dw = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    ctx.step(du, dw, 0.0, wl.dt, wl.sweeps, wl.tol)
    U = torch.empty((wl.M, wl.n), dtype=torch.float64, device=dev)
    Wn = torch.empty((wl.M, wl.n_pairs), dtype=torch.float64, device=dev)
    ctx.nodes(U, Wn)
    assert torch.equal(U[-1], du) and torch.equal(Wn[-1], dw)
    hu, hw = wl.u0.copy(), wl.w0.copy()
    ctx.step_host(hu, hw, 0.0, wl.dt, wl.sweeps, wl.tol)
    assert np.array_equal(hu, du.cpu().numpy()) and np.array_equal(hw, dw.cpu().numpy())
    ctx.close()


def test_emi_context_rejects_monodomain_only_calls(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import SdcError
    wl = emi_tiny("two_cells")
    ctx = _ctx(wl, torch, dev)
    with pytest.raises(SdcError):
        ctx.set_stimulus([0], 1.0, 0.0, 1.0)
    with pytest.raises(SdcError):
        ctx.set_dof_scale(np.ones(wl.n))
    du = torch.tensor(wl.u0, dtype=torch.float64, device=dev)
    dw = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    tp = ctx.new_tape(wl.sweeps, dev)
    with pytest.raises(SdcError):
        ctx.step_taped(du, dw, 0.0, wl.dt, wl.sweeps, wl.tol, tp)
    ctx.close()


def test_emi_parity_full_size_cells(torch_dev):
    """Two 100x20x20 um cells on 2 um voxels (53,274 dofs): the node solves
    run on the shared-memory PCG variant over many blocks; one adaptive step
    against the oracle."""
    torch, dev = torch_dev
    from workloads.emi import emi_bricks
    wl = emi_bricks(cells=(2, 1, 1))
    assert wl.n > 50000
    assert _run(wl, torch, dev, 1, wl.tol)


@pytest.mark.slow
def test_emi_bricks_full_size_properties(torch_dev):
    """The 8x4x4-cell workload at full size (1,471,260 dofs) in the launch
    configuration the benchmark times: a step is bitwise reproducible, every
    node solve met the CG tolerance, the sets are nested, and adaptive and
    plain SDC agree to the order of TOL."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import default_options, Context
    from workloads.emi import emi_bricks
    wl = emi_bricks()
    opts = default_options(profile=1, cg_rtol=wl.cg_rtol, alpha=wl.alpha, cg_maxit=100000)
    ctx = Context.from_emi(wl, options=opts, stream=torch.cuda.current_stream(dev).cuda_stream)
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    outs = []
    for tol in (wl.tol, wl.tol, 0.0):
        u, w = t64(wl.u0), t64(wl.w0)
        st = ctx.step(u, w, 0.0, wl.dt, wl.sweeps, tol)
        assert st.cg_relres_max <= wl.cg_rtol
        acts = [ctx.active(k) for k in range(1, wl.sweeps)]
        for a, b in zip(acts[1:], acts[:-1]):
            assert np.all(np.isin(a, b))
        outs.append((u.cpu().numpy(), w.cpu().numpy(), list(st.n_active[:wl.sweeps])))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2] and outs[0][2][-1] < wl.n
    assert np.abs(outs[0][0] - outs[2][0]).max() <= 10 * wl.tol
    ctx.close()


@pytest.mark.parametrize("variant,cluster", [(0, 20000), (1, 0)])
def test_emi_parity_2d_branched_cells(torch_dev, variant, cluster):
    """The 2D cell-by-cell mesh (triangles, edge membranes) of the branched
    myocytes at 10 um pixels, gating held at w = 0 as in the paper's EMI runs.
    Its node solves take 300-400 CG iterations; at that length the iteration
    where the recursively updated residual of a finite-precision CG crosses
    rtol depends on the rounding of its sums and recurrences (the oracle runs
    the textbook recurrences summed in index order; the kernels run the
    Chronopoulos-Gear recurrences, exact sums, Jacobi or scaled form), so counts
    agree to 15 % here while the states agree to 1e-10 and the active sets
    exactly."""
    torch, dev = torch_dev
    from workloads.emi import emi_tiny
    wl = emi_tiny("branched_2d")
    assert wl.mesh.dim == 2
    assert _run(wl, torch, dev, 3, wl.tol, w_frozen=True, iters_rel=0.15, cg_variant=variant,
                cg_cluster_rows=cluster)
