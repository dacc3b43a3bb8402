"""GPU parity of the CUDA library against the CPU oracle, element by element on
the same seeded inputs, through the C ABI.

Tolerance: 1e-10 relative in the max norm for v and w (every collocation node),
active index lists identical.  Each GPU step starts from the oracle's state so
rounding differences do not accumulate across steps; the CG tolerance is the
workload's (1e-10).
"""

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


def _ctx(wl, torch, dev, **opts):
    from paper_2311_07206_gb300 import Context, default_options
    o = default_options(**opts)
    return Context.from_workload(wl, options=o, stream=torch.cuda.current_stream(dev).cuda_stream)


def _relmax(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def _compare_step(ctx, S, wl, v, w, t, sweeps, tol, torch, dev, cg_rtol=None, nodes=True):
    """One step from (v, w) on both sides; returns the oracle's result."""
    cg_rtol = wl.cg_rtol if cg_rtol is None else cg_rtol
    dv = torch.tensor(v, dtype=torch.float64, device=dev)
    dw = torch.tensor(w, dtype=torch.float64, device=dev)
    st = ctx.step(dv, dw, t, wl.dt, sweeps, tol)
    r = S.step(wl.ionic, wl.M, v, w, wl.dt, sweeps, tol, alpha=wl.alpha, cg_rtol=cg_rtol,
               istim=wl.stim_vector(t), want_log=True, want_nodes=nodes)
    assert r["status"] == 0
    gv, gw = dv.cpu().numpy(), dw.cpu().numpy()
    assert _relmax(gv, r["v"]) <= RTOL
    assert _relmax(gw, r["w"]) <= RTOL
    assert list(st.n_active[:sweeps]) == list(r["stats"].n_active[:sweeps])
    for k in range(sweeps):
        if r["stats"].n_active[k]:
            assert np.array_equal(ctx.active(k), r["active"][k]), "active set of sweep %d" % k
    if nodes:
        Vg = torch.empty((wl.M, wl.n), dtype=torch.float64, device=dev)
        Wg = torch.empty_like(Vg)
        ctx.nodes(Vg, Wg)
        assert _relmax(Vg.cpu().numpy(), r["V"]) <= RTOL
        assert _relmax(Wg.cpu().numpy(), r["W"]) <= RTOL
    # CG iteration counts agree (a tie at the stopping test may shift one by 1).
    # On systems with fewer rows than a few iterations CG terminates at the
    # rounding floor, where the pipelined recurrences may take an extra step
    # or two before their residual estimate passes the test.
    for k in range(sweeps):
        for m in range(wl.M):
            a, b = st.cg_iters[k][m], r["stats"].cg_iters[k * 8 + m]
            assert abs(a - b) <= 1 or wl.n <= 2 * max(a, b), (k, m, a, b)
    return r, st


# ------------------------------------------------------------------ assembly
def _small_slab():
    wl = W.w1_slab()
    mesh = W.kuhn3d(41, 15, 7, 0.1)
    stim = np.nonzero((mesh.xyz <= 1.5 + 1e-12).all(axis=1))[0].astype(np.int32)
    return W.Workload("slab_41x15x7", mesh, wl.sigma, wl.ionic, M=4, dt=0.05, sweeps=5, tol=1e-5,
                      steps=20, v0=np.zeros(mesh.n_nodes), w0=np.zeros(mesh.n_nodes),
                      stim_nodes=stim, stim_amp=2.0, stim_t_on=0.0, stim_t_off=1.0)


@pytest.mark.parametrize("case", ["w0", "slab", "tissue", "scaled"])
def test_assembly_matches_oracle(torch_dev, case):
    torch, dev = torch_dev
    if case == "w0":
        wl = W.w0_square()
    elif case == "slab":
        wl = _small_slab()
    elif case == "tissue":
        wl = W.w5_tissue(h=0.6)
    else:
        wl = W.w4_slab()
    ctx = _ctx(wl, torch, dev)
    rp, ci, val, mass = ctx.matrix()
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, wl.dof_scale)
    orp, oci, oval, omass = S.matrix()
    np.testing.assert_allclose(mass, omass, rtol=1e-13, atol=0)
    kd = np.array([oval[orp[i]:orp[i + 1]][oci[orp[i]:orp[i + 1]] == i][0] for i in range(wl.n)])
    for i in range(wl.n):
        gc, gv = ci[rp[i]:rp[i + 1]], val[rp[i]:rp[i + 1]]
        oc, ov = oci[orp[i]:orp[i + 1]], oval[orp[i]:orp[i + 1]]
        full = dict(zip(oc.tolist(), ov.tolist()))
        assert set(gc.tolist()) <= set(full)
        for c, v in zip(gc.tolist(), gv.tolist()):
            assert abs(v - full[c]) <= 1e-13 * kd[i]
        for c, v in full.items():
            if c not in set(gc.tolist()):   # dropped: rounding residue only
                assert abs(v) <= 1e-12 * np.sqrt(kd[i] * kd[c])
    ctx.close()


# ------------------------------------------------------------------ step parity
@pytest.mark.parametrize("variant,cluster,pipe,scaled", [(1, 0, 1, 1), (2, 0, 1, 1),
                                                          (2, 0, 1, 0), (0, 1 << 30, 1, 1),
                                                          (1, 0, 0, 1), (2, 0, 0, 1)])
@pytest.mark.parametrize("tol", [0.0, 1e-4])
def test_step_parity_2d_square(torch_dev, tol, variant, cluster, pipe, scaled):
    """Pipelined (pipe = 1) and classical (pipe = 0) arrangements of the CG in
    every variant it has; the pipelined shared-memory solve in the
    symmetrically scaled (scaled = 1) and the Jacobi form."""
    torch, dev = torch_dev
    wl = W.w0_square()
    ctx = _ctx(wl, torch, dev, cg_variant=variant, cg_cluster_rows=cluster, cg_pipelined=pipe,
               cg_scaled=scaled)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(12):
        r, st = _compare_step(ctx, S, wl, v, w, n * wl.dt, wl.sweeps, tol, torch, dev)
        v, w = r["v"], r["w"]
    if tol > 0:
        assert st.n_active[1] < wl.n
    ctx.close()


@pytest.mark.parametrize("variant,rows,cluster,pipe,scaled",
                         [(1, 0, 0, 1, 1), (1, 0, 0, 1, 0), (2, 0, 0, 1, 1), (2, 64, 0, 1, 1),
                          (2, 4096, 0, 1, 1),
                          (2, 0, 0, 1, 0), (2, 64, 0, 1, 0), (2, 0, 1 << 30, 1, 1),
                          (1, 0, 0, 0, 1), (1, 0, 0, 0, 0), (2, 64, 0, 0, 1),
                          (2, 64, 0, 0, 0)])
def test_step_parity_3d_slab_with_stimulus(torch_dev, variant, rows, cluster, pipe, scaled):
    """Every CG variant: global vectors; per-block shared memory with 64 rows
    per block (many blocks, tiny chunks) and with 4096 rows per block (fewest
    blocks), in the symmetrically scaled (scaled = 1) and the Jacobi form; one
    thread-block cluster for every solve; pipelined (pipe = 1) and classical
    (pipe = 0) arrangements."""
    torch, dev = torch_dev
    wl = _small_slab()
    ctx = _ctx(wl, torch, dev, cg_variant=variant, cg_rows_per_block=rows,
               cg_cluster_rows=cluster, cg_pipelined=pipe, cg_scaled=scaled)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(24):   # stimulus on for the first 20 steps, then off
        t = n * wl.dt
        r, st = _compare_step(ctx, S, wl, v, w, t, wl.sweeps, wl.tol, torch, dev,
                              nodes=(n % 6 == 0))
        v, w = r["v"], r["w"]
    assert v.max() > 0.5
    ctx.close()


@pytest.mark.parametrize("M", range(1, 9))
def test_step_parity_every_M(torch_dev, M):
    torch, dev = torch_dev
    wl = W.w0_square(n=19, length=5.625)
    wl.M = M
    ctx = _ctx(wl, torch, dev)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(3):
        r, _ = _compare_step(ctx, S, wl, v, w, n * wl.dt, 3, 1e-3, torch, dev)
        v, w = r["v"], r["w"]
    ctx.close()


@pytest.mark.parametrize("case", ["one_triangle", "one_tet", "ragged_33x31", "ragged_3d"])
def test_step_parity_edge_meshes(torch_dev, case):
    """Meshes with 3 or 4 nodes and node counts that are no multiple of any
    block size (ragged tails in every kernel)."""
    torch, dev = torch_dev
    if case == "one_triangle":
        mesh = W.Mesh(2, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]),
                      np.array([[0, 1, 2]], np.int32))
    elif case == "one_tet":
        mesh = W.Mesh(3, np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]),
                      np.array([[0, 1, 2, 3]], np.int32))
    elif case == "ragged_33x31":
        mesh = W.grid2d(33, 31, 0.3125)
    else:
        mesh = W.kuhn3d(13, 7, 5, 0.2)
    n = mesh.n_nodes
    v0 = np.zeros(n)
    v0[: max(1, n // 7)] = 1.0
    wl = W.Workload(case, mesh, np.eye(3), dict(W.AP_BENCH), M=3, dt=0.1, sweeps=4, tol=1e-4,
                    steps=4, v0=v0, w0=np.zeros(n))
    ctx = _ctx(wl, torch, dev)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for k in range(4):
        r, _ = _compare_step(ctx, S, wl, v, w, k * wl.dt, wl.sweeps, wl.tol, torch, dev)
        v, w = r["v"], r["w"]
    ctx.close()


def test_empty_active_sets_and_single_sweep(torch_dev):
    torch, dev = torch_dev
    wl = W.w0_square(n=21, length=6.25)
    ctx = _ctx(wl, torch, dev)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    # TOL so large that every dof drops after the first sweep
    r, st = _compare_step(ctx, S, wl, wl.v0, wl.w0, 0.0, 4, 1e300, torch, dev)
    assert list(st.n_active[:4]) == [wl.n, 0, 0, 0]
    r, st = _compare_step(ctx, S, wl, wl.v0, wl.w0, 0.0, 1, 1e-4, torch, dev)
    ctx.close()


@pytest.mark.parametrize("tol", [0.0, 1e-4])
def test_step_parity_implicit_euler_qhat(torch_dev, tol):
    """The implicit-Euler preconditioner of the sweeps (option sdc_qhat = 1)
    against the oracle's (qhat="ie")."""
    torch, dev = torch_dev
    wl = W.w0_square()
    ctx = _ctx(wl, torch, dev, sdc_qhat=1)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(6):
        dv = torch.tensor(v, dtype=torch.float64, device=dev)
        dw = torch.tensor(w, dtype=torch.float64, device=dev)
        st = ctx.step(dv, dw, n * wl.dt, wl.dt, wl.sweeps, tol)
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, tol, alpha=wl.alpha,
                   cg_rtol=wl.cg_rtol, istim=wl.stim_vector(n * wl.dt), want_log=True, qhat="ie")
        assert r["status"] == 0
        assert _relmax(dv.cpu().numpy(), r["v"]) <= RTOL
        assert _relmax(dw.cpu().numpy(), r["w"]) <= RTOL
        for k in range(wl.sweeps):
            if r["stats"].n_active[k]:
                assert np.array_equal(ctx.active(k), r["active"][k])
        v, w = r["v"], r["w"]
    ctx.close()


def test_tol_zero_is_plain_and_deterministic(torch_dev):
    torch, dev = torch_dev
    wl = W.w0_square()
    outs = []
    for alpha in (0.1, 0.0, 0.1):
        ctx = _ctx(wl, torch, dev, alpha=alpha)
        v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
        w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
        for n in range(5):
            ctx.step(v, w, n * wl.dt, wl.dt, wl.sweeps, 0.0)
        outs.append((v.cpu().numpy(), w.cpu().numpy()))
        ctx.close()
    for a, b in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(b, outs[0][1])


def test_host_entry_point_equals_device_entry_point(torch_dev):
    torch, dev = torch_dev
    wl = _small_slab()
    ctx = _ctx(wl, torch, dev)
    v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    hv, hw = wl.v0.copy(), wl.w0.copy()
    for n in range(6):
        ctx.step(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol)
        ctx.step_host(hv, hw, n * wl.dt, wl.dt, wl.sweeps, wl.tol)
    assert np.array_equal(v.cpu().numpy(), hv) and np.array_equal(w.cpu().numpy(), hw)
    ctx.close()


# ------------------------------------------------------------------ error paths
def test_error_statuses(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import SdcError
    from paper_2311_07206_gb300 import binding as B
    wl = W.w0_square(n=17, length=5.0)
    ctx = _ctx(wl, torch, dev)
    v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    for args in ((0.0, -0.1, 4, 1e-4), (0.0, 0.1, 0, 1e-4), (0.0, 0.1, 65, 1e-4), (0.0, 0.1, 4, -1.0)):
        with pytest.raises(SdcError) as e:
            ctx.step(v, w, *args)
        assert e.value.status == B.SDC_E_INVALID
    # non-finite input
    vb = v.clone()
    vb[3] = float("nan")
    with pytest.raises(SdcError) as e:
        ctx.step(vb, w.clone(), 0.0, 0.1, 4, 1e-4)
    assert e.value.status == B.SDC_E_NONFINITE
    # a node system with a non-positive diagonal: dI/dv = ... + w is hugely negative
    wb = w.clone()
    wb[5] = -1e6
    with pytest.raises(SdcError) as e:
        ctx.step(v.clone(), wb, 0.0, 0.1, 4, 1e-4)
    assert e.value.status == B.SDC_E_DOMAIN
    ctx.close()
    # CG iteration cap
    ctx = _ctx(wl, torch, dev, cg_maxit=1)
    with pytest.raises(SdcError) as e:
        ctx.step(v.clone(), w.clone(), 0.0, 0.1, 4, 1e-4)
    assert e.value.status == B.SDC_E_CG_NOCONV
    ctx.close()
    # invalid mesh
    with pytest.raises(SdcError) as e:
        from paper_2311_07206_gb300 import Context
        Context(2, np.zeros((3, 2)), np.array([[0, 1, 2]], np.int32))   # degenerate triangle
    assert e.value.status == B.SDC_E_INVALID


@pytest.mark.parametrize("variant", [1, 2])
def test_barrier_timeout_is_reported_and_context_recovers(torch_dev, variant):
    """Fault injection: one CG block never arrives at the grid barrier; the
    other blocks' waits are bounded (spin budget ~1 ms), the step reports
    SDC_E_TIMEOUT, and the same context then steps normally."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import SdcError
    from paper_2311_07206_gb300 import binding as B
    wl = W.w0_square()
    bad = _ctx(wl, torch, dev, inject_fault=1, spin_budget=2_000_000, cg_variant=variant,
               cg_rows_per_block=256)
    v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    with pytest.raises(SdcError) as e:
        bad.step(v, w, 0.0, wl.dt, wl.sweeps, wl.tol)
    assert e.value.status == B.SDC_E_TIMEOUT
    bad.close()
    good = _ctx(wl, torch, dev, cg_variant=variant)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    _compare_step(good, S, wl, wl.v0, wl.w0, 0.0, wl.sweeps, wl.tol, torch, dev)
    good.close()


# ------------------------------------------------------------------ full size
@pytest.mark.slow
def test_full_size_slab_parity(torch_dev):
    """The 201x71x31 slab (442k dofs, M = 4, 5 sweeps, TOL = 1e-5): the first
    steps under stimulus, and steps from a state reached after 200 GPU steps
    (t = 10 ms, fronts inside the slab), each compared with the oracle."""
    torch, dev = torch_dev
    wl = W.w1_slab()
    ctx = _ctx(wl, torch, dev)
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    v, w = wl.v0.copy(), wl.w0.copy()
    for n in range(2):
        r, _ = _compare_step(ctx, S, wl, v, w, n * wl.dt, wl.sweeps, wl.tol, torch, dev,
                             nodes=False)
        v, w = r["v"], r["w"]
    dv = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    dw = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    for n in range(200):
        ctx.step(dv, dw, n * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
    v, w = dv.cpu().numpy(), dw.cpu().numpy()
    assert 0.05 < (v > 0.5).mean() < 0.95
    for n in range(200, 202):
        r, st = _compare_step(ctx, S, wl, v, w, n * wl.dt, wl.sweeps, wl.tol, torch, dev,
                              nodes=False)
        v, w = r["v"], r["w"]
    assert st.n_active[2] < st.n_active[1] < wl.n
    ctx.close()
