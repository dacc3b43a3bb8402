"""Discrete adjoint of the adaptive SDC step (active sets recorded in the
forward pass and held fixed).

Gradients of L = sum_n sum_probes (v_n - target_n)^2 with respect to the
per-node conductivity scale s and the Aliev-Panfilov parameters (k = ga = gs,
a) are checked against fourth-order central differences of the loss with the
same active sets replayed: once with the library's own forward, once with the
oracle's forward (independent code).  Relative agreement 1e-6.
"""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-6


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_07206_gb300 import build as b
    b.build()
    return torch, torch.device("cuda:0")


def _problem(kind):
    rng = np.random.default_rng(20231107)
    if kind == "2d":
        wl = W.w0_square(tol=1e-3, n=13, length=3.75)
        wl.sweeps, wl.dt = 4, 0.1
    else:
        mesh = W.kuhn3d(9, 5, 4, 0.2)
        stim = np.nonzero((mesh.xyz <= 0.4 + 1e-12).all(axis=1))[0].astype(np.int32)
        n = mesh.n_nodes
        wl = W.Workload("slab_9x5x4", mesh, np.diag([1.0, 0.25, 0.25]), dict(W.AP_BENCH), M=3,
                        dt=0.05, sweeps=4, tol=1e-3, steps=4, v0=np.zeros(n), w0=np.zeros(n),
                        stim_nodes=stim, stim_amp=2.0, stim_t_on=0.0, stim_t_off=1.0)
    wl.cg_rtol = 1e-13
    wl.dof_scale = 1.0 + 0.1 * rng.standard_normal(wl.n)
    probes = np.sort(rng.choice(wl.n, size=min(20, wl.n // 2), replace=False))
    return wl, probes, rng


def _setup(torch, dev, kind, steps):
    from paper_2311_07206_gb300 import Context, default_options
    wl, probes, rng = _problem(kind)
    ctx = Context.from_workload(wl, options=default_options(cg_rtol=1e-13),
                                stream=torch.cuda.current_stream(dev).cuda_stream)
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    # targets: the run with the nominal scale, shifted
    ctx.set_dof_scale(None)
    v, w = t64(wl.v0), t64(wl.w0)
    targets = []
    for n in range(steps):
        ctx.step(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
        targets.append(v[t64(probes).long()].clone() + 0.01)
    return wl, ctx, t64(probes).long(), targets, rng, t64


def _record(ctx, wl, torch, dev, t64, steps, scale, k, a):
    """Forward run at (scale, k, a) recording one tape per step."""
    from paper_2311_07206_gb300.autodiff import _set_params
    _set_params(ctx, wl, t64(scale), k, a)
    v, w = t64(wl.v0), t64(wl.w0)
    tapes = []
    for n in range(steps):
        tp = ctx.new_tape(wl.sweeps, dev)
        ctx.step_taped(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, tp)
        tapes.append(tp)
    return tapes


def _fd(loss_at, h):
    return (-loss_at(2 * h) + 8 * loss_at(h) - 8 * loss_at(-h) + loss_at(-2 * h)) / (12 * h)


def _close(fd, ad):
    return abs(fd - ad) <= REL * max(abs(fd), abs(ad)) + 1e-13


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_adjoint_gradient_matches_replayed_finite_differences(torch_dev, kind):
    torch, dev = torch_dev
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss, _set_params, replayed_loss
    steps = 4
    wl, ctx, probes, targets, rng, t64 = _setup(torch, dev, kind, steps)
    k0, a0 = wl.ionic["ga"], wl.ionic["a"]
    s0 = wl.dof_scale.copy()
    scale = t64(s0).requires_grad_(True)
    ka = t64([k0, a0]).requires_grad_(True)
    L = TrajectoryLoss.apply(scale, ka, ctx, wl, steps, probes, targets, 2)
    L.backward()
    gs = scale.grad.cpu().numpy()
    gka = ka.grad.cpu().numpy()
    assert np.abs(gs).max() > 0 and np.all(np.isfinite(gs)) and np.all(np.isfinite(gka))
    tapes = _record(ctx, wl, torch, dev, t64, steps, s0, k0, a0)
    # the adaptive sets really shrink in this problem
    assert any(tp.n_active[k] < wl.n for tp in tapes for k in range(1, wl.sweeps))
    v0, w0 = t64(wl.v0), t64(wl.w0)

    def loss(sc, k, a):
        _set_params(ctx, wl, t64(sc), k, a)
        return replayed_loss(ctx, wl, v0, w0, steps, probes, targets, tapes)

    assert abs(loss(s0, k0, a0) - L.item()) <= 1e-12 * abs(L.item())
    for _ in range(3):
        d = rng.standard_normal(wl.n)
        d /= np.linalg.norm(d)
        fd = _fd(lambda h: loss(s0 + h * d, k0, a0), 1e-4)
        assert _close(fd, gs @ d), (fd, gs @ d)
    fd_k = _fd(lambda h: loss(s0, k0 + h, a0), 1e-4 * k0)
    assert _close(fd_k, gka[0]), (fd_k, gka[0])
    fd_a = _fd(lambda h: loss(s0, k0, a0 + h), 1e-4 * a0)
    assert _close(fd_a, gka[1]), (fd_a, gka[1])
    ctx.close()


def test_adjoint_matches_oracle_finite_differences(torch_dev):
    """The same gradient against the oracle's forward (independent code),
    replaying the active sets recorded on the GPU."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss
    steps = 3
    wl, ctx, probes, targets, rng, t64 = _setup(torch, dev, "2d", steps)
    k0, a0 = wl.ionic["ga"], wl.ionic["a"]
    s0 = wl.dof_scale.copy()
    scale = t64(s0).requires_grad_(True)
    ka = t64([k0, a0]).requires_grad_(True)
    L = TrajectoryLoss.apply(scale, ka, ctx, wl, steps, probes, targets, 1)
    L.backward()
    gs = scale.grad.cpu().numpy()
    gka = ka.grad.cpu().numpy()
    tapes = _record(ctx, wl, torch, dev, t64, steps, s0, k0, a0)
    lists = []
    for tp in tapes:
        acts = tp._act.cpu().numpy().reshape(wl.sweeps, wl.n)
        lists.append([None] + [acts[k, :tp.n_active[k]].copy() for k in range(1, wl.sweeps)])
    pr = probes.cpu().numpy()
    tg = [t.cpu().numpy() for t in targets]

    def oracle_loss(sc, k, a):
        S = oracle.System.from_mesh(wl.mesh, wl.sigma, sc)
        ion = dict(wl.ionic)
        ion["ga"] = ion["gs"] = k
        ion["a"] = a
        v, w = wl.v0.copy(), wl.w0.copy()
        total = 0.0
        for n in range(steps):
            r = S.step_forced(ion, wl.M, v, w, wl.dt, wl.sweeps, lists[n], cg_rtol=1e-13,
                              istim=wl.stim_vector(n * wl.dt))
            assert r["status"] == 0
            v, w = r["v"], r["w"]
            total += float(np.sum((v[pr] - tg[n]) ** 2))
        return total

    assert abs(oracle_loss(s0, k0, a0) - L.item()) <= 1e-10 * abs(L.item())
    d = rng.standard_normal(wl.n)
    d /= np.linalg.norm(d)
    fd = _fd(lambda h: oracle_loss(s0 + h * d, k0, a0), 1e-4)
    assert _close(fd, gs @ d), (fd, gs @ d)
    fd_k = _fd(lambda h: oracle_loss(s0, k0 + h, a0), 1e-4 * k0)
    assert _close(fd_k, gka[0]), (fd_k, gka[0])
    ctx.close()


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_adjoint_dot_product_with_oracle_tangent(torch_dev, kind):
    """Dot-product test of the adjoint against the oracle's tangent (forward
    mode, independent code): for the loss L over the trajectory, the GPU's
    <grad L, d> equals the oracle's directional derivative dL/d(eps) along d,
    for conductivity-scale directions and for (k, a), with the active sets the
    GPU recorded.  Both sides differentiate solves converged to 1e-13, so they
    agree far below the finite-difference tolerance (1e-8 relative)."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss
    steps = 3
    wl, ctx, probes, targets, rng, t64 = _setup(torch, dev, kind, steps)
    k0, a0 = wl.ionic["ga"], wl.ionic["a"]
    s0 = wl.dof_scale.copy()
    scale = t64(s0).requires_grad_(True)
    ka = t64([k0, a0]).requires_grad_(True)
    L = TrajectoryLoss.apply(scale, ka, ctx, wl, steps, probes, targets, 1)
    L.backward()
    gs = scale.grad.cpu().numpy()
    gka = ka.grad.cpu().numpy()
    tapes = _record(ctx, wl, torch, dev, t64, steps, s0, k0, a0)
    lists = []
    for tp in tapes:
        acts = tp._act.cpu().numpy().reshape(wl.sweeps, wl.n)
        lists.append([None] + [acts[k, :tp.n_active[k]].copy() for k in range(1, wl.sweeps)])
    pr = probes.cpu().numpy()
    tg = [t.cpu().numpy() for t in targets]
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, s0)

    def tangent(ds=None, dion=None):
        Sd = oracle.System.from_mesh(wl.mesh, wl.sigma, ds) if ds is not None else None
        v, w = wl.v0.copy(), wl.w0.copy()
        dv, dw = np.zeros(wl.n), np.zeros(wl.n)
        total, dtotal = 0.0, 0.0
        for n in range(steps):
            r = S.step_tangent(wl.ionic, wl.M, v, dv, w, dw, wl.dt, wl.sweeps, lists[n],
                               dionic=dion, dscale_system=Sd, cg_rtol=1e-13,
                               istim=wl.stim_vector(n * wl.dt))
            assert r["status"] == 0
            v, w, dv, dw = r["v"], r["w"], r["dv"], r["dw"]
            e = v[pr] - tg[n]
            total += float(np.sum(e ** 2))
            dtotal += float(np.sum(2.0 * e * dv[pr]))
        return total, dtotal

    for _ in range(2):
        d = rng.standard_normal(wl.n)
        d /= np.linalg.norm(d)
        total, dl = tangent(ds=d)
        assert abs(total - L.item()) <= 1e-10 * abs(L.item())
        assert abs(dl - gs @ d) <= 1e-8 * max(abs(dl), abs(gs @ d)), (dl, gs @ d)
    zero = {k: 0.0 for k in wl.ionic}
    _, dk = tangent(dion=dict(zero, ga=1.0, gs=1.0))
    assert abs(dk - gka[0]) <= 1e-8 * max(abs(dk), abs(gka[0])), (dk, gka[0])
    _, da = tangent(dion=dict(zero, a=1.0))
    assert abs(da - gka[1]) <= 1e-8 * max(abs(da), abs(gka[1])), (da, gka[1])
    ctx.close()


def test_checkpoint_interval_does_not_change_the_gradient(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss
    steps = 5
    wl, ctx, probes, targets, rng, t64 = _setup(torch, dev, "2d", steps)
    grads = []
    for ck in (1, 2, 5):
        scale = t64(wl.dof_scale).requires_grad_(True)
        ka = t64([wl.ionic["ga"], wl.ionic["a"]]).requires_grad_(True)
        L = TrajectoryLoss.apply(scale, ka, ctx, wl, steps, probes, targets, ck)
        L.backward()
        grads.append((L.item(), scale.grad.cpu().numpy(), ka.grad.cpu().numpy()))
    for L, gs, gka in grads[1:]:
        assert L == grads[0][0]
        assert np.array_equal(gs, grads[0][1]) and np.array_equal(gka, grads[0][2])
    ctx.close()


def test_backward_uses_the_forward_parameters(torch_dev):
    """Two applications with different parameters before the first backward:
    the first gradient equals the one taken alone, and backward leaves the
    context with the parameters it held before (the second application's)."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss
    steps = 3
    wl, ctx, probes, targets, rng, t64 = _setup(torch, dev, "2d", steps)
    k0, a0 = wl.ionic["ga"], wl.ionic["a"]
    s0 = wl.dof_scale.copy()
    s1 = s0 * (1.0 + 0.05 * rng.standard_normal(wl.n))

    def grad_at(sc, k, a):
        scale = t64(sc).requires_grad_(True)
        ka = t64([k, a]).requires_grad_(True)
        return scale, ka, TrajectoryLoss.apply(scale, ka, ctx, wl, steps, probes, targets, 2)

    scale, ka, L = grad_at(s0, k0, a0)
    L.backward()
    alone = (scale.grad.cpu().numpy().copy(), ka.grad.cpu().numpy().copy())

    scale_a, ka_a, La = grad_at(s0, k0, a0)
    scale_b, ka_b, Lb = grad_at(s1, 1.1 * k0, 0.9 * a0)
    assert La.item() != Lb.item()
    La.backward()
    assert np.array_equal(scale_a.grad.cpu().numpy(), alone[0])
    assert np.array_equal(ka_a.grad.cpu().numpy(), alone[1])
    assert np.array_equal(ctx.dof_scale, s1)
    assert ctx.ionic["ga"] == 1.1 * k0 and ctx.ionic["a"] == 0.9 * a0
    Lb.backward()
    assert np.all(np.isfinite(scale_b.grad.cpu().numpy()))
    ctx.close()
