"""Kernel-level GPU tests of the restricted Jacobi-PCG (the node systems of
eq. final-sdc, Sec. 3.2 / Sec. 4.2) through sdc_pcg_solve, against dense
numpy solves of the same systems."""

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


def _laplacian_system(n, seed):
    """Weighted graph Laplacian with ragged degrees (symmetric, zero row sums,
    negative off-diagonals) and a positive lumped mass."""
    rng = np.random.default_rng(seed)
    edges = set()
    for i in range(n):
        for _ in range(rng.integers(1, 6)):
            j = int(rng.integers(0, n))
            if j != i:
                edges.add((min(i, j), max(i, j)))
    K = np.zeros((n, n))
    for i, j in edges:
        w = rng.uniform(0.1, 2.0)
        K[i, j] -= w
        K[j, i] -= w
        K[i, i] += w
        K[j, j] += w
    mass = rng.uniform(0.5, 1.5, n)
    rp = [0]
    ci, val = [], []
    for i in range(n):
        nz = np.nonzero(K[i])[0]
        ci.extend(nz.tolist())
        val.extend(K[i, nz].tolist())
        rp.append(len(ci))
    return K, mass, np.array(rp), np.array(ci, np.int32), np.array(val)


def _mesh_system():
    wl = W.w0_square()
    S = oracle.System.from_mesh(wl.mesh, wl.sigma)
    rp, ci, val, mass = S.matrix()
    K, _ = S.dense()
    return K, mass, rp, ci, val


def _solve(torch, dev, K, mass, rp, ci, val, J, c, b, rtol=1e-13, maxit=20000):
    from paper_2311_07206_gb300 import binding
    n = len(mass)
    kdiag, ev, ec, el, ld, width = binding.csr_to_ell(rp, ci, val, n)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    it, rr = binding.pcg_solve(n, t(ev), t(ec, torch.int32), t(el, torch.int32), ld, width,
                               t(kdiag), t(mass), t(J), c, t(b), x, rtol=rtol, maxit=maxit,
                               stream=torch.cuda.current_stream(dev).cuda_stream)
    return x.cpu().numpy(), it, rr


@pytest.mark.parametrize("system", ["mesh", "graph"])
def test_pcg_solve_matches_dense_solve(torch_dev, system):
    torch, dev = torch_dev
    if system == "mesh":
        K, mass, rp, ci, val = _mesh_system()
    else:
        K, mass, rp, ci, val = _laplacian_system(3001, seed=11)
    n = len(mass)
    rng = np.random.default_rng(5)
    J = rng.uniform(-0.5, 2.0, n)
    c = 0.05 * 0.2
    b = rng.standard_normal(n)
    x, it, rr = _solve(torch, dev, K, mass, rp, ci, val, J, c, b)
    A = np.diag(mass * (1 + c * J)) + c * K
    ref = np.linalg.solve(A, b)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    assert 0 < it < 1000 and rr <= 1e-13


@pytest.mark.parametrize("n", [40, 300, 1000])
def test_pcg_solve_small_systems_with_padded_ld(torch_dev, n):
    """One to four blocks, and an ELL leading dimension above n (rounded up to 32,
    and 64 more): the second buffer of the published m vector lies ld after the
    first, so the workspace must hold 2 ld for it."""
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import binding
    K, mass, rp, ci, val = _laplacian_system(n, seed=n)
    rng = np.random.default_rng(n)
    J = rng.uniform(-0.5, 2.0, n)
    c = 0.1
    b = rng.standard_normal(n)
    A = np.diag(mass * (1 + c * J)) + c * K
    ref = np.linalg.solve(A, b)
    kdiag, ev, ec, el, ld, width = binding.csr_to_ell(rp, ci, val, n)
    for pad in (0, 64):
        ld2 = ld + pad
        ev2 = np.zeros((ev.shape[0], ld2))
        ec2 = np.zeros((ec.shape[0], ld2), np.int32)
        ev2[:, :ld], ec2[:, :ld] = ev, ec
        t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        it, rr = binding.pcg_solve(n, t(ev2), t(ec2, torch.int32), t(el, torch.int32), ld2, width,
                                   t(kdiag), t(mass), t(J), c, t(b), x, rtol=1e-13, maxit=2000,
                                   stream=torch.cuda.current_stream(dev).cuda_stream)
        assert np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
        assert 0 < it < 200 and rr <= 1e-13


def test_pcg_solve_zero_rhs_and_errors(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import SdcError, binding
    K, mass, rp, ci, val = _laplacian_system(257, seed=3)
    n = len(mass)
    J = np.zeros(n)
    x, it, rr = _solve(torch, dev, K, mass, rp, ci, val, J, 0.1, np.zeros(n))
    assert it == 0 and np.all(x == 0.0)
    b = np.ones(n)
    with pytest.raises(SdcError) as e:
        _solve(torch, dev, K, mass, rp, ci, val, J, 0.1, b, maxit=1)
    assert e.value.status == binding.SDC_E_CG_NOCONV
    Jbad = J.copy()
    Jbad[7] = -1e6
    with pytest.raises(SdcError) as e:
        _solve(torch, dev, K, mass, rp, ci, val, Jbad, 0.1, b)
    assert e.value.status == binding.SDC_E_DOMAIN
    with pytest.raises(SdcError) as e:
        binding.pcg_solve(0, 0, 0, 0, 32, 1, 0, 0, 0, 0.1, 0, 0)
    assert e.value.status == binding.SDC_E_INVALID
