"""sdc_pcg_solve_noalloc against sdc_pcg_solve.

The no-allocation entry point serves callers whose device memory is owned by
a host framework's pool, or whose time-critical loop must not call
cudaMalloc/cudaFree; it keeps its workspace in a static device array of the
library.  This test calls it through the C ABI twice in a row on the same node
system (the second call reuses the array left by the first) and compares both
solutions with the allocating entry point's, element by element, within the
parity tolerance of the other GPU tests.  It also checks that a system larger
than the static workspace is refused before any device work.

The file name puts it last in collection order; it does not depend on any
other test having run.
"""

import numpy as np
import pytest

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


def _system():
    """Node system of the 2D square's first sweep, node 1: stiffness and lumped
    mass from the library's own assembly, a seeded J and right-hand side."""
    import workloads as W
    from paper_2311_07206_gb300 import Context
    wl = W.w0_square()
    ctx = Context.from_workload(wl)
    rp, ci, val, mass = ctx.matrix()
    ctx.close()
    rng = np.random.default_rng(2311)
    J = rng.uniform(-0.5, 2.0, wl.n)
    b = rng.standard_normal(wl.n)
    return rp, ci, val, mass, J, b


def test_noalloc_solve_matches_allocating_solve_twice(torch_dev):
    torch, dev = torch_dev
    from paper_2311_07206_gb300 import binding
    rp, ci, val, mass, J, b = _system()
    n = len(mass)
    assert n <= binding.SDC_PCG_NOALLOC_MAX_ROWS
    kdiag, ev, ec, el, ld, width = binding.csr_to_ell(rp, ci, val, n)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
    args = (n, t(ev), t(ec, torch.int32), t(el, torch.int32), ld, width, t(kdiag), t(mass), t(J),
            0.05 * 0.2, t(b))
    stream = torch.cuda.current_stream(dev).cuda_stream
    x_ref = torch.zeros(n, dtype=torch.float64, device=dev)
    it_ref, _ = binding.pcg_solve(*args, x_ref, rtol=1e-12, stream=stream)
    ref = x_ref.cpu().numpy()
    assert it_ref > 0 and np.abs(ref).max() > 0
    for call in range(2):
        x = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        it, rr = binding.pcg_solve_noalloc(*args, x, rtol=1e-12, stream=stream)
        got = x.cpu().numpy()
        assert np.abs(got - ref).max() <= RTOL * np.abs(ref).max(), "call %d" % call
        assert abs(it - it_ref) <= 1 and rr <= 1e-12


def test_noalloc_rejects_oversized_system(torch_dev):
    from paper_2311_07206_gb300 import SdcError, binding
    n = binding.SDC_PCG_NOALLOC_MAX_ROWS + 1
    with pytest.raises(SdcError) as e:
        binding.pcg_solve_noalloc(n, 0, 0, 0, n, 1, 0, 0, 0, 0.1, 0, 0)
    assert e.value.status == binding.SDC_E_INVALID
    assert "static workspace" in str(e.value)


def test_noalloc_rejects_an_ld_beyond_the_workspace(torch_dev):
    """The published m vector takes two buffers ld apart in the static array:
    9 n + ld beyond its ten vectors is refused before any device work."""
    from paper_2311_07206_gb300 import SdcError, binding
    n = 1000
    ld = 10 * binding.SDC_PCG_NOALLOC_MAX_ROWS
    with pytest.raises(SdcError) as e:
        binding.pcg_solve_noalloc(n, 0, 0, 0, ld, 1, 0, 0, 0, 0.1, 0, 0)
    assert e.value.status == binding.SDC_E_INVALID
    assert "too large" in str(e.value)
