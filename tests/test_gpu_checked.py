"""The checked build of the library (libsdc_gb300_checked.so, built with
SDC_CHECKED=1): every gathered index in the kernels (ELL columns, active-list
entries, permutation entries, membrane-pair ends, position-table lookups,
element vertices) is tested against its bound; an index outside it is recorded,
replaced by an in-bounds one, and turns the call's status into SDC_E_INVALID.

1. The GPU tests of the small cases run again in a child process whose binding
   loads the checked build (SDC_GB300_LIB): 2D and 3D steps against the oracle,
   the 3- and 4-node meshes and the ragged 33 x 31 and 3D meshes, every M,
   empty sets, error statuses and the bounded-wait fault path, the cell-by-cell
   two-cell, grid and branched cases with and without the two-level
   preconditioner, the PCG kernel tests, batches and the adjoint.  No check may fire (a firing check fails the call), and every parity
   bar is the test's own.
2. A node system one of whose column indices lies outside the matrix is solved
   by the checked build only: the call returns SDC_E_INVALID naming the check
   site, and the next, valid call succeeds.  The bad index is chosen inside the
   arrays' allocations as well.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_07206_gb300 import build as b
    b.build()
    return b.build(checked=True)


def _env(lib):
    env = dict(os.environ)
    env["SDC_GB300_LIB"] = lib
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


def test_small_cases_pass_under_the_checked_build(checked_lib):
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_kernels.py", "tests/test_gpu_emi.py",
             "tests/test_gpu_emi_coarse.py", "tests/test_gpu_batch.py",
             "tests/test_gpu_adjoint.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-q", "-x",
                        "-m", "gpu and not slow", "-k", "not full_size"],
                       cwd=ROOT, env=_env(checked_lib), capture_output=True, text=True,
                       timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail


CHILD = r"""
import numpy as np, torch
from paper_2311_07206_gb300 import binding
assert binding.LIB_PATH.endswith("libsdc_gb300_checked.so"), binding.LIB_PATH
dev = torch.device("cuda:0")
rng = np.random.default_rng(7)
n = 40
K = np.zeros((n, n))
for i in range(n):
    for j in (i - 1, i + 1, i + 7):
        if 0 <= j < n and j != i:
            w = rng.uniform(0.5, 1.5)
            K[i, j] -= w; K[j, i] -= w; K[i, i] += w; K[j, j] += w
rp, ci, val = [0], [], []
for i in range(n):
    nz = np.nonzero(K[i])[0]
    ci += nz.tolist(); val += K[i, nz].tolist(); rp.append(len(ci))
kdiag, ev, ec, el, ld, width = binding.csr_to_ell(np.array(rp), np.array(ci, np.int32),
                                                  np.array(val), n)
t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
mass = np.ones(n)
b_rhs = rng.uniform(-1, 1, n)
args = lambda col: (n, t(ev), t(col, torch.int32), t(el, torch.int32), ld, width, t(kdiag),
                    t(mass), t(np.zeros(n)), 0.1, t(b_rhs))
stream = torch.cuda.current_stream(dev).cuda_stream


def solve(col):
    x = torch.zeros(64, dtype=torch.float64, device=dev)[:n]
    it, rr = binding.pcg_solve(*args(col), x, rtol=1e-10, maxit=500, stream=stream)
    return x.cpu().numpy(), it, rr


x1, it1, rr1 = solve(ec)
A = np.eye(n) + 0.1 * K
assert np.abs(A @ x1 - b_rhs).max() <= 1e-8, np.abs(A @ x1 - b_rhs).max()
bad = np.array(ec, copy=True)
bad.reshape(-1)[0 * ld + 5] = n + 3   # slot 0 of row 5 (slot-major): a column past the last row
try:
    solve(bad)
    raise SystemExit("the out-of-range column was not reported")
except binding.SdcError as e:
    assert e.status == binding.SDC_E_INVALID, e
    assert "checked build" in str(e) and "index %d" % (n + 3) in str(e), e
x2, it2, rr2 = solve(ec)
assert it2 == it1 and np.array_equal(x1, x2), (it1, it2, rr1, rr2)
print("checked ok")
"""


def test_out_of_range_column_is_reported_by_the_checked_build(checked_lib):
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=_env(checked_lib),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout + r.stderr)[-3000:]
