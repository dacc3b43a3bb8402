"""Pins of the oracle's two-level preconditioner for the cell-by-cell node
systems (Sec. 6: block preconditioning of EMI systems; blocks = the subdomains
holding active dofs):
    z = D^-1 r + Z E^-1 Z' r,   Z = subdomain indicator vectors on the active set,
                                E = Z' A Z.

Expected values come from what the definition fixes:
1. With an empty coarse space (every label -1) the preconditioner is Jacobi, and
   the solve and the whole EMI step equal the Jacobi ones bitwise.
2. The coarse part is exact on the constant-per-subdomain subspace: for
   r = A Z y, z - D^-1 r = Z y (A, Z, y built here with scipy), on all dofs and on
   a restricted active set.
3. The preconditioned CG converges to the dense solve (numpy) of the two-cell
   node system, in fewer iterations than Jacobi-PCG, and the EMI step with it
   reaches the state of the Jacobi step within the solves' tolerance.
The subdomain labels of the cell-by-cell workloads are the connected components
of the stiffness matrix's graph (each subdomain's mesh is connected, and only
membrane pairs join subdomains), which is how the library finds them.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

import oracle
from workloads.emi import coarse_blocks, emi_tiny


def _node_system(wl, c=None, seed=0):
    """Node operator A = B + c (K + R + D) of the first node (M = 3) with the pair
    Jacobians at a seeded state, as a scipy CSR matrix."""
    S = oracle.System.from_mesh(wl.mesh)
    ptr, col, val, _ = S.matrix()
    n = wl.n
    K = sp.csr_matrix((val, col, ptr), shape=(n, n))
    _, _, Qh = oracle.collocation(3)
    c = wl.dt * Qh[0, 0] if c is None else c
    rng = np.random.default_rng(seed)
    p = wl.ionic
    v = rng.uniform(-0.1, 1.0, wl.n_pairs)
    J = np.where(wl.pair_kind == 0,
                 p["ga"] * (3 * v * v - 2 * (1 + p["a"]) * v + p["a"]) + 0.02, wl.g_gap)
    coef = wl.pair_area * (wl.Cm + c * J)
    pk, pl = wl.pair_k, wl.pair_l
    Bp = sp.csr_matrix((np.concatenate([coef, coef, -coef, -coef]),
                        (np.concatenate([pk, pl, pk, pl]), np.concatenate([pk, pl, pl, pk]))),
                       shape=(n, n))
    A = (Bp + c * (K + sp.diags(wl.robin))).tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("kind", ["two_cells", "grid", "branched_2d"])
def test_subdomain_labels_are_the_stiffness_graph_components(kind):
    wl = emi_tiny(kind)
    S = oracle.System.from_mesh(wl.mesh)
    ptr, col, val, _ = S.matrix()
    K = sp.csr_matrix((val, col, ptr), shape=(wl.n, wl.n))
    ncomp, comp = csgraph.connected_components(K != 0, directed=False)
    assert ncomp == len(np.unique(wl.labels))
    # the same partition: every component carries one label and vice versa
    pairs = set(zip(comp.tolist(), wl.labels.tolist()))
    assert len(pairs) == ncomp


def test_empty_coarse_space_is_jacobi_bitwise():
    wl = emi_tiny("two_cells")
    A = _node_system(wl)
    b = np.random.default_rng(1).standard_normal(wl.n)
    x0, it0, rc0 = oracle.pcg_csr(A.indptr, A.indices, A.data, b, rtol=1e-12)
    x1, it1, rc1 = oracle.pcg_csr(A.indptr, A.indices, A.data, b, dom=np.full(wl.n, -1),
                                  rtol=1e-12)
    assert rc0 == rc1 == 0 and it0 == it1 and np.array_equal(x0, x1)
    # the whole step
    S = oracle.System.from_mesh(wl.mesh)
    plain = S.step_emi(wl, wl.u0, wl.w0)
    wl2 = emi_tiny("two_cells")
    wl2.labels = np.full(wl2.n, -1, np.int32)
    empty = S.step_emi(wl2, wl2.u0, wl2.w0, coarse=True)
    assert plain["status"] == empty["status"] == 0
    assert np.array_equal(plain["u"], empty["u"]) and np.array_equal(plain["w"], empty["w"])


@pytest.mark.parametrize("kind", ["two_cells", "grid"])
@pytest.mark.parametrize("restricted", [False, True])
def test_coarse_part_is_exact_on_subdomain_constants(kind, restricted):
    wl = emi_tiny(kind)
    A = _node_system(wl, seed=2)
    n = wl.n
    rng = np.random.default_rng(3)
    act = np.arange(n)
    if restricted:
        act = np.sort(rng.choice(n, size=n * 2 // 3, replace=False))
    Aa = A[act][:, act]
    lab = wl.labels[act]
    q = lab.max() + 1
    Z = sp.csr_matrix((np.ones(len(act)), (np.arange(len(act)), lab)), shape=(len(act), q))
    present = np.unique(lab)
    y = np.zeros(q)
    y[present] = rng.standard_normal(len(present))
    r_act = Aa @ (Z @ y)
    r = np.zeros(n)
    r[act] = r_act
    z = oracle.two_level_apply(A.indptr, A.indices, A.data, r, wl.labels, act=act)
    d = Aa.diagonal()
    # On a whole subdomain the stiffness part of A Z y (and of E) cancels exactly in
    # exact arithmetic (zero row sums); in FP64 it leaves a residue of ~1e-16 of the
    # stiffness diagonal against the much smaller membrane and Robin terms, ~1e-10
    # relative on these meshes.  A wrong E, label map or missing Jacobi term is O(1).
    np.testing.assert_allclose(z[act] - r_act / d, Z @ y, rtol=0,
                               atol=1e-8 * np.abs(Z @ y).max())
    off = np.setdiff1d(np.arange(n), act)
    assert np.all(z[off] == 0.0)


@pytest.mark.parametrize("kind", ["two_cells", "grid"])
def test_two_level_pcg_matches_dense_solve_in_fewer_iterations(kind):
    wl = emi_tiny(kind)
    A = _node_system(wl, seed=4)
    b = np.random.default_rng(5).standard_normal(wl.n)
    ref = np.linalg.solve(A.toarray(), b)
    xj, itj, rcj = oracle.pcg_csr(A.indptr, A.indices, A.data, b, rtol=1e-12)
    x2, it2, rc2 = oracle.pcg_csr(A.indptr, A.indices, A.data, b, dom=wl.labels, rtol=1e-12)
    assert rcj == rc2 == 0
    scale = np.abs(ref).max()
    assert np.abs(x2 - ref).max() <= 1e-9 * scale
    assert np.abs(xj - ref).max() <= 1e-9 * scale
    assert it2 < itj, (it2, itj)


def test_emi_step_with_two_level_preconditioner():
    wl = emi_tiny("two_cells")
    S = oracle.System.from_mesh(wl.mesh)
    jac = S.step_emi(wl, wl.u0, wl.w0, tol=0.0, cg_rtol=1e-13)
    two = S.step_emi(wl, wl.u0, wl.w0, tol=0.0, cg_rtol=1e-13, coarse=True)
    assert jac["status"] == two["status"] == 0
    scale = max(1.0, np.abs(jac["u"]).max())
    assert np.abs(two["u"] - jac["u"]).max() <= 1e-10 * scale
    assert np.abs(two["w"] - jac["w"]).max() <= 1e-10
    it_j = sum(jac["stats"].cg_iters[k * 8 + m] for k in range(wl.sweeps) for m in range(wl.M))
    it_2 = sum(two["stats"].cg_iters[k * 8 + m] for k in range(wl.sweeps) for m in range(wl.M))
    assert it_2 < it_j, (it_2, it_j)


def test_block_major_renumbering_is_a_relabelling():
    """Numbering the dofs block by block (workloads.emi.block_major) permutes the
    step's result and changes nothing else: the oracle's step of the renumbered
    workload equals the permuted step of the original to rounding, with the same
    active-set sizes."""
    from workloads.emi import block_major, coarse_blocks, renumber
    wl = emi_tiny("grid")
    blocks = coarse_blocks(wl, split=(4, 2, 2))
    order, b2 = block_major(wl, blocks)
    assert np.array_equal(np.sort(order), np.arange(wl.n))
    assert np.all(np.diff(b2) >= 0)                       # blocks contiguous
    w2 = renumber(wl, order)
    S1 = oracle.System.from_mesh(wl.mesh)
    S2 = oracle.System.from_mesh(w2.mesh)
    r1 = S1.step_emi(wl, wl.u0, wl.w0)
    r2 = S2.step_emi(w2, w2.u0, w2.w0)
    assert r1["status"] == r2["status"] == 0
    scale = max(1.0, np.abs(r1["u"]).max())
    assert np.abs(r1["u"][order] - r2["u"]).max() <= 1e-12 * scale
    assert np.abs(r1["w"] - r2["w"]).max() <= 1e-12
    assert list(r1["stats"].n_active) == list(r2["stats"].n_active)


def test_block_labels_need_not_be_consecutive_and_one_block_is_allowed():
    """Labels are only names: spreading them out (unused labels between) changes
    nothing, bitwise; a single block (one coarse vector, every active dof) is a
    valid coarse space whose step agrees with the Jacobi step within the solves'
    tolerance."""
    wl = emi_tiny("grid")
    blocks = coarse_blocks(wl, split=(4, 2, 2))
    S = oracle.System.from_mesh(wl.mesh)
    a = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=blocks)
    b = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=2 * blocks + 3)
    assert a["status"] == b["status"] == 0
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["w"], b["w"])
    assert list(a["stats"].cg_iters) == list(b["stats"].cg_iters)
    one = S.step_emi(wl, wl.u0, wl.w0, tol=0.0, cg_rtol=1e-13, coarse=np.zeros(wl.n, np.int32))
    jac = S.step_emi(wl, wl.u0, wl.w0, tol=0.0, cg_rtol=1e-13)
    assert one["status"] == jac["status"] == 0
    scale = max(1.0, np.abs(jac["u"]).max())
    assert np.abs(one["u"] - jac["u"]).max() <= 1e-10 * scale


def test_coarse_min_rows_chooses_the_preconditioner_per_sweep():
    """coarse_min_rows: sweeps with fewer active dofs solve with Jacobi alone.  Above
    every sweep's size it is the Jacobi step bitwise, at 0 the two-level step bitwise;
    between the first and the second sweep's sizes the first sweep keeps the
    two-level solves (same iteration counts, same next active set) and the step ends
    within the solves' and the sweeps' tolerance of the two-level one."""
    wl = emi_tiny("grid")
    blocks = coarse_blocks(wl, split=(4, 2, 2))
    S = oracle.System.from_mesh(wl.mesh)
    jac = S.step_emi(wl, wl.u0, wl.w0, want_log=True)
    two = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=blocks)
    off = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=blocks, coarse_min_rows=10 ** 9)
    on = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=blocks, coarse_min_rows=0)
    assert np.array_equal(off["u"], jac["u"]) and np.array_equal(off["w"], jac["w"])
    assert np.array_equal(on["u"], two["u"]) and np.array_equal(on["w"], two["w"])
    n0, n1 = two["stats"].n_active[0], two["stats"].n_active[1]
    assert n1 < n0
    mid = S.step_emi(wl, wl.u0, wl.w0, want_log=True, coarse=blocks, coarse_min_rows=n1 + 1)
    assert mid["status"] == 0
    assert [mid["stats"].cg_iters[m] for m in range(wl.M)] == \
        [two["stats"].cg_iters[m] for m in range(wl.M)]
    assert mid["stats"].n_active[1] == n1
    scale = max(1.0, np.abs(two["u"]).max())
    assert np.abs(mid["u"] - two["u"]).max() <= 10 * wl.tol * scale
