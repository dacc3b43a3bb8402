"""Pins of the oracle's P1 assembly (Sec. 2.2, eq. abstract monodomain) and of
its Aliev-Panfilov model (Sec. 5.1.1).

Expected values come from closed forms: the finite-difference stencils that P1
elements reduce to on these structured meshes, exactness of P1 on linear
fields, measure of the domain, and root / nullcline / derivative properties of
the ionic model (derivatives checked by central differences).
"""

import numpy as np
import pytest

import oracle
from workloads import AP_BENCH, AP_PAPER, grid2d, kuhn3d


def _assemble(mesh, sigma, scale=None):
    S = oracle.System.from_mesh(mesh, sigma, scale)
    return S, S.dense()


def test_2d_right_triangles_give_five_point_stencil():
    n, h = 6, 0.3125
    mesh = grid2d(n, n, h)
    dx, dy = 1.3, 0.4
    _, (K, m) = _assemble(mesh, np.diag([dx, dy, 1.0]))
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            r = i + n * j
            row = K[r]
            assert row[r] == pytest.approx(2 * dx + 2 * dy, rel=1e-14)
            assert row[r - 1] == pytest.approx(-dx, rel=1e-14)
            assert row[r + 1] == pytest.approx(-dx, rel=1e-14)
            assert row[r - n] == pytest.approx(-dy, rel=1e-14)
            assert row[r + n] == pytest.approx(-dy, rel=1e-14)
            # hypotenuse couplings cancel exactly for diagonal D
            assert row[r + n + 1] == 0.0 and row[r - n - 1] == 0.0
            assert m[r] == pytest.approx(h * h, rel=1e-14)
    assert m.sum() == pytest.approx(((n - 1) * h) ** 2, rel=1e-14)
    np.testing.assert_allclose(K, K.T, atol=0)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-14)


def test_3d_kuhn_gives_seven_point_stencil():
    nx, ny, nz, h = 5, 4, 4, 0.1
    mesh = kuhn3d(nx, ny, nz, h)
    D = np.diag([1.0, 0.25, 0.25])
    _, (K, m) = _assemble(mesh, D)
    off = {1: -D[0, 0] * h, nx: -D[1, 1] * h, nx * ny: -D[2, 2] * h}
    for k in range(1, nz - 1):
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                r = i + nx * (j + ny * k)
                for s, val in off.items():
                    assert K[r, r + s] == pytest.approx(val, rel=1e-12)
                    assert K[r, r - s] == pytest.approx(val, rel=1e-12)
                assert K[r, r] == pytest.approx(-2 * sum(off.values()), rel=1e-12)
                # face- and body-diagonal couplings vanish up to rounding of the coordinates
                others = np.delete(K[r], [r, r + 1, r - 1, r + nx, r - nx, r + nx * ny, r - nx * ny])
                assert np.abs(others).max() <= 1e-13 * K[r, r]
                assert m[r] == pytest.approx(h ** 3, rel=1e-12)
    vol = (nx - 1) * (ny - 1) * (nz - 1) * h ** 3
    assert m.sum() == pytest.approx(vol, rel=1e-13)
    np.testing.assert_allclose(K, K.T, atol=1e-18)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_fields_on_distorted_mesh(dim):
    """P1 reproduces linear fields: interior rows of K a.x vanish and the energy
    a^T K a equals |Omega| a^T D a (catches wrong gradients, volumes, or a
    transposed tensor)."""
    rng = np.random.default_rng(7)
    mesh = grid2d(5, 6, 0.25) if dim == 2 else kuhn3d(4, 3, 5, 0.2)
    # random affine map keeps the simplices affine images of the originals
    T = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    mesh.xyz = mesh.xyz @ T.T
    D = rng.standard_normal((3, 3))
    D = D @ D.T + 0.5 * np.eye(3)
    D[0, 1] += 0.2      # slightly non-symmetric: a^T D a uses the symmetric part only
    _, (K, m) = _assemble(mesh, D)
    a = rng.standard_normal(dim)
    u = mesh.xyz @ a
    Ku = K @ u
    vol = m.sum()
    Dd = D[:dim, :dim]
    assert u @ Ku == pytest.approx(vol * (a @ Dd @ a), rel=1e-12)
    # interior nodes (of the original grid) carry no flux
    nx = 5 if dim == 2 else 4
    if dim == 2:
        interior = [i + 5 * j for j in range(1, 5) for i in range(1, 4)]
    else:
        interior = [i + 4 * (j + 3 * k) for k in range(1, 4) for j in range(1, 2) for i in range(1, 3)]
    np.testing.assert_allclose(Ku[interior], 0.0, atol=1e-12)
    assert nx > 0


def test_dof_scale_uses_element_mean():
    mesh = grid2d(4, 4, 0.5)
    s = np.linspace(0.5, 1.5, mesh.n_nodes)
    _, (K1, _) = _assemble(mesh, np.eye(3))
    _, (Ks, _) = _assemble(mesh, np.eye(3), s)
    # a single element's contribution scales by the mean of its vertex scales:
    # compare against per-element assembly with constant scale
    K_ref = np.zeros_like(K1)
    for e in mesh.elems:
        sub = grid2d(4, 4, 0.5)
        sub.elems = e[None, :].astype(np.int32)
        _, (Ke, _) = _assemble(sub, np.eye(3))
        K_ref += s[e].mean() * Ke
    np.testing.assert_allclose(Ks, K_ref, atol=1e-14)


@pytest.mark.parametrize("p", [AP_BENCH, AP_PAPER])
def test_aliev_panfilov_roots_and_nullcline(p):
    for v in (0.0, p["a"], 1.0):
        assert oracle.ionic_eval(p, v, 0.0)[0] == pytest.approx(0.0, abs=1e-15)
    for v, w in [(0.3, 0.7), (0.9, 1.2), (-0.05, 0.1)]:
        I0 = oracle.ionic_eval(p, v, 0.0)[0]
        assert oracle.ionic_eval(p, v, w)[0] - I0 == pytest.approx(v * w, rel=1e-13)
        # w on the nullcline w* = -gs v (v - a - 1) makes R vanish
        wstar = -p["gs"] * v * (v - p["a"] - 1.0)
        assert oracle.ionic_eval(p, v, wstar)[3] == pytest.approx(0.0, abs=1e-14)
    # resting state (0, 0) is an equilibrium
    out = oracle.ionic_eval(p, 0.0, 0.0)
    assert out[0] == 0.0 and out[3] == 0.0
    # the 1/4 prefactor of the paper's R scales the whole rate
    q = dict(p)
    q["cw"] = 1.0
    assert oracle.ionic_eval(p, 0.4, 0.2)[3] == pytest.approx(p["cw"] * oracle.ionic_eval(q, 0.4, 0.2)[3], rel=1e-14)


@pytest.mark.parametrize("p", [AP_BENCH, AP_PAPER])
@pytest.mark.parametrize("vw", [(0.05, 0.0), (0.4, 0.3), (0.95, 1.1), (0.2, 2.0)])
def test_aliev_panfilov_derivatives_by_central_differences(p, vw):
    v, w = vw
    h = 1e-6
    f = lambda a, b: oracle.ionic_eval(p, a, b)
    d = f(v, w)
    dIdv = (f(v + h, w)[0] - f(v - h, w)[0]) / (2 * h)
    dIdw = (f(v, w + h)[0] - f(v, w - h)[0]) / (2 * h)
    dRdv = (f(v + h, w)[3] - f(v - h, w)[3]) / (2 * h)
    dRdw = (f(v, w + h)[3] - f(v, w - h)[3]) / (2 * h)
    assert d[1] == pytest.approx(dIdv, rel=1e-7, abs=1e-8)
    assert d[2] == pytest.approx(dIdw, rel=1e-7, abs=1e-8)
    assert d[4] == pytest.approx(dRdv, rel=1e-7, abs=1e-8)
    assert d[5] == pytest.approx(dRdw, rel=1e-7, abs=1e-8)
