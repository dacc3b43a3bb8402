"""Pins of the oracle's collocation data (Sec. 3.1: Radau-IIA grid, order 2M-1,
L-stability; LU-trick preconditioner cited in Sec. 3.1 after eq. SDC).

Every expected value here comes from mathematics the paper relies on, not from
the oracle: textbook Radau-IIA tableaux, polynomial exactness, numpy's own
Legendre root finder, and the nilpotency the LU trick is designed for.
"""

import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle


def test_radau3_closed_form():
    # 3-stage Radau IIA (Hairer & Wanner, Solving ODEs II, Sec. IV.5, Table 5.6).
    s6 = math.sqrt(6.0)
    tau, Q, Qh = oracle.collocation(3)
    np.testing.assert_allclose(tau, [(4 - s6) / 10, (4 + s6) / 10, 1.0], rtol=0, atol=1e-15)
    A = np.array([[(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225],
                  [(296 + 169 * s6) / 1800, (88 + 7 * s6) / 360, (-2 - 3 * s6) / 225],
                  [(16 - s6) / 36, (16 + s6) / 36, 1 / 9]])
    np.testing.assert_allclose(Q, A, rtol=0, atol=1e-15)


def test_radau2_and_1_closed_form():
    tau, Q, Qh = oracle.collocation(2)
    np.testing.assert_allclose(tau, [1 / 3, 1.0], atol=1e-15)
    np.testing.assert_allclose(Q, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)
    tau, Q, Qh = oracle.collocation(1)   # implicit Euler
    assert tau.tolist() == [1.0] and Q.tolist() == [[1.0]] and Qh.tolist() == [[1.0]]


@pytest.mark.parametrize("M", range(1, 9))
def test_nodes_match_numpy_legendre_roots(M):
    # zeros of P_M(x) - P_{M-1}(x) on [-1, 1], mapped by tau = (x+1)/2
    c = np.zeros(M + 1)
    c[M] = 1.0
    c[M - 1] = -1.0
    x = np.sort(npleg.legroots(c).real)
    tau, _, _ = oracle.collocation(M)
    np.testing.assert_allclose(tau, (x + 1) / 2, atol=1e-13)
    assert tau[-1] == 1.0
    assert np.all(np.diff(tau) > 0) and tau[0] > 0


@pytest.mark.parametrize("M", range(1, 9))
def test_stage_order_and_quadrature_exactness(M):
    tau, Q, _ = oracle.collocation(M)
    # stage order M: sum_j Q_mj tau_j^p = tau_m^{p+1} / (p+1), p <= M-1
    for p in range(M):
        np.testing.assert_allclose(Q @ tau ** p, tau ** (p + 1) / (p + 1), atol=2e-14)
    # weights b = last row of Q integrate degree <= 2M-2 exactly and fail at 2M-1
    b = Q[-1]
    for p in range(2 * M - 1):
        assert abs(b @ tau ** p - 1.0 / (p + 1)) < 2e-14
    assert abs(b @ tau ** (2 * M - 1) - 1.0 / (2 * M)) > 1e-11


@pytest.mark.parametrize("M", range(1, 9))
def test_lu_trick(M):
    _, Q, Qh = oracle.collocation(M)
    assert np.allclose(np.triu(Qh, 1), 0.0, atol=0)
    assert np.all(np.diag(Qh) > 0)
    # Q = Qhat L^T with L unit lower triangular, i.e. Qhat^{-1} Q is unit upper triangular
    U = np.linalg.solve(Qh, Q)
    np.testing.assert_allclose(np.tril(U, -1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.diag(U), 1.0, atol=1e-12)
    # stiff-limit iteration matrix E = I - Qhat^{-1} Q is nilpotent
    E = np.eye(M) - U
    np.testing.assert_allclose(np.linalg.matrix_power(E, M), 0.0, atol=1e-12)
