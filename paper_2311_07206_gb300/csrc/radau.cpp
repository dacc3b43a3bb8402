// Radau-IIA collocation data for the library (Sec. 3.1), computed on the host
// in long double once per context.
//
// Nodes: tau_M = 1 and the M-1 interior nodes are the zeros of the Jacobi
// polynomial P^{(1,0)}_{M-1} mapped from [-1, 1] to [0, 1] (Gauss-Radau rule
// with the fixed node at the right end).  The zeros are found largest first by
// Newton's method started right of every zero, with the found zeros divided
// out (for a polynomial with only real zeros this converges monotonically).
//
// Q: the cumulative collocation quadrature, Q_mj = integral over [0, tau_m] of
// the j-th Lagrange polynomial on tau_1..tau_M.  Row m is the unique solution of
// the moment conditions sum_j Q_mj tau_j^p = tau_m^(p+1)/(p+1), p = 0..M-1
// (a transposed Vandermonde system, solved by Gaussian elimination with
// partial pivoting).
//
// Qhat: the LU trick cited in Sec. 3.1 (after eq. SDC): factor Q^T = L U with
// unit lower L and take Qhat = U^T, which is lower triangular, so the node
// systems decouple and sweep sequentially.

#include <cmath>

#include "sdc_internal.h"

namespace sdc {
namespace {

// P^{(1,0)}_n(x) and its derivative by the three-term recurrence of the
// Jacobi polynomials with alpha = 1, beta = 0.
void jacobi10(int n, long double x, long double& p, long double& dp) {
    long double p0 = 1.0L, d0 = 0.0L;
    if (n == 0) { p = p0; dp = d0; return; }
    long double p1 = (3.0L * x + 1.0L) / 2.0L, d1 = 1.5L;
    for (int k = 2; k <= n; ++k) {
        // 2k(k+1)(2k-1) P_k = 2k[(2k+1)(2k-1) x + 1] P_{k-1} - 2k(k-1)(2k+1) P_{k-2}
        const long double a = 2.0L * k * (k + 1) * (2 * k - 1);
        const long double b = 2.0L * k * ((2.0L * k + 1) * (2 * k - 1) * x + 1.0L);
        const long double bx = 2.0L * k * (2.0L * k + 1) * (2 * k - 1);
        const long double c = 2.0L * k * (k - 1) * (2 * k + 1);
        const long double p2 = (b * p1 - c * p0) / a;
        const long double d2 = (bx * p1 + b * d1 - c * d0) / a;
        p0 = p1; d0 = d1; p1 = p2; d1 = d2;
    }
    p = p1;
    dp = d1;
}

}  // namespace

bool radau_collocation(int M, double* tau_out, double* Q_out, double* Qh_out) {
    if (M < 1 || M > kMaxM) return false;
    long double x[kMaxM];
    const int n = M - 1;
    for (int r = 0; r < n; ++r) {
        long double xr = 1.0L;     // right of every zero of P^{(1,0)}_n
        for (int it = 0; it < 200; ++it) {
            long double p, dp;
            jacobi10(n, xr, p, dp);
            long double ratio = dp / p;
            for (int q = 0; q < r; ++q) ratio -= 1.0L / (xr - x[q]);
            const long double step = 1.0L / ratio;
            xr -= step;
            if (std::fabs((double)step) < 1e-19) break;
        }
        x[r] = xr;
    }
    long double tau[kMaxM];
    for (int r = 0; r < n; ++r) tau[n - 1 - r] = (x[r] + 1.0L) / 2.0L;   // ascending
    tau[M - 1] = 1.0L;
    for (int j = 1; j < M; ++j)
        if (!(tau[j] > tau[j - 1]) || !(tau[0] > 0.0L)) return false;

    // Q rows from the moment conditions: V^T q_m = mu_m with V_{jp} = tau_j^p
    long double Q[kMaxM][kMaxM];
    for (int m = 0; m < M; ++m) {
        long double A[kMaxM][kMaxM + 1];
        for (int p = 0; p < M; ++p) {
            for (int j = 0; j < M; ++j) A[p][j] = std::pow(tau[j], (long double)p);
            A[p][M] = std::pow(tau[m], (long double)(p + 1)) / (long double)(p + 1);
        }
        for (int c = 0; c < M; ++c) {
            int piv = c;
            for (int r = c + 1; r < M; ++r)
                if (std::fabs((double)A[r][c]) > std::fabs((double)A[piv][c])) piv = r;
            if (piv != c)
                for (int k = 0; k <= M; ++k) { long double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            for (int r = c + 1; r < M; ++r) {
                const long double l = A[r][c] / A[c][c];
                for (int k = c; k <= M; ++k) A[r][k] -= l * A[c][k];
            }
        }
        for (int c = M - 1; c >= 0; --c) {
            long double s = A[c][M];
            for (int k = c + 1; k < M; ++k) s -= A[c][k] * Q[m][k];
            Q[m][c] = s / A[c][c];
        }
    }
    // LU trick: Q^T = L U, Qhat = U^T
    long double U[kMaxM][kMaxM] = {}, L[kMaxM][kMaxM] = {};
    for (int i = 0; i < M; ++i) {
        for (int j = i; j < M; ++j) {
            long double s = Q[j][i];                 // (Q^T)_{ij}
            for (int k = 0; k < i; ++k) s -= L[i][k] * U[k][j];
            U[i][j] = s;
        }
        if (!(std::fabs((double)U[i][i]) > 1e-14)) return false;
        L[i][i] = 1.0L;
        for (int j = i + 1; j < M; ++j) {
            long double s = Q[i][j];                 // (Q^T)_{ji}
            for (int k = 0; k < i; ++k) s -= L[j][k] * U[k][i];
            L[j][i] = s / U[i][i];
        }
    }
    for (int m = 0; m < M; ++m) {
        tau_out[m] = (double)tau[m];
        for (int j = 0; j < M; ++j) {
            Q_out[m * M + j] = (double)Q[m][j];
            Qh_out[m * M + j] = (double)U[j][m];
        }
    }
    return true;
}

}  // namespace sdc
