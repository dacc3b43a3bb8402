// Plain FP64 CPU oracle for the adaptive SDC step (test infrastructure).
//
// This file is the parity authority for the CUDA library.  It is slow on
// purpose: single-threaded loops in the order the paper states the method, no
// BLAS, no blocking, no fusion.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load it; the library never does, and this file
// shares no code, header or constant table with the library.
//
// What it computes (paper sections in brackets):
//   * right Radau-IIA collocation nodes tau_1..tau_M with tau_M = 1, the
//     cumulative quadrature matrix Q_mj = int_0^{tau_m} l_j, and the LU-trick
//     lower-triangular preconditioner Qhat = U^T where Q^T = L U     [Sec. 3.1]
//   * P1 finite elements: stiffness K, lumped mass m                 [Sec. 2.2]
//   * Aliev-Panfilov current I_ion and gating rate R                [Sec. 5.1.1]
//   * one SDC time step with operator-splitting sweeps (v then w) and
//     nested algebraic active sets I_{k+1} = {i in I_k : |dv_i| >= TOL_drop}
//                                                  [Sec. 3.2, eq. final-sdc; Sec. 4.2]
//   * Jacobi-preconditioned CG on the restricted systems            [Sec. 4.2]
//   * for cell-by-cell systems, optionally the additive two-level
//     preconditioner over the subdomains (block preconditioning)     [Sec. 6]
//   * a dense Newton solve of the full collocation system (tiny meshes),
//     the fixed point the SDC sweeps converge to                     [Sec. 3.1]
//
// Readings where the paper is ambiguous or garbled (each also listed in the
// design notes):
//   - Q is built on tau_1..tau_M only (standard Radau-IIA collocation); the
//     node-to-node form S_i = Q_{i+1} - Q_i of eq. SDC Integration is equivalent.
//   - the w correction of eq. final-sdc is read in its Newton-consistent form
//     eps_m = (s_m + dt sum_{j<m} Qhat_mj dR_j eps_j) / (1 - dt Qhat_mm dR_m).
//   - the predictor spreads the step's initial value to all nodes.
//   - selection uses max over the M nodes of |dv_{m,i}| (v only).
//   - the ionic load is lumped: b_i = m_i (I_ion(v_i, w_i) - I_stim,i).
//
// All parts are pinned by the CPU tests (Radau closed forms and exactness,
// LU-trick nilpotency, SDC fixed point == direct collocation solve, Pade
// stability function, observed time order, assembly stencils, conservation,
// adaptivity invariants).

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

// --------------------------------------------------------------------------
// Collocation (Sec. 3.1)
// --------------------------------------------------------------------------

// Legendre polynomial P_n(x) by the three-term recurrence.
long double legendre(int n, long double x) {
    if (n == 0) return 1.0L;
    long double p0 = 1.0L, p1 = x;
    for (int k = 1; k < n; ++k) {
        long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// Radau right polynomial on [-1, 1]: P_M(x) - P_{M-1}(x); its zeros map to the
// Radau-IIA nodes by tau = (x + 1) / 2, and x = 1 is always one of them.
long double radau_poly(int M, long double x) { return legendre(M, x) - legendre(M - 1, x); }

// Nodes by sign-change bracketing on a fine grid, then bisection.
bool radau_nodes(int M, std::vector<long double>& tau) {
    tau.clear();
    const int samples = 40000;
    const long double lo = -1.0L, hi = 1.0L - 1e-3L;
    long double xa = lo, fa = radau_poly(M, xa);
    for (int s = 1; s <= samples; ++s) {
        long double xb = lo + (hi - lo) * s / samples;
        long double fb = radau_poly(M, xb);
        if (fa == 0.0L) {
            tau.push_back((xa + 1.0L) / 2.0L);
        } else if ((fa < 0) != (fb < 0) && fb != 0.0L) {
            long double a = xa, b = xb, f_a = fa;
            for (int it = 0; it < 200; ++it) {
                long double c = 0.5L * (a + b);
                long double fc = radau_poly(M, c);
                if (fc == 0.0L) { a = b = c; break; }
                if ((fc < 0) == (f_a < 0)) { a = c; f_a = fc; } else { b = c; }
            }
            tau.push_back((0.5L * (a + b) + 1.0L) / 2.0L);
        }
        xa = xb;
        fa = fb;
    }
    tau.push_back(1.0L);
    return (int)tau.size() == M;
}

// Q[m][j] = integral over [0, tau_m] of the Lagrange polynomial l_j on tau_1..tau_M.
void quadrature_matrix(const std::vector<long double>& tau, std::vector<long double>& Q) {
    const int M = (int)tau.size();
    Q.assign(M * M, 0.0L);
    for (int j = 0; j < M; ++j) {
        // monomial coefficients of l_j(s) = prod_{k != j} (s - tau_k) / (tau_j - tau_k)
        std::vector<long double> c(1, 1.0L);
        for (int k = 0; k < M; ++k) {
            if (k == j) continue;
            long double den = tau[j] - tau[k];
            std::vector<long double> nc(c.size() + 1, 0.0L);
            for (size_t p = 0; p < c.size(); ++p) {
                nc[p + 1] += c[p] / den;
                nc[p] -= c[p] * tau[k] / den;
            }
            c.swap(nc);
        }
        for (int m = 0; m < M; ++m) {
            long double s = 0.0L, tp = tau[m];
            for (size_t p = 0; p < c.size(); ++p) {
                s += c[p] * tp / (long double)(p + 1);
                tp *= tau[m];
            }
            Q[m * M + j] = s;
        }
    }
}

// LU trick: Q^T = L U (Doolittle, unit lower L, no pivoting); Qhat = U^T.
bool lu_trick(int M, const std::vector<long double>& Q, std::vector<long double>& Qhat) {
    std::vector<long double> A(M * M), L(M * M, 0.0L), U(M * M, 0.0L);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) A[i * M + j] = Q[j * M + i];
    for (int i = 0; i < M; ++i) {
        for (int j = i; j < M; ++j) {
            long double s = A[i * M + j];
            for (int k = 0; k < i; ++k) s -= L[i * M + k] * U[k * M + j];
            U[i * M + j] = s;
        }
        if (std::fabs((double)U[i * M + i]) < 1e-14) return false;
        L[i * M + i] = 1.0L;
        for (int j = i + 1; j < M; ++j) {
            long double s = A[j * M + i];
            for (int k = 0; k < i; ++k) s -= L[j * M + k] * U[k * M + i];
            L[j * M + i] = s / U[i * M + i];
        }
    }
    Qhat.assign(M * M, 0.0L);
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j) Qhat[m * M + j] = U[j * M + m];
    return true;
}

struct Collocation {
    int M = 0;
    std::vector<double> tau, Q, Qhat;  // row-major M x M
};

// qhat = 0: LU trick (Qhat = U^T with Q^T = L U); qhat = 1: implicit Euler, the
// right-looking rectangle rule of Sec. 3.1 in cumulative form,
// Qhat_mj = tau_j - tau_{j-1} for j <= m (tau_0 = 0), i.e. z_m = z_0 + sum_{j<=m} dtau_j f(z_j).
bool make_collocation(int M, Collocation& c, int qhat = 0) {
    if (M < 1 || M > 8 || qhat < 0 || qhat > 1) return false;
    std::vector<long double> tau, Q, Qh;
    if (!radau_nodes(M, tau)) return false;
    quadrature_matrix(tau, Q);
    if (qhat == 0) {
        if (!lu_trick(M, Q, Qh)) return false;
    } else {
        Qh.assign((size_t)M * M, 0.0L);
        for (int m = 0; m < M; ++m)
            for (int j = 0; j <= m; ++j) Qh[(size_t)m * M + j] = tau[j] - (j > 0 ? tau[j - 1] : 0.0L);
    }
    c.M = M;
    c.tau.assign(tau.begin(), tau.end());
    c.Q.assign(Q.begin(), Q.end());
    c.Qhat.assign(Qh.begin(), Qh.end());
    return true;
}

// --------------------------------------------------------------------------
// Sparse matrix and P1 assembly (Sec. 2.2)
// --------------------------------------------------------------------------

struct Csr {
    int n = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};

struct System {
    Csr K;                      // stiffness (includes the diagonal)
    std::vector<double> mass;   // lumped mass (diagonal)
};

double det3(const double a[3][3]) {
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

// K = sum_e sbar_e |e| G_e^T D_e G_e and m_i = sum_{e containing i} |e| / (d+1).
// Duplicate contributions are summed in element order.
bool assemble(int dim, int n_nodes, const double* xyz, int n_elems, const int* elems,
              const double* sigma9, const double* elem_sigma9, const double* dof_scale,
              System& sys) {
    if (dim != 2 && dim != 3) return false;
    const int nv = dim + 1;
    std::vector<std::vector<std::pair<int, double>>> rows(n_nodes);
    sys.mass.assign(n_nodes, 0.0);
    for (int e = 0; e < n_elems; ++e) {
        const int* vtx = elems + (size_t)e * nv;
        for (int a = 0; a < nv; ++a)
            if (vtx[a] < 0 || vtx[a] >= n_nodes) return false;
        // Jacobian: column c = x_{c+1} - x_0
        double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c)
                J[r][c] = xyz[(size_t)vtx[c + 1] * dim + r] - xyz[(size_t)vtx[0] * dim + r];
        double det = det3(J);
        if (det == 0.0) return false;
        double vol = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
        // inverse by cofactors: inv[r][c] = cof[c][r] / det
        double inv[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
                inv[r][c] = (J[r1][c1] * J[r2][c2] - J[r1][c2] * J[r2][c1]) / det;
            }
        // gradients of the barycentric coordinates: grad l_{c+1} = row c of inv
        double g[4][3] = {{0}};
        for (int c = 0; c < dim; ++c)
            for (int r = 0; r < dim; ++r) g[c + 1][r] = inv[c][r];
        for (int r = 0; r < dim; ++r) {
            double s = 0.0;
            for (int c = 1; c <= dim; ++c) s += g[c][r];
            g[0][r] = -s;
        }
        const double* D = elem_sigma9 ? elem_sigma9 + (size_t)e * 9 : sigma9;
        double sbar = 1.0;
        if (dof_scale) {
            double s = 0.0;
            for (int a = 0; a < nv; ++a) s += dof_scale[vtx[a]];
            sbar = s / nv;
        }
        for (int a = 0; a < nv; ++a) {
            sys.mass[vtx[a]] += vol / nv;
            for (int b = 0; b < nv; ++b) {
                double s = 0.0;
                for (int r = 0; r < dim; ++r)
                    for (int c = 0; c < dim; ++c) s += g[a][r] * D[r * 3 + c] * g[b][c];
                double kab = sbar * vol * s;
                auto& row = rows[vtx[a]];
                bool found = false;
                for (auto& ent : row)
                    if (ent.first == vtx[b]) { ent.second += kab; found = true; break; }
                if (!found) row.push_back({vtx[b], kab});
            }
        }
    }
    sys.K.n = n_nodes;
    sys.K.ptr.assign(n_nodes + 1, 0);
    sys.K.col.clear();
    sys.K.val.clear();
    for (int i = 0; i < n_nodes; ++i) {
        auto& row = rows[i];
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
                      return x.first < y.first;
                  });
        for (auto& ent : row) {
            sys.K.col.push_back(ent.first);
            sys.K.val.push_back(ent.second);
        }
        sys.K.ptr[i + 1] = (int)sys.K.col.size();
    }
    return true;
}

// --------------------------------------------------------------------------
// Aliev-Panfilov ionic model (Sec. 5.1.1)
// --------------------------------------------------------------------------

struct Ionic {
    double ga, gs, a, eps, mu1, mu2, cw;
};

inline double ion_I(const Ionic& p, double v, double w) {
    return p.ga * v * (v - p.a) * (v - 1.0) + v * w;
}
inline double ion_dIdv(const Ionic& p, double v, double w) {
    return p.ga * (3.0 * v * v - 2.0 * (1.0 + p.a) * v + p.a) + w;
}
inline double ion_dIdw(const Ionic&, double v, double) { return v; }
inline double ion_R(const Ionic& p, double v, double w) {
    double E = p.eps + p.mu1 * w / (v + p.mu2);
    double G = -w - p.gs * v * (v - p.a - 1.0);
    return p.cw * E * G;
}
inline double ion_dRdv(const Ionic& p, double v, double w) {
    double E = p.eps + p.mu1 * w / (v + p.mu2);
    double G = -w - p.gs * v * (v - p.a - 1.0);
    double dE = -p.mu1 * w / ((v + p.mu2) * (v + p.mu2));
    double dG = -p.gs * (2.0 * v - p.a - 1.0);
    return p.cw * (dE * G + E * dG);
}
inline double ion_dRdw(const Ionic& p, double v, double w) {
    double E = p.eps + p.mu1 * w / (v + p.mu2);
    double G = -w - p.gs * v * (v - p.a - 1.0);
    double dE = p.mu1 / (v + p.mu2);
    return p.cw * (dE * G - E);
}

// --------------------------------------------------------------------------
// Status codes (same meaning as the library's, defined independently)
// --------------------------------------------------------------------------
enum { ORA_OK = 0, ORA_INVALID = -1, ORA_CG_NOCONV = -4, ORA_NONFINITE = -6, ORA_DOMAIN = -7 };

// --------------------------------------------------------------------------
// Jacobi PCG on A = diag(dA_off) + c K restricted to the active set (Sec. 4.2)
// x, b are full-length; entries outside the active set are zero and stay zero.
// dA holds the full diagonal of A for active rows.
// --------------------------------------------------------------------------
int pcg(const Csr& K, double c, const std::vector<double>& dA, const std::vector<int>& act,
        const std::vector<double>& b, std::vector<double>& x,
        double rtol, int maxit, int& iters, double& relres) {
    const int n = K.n;
    std::vector<double> r(n, 0.0), z(n, 0.0), p(n, 0.0), q(n, 0.0);
    for (int i : act) {
        x[i] = 0.0;
        r[i] = b[i];
        z[i] = r[i] / dA[i];
        p[i] = z[i];
    }
    double rho = 0.0;
    for (int i : act) rho += r[i] * z[i];
    const double rho0 = rho;
    iters = 0;
    relres = 0.0;
    if (rho0 == 0.0) return ORA_OK;
    if (!std::isfinite(rho0)) return ORA_NONFINITE;
    for (int it = 1; it <= maxit; ++it) {
        // q = A p on the active rows; p is zero off the active set.
        for (int i : act) {
            double s = 0.0;
            for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k) {
                int j = K.col[k];
                if (j == i) continue;
                s += K.val[k] * p[j];
            }
            q[i] = dA[i] * p[i] + c * s;
        }
        double pq = 0.0;
        for (int i : act) pq += p[i] * q[i];
        double alpha = rho / pq;
        for (int i : act) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = r[i] / dA[i];
        }
        double rho_new = 0.0;
        for (int i : act) rho_new += r[i] * z[i];
        iters = it;
        relres = std::sqrt(std::fabs(rho_new) / rho0);
        if (!std::isfinite(rho_new)) return ORA_NONFINITE;
        if (std::sqrt(rho_new) <= rtol * std::sqrt(rho0)) return ORA_OK;
        double beta = rho_new / rho;
        rho = rho_new;
        for (int i : act) p[i] = z[i] + beta * p[i];
    }
    return ORA_CG_NOCONV;
}

// Additive two-level preconditioner for the cell-by-cell node systems (the block
// preconditioning Sec. 6 proposes for EMI systems): blocks are the subdomains (each
// cell, the extracellular space), and the blocks selected are those holding active
// dofs.  With Z the n x q matrix of their indicator vectors restricted to the active
// set and E = Z' A Z (q x q, symmetric positive definite),
//     z = D^-1 r + Z E^-1 Z' r.
// The Jacobi part is the one-level preconditioner of pcg(); the coarse part removes
// the near-constant modes of the floating subdomains.
struct TwoLevel {
    int q = 0;                  // selected subdomains (coarse vectors)
    std::vector<int> cls;       // per dof: coarse index, -1 outside the coarse space
    std::vector<double> L;      // Cholesky factor of E, q x q row-major, lower

    // dom[i]: subdomain label of dof i (labels >= 0; -1: in no block).  Returns
    // false when E is not positive definite.
    template <class Op>
    bool build(int n, const int* dom, const std::vector<int>& act, Op apply) {
        std::vector<int> labels;
        for (int i : act)
            if (dom[i] >= 0) labels.push_back(dom[i]);
        std::sort(labels.begin(), labels.end());
        labels.erase(std::unique(labels.begin(), labels.end()), labels.end());
        q = (int)labels.size();
        cls.assign(n, -1);
        for (int i : act)
            if (dom[i] >= 0)
                cls[i] = (int)(std::lower_bound(labels.begin(), labels.end(), dom[i]) -
                               labels.begin());
        // E = Z' A Z, one column per application of A to an indicator vector
        std::vector<double> E((size_t)q * q, 0.0), zb(n, 0.0), y(n, 0.0);
        for (int b = 0; b < q; ++b) {
            for (int i : act) zb[i] = cls[i] == b ? 1.0 : 0.0;
            apply(zb, y);
            for (int i : act)
                if (cls[i] >= 0) E[(size_t)cls[i] * q + b] += y[i];
        }
        // Cholesky E = L L'
        L.assign((size_t)q * q, 0.0);
        for (int a = 0; a < q; ++a) {
            for (int b = 0; b <= a; ++b) {
                double s = E[(size_t)a * q + b];
                for (int k = 0; k < b; ++k) s -= L[(size_t)a * q + k] * L[(size_t)b * q + k];
                if (a == b) {
                    if (!(s > 0.0)) return false;
                    L[(size_t)a * q + a] = std::sqrt(s);
                } else {
                    L[(size_t)a * q + b] = s / L[(size_t)b * q + b];
                }
            }
        }
        return true;
    }

    // z += Z E^-1 Z' r on the active rows
    void add(const std::vector<int>& act, const std::vector<double>& r,
             std::vector<double>& z) const {
        if (q == 0) return;
        std::vector<double> t(q, 0.0), y(q, 0.0);
        for (int i : act)
            if (cls[i] >= 0) t[cls[i]] += r[i];
        for (int a = 0; a < q; ++a) {           // L y' = t
            double s = t[a];
            for (int k = 0; k < a; ++k) s -= L[(size_t)a * q + k] * y[k];
            y[a] = s / L[(size_t)a * q + a];
        }
        for (int a = q - 1; a >= 0; --a) {      // L' y = y'
            double s = y[a];
            for (int k = a + 1; k < q; ++k) s -= L[(size_t)k * q + a] * y[k];
            y[a] = s / L[(size_t)a * q + a];
        }
        for (int i : act)
            if (cls[i] >= 0) z[i] += y[cls[i]];
    }
};

// PCG with the operator given as a function y = A x on the active rows (x is zero
// off the active set), same iteration and stopping rule as pcg(): Jacobi
// preconditioner, and the coarse part of a two-level one when tl is given.
template <class Op>
int pcg_op(int n, Op apply, const std::vector<double>& diag, const std::vector<int>& act,
           const std::vector<double>& b, std::vector<double>& x, double rtol, int maxit,
           int& iters, double& relres, const TwoLevel* tl = nullptr) {
    std::vector<double> r(n, 0.0), z(n, 0.0), p(n, 0.0), q(n, 0.0);
    for (int i : act) {
        x[i] = 0.0;
        r[i] = b[i];
        z[i] = r[i] / diag[i];
    }
    if (tl) tl->add(act, r, z);
    for (int i : act) p[i] = z[i];
    double rho = 0.0;
    for (int i : act) rho += r[i] * z[i];
    const double rho0 = rho;
    iters = 0;
    relres = 0.0;
    if (rho0 == 0.0) return ORA_OK;
    if (!std::isfinite(rho0)) return ORA_NONFINITE;
    for (int it = 1; it <= maxit; ++it) {
        apply(p, q);
        double pq = 0.0;
        for (int i : act) pq += p[i] * q[i];
        double alpha = rho / pq;
        for (int i : act) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = r[i] / diag[i];
        }
        if (tl) tl->add(act, r, z);
        double rho_new = 0.0;
        for (int i : act) rho_new += r[i] * z[i];
        iters = it;
        relres = std::sqrt(std::fabs(rho_new) / rho0);
        if (!std::isfinite(rho_new)) return ORA_NONFINITE;
        if (std::sqrt(rho_new) <= rtol * std::sqrt(rho0)) return ORA_OK;
        double beta = rho_new / rho;
        rho = rho_new;
        for (int i : act) p[i] = z[i] + beta * p[i];
    }
    return ORA_CG_NOCONV;
}

double kdiag(const Csr& K, int i) {
    for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k)
        if (K.col[k] == i) return K.val[k];
    return 0.0;
}

// (K x)_i over the full row (all neighbours, their current values)
double krow(const Csr& K, int i, const double* x) {
    double s = 0.0;
    for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k) s += K.val[k] * x[K.col[k]];
    return s;
}

}  // namespace

// ==========================================================================
// C API (loaded with ctypes by the tests and the benchmark's CPU leg)
// ==========================================================================

extern "C" {

typedef struct { double ga, gs, a, eps, mu1, mu2, cw; } ora_ionic;
// energy_stop: end the sweeps once the energy norm of the sweep's corrections,
// sum over the nodes of dv_m' A~_m dv_m (A~_m the node system matrix), is at most
// ((1 - rho) / rho * TOL)^2 (Sec. 3.2); rho > 0 is the SDC contraction, rho = 0
// estimates it after each sweep as sqrt(E_k / E_{k-1}) (no stop after the first).
// qhat: 0 LU trick, 1 implicit Euler (make_collocation)
// drop_rule: 0 TOL_drop = alpha TOL; 1 the a priori drop tolerance of Sec. 4.1
// (drop_tolerance below) with the given rho > 0 and c from the first sweep
// coarse_min_rows: cell-by-cell steps with blocks: sweeps with fewer active dofs
// solve with Jacobi alone
typedef struct {
    double alpha; double cg_rtol; int cg_maxit; int reaction_implicit; int w_frozen;
    int energy_stop; double rho; int qhat; int drop_rule; int coarse_min_rows;
} ora_opts;
#define ORA_MAX_SWEEPS 64
#define ORA_MAX_M 8
typedef struct {
    int sweeps_run;
    int n_active[ORA_MAX_SWEEPS];
    int cg_iters[ORA_MAX_SWEEPS * ORA_MAX_M];
    double cg_relres_max;
    double min_margin;
    double energy[ORA_MAX_SWEEPS];   // sum over the nodes of dv_m' A~_m dv_m
    double tol_drop;                 // the drop tolerance the selections used
} ora_stats;

// A priori drop tolerance of Sec. 4.1 (Eq. drop-tolerance with Theorems 1 and 2):
//   TOL_drop = exp(-eta T) (1 - rho) / (r + 1) TOL,
// r the least integer >= 0 with r >= log((1 - rho) TOL / c) / log(rho) (Eq. r-condition),
// c = ||dv^0||_inf the first correction (the linear-convergence constant at k = 0, Sec. 4.2),
// eta = max(0, -min dI/dv) / Cm over the linearisation of the correction equation,
// T = dt, the interval the correction equation of one step is posed on.
static double drop_tolerance(double c, double neg_jmin, double Cm, double rho, double tol,
                             double dt) {
    if (!(tol > 0.0)) return 0.0;
    double r = 0.0;
    if (c > 0.0) r = std::max(0.0, std::ceil(std::log((1.0 - rho) * tol / c) / std::log(rho)));
    const double eta = std::max(0.0, neg_jmin) / Cm;
    return std::exp(-eta * dt) * (1.0 - rho) / (r + 1.0) * tol;
}

int ora_collocation(int M, double* tau, double* Q, double* Qhat) {
    Collocation c;
    if (!make_collocation(M, c)) return ORA_INVALID;
    for (int i = 0; i < M; ++i) tau[i] = c.tau[i];
    for (int i = 0; i < M * M; ++i) {
        Q[i] = c.Q[i];
        Qhat[i] = c.Qhat[i];
    }
    return ORA_OK;
}

void ora_ionic_eval(const ora_ionic* ip, double v, double w, double* out6) {
    Ionic p{ip->ga, ip->gs, ip->a, ip->eps, ip->mu1, ip->mu2, ip->cw};
    out6[0] = ion_I(p, v, w);
    out6[1] = ion_dIdv(p, v, w);
    out6[2] = ion_dIdw(p, v, w);
    out6[3] = ion_R(p, v, w);
    out6[4] = ion_dRdv(p, v, w);
    out6[5] = ion_dRdw(p, v, w);
}

void* ora_create_fem(int dim, int n_nodes, const double* xyz, int n_elems, const int* elems,
                     const double* sigma9, const double* elem_sigma9, const double* dof_scale) {
    System* s = new System();
    if (!assemble(dim, n_nodes, xyz, n_elems, elems, sigma9, elem_sigma9, dof_scale, *s)) {
        delete s;
        return nullptr;
    }
    return s;
}

void* ora_create_matrix(int n, const int* ptr, const int* col, const double* val,
                        const double* mass) {
    System* s = new System();
    s->K.n = n;
    s->K.ptr.assign(ptr, ptr + n + 1);
    s->K.col.assign(col, col + ptr[n]);
    s->K.val.assign(val, val + ptr[n]);
    s->mass.assign(mass, mass + n);
    return s;
}

int ora_n(void* h) { return ((System*)h)->K.n; }
int ora_nnz(void* h) { return (int)((System*)h)->K.col.size(); }

void ora_get_matrix(void* h, int* ptr, int* col, double* val, double* mass) {
    System* s = (System*)h;
    std::copy(s->K.ptr.begin(), s->K.ptr.end(), ptr);
    std::copy(s->K.col.begin(), s->K.col.end(), col);
    std::copy(s->K.val.begin(), s->K.val.end(), val);
    std::copy(s->mass.begin(), s->mass.end(), mass);
}

void ora_destroy(void* h) { delete (System*)h; }

// One SDC time step of length dt from (v, w) at the step start; on return
// (v, w) hold the values at the last collocation node (tau_M = 1).
// istim: per-node stimulus current for this step (NULL = none).
// active_log (optional): concatenated ascending active lists of every sweep.
// Vn, Wn (optional): all collocation-node values after the last sweep, [M][N].
// forced_counts / forced_lists (optional, for derivative checks): the active
// sets to use instead of selecting them, |I_k| = forced_counts[k], the lists of
// sweeps 1..sweeps-1 concatenated in forced_lists (I_0 is every dof).
int ora_step_forced(void* h, const ora_ionic* ip, int M, const double* istim, double* v, double* w,
                    double dt, int sweeps, double tol, const ora_opts* o, ora_stats* st,
                    int* active_log, double* Vn, double* Wn, const int* forced_counts,
                    const int* forced_lists);

int ora_step(void* h, const ora_ionic* ip, int M, const double* istim, double* v, double* w,
             double dt, int sweeps, double tol, const ora_opts* o, ora_stats* st,
             int* active_log, double* Vn, double* Wn) {
    return ora_step_forced(h, ip, M, istim, v, w, dt, sweeps, tol, o, st, active_log, Vn, Wn,
                           nullptr, nullptr);
}

int ora_step_forced(void* h, const ora_ionic* ip, int M, const double* istim, double* v, double* w,
                    double dt, int sweeps, double tol, const ora_opts* o, ora_stats* st,
                    int* active_log, double* Vn, double* Wn, const int* forced_counts,
                    const int* forced_lists) {
    System& S = *(System*)h;
    const Csr& K = S.K;
    const int N = K.n;
    Collocation col;
    if (!make_collocation(M, col, o->qhat) || sweeps < 0 || sweeps > ORA_MAX_SWEEPS || tol < 0 ||
        dt <= 0)
        return ORA_INVALID;
    const std::vector<double>& Q = col.Q;
    const std::vector<double>& Qh = col.Qhat;
    Ionic p{ip->ga, ip->gs, ip->a, ip->eps, ip->mu1, ip->mu2, ip->cw};
    double tol_drop = o->alpha * tol;
    if (o->drop_rule && !(o->rho > 0.0 && o->rho < 1.0)) return ORA_INVALID;

    std::vector<double> v0(v, v + N), w0(w, w + N);
    // collocation iterates V[m][i], W[m][i], spread predictor
    std::vector<double> V((size_t)M * N), W((size_t)M * N);
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < N; ++i) {
            V[(size_t)m * N + i] = v0[i];
            W[(size_t)m * N + i] = w0[i];
        }
    std::vector<int> act(N);
    for (int i = 0; i < N; ++i) act[i] = i;
    std::vector<double> f((size_t)M * N), J((size_t)M * N), r((size_t)M * N),
        delta((size_t)M * N), b(N), dA(N), Kd(N);
    for (int i = 0; i < N; ++i) Kd[i] = kdiag(K, i);
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->min_margin = INFINITY;
    }
    size_t log_pos = 0;
    int status = ORA_OK;

    double energy_prev = 0.0;
    for (int k = 0; k < sweeps; ++k) {
        if (st) {
            st->n_active[k] = (int)act.size();
            st->sweeps_run = k + 1;
        }
        if (active_log) {
            std::copy(act.begin(), act.end(), active_log + log_pos);
            log_pos += act.size();
        }
        if (act.empty()) continue;
        double energy = 0.0;
        // residual of the collocation system at the current iterate (active rows only)
        for (int m = 0; m < M; ++m)
            for (int i : act) {
                double vm = V[(size_t)m * N + i], wm = W[(size_t)m * N + i];
                double s = istim ? istim[i] : 0.0;
                f[(size_t)m * N + i] = -krow(K, i, &V[(size_t)m * N]) - S.mass[i] * (ion_I(p, vm, wm) - s);
                J[(size_t)m * N + i] = o->reaction_implicit ? ion_dIdv(p, vm, wm) : 0.0;
            }
        for (int m = 0; m < M; ++m)
            for (int i : act) {
                double q = 0.0;
                for (int j = 0; j < M; ++j) q += Q[m * M + j] * f[(size_t)j * N + i];
                r[(size_t)m * N + i] = S.mass[i] * v0[i] + dt * q - S.mass[i] * V[(size_t)m * N + i];
            }
        std::fill(delta.begin(), delta.end(), 0.0);
        // sequential node solves (lower-triangular Qhat)
        for (int m = 0; m < M; ++m) {
            for (int i : act) {
                double corr = 0.0;
                for (int j = 0; j < m; ++j) {
                    const double* dj = &delta[(size_t)j * N];
                    corr += Qh[m * M + j] * (krow(K, i, dj) + S.mass[i] * J[(size_t)j * N + i] * dj[i]);
                }
                b[i] = r[(size_t)m * N + i] - dt * corr;
            }
            const double c = dt * Qh[m * M + m];
            for (int i : act) {
                dA[i] = S.mass[i] * (1.0 + c * J[(size_t)m * N + i]) + c * Kd[i];
                if (!std::isfinite(dA[i])) return ORA_NONFINITE;
                if (!(dA[i] > 0.0)) return ORA_DOMAIN;
            }
            std::vector<double> x(N, 0.0);
            int iters = 0;
            double relres = 0.0;
            int rc = pcg(K, c, dA, act, b, x, o->cg_rtol, o->cg_maxit, iters, relres);
            if (st) {
                st->cg_iters[k * ORA_MAX_M + m] = iters;
                st->cg_relres_max = std::max(st->cg_relres_max, relres);
            }
            if (rc != ORA_OK) return rc;
            for (int i : act) delta[(size_t)m * N + i] = x[i];
            // energy norm of this node's correction in its own system matrix
            for (int i : act) {
                double s = 0.0;
                for (int q = K.ptr[i]; q < K.ptr[i + 1]; ++q)
                    if (K.col[q] != i) s += K.val[q] * x[K.col[q]];
                energy += x[i] * (dA[i] * x[i] + c * s);
            }
        }
        if (st) st->energy[k] = energy;
        if (o->drop_rule && k == 0) {
            // c and eta from the first sweep (all dofs active)
            double cmax = 0.0, neg_jmin = 0.0;
            for (int m = 0; m < M; ++m)
                for (int i : act) {
                    cmax = std::max(cmax, std::fabs(delta[(size_t)m * N + i]));
                    neg_jmin = std::max(neg_jmin, -J[(size_t)m * N + i]);
                }
            tol_drop = drop_tolerance(cmax, neg_jmin, 1.0, o->rho, tol, dt);
        }
        // v update on the active rows; inactive rows are held fixed
        for (int m = 0; m < M; ++m)
            for (int i : act) V[(size_t)m * N + i] += delta[(size_t)m * N + i];
        // pointwise w sweep with the updated v and the old w
        if (!o->w_frozen) {
            for (int i : act) {
                double g[ORA_MAX_M], d[ORA_MAX_M], s[ORA_MAX_M], eps[ORA_MAX_M];
                for (int m = 0; m < M; ++m) {
                    double vm = V[(size_t)m * N + i], wm = W[(size_t)m * N + i];
                    if (vm + p.mu2 <= 0.0) return ORA_DOMAIN;
                    g[m] = ion_R(p, vm, wm);
                    d[m] = ion_dRdw(p, vm, wm);
                }
                for (int m = 0; m < M; ++m) {
                    double q = 0.0;
                    for (int j = 0; j < M; ++j) q += Q[m * M + j] * g[j];
                    s[m] = w0[i] + dt * q - W[(size_t)m * N + i];
                }
                for (int m = 0; m < M; ++m) {
                    double acc = s[m];
                    for (int j = 0; j < m; ++j) acc += dt * Qh[m * M + j] * d[j] * eps[j];
                    double den = 1.0 - dt * Qh[m * M + m] * d[m];
                    if (!(den > 0.0)) return ORA_DOMAIN;
                    eps[m] = acc / den;
                }
                for (int m = 0; m < M; ++m) W[(size_t)m * N + i] += eps[m];
            }
        }
        // nested selection: keep i in I_k with max_m |dv_{m,i}| >= TOL_drop
        std::vector<int> next;
        for (int i : act) {
            double amax = 0.0;
            for (int m = 0; m < M; ++m) amax = std::max(amax, std::fabs(delta[(size_t)m * N + i]));
            if (!std::isfinite(amax)) return ORA_NONFINITE;
            if (st && tol_drop > 0.0) st->min_margin = std::min(st->min_margin, std::fabs(amax - tol_drop));
            if (amax >= tol_drop) next.push_back(i);
        }
        if (o->energy_stop) {
            // Sec. 3.2: geometric-series estimate of the remaining energy-norm error
            double rho = o->rho;
            if (!(rho > 0.0)) rho = k > 0 && energy_prev > 0.0 ? std::sqrt(energy / energy_prev) : 0.0;
            energy_prev = energy;
            if (rho > 0.0 && rho < 1.0) {
                const double lim = (1.0 - rho) / rho * tol;
                if (energy <= lim * lim) break;
            }
        }
        if (forced_counts) {
            // replace the selection by the given set of the next sweep
            next.clear();
            if (k + 1 < sweeps) {
                size_t off = 0;
                for (int kk = 1; kk <= k; ++kk) off += (size_t)forced_counts[kk];
                next.assign(forced_lists + off, forced_lists + off + forced_counts[k + 1]);
            }
        }
        act.swap(next);
    }
    for (int i = 0; i < N; ++i) {
        v[i] = V[(size_t)(M - 1) * N + i];
        w[i] = W[(size_t)(M - 1) * N + i];
    }
    if (Vn) std::copy(V.begin(), V.end(), Vn);
    if (Wn) std::copy(W.begin(), W.end(), Wn);
    if (st) st->tol_drop = tol_drop;
    return status;
}

// One SDC step of the cell-by-cell (EMI) system (Sec. 2.1, eq. abstract reaction
// diffusion / abstract gating) in the abstract form B u' = -A u - b(u, w) of
// Sec. 3:
//   A = K + diag(robin)                 (stiffness of every subdomain, Robin term)
//   B = sum_p area_p Cm (e_k - e_l)(e_k - e_l)^T              (membrane capacitance)
//   b = sum_p area_p I_p(u_k - u_l, w_p) (e_k - e_l),  I_p = I_ion (kind 0) or g_gap v (kind 1)
//   w_p' = R(u_k - u_l, w_p) on the cell-ECS pairs (kind 0).
// The sweep is that of ora_step with B in place of the lumped mass and the
// pair Jacobian sum_p area_p dI_p/dv (e_k - e_l)(e_k - e_l)^T in place of the
// lumped ionic Jacobian; the gating sweep runs over the pairs with an active
// endpoint; selection uses |du| of every potential dof.
// PCG on an explicit CSR matrix A (rows ptr/col/val, n x n, symmetric positive
// definite on the active rows act[0..n_act)): Jacobi, plus the two-level coarse part
// over the subdomain labels dom when dom is given.  x: n entries (zero off the
// active set on return).
int ora_pcg_csr(int n, const int* ptr, const int* col, const double* val, int n_act,
                const int* act_list, const int* dom, const double* b_in, double* x_out,
                double rtol, int maxit, int* iters_out) {
    std::vector<int> act(act_list, act_list + n_act);
    std::vector<char> on(n, 0);
    for (int i : act) on[i] = 1;
    std::vector<double> diag(n, 0.0), b(n, 0.0), x(n, 0.0);
    for (int i : act) {
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (col[k] == i) diag[i] += val[k];
        b[i] = b_in[i];
        if (!(diag[i] > 0.0)) return ORA_DOMAIN;
    }
    auto apply = [&](const std::vector<double>& v, std::vector<double>& y) {
        for (int i : act) {
            double s = 0.0;
            for (int k = ptr[i]; k < ptr[i + 1]; ++k)
                if (on[col[k]]) s += val[k] * v[col[k]];
            y[i] = s;
        }
    };
    TwoLevel tl;
    if (dom && !tl.build(n, dom, act, apply)) return ORA_DOMAIN;
    int iters = 0;
    double relres = 0.0;
    const int rc = pcg_op(n, apply, diag, act, b, x, rtol, maxit, iters, relres,
                          dom ? &tl : nullptr);
    for (int i = 0; i < n; ++i) x_out[i] = x[i];
    if (iters_out) *iters_out = iters;
    return rc;
}

// z = D^-1 r + Z E^-1 Z' r of the two-level preconditioner on an explicit CSR matrix
// restricted to act[0..n_act) (z: n entries).
int ora_two_level_apply(int n, const int* ptr, const int* col, const double* val, int n_act,
                        const int* act_list, const int* dom, const double* r_in, double* z_out) {
    std::vector<int> act(act_list, act_list + n_act);
    std::vector<char> on(n, 0);
    for (int i : act) on[i] = 1;
    auto apply = [&](const std::vector<double>& v, std::vector<double>& y) {
        for (int i : act) {
            double s = 0.0;
            for (int k = ptr[i]; k < ptr[i + 1]; ++k)
                if (on[col[k]]) s += val[k] * v[col[k]];
            y[i] = s;
        }
    };
    TwoLevel tl;
    if (!tl.build(n, dom, act, apply)) return ORA_DOMAIN;
    std::vector<double> r(r_in, r_in + n), z(n, 0.0);
    for (int i : act) {
        double d = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (col[k] == i) d += val[k];
        z[i] = r[i] / d;
    }
    tl.add(act, r, z);
    for (int i = 0; i < n; ++i) z_out[i] = z[i];
    return ORA_OK;
}

int ora_step_emi(void* h, const ora_ionic* ip, double Cm, double g_gap, int M, int n_pairs,
                 const int* pk, const int* pl, const double* parea, const int* pkind,
                 const double* robin, double* u, double* w, double dt, int sweeps, double tol,
                 const ora_opts* o, ora_stats* st, int* active_log, const int* dom) {
    System& S = *(System*)h;
    const Csr& K = S.K;
    const int N = K.n, NP = n_pairs;
    Collocation col;
    if (!make_collocation(M, col, o->qhat) || sweeps < 0 || sweeps > ORA_MAX_SWEEPS || tol < 0 ||
        dt <= 0)
        return ORA_INVALID;
    const std::vector<double>& Q = col.Q;
    const std::vector<double>& Qh = col.Qhat;
    Ionic p{ip->ga, ip->gs, ip->a, ip->eps, ip->mu1, ip->mu2, ip->cw};
    double tol_drop = o->alpha * tol;
    if (o->drop_rule && !(o->rho > 0.0 && o->rho < 1.0)) return ORA_INVALID;
    // pairs incident to each node, with the sign of the node in v = u_k - u_l
    std::vector<std::vector<std::pair<int, int>>> inc(N);
    for (int q = 0; q < NP; ++q) {
        inc[pk[q]].push_back({q, +1});
        inc[pl[q]].push_back({q, -1});
    }
    auto partner = [&](int q, int i) { return pk[q] == i ? pl[q] : pk[q]; };
    std::vector<double> u0(u, u + N), w0(w, w + NP);
    std::vector<double> U((size_t)M * N), Wp((size_t)M * NP);
    for (int m = 0; m < M; ++m) {
        for (int i = 0; i < N; ++i) U[(size_t)m * N + i] = u0[i];
        for (int q = 0; q < NP; ++q) Wp[(size_t)m * NP + q] = w0[q];
    }
    std::vector<int> act(N);
    for (int i = 0; i < N; ++i) act[i] = i;
    std::vector<char> on(N, 1);
    std::vector<double> Ip((size_t)M * NP), Jp((size_t)M * NP), f((size_t)M * N), r((size_t)M * N),
        delta((size_t)M * N), b(N), diag(N), Kd(N);
    for (int i = 0; i < N; ++i) Kd[i] = kdiag(K, i) + (robin ? robin[i] : 0.0);
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->min_margin = INFINITY;
    }
    size_t log_pos = 0;
    // (A x)_i over the full row: K plus the Robin diagonal
    auto arow = [&](int i, const double* x) {
        return krow(K, i, x) + (robin ? robin[i] : 0.0) * x[i];
    };
    double energy_prev = 0.0;
    for (int k = 0; k < sweeps; ++k) {
        if (st) {
            st->n_active[k] = (int)act.size();
            st->sweeps_run = k + 1;
        }
        if (active_log) {
            std::copy(act.begin(), act.end(), active_log + log_pos);
            log_pos += act.size();
        }
        if (act.empty()) continue;
        double energy = 0.0;
        for (int m = 0; m < M; ++m)
            for (int q = 0; q < NP; ++q) {
                const double v = U[(size_t)m * N + pk[q]] - U[(size_t)m * N + pl[q]];
                const double wq = Wp[(size_t)m * NP + q];
                if (pkind[q] == 0) {
                    Ip[(size_t)m * NP + q] = ion_I(p, v, wq);
                    Jp[(size_t)m * NP + q] = o->reaction_implicit ? ion_dIdv(p, v, wq) : 0.0;
                } else {
                    Ip[(size_t)m * NP + q] = g_gap * v;
                    Jp[(size_t)m * NP + q] = o->reaction_implicit ? g_gap : 0.0;
                }
            }
        for (int m = 0; m < M; ++m)
            for (int i : act) {
                double s = -arow(i, &U[(size_t)m * N]);
                for (auto& e : inc[i]) s -= e.second * parea[e.first] * Ip[(size_t)m * NP + e.first];
                f[(size_t)m * N + i] = s;
            }
        for (int m = 0; m < M; ++m)
            for (int i : act) {
                double bt = 0.0;
                for (auto& e : inc[i]) {
                    const int j = partner(e.first, i);
                    bt += parea[e.first] * Cm *
                          ((u0[i] - u0[j]) - (U[(size_t)m * N + i] - U[(size_t)m * N + j]));
                }
                double qs = 0.0;
                for (int j = 0; j < M; ++j) qs += Q[m * M + j] * f[(size_t)j * N + i];
                r[(size_t)m * N + i] = bt + dt * qs;
            }
        std::fill(delta.begin(), delta.end(), 0.0);
        for (int m = 0; m < M; ++m) {
            for (int i : act) {
                double corr = 0.0;
                for (int j = 0; j < m; ++j) {
                    const double* dj = &delta[(size_t)j * N];
                    double pj = 0.0;
                    for (auto& e : inc[i])
                        pj += parea[e.first] * Jp[(size_t)j * NP + e.first] *
                              (dj[i] - dj[partner(e.first, i)]);
                    corr += Qh[m * M + j] * (arow(i, dj) + pj);
                }
                b[i] = r[(size_t)m * N + i] - dt * corr;
            }
            const double c = dt * Qh[m * M + m];
            for (int i : act) {
                double d = c * Kd[i];
                for (auto& e : inc[i]) d += parea[e.first] * (Cm + c * Jp[(size_t)m * NP + e.first]);
                diag[i] = d;
                if (!std::isfinite(d)) return ORA_NONFINITE;
                if (!(d > 0.0)) return ORA_DOMAIN;
            }
            auto apply = [&](const std::vector<double>& x, std::vector<double>& y) {
                for (int i : act) {
                    double s = c * arow(i, x.data());
                    for (auto& e : inc[i])
                        s += parea[e.first] * (Cm + c * Jp[(size_t)m * NP + e.first]) *
                             (x[i] - x[partner(e.first, i)]);
                    y[i] = s;
                }
            };
            std::vector<double> x(N, 0.0);
            int iters = 0;
            double relres = 0.0;
            // dom given (and enough active dofs): the two-level preconditioner over the
            // subdomains of the active set
            const bool two = dom && (long long)act.size() >= o->coarse_min_rows;
            TwoLevel tl;
            if (two && !tl.build(N, dom, act, apply)) return ORA_DOMAIN;
            const int rc = pcg_op(N, apply, diag, act, b, x, o->cg_rtol, o->cg_maxit, iters, relres,
                                  two ? &tl : nullptr);
            if (st) {
                st->cg_iters[k * ORA_MAX_M + m] = iters;
                st->cg_relres_max = std::max(st->cg_relres_max, relres);
            }
            if (rc != ORA_OK) return rc;
            for (int i : act) delta[(size_t)m * N + i] = x[i];
            // energy norm of this node's correction in its own system matrix
            std::vector<double> ax(N, 0.0);
            apply(x, ax);
            for (int i : act) energy += x[i] * ax[i];
        }
        if (st) st->energy[k] = energy;
        if (o->drop_rule && k == 0) {
            // c from the first sweep; eta from the pair Jacobians (membrane currents
            // and gap junctions) over C_m
            double cmax = 0.0, neg_jmin = 0.0;
            for (int m = 0; m < M; ++m) {
                for (int i : act) cmax = std::max(cmax, std::fabs(delta[(size_t)m * N + i]));
                for (int q = 0; q < NP; ++q) neg_jmin = std::max(neg_jmin, -Jp[(size_t)m * NP + q]);
            }
            tol_drop = drop_tolerance(cmax, neg_jmin, Cm, o->rho, tol, dt);
        }
        for (int m = 0; m < M; ++m)
            for (int i : act) U[(size_t)m * N + i] += delta[(size_t)m * N + i];
        if (!o->w_frozen) {
            for (int q = 0; q < NP; ++q) {
                if (pkind[q] != 0 || !(on[pk[q]] || on[pl[q]])) continue;
                double g[ORA_MAX_M], d[ORA_MAX_M], s[ORA_MAX_M], eps[ORA_MAX_M];
                for (int m = 0; m < M; ++m) {
                    const double v = U[(size_t)m * N + pk[q]] - U[(size_t)m * N + pl[q]];
                    const double wq = Wp[(size_t)m * NP + q];
                    if (v + p.mu2 <= 0.0) return ORA_DOMAIN;
                    g[m] = ion_R(p, v, wq);
                    d[m] = ion_dRdw(p, v, wq);
                }
                for (int m = 0; m < M; ++m) {
                    double qs = 0.0;
                    for (int j = 0; j < M; ++j) qs += Q[m * M + j] * g[j];
                    s[m] = w0[q] + dt * qs - Wp[(size_t)m * NP + q];
                }
                for (int m = 0; m < M; ++m) {
                    double acc = s[m];
                    for (int j = 0; j < m; ++j) acc += dt * Qh[m * M + j] * d[j] * eps[j];
                    const double den = 1.0 - dt * Qh[m * M + m] * d[m];
                    if (!(den > 0.0)) return ORA_DOMAIN;
                    eps[m] = acc / den;
                }
                for (int m = 0; m < M; ++m) Wp[(size_t)m * NP + q] += eps[m];
            }
        }
        std::vector<int> next;
        for (int i : act) {
            double amax = 0.0;
            for (int m = 0; m < M; ++m) amax = std::max(amax, std::fabs(delta[(size_t)m * N + i]));
            if (!std::isfinite(amax)) return ORA_NONFINITE;
            if (st && tol_drop > 0.0) st->min_margin = std::min(st->min_margin, std::fabs(amax - tol_drop));
            if (amax >= tol_drop) next.push_back(i);
        }
        if (o->energy_stop) {
            // Sec. 3.2: geometric-series estimate of the remaining energy-norm error
            double rho = o->rho;
            if (!(rho > 0.0)) rho = k > 0 && energy_prev > 0.0 ? std::sqrt(energy / energy_prev) : 0.0;
            energy_prev = energy;
            if (rho > 0.0 && rho < 1.0) {
                const double lim = (1.0 - rho) / rho * tol;
                if (energy <= lim * lim) break;
            }
        }
        for (int i : act) on[i] = 0;
        for (int i : next) on[i] = 1;
        act.swap(next);
    }
    for (int i = 0; i < N; ++i) u[i] = U[(size_t)(M - 1) * N + i];
    for (int q = 0; q < NP; ++q) w[q] = Wp[(size_t)(M - 1) * NP + q];
    if (st) st->tol_drop = tol_drop;
    return ORA_OK;
}

// Dense Newton solve of the full collocation system (Sec. 3.1):
//   m (v_m - v_0) = dt sum_j Q_mj f(v_j, w_j),   w_m - w_0 = dt sum_j Q_mj R(v_j, w_j)
// for tiny systems only (2 N M unknowns, dense LU with partial pivoting).
int ora_collocation_solve(void* h, const ora_ionic* ip, int M, const double* istim, double* v,
                          double* w, double dt, double* Vn, double* Wn, int* newton_iters) {
    System& S = *(System*)h;
    const Csr& K = S.K;
    const int N = K.n;
    const int U = 2 * N * M;
    if (U > 4000) return ORA_INVALID;
    Collocation col;
    if (!make_collocation(M, col)) return ORA_INVALID;
    const std::vector<double>& Q = col.Q;
    Ionic p{ip->ga, ip->gs, ip->a, ip->eps, ip->mu1, ip->mu2, ip->cw};
    std::vector<double> v0(v, v + N), w0(w, w + N);
    std::vector<double> Z(U);
    auto iv = [&](int m, int i) { return m * N + i; };
    auto iw = [&](int m, int i) { return N * M + m * N + i; };
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < N; ++i) {
            Z[iv(m, i)] = v0[i];
            Z[iw(m, i)] = w0[i];
        }
    std::vector<double> G(U), A((size_t)U * U), dz(U);
    std::vector<int> piv(U);
    int it;
    for (it = 0; it < 50; ++it) {
        // residual
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < N; ++i) {
                double qv = 0.0, qw = 0.0;
                for (int j = 0; j < M; ++j) {
                    double vj = Z[iv(j, i)], wj = Z[iw(j, i)];
                    double Kv = 0.0;
                    for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k) Kv += K.val[k] * Z[iv(j, K.col[k])];
                    double fj = -Kv - S.mass[i] * (ion_I(p, vj, wj) - (istim ? istim[i] : 0.0));
                    qv += Q[m * M + j] * fj;
                    qw += Q[m * M + j] * ion_R(p, vj, wj);
                }
                G[iv(m, i)] = S.mass[i] * (Z[iv(m, i)] - v0[i]) - dt * qv;
                G[iw(m, i)] = (Z[iw(m, i)] - w0[i]) - dt * qw;
            }
        // Jacobian
        std::fill(A.begin(), A.end(), 0.0);
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < N; ++i) {
                size_t rv = (size_t)iv(m, i) * U, rw = (size_t)iw(m, i) * U;
                A[rv + iv(m, i)] += S.mass[i];
                A[rw + iw(m, i)] += 1.0;
                for (int j = 0; j < M; ++j) {
                    double vj = Z[iv(j, i)], wj = Z[iw(j, i)];
                    double q = dt * Q[m * M + j];
                    for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k) A[rv + iv(j, K.col[k])] += q * K.val[k];
                    A[rv + iv(j, i)] += q * S.mass[i] * ion_dIdv(p, vj, wj);
                    A[rv + iw(j, i)] += q * S.mass[i] * ion_dIdw(p, vj, wj);
                    A[rw + iv(j, i)] -= q * ion_dRdv(p, vj, wj);
                    A[rw + iw(j, i)] -= q * ion_dRdw(p, vj, wj);
                }
            }
        // LU with partial pivoting, solve A dz = -G
        for (int c = 0; c < U; ++c) {
            int best = c;
            for (int r2 = c + 1; r2 < U; ++r2)
                if (std::fabs(A[(size_t)r2 * U + c]) > std::fabs(A[(size_t)best * U + c])) best = r2;
            piv[c] = best;
            if (best != c) {
                for (int k = 0; k < U; ++k) std::swap(A[(size_t)c * U + k], A[(size_t)best * U + k]);
            }
            double d = A[(size_t)c * U + c];
            if (d == 0.0) return ORA_INVALID;
            for (int r2 = c + 1; r2 < U; ++r2) {
                double l = A[(size_t)r2 * U + c] / d;
                A[(size_t)r2 * U + c] = l;
                if (l != 0.0)
                    for (int k = c + 1; k < U; ++k) A[(size_t)r2 * U + k] -= l * A[(size_t)c * U + k];
            }
        }
        for (int i = 0; i < U; ++i) dz[i] = -G[i];
        for (int c = 0; c < U; ++c) {
            if (piv[c] != c) std::swap(dz[c], dz[piv[c]]);
            for (int r2 = c + 1; r2 < U; ++r2) dz[r2] -= A[(size_t)r2 * U + c] * dz[c];
        }
        for (int c = U - 1; c >= 0; --c) {
            double s = dz[c];
            for (int k = c + 1; k < U; ++k) s -= A[(size_t)c * U + k] * dz[k];
            dz[c] = s / A[(size_t)c * U + c];
        }
        double nrm = 0.0, zn = 1.0;
        for (int i = 0; i < U; ++i) {
            Z[i] += dz[i];
            nrm = std::max(nrm, std::fabs(dz[i]));
            zn = std::max(zn, std::fabs(Z[i]));
        }
        if (nrm <= 1e-15 * zn) { ++it; break; }
    }
    if (newton_iters) *newton_iters = it;
    for (int i = 0; i < N; ++i) {
        v[i] = Z[iv(M - 1, i)];
        w[i] = Z[iw(M - 1, i)];
    }
    if (Vn)
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < N; ++i) Vn[(size_t)m * N + i] = Z[iv(m, i)];
    if (Wn)
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < N; ++i) Wn[(size_t)m * N + i] = Z[iw(m, i)];
    return ORA_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------
// Tangent (forward mode) of one step with the active sets given (derivative
// checks of the library's discrete adjoint).  Every quantity carries a value and
// a directional derivative (dual numbers); the step is the one of
// ora_step_forced in the same order of operations, so the value parts equal
// that function's results bitwise.  The direction may move the initial state
// (dv, dw), the Aliev-Panfilov parameters (dip) and the per-node conductivity
// scale: K is linear in the scale (K = sum_e sbar_e K_e), so the derivative of K
// along a scale direction d is the matrix assembled with scale d on the same
// pattern (handle hd; NULL for none).  Each CG solve differentiates its own
// iterations, stopped by the values' test: with a tight rtol its derivative is
// that of the exact solve to the same order.
// --------------------------------------------------------------------------
namespace {

struct Dual {
    double v, d;
    Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }

struct IonicD {
    Dual ga, gs, a, eps, mu1, mu2, cw;
};
// the model of Sec. 5.1.1, written as in ion_I / ion_dIdv / ion_R / ion_dRdw
inline Dual dion_I(const IonicD& p, Dual v, Dual w) {
    return p.ga * v * (v - p.a) * (v - 1.0) + v * w;
}
inline Dual dion_dIdv(const IonicD& p, Dual v, Dual w) {
    return p.ga * (3.0 * v * v - 2.0 * (1.0 + p.a) * v + p.a) + w;
}
inline Dual dion_R(const IonicD& p, Dual v, Dual w) {
    Dual E = p.eps + p.mu1 * w / (v + p.mu2);
    Dual G = -w - p.gs * v * (v - p.a - 1.0);
    return p.cw * E * G;
}
inline Dual dion_dRdw(const IonicD& p, Dual v, Dual w) {
    Dual E = p.eps + p.mu1 * w / (v + p.mu2);
    Dual G = -w - p.gs * v * (v - p.a - 1.0);
    Dual dE = p.mu1 / (v + p.mu2);
    return p.cw * (dE * G - E);
}

// K with its derivative along the scale direction, entry by entry (same pattern)
struct CsrD {
    const Csr* K;
    const Csr* Kd;   // may be null
    Dual val(int k) const { return Dual(K->val[k], Kd ? Kd->val[k] : 0.0); }
};
Dual dkrow(const CsrD& K, int i, const Dual* x) {
    Dual s = 0.0;
    for (int k = K.K->ptr[i]; k < K.K->ptr[i + 1]; ++k) s += K.val(k) * x[K.K->col[k]];
    return s;
}
Dual dkdiag(const CsrD& K, int i) {
    for (int k = K.K->ptr[i]; k < K.K->ptr[i + 1]; ++k)
        if (K.K->col[k] == i) return K.val(k);
    return Dual(0.0);
}

// pcg() in dual numbers: the same iteration, stopped by the values' test
int dpcg(const CsrD& K, double c, const std::vector<Dual>& dA, const std::vector<int>& act,
         const std::vector<Dual>& b, std::vector<Dual>& x, double rtol, int maxit, int& iters) {
    const int n = K.K->n;
    std::vector<Dual> r(n), z(n), p(n), q(n);
    for (int i : act) {
        x[i] = 0.0;
        r[i] = b[i];
        z[i] = r[i] / dA[i];
        p[i] = z[i];
    }
    Dual rho = 0.0;
    for (int i : act) rho += r[i] * z[i];
    const Dual rho0 = rho;
    iters = 0;
    if (rho0.v == 0.0) return ORA_OK;
    if (!std::isfinite(rho0.v)) return ORA_NONFINITE;
    for (int it = 1; it <= maxit; ++it) {
        for (int i : act) {
            Dual s = 0.0;
            for (int k = K.K->ptr[i]; k < K.K->ptr[i + 1]; ++k) {
                int j = K.K->col[k];
                if (j == i) continue;
                s += K.val(k) * p[j];
            }
            q[i] = dA[i] * p[i] + c * s;
        }
        Dual pq = 0.0;
        for (int i : act) pq += p[i] * q[i];
        Dual alpha = rho / pq;
        for (int i : act) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = r[i] / dA[i];
        }
        Dual rho_new = 0.0;
        for (int i : act) rho_new += r[i] * z[i];
        iters = it;
        if (!std::isfinite(rho_new.v)) return ORA_NONFINITE;
        if (std::sqrt(rho_new.v) <= rtol * std::sqrt(rho0.v)) return ORA_OK;
        Dual beta = rho_new / rho;
        rho = rho_new;
        for (int i : act) p[i] = z[i] + beta * p[i];
    }
    return ORA_CG_NOCONV;
}

}  // namespace

extern "C" {

// Tangent of ora_step_forced (forced sets required, no energy stop or drop rule):
// on return v, w hold the step's result and dv, dw its derivative along the
// direction (dv, dw on entry: the initial state's direction; dip: the ionic
// parameters' direction, NULL = none; hd: matrix of the scale direction, NULL =
// none).  iters (optional, sweeps * ORA_MAX_M): CG iterations of each solve.
int ora_step_tangent(void* h, void* hd, const ora_ionic* ip, const ora_ionic* dip, int M,
                     const double* istim, double* v, double* dv, double* w, double* dw, double dt,
                     int sweeps, const ora_opts* o, const int* forced_counts,
                     const int* forced_lists, int* iters_out) {
    System& S = *(System*)h;
    const Csr& K0 = S.K;
    const int N = K0.n;
    Collocation col;
    if (!make_collocation(M, col, o->qhat) || sweeps < 0 || sweeps > ORA_MAX_SWEEPS || dt <= 0 ||
        !forced_counts)
        return ORA_INVALID;
    const Csr* Kd = nullptr;
    if (hd) {
        Kd = &((System*)hd)->K;
        if (Kd->n != N || Kd->ptr != K0.ptr || Kd->col != K0.col) return ORA_INVALID;
    }
    const CsrD K{&K0, Kd};
    const std::vector<double>& Q = col.Q;
    const std::vector<double>& Qh = col.Qhat;
    auto dual = [&](double x, double dx) { return Dual(x, dip ? dx : 0.0); };
    const ora_ionic z{0, 0, 0, 0, 0, 0, 0};
    const ora_ionic& di = dip ? *dip : z;
    IonicD p{dual(ip->ga, di.ga), dual(ip->gs, di.gs), dual(ip->a, di.a), dual(ip->eps, di.eps),
             dual(ip->mu1, di.mu1), dual(ip->mu2, di.mu2), dual(ip->cw, di.cw)};
    std::vector<Dual> v0(N), w0(N);
    for (int i = 0; i < N; ++i) {
        v0[i] = Dual(v[i], dv[i]);
        w0[i] = Dual(w[i], dw[i]);
    }
    std::vector<Dual> V((size_t)M * N), W((size_t)M * N);
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < N; ++i) {
            V[(size_t)m * N + i] = v0[i];
            W[(size_t)m * N + i] = w0[i];
        }
    std::vector<int> act(N);
    for (int i = 0; i < N; ++i) act[i] = i;
    std::vector<Dual> f((size_t)M * N), J((size_t)M * N), r((size_t)M * N), delta((size_t)M * N),
        b(N), dA(N), Kdg(N);
    for (int i = 0; i < N; ++i) Kdg[i] = dkdiag(K, i);
    for (int k = 0; k < sweeps; ++k) {
        if (act.empty()) continue;   // as in ora_step_forced: an emptied set stays empty
        {
            for (int m = 0; m < M; ++m)
                for (int i : act) {
                    Dual vm = V[(size_t)m * N + i], wm = W[(size_t)m * N + i];
                    double s = istim ? istim[i] : 0.0;
                    f[(size_t)m * N + i] =
                        -dkrow(K, i, &V[(size_t)m * N]) - S.mass[i] * (dion_I(p, vm, wm) - s);
                    J[(size_t)m * N + i] = o->reaction_implicit ? dion_dIdv(p, vm, wm) : Dual(0.0);
                }
            for (int m = 0; m < M; ++m)
                for (int i : act) {
                    Dual q = 0.0;
                    for (int j = 0; j < M; ++j) q += Q[m * M + j] * f[(size_t)j * N + i];
                    r[(size_t)m * N + i] =
                        S.mass[i] * v0[i] + dt * q - S.mass[i] * V[(size_t)m * N + i];
                }
            std::fill(delta.begin(), delta.end(), Dual(0.0));
            for (int m = 0; m < M; ++m) {
                for (int i : act) {
                    Dual corr = 0.0;
                    for (int j = 0; j < m; ++j) {
                        const Dual* dj = &delta[(size_t)j * N];
                        corr += Qh[m * M + j] *
                                (dkrow(K, i, dj) + S.mass[i] * J[(size_t)j * N + i] * dj[i]);
                    }
                    b[i] = r[(size_t)m * N + i] - dt * corr;
                }
                const double c = dt * Qh[m * M + m];
                for (int i : act) {
                    dA[i] = S.mass[i] * (1.0 + c * J[(size_t)m * N + i]) + c * Kdg[i];
                    if (!std::isfinite(dA[i].v)) return ORA_NONFINITE;
                    if (!(dA[i].v > 0.0)) return ORA_DOMAIN;
                }
                std::vector<Dual> x(N);
                int iters = 0;
                const int rc = dpcg(K, c, dA, act, b, x, o->cg_rtol, o->cg_maxit, iters);
                if (iters_out) iters_out[k * ORA_MAX_M + m] = iters;
                if (rc != ORA_OK) return rc;
                for (int i : act) delta[(size_t)m * N + i] = x[i];
            }
            for (int m = 0; m < M; ++m)
                for (int i : act) V[(size_t)m * N + i] += delta[(size_t)m * N + i];
            if (!o->w_frozen) {
                for (int i : act) {
                    Dual g[ORA_MAX_M], d[ORA_MAX_M], s[ORA_MAX_M], eps[ORA_MAX_M];
                    for (int m = 0; m < M; ++m) {
                        Dual vm = V[(size_t)m * N + i], wm = W[(size_t)m * N + i];
                        if ((vm + p.mu2).v <= 0.0) return ORA_DOMAIN;
                        g[m] = dion_R(p, vm, wm);
                        d[m] = dion_dRdw(p, vm, wm);
                    }
                    for (int m = 0; m < M; ++m) {
                        Dual q = 0.0;
                        for (int j = 0; j < M; ++j) q += Q[m * M + j] * g[j];
                        s[m] = w0[i] + dt * q - W[(size_t)m * N + i];
                    }
                    for (int m = 0; m < M; ++m) {
                        Dual acc = s[m];
                        for (int j = 0; j < m; ++j) acc += dt * Qh[m * M + j] * d[j] * eps[j];
                        Dual den = 1.0 - dt * Qh[m * M + m] * d[m];
                        if (!(den.v > 0.0)) return ORA_DOMAIN;
                        eps[m] = acc / den;
                    }
                    for (int m = 0; m < M; ++m) W[(size_t)m * N + i] += eps[m];
                }
            }
        }
        // the given set of the next sweep
        std::vector<int> next;
        if (k + 1 < sweeps) {
            size_t off = 0;
            for (int kk = 1; kk <= k; ++kk) off += (size_t)forced_counts[kk];
            next.assign(forced_lists + off, forced_lists + off + forced_counts[k + 1]);
        }
        act.swap(next);
    }
    for (int i = 0; i < N; ++i) {
        v[i] = V[(size_t)(M - 1) * N + i].v;
        dv[i] = V[(size_t)(M - 1) * N + i].d;
        w[i] = W[(size_t)(M - 1) * N + i].v;
        dw[i] = W[(size_t)(M - 1) * N + i].d;
    }
    return ORA_OK;
}

}  // extern "C"
