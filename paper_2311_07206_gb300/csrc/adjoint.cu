// Discrete adjoint of one adaptive SDC step (Sec. 3.2 eq. final-sdc, Sec. 4.2)
// with the active sets of the forward step held fixed (recorded on a tape).
//
// The forward step is a composition of differentiable maps once the index
// sets I_k are fixed and every node solve is read as the exact solution of its
// linear system.  The reverse pass visits the sweeps k = K-1 .. 0 and, inside a
// sweep, the forward operations backwards:
//   w sweep          pointwise reverse of the LU-trick recursion for w
//   v update         V' = V + dv on I_k: the adjoint passes through
//   node solves      m = M-1 .. 0: A_m bbar_m = dvbar_m (A_m symmetric: the same
//                    restricted Jacobi-PCG), then the coupling into earlier
//                    nodes dvbar_j -= dt Qhat_mj (K bbar_m + mass J_j bbar_m)
//   residual         rbar_m = bbar_m; fbar_j = dt sum_m Q_mj rbar_m; vbar0 +=
//                    mass sum_m rbar_m; Vbar_j -= K fbar_j (full rows: dropped
//                    neighbours receive their share); ionic terms
// followed by the reverse of the predictor (vbar0 += sum_m Vbar_m).
// Parameter gradients: the per-node conductivity scale s enters K through the
// element means sbar_e, so dL/dsbar_e = sum over (u, v) pairs of u_e^T Khat_e v_e
// with Khat_e the unscaled element matrix; the Aliev-Panfilov parameters
// (ga, gs, a) enter I_ion, dI/dv, R and dR/dw pointwise.

#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "sdc_internal.h"

namespace sdc {
namespace {

constexpr int kAdjBlock = 256;

inline int nb(int n, int b) { return (n + b - 1) / b; }

// Aliev-Panfilov derivatives needed by the adjoint.  p = (ga, gs, a).
struct ApDer {
    double I, Iv, Iw, Ivv, Ivw, I_ga, I_a, Iv_ga, Iv_a;
    double R, Rv, Rw, Rwv, Rww, R_gs, R_a, Rw_gs, Rw_a;
};

__device__ __forceinline__ ApDer ap_der(const Ionic& p, double v, double w) {
    ApDer d;
    const double vm1 = v - 1.0, vma = v - p.a;
    d.I = p.ga * v * vma * vm1 + v * w;
    d.Iv = p.ga * (3.0 * v * v - 2.0 * (1.0 + p.a) * v + p.a) + w;
    d.Iw = v;
    d.Ivv = p.ga * (6.0 * v - 2.0 * (1.0 + p.a));
    d.Ivw = 1.0;
    d.I_ga = v * vma * vm1;
    d.I_a = -p.ga * v * vm1;
    d.Iv_ga = 3.0 * v * v - 2.0 * (1.0 + p.a) * v + p.a;
    d.Iv_a = p.ga * (1.0 - 2.0 * v);
    const double inv = 1.0 / (v + p.mu2);
    const double E = p.eps + p.mu1 * w * inv;
    const double Ew = p.mu1 * inv;
    const double Ev = -p.mu1 * w * inv * inv;
    const double Ewv = -p.mu1 * inv * inv;
    const double G = -w - p.gs * v * (v - p.a - 1.0);
    const double Gv = -p.gs * (2.0 * v - p.a - 1.0);
    const double G_gs = -v * (v - p.a - 1.0);
    const double G_a = p.gs * v;
    d.R = p.cw * E * G;
    d.Rv = p.cw * (Ev * G + E * Gv);
    d.Rw = p.cw * (Ew * G - E);
    d.Rwv = p.cw * (Ewv * G + Ew * Gv - Ev);
    d.Rww = -2.0 * p.cw * Ew;
    d.R_gs = p.cw * E * G_gs;
    d.R_a = p.cw * E * G_a;
    d.Rw_gs = p.cw * Ew * G_gs;
    d.Rw_a = p.cw * Ew * G_a;
    return d;
}

// per-block partial sums of the three ionic-parameter gradients
__device__ __forceinline__ void block_sum3(double a, double b, double c, double* out3) {
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
        sh[2][wid] = c;
    }
    __syncthreads();
    if (wid == 0) {
        double x = lane < nw ? sh[0][lane] : 0.0;
        double y = lane < nw ? sh[1][lane] : 0.0;
        double z = lane < nw ? sh[2][lane] : 0.0;
        x = warp_sum(x);
        y = warp_sum(y);
        z = warp_sum(z);
        if (lane == 0) {
            out3[3 * blockIdx.x + 0] = x;
            out3[3 * blockIdx.x + 1] = y;
            out3[3 * blockIdx.x + 2] = z;
        }
    }
}

// fixed-order sum of nblk block partials into the running accumulator acc[3]
__global__ void k_sum3(int nblk, const double* __restrict__ part, double* __restrict__ acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < nblk; ++i) {
        a += part[3 * i];
        b += part[3 * i + 1];
        c += part[3 * i + 2];
    }
    acc[0] += a;
    acc[1] += b;
    acc[2] += c;
}

__global__ void k_adj_init(int N, int M, const double* __restrict__ lv,
                           const double* __restrict__ lw, double* __restrict__ Vb,
                           double* __restrict__ Wb, double* __restrict__ lv0,
                           double* __restrict__ lw0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int m = 0; m < M; ++m) {
        Vb[(size_t)i * M + m] = m == M - 1 ? lv[i] : 0.0;
        Wb[(size_t)i * M + m] = m == M - 1 ? lw[i] : 0.0;
    }
    lv0[i] = 0.0;
    lw0[i] = 0.0;
}

// Reverse of the pointwise w sweep on the active rows.  Vn: v after the sweep,
// Wo / Wn: w before / after; Wb is replaced by the adjoint of w before the
// sweep, Vb (adjoint of v after the sweep) and lw0 accumulate.
template <int M>
__global__ void k_adj_wsweep(int n, const int* __restrict__ act, const double* __restrict__ Vn,
                             const double* __restrict__ Wo, const double* __restrict__ Wn,
                             double dt, Ionic ion, Coll co, double* __restrict__ Vb,
                             double* __restrict__ Wb, double* __restrict__ lw0,
                             double* __restrict__ part3, int N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double gga = 0.0, ggs = 0.0, ga_ = 0.0;
    if (p < n) {
        const int g = act ? sdc_idx(act[p], N, 201) : p;
        ApDer d[M];
        double eps[M], den[M], eb[M], Nb[M], sb[M], gb[M], db[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            d[m] = ap_der(ion, Vn[(size_t)g * M + m], Wo[(size_t)g * M + m]);
            eps[m] = Wn[(size_t)g * M + m] - Wo[(size_t)g * M + m];
            den[m] = 1.0 - dt * co.Qh[m * kMaxM + m] * d[m].Rw;
            eb[m] = Wb[(size_t)g * M + m];     // adjoint of W' = W + eps
            gb[m] = 0.0;
            db[m] = 0.0;
        }
        // eps_m = N_m / den_m,  N_m = s_m + dt sum_{j<m} Qh_mj d_j eps_j
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
            Nb[m] = eb[m] / den[m];
            const double denb = -eb[m] * eps[m] / den[m];
            db[m] += denb * (-dt * co.Qh[m * kMaxM + m]);
            sb[m] = Nb[m];
#pragma unroll
            for (int j = 0; j < m; ++j) {
                db[j] += Nb[m] * dt * co.Qh[m * kMaxM + j] * eps[j];
                eb[j] += Nb[m] * dt * co.Qh[m * kMaxM + j] * d[j].Rw;
            }
        }
        // s_m = w0 + dt sum_j Q_mj g_j - W_m
        double w0b = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            w0b += sb[m];
#pragma unroll
            for (int j = 0; j < M; ++j) gb[j] += dt * co.Q[m * kMaxM + j] * sb[m];
        }
        lw0[g] += w0b;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            // W' = W + eps: adjoint of W is eb (direct) - sb (via s) + chain through g, d
            const double wb = Wb[(size_t)g * M + m] - sb[m] + gb[m] * d[m].Rw + db[m] * d[m].Rww;
            Wb[(size_t)g * M + m] = wb;
            Vb[(size_t)g * M + m] += gb[m] * d[m].Rv + db[m] * d[m].Rwv;
            ggs += gb[m] * d[m].R_gs + db[m] * d[m].Rw_gs;
            ga_ += gb[m] * d[m].R_a + db[m] * d[m].Rw_a;
        }
    }
    block_sum3(gga, ggs, ga_, part3);
}

// Per-sweep quantities of the active rows (compact): J, dv, mass, K_ii, and the
// adjoint of dv gathered from Vb.
template <int M>
__global__ void k_adj_prep(int n, const int* __restrict__ act, const double* __restrict__ Vo,
                           const double* __restrict__ Wo, const double* __restrict__ Vn,
                           const double* __restrict__ kdiag, const double* __restrict__ mass,
                           const double* __restrict__ Vb, Ionic ion, int reaction_implicit,
                           int ld, double* __restrict__ J, double* __restrict__ D,
                           double* __restrict__ mc, double* __restrict__ kdc,
                           double* __restrict__ Db, double* __restrict__ Jb, int N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int g = act ? sdc_idx(act[p], N, 202) : p;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const double v = Vo[(size_t)g * M + m], w = Wo[(size_t)g * M + m];
        J[(size_t)m * ld + p] = reaction_implicit ? ap_dIdv(ion, v, w) : 0.0;
        D[(size_t)m * ld + p] = Vn[(size_t)g * M + m] - v;
        Db[(size_t)m * ld + p] = Vb[(size_t)g * M + m];
        Jb[(size_t)m * ld + p] = 0.0;
    }
    mc[p] = mass[g];
    kdc[p] = kdiag[g];
}

// After the reverse solve of node m (x = bbar_m): adjoint of J through A_m and
// through the couplings b_m uses for j < m; the conductivity pairs; and the
// full-length copy of bbar_m.
template <int M>
__global__ void k_adj_node_post(int n, const int* __restrict__ act, int m, double dt, Coll co,
                                int ld, int N, const double* __restrict__ x,
                                const double* __restrict__ D, const double* __restrict__ mc,
                                double* __restrict__ Jb, double* __restrict__ bfull,
                                double* __restrict__ vkfull) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int g = act ? sdc_idx(act[p], N, 203) : p;
    const double xb = x[p];
    const double cm = dt * co.Qh[m * kMaxM + m];
    const double dm = D[(size_t)m * ld + p];
    Jb[(size_t)m * ld + p] += -mc[p] * cm * xb * dm;
    double vk = -cm * dm;
    for (int j = 0; j < m; ++j) {
        const double dj = D[(size_t)j * ld + p];
        Jb[(size_t)j * ld + p] += -dt * co.Qh[m * kMaxM + j] * mc[p] * dj * xb;
        vk += -dt * co.Qh[m * kMaxM + j] * dj;
    }
    bfull[(size_t)m * N + g] = xb;
    vkfull[(size_t)m * N + g] = vk;
}

// Reverse of the residual on the active rows: rbar_m = bbar_m.
template <int M>
__global__ void k_adj_residual(int n, const int* __restrict__ act, int ld, int N, double dt,
                               Coll co, Ionic ion, int reaction_implicit,
                               const double* __restrict__ X, const double* __restrict__ Jb,
                               const double* __restrict__ Vo, const double* __restrict__ Wo,
                               const double* __restrict__ mass, double* __restrict__ Vb,
                               double* __restrict__ Wb, double* __restrict__ lv0,
                               double* __restrict__ ffull, double* __restrict__ part3) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double gga = 0.0, ggs = 0.0, ga_ = 0.0;
    if (p < n) {
        const int g = act ? sdc_idx(act[p], N, 204) : p;
        const double mi = mass[g];
        double rb[M], fb[M];
        double rsum = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            rb[m] = X[(size_t)m * ld + p];
            rsum += rb[m];
            fb[m] = 0.0;
        }
        lv0[g] += mi * rsum;
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int j = 0; j < M; ++j) fb[j] += dt * co.Q[m * kMaxM + j] * rb[m];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const ApDer d = ap_der(ion, Vo[(size_t)g * M + j], Wo[(size_t)g * M + j]);
            const double jb = reaction_implicit ? Jb[(size_t)j * ld + p] : 0.0;
            // r_j = ... - mass V_j ;  f_j = -K V_j - mass (I - stim) ;  J_j = dI/dv
            Vb[(size_t)g * M + j] += -mi * rb[j] - mi * d.Iv * fb[j] + jb * d.Ivv;
            Wb[(size_t)g * M + j] += -mi * d.Iw * fb[j] + jb * d.Ivw;
            gga += -mi * d.I_ga * fb[j] + jb * d.Iv_ga;
            ga_ += -mi * d.I_a * fb[j] + jb * d.Iv_a;
            ffull[(size_t)j * N + g] = fb[j];
        }
    }
    block_sum3(gga, ggs, ga_, part3);
}

// Vb_j -= K fbar_j over every row (fbar is zero off the active set).
template <int M>
__global__ void k_adj_kfull(int N, const double* __restrict__ kval, const int* __restrict__ kcol,
                            const int* __restrict__ klen, int ldk, const double* __restrict__ kdiag,
                            const double* __restrict__ ffull, double* __restrict__ Vb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = kdiag[i] * ffull[(size_t)m * N + i];
    const int len = klen[i];
    for (int t = 0; t < len; ++t) {
        const double a = kval[(size_t)t * ldk + i];
        const int j = sdc_idx(kcol[(size_t)t * ldk + i], N, 205);
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] += a * ffull[(size_t)m * N + j];
    }
#pragma unroll
    for (int m = 0; m < M; ++m) Vb[(size_t)i * M + m] -= acc[m];
}

// dL/dsbar_e += sum_m bbar_m^T Khat_e vk_m - sum_j fbar_j^T Khat_e V_j
template <int M>
__global__ void k_adj_elem(int NE, int dim, const double* __restrict__ xyz,
                           const int* __restrict__ elem, const double* __restrict__ sig9,
                           const double* __restrict__ esig9, int N,
                           const double* __restrict__ bfull, const double* __restrict__ vkfull,
                           const double* __restrict__ ffull, const double* __restrict__ Vo,
                           double* __restrict__ ge) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NE) return;
    const int nv = dim + 1;
    const int* vt = elem + (size_t)e * nv;
    double grad[4][3], vol;
    if (!p1_gradients(dim, xyz, vt, grad, vol)) return;
    const double* Dm = esig9 ? esig9 + (size_t)e * 9 : sig9;
    double Ke[4][4];
    for (int a = 0; a < nv; ++a) {
        double Dg[3] = {0, 0, 0};
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) Dg[c] += grad[a][r] * Dm[r * 3 + c];
        for (int b = 0; b < nv; ++b) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += Dg[c] * grad[b][c];
            Ke[a][b] = vol * s;
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        for (int a = 0; a < nv; ++a) {
            const double ub = bfull[(size_t)m * N + vt[a]];
            const double uf = ffull[(size_t)m * N + vt[a]];
            if (ub == 0.0 && uf == 0.0) continue;
            double kb = 0.0, kf = 0.0;
            for (int b = 0; b < nv; ++b) {
                kb += Ke[a][b] * vkfull[(size_t)m * N + vt[b]];
                kf += Ke[a][b] * Vo[(size_t)vt[b] * M + m];
            }
            acc += ub * kb - uf * kf;
        }
    }
    ge[e] += acc;
}

// dL/ds_a += sum over elements e containing a of dL/dsbar_e / (d + 1)
__global__ void k_adj_scale_nodes(int N, int nv, const int* __restrict__ n2e_ptr,
                                  const int* __restrict__ n2e, const double* __restrict__ ge,
                                  double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int k = n2e_ptr[i]; k < n2e_ptr[i + 1]; ++k) s += ge[n2e[k]];
    grad[i] += s / nv;
}

__global__ void k_adj_spread_back(int N, int M, const double* __restrict__ Vb,
                                  const double* __restrict__ Wb, double* __restrict__ lv0,
                                  double* __restrict__ lw0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double a = 0.0, b = 0.0;
    for (int m = 0; m < M; ++m) {
        a += Vb[(size_t)i * M + m];
        b += Wb[(size_t)i * M + m];
    }
    lv0[i] += a;
    lw0[i] += b;
}

__global__ void k_pos_set(int n, const int* __restrict__ act, int* __restrict__ pos, int reset,
                          int N) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    pos[sdc_idx(act[q], N, 206)] = reset ? -1 : q;
}

// restricted matrix of an arbitrary active list, straight from the global K
__global__ void k_extract_global(int n, const int* __restrict__ act, const int* __restrict__ pos,
                                 const double* __restrict__ kval, const int* __restrict__ kcol,
                                 const int* __restrict__ klen, int ldk, double* __restrict__ nval,
                                 int* __restrict__ ncol, int* __restrict__ nlen, int ldn, int N) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int g = sdc_idx(act[q], N, 207);
    const int len = klen[g];
    int c = 0;
    for (int t = 0; t < len; ++t) {
        const int jn = pos[sdc_idx(kcol[(size_t)t * ldk + g], N, 208)];
        if (jn >= 0) {
            nval[(size_t)c * ldn + q] = kval[(size_t)t * ldk + g];
            ncol[(size_t)c * ldn + q] = jn;
            ++c;
        }
    }
    nlen[q] = c;
}

// old compact row -> position in a replayed next list (pos holds that list)
__global__ void k_replay_map(int n_old, const int* __restrict__ act_old,
                             const int* __restrict__ pos, int* __restrict__ map, int N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_old) return;
    map[p] = pos[act_old ? sdc_idx(act_old[p], N, 209) : p];
}

template <class F>
void dispatch_M(int M, F&& f) {
    switch (M) {
        case 1: f(std::integral_constant<int, 1>()); break;
        case 2: f(std::integral_constant<int, 2>()); break;
        case 3: f(std::integral_constant<int, 3>()); break;
        case 4: f(std::integral_constant<int, 4>()); break;
        case 5: f(std::integral_constant<int, 5>()); break;
        case 6: f(std::integral_constant<int, 6>()); break;
        case 7: f(std::integral_constant<int, 7>()); break;
        case 8: f(std::integral_constant<int, 8>()); break;
        default: break;
    }
}

}  // namespace

void launch_pos_set(int n, const int* act, int* pos, int reset, int N, cudaStream_t s) {
    if (n > 0) k_pos_set<<<nb(n, kAdjBlock), kAdjBlock, 0, s>>>(n, act, pos, reset, N);
}

void launch_replay_map(int n_old, const int* act_old, const int* pos, int* map, int N,
                       cudaStream_t s) {
    if (n_old > 0)
        k_replay_map<<<nb(n_old, kAdjBlock), kAdjBlock, 0, s>>>(n_old, act_old, pos, map, N);
}

void launch_extract_global(int n, const int* act, const int* pos, const Ell& K, Ell& out, int N,
                           cudaStream_t s) {
    if (n > 0)
        k_extract_global<<<nb(n, kAdjBlock), kAdjBlock, 0, s>>>(n, act, pos, K.val, K.col, K.len,
                                                                K.ld, out.val, out.col, out.len,
                                                                out.ld, N);
}

int adjoint_step(const AdjointArgs& a, StepBuffers& B, AdjointBuffers& W, cudaStream_t s) {
    const int N = B.N, M = B.M, ld = B.ld;
    const MeshDev& md = *a.mesh;
    const Ell& K = *a.K;
    cudaMemsetAsync(W.iacc, 0, 3 * sizeof(double), s);
    if (a.grad_scale) cudaMemsetAsync(W.ge, 0, (size_t)md.n_elems * sizeof(double), s);
    k_adj_init<<<nb(N, kAdjBlock), kAdjBlock, 0, s>>>(N, M, a.lam_v, a.lam_w, W.Vb, W.Wb,
                                                     a.lam_v0, a.lam_w0);
    // state before sweep 0: the predictor (spread of v0, w0)
    launch_spread(N, M, a.v0, a.w0, W.V0, W.W0, s);
    int status = SDC_OK;
    for (int k = a.sweeps - 1; k >= 0 && status == SDC_OK; --k) {
        const int n = a.n_active[k];
        if (n == 0) continue;
        const double* Vo = k == 0 ? W.V0 : a.tape_V + (size_t)(k - 1) * N * M;
        const double* Wo = k == 0 ? W.W0 : a.tape_W + (size_t)(k - 1) * N * M;
        const double* Vn = a.tape_V + (size_t)k * N * M;
        const double* Wn = a.tape_W + (size_t)k * N * M;
        const int* act = k == 0 ? nullptr : a.tape_act + (size_t)k * N;
        const int nbk = nb(n, kAdjBlock);
        // restricted matrix of I_k
        const Ell* A = &K;
        if (act) {
            launch_pos_set(n, act, W.pos, 0, N, s);
            launch_extract_global(n, act, W.pos, K, B.A[0], N, s);
            launch_pos_set(n, act, W.pos, 1, N, s);
            A = &B.A[0];
        }
        dispatch_M(M, [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            if (!a.w_frozen) {
                k_adj_wsweep<MM><<<nbk, kAdjBlock, 0, s>>>(n, act, Vn, Wo, Wn, a.dt, a.ion, a.co,
                                                           W.Vb, W.Wb, a.lam_w0, W.part3, N);
                k_sum3<<<1, 32, 0, s>>>(nbk, W.part3, W.iacc);
            }
            k_adj_prep<MM><<<nbk, kAdjBlock, 0, s>>>(n, act, Vo, Wo, Vn, a.kdiag, a.mass, W.Vb,
                                                     a.ion, a.reaction_implicit, ld, B.J, B.D,
                                                     B.mc, B.kdc, B.R, W.Jb, N);
        });
        cudaMemsetAsync(W.bfull, 0, (size_t)M * N * sizeof(double), s);
        cudaMemsetAsync(W.vkfull, 0, (size_t)M * N * sizeof(double), s);
        cudaMemsetAsync(W.ffull, 0, (size_t)M * N * sizeof(double), s);
        for (int m = M - 1; m >= 0 && status == SDC_OK; --m) {
            PcgRole role{};
            role.b = B.R + (size_t)m * ld;            // dvbar_m (coupled)
            role.x = W.X + (size_t)m * ld;            // bbar_m
            role.J = B.J + (size_t)m * ld;
            role.Jall = B.J;
            role.R = B.R;
            role.epi_lo = 0;
            role.epi_hi = m;
            role.epi_target_J = 1;
            for (int j = 0; j < kMaxM; ++j) role.qh[j] = j < M ? a.co.Qh[m * kMaxM + j] : 0.0;
            role.c = a.dt * a.co.Qh[m * kMaxM + m];
            role.iters_out = W.iters + (size_t)k * kMaxM + m;
            role.relres_out = W.relres + (size_t)k * kMaxM + m;
            if (launch_pcg_role(n, *A, role, a.dt, M, a.rtol, a.maxit, *a.cfg, B, s) != SDC_OK) {
                status = SDC_E_CUDA;
                break;
            }
            dispatch_M(M, [&](auto mc) {
                constexpr int MM = decltype(mc)::value;
                k_adj_node_post<MM><<<nbk, kAdjBlock, 0, s>>>(n, act, m, a.dt, a.co, ld, N,
                                                              W.X + (size_t)m * ld, B.D, B.mc,
                                                              W.Jb, W.bfull, W.vkfull);
            });
        }
        if (status != SDC_OK) break;
        dispatch_M(M, [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            k_adj_residual<MM><<<nbk, kAdjBlock, 0, s>>>(n, act, ld, N, a.dt, a.co, a.ion,
                                                         a.reaction_implicit, W.X, W.Jb, Vo, Wo,
                                                         a.mass, W.Vb, W.Wb, a.lam_v0, W.ffull,
                                                         W.part3);
            k_sum3<<<1, 32, 0, s>>>(nbk, W.part3, W.iacc);
            k_adj_kfull<MM><<<nb(N, kAdjBlock), kAdjBlock, 0, s>>>(N, K.val, K.col, K.len, K.ld,
                                                                  a.kdiag, W.ffull, W.Vb);
            if (a.grad_scale)
                k_adj_elem<MM><<<nb(md.n_elems, 128), 128, 0, s>>>(
                    md.n_elems, md.dim, md.xyz, md.elem, md.sig, md.esig, N, W.bfull, W.vkfull,
                    W.ffull, Vo, W.ge);
        });
    }
    if (status != SDC_OK) return status;
    k_adj_spread_back<<<nb(N, kAdjBlock), kAdjBlock, 0, s>>>(N, M, W.Vb, W.Wb, a.lam_v0,
                                                            a.lam_w0);
    if (a.grad_scale)
        k_adj_scale_nodes<<<nb(N, kAdjBlock), kAdjBlock, 0, s>>>(N, md.dim + 1, md.n2e_ptr,
                                                                md.n2e, W.ge, a.grad_scale);
    return SDC_OK;
}

}  // namespace sdc

namespace sdc {
SDC_CHECK_READER(check_take_adjoint)
}  // namespace sdc
