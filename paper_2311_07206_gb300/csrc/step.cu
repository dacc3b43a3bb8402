// Kernels of one SDC sweep (Sec. 3.2, eq. final-sdc) on the active index set
// I_k (Sec. 4.2).  Compact row p of sweep k is global dof act[p] (act = NULL
// means the identity, used for the first sweep, which always covers every dof).
//
//   residual : f_j = -(K v_j) - m (I_ion(v_j, w_j) - I_stim), J_j = dI/dv,
//              r_m = m v0 + dt sum_j Q_mj f_j - m v_m         (full rows of K,
//              dropped neighbours enter with their current values)
//   pcg      : node system (diag(m (1 + c J_m)) + c K)[I, I] dv_m = b_m, c = dt Qhat_mm,
//              Jacobi-PCG in one cooperative launch; its epilogue applies the
//              LU-trick coupling b_m' -= dt Qhat_m'm (K dv_m + m J_m dv_m), m' > m
//   update   : v_m += dv_m, pointwise w sweep, selection flag max_m|dv_m| >= TOL_drop
//   select   : stable compaction of the flagged rows (warp ballot + block scan)
//   extract  : K[I_{k+1}, I_{k+1}] from K[I_k, I_k] through the old->new row map

#include <cfloat>

#include "device_common.cuh"
#include "sdc_internal.h"

namespace sdc {
namespace {

__global__ void k_spread(int N, int M, const double* __restrict__ v0, const double* __restrict__ w0,
                         double* __restrict__ V, double* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = v0[i], b = w0[i];
    for (int m = 0; m < M; ++m) {
        V[(size_t)i * M + m] = a;
        W[(size_t)i * M + m] = b;
    }
}

__global__ void k_final(int N, int M, const double* __restrict__ V, const double* __restrict__ W,
                        double* __restrict__ v, double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    v[i] = V[(size_t)i * M + M - 1];
    w[i] = W[(size_t)i * M + M - 1];
}

__global__ void k_nodes_out(int N, int M, const double* __restrict__ V, const double* __restrict__ W,
                            double* __restrict__ Vo, double* __restrict__ Wo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int m = 0; m < M; ++m) {
        Vo[(size_t)m * N + i] = V[(size_t)i * M + m];
        Wo[(size_t)m * N + i] = W[(size_t)i * M + m];
    }
}

template <int M>
__global__ void k_residual(int n, const int* __restrict__ act, const double* __restrict__ kval,
                           const int* __restrict__ kcol, const int* __restrict__ klen, int ldk,
                           const double* __restrict__ kdiag, const double* __restrict__ mass,
                           const double* __restrict__ stim, double stim_on,
                           const double* __restrict__ V, const double* __restrict__ W,
                           const double* __restrict__ v0, double dt, Ionic ion, Coll co,
                           int reaction_implicit, int ld, double* __restrict__ R,
                           double* __restrict__ Jout, double* __restrict__ mc,
                           double* __restrict__ kdc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int g = act ? act[p] : p;
    const double kd = kdiag[g];
    double vm[M], kv[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        vm[m] = V[(size_t)g * M + m];
        kv[m] = kd * vm[m];
    }
    const int len = klen[g];
    for (int t = 0; t < len; ++t) {
        const double a = kval[(size_t)t * ldk + g];
        const int j = kcol[(size_t)t * ldk + g];
#pragma unroll
        for (int m = 0; m < M; ++m) kv[m] += a * V[(size_t)j * M + m];
    }
    const double mi = mass[g];
    const double s = stim ? stim[g] * stim_on : 0.0;
    double f[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const double wm = W[(size_t)g * M + m];
        f[m] = -kv[m] - mi * (ap_I(ion, vm[m], wm) - s);
        Jout[(size_t)m * ld + p] = reaction_implicit ? ap_dIdv(ion, vm[m], wm) : 0.0;
    }
    const double base = mi * v0[g];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        double q = 0.0;
#pragma unroll
        for (int j = 0; j < M; ++j) q += co.Q[m * kMaxM + j] * f[j];
        R[(size_t)m * ld + p] = base + dt * q - mi * vm[m];
    }
    mc[p] = mi;
    kdc[p] = kd;
}

struct CgParams {
    int n, ld;
    const double* aval;
    const int* acol;
    const int* alen;
    const double* mc;
    const double* kdc;
    const double* J;     // J of this node, compact
    double c;            // dt * Qhat_mm
    const double* b;     // right-hand side of this node
    double* x;           // correction of this node (output)
    double* r;
    double* z;
    double* p;
    double* q;
    double* dA;
    double* part;
    unsigned* bar;
    int* err;
    double rtol;
    int maxit;
    long long budget;
    int* iters_out;
    double* relres_out;
    // epilogue: LU-trick coupling into the later nodes' right-hand sides
    int m, M;
    double dt;
    double* R;
    double qh[kMaxM];    // Qhat[m'][m], m' = 0..M-1
    int inject_fault;    // testing hook: the last block skips the first barrier
};

// Jacobi-PCG on the restricted node system, whole solve in one cooperative
// launch.  Rows are processed grid-stride; each thread owns the same rows in
// every phase.  Per iteration: q = A p with p.q (barrier), x/r/z updates with
// r.z (barrier), p = z + beta p (barrier).  Partial sums are reduced in a fixed
// order by every block, so all blocks take identical decisions.
__global__ void __launch_bounds__(1024) k_pcg(CgParams P) {
    __shared__ double sh[32];
    const int G = gridDim.x;
    const int stride = G * blockDim.x;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int ld = P.ld;
    unsigned epoch = 0;
    int buf = 0;

    double part = 0.0;
    for (int i = i0; i < P.n; i += stride) {
        const double d = P.mc[i] * (1.0 + P.c * P.J[i]) + P.c * P.kdc[i];
        if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        P.dA[i] = d;
        const double r = P.b[i];
        const double z = r / d;
        P.r[i] = r;
        P.p[i] = z;
        P.x[i] = 0.0;
        part += r * z;
    }
    double s = block_sum(part, sh);
    if (threadIdx.x == 0) P.part[buf * G + blockIdx.x] = s;
    if (P.inject_fault && blockIdx.x == G - 1) {
        // leave without arriving: every other block's bounded wait runs out
        if (G == 1 && threadIdx.x == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_sync(P.bar, epoch, P.budget, P.err)) return;
    const double rho0 = sum_partials(P.part + buf * G, G);
    buf ^= 1;

    int it = 0;
    double relres = 0.0;
    bool done = (rho0 == 0.0);
    if (!isfinite(rho0)) {
        if (i0 == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    const double thresh = P.rtol * sqrt(rho0);
    double rho = rho0;
    while (!done) {
        if (it >= P.maxit) {
            if (i0 == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        // q = A p, p.q
        part = 0.0;
        for (int i = i0; i < P.n; i += stride) {
            const int len = P.alen[i];
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.p + P.acol[(size_t)t * ld + i]);
            const double pi = __ldcg(P.p + i);
            const double qi = P.dA[i] * pi + P.c * acc;
            P.q[i] = qi;
            part += pi * qi;
        }
        s = block_sum(part, sh);
        if (threadIdx.x == 0) P.part[buf * G + blockIdx.x] = s;
        if (!grid_sync(P.bar, epoch, P.budget, P.err)) return;
        const double pq = sum_partials(P.part + buf * G, G);
        buf ^= 1;
        const double alpha = rho / pq;
        // x += alpha p, r -= alpha q, z = r / diag, r.z
        part = 0.0;
        for (int i = i0; i < P.n; i += stride) {
            const double pi = __ldcg(P.p + i);
            P.x[i] += alpha * pi;
            const double r = P.r[i] - alpha * P.q[i];
            P.r[i] = r;
            const double z = r / P.dA[i];
            P.z[i] = z;
            part += r * z;
        }
        s = block_sum(part, sh);
        if (threadIdx.x == 0) P.part[buf * G + blockIdx.x] = s;
        if (!grid_sync(P.bar, epoch, P.budget, P.err)) return;
        const double rho_new = sum_partials(P.part + buf * G, G);
        buf ^= 1;
        relres = sqrt(fabs(rho_new) / rho0);
        if (!isfinite(rho_new)) {
            if (i0 == 0) raise_error(P.err, SDC_E_NONFINITE);
            return;
        }
        if (sqrt(rho_new) <= thresh) break;
        const double beta = rho_new / rho;
        rho = rho_new;
        for (int i = i0; i < P.n; i += stride) P.p[i] = P.z[i] + beta * __ldcg(P.p + i);
        if (!grid_sync(P.bar, epoch, P.budget, P.err)) return;
    }
    if (i0 == 0) {
        *P.iters_out = it;
        *P.relres_out = relres;
    }
    // x is complete in every block: the last barrier followed its update.
    if (P.m + 1 < P.M) {
        for (int i = i0; i < P.n; i += stride) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.x + P.acol[(size_t)t * ld + i]);
            const double corr = P.kdc[i] * xi + acc + P.mc[i] * P.J[i] * xi;
            for (int mm = P.m + 1; mm < P.M; ++mm)
                P.R[(size_t)mm * ld + i] -= P.dt * P.qh[mm] * corr;
        }
    }
}

template <int M>
__global__ void k_update(int n, const int* __restrict__ act, const double* __restrict__ D, int ld,
                         double* __restrict__ V, double* __restrict__ W,
                         const double* __restrict__ w0, double dt, Ionic ion, Coll co,
                         double tol_drop, int w_frozen, int* __restrict__ flag,
                         int* __restrict__ blockcnt, double* __restrict__ blockmarg,
                         int* __restrict__ err) {
    __shared__ int wc[32];
    __shared__ double wmg[32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    double margin = DBL_MAX;
    if (p < n) {
        const int g = act ? act[p] : p;
        double vm[M];
        double amax = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double d = D[(size_t)m * ld + p];
            vm[m] = V[(size_t)g * M + m] + d;
            V[(size_t)g * M + m] = vm[m];
            amax = fmax(amax, fabs(d));
        }
        if (!w_frozen) {
            double wm[M], gR[M], dR[M], e[M];
            const double wz = w0[g];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                wm[m] = W[(size_t)g * M + m];
                if (!(vm[m] + ion.mu2 > 0.0)) raise_error(err, SDC_E_DOMAIN);
                ap_R_dRdw(ion, vm[m], wm[m], gR[m], dR[m]);
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                double q = 0.0;
#pragma unroll
                for (int j = 0; j < M; ++j) q += co.Q[m * kMaxM + j] * gR[j];
                double acc = wz + dt * q - wm[m];
#pragma unroll
                for (int j = 0; j < m; ++j) acc += dt * co.Qh[m * kMaxM + j] * dR[j] * e[j];
                const double den = 1.0 - dt * co.Qh[m * kMaxM + m] * dR[m];
                if (!(den > 0.0)) raise_error(err, SDC_E_DOMAIN);
                e[m] = acc / den;
            }
#pragma unroll
            for (int m = 0; m < M; ++m) W[(size_t)g * M + m] = wm[m] + e[m];
        }
        if (!isfinite(amax)) raise_error(err, SDC_E_NONFINITE);
        keep = amax >= tol_drop ? 1 : 0;
        if (tol_drop > 0.0) margin = fabs(amax - tol_drop);
        flag[p] = keep;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    margin = warp_min(margin);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        wc[wid] = __popc(bal);
        wmg[wid] = margin;
    }
    __syncthreads();
    if (wid == 0) {
        int c = lane < nw ? wc[lane] : 0;
        double mg = lane < nw ? wmg[lane] : DBL_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        mg = warp_min(mg);
        if (lane == 0) {
            blockcnt[blockIdx.x] = c;
            blockmarg[blockIdx.x] = mg;
        }
    }
}

// Exclusive scan of the per-block counts (single block), total -> sc->count,
// min margin -> sc->margin.
__global__ void k_scan_counts(int nb, const int* __restrict__ cnt, int* __restrict__ off,
                              const double* __restrict__ marg, DevScalars* sc) {
    __shared__ int ssum[1024];
    __shared__ double smin[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (nb + T - 1) / T;
    const int b0 = t * per, b1 = min(nb, b0 + per);
    int local = 0;
    double mg = DBL_MAX;
    for (int b = b0; b < b1; ++b) {
        local += cnt[b];
        mg = fmin(mg, marg[b]);
    }
    ssum[t] = local;
    smin[t] = mg;
    __syncthreads();
    // inclusive Hillis-Steele scan over T entries
    for (int o = 1; o < T; o <<= 1) {
        const int v = t >= o ? ssum[t - o] : 0;
        __syncthreads();
        ssum[t] += v;
        __syncthreads();
    }
    int run = ssum[t] - local;
    for (int b = b0; b < b1; ++b) {
        off[b] = run;
        run += cnt[b];
    }
    for (int o = T / 2; o > 0; o >>= 1) {
        if (t < o) smin[t] = fmin(smin[t], smin[t + o]);
        __syncthreads();
    }
    if (t == T - 1) sc->count = ssum[T - 1];
    if (t == 0) sc->margin = fmin(sc->margin, smin[0]);
}

__global__ void k_scatter(int n, const int* __restrict__ act, const int* __restrict__ flag,
                          const int* __restrict__ blockoff, int* __restrict__ act_next,
                          int* __restrict__ map) {
    __shared__ int woff[32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int keep = p < n ? flag[p] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) woff[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        const int c = lane < nw ? woff[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < nw) woff[lane] = incl - c;
    }
    __syncthreads();
    if (p < n) {
        const int pos = blockoff[blockIdx.x] + woff[wid] + pre;
        if (keep) act_next[pos] = act ? act[p] : p;
        map[p] = keep ? pos : -1;
    }
}

__global__ void k_extract(int n_old, const double* __restrict__ oval, const int* __restrict__ ocol,
                          const int* __restrict__ olen, int old_ld, const int* __restrict__ map,
                          double* __restrict__ nval, int* __restrict__ ncol, int* __restrict__ nlen,
                          int new_ld, unsigned long long* nnz) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (p < n_old) {
        const int qrow = map[p];
        if (qrow >= 0) {
            const int len = olen[p];
            for (int t = 0; t < len; ++t) {
                const int jn = map[ocol[(size_t)t * old_ld + p]];
                if (jn >= 0) {
                    nval[(size_t)cnt * new_ld + qrow] = oval[(size_t)t * old_ld + p];
                    ncol[(size_t)cnt * new_ld + qrow] = jn;
                    ++cnt;
                }
            }
            nlen[qrow] = cnt;
        }
    }
    // block-aggregated count (integer: order independent)
    unsigned long long c = (unsigned long long)cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nnz, c);
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

inline int nblk(int n, int b) { return (n + b - 1) / b; }

}  // namespace

void launch_spread(int N, int M, const double* v0, const double* w0, double* V, double* W,
                   cudaStream_t s) {
    k_spread<<<nblk(N, 256), 256, 0, s>>>(N, M, v0, w0, V, W);
}

void launch_final(int N, int M, const double* V, const double* W, double* v, double* w,
                  cudaStream_t s) {
    k_final<<<nblk(N, 256), 256, 0, s>>>(N, M, V, W, v, w);
}

void launch_nodes_out(int N, int M, const double* V, const double* W, double* Vo, double* Wo,
                      cudaStream_t s) {
    k_nodes_out<<<nblk(N, 256), 256, 0, s>>>(N, M, V, W, Vo, Wo);
}

void launch_residual(int M, int n, const int* act, const Ell& K, const double* kdiag,
                     const double* mass, const double* stim, double stim_on, const double* V,
                     const double* W, const double* v0, double dt, const Ionic& ion,
                     const Coll& co, int reaction_implicit, StepBuffers& B, cudaStream_t s) {
    dispatch_M(M, [&](auto mc) {
        constexpr int MM = decltype(mc)::value;
        k_residual<MM><<<nblk(n, 128), 128, 0, s>>>(n, act, K.val, K.col, K.len, K.ld, kdiag, mass,
                                                      stim, stim_on, V, W, v0, dt, ion, co,
                                                      reaction_implicit, B.ld, B.R, B.J, B.mc, B.kdc);
    });
}

int pcg_max_blocks(int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg, block, 0);
    return sms * per;
}

int launch_pcg(int n, const Ell& A, int m, double dt, const Coll& co, double rtol, int maxit,
               long long budget, int sweep, int block, int max_blocks, int inject_fault,
               StepBuffers& B, cudaStream_t s) {
    CgParams P;
    P.n = n;
    P.ld = B.ld;
    P.aval = A.val;
    P.acol = A.col;
    P.alen = A.len;
    P.mc = B.mc;
    P.kdc = B.kdc;
    P.J = B.J + (size_t)m * B.ld;
    P.c = dt * co.Qh[m * kMaxM + m];
    P.b = B.R + (size_t)m * B.ld;
    P.x = B.D + (size_t)m * B.ld;
    P.r = B.r;
    P.z = B.z;
    P.p = B.p;
    P.q = B.q;
    P.dA = B.dA;
    P.part = B.part;
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = budget;
    P.iters_out = &B.sc->cg_iters[sweep * kMaxM + m];
    P.relres_out = &B.sc->cg_relres[sweep * kMaxM + m];
    P.m = m;
    P.M = co.M;
    P.dt = dt;
    P.R = B.R;
    for (int j = 0; j < kMaxM; ++j) P.qh[j] = j < co.M ? co.Qh[j * kMaxM + m] : 0.0;
    P.inject_fault = inject_fault;
    int grid = std::min(max_blocks, nblk(n, block));
    if (grid < 1) grid = 1;
    cudaMemsetAsync(&B.sc->bar, 0, sizeof(unsigned), s);
    void* args[] = {&P};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pcg, dim3(grid), dim3(block), args,
                                                0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

void launch_update(int M, int n, const int* act, const double* w0, double dt, const Ionic& ion,
                   const Coll& co, double tol_drop, int w_frozen, StepBuffers& B, cudaStream_t s) {
    dispatch_M(M, [&](auto mc) {
        constexpr int MM = decltype(mc)::value;
        k_update<MM><<<nblk(n, kUpdateBlock), kUpdateBlock, 0, s>>>(
            n, act, B.D, B.ld, B.V, B.W, w0, dt, ion, co, tol_drop, w_frozen, B.flag, B.blockcnt,
            B.blockmarg, &B.sc->err);
    });
}

void launch_select(int n, const int* act, int* act_next, StepBuffers& B, cudaStream_t s) {
    const int nb = nblk(n, kUpdateBlock);
    k_scan_counts<<<1, 1024, 0, s>>>(nb, B.blockcnt, B.blockoff, B.blockmarg, B.sc);
    k_scatter<<<nb, kUpdateBlock, 0, s>>>(n, act, B.flag, B.blockoff, act_next, B.map);
}

void launch_extract(int n_old, const Ell& Aold, const int* map, Ell& Anew, StepBuffers& B,
                    cudaStream_t s) {
    cudaMemsetAsync(&B.sc->nnz, 0, sizeof(unsigned long long), s);
    k_extract<<<nblk(n_old, 256), 256, 0, s>>>(n_old, Aold.val, Aold.col, Aold.len, Aold.ld, map,
                                               Anew.val, Anew.col, Anew.len, Anew.ld, &B.sc->nnz);
}

}  // namespace sdc
