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
#include <cstdint>

#include <cooperative_groups.h>

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

__global__ void k_perm_gather(int N, const int* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[sdc_idx(perm[i], N, 1)];
}
__global__ void k_perm_scatter(int N, const int* __restrict__ perm, const double* __restrict__ src,
                               double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[sdc_idx(perm[i], N, 2)] = src[i];
}
__global__ void k_nodes_out_perm(int N, int M, const int* __restrict__ perm,
                                 const double* __restrict__ X, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int o = sdc_idx(perm[i], N, 3);
    for (int m = 0; m < M; ++m) out[(size_t)m * N + o] = X[(size_t)i * M + m];
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
                           double* __restrict__ kdc, const int* __restrict__ n_dev, int N) {
    if (n_dev) n = *n_dev;   // device-driven sweeps: |I_k| from the device, grid for N
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int g = act ? sdc_idx(act[p], N, 4) : p;
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
        const int j = sdc_idx(kcol[(size_t)t * ldk + g], N, 5);
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

// One block's share of a batched PCG launch.
struct SegBlock {
    int row0, row1;   // compact rows of the instance
    int blk0, nblk;   // the instance's first block and block count
    int seg;          // instance index
};

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
    // CG vectors of the global-vector variant (the shared-memory variants keep
    // their rows on chip): residual r, u = D^-1 r, w = A u, the recurrences
    // p, s = A p, z = A D^-1 s, and nv = A m
    double* r;
    double* u;           // also: u published for the initial product A u
    double* w;
    double* p;
    double* s;
    double* z;
    double* nv;
    double* m;           // m = D^-1 w, published for the neighbours' gathers, two buffers of ld
    double* idA;         // reciprocal of the diagonal (Jacobi preconditioner)
    double* part;        // per-block exact-sum records, two buffers
    unsigned* bar;
    int* err;
    double rtol;
    int maxit;
    long long budget;
    int* iters_out;
    double* relres_out;
    double* energy_out;  // x' A x of the solution (may be null)
    // epilogue: LU-trick coupling into the later nodes' right-hand sides
    int m_node, M;
    double dt;
    double* R;
    double qh[kMaxM];    // coupling coefficient per target node
    // targets [epi_lo, epi_hi): R[t] -= dt qh[t] (K x + mass J' x), with J' this
    // node's J (forward sweep, targets after m) or the target's own J taken from
    // Jall (reverse sweep, targets before m)
    int epi_lo, epi_hi, epi_target_J;
    const double* Jall;
    int inject_fault;    // testing hook: the last block skips the first barrier
    int L;               // rows per block (shared-memory variants)
    // symmetrically scaled form (k_pcg_scaled): s = diag^-1/2 per row and the
    // scaled off-diagonal values c s_i a_ij s_j, rebuilt per solve (null: not used)
    double* sv;
    double* sval;
};

// LU-trick coupling of one solved row into the right-hand sides of other nodes.
__device__ __forceinline__ void cg_couple_row(const CgParams& P, int i, double xi, double kx) {
    const double base = P.kdc[i] * xi + kx;
    for (int t = P.epi_lo; t < P.epi_hi; ++t) {
        const double Jt = P.epi_target_J ? P.Jall[(size_t)t * P.ld + i] : P.J[i];
        P.R[(size_t)t * P.ld + i] -= P.dt * P.qh[t] * (base + P.mc[i] * Jt * xi);
    }
}

// Off-diagonal product of row i over its ELL slots, acc + sum_k val(k) x(col(k))
// in slot order (the same FMAs, in the same order, as a plain slot loop).  The
// column and value loads of CH slots, and then their gathers, are all issued
// before the first multiply, so a row costs two memory round trips per CH slots
// instead of two per slot: the latency that bounds an iteration when a thread
// has one or two rows.  CH follows the register budget of the block size
// (1024-thread blocks have 64 registers per thread).
template <int MAXT>
struct EllChunk {
    static constexpr int value = MAXT > 512 ? 3 : 6;
};

template <int CH, class Val, class Gather>
__device__ __forceinline__ double ell_row_dot(double acc, int len, size_t i, int ld,
                                              const int* __restrict__ col, int ncol, Val&& val,
                                              Gather&& gather) {
    for (int k0 = 0; k0 < len; k0 += CH) {
        int j[CH];
        double a[CH], x[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (k0 + k < len) {
                const size_t q = (size_t)(k0 + k) * ld + i;
                j[k] = sdc_idx(__ldg(col + q), ncol, 6);
                a[k] = val(q);
            }
        }
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (k0 + k < len) x[k] = gather(j[k]);
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (k0 + k < len) acc += a[k] * x[k];
    }
    return acc;
}

// Shared per-block state of a CG solve.  The scalars are derived by lane 0
// of warps 0 and 1 from each pair of grid-wide sums (a few FP64 operations
// per block, not per thread: the FP64 pipe is the scarce unit on this part).
struct CgShared {
    XsScratch xs;           // exact block sums
    double alpha, beta, den, gamma0, rzmax, rn;
    double energy;          // x' A x of the iterate: sum of alpha_t gamma_t over the steps taken
    double inv_g[2];        // 1 / gamma of the last two sums (warp 1)
    int ok, state;          // state: 0 iterating, 1 converged, 2 non-finite
};

// The stopping test sqrt(r.u) <= rtol sqrt(r0.u0) is evaluated as
// r.u <= rzmax with rzmax the largest double whose correctly rounded square
// root does not exceed the threshold (sqrt is monotone), found once per solve:
// the same decision without a square root per iteration.
__device__ __forceinline__ double largest_with_sqrt_at_most(double thresh) {
    double r = thresh * thresh;
    for (int k = 0; k < 64 && !(sqrt(r) <= thresh); ++k) r = nextafter(r, 0.0);
    for (int k = 0; k < 64; ++k) {
        const double up = nextafter(r, INFINITY);
        if (!(sqrt(up) <= thresh)) break;
        r = up;
    }
    return r;
}

// Scalars of sum number t from gamma = r.u and delta = w.u:
//   t = 0:  alpha = gamma / delta, beta = 0, den = delta
//   t > 0:  beta = gamma / gamma_old, den = delta - beta^2 den_old,
//           alpha = gamma / den
// (den_t = delta_t - beta_t gamma_t / alpha_{t-1}, since
// alpha_{t-1} = gamma_{t-1} / den_{t-1}).  Warp 0 lane 0 runs this chain;
// warp 1 lane 0 meanwhile forms 1/gamma for the next beta and, on the first
// sum, the stopping bound, so the chain holds one division.
__device__ __forceinline__ void cg_scalars(CgShared& S, int wid, int t, double g, double d,
                                           double rtol) {
    if (wid == 0) {
        S.rn = g;
        if (t == 0) {
            S.gamma0 = g;
            S.energy = 0.0;
        }
        if (!isfinite(g) || !isfinite(d)) {
            S.state = 2;
        } else if (t == 0 ? g == 0.0 : (g >= 0.0 && g <= S.rzmax)) {
            S.state = 1;
        } else {
            const double beta = t == 0 ? 0.0 : g * S.inv_g[(t - 1) & 1];
            const double den = t == 0 ? d : fma(-beta, beta * S.den, d);
            S.alpha = g / den;
            S.beta = beta;
            S.den = den;
            S.state = 0;
            // the iterate is x = sum_t alpha_t p_t with A-conjugate p_t, so
            // x' A x = sum_t alpha_t^2 p_t' A p_t = sum_t alpha_t gamma_t
            S.energy = fma(S.alpha, g, S.energy);
        }
    } else {
        S.inv_g[t & 1] = 1.0 / g;
        if (t == 0) S.rzmax = largest_with_sqrt_at_most(rtol * sqrt(g));
    }
}
// Sec. 3.2 energy-norm termination: in exact arithmetic the CG iterate from
// x0 = 0 has x' A x = sum_t alpha_t gamma_t, so the norm needs no product.
// final relative preconditioned residual sqrt(r.u / r0.u0)
__device__ __forceinline__ double cg_relres(const CgShared& S) {
    return S.gamma0 > 0.0 ? sqrt(fabs(S.rn) / S.gamma0) : 0.0;
}

// Block part of a group sum: exact block sums of (a, b); thread 0 publishes
// them to part[bidx] and arrives at the group barrier, which also publishes
// every global write the block made before it.  Returns false (in every
// thread) after a barrier timeout.
__device__ __forceinline__ bool cg_publish_arrive(double a, double b, CgShared& S, XsRecord* part,
                                                  unsigned* bar, int nblk, int bidx,
                                                  unsigned& epoch, long long budget, int* err) {
    int fa, fb;
    __int128 qa, qb;
    xs_block_sum2(a, b, S.xs, fa, fb, qa, qb);
    epoch += nblk;
    if (threadIdx.x == 0) {
        xs_store(part + bidx, fa, fb, qa, qb);
        S.ok = barrier_arrive_wait(bar, epoch, budget, err);
    }
    __syncthreads();
    return S.ok != 0;
}

// Jacobi-PCG on the restricted node system in the pipelined arrangement of
// Ghysels and Vanroose (2014), whole solve in one cooperative launch.
//
// With u = D^-1 r, w = A u and m = D^-1 w, an iteration needs the two dot
// products gamma = r.u and delta = w.u and one product n = A m, and the
// product does not depend on the iteration's scalars.  So one grid-wide
// synchronisation per iteration both publishes m for the neighbours' gathers
// and completes the sums: after it, warps 0 and 1 add the blocks' exact
// partial sums and derive alpha and beta while the other warps form n = A m.
// Per iteration:
//   U+L (local): z = n + beta z, s = w + beta s, p = u + beta p,
//                x += alpha p, r -= alpha s, w -= alpha z, then u = D^-1 r
//                and m = D^-1 w directly (not by recurrence: exact relations
//                that keep u consistent with r), r.u, w.u; m is published
//   sync:        exact block sums, group barrier
//   S (overlap): n = A m (the diagonal part of A m is D m = w)  ||  totals,
//                convergence test on r.u, beta and alpha
// The iterates are those of standard preconditioned CG in exact arithmetic.
// m is published to two alternating buffers: a block may write the next m
// while a slower neighbour still gathers the current one.
//
// One group of `nblk` blocks solves rows [row0, row1) in contiguous chunks of
// Lg rows per block: the whole launch, or one instance of a batched launch.
// `part` points at the group's first record of buffer 0; buffer 1 is
// `pstride` records further.  Threads [sp0, B) form the products while warps
// 0 and 1 sum; blocks under 256 threads do both in turn.
__device__ __forceinline__ void pcg_group(const CgParams& P, CgShared& S, int row0, int row1,
                                          int nblk, int bidx, unsigned* bar, XsRecord* part,
                                          int pstride, int* iters_out, double* relres_out) {
    const int B = blockDim.x, t = threadIdx.x;
    const int Lg = (row1 - row0 + nblk - 1) / nblk;
    const int c0 = row0 + bidx * Lg;
    const int c1 = min(row1, c0 + Lg);
    const bool lead = (bidx == 0 && t == 0);
    const int sp0 = B >= 256 ? 64 : 0;
    const int ld = P.ld;
    const double c = P.c;
    double* const mbuf[2] = {P.m, P.m + ld};
    unsigned epoch = 0;
    int buf = 0;

    for (int i = c0 + t; i < c1; i += B) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        P.idA[i] = id;
        const double r = P.b[i];
        P.r[i] = r;
        P.u[i] = r * id;
        P.p[i] = 0.0;
        P.s[i] = 0.0;
        P.z[i] = 0.0;
        P.x[i] = 0.0;
    }
    if (P.inject_fault && bidx == nblk - 1) {
        // leave without arriving: every other block's bounded wait runs out
        if (nblk == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    // w = A u; first r.u, w.u and m
    double ga = 0.0, de = 0.0;
    for (int i = c0 + t; i < c1; i += B) {
        const int len = P.alen[i];
        double acc = 0.0;
        for (int k = 0; k < len; ++k)
            acc += P.aval[(size_t)k * ld + i] * __ldcg(P.u + sdc_idx(P.acol[(size_t)k * ld + i], P.n, 11));
        const double ri = P.r[i], ui = P.u[i];
        const double wi = ri + c * acc;
        P.w[i] = wi;
        ga += ri * ui;
        de += wi * ui;
        mbuf[0][i] = P.idA[i] * wi;
    }
    int it = 0, nsum = 0;
    while (true) {
        if (!cg_publish_arrive(ga, de, S, part + buf * pstride, bar, nblk, bidx, epoch,
                               P.budget, P.err))
            return;
        const double* mc = mbuf[nsum & 1];
        auto totals = [&]() {
            double g, d;
            xs_group_total(nblk, [&](int k) { return xs_load_cg(part + buf * pstride + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        };
        if (sp0 > 0 && t < 64) totals();
        if (t >= sp0) {
            for (int i = c0 + t - sp0; i < c1; i += B - sp0) {
                const int len = P.alen[i];
                double acc = 0.0;
                for (int k = 0; k < len; ++k)
                    acc += P.aval[(size_t)k * ld + i] * __ldcg(mc + sdc_idx(P.acol[(size_t)k * ld + i], P.n, 12));
                P.nv[i] = P.w[i] + c * acc;
            }
        }
        if (sp0 == 0 && t < 64) totals();
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        double* mn = mbuf[nsum & 1];
        ga = de = 0.0;
        for (int i = c0 + t; i < c1; i += B) {
            // every operand of the row loaded before the first store (the vectors may
            // alias as far as the compiler knows)
            const double id = P.idA[i];
            const double wi = P.w[i], ui = P.u[i], ni = P.nv[i], z0 = P.z[i], s0 = P.s[i],
                         p0 = P.p[i], xi = P.x[i], r0 = P.r[i];
            const double zi = ni + beta * z0;
            const double si = wi + beta * s0;
            const double pi = ui + beta * p0;
            P.z[i] = zi;
            P.s[i] = si;
            P.p[i] = pi;
            P.x[i] = xi + alpha * pi;
            const double r2 = r0 - alpha * si;
            const double w2 = wi - alpha * zi;
            const double u2 = id * r2;
            P.r[i] = r2;
            P.u[i] = u2;
            P.w[i] = w2;
            ga += r2 * u2;
            de += w2 * u2;
            mn[i] = id * w2;
        }
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *iters_out = it;
        *relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x is complete and visible in every block: the last group barrier followed its update.
    if (P.epi_lo < P.epi_hi) {
        for (int i = c0 + t; i < c1; i += B) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += P.aval[(size_t)k * ld + i] * __ldcg(P.x + sdc_idx(P.acol[(size_t)k * ld + i], P.n, 13));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

// The symmetrically scaled form of pcg_group (see k_pcg_scaled): CG on
// I + c S K_off S with S = diag^-1/2, vectors in global memory, any size.
__device__ __forceinline__ void pcg_group_scaled(const CgParams& P, CgShared& S, int nblk,
                                                 int bidx) {
    const int B = blockDim.x, t = threadIdx.x;
    const int n = P.n;
    const int Lg = (n + nblk - 1) / nblk;
    const int c0 = bidx * Lg;
    const int c1 = min(n, c0 + Lg);
    const bool lead = (bidx == 0 && t == 0);
    const int sp0 = B >= 256 ? 64 : 0;
    const int ld = P.ld;
    const double c = P.c;
    double* const mbuf[2] = {P.m, P.m + ld};
    double* __restrict__ sg = P.sv;
    double* __restrict__ sval = P.sval;
    XsRecord* const part = reinterpret_cast<XsRecord*>(P.part);
    unsigned epoch = 0;
    int buf = 0;

    for (int i = c0 + t; i < c1; i += B) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        double si = 0.0;
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        else si = rsqrt(d);
        sg[i] = si;
        const double r = si * P.b[i];
        P.r[i] = r;
        P.u[i] = r;
        P.p[i] = 0.0;
        P.s[i] = 0.0;
        P.z[i] = 0.0;
        P.x[i] = 0.0;
    }
    if (P.inject_fault && bidx == nblk - 1) {
        if (nblk == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!group_barrier(P.bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    double ga = 0.0, de = 0.0;
    for (int i = c0 + t; i < c1; i += B) {
        const int len = P.alen[i];
        const double csi = c * __ldcg(sg + i);
        const double ri = __ldcg(P.r + i);
        double acc = ri;
        for (int k = 0; k < len; ++k) {
            const size_t q = (size_t)k * ld + i;
            const int j = sdc_idx(P.acol[q], P.n, 14);
            const double a = csi * P.aval[q] * __ldcg(sg + j);
            sval[q] = a;
            acc += a * __ldcg(P.u + j);
        }
        P.w[i] = acc;
        ga += ri * ri;
        de += acc * ri;
        mbuf[0][i] = acc;
    }
    int it = 0, nsum = 0;
    while (true) {
        if (!cg_publish_arrive(ga, de, S, part + buf * nblk, P.bar, nblk, bidx, epoch,
                               P.budget, P.err))
            return;
        const double* mc = mbuf[nsum & 1];
        auto totals = [&]() {
            double g, d;
            xs_group_total(nblk, [&](int k) { return xs_load_cg(part + buf * nblk + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        };
        if (sp0 > 0 && t < 64) totals();
        if (t >= sp0) {
            for (int i = c0 + t - sp0; i < c1; i += B - sp0) {
                const int len = P.alen[i];
                double acc = P.w[i];
                for (int k = 0; k < len; ++k) {
                    const size_t q = (size_t)k * ld + i;
                    acc += __ldcg(sval + q) * __ldcg(mc + sdc_idx(P.acol[q], P.n, 15));
                }
                P.nv[i] = acc;
            }
        }
        if (sp0 == 0 && t < 64) totals();
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        double* mn = mbuf[nsum & 1];
        ga = de = 0.0;
        for (int i = c0 + t; i < c1; i += B) {
            // every operand of the row loaded before the first store
            const double wi = P.w[i], ri = P.r[i], ni = P.nv[i], z0 = P.z[i], s0 = P.s[i],
                         p0 = P.p[i], xi = P.x[i];
            const double zi = ni + beta * z0;
            const double si = wi + beta * s0;
            const double pi = ri + beta * p0;
            P.z[i] = zi;
            P.s[i] = si;
            P.p[i] = pi;
            P.x[i] = xi + alpha * pi;
            const double r2 = ri - alpha * si;
            const double w2 = wi - alpha * zi;
            P.r[i] = r2;
            P.w[i] = w2;
            ga += r2 * r2;
            de += w2 * r2;
            mn[i] = w2;
        }
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x = S x~ on this block's rows; the epilogue gathers neighbours' x after a barrier
    for (int i = c0 + t; i < c1; i += B) P.x[i] = __ldcg(sg + i) * __ldcg(P.x + i);
    if (P.epi_lo < P.epi_hi) {
        if (!group_barrier(P.bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
        for (int i = c0 + t; i < c1; i += B) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += P.aval[(size_t)k * ld + i] * __ldcg(P.x + sdc_idx(P.acol[(size_t)k * ld + i], P.n, 16));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgs(CgParams P) {
    __shared__ CgShared S;
    pcg_group_scaled(P, S, (int)gridDim.x, (int)blockIdx.x);
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcg(CgParams P) {
    __shared__ CgShared S;
    pcg_group(P, S, 0, P.n, (int)gridDim.x, (int)blockIdx.x, P.bar,
              reinterpret_cast<XsRecord*>(P.part), (int)gridDim.x, P.iters_out, P.relres_out);
}

// Batched variant: independent solves of the instances of a batch (disjoint
// diagonal blocks of the system) in one cooperative launch.  Block b works on
// the group tab[b] describes: that instance's compact rows, its own barrier
// counter and partial-sum records, its own iteration count.  Groups never
// wait for each other, so a converged instance's blocks leave early.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcg_batch(CgParams P, const SegBlock* __restrict__ tab,
                                                        unsigned* __restrict__ bars,
                                                        int* __restrict__ seg_iters,
                                                        double* __restrict__ seg_relres) {
    __shared__ CgShared S;
    const SegBlock g = tab[blockIdx.x];
    if (g.nblk == 0) return;   // no group: a planned launch's spare block
    pcg_group(P, S, g.row0, g.row1, g.nblk, (int)blockIdx.x - g.blk0, bars + g.seg,
              reinterpret_cast<XsRecord*>(P.part) + g.blk0, (int)gridDim.x, seg_iters + g.seg,
              seg_relres + g.seg);
}

// Compact boundaries of the batch instances in a sorted active list:
// bounds[s] = first position p with act[p] >= inst_off[s] (lower bound).
__global__ void k_seg_bounds(const int* __restrict__ count, const int* __restrict__ act, int nseg,
                             const int* __restrict__ inst_off, int* __restrict__ bounds) {
    const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (sidx > nseg) return;
    const int n = *count;
    const int key = inst_off[sidx];
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (act[mid] < key) lo = mid + 1; else hi = mid;
    }
    bounds[sidx] = lo;
}

// Shared-memory variant of the same iteration for n <= gridDim.x * L rows:
// block b owns the contiguous rows [b L, b L + L); their r, u, w, p, s, z, n
// and reciprocal diagonal stay in shared memory for the whole solve.  m is
// published to global memory (coalesced, two buffers) for the neighbours'
// gathers and x is accumulated in place in global memory; the matrix is read
// through the read-only path.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcg_smem(CgParams P) {
    extern __shared__ double sm[];
    __shared__ CgShared S;
    const int G = gridDim.x, B = blockDim.x, t = threadIdx.x;
    const int L = P.L, ld = P.ld;
    const int r0 = blockIdx.x * L;
    const int nl = max(0, min(P.n - r0, L));
    const int sp0 = B >= 256 ? 64 : 0;
    // per-row vectors in shared memory (addressed from one base: fewer live registers)
#define SR(l) sm[(l)]
#define SU(l) sm[L + (l)]
#define SW(l) sm[2 * L + (l)]
#define SP(l) sm[3 * L + (l)]
#define SS(l) sm[4 * L + (l)]
#define SZ(l) sm[5 * L + (l)]
#define SN(l) sm[6 * L + (l)]
#define SI(l) sm[7 * L + (l)]
    double* __restrict__ ug = P.u;
    double* __restrict__ xg = P.x;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    XsRecord* const rec = reinterpret_cast<XsRecord*>(P.part);
    unsigned epoch = 0;
    int buf = 0;

    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        SI(l) = id;
        const double r = P.b[i];
        const double u = r * id;
        SR(l) = r;
        SU(l) = u;
        ug[i] = u;
        SP(l) = 0.0;
        SS(l) = 0.0;
        SZ(l) = 0.0;
        xg[i] = 0.0;
    }
    if (P.inject_fault && blockIdx.x == G - 1) {
        if (G == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    double ga = 0.0, de = 0.0;
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const int len = __ldg(alen + i);
        double acc = 0.0;
        for (int k = 0; k < len; ++k)
            acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(ug + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 41));
        const double ri = SR(l), ui = SU(l);
        const double wi = ri + c * acc;
        SW(l) = wi;
        ga += ri * ui;
        de += wi * ui;
        P.m[i] = SI(l) * wi;
    }
    int it = 0, nsum = 0;
    while (true) {
        if (!cg_publish_arrive(ga, de, S, rec + buf * G, P.bar, G, (int)blockIdx.x, epoch,
                               P.budget, P.err))
            return;
        const double* mc = P.m + (nsum & 1) * (size_t)ld;
        auto totals = [&]() {
            double g, d;
            xs_group_total(G, [&](int k) { return xs_load_cg(rec + buf * G + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        };
        if (sp0 > 0 && t < 64) totals();
        if (t >= sp0) {
            for (int l = t - sp0; l < nl; l += B - sp0) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                double acc = 0.0;
                for (int k = 0; k < len; ++k)
                    acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(mc + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 42));
                SN(l) = SW(l) + c * acc;
            }
        }
        if (sp0 == 0 && t < 64) totals();
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        double* mn = P.m + (nsum & 1) * (size_t)ld;
        ga = de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const double id = SI(l);
            const double wi = SW(l), ui = SU(l);
            const double zi = SN(l) + beta * SZ(l);
            const double s_i = wi + beta * SS(l);
            const double pi = ui + beta * SP(l);
            SZ(l) = zi;
            SS(l) = s_i;
            SP(l) = pi;
            xg[i] += alpha * pi;
            const double r2 = SR(l) - alpha * s_i;
            const double w2 = wi - alpha * zi;
            const double u2 = id * r2;
            SR(l) = r2;
            SU(l) = u2;
            SW(l) = w2;
            ga += r2 * u2;
            de += w2 * u2;
            mn[i] = id * w2;
        }
    }
    if (S.state == 2) {
        if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (blockIdx.x == 0 && t == 0) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x is complete and visible: the last grid barrier followed its last update
    if (P.epi_lo < P.epi_hi) {
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = __ldcg(xg + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(xg + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 43));
            cg_couple_row(P, i, xi, acc);
        }
    }
}
#undef SR
#undef SU
#undef SW
#undef SP
#undef SS
#undef SZ
#undef SN
#undef SI

// Symmetrically scaled form of the pipelined shared-memory solve.  Jacobi-PCG
// on A = diag(d) + c K_off is CG on S A S = I + c S K_off S with S = diag(d)^-1/2,
// x = S x~, b~ = S b: the same iterates, the same stopping quantity
// (r~.r~ = r.D^-1 r) and the same energy (x~' S A S x~ = x' A x).  Per
// row-iteration it saves the two preconditioner products (u = D^-1 r, m = D^-1 w)
// and the scaling of the product by c, and keeps six vectors on chip instead of
// eight (4800 rows per block).  The scaled off-diagonals c s_i a_ij s_j are
// written once per solve to P.sval (each block its own rows, after a grid barrier
// that publishes s).  Per row-iteration: len FMAs of the product (started from
// w_i, the unit diagonal), six recurrence FMAs, two dot FMAs.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcg_scaled(CgParams P) {
    extern __shared__ double sm[];
    __shared__ CgShared S;
    const int G = gridDim.x, B = blockDim.x, t = threadIdx.x;
    const int L = P.L, ld = P.ld;
    const int r0 = blockIdx.x * L;
    const int nl = max(0, min(P.n - r0, L));
    const int sp0 = B >= 256 ? 64 : 0;
#define SR(l) sm[(l)]
#define SW(l) sm[L + (l)]
#define SP(l) sm[2 * L + (l)]
#define SS(l) sm[3 * L + (l)]
#define SZ(l) sm[4 * L + (l)]
#define SN(l) sm[5 * L + (l)]
    double* __restrict__ ug = P.u;
    double* __restrict__ xg = P.x;
    double* __restrict__ sg = P.sv;
    double* __restrict__ sval = P.sval;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    XsRecord* const rec = reinterpret_cast<XsRecord*>(P.part);
    unsigned epoch = 0;
    int buf = 0;

    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        double si = 0.0;
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        else si = rsqrt(d);
        sg[i] = si;
        const double r = si * P.b[i];
        SR(l) = r;
        ug[i] = r;
        SP(l) = 0.0;
        SS(l) = 0.0;
        SZ(l) = 0.0;
        xg[i] = 0.0;
    }
    if (P.inject_fault && blockIdx.x == G - 1) {
        if (G == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    // scaled rows of this block, and w = (I + c S K_off S) r~
    double ga = 0.0, de = 0.0;
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const int len = __ldg(alen + i);
        const double csi = c * __ldcg(sg + i);
        const double ri = SR(l);
        double acc = ri;
        for (int k0 = 0; k0 < len; k0 += EllChunk<MAXT>::value) {
            int j[EllChunk<MAXT>::value];
            double av[EllChunk<MAXT>::value], sj[EllChunk<MAXT>::value], uj[EllChunk<MAXT>::value];
#pragma unroll
            for (int k = 0; k < EllChunk<MAXT>::value; ++k) {
                if (k0 + k < len) {
                    const size_t q = (size_t)(k0 + k) * ld + i;
                    j[k] = sdc_idx(__ldg(acol + q), P.n, 44);
                    av[k] = __ldg(aval + q);
                }
            }
#pragma unroll
            for (int k = 0; k < EllChunk<MAXT>::value; ++k) {
                if (k0 + k < len) {
                    sj[k] = __ldcg(sg + j[k]);
                    uj[k] = __ldcg(ug + j[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < EllChunk<MAXT>::value; ++k) {
                if (k0 + k < len) {
                    const double a = csi * av[k] * sj[k];
                    sval[(size_t)(k0 + k) * ld + i] = a;
                    acc += a * uj[k];
                }
            }
        }
        SW(l) = acc;
        ga += ri * ri;
        de += acc * ri;
        P.m[i] = acc;
    }
    int it = 0, nsum = 0;
    while (true) {
        if (!cg_publish_arrive(ga, de, S, rec + buf * G, P.bar, G, (int)blockIdx.x, epoch,
                               P.budget, P.err))
            return;
        const double* mc = P.m + (nsum & 1) * (size_t)ld;
        auto totals = [&]() {
            double g, d;
            xs_group_total(G, [&](int k) { return xs_load_cg(rec + buf * G + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        };
        if (sp0 > 0 && t < 64) totals();
        if (t >= sp0) {
            for (int l = t - sp0; l < nl; l += B - sp0) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                SN(l) = ell_row_dot<EllChunk<MAXT>::value>(SW(l), len, (size_t)i, ld, acol, P.n,
                                    [&](size_t q) { return __ldcg(sval + q); },
                                    [&](int j) { return __ldcg(mc + j); });
            }
        }
        if (sp0 == 0 && t < 64) totals();
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        double* mn = P.m + (nsum & 1) * (size_t)ld;
        ga = de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const double wi = SW(l), ri = SR(l);
            const double zi = SN(l) + beta * SZ(l);
            const double s_i = wi + beta * SS(l);
            const double pi = ri + beta * SP(l);
            SZ(l) = zi;
            SS(l) = s_i;
            SP(l) = pi;
            xg[i] += alpha * pi;
            const double r2 = ri - alpha * s_i;
            const double w2 = wi - alpha * zi;
            SR(l) = r2;
            SW(l) = w2;
            ga += r2 * r2;
            de += w2 * r2;
            mn[i] = w2;
        }
    }
    if (S.state == 2) {
        if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (blockIdx.x == 0 && t == 0) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x = S x~ on this block's rows; the epilogue gathers neighbours' x after a barrier
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        xg[i] = __ldcg(sg + i) * __ldcg(xg + i);
    }
    if (P.epi_lo < P.epi_hi) {
        if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = __ldcg(xg + i);
            const double acc = ell_row_dot<EllChunk<MAXT>::value>(0.0, len, (size_t)i, ld, acol, P.n,
                                           [&](size_t q) { return __ldg(aval + q); },
                                           [&](int j) { return __ldcg(xg + j); });
            cg_couple_row(P, i, xi, acc);
        }
    }
}
#undef SR
#undef SW
#undef SP
#undef SS
#undef SZ
#undef SN

// Thread-block-cluster variant for small active sets (n <= C * L rows, one
// cluster of C CTAs).  The same iteration as k_pcg_smem; m of other CTAs is
// read from their shared memory (distributed shared memory, two buffers),
// the blocks' exact partial sums are exchanged through shared memory, and the
// hardware cluster barrier replaces the global arrival counter, so the
// iteration loop touches no global memory besides the read-only matrix and x.
// Every CTA takes the same decisions (same totals) and leaves only after a
// final cluster barrier, so no CTA reads the shared memory of one that has
// exited.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcg_cluster(CgParams P) {
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    extern __shared__ double sm[];
    __shared__ CgShared S;
    __shared__ XsRecord crec[2];
    __shared__ double* mr[2][16];
    __shared__ XsRecord* pr[16];
    const int B = blockDim.x, t = threadIdx.x;
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int L = P.L, ld = P.ld;
    const int r0 = rank * L;
    const int nl = max(0, min(P.n - r0, L));
    const int sp0 = B >= 256 ? 64 : 0;
    double* __restrict__ sr = sm;
    double* __restrict__ su = sm + L;
    double* __restrict__ sw = sm + 2 * L;
    double* __restrict__ sp = sm + 3 * L;
    double* __restrict__ ss = sm + 4 * L;
    double* __restrict__ sz = sm + 5 * L;
    double* __restrict__ sn = sm + 6 * L;
    double* __restrict__ si = sm + 7 * L;
    double* const smb[2] = {sm + 8 * L, sm + 9 * L};
    double* __restrict__ xg = P.x;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    if (t < C) {
        mr[0][t] = cl.map_shared_rank(smb[0], t);
        mr[1][t] = cl.map_shared_rank(smb[1], t);
        pr[t] = cl.map_shared_rank(crec, t);
    }
    // the initial product A u gathers u through the second buffer
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        si[l] = id;
        const double r = P.b[i];
        const double u = r * id;
        sr[l] = r;
        su[l] = u;
        smb[1][l] = u;
        sp[l] = 0.0;
        ss[l] = 0.0;
        sz[l] = 0.0;
        xg[i] = 0.0;
    }
    cl.sync();
    double ga = 0.0, de = 0.0;
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const int len = __ldg(alen + i);
        const double acc = ell_row_dot<EllChunk<MAXT>::value>(0.0, len, (size_t)i, ld, acol, P.n,
                                       [&](size_t q) { return __ldg(aval + q); },
                                       [&](int j) {
                                           const int owner = j / L;
                                           return mr[1][owner][j - owner * L];
                                       });
        const double ri = sr[l], ui = su[l];
        const double wi = ri + c * acc;
        sw[l] = wi;
        ga += ri * ui;
        de += wi * ui;
        smb[0][l] = si[l] * wi;
    }
    int it = 0, nsum = 0, buf = 0;
    while (true) {
        {
            int fa, fb;
            __int128 qa, qb;
            xs_block_sum2(ga, de, S.xs, fa, fb, qa, qb);
            if (t == 0) xs_store(&crec[buf], fa, fb, qa, qb);
        }
        cl.sync();   // m and the partial sums of every CTA are visible
        const int cb = nsum & 1;
        auto totals = [&]() {
            double g, d;
            xs_group_total(C, [&](int k) { return pr[k][buf]; }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        };
        if (sp0 > 0 && t < 64) totals();
        if (t >= sp0) {
            for (int l = t - sp0; l < nl; l += B - sp0) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                const double acc = ell_row_dot<EllChunk<MAXT>::value>(0.0, len, (size_t)i, ld, acol, P.n,
                                               [&](size_t q) { return __ldg(aval + q); },
                                               [&](int j) {
                                                   const int owner = j / L;
                                                   return mr[cb][owner][j - owner * L];
                                               });
                sn[l] = sw[l] + c * acc;
            }
        }
        if (sp0 == 0 && t < 64) totals();
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (rank == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        double* mn = smb[cb ^ 1];
        ga = de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const double id = si[l];
            const double wi = sw[l], ui = su[l];
            const double zi = sn[l] + beta * sz[l];
            const double s_i = wi + beta * ss[l];
            const double pi = ui + beta * sp[l];
            sz[l] = zi;
            ss[l] = s_i;
            sp[l] = pi;
            xg[i] += alpha * pi;
            const double r2 = sr[l] - alpha * s_i;
            const double w2 = wi - alpha * zi;
            const double u2 = id * r2;
            sr[l] = r2;
            su[l] = u2;
            sw[l] = w2;
            ga += r2 * u2;
            de += w2 * u2;
            mn[l] = id * w2;
        }
    }
    if (S.state == 2) {
        if (rank == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
    } else {
        if (rank == 0 && t == 0) {
            *P.iters_out = it;
            *P.relres_out = cg_relres(S);
            if (P.energy_out) *P.energy_out = S.energy;
        }
        if (P.epi_lo < P.epi_hi) {
            // every CTA's x is final: its last update preceded the last cluster barrier
            for (int l = t; l < nl; l += B) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                const double xi = __ldcg(xg + i);
                const double acc = ell_row_dot<EllChunk<MAXT>::value>(0.0, len, (size_t)i, ld, acol, P.n,
                                               [&](size_t q) { return __ldg(aval + q); },
                                               [&](int j) { return __ldcg(xg + j); });
                cg_couple_row(P, i, xi, acc);
            }
        }
    }
    cl.sync();   // nobody leaves while another CTA may still read its shared memory
}

// ---- classical arrangement (Chronopoulos and Gear, 1989) ----------------------
// The same Jacobi-PCG with two synchronisation points per iteration and no
// pipelining: u = D^-1 r is published, a grid barrier, then w = A u and the
// two dot products r.u, w.u summed in one grid reduction, after which
// s = w + beta s and p = u + beta p give the update.  Its recurrences carry
// fewer vectors than the pipelined form, so its rounding stays close to that
// of textbook CG over long, ill-conditioned solves (cell-by-cell systems).
__device__ __forceinline__ void pcgc_group(const CgParams& P, CgShared& S, int row0, int row1,
                                           int nblk, int bidx, unsigned* bar, XsRecord* part,
                                           int pstride, int* iters_out, double* relres_out) {
    const int t = threadIdx.x;
    const int stride = nblk * blockDim.x;
    const int i0 = row0 + bidx * blockDim.x + t;
    const bool lead = (bidx == 0 && t == 0);
    const int ld = P.ld;
    const double c = P.c;
    unsigned epoch = 0;
    int buf = 0;

    for (int i = i0; i < row1; i += stride) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        P.idA[i] = id;
        const double r = P.b[i];
        P.r[i] = r;
        P.u[i] = r * id;
        P.p[i] = 0.0;
        P.s[i] = 0.0;
        P.x[i] = 0.0;
    }
    if (P.inject_fault && bidx == nblk - 1) {
        // leave without arriving: every other block's bounded wait runs out
        if (nblk == 1 && threadIdx.x == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    int it = 0, nsum = 0;
    while (true) {
        // phase 2: w = A u, r.u, w.u
        double ga = 0.0, de = 0.0;
        for (int i = i0; i < row1; i += stride) {
            const int len = P.alen[i];
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.u + sdc_idx(P.acol[(size_t)t * ld + i], P.n, 17));
            const double ri = P.r[i];
            const double ui = P.u[i];
            const double wi = ri + c * acc;
            P.w[i] = wi;
            ga += ri * ui;
            de += wi * ui;
        }
        if (!cg_publish_arrive(ga, de, S, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                               P.err))
            return;
        if (t < 64) {
            double g, d;
            xs_group_total(nblk, [&](int k) { return xs_load_cg(part + buf * pstride + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        }
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        // phase 1: p, s, x, r, u
        const double alpha = S.alpha, beta = S.beta;
        for (int i = i0; i < row1; i += stride) {
            // every operand of the row loaded before the first store
            const double ui = P.u[i], p0 = P.p[i], wi = P.w[i], s0 = P.s[i], xi = P.x[i],
                         r0 = P.r[i], id = P.idA[i];
            const double pi = ui + beta * p0;
            const double si = wi + beta * s0;
            const double r = r0 - alpha * si;
            P.p[i] = pi;
            P.s[i] = si;
            P.x[i] = xi + alpha * pi;
            P.r[i] = r;
            P.u[i] = r * id;
        }
        if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *iters_out = it;
        *relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x is complete in every block of the group: the last group sum followed its update.
    if (P.epi_lo < P.epi_hi) {
        for (int i = i0; i < row1; i += stride) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.x + sdc_idx(P.acol[(size_t)t * ld + i], P.n, 18));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

// The symmetrically scaled form of pcgc_group (see k_pcg_scaled): classical
// arrangement of CG on I + c S K_off S, S = diag^-1/2, vectors in global memory.
// Per row-iteration z-bar + 6 FP64 operations instead of z-bar + 8 (no u = D^-1 r,
// no scaling of the product by c).  Each thread owns the same rows in every loop,
// so the scaled values it writes once per solve are read back by itself.
__device__ __forceinline__ void pcgc_group_scaled(const CgParams& P, CgShared& S, int row0,
                                                  int row1, int nblk, int bidx, unsigned* bar,
                                                  XsRecord* part, int pstride, int* iters_out,
                                                  double* relres_out) {
    const int t = threadIdx.x;
    const int n = row1;
    const int stride = nblk * blockDim.x;
    const int i0 = row0 + bidx * blockDim.x + t;
    const bool lead = (bidx == 0 && t == 0);
    const int ld = P.ld;
    const double c = P.c;
    double* __restrict__ sg = P.sv;
    double* __restrict__ sval = P.sval;
    unsigned epoch = 0;
    int buf = 0;

    for (int i = i0; i < n; i += stride) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        double si = 0.0;
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        else si = rsqrt(d);
        sg[i] = si;
        P.r[i] = si * P.b[i];
        P.p[i] = 0.0;
        P.s[i] = 0.0;
        P.x[i] = 0.0;
    }
    if (P.inject_fault && bidx == nblk - 1) {
        if (nblk == 1 && threadIdx.x == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    for (int i = i0; i < n; i += stride) {
        const int len = P.alen[i];
        const double csi = c * __ldcg(sg + i);
        for (int k = 0; k < len; ++k) {
            const size_t q = (size_t)k * ld + i;
            sval[q] = csi * P.aval[q] * __ldcg(sg + sdc_idx(P.acol[q], P.n, 19));
        }
    }
    int it = 0, nsum = 0;
    while (true) {
        // w = (I + c S K_off S) r, r.r, w.r
        double ga = 0.0, de = 0.0;
        for (int i = i0; i < n; i += stride) {
            const int len = P.alen[i];
            const double ri = __ldcg(P.r + i);
            double acc = ri;
            for (int k = 0; k < len; ++k) {
                const size_t q = (size_t)k * ld + i;
                acc += sval[q] * __ldcg(P.r + sdc_idx(P.acol[q], P.n, 20));
            }
            P.w[i] = acc;
            ga += ri * ri;
            de += acc * ri;
        }
        if (!cg_publish_arrive(ga, de, S, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                               P.err))
            return;
        if (t < 64) {
            double g, d;
            xs_group_total(nblk, [&](int k) { return xs_load_cg(part + buf * pstride + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        }
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        for (int i = i0; i < n; i += stride) {
            // every operand of the row loaded before the first store
            const double ri = P.r[i], p0 = P.p[i], wi = P.w[i], s0 = P.s[i], xi = P.x[i];
            const double pi = ri + beta * p0;
            const double si = wi + beta * s0;
            P.p[i] = pi;
            P.s[i] = si;
            P.x[i] = xi + alpha * pi;
            P.r[i] = ri - alpha * si;
        }
        if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *iters_out = it;
        *relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    for (int i = i0; i < n; i += stride) P.x[i] = __ldcg(sg + i) * __ldcg(P.x + i);
    if (P.epi_lo < P.epi_hi) {
        if (!group_barrier(bar, nblk, epoch, P.budget, P.err, &S.ok)) return;
        for (int i = i0; i < n; i += stride) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += P.aval[(size_t)k * ld + i] * __ldcg(P.x + sdc_idx(P.acol[(size_t)k * ld + i], P.n, 21));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgcs(CgParams P) {
    __shared__ CgShared S;
    pcgc_group_scaled(P, S, 0, P.n, (int)gridDim.x, (int)blockIdx.x, P.bar,
                      reinterpret_cast<XsRecord*>(P.part), (int)gridDim.x, P.iters_out,
                      P.relres_out);
}

// Batched form of the scaled classical arrangement (one group of blocks per instance).
// ---- two-level preconditioner (cell-by-cell node solves, Sec. 6) ------------------
// The classical scaled arrangement of pcgc_group_scaled with the preconditioned
// residual u = r + Y E^-1 t, t = Y' r, in place of u = r: in the scaled variables
// x = S x~ the block indicators Z become Y = S^-1 Z (Y_i = sqrt(d_i) on the rows of its
// block) and D^-1 becomes the identity.  The compact rows, sorted by block (crow), run in
// tiles of kCoarseTile positions, tile j on CTA j mod G and position j kCoarseTile + t on
// thread t, so that the grid sweeps one window of the vectors at a time (the row order of
// the Jacobi kernels); each tile is cut at the block boundaries into pieces.
// t is carried by the recurrences of the CG vectors it is a linear image of:
//     Y' s <- Y' w + beta Y' s,   t <- t - alpha Y' s,
// so an iteration needs Y' w only, taken per piece in the product and published by
// the grid sum of the dot products.  Per iteration: the product, the dot products and
// the pieces' Y' w (one grid sum); in every CTA the two recurrences over the blocks
// with active rows (the same arithmetic in the same order in every CTA), then
// y = E^-1 t for the blocks of its pieces (a warp per piece); the update of p, s, x,
// r and u = r + Y y on its rows (one grid barrier, publishing u).  t starts as Y' r
// of the initial residual.  Piece sums are exact: each warp sums its rows of a piece
// in 128-bit fixed point, and the warps' records of a piece are added as integers.
// So are the rows of E^-1 t.
struct CoarseParams {
    int q;
    int qn;                // blocks with active rows
    int pmax;              // most pieces of one CTA
    int ptot;              // pieces of the sweep
    int ntiles;            // tiles of the sweep
    int tmax;              // most tiles of one CTA
    int stage;             // 1: the CTA's rows of crow are staged in shared memory
    const int* crow;
    const int* tp;         // [ntiles + 1] pieces of each tile
    const int* piece;      // [3 ptot]: block, first and end position in crow (position order)
    const int* blk_ptr;    // [q + 1] pieces of each block
    const int* nzb;        // [qn] the blocks with active rows, ascending
    const double* Einv;
    double* tpiece;        // [ptot] sums of each piece
};

// a warp's exact partial sum of one piece (shared memory)
struct __align__(16) XsPieceRec {
    __int128 q;
    int f;
    int tag;               // the piece it belongs to; -1: never written
    int pad[2];
};

// dynamic shared memory of k_pcgcs_coarse: records (piece l of tile m, warp w at
// l + 32 m + w), y, the staged piece sums, own pieces, their global ids, first piece of
// each own tile, blocks with active rows and their first pieces, and (stage) the rows
// of the own tiles
inline size_t coarse_smem_bytes(int pmax, int qn, int ptot, int tmax, bool stage) {
    return (size_t)(pmax + 32 * tmax) * sizeof(XsPieceRec) + (size_t)pmax * 8 +
           (size_t)ptot * 8 + (size_t)pmax * 16 + (size_t)(tmax + 1) * 4 +
           (size_t)(2 * qn + 1) * 4 + (stage ? (size_t)tmax * kCoarseTile * 4 : 0);
}
constexpr size_t kCoarseSmemMax = 200 * 1024;   // dynamic shared memory budget of the launch

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgcs_coarse(CgParams P, CoarseParams C) {
    static_assert(MAXT == kCoarseTile, "one position of a tile per thread");
    __shared__ CgShared S;
    __shared__ double tr[kMaxCoarseBlocks];   // t = Y' r of every block with active rows
    __shared__ double ts[kMaxCoarseBlocks];   // Y' s
    extern __shared__ __align__(16) unsigned char dyn[];
    const int t = threadIdx.x, B = blockDim.x, G = gridDim.x, bidx = blockIdx.x;
    const int lane = t & 31, wid = t >> 5, nw = B >> 5;
    const bool lead = bidx == 0 && t == 0;
    const int ld = P.ld, n = P.n, q = C.q, qn = C.qn;
    const double c = P.c;
    double* __restrict__ sg = P.sv;     // diag^-1/2
    double* __restrict__ yv = P.idA;    // diag^1/2: the block indicators in scaled variables
    double* __restrict__ sval = P.sval;
    XsRecord* const rec = reinterpret_cast<XsRecord*>(P.part);
    const int ntl = C.ntiles > bidx ? (C.ntiles - bidx + G - 1) / G : 0;   // own tiles
    XsPieceRec* const recs = reinterpret_cast<XsPieceRec*>(dyn);   // [pmax + 32 tmax]
    double* const ysh = reinterpret_cast<double*>(recs + C.pmax + 32 * C.tmax);   // [pmax]
    double* const stp = ysh + C.pmax;                                  // [ptot]
    int* const spc = reinterpret_cast<int*>(stp + C.ptot);             // [3 pmax] own pieces
    int* const sid = spc + 3 * C.pmax;                                 // [pmax] their ids
    int* const stile = sid + C.pmax;                                   // [tmax + 1]
    int* const snz = stile + C.tmax + 1;                               // [qn]
    int* const sbp = snz + qn;                                         // [qn + 1]
    int* const srow = sbp + qn + 1;                    // [tmax kCoarseTile] (stage) own rows
    if (t == 0) {
        int np = 0;
        for (int m = 0; m < ntl; ++m) {
            const int j = bidx + m * G;
            stile[m] = np;
            np += C.tp[j + 1] - C.tp[j];
        }
        stile[ntl] = np;
    }
    for (int m = t; m < qn; m += B) {
        const int a = sdc_idx(C.nzb[m], q, 73);
        snz[m] = a;
        sbp[m] = C.blk_ptr[a];
    }
    if (t == 0) sbp[qn] = C.blk_ptr[q];
    for (int j = t; j < C.pmax + 32 * C.tmax; j += B) recs[j].tag = -1;
    if (C.stage)
        for (int m = 0; m < ntl; ++m) {
            const int k = (bidx + m * G) * kCoarseTile + t;
            srow[m * kCoarseTile + t] = k < n ? sdc_idx(C.crow[k], n, 70) : 0;
        }
    __syncthreads();
    const int np = stile[ntl];
    for (int m = 0; m < ntl; ++m) {
        const int e0 = C.tp[bidx + m * G], l0 = stile[m], cnt = stile[m + 1] - l0;
        for (int u = t; u < cnt; u += B) {
            const int e = sdc_idx(e0 + u, C.ptot, 74);
            sid[l0 + u] = e;
            spc[3 * (l0 + u)] = C.piece[3 * e];
            spc[3 * (l0 + u) + 1] = C.piece[3 * e + 1];
            spc[3 * (l0 + u) + 2] = C.piece[3 * e + 2];
        }
    }
    __syncthreads();
    unsigned epoch = 0;
    int buf = 0;
    // compact row at position k of own tile m (thread t: k = tile start + t)
    auto row_at = [&](int m, int k) {
        return C.stage ? srow[m * kCoarseTile + t] : sdc_idx(C.crow[k], n, 70);
    };
    // f(l, i) over this thread's rows: own piece l, compact row i
    auto for_rows = [&](auto&& f) {
        int l = 0;
        for (int m = 0; m < ntl; ++m) {
            const int k = (bidx + m * G) * kCoarseTile + t;
            if (k >= n) break;
            while (spc[3 * l + 2] <= k) ++l;
            f(l, row_at(m, k));
        }
    };
    // sum of g(i) = (a, b) -> a b over each own piece, exactly, into tpiece
    auto piece_sums = [&](auto&& g) {
        for (int m = 0; m < ntl; ++m) {
            const int j = bidx + m * G;
            const int base = j * kCoarseTile + 32 * wid, end = min(n, (j + 1) * kCoarseTile);
            if (base >= end) continue;           // no rows of this warp in the tile
            int l = stile[m];
            while (spc[3 * l + 2] <= base) ++l;  // the piece holding the warp's first row
            int pend = spc[3 * l + 2];
            const int k = base + lane;
            double v = 0.0;
            if (k < end) {
                const double2 ab = g(row_at(m, k));
                v = ab.x * ab.y;
            }
            bool used = k >= end;
            while (true) {
                double part = 0.0;
                if (!used && k < pend) {
                    part = v;
                    used = true;
                }
                const int F = __reduce_max_sync(0xffffffffu, xs_field(part));
                const __int128 qv = xs_warp_sum(xs_fixed(part, F));
                if (lane == 0) {
                    XsPieceRec& R = recs[l + 32 * m + wid];
                    R.q = qv;
                    R.f = F;
                    R.tag = l;
                }
                if (__all_sync(0xffffffffu, used)) break;
                ++l;
                pend = spc[3 * l + 2];
            }
        }
        __syncthreads();
        for (int l = wid; l < np; l += nw) {
            const int m = (spc[3 * l + 1] / kCoarseTile - bidx) / G;
            const XsPieceRec R = recs[l + 32 * m + lane];
            const bool on = lane < nw && R.tag == l;
            const int f = on ? R.f : 1;
            const int F = __reduce_max_sync(0xffffffffu, f);
            const int d = F - f;
            __int128 qv = 0;
            if (on) qv = d >= 127 ? (R.q < 0 ? (__int128)-1 : (__int128)0) : xs_sar(R.q, d);
            qv = xs_warp_sum(qv);
            if (lane == 0) C.tpiece[sid[l]] = xs_to_double(qv, F);
        }
    };
    // the blocks' totals of the published piece sums; first: t = total, Y's = 0,
    // else the recurrences
    auto coarse_t = [&](bool first, double alpha, double beta) {
        const int ptot = sbp[qn];
        for (int e = t; e < ptot; e += B) stp[e] = __ldcg(C.tpiece + e);
        __syncthreads();
        for (int m = t; m < qn; m += B) {
            const int a = snz[m];
            double tw = 0.0;
            for (int e = sbp[m]; e < sbp[m + 1]; ++e) tw += stp[e];
            if (first) {
                tr[a] = tw;
                ts[a] = 0.0;
            } else {
                const double sa = tw + beta * ts[a];
                ts[a] = sa;
                tr[a] -= alpha * sa;
            }
        }
        __syncthreads();
    };
    // y = E^-1 t on the blocks of this CTA's pieces, a warp per piece (t vanishes
    // outside the blocks with active rows)
    auto coarse_y = [&]() {
        for (int l = wid; l < np; l += nw) {
            const double* ra = C.Einv + (size_t)spc[3 * l] * q;
            double pa = 0.0;
            for (int m = lane; m < qn; m += 32) {
                const int j = snz[m];
                pa += __ldg(ra + j) * tr[j];
            }
            const int F = __reduce_max_sync(0xffffffffu, xs_field(pa));
            const __int128 qv = xs_warp_sum(xs_fixed(pa, F));
            if (lane == 0) ysh[l] = xs_to_double(qv, F);
        }
        __syncthreads();
    };
    for_rows([&](int, int i) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        double si = 0.0;
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        else si = rsqrt(d);
        sg[i] = si;
        yv[i] = d * si;
        P.r[i] = si * P.b[i];
        P.p[i] = 0.0;
        P.s[i] = 0.0;
        P.x[i] = 0.0;
    });
    if (!group_barrier(P.bar, G, epoch, P.budget, P.err, &S.ok)) return;
    for_rows([&](int, int i) {
        const int len = P.alen[i];
        const double csi = c * sg[i];
        for (int k = 0; k < len; ++k) {
            const size_t qq = (size_t)k * ld + i;
            sval[qq] = csi * P.aval[qq] * __ldcg(sg + sdc_idx(P.acol[qq], n, 71));
        }
    });
    // t = Y' r, y, u = r + Y y
    piece_sums([&](int i) { return make_double2(yv[i], P.r[i]); });
    if (!group_barrier(P.bar, G, epoch, P.budget, P.err, &S.ok)) return;
    coarse_t(true, 0.0, 0.0);
    coarse_y();
    for_rows([&](int l, int i) { P.u[i] = P.r[i] + yv[i] * ysh[l]; });
    if (!group_barrier(P.bar, G, epoch, P.budget, P.err, &S.ok)) return;
    int it = 0, nsum = 0;
    while (true) {
        // w = (I + c S K_off S) u, r.u, w.u, and Y' w per piece
        double ga = 0.0, de = 0.0;
        piece_sums([&](int i) {
            // every operand of the row loaded before the first store (the vectors may
            // alias as far as the compiler knows)
            const int len = P.alen[i];
            const double ui = __ldcg(P.u + i), ri = P.r[i], yi = yv[i];
            double acc = ui;
            for (int k = 0; k < len; ++k) {
                const size_t qq = (size_t)k * ld + i;
                acc += sval[qq] * __ldcg(P.u + sdc_idx(P.acol[qq], n, 72));
            }
            P.w[i] = acc;
            ga += ri * ui;
            de += acc * ui;
            return make_double2(yi, acc);
        });
        if (!cg_publish_arrive(ga, de, S, rec + buf * G, P.bar, G, bidx, epoch, P.budget, P.err))
            return;
        if (t < 64) {
            double g, d;
            xs_group_total(G, [&](int k) { return xs_load_cg(rec + buf * G + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        }
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        coarse_t(false, alpha, beta);
        coarse_y();
        for_rows([&](int l, int i) {
            const double ui = P.u[i], p0 = P.p[i], wi = P.w[i], s0 = P.s[i], xi = P.x[i],
                         r0 = P.r[i], yi = yv[i];
            const double pi = ui + beta * p0;
            const double si = wi + beta * s0;
            const double ri = r0 - alpha * si;
            P.p[i] = pi;
            P.s[i] = si;
            P.x[i] = xi + alpha * pi;
            P.r[i] = ri;
            P.u[i] = ri + yi * ysh[l];
        });
        if (!group_barrier(P.bar, G, epoch, P.budget, P.err, &S.ok)) return;
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    for_rows([&](int, int i) { P.x[i] = sg[i] * P.x[i]; });
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgcs_batch(CgParams P, const SegBlock* __restrict__ tab,
                                                          unsigned* __restrict__ bars,
                                                          int* __restrict__ seg_iters,
                                                          double* __restrict__ seg_relres) {
    __shared__ CgShared S;
    const SegBlock g = tab[blockIdx.x];
    if (g.nblk == 0) return;   // no group: a planned launch's spare block
    pcgc_group_scaled(P, S, g.row0, g.row1, g.nblk, (int)blockIdx.x - g.blk0, bars + g.seg,
                      reinterpret_cast<XsRecord*>(P.part) + g.blk0, (int)gridDim.x,
                      seg_iters + g.seg, seg_relres + g.seg);
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgc(CgParams P) {
    __shared__ CgShared S;
    pcgc_group(P, S, 0, P.n, (int)gridDim.x, (int)blockIdx.x, P.bar,
               reinterpret_cast<XsRecord*>(P.part), (int)gridDim.x, P.iters_out, P.relres_out);
}

// Batched form of the classical arrangement (one group of blocks per instance).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgc_batch(CgParams P, const SegBlock* __restrict__ tab,
                                                         unsigned* __restrict__ bars,
                                                         int* __restrict__ seg_iters,
                                                         double* __restrict__ seg_relres) {
    __shared__ CgShared S;
    const SegBlock g = tab[blockIdx.x];
    if (g.nblk == 0) return;   // no group: a planned launch's spare block
    pcgc_group(P, S, g.row0, g.row1, g.nblk, (int)blockIdx.x - g.blk0, bars + g.seg,
               reinterpret_cast<XsRecord*>(P.part) + g.blk0, (int)gridDim.x, seg_iters + g.seg,
               seg_relres + g.seg);
}

// Shared-memory form of the classical arrangement (rows as in k_pcg_smem;
// r, u, p, s, w and the reciprocal diagonal on chip, u published).
// Shared-memory form of pcgc_group_scaled: rows as in k_pcgc_smem, r, p, s, w on
// chip (four vectors), r published for the neighbours' products.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgc_scaled(CgParams P) {
    extern __shared__ double sm[];
    __shared__ CgShared S;
    const int G = gridDim.x, B = blockDim.x, t = threadIdx.x;
    const int L = P.L, ld = P.ld;
    const int r0 = blockIdx.x * L;
    const int nl = max(0, min(P.n - r0, L));
    double* __restrict__ sr = sm;
    double* __restrict__ sp = sm + L;
    double* __restrict__ ss = sm + 2 * L;
    double* __restrict__ sw = sm + 3 * L;
    double* __restrict__ ug = P.u;
    double* __restrict__ xg = P.x;
    double* __restrict__ sg = P.sv;
    double* __restrict__ sval = P.sval;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    unsigned epoch = 0;
    int buf = 0;

    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        double si = 0.0;
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        else si = rsqrt(d);
        sg[i] = si;
        const double r = si * P.b[i];
        sr[l] = r;
        ug[i] = r;
        sp[l] = 0.0;
        ss[l] = 0.0;
        xg[i] = 0.0;
    }
    if (P.inject_fault && blockIdx.x == G - 1) {
        if (G == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    // scaled rows: written and read back by the same thread (same row mapping in every loop)
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const int len = __ldg(alen + i);
        const double csi = c * __ldcg(sg + i);
        for (int k = 0; k < len; ++k) {
            const size_t q = (size_t)k * ld + i;
            sval[q] = csi * __ldg(aval + q) * __ldcg(sg + sdc_idx(__ldg(acol + q), P.n, 45));
        }
    }
    XsRecord* const rec = reinterpret_cast<XsRecord*>(P.part);
    int it = 0, nsum = 0;
    while (true) {
        double ga = 0.0, de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double ri = sr[l];
            double acc = ri;
            for (int k = 0; k < len; ++k) {
                const size_t q = (size_t)k * ld + i;
                acc += sval[q] * __ldcg(ug + sdc_idx(__ldg(acol + q), P.n, 46));
            }
            sw[l] = acc;
            ga += ri * ri;
            de += acc * ri;
        }
        if (!cg_publish_arrive(ga, de, S, rec + buf * G, P.bar, G, (int)blockIdx.x, epoch,
                               P.budget, P.err))
            return;
        if (t < 64) {
            double g, d;
            xs_group_total(G, [&](int k) { return xs_load_cg(rec + buf * G + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        }
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        for (int l = t; l < nl; l += B) {
            const double ri = sr[l];
            const double pi = ri + beta * sp[l];
            const double s_i = sw[l] + beta * ss[l];
            sp[l] = pi;
            ss[l] = s_i;
            xg[r0 + l] += alpha * pi;
            const double r = ri - alpha * s_i;
            sr[l] = r;
            ug[r0 + l] = r;
        }
        if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    }
    if (S.state == 2) {
        if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (blockIdx.x == 0 && t == 0) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        xg[i] = __ldcg(sg + i) * __ldcg(xg + i);
    }
    if (P.epi_lo < P.epi_hi) {
        if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = __ldcg(xg + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(xg + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 47));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pcgc_smem(CgParams P) {
    extern __shared__ double sm[];
    __shared__ CgShared S;
    const int G = gridDim.x, B = blockDim.x, t = threadIdx.x;
    const int L = P.L, ld = P.ld;
    const int r0 = blockIdx.x * L;
    const int nl = max(0, min(P.n - r0, L));
    double* __restrict__ sr = sm;
    double* __restrict__ su = sm + L;
    double* __restrict__ sp = sm + 2 * L;
    double* __restrict__ ss = sm + 3 * L;
    double* __restrict__ sw = sm + 4 * L;
    double* __restrict__ si = sm + 5 * L;
    double* __restrict__ ug = P.u;
    double* __restrict__ xg = P.x;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    unsigned epoch = 0;
    int buf = 0;

    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        si[l] = id;
        const double r = P.b[i];
        const double u = r * id;
        sr[l] = r;
        su[l] = u;
        ug[i] = u;
        sp[l] = 0.0;
        ss[l] = 0.0;
        xg[i] = 0.0;
    }
    if (P.inject_fault && blockIdx.x == G - 1) {
        if (G == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    XsRecord* const rec = reinterpret_cast<XsRecord*>(P.part);
    int it = 0, nsum = 0;
    while (true) {
        double ga = 0.0, de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(ug + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 48));
            const double ri = sr[l], ui = su[l];
            const double wi = ri + c * acc;
            sw[l] = wi;
            ga += ri * ui;
            de += wi * ui;
        }
        if (!cg_publish_arrive(ga, de, S, rec + buf * G, P.bar, G, (int)blockIdx.x, epoch,
                               P.budget, P.err))
            return;
        if (t < 64) {
            double g, d;
            xs_group_total(G, [&](int k) { return xs_load_cg(rec + buf * G + k); }, S.xs, g, d);
            if ((t & 31) == 0) cg_scalars(S, t >> 5, nsum, g, d, P.rtol);
        }
        __syncthreads();
        ++nsum;
        buf ^= 1;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        const double alpha = S.alpha, beta = S.beta;
        for (int l = t; l < nl; l += B) {
            const double pi = su[l] + beta * sp[l];
            const double s_i = sw[l] + beta * ss[l];
            sp[l] = pi;
            ss[l] = s_i;
            xg[r0 + l] += alpha * pi;
            const double r = sr[l] - alpha * s_i;
            sr[l] = r;
            const double u = r * si[l];
            su[l] = u;
            ug[r0 + l] = u;
        }
        if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
    }
    if (S.state == 2) {
        if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (blockIdx.x == 0 && t == 0) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
        if (P.energy_out) *P.energy_out = S.energy;
    }
    // x is complete and visible: the last grid sum followed its last update
    if (P.epi_lo < P.epi_hi) {
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = __ldcg(xg + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(xg + sdc_idx(__ldg(acol + (size_t)k * ld + i), P.n, 49));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

template <int M>
__global__ void k_update(int n, const int* __restrict__ act, const double* __restrict__ D, int ld,
                         double* __restrict__ V, double* __restrict__ W,
                         const double* __restrict__ w0, double dt, Ionic ion, Coll co,
                         double tol_drop, int w_frozen, int* __restrict__ flag,
                         int* __restrict__ blockcnt, double* __restrict__ blockmarg,
                         int* __restrict__ err, const double* __restrict__ tol_drop_dev,
                         const int* __restrict__ n_dev, int N) {
    __shared__ int wc[32];
    if (tol_drop_dev) tol_drop = *tol_drop_dev;
    if (n_dev) n = *n_dev;
    __shared__ double wmg[32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    double margin = DBL_MAX;
    if (p < n) {
        const int g = act ? sdc_idx(act[p], N, 61) : p;
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
            // two divisions per row instead of 2 M (FP64 division is a long sequence on this
            // part): the M reciprocals 1 / (v + mu2), then the M reciprocals of the denominators
            double wm[M], gR[M], dR[M], e[M], xs[M], inv[M];
            const double wz = w0[g];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                wm[m] = W[(size_t)g * M + m];
                xs[m] = vm[m] + ion.mu2;
                if (!(xs[m] > 0.0)) raise_error(err, SDC_E_DOMAIN);
            }
            batch_reciprocal<M>(xs, inv);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                ap_R_dRdw_inv(ion, vm[m], wm[m], inv[m], gR[m], dR[m]);
                xs[m] = 1.0 - dt * co.Qh[m * kMaxM + m] * dR[m];
                if (!(xs[m] > 0.0)) raise_error(err, SDC_E_DOMAIN);
            }
            batch_reciprocal<M>(xs, inv);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                double q = 0.0;
#pragma unroll
                for (int j = 0; j < M; ++j) q += co.Q[m * kMaxM + j] * gR[j];
                double acc = wz + dt * q - wm[m];
#pragma unroll
                for (int j = 0; j < m; ++j) acc += dt * co.Qh[m * kMaxM + j] * dR[j] * e[j];
                e[m] = acc * inv[m];
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
                          int* __restrict__ map, const int* __restrict__ n_dev) {
    __shared__ int woff[32];
    if (n_dev) n = *n_dev;
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
                          int new_ld, unsigned long long* nnz, const int* __restrict__ n_dev) {
    if (n_dev) n_old = *n_dev;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (p < n_old) {
        const int qrow = map[p];
        if (qrow >= 0) {
            const int len = olen[p];
            for (int t = 0; t < len; ++t) {
                const int jn = map[sdc_idx(ocol[(size_t)t * old_ld + p], n_old, 62)];
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

void launch_perm_gather(int N, const int* perm, const double* src, double* dst, cudaStream_t s) {
    if (N > 0) k_perm_gather<<<nblk(N, 256), 256, 0, s>>>(N, perm, src, dst);
}
void launch_perm_scatter(int N, const int* perm, const double* src, double* dst, cudaStream_t s) {
    if (N > 0) k_perm_scatter<<<nblk(N, 256), 256, 0, s>>>(N, perm, src, dst);
}
void launch_nodes_out_perm(int N, int M, const int* perm, const double* X, double* out,
                           cudaStream_t s) {
    if (N > 0) k_nodes_out_perm<<<nblk(N, 256), 256, 0, s>>>(N, M, perm, X, out);
}

void launch_nodes_out(int N, int M, const double* V, const double* W, double* Vo, double* Wo,
                      cudaStream_t s) {
    k_nodes_out<<<nblk(N, 256), 256, 0, s>>>(N, M, V, W, Vo, Wo);
}

void launch_residual(int M, int n, const int* act, const Ell& K, const double* kdiag,
                     const double* mass, const double* stim, double stim_on, const double* V,
                     const double* W, const double* v0, double dt, const Ionic& ion,
                     const Coll& co, int reaction_implicit, StepBuffers& B, cudaStream_t s,
                     const int* n_dev) {
    if (n < 1) return;
    dispatch_M(M, [&](auto mc) {
        constexpr int MM = decltype(mc)::value;
        k_residual<MM><<<nblk(n, 128), 128, 0, s>>>(n, act, K.val, K.col, K.len, K.ld, kdiag, mass,
                                                      stim, stim_on, V, W, v0, dt, ion, co,
                                                      reaction_implicit, B.ld, B.R, B.J, B.mc, B.kdc,
                                                      n_dev, B.N);
    });
}

int launch_pcg_params(CgParams& P, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s);

using PcgKernel = void (*)(CgParams);
using PcgBatchKernel = void (*)(CgParams, const SegBlock*, unsigned*, int*, double*);

// instantiation for a block size: the register budget follows the largest block
PcgKernel pcg_general_kernel(int block) {
    return block > 512 ? k_pcg<1024> : block > 256 ? k_pcg<512> : k_pcg<256>;
}
PcgKernel pcg_smem_kernel(int block) { return block > 512 ? k_pcg_smem<1024> : k_pcg_smem<512>; }
PcgKernel pcgc_scaled_kernel(int block) {
    return block > 512 ? k_pcgc_scaled<1024> : k_pcgc_scaled<512>;
}
PcgKernel pcgcs_general_kernel(int block) {
    return block > 512 ? k_pcgcs<1024> : block > 256 ? k_pcgcs<512> : k_pcgcs<256>;
}
PcgKernel pcgs_general_kernel(int block) {
    return block > 512 ? k_pcgs<1024> : block > 256 ? k_pcgs<512> : k_pcgs<256>;
}
PcgKernel pcg_scaled_kernel(int block) {
    return block > 512 ? k_pcg_scaled<1024> : k_pcg_scaled<512>;
}
PcgKernel pcg_cluster_kernel(int block) {
    return block > 512 ? k_pcg_cluster<1024> : k_pcg_cluster<512>;
}
PcgKernel pcgc_general_kernel(int block) {
    return block > 512 ? k_pcgc<1024> : block > 256 ? k_pcgc<512> : k_pcgc<256>;
}
PcgKernel pcgc_smem_kernel(int block) { return block > 512 ? k_pcgc_smem<1024> : k_pcgc_smem<512>; }
// Batches: the 64-register instantiation whatever the block size, so that
// several blocks share an SM and one cooperative wave holds more instances.
PcgBatchKernel pcg_batch_kernel(int, bool pipelined, bool scaled = false) {
    return pipelined ? k_pcg_batch<1024> : scaled ? k_pcgcs_batch<1024> : k_pcgc_batch<1024>;
}

// opt-in dynamic shared memory of the on-chip variants (set once per instantiation)
void pcg_smem_attrs() {
    static bool done = false;
    if (done) return;
    for (PcgKernel k : {k_pcg_smem<512>, k_pcg_smem<1024>})
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemVectors * kSmemRows * sizeof(double)));
    for (PcgKernel k : {k_pcgc_smem<512>, k_pcgc_smem<1024>})
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemVectorsC * kSmemRowsC * sizeof(double)));
    for (PcgKernel k : {k_pcg_scaled<512>, k_pcg_scaled<1024>})
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemVectorsS * kSmemRowsS * sizeof(double)));
    for (PcgKernel k : {k_pcgc_scaled<512>, k_pcgc_scaled<1024>})
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemVectorsCS * kSmemRowsC * sizeof(double)));
    for (PcgKernel k : {k_pcg_cluster<512>, k_pcg_cluster<1024>}) {
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kClusterVectors * kClusterRows * sizeof(double)));
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    done = true;
}

int pcg_max_blocks(int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_general_kernel(block), block, 0);
    // the other general-vector kernels share the grid limit: take the smallest occupancy
    for (PcgKernel k : {pcgs_general_kernel(block), pcgc_general_kernel(block),
                        pcgcs_general_kernel(block)}) {
        int q = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, block, 0);
        per = std::min(per, q);
    }
    return sms * per;
}

int pcg_cluster_size(int block) {
    pcg_smem_attrs();
    for (int C = 16; C >= 2; C /= 2) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(C);
        lc.blockDim = dim3(block);
        lc.dynamicSmemBytes = (size_t)kClusterVectors * kClusterRows * sizeof(double);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)pcg_cluster_kernel(block), &lc) ==
                cudaSuccess &&
            nclusters >= 1)
            return C;
        cudaGetLastError();
    }
    return 0;
}

int pcg_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// CG vectors of a context's step buffers
void set_cg_vectors(CgParams& P, StepBuffers& B) {
    P.r = B.r;
    P.u = B.u;
    P.w = B.w;
    P.p = B.p;
    P.s = B.s;
    P.z = B.z;
    P.nv = B.nv;
    P.m = B.m;
    P.idA = B.idA;
    P.part = B.part;
}

// buffers of the scaled form, when the context has them and they hold A's width
void set_scaled_buffers(CgParams& P, const Ell& A, StepBuffers& B) {
    const bool fits = B.sv && B.sval && A.width <= B.sval_width && A.ld == B.ld;
    P.sv = fits ? B.sv : nullptr;
    P.sval = fits ? B.sval : nullptr;
}

int launch_pcg(int n, const Ell& A, int m, double dt, const Coll& co, double rtol, int maxit,
               int sweep, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
    CgParams P{};
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
    set_cg_vectors(P, B);
    set_scaled_buffers(P, A, B);
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = &B.sc->cg_iters[sweep * kMaxM + m];
    P.relres_out = &B.sc->cg_relres[sweep * kMaxM + m];
    P.energy_out = &B.sc->cg_energy[sweep * kMaxM + m];
    P.m_node = m;
    P.M = co.M;
    P.epi_lo = m + 1;
    P.epi_hi = co.M;
    P.epi_target_J = 0;
    P.Jall = B.J;
    P.dt = dt;
    P.R = B.R;
    for (int j = 0; j < kMaxM; ++j) P.qh[j] = j < co.M ? co.Qh[j * kMaxM + m] : 0.0;
    P.inject_fault = cfg.inject_fault;
    P.L = 0;
    return launch_pcg_params(P, cfg, B, s);
}

int launch_pcg_coarse(int n, const Ell& A, const PcgRole& role, double rtol, int maxit,
                      const CoarseDev& C, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
    CgParams P{};
    P.n = n;
    P.ld = B.ld;
    P.aval = A.val;
    P.acol = A.col;
    P.alen = A.len;
    P.mc = B.mc;
    P.kdc = B.kdc;
    P.J = role.J;
    P.c = role.c;
    P.b = role.b;
    P.x = role.x;
    set_cg_vectors(P, B);
    set_scaled_buffers(P, A, B);
    if (!P.sv || !P.sval || role.epi_lo < role.epi_hi || C.G < 1 || C.q < 1 || C.qn > C.q ||
        C.ntiles < 1 || C.tmax < 1 || C.pmax < 1 || C.ptot < 1)
        return SDC_E_INVALID;
    if (reinterpret_cast<uintptr_t>(P.part) % 16 != 0 || C.G > B.max_blocks) return SDC_E_INVALID;
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = role.iters_out;
    P.relres_out = role.relres_out;
    P.energy_out = role.energy_out;
    P.M = 1;
    cudaMemsetAsync(&B.sc->bar, 0, sizeof(unsigned), s);
    CoarseParams CP;
    CP.q = C.q;
    CP.qn = C.qn;
    CP.pmax = C.pmax;
    CP.ptot = C.ptot;
    CP.ntiles = C.ntiles;
    CP.tmax = C.tmax;
    CP.stage = coarse_smem_bytes(C.pmax, C.qn, C.ptot, C.tmax, true) <= kCoarseSmemMax;
    CP.crow = C.crow;
    CP.tp = C.tp;
    CP.piece = C.piece;
    CP.blk_ptr = C.blk_ptr;
    CP.nzb = C.nzb;
    CP.Einv = C.Einv;
    CP.tpiece = C.tpiece;
    void* args[] = {&P, &CP};
    const int blk = kCoarseTile;
    const void* k = (const void*)k_pcgcs_coarse<kCoarseTile>;
    const size_t smem = coarse_smem_bytes(C.pmax, C.qn, C.ptot, C.tmax, CP.stage != 0);
    if (smem > kCoarseSmemMax) return SDC_E_INVALID;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return SDC_E_CUDA;
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(C.G), dim3(blk), args, smem, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

int launch_pcg_role(int n, const Ell& A, const PcgRole& role, double dt, int M, double rtol,
                    int maxit, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
    CgParams P{};
    P.n = n;
    P.ld = B.ld;
    P.aval = A.val;
    P.acol = A.col;
    P.alen = A.len;
    P.mc = B.mc;
    P.kdc = B.kdc;
    P.J = role.J;
    P.c = role.c;
    P.b = role.b;
    P.x = role.x;
    set_cg_vectors(P, B);
    set_scaled_buffers(P, A, B);
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = role.iters_out;
    P.relres_out = role.relres_out;
    P.energy_out = role.energy_out;
    P.m_node = 0;
    P.M = M;
    P.epi_lo = role.epi_lo;
    P.epi_hi = role.epi_hi;
    P.epi_target_J = role.epi_target_J;
    P.Jall = role.Jall;
    P.dt = dt;
    P.R = role.R;
    for (int j = 0; j < kMaxM; ++j) P.qh[j] = role.qh[j];
    P.inject_fault = 0;
    P.L = 0;
    PcgConfig c2 = cfg;
    c2.inject_fault = 0;
    return launch_pcg_params(P, c2, B, s);
}

int launch_pcg_params(CgParams& P, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
    const int n = P.n;
    // the exact-sum records are read with 16-byte loads
    if (reinterpret_cast<uintptr_t>(P.part) % 16 != 0) return SDC_E_INVALID;
    cudaMemsetAsync(&B.sc->bar, 0, sizeof(unsigned), s);
    void* args[] = {&P};
    // automatic arrangement: the pipelined form pays off where the vectors live on chip;
    // for the global-vector variant (solves above the on-chip capacity) its extra vector
    // traffic outweighs the saved synchronisation
    const bool on_chip = cfg.variant != 1 && n <= cfg.sms * kSmemRows;
    if (!cfg.pipelined || (cfg.general_classical && !on_chip)) {
        // classical arrangement: shared-memory form when it fits, else global vectors
        if (cfg.variant != 1 && n <= cfg.sms * kSmemRowsC) {
            const int rpb = cfg.rows_per_block > 0 ? cfg.rows_per_block : kSmemRowsDefault;
            int grid = std::max(nblk(n, kSmemRowsC), nblk(n, rpb));
            grid = std::min(grid, cfg.sms);
            if (cfg.max_blocks > 0) grid = std::min(grid, cfg.max_blocks);
            grid = std::max(std::max(grid, nblk(n, kSmemRowsC)), 1);
            P.L = nblk(n, grid);
            const int blk = n >= cfg.big_rows ? 1024 : cfg.smem_block;
            pcg_smem_attrs();
            const bool sc = cfg.scaled && P.sv && P.sval;
            cudaError_t e = cudaLaunchCooperativeKernel(
                (const void*)(sc ? pcgc_scaled_kernel(blk) : pcgc_smem_kernel(blk)), dim3(grid),
                dim3(blk), args,
                (size_t)(sc ? kSmemVectorsCS : kSmemVectorsC) * P.L * sizeof(double), s);
            return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
        }
        int grid = std::min(cfg.max_blocks_general, nblk(n, cfg.block));
        if (grid < 1) grid = 1;
        const PcgKernel kg = cfg.scaled && P.sv && P.sval ? pcgcs_general_kernel(cfg.block)
                                                          : pcgc_general_kernel(cfg.block);
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)kg, dim3(grid), dim3(cfg.block),
                                                    args, 0, s);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    // cluster variant: one cluster of cfg.cluster CTAs for small active sets
    if (cfg.variant != 1 && cfg.cluster > 0 && !cfg.inject_fault && n <= cfg.cluster_rows &&
        n <= cfg.cluster * kClusterRows) {
        pcg_smem_attrs();
        // enough CTAs for the FP64 work, never more rows per CTA than fit
        int C = std::min(cfg.cluster,
                         std::max(nblk(n, cfg.cluster_rows_per_cta), nblk(n, kClusterRows)));
        C = std::max(C, 1);
        P.L = nblk(n, C);
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(C);
        lc.blockDim = dim3(cfg.smem_block);
        lc.dynamicSmemBytes = (size_t)kClusterVectors * P.L * sizeof(double);
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&lc, pcg_cluster_kernel(cfg.smem_block), P);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    // symmetrically scaled shared-memory form: one block per SM at most.  Up to the Jacobi
    // form's capacity only: above it (the 686k-row tissue mesh) 4,500 on-chip rows per block
    // leave too little L1 for the irregular gathers and the global-vector kernel is faster
    // (16.1 against 18.9 ms of PCG per step)
    if (cfg.variant != 1 && cfg.scaled && P.sv && P.sval && n <= cfg.sms * kSmemRows) {
        const int rpb = cfg.rows_per_block > 0 ? cfg.rows_per_block : kSmemRowsDefault;
        int grid = std::max(nblk(n, kSmemRowsS), nblk(n, rpb));
        grid = std::min(grid, cfg.sms);
        if (cfg.max_blocks > 0) grid = std::min(grid, cfg.max_blocks);
        grid = std::max(std::max(grid, nblk(n, kSmemRowsS)), 1);
        P.L = nblk(n, grid);
        const size_t smem = (size_t)kSmemVectorsS * P.L * sizeof(double);
        const int blk = n >= cfg.big_rows ? 1024 : cfg.smem_block;
        pcg_smem_attrs();
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_scaled_kernel(blk),
                                                    dim3(grid), dim3(blk), args, smem, s);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    // shared-memory variant: one block per SM at most, each owning <= kSmemRows rows
    const bool smem_ok = cfg.variant != 1 && n <= cfg.sms * kSmemRows;
    if (smem_ok && cfg.variant != 1) {
        const int rpb = cfg.rows_per_block > 0 ? cfg.rows_per_block : kSmemRowsDefault;
        int grid = std::max(nblk(n, kSmemRows), nblk(n, rpb));
        grid = std::min(grid, cfg.sms);
        if (cfg.max_blocks > 0) grid = std::min(grid, cfg.max_blocks);
        grid = std::max(grid, nblk(n, kSmemRows));
        grid = std::max(grid, 1);
        P.L = nblk(n, grid);
        const size_t smem = (size_t)kSmemVectors * P.L * sizeof(double);
        // the largest systems keep every SM's FP64 pipe busy with 32 warps;
        // smaller ones favour shorter block-level reductions
        const int blk = n >= cfg.big_rows ? 1024 : cfg.smem_block;
        pcg_smem_attrs();
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_smem_kernel(blk), dim3(grid),
                                                    dim3(blk), args, smem, s);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    int grid = std::min(cfg.max_blocks_general, nblk(n, cfg.block));
    if (grid < 1) grid = 1;
    const PcgKernel kg = cfg.scaled && P.sv && P.sval ? pcgs_general_kernel(cfg.block)
                                                      : pcg_general_kernel(cfg.block);
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)kg, dim3(grid), dim3(cfg.block),
                                                args, 0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

int pcg_batch_max_blocks(int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_batch_kernel(block, true), block, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, pcg_batch_kernel(block, false), block, 0);
    int per3 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per3, pcg_batch_kernel(block, false, true), block,
                                                  0);
    per2 = std::min(per2, per3);
    per = std::min(per, per2);
    return sms * per;
}

void launch_seg_bounds(const int* act, const int* count, StepBuffers& B, cudaStream_t s,
                       int* bounds_out) {
    k_seg_bounds<<<nblk(B.nseg + 1, 128), 128, 0, s>>>(count, act, B.nseg, B.inst_off,
                                                        bounds_out ? bounds_out : B.bounds);
}

// Start of a captured batched step: margin, |I_0| = N and the sweep-0 boundaries.
__global__ void k_graph_init(DevScalars* sc, int* nk, int N, const int* __restrict__ inst_off,
                             int* __restrict__ bounds0, int nseg) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        sc->margin = DBL_MAX;
        nk[0] = N;
    }
    for (int i = t; i <= nseg; i += gridDim.x * blockDim.x) bounds0[i] = inst_off[i];
}

void launch_graph_init(StepBuffers& B, cudaStream_t s) {
    k_graph_init<<<1, 256, 0, s>>>(B.sc, B.nk, B.N, B.inst_off, B.bounds_k, B.nseg);
}

// Block plan of a batched solve from the device boundaries (one block).  Every non-empty
// instance gets max(1, ceil(rows / rpb)) blocks; when that exceeds the grid G, each keeps
// one block and the remaining G - (non-empty instances) are shared in proportion to the
// extra blocks it asked for (rounded down), so the total never exceeds G (the host checks
// nseg <= G).  Table entries past the total get nblk = 0.
__global__ void k_batch_plan(int nseg, const int* __restrict__ bounds, int G, int rpb,
                             SegBlock* __restrict__ tab, int* __restrict__ want,
                             int* __restrict__ first) {
    __shared__ int total_s;
    if (threadIdx.x == 0) {
        long long tot = 0, extra = 0;
        int nonempty = 0;
        for (int g = 0; g < nseg; ++g) {
            const int r = bounds[g + 1] - bounds[g];
            const int w = r > 0 ? max(1, (r + rpb - 1) / rpb) : 0;
            want[g] = w;
            nonempty += r > 0;
            tot += w;
            extra += w > 0 ? w - 1 : 0;
        }
        if (tot > G) {
            const long long budget = G - nonempty;
            for (int g = 0; g < nseg; ++g)
                if (want[g] > 0) want[g] = 1 + (int)((long long)(want[g] - 1) * budget / extra);
        }
        int run = 0;
        for (int g = 0; g < nseg; ++g) {
            first[g] = run;
            run += want[g];
        }
        total_s = run;
    }
    __syncthreads();
    const int total = total_s;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        SegBlock e{0, 0, 0, 0, 0};
        if (b < total) {
            // the last instance whose first block is <= b: a non-empty one (an empty
            // instance shares its first block with the next non-empty instance)
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (first[mid] <= b) lo = mid; else hi = mid - 1;
            }
            e = SegBlock{bounds[lo], bounds[lo + 1], first[lo], want[lo], lo};
        }
        tab[b] = e;
    }
}

// Parameters of a batched node solve (the groups come from the block table)
CgParams batch_params(int n, const Ell& A, int m, double dt, const Coll& co, double rtol,
                      int maxit, const PcgConfig& cfg, StepBuffers& B) {
    CgParams P{};
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
    set_cg_vectors(P, B);
    set_scaled_buffers(P, A, B);
    P.bar = nullptr;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = nullptr;
    P.relres_out = nullptr;
    P.energy_out = nullptr;
    P.m_node = m;
    P.M = co.M;
    P.epi_lo = m + 1;
    P.epi_hi = co.M;
    P.epi_target_J = 0;
    P.Jall = B.J;
    P.dt = dt;
    P.R = B.R;
    for (int j = 0; j < kMaxM; ++j) P.qh[j] = j < co.M ? co.Qh[j * kMaxM + m] : 0.0;
    P.inject_fault = 0;
    P.L = 0;
    return P;
}

int launch_pcg_batch(int n, const Ell& A, int m, double dt, const Coll& co, double rtol,
                     int maxit, int sweep, const PcgConfig& cfg, const std::vector<int>& bounds,
                     StepBuffers& B, cudaStream_t s) {
    const int nseg = (int)bounds.size() - 1;
    const int Gmax = cfg.max_blocks_batch;
    // blocks per instance: proportional to its active rows, at least one
    std::vector<int> want(nseg, 0);
    long long total = 0;
    for (int g = 0; g < nseg; ++g) {
        const int r = bounds[g + 1] - bounds[g];
        if (r > 0) want[g] = std::max(1, nblk(r, cfg.batch_rows_per_block));
        total += want[g];
    }
    if (total > Gmax) {
        const double f = (double)Gmax / (double)total;
        for (int g = 0; g < nseg; ++g)
            if (want[g] > 0) want[g] = std::max(1, (int)(want[g] * f));
    }
    CgParams P = batch_params(n, A, m, dt, co, rtol, maxit, cfg, B);
    int* seg_iters = B.seg_iters + (size_t)(sweep * kMaxM + m) * nseg;
    double* seg_relres = B.seg_relres + (size_t)(sweep * kMaxM + m) * nseg;
    cudaMemsetAsync(B.bars, 0, nseg * sizeof(unsigned), s);
    // waves of instances whose blocks fit in one cooperative grid
    std::vector<SegBlock> tab;
    int g = 0;
    while (g < nseg) {
        tab.clear();
        while (g < nseg) {
            if (want[g] == 0) { ++g; continue; }
            if (!tab.empty() && (int)tab.size() + want[g] > Gmax) break;
            const int blk0 = (int)tab.size();
            const int nb = std::min(want[g], Gmax);
            for (int b = 0; b < nb; ++b) tab.push_back({bounds[g], bounds[g + 1], blk0, nb, g});
            ++g;
        }
        if (tab.empty()) break;
        if (cudaMemcpyAsync(B.segtab, tab.data(), tab.size() * sizeof(SegBlock),
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SDC_E_CUDA;
        const SegBlock* dtab = reinterpret_cast<const SegBlock*>(B.segtab);
        void* args[] = {&P, (void*)&dtab, &B.bars, &seg_iters, &seg_relres};
        cudaError_t e = cudaLaunchCooperativeKernel(
            (const void*)pcg_batch_kernel(cfg.batch_block, cfg.batch_pipelined,
                                          cfg.scaled && P.sv && P.sval),
                                                    dim3((int)tab.size()),
                                                    dim3(cfg.batch_block), args, 0, s);
        if (e != cudaSuccess) return SDC_E_CUDA;
    }
    return SDC_OK;
}

int launch_pcg_batch_planned(const Ell& A, int m, double dt, const Coll& co, double rtol,
                             int maxit, int sweep, const PcgConfig& cfg, const int* bounds_dev,
                             bool plan, StepBuffers& B, cudaStream_t s) {
    const int nseg = B.nseg;
    const int G = cfg.max_blocks_batch;
    if (nseg < 1 || nseg > G || G > B.segtab_cap) return SDC_E_INVALID;
    SegBlock* tab = reinterpret_cast<SegBlock*>(B.segtab);
    if (plan)
        k_batch_plan<<<1, 256, 0, s>>>(nseg, bounds_dev, G, cfg.batch_rows_per_block, tab, B.plan,
                                       B.plan + nseg);
    CgParams P = batch_params(B.N, A, m, dt, co, rtol, maxit, cfg, B);
    int* seg_iters = B.seg_iters + (size_t)(sweep * kMaxM + m) * nseg;
    double* seg_relres = B.seg_relres + (size_t)(sweep * kMaxM + m) * nseg;
    cudaMemsetAsync(B.bars, 0, nseg * sizeof(unsigned), s);
    const SegBlock* dtab = tab;
    void* args[] = {&P, (void*)&dtab, &B.bars, &seg_iters, &seg_relres};
    cudaError_t e = cudaLaunchCooperativeKernel(
        (const void*)pcg_batch_kernel(cfg.batch_block, cfg.batch_pipelined,
                                      cfg.scaled && P.sv && P.sval),
        dim3(G), dim3(cfg.batch_block), args, 0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

int launch_pcg_standalone(int n, const Ell& A, const double* kdiag, const double* mass,
                          const double* J, double c, const double* b, double* x, double rtol,
                          int maxit, long long budget, int block, const PcgScratch& w,
                          cudaStream_t s) {
    CgParams P{};
    P.n = n;
    P.ld = A.ld;
    P.aval = A.val;
    P.acol = A.col;
    P.alen = A.len;
    P.mc = mass;
    P.kdc = kdiag;
    P.J = J;
    P.c = c;
    P.b = b;
    P.x = x;
    P.r = w.r;
    P.u = w.u;
    P.w = w.w;
    P.p = w.p;
    P.s = w.s;
    P.z = w.z;
    P.nv = w.nv;
    P.m = w.m;
    P.idA = w.idA;
    P.part = w.part;
    P.bar = w.bar;
    P.err = w.err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = budget;
    P.iters_out = w.iters;
    P.relres_out = w.relres;
    P.energy_out = nullptr;
    P.m_node = 0;
    P.M = 1;            // no coupling into other nodes
    P.epi_lo = 0;
    P.epi_hi = 0;
    P.epi_target_J = 0;
    P.Jall = nullptr;
    P.dt = 0.0;
    P.R = nullptr;
    for (int j = 0; j < kMaxM; ++j) P.qh[j] = 0.0;
    P.inject_fault = 0;
    P.L = 0;
    if (reinterpret_cast<uintptr_t>(w.part) % 16 != 0) return SDC_E_INVALID;
    int grid = std::min(std::min(w.max_blocks, pcg_max_blocks(block)), nblk(n, block));
    if (grid < 1) grid = 1;
    void* args[] = {&P};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_general_kernel(block), dim3(grid),
                                                dim3(block), args,
                                                0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

void launch_update(int M, int n, const int* act, const double* w0, double dt, const Ionic& ion,
                   const Coll& co, double tol_drop, int w_frozen, StepBuffers& B, cudaStream_t s,
                   const double* tol_drop_dev, const int* n_dev) {
    dispatch_M(M, [&](auto mc) {
        constexpr int MM = decltype(mc)::value;
        k_update<MM><<<nblk(n, kUpdateBlock), kUpdateBlock, 0, s>>>(
            n, act, B.D, B.ld, B.V, B.W, w0, dt, ion, co, tol_drop, w_frozen, B.flag, B.blockcnt,
            B.blockmarg, &B.sc->err, tol_drop_dev, n_dev, B.N);
    });
}

// Inputs of the a priori drop tolerance (Sec. 4.1): c = max over nodes and rows of |dv|
// of the first sweep, and max(0, -dI/dv) over its linearisation.  Both are >= 0, so
// their IEEE bit patterns order like the values and atomicMax on the bits takes the max.
__global__ void k_drop_inputs(int n, int M, const double* __restrict__ D, int ld, int nj,
                              const double* __restrict__ J, int ldj,
                              unsigned long long* cbits, unsigned long long* ebits) {
    double cm = 0.0, em = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        for (int m = 0; m < M; ++m) cm = fmax(cm, fabs(D[(size_t)m * ld + p]));
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nj; p += stride)
        for (int m = 0; m < M; ++m) em = fmax(em, -J[(size_t)m * ldj + p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(cbits, (unsigned long long)__double_as_longlong(cm));
        atomicMax(ebits, (unsigned long long)__double_as_longlong(em));
    }
}

// TOL_drop = exp(-eta dt) (1 - rho) / (r + 1) TOL (Eq. drop-tolerance), r the least
// integer >= 0 with r >= log((1 - rho) TOL / c) / log(rho) (Eq. r-condition), eta =
// max(0, -dI/dv) / Cm.
__global__ void k_drop_final(const unsigned long long* cbits, const unsigned long long* ebits,
                             double Cm, double rho, double TOL, double dt, double* out) {
    if (threadIdx.x != 0) return;
    const double c = __longlong_as_double((long long)*cbits);
    const double eta = __longlong_as_double((long long)*ebits) / Cm;
    double r = 0.0;
    if (c > 0.0) r = fmax(0.0, ceil(log((1.0 - rho) * TOL / c) / log(rho)));
    *out = TOL > 0.0 ? exp(-eta * dt) * (1.0 - rho) / (r + 1.0) * TOL : 0.0;
}

void launch_drop_rule(int n, int M, const double* D, int ld, int nj, const double* J, int ldj,
                      double Cm, double rho, double TOL, double dt, StepBuffers& B,
                      cudaStream_t s) {
    const int rows = n > nj ? n : nj;
    int nb = nblk(rows, 256);
    if (nb > 1216) nb = 1216;                 // 8 blocks per SM, grid-stride beyond
    if (nb < 1) nb = 1;
    k_drop_inputs<<<nb, 256, 0, s>>>(n, M, D, ld, nj, J, ldj, &B.sc->drop_c, &B.sc->drop_eta);
    k_drop_final<<<1, 32, 0, s>>>(&B.sc->drop_c, &B.sc->drop_eta, Cm, rho, TOL, dt,
                                  &B.sc->tol_drop);
}

void launch_select(int n, const int* act, int* act_next, StepBuffers& B, cudaStream_t s,
                   const int* n_dev) {
    const int nb = nblk(n, kUpdateBlock);
    k_scan_counts<<<1, 1024, 0, s>>>(nb, B.blockcnt, B.blockoff, B.blockmarg, B.sc);
    k_scatter<<<nb, kUpdateBlock, 0, s>>>(n, act, B.flag, B.blockoff, act_next, B.map, n_dev);
}

void launch_extract(int n_old, const Ell& Aold, const int* map, Ell& Anew, StepBuffers& B,
                    cudaStream_t s, const int* n_dev) {
    cudaMemsetAsync(&B.sc->nnz, 0, sizeof(unsigned long long), s);
    k_extract<<<nblk(n_old, 256), 256, 0, s>>>(n_old, Aold.val, Aold.col, Aold.len, Aold.ld, map,
                                               Anew.val, Anew.col, Anew.len, Anew.ld, &B.sc->nnz,
                                               n_dev);
}

}  // namespace sdc

namespace sdc {
SDC_CHECK_READER(check_take_step)
}  // namespace sdc
