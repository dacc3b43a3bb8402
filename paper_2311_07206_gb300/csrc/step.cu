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
    double* r;
    double* z;
    double* p;
    double* q;
    double* dA;          // diagonal of the node system
    double* idA;         // its reciprocal (Jacobi preconditioner)
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
    double qh[kMaxM];    // coupling coefficient per target node
    // targets [epi_lo, epi_hi): R[t] -= dt qh[t] (K x + mass J' x), with J' this
    // node's J (forward sweep, targets after m) or the target's own J taken from
    // Jall (reverse sweep, targets before m)
    int epi_lo, epi_hi, epi_target_J;
    const double* Jall;
    int inject_fault;    // testing hook: the last block skips the first barrier
    int L;               // rows per block (shared-memory variant)
};

// LU-trick coupling of one solved row into the right-hand sides of other nodes.
__device__ __forceinline__ void cg_couple_row(const CgParams& P, int i, double xi, double kx) {
    const double base = P.kdc[i] * xi + kx;
    for (int t = P.epi_lo; t < P.epi_hi; ++t) {
        const double Jt = P.epi_target_J ? P.Jall[(size_t)t * P.ld + i] : P.J[i];
        P.R[(size_t)t * P.ld + i] -= P.dt * P.qh[t] * (base + P.mc[i] * Jt * xi);
    }
}


// Shared per-block scalars of a CG solve.  Lane 0 of warp 0 derives them from
// each grid-wide sum (one FP64 division / square root per block, not per
// thread: the FP64 pipe is the scarce unit on this part).
struct CgShared {
    double red[1024];   // per-thread partial sums
    double alpha, beta, rho, rho0, thresh, rzmax, rn;
    int ok, state;      // state: 0 iterating, 1 converged, 2 non-finite
};

// The stopping test sqrt(r.z) <= rtol sqrt(r0.z0) is evaluated as
// r.z <= rzmax with rzmax the largest double whose correctly rounded square
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

__device__ __forceinline__ void cg_after_rho0(CgShared& S, double tot, double rtol) {
    S.rho0 = tot;
    S.rho = tot;
    S.rn = tot;
    S.thresh = rtol * sqrt(tot);
    S.rzmax = largest_with_sqrt_at_most(S.thresh);
    S.state = !isfinite(tot) ? 2 : (tot == 0.0 ? 1 : 0);
}
__device__ __forceinline__ void cg_after_pq(CgShared& S, double pq) { S.alpha = S.rho / pq; }
__device__ __forceinline__ void cg_after_rz(CgShared& S, double rn) {
    S.rn = rn;
    if (!isfinite(rn)) {
        S.state = 2;
    } else if (rn >= 0.0 && rn <= S.rzmax) {
        S.state = 1;
    } else {
        S.beta = rn / S.rho;
        S.rho = rn;
    }
}
// final relative preconditioned residual sqrt(r.z / r0.z0)
__device__ __forceinline__ double cg_relres(const CgShared& S) {
    return S.rho0 > 0.0 ? sqrt(fabs(S.rn) / S.rho0) : 0.0;
}

// Jacobi-PCG on the restricted node system (diagonal preconditioner), whole
// solve in one cooperative launch, vectors in global memory (any size).
//
// The iteration is the standard preconditioned CG, arranged with two grid-wide
// synchronisation points per iteration: the matrix is applied to z = D^-1 r,
// and p and q = A p follow from p = z + beta p, q = A z + beta q (the same
// iterates in exact arithmetic as q = A p; rounding differs only in the order
// of the additions).  Per iteration:
//   phase A: s = A z (gathers z of neighbouring rows), p, q updates, p.q
//            -> grid sum, alpha = rho / p.q
//   phase B: x += alpha p, r -= alpha q, z = D^-1 r (published), r.z
//            -> grid sum, convergence test, beta
// Rows are processed grid-stride; each thread owns the same rows in every
// phase.  Block totals are added in a fixed order by every block, so all
// blocks take identical decisions.
// One group of `nblk` blocks solves rows [row0, row1): the whole launch, or
// one instance of a batched launch.  `part` points at the group's first
// partial-sum slot of buffer 0; buffer 1 is `pstride` doubles further.
__device__ __forceinline__ void pcg_group(const CgParams& P, CgShared& S, int row0, int row1,
                                          int nblk, int bidx, unsigned* bar, double* part,
                                          int pstride, int* iters_out, double* relres_out) {
    const int stride = nblk * blockDim.x;
    const int i0 = row0 + bidx * blockDim.x + threadIdx.x;
    const bool lead = (bidx == 0 && threadIdx.x == 0);
    const int ld = P.ld;
    const double c = P.c;
    unsigned epoch = 0;
    int buf = 0;

    double acc_part = 0.0;
    for (int i = i0; i < row1; i += stride) {
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        P.dA[i] = d;
        P.idA[i] = id;
        const double r = P.b[i];
        const double z = r * id;
        P.r[i] = r;
        P.z[i] = z;
        P.p[i] = 0.0;
        P.q[i] = 0.0;
        P.x[i] = 0.0;
        acc_part += r * z;
    }
    if (P.inject_fault && bidx == nblk - 1) {
        // leave without arriving: every other block's bounded wait runs out
        if (nblk == 1 && threadIdx.x == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!group_reduce(acc_part, S.red, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                      P.err, &S.ok, [&](double t) { cg_after_rho0(S, t, P.rtol); }))
        return;
    buf ^= 1;
    int it = 0;
    double beta = 0.0;
    while (S.state == 0) {
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        // s = A z; p = z + beta p; q = s + beta q; p.q
        acc_part = 0.0;
        for (int i = i0; i < row1; i += stride) {
            const int len = P.alen[i];
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.z + P.acol[(size_t)t * ld + i]);
            const double zi = __ldcg(P.z + i);
            const double si = P.dA[i] * zi + c * acc;
            const double pi = zi + beta * P.p[i];
            const double qi = si + beta * P.q[i];
            P.p[i] = pi;
            P.q[i] = qi;
            acc_part += pi * qi;
        }
        if (!group_reduce(acc_part, S.red, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                          P.err, &S.ok, [&](double t) { cg_after_pq(S, t); }))
            return;
        buf ^= 1;
        const double alpha = S.alpha;
        // x += alpha p, r -= alpha q, z = D^-1 r, r.z
        acc_part = 0.0;
        for (int i = i0; i < row1; i += stride) {
            P.x[i] += alpha * P.p[i];
            const double r = P.r[i] - alpha * P.q[i];
            P.r[i] = r;
            const double z = r * P.idA[i];
            P.z[i] = z;
            acc_part += r * z;
        }
        if (!group_reduce(acc_part, S.red, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                          P.err, &S.ok, [&](double t) { cg_after_rz(S, t); }))
            return;
        buf ^= 1;
        beta = S.beta;
    }
    if (S.state == 2) {
        if (lead) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (lead) {
        *iters_out = it;
        *relres_out = cg_relres(S);
    }
    // x is complete in every block of the group: the last group sum followed its update.
    if (P.epi_lo < P.epi_hi) {
        for (int i = i0; i < row1; i += stride) {
            const int len = P.alen[i];
            const double xi = __ldcg(P.x + i);
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.x + P.acol[(size_t)t * ld + i]);
            cg_couple_row(P, i, xi, acc);
        }
    }
}

__global__ void __launch_bounds__(1024, 1) k_pcg(CgParams P) {
    __shared__ CgShared S;
    pcg_group(P, S, 0, P.n, (int)gridDim.x, (int)blockIdx.x, P.bar, P.part, (int)gridDim.x,
              P.iters_out, P.relres_out);
}

// Batched variant: independent solves of the instances of a batch (disjoint
// diagonal blocks of the system) in one cooperative launch.  Block b works on
// the group tab[b] describes: that instance's compact rows, its own barrier
// counter and partial-sum slots, its own iteration count.  Groups never wait
// for each other, so a converged instance's blocks leave early.
__global__ void __launch_bounds__(1024, 1) k_pcg_batch(CgParams P, const SegBlock* __restrict__ tab,
                                                        unsigned* __restrict__ bars,
                                                        int* __restrict__ seg_iters,
                                                        double* __restrict__ seg_relres) {
    __shared__ CgShared S;
    const SegBlock g = tab[blockIdx.x];
    pcg_group(P, S, g.row0, g.row1, g.nblk, (int)blockIdx.x - g.blk0, bars + g.seg,
              P.part + g.blk0, (int)gridDim.x, seg_iters + g.seg, seg_relres + g.seg);
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
// block b owns the contiguous rows [b L, b L + L); their x, r, z, p, q,
// diagonal and reciprocal diagonal stay in shared memory for the whole solve.
// Only z is published to global memory (coalesced) for the neighbours'
// gathers; the matrix is read through the read-only path.
__global__ void __launch_bounds__(1024, 1) k_pcg_smem(CgParams P) {
    extern __shared__ double sm[];
    __shared__ CgShared S;
    const int G = gridDim.x, B = blockDim.x, t = threadIdx.x;
    const int L = P.L, ld = P.ld;
    const int r0 = blockIdx.x * L;
    const int nl = max(0, min(P.n - r0, L));
    double* __restrict__ sx = sm;
    double* __restrict__ sr = sm + L;
    double* __restrict__ sz = sm + 2 * L;
    double* __restrict__ sp = sm + 3 * L;
    double* __restrict__ sq = sm + 4 * L;
    double* __restrict__ sd = sm + 5 * L;
    double* __restrict__ si = sm + 6 * L;
    double* __restrict__ zg = P.z;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    unsigned epoch = 0;
    int buf = 0;

    double part = 0.0;
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        sd[l] = d;
        si[l] = id;
        const double r = P.b[i];
        const double z = r * id;
        sr[l] = r;
        sz[l] = z;
        zg[i] = z;
        sp[l] = 0.0;
        sq[l] = 0.0;
        sx[l] = 0.0;
        part += r * z;
    }
    if (P.inject_fault && blockIdx.x == G - 1) {
        if (G == 1 && t == 0) raise_error(P.err, SDC_E_TIMEOUT);
        return;
    }
    if (!grid_reduce(part, S.red, P.part + buf * G, P.bar, epoch, P.budget, P.err, &S.ok,
                     [&](double tot) { cg_after_rho0(S, tot, P.rtol); }))
        return;
    buf ^= 1;
    int it = 0;
    double beta = 0.0;
    while (S.state == 0) {
        if (it >= P.maxit) {
            if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        part = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(zg + __ldg(acol + (size_t)k * ld + i));
            const double zi = sz[l];
            const double s_i = sd[l] * zi + c * acc;
            const double pi = zi + beta * sp[l];
            const double qi = s_i + beta * sq[l];
            sp[l] = pi;
            sq[l] = qi;
            part += pi * qi;
        }
        if (!grid_reduce(part, S.red, P.part + buf * G, P.bar, epoch, P.budget, P.err, &S.ok,
                         [&](double tot) { cg_after_pq(S, tot); }))
            return;
        buf ^= 1;
        const double alpha = S.alpha;
        part = 0.0;
        for (int l = t; l < nl; l += B) {
            sx[l] += alpha * sp[l];
            const double r = sr[l] - alpha * sq[l];
            sr[l] = r;
            const double z = r * si[l];
            sz[l] = z;
            zg[r0 + l] = z;
            part += r * z;
        }
        if (!grid_reduce(part, S.red, P.part + buf * G, P.bar, epoch, P.budget, P.err, &S.ok,
                         [&](double tot) { cg_after_rz(S, tot); }))
            return;
        buf ^= 1;
        beta = S.beta;
    }
    if (S.state == 2) {
        if (blockIdx.x == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
        return;
    }
    if (blockIdx.x == 0 && t == 0) {
        *P.iters_out = it;
        *P.relres_out = cg_relres(S);
    }
    for (int l = t; l < nl; l += B) P.x[r0 + l] = sx[l];
    if (P.epi_lo < P.epi_hi) {
        if (!grid_barrier(P.bar, epoch, P.budget, P.err, &S.ok)) return;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = sx[l];
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(P.x + __ldg(acol + (size_t)k * ld + i));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

// Thread-block-cluster variant for small active sets (n <= C * L rows, one
// cluster of C CTAs).  The same iteration as k_pcg_smem; z and x of other CTAs
// are read from their shared memory (distributed shared memory), block totals
// are exchanged through shared memory, and the hardware cluster barrier
// replaces the global arrival counter, so the iteration loop touches no global
// memory besides the (read-only) matrix.  Every CTA takes the same decisions
// (same totals, same order) and leaves only after a final cluster barrier, so
// no CTA reads the shared memory of one that has exited.
__global__ void __launch_bounds__(1024, 1) k_pcg_cluster(CgParams P) {
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    extern __shared__ double sm[];
    __shared__ CgShared S;
    __shared__ double cpart[2];
    __shared__ double* zr[16];
    __shared__ double* xr[16];
    __shared__ double* pr[16];
    const int B = blockDim.x, t = threadIdx.x;
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int L = P.L, ld = P.ld;
    const int r0 = rank * L;
    const int nl = max(0, min(P.n - r0, L));
    const int nact = min(B, nl);
    double* __restrict__ sx = sm;
    double* __restrict__ sr = sm + L;
    double* __restrict__ sz = sm + 2 * L;
    double* __restrict__ sp = sm + 3 * L;
    double* __restrict__ sq = sm + 4 * L;
    double* __restrict__ sd = sm + 5 * L;
    double* __restrict__ si = sm + 6 * L;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    if (t < C) {
        zr[t] = cl.map_shared_rank(sz, t);
        xr[t] = cl.map_shared_rank(sx, t);
        pr[t] = cl.map_shared_rank(cpart, t);
    }
    int buf = 0;
    // cluster-wide sum; lane 0 of warp 0 derives the scalars from the total
    auto reduce = [&](double v, auto&& on_total) {
        S.red[t] = v;
        __syncthreads();
        if (t < 32) {
            double s = 0.0;
            for (int i = t; i < nact; i += 32) s += S.red[i];
            s = warp_sum(s);
            if (t == 0) cpart[buf] = s;
        }
        cl.sync();
        if (t < 32) {
            double tot = t < C ? pr[t][buf] : 0.0;
            tot = warp_sum(tot);
            if (t == 0) on_total(tot);
        }
        buf ^= 1;
        __syncthreads();
    };

    double part = 0.0;
    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        sd[l] = d;
        si[l] = id;
        const double r = P.b[i];
        const double z = r * id;
        sr[l] = r;
        sz[l] = z;
        sp[l] = 0.0;
        sq[l] = 0.0;
        sx[l] = 0.0;
        part += r * z;
    }
    reduce(part, [&](double tot) { cg_after_rho0(S, tot, P.rtol); });
    int it = 0;
    double beta = 0.0;
    while (S.state == 0) {
        if (it >= P.maxit) {
            if (rank == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        part = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k) {
                const int j = __ldg(acol + (size_t)k * ld + i);
                const int owner = j / L;
                acc += __ldg(aval + (size_t)k * ld + i) * zr[owner][j - owner * L];
            }
            const double zi = sz[l];
            const double s_i = sd[l] * zi + c * acc;
            const double pi = zi + beta * sp[l];
            const double qi = s_i + beta * sq[l];
            sp[l] = pi;
            sq[l] = qi;
            part += pi * qi;
        }
        reduce(part, [&](double tot) { cg_after_pq(S, tot); });
        const double alpha = S.alpha;
        part = 0.0;
        for (int l = t; l < nl; l += B) {
            sx[l] += alpha * sp[l];
            const double r = sr[l] - alpha * sq[l];
            sr[l] = r;
            const double z = r * si[l];
            sz[l] = z;
            part += r * z;
        }
        reduce(part, [&](double tot) { cg_after_rz(S, tot); });
        beta = S.beta;
    }
    if (S.state == 2) {
        if (rank == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
    } else {
        if (rank == 0 && t == 0) {
            *P.iters_out = it;
            *P.relres_out = cg_relres(S);
        }
        for (int l = t; l < nl; l += B) P.x[r0 + l] = sx[l];
        if (P.epi_lo < P.epi_hi) {
            cl.sync();   // every CTA's x is final
            for (int l = t; l < nl; l += B) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                const double xi = sx[l];
                double acc = 0.0;
                for (int k = 0; k < len; ++k) {
                    const int j = __ldg(acol + (size_t)k * ld + i);
                    const int owner = j / L;
                    acc += __ldg(aval + (size_t)k * ld + i) * xr[owner][j - owner * L];
                }
                cg_couple_row(P, i, xi, acc);
            }
        }
    }
    cl.sync();   // nobody leaves while another CTA may still read its shared memory
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

int launch_pcg_params(CgParams& P, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s);

int pcg_max_blocks(int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg, block, 0);
    return sms * per;
}

int pcg_cluster_size(int block) {
    cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(7 * kSmemRows * sizeof(double)));
    cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int C = 16; C >= 2; C /= 2) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(C);
        lc.blockDim = dim3(block);
        lc.dynamicSmemBytes = (size_t)7 * kSmemRows * sizeof(double);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_pcg_cluster, &lc) == cudaSuccess &&
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

int launch_pcg(int n, const Ell& A, int m, double dt, const Coll& co, double rtol, int maxit,
               int sweep, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
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
    P.idA = B.idA;
    P.part = B.part;
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = &B.sc->cg_iters[sweep * kMaxM + m];
    P.relres_out = &B.sc->cg_relres[sweep * kMaxM + m];
    P.m = m;
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

int launch_pcg_role(int n, const Ell& A, const PcgRole& role, double dt, int M, double rtol,
                    int maxit, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s) {
    CgParams P;
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
    P.r = B.r;
    P.z = B.z;
    P.p = B.p;
    P.q = B.q;
    P.dA = B.dA;
    P.idA = B.idA;
    P.part = B.part;
    P.bar = &B.sc->bar;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = role.iters_out;
    P.relres_out = role.relres_out;
    P.m = 0;
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
    cudaMemsetAsync(&B.sc->bar, 0, sizeof(unsigned), s);
    void* args[] = {&P};
    // cluster variant: one cluster of cfg.cluster CTAs for small active sets
    if (cfg.variant != 1 && cfg.cluster > 0 && !cfg.inject_fault && n <= cfg.cluster_rows &&
        n <= cfg.cluster * kSmemRows) {
        static bool cattr_set = false;
        if (!cattr_set) {
            cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(7 * kSmemRows * sizeof(double)));
            cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cattr_set = true;
        }
        // enough CTAs for the FP64 work, never more rows per CTA than fit
        int C = std::min(cfg.cluster, std::max(nblk(n, cfg.cluster_rows_per_cta), nblk(n, kSmemRows)));
        C = std::max(C, 1);
        P.L = nblk(n, C);
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(C);
        lc.blockDim = dim3(cfg.smem_block);
        lc.dynamicSmemBytes = (size_t)7 * P.L * sizeof(double);
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&lc, k_pcg_cluster, P);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    // shared-memory variant: one block per SM at most, each owning <= kSmemRows rows
    const bool smem_ok = cfg.variant != 1 && n <= cfg.sms * kSmemRows;
    if (smem_ok && cfg.variant != 1) {
        const int rpb = cfg.rows_per_block > 0 ? cfg.rows_per_block : 512;
        int grid = std::max(nblk(n, kSmemRows), nblk(n, rpb));
        grid = std::min(grid, cfg.sms);
        if (cfg.max_blocks > 0) grid = std::min(grid, cfg.max_blocks);
        grid = std::max(grid, nblk(n, kSmemRows));
        grid = std::max(grid, 1);
        P.L = nblk(n, grid);
        const size_t smem = (size_t)7 * P.L * sizeof(double);
        // the largest systems keep every SM's FP64 pipe busy with 32 warps;
        // smaller ones favour shorter block-level reductions
        const int blk = n >= cfg.big_rows ? 1024 : cfg.smem_block;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_pcg_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(7 * kSmemRows * sizeof(double)));
            attr_set = true;
        }
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pcg_smem, dim3(grid),
                                                    dim3(blk), args, smem, s);
        return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
    }
    int grid = std::min(cfg.max_blocks_general, nblk(n, cfg.block));
    if (grid < 1) grid = 1;
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pcg, dim3(grid), dim3(cfg.block),
                                                args, 0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

int pcg_batch_max_blocks(int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_batch, block, 0);
    return sms * per;
}

void launch_seg_bounds(const int* act, const int* count, StepBuffers& B, cudaStream_t s) {
    k_seg_bounds<<<nblk(B.nseg + 1, 128), 128, 0, s>>>(count, act, B.nseg, B.inst_off, B.bounds);
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
    P.idA = B.idA;
    P.part = B.part;
    P.bar = nullptr;
    P.err = &B.sc->err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = cfg.budget;
    P.iters_out = nullptr;
    P.relres_out = nullptr;
    P.m = m;
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
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pcg_batch, dim3((int)tab.size()),
                                                    dim3(cfg.block), args, 0, s);
        if (e != cudaSuccess) return SDC_E_CUDA;
    }
    return SDC_OK;
}

int launch_pcg_standalone(int n, const Ell& A, const double* kdiag, const double* mass,
                          const double* J, double c, const double* b, double* x, double rtol,
                          int maxit, long long budget, int block, const PcgScratch& w,
                          cudaStream_t s) {
    CgParams P;
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
    P.z = w.z;
    P.p = w.p;
    P.q = w.q;
    P.dA = w.dA;
    P.idA = w.idA;
    P.part = w.part;
    P.bar = w.bar;
    P.err = w.err;
    P.rtol = rtol;
    P.maxit = maxit;
    P.budget = budget;
    P.iters_out = w.iters;
    P.relres_out = w.relres;
    P.m = 0;
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
    int grid = std::min(std::min(w.max_blocks, pcg_max_blocks(block)), nblk(n, block));
    if (grid < 1) grid = 1;
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
