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
    // CG vectors (global-vector variant; the shared-memory variants keep their
    // own rows on chip and publish u only)
    double* r;           // residual
    double* u;           // D^-1 r (published for the neighbours' gathers)
    double* p;           // search direction
    double* s;           // A p
    double* w;           // A u
    double* idA;         // reciprocal of the diagonal (Jacobi preconditioner)
    double* part;        // per-block partial sums, two per block, two buffers
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
    int L;               // rows per block (shared-memory variants)
};

// LU-trick coupling of one solved row into the right-hand sides of other nodes.
__device__ __forceinline__ void cg_couple_row(const CgParams& P, int i, double xi, double kx) {
    const double base = P.kdc[i] * xi + kx;
    for (int t = P.epi_lo; t < P.epi_hi; ++t) {
        const double Jt = P.epi_target_J ? P.Jall[(size_t)t * P.ld + i] : P.J[i];
        P.R[(size_t)t * P.ld + i] -= P.dt * P.qh[t] * (base + P.mc[i] * Jt * xi);
    }
}

// Shared per-block state of a CG solve.  The scalars are derived by lane 0 of
// warp 0 from each pair of grid-wide sums (one FP64 division chain per block,
// not per thread: the FP64 pipe is the scarce unit on this part).
struct CgShared {
    double red[2 * 1024];   // per-thread partial sums of the two dot products
    double wsum[8];         // per-warp totals of the block sum
    double alpha, beta, inv_gamma, inv_alpha, gamma0, thresh, rzmax, rn;
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

// Scalars of the Chronopoulos-Gear iteration from gamma = r.u and
// delta = w.u (u = D^-1 r, w = A u):
//   first:  alpha = gamma / delta, beta = 0
//   later:  beta = gamma / gamma_old,
//           alpha = gamma / (delta - beta gamma / alpha_old)
// 1/gamma and 1/alpha are kept so that a step needs one division chain.
__device__ __forceinline__ void cg_first(CgShared& S, double g, double d, double rtol) {
    S.gamma0 = g;
    S.rn = g;
    S.beta = 0.0;
    S.thresh = rtol * sqrt(g);
    S.rzmax = largest_with_sqrt_at_most(S.thresh);
    if (!isfinite(g) || !isfinite(d)) {
        S.state = 2;
    } else if (g == 0.0) {
        S.state = 1;
    } else {
        S.state = 0;
        S.alpha = g / d;
        S.inv_gamma = 1.0 / g;
        S.inv_alpha = d * S.inv_gamma;
    }
}
__device__ __forceinline__ void cg_next(CgShared& S, double g, double d) {
    S.rn = g;
    if (!isfinite(g) || !isfinite(d)) {
        S.state = 2;
    } else if (g >= 0.0 && g <= S.rzmax) {
        S.state = 1;
    } else {
        const double beta = g * S.inv_gamma;
        const double den = d - beta * g * S.inv_alpha;
        S.alpha = g / den;
        S.inv_gamma = 1.0 / g;
        S.inv_alpha = den * S.inv_gamma;
        S.beta = beta;
    }
}
// final relative preconditioned residual sqrt(r.u / r0.u0)
__device__ __forceinline__ double cg_relres(const CgShared& S) {
    return S.gamma0 > 0.0 ? sqrt(fabs(S.rn) / S.gamma0) : 0.0;
}

// Block sum of two values per thread in a fixed order, result in thread 0.
// Thread t stores (a, b) at red[t], red[1024 + t]; warp w < W = min(4, B/32)
// adds the warp-rows w, w + W, w + 2W, ... of the block (a balanced tree over
// at most 8 values per lane, then a shuffle tree), and thread 0 adds the W
// warp totals in order.  Four summing warps keep every SM sub-partition's
// FP64 unit busy with a short dependency chain.
__device__ __forceinline__ void block_sum2(double a, double b, CgShared& S, double& sa,
                                           double& sb) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int nw = blockDim.x >> 5;
    const int W = min(4, nw);
    S.red[t] = a;
    S.red[1024 + t] = b;
    __syncthreads();
    if (wid < W) {
        const int cnt = (nw - wid + W - 1) / W;   // warp-rows of this warp (<= 8)
        double x[8], y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int at = (wid + k * W) * 32 + lane;
            x[k] = k < cnt ? S.red[at] : 0.0;
            y[k] = k < cnt ? S.red[1024 + at] : 0.0;
        }
        if (cnt > 4) {
#pragma unroll
            for (int k = 0; k < 4; ++k) { x[k] += x[k + 4]; y[k] += y[k + 4]; }
        }
        if (cnt > 2) {
            x[0] += x[2]; y[0] += y[2];
            x[1] += x[3]; y[1] += y[3];
        }
        if (cnt > 1) { x[0] += x[1]; y[0] += y[1]; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
            y[0] += __shfl_xor_sync(0xffffffffu, y[0], o);
        }
        if (lane == 0) {
            S.wsum[wid] = x[0];
            S.wsum[4 + wid] = y[0];
        }
    }
    __syncthreads();
    sa = sb = 0.0;
    if (t == 0) {
        if (W == 4) {
            sa = (S.wsum[0] + S.wsum[1]) + (S.wsum[2] + S.wsum[3]);
            sb = (S.wsum[4] + S.wsum[5]) + (S.wsum[6] + S.wsum[7]);
        } else {
            for (int k = 0; k < W; ++k) { sa += S.wsum[k]; sb += S.wsum[4 + k]; }
        }
    }
}

// Sum of two values per thread over a group of `nblk` blocks (the whole grid,
// or one instance's share of a batched launch), fused with the group barrier.
// Thread 0 publishes the block's pair to part[2 bidx], arrives and waits;
// warp 0 then adds the nblk pairs in index order (bitwise identical in every
// block) and lane 0 runs on_total(a, b), which stores the iteration's scalars
// in shared memory.  A closing CTA barrier makes them visible to the block.
// Returns false after a barrier timeout.
template <class F>
__device__ __forceinline__ bool group_reduce2(double a, double b, CgShared& S, double* part,
                                              unsigned* bar, int nblk, int bidx, unsigned& epoch,
                                              long long budget, int* err, F&& on_total) {
    double sa, sb;
    block_sum2(a, b, S, sa, sb);
    epoch += nblk;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int ok = 1;
        if (lane == 0) {
            part[2 * bidx] = sa;
            part[2 * bidx + 1] = sb;
            ok = barrier_arrive_wait(bar, epoch, budget, err);
        }
        __syncwarp();
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
            double ta = 0.0, tb = 0.0;
            const double2* p2 = reinterpret_cast<const double2*>(part);
            for (int i = lane; i < nblk; i += 32) {
                const double2 v = __ldcg(p2 + i);
                ta += v.x;
                tb += v.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ta += __shfl_xor_sync(0xffffffffu, ta, o);
                tb += __shfl_xor_sync(0xffffffffu, tb, o);
            }
            if (lane == 0) on_total(ta, tb);
        }
        if (lane == 0) S.ok = ok;
    }
    __syncthreads();
    return S.ok != 0;
}

// Jacobi-PCG on the restricted node system, whole solve in one cooperative
// launch, vectors in global memory (any size).
//
// The iteration is preconditioned CG in the arrangement of Chronopoulos and
// Gear (1989): with u = D^-1 r and w = A u, both dot products of an iteration,
// gamma = r.u and delta = w.u, are summed in one grid-wide reduction, and
// s = A p follows from the recurrence s = w + beta s.  Per iteration:
//   phase 1: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s,
//            u = D^-1 r (published) -> grid barrier
//   phase 2: w = A u (gathers u of neighbouring rows; the diagonal part of
//            A u is D u = r), r.u and w.u -> one grid sum of two values,
//            convergence test on r.u, then beta and alpha
// The iterates are those of standard preconditioned CG in exact arithmetic.
// Rows are processed grid-stride; each thread owns the same rows in every
// phase.  Block totals are added in a fixed order by every block, so all
// blocks take identical decisions.
// One group of `nblk` blocks solves rows [row0, row1): the whole launch, or
// one instance of a batched launch.  `part` points at the group's first
// partial-sum pair of buffer 0; buffer 1 is `pstride` doubles further.
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
    int it = 0;
    bool first = true;
    while (true) {
        // phase 2: w = A u, r.u, w.u
        double ga = 0.0, de = 0.0;
        for (int i = i0; i < row1; i += stride) {
            const int len = P.alen[i];
            double acc = 0.0;
            for (int t = 0; t < len; ++t)
                acc += P.aval[(size_t)t * ld + i] * __ldcg(P.u + P.acol[(size_t)t * ld + i]);
            const double ri = P.r[i];
            const double ui = P.u[i];
            const double wi = ri + c * acc;
            P.w[i] = wi;
            ga += ri * ui;
            de += wi * ui;
        }
        if (!group_reduce2(ga, de, S, part + buf * pstride, bar, nblk, bidx, epoch, P.budget,
                           P.err, [&](double g, double d) {
                               if (first) cg_first(S, g, d, P.rtol);
                               else cg_next(S, g, d);
                           }))
            return;
        buf ^= 1;
        first = false;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (lead) raise_error(P.err, SDC_E_CG_NOCONV);
            break;
        }
        ++it;
        // phase 1: p, s, x, r, u
        const double alpha = S.alpha, beta = S.beta;
        for (int i = i0; i < row1; i += stride) {
            const double pi = P.u[i] + beta * P.p[i];
            const double si = P.w[i] + beta * P.s[i];
            P.p[i] = pi;
            P.s[i] = si;
            P.x[i] += alpha * pi;
            const double r = P.r[i] - alpha * si;
            P.r[i] = r;
            P.u[i] = r * P.idA[i];
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
    pcg_group(P, S, 0, P.n, (int)gridDim.x, (int)blockIdx.x, P.bar, P.part, 2 * (int)gridDim.x,
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
              P.part + 2 * g.blk0, 2 * (int)gridDim.x, seg_iters + g.seg, seg_relres + g.seg);
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
// block b owns the contiguous rows [b L, b L + L); their r, u, p, s, w and
// reciprocal diagonal stay in shared memory for the whole solve.  u is
// published to global memory (coalesced) for the neighbours' gathers and x is
// accumulated in place in global memory; the matrix is read through the
// read-only path.
__global__ void __launch_bounds__(1024, 1) k_pcg_smem(CgParams P) {
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
    int it = 0;
    bool first = true;
    while (true) {
        double ga = 0.0, de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(ug + __ldg(acol + (size_t)k * ld + i));
            const double ri = sr[l], ui = su[l];
            const double wi = ri + c * acc;
            sw[l] = wi;
            ga += ri * ui;
            de += wi * ui;
        }
        if (!group_reduce2(ga, de, S, P.part + buf * 2 * G, P.bar, G, (int)blockIdx.x, epoch,
                           P.budget, P.err, [&](double g, double d) {
                               if (first) cg_first(S, g, d, P.rtol);
                               else cg_next(S, g, d);
                           }))
            return;
        buf ^= 1;
        first = false;
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
    }
    // x is complete and visible: the last grid sum followed its last update
    if (P.epi_lo < P.epi_hi) {
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            const double xi = __ldcg(xg + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k)
                acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(xg + __ldg(acol + (size_t)k * ld + i));
            cg_couple_row(P, i, xi, acc);
        }
    }
}

// Thread-block-cluster variant for small active sets (n <= C * L rows, one
// cluster of C CTAs).  The same iteration as k_pcg_smem; u of other CTAs is
// read from their shared memory (distributed shared memory), block totals are
// exchanged through shared memory, and the hardware cluster barrier replaces
// the global arrival counter, so the iteration loop touches no global memory
// besides the (read-only) matrix and x.  Every CTA takes the same decisions
// (same totals, same order) and leaves only after a final cluster barrier, so
// no CTA reads the shared memory of one that has exited.
__global__ void __launch_bounds__(1024, 1) k_pcg_cluster(CgParams P) {
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    extern __shared__ double sm[];
    __shared__ CgShared S;
    __shared__ double cpart[4];
    __shared__ double* ur[16];
    __shared__ double* pr[16];
    const int B = blockDim.x, t = threadIdx.x;
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int L = P.L, ld = P.ld;
    const int r0 = rank * L;
    const int nl = max(0, min(P.n - r0, L));
    double* __restrict__ sr = sm;
    double* __restrict__ su = sm + L;
    double* __restrict__ sp = sm + 2 * L;
    double* __restrict__ ss = sm + 3 * L;
    double* __restrict__ sw = sm + 4 * L;
    double* __restrict__ si = sm + 5 * L;
    double* __restrict__ xg = P.x;
    const double* __restrict__ aval = P.aval;
    const int* __restrict__ acol = P.acol;
    const int* __restrict__ alen = P.alen;
    const double c = P.c;
    if (t < C) {
        ur[t] = cl.map_shared_rank(su, t);
        pr[t] = cl.map_shared_rank(cpart, t);
    }
    int buf = 0;
    // cluster-wide sum of two values; lane 0 of warp 0 derives the scalars
    auto reduce2 = [&](double a, double b, auto&& on_total) {
        double sa, sb;
        block_sum2(a, b, S, sa, sb);
        if (t == 0) {
            cpart[2 * buf] = sa;
            cpart[2 * buf + 1] = sb;
        }
        cl.sync();
        if (t < 32) {
            double ta = t < C ? pr[t][2 * buf] : 0.0;
            double tb = t < C ? pr[t][2 * buf + 1] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ta += __shfl_xor_sync(0xffffffffu, ta, o);
                tb += __shfl_xor_sync(0xffffffffu, tb, o);
            }
            if (t == 0) on_total(ta, tb);
        }
        buf ^= 1;
        __syncthreads();
    };

    for (int l = t; l < nl; l += B) {
        const int i = r0 + l;
        const double d = P.mc[i] * (1.0 + c * P.J[i]) + c * P.kdc[i];
        if (!isfinite(d)) raise_error(P.err, SDC_E_NONFINITE);
        else if (!(d > 0.0)) raise_error(P.err, SDC_E_DOMAIN);
        const double id = 1.0 / d;
        si[l] = id;
        const double r = P.b[i];
        sr[l] = r;
        su[l] = r * id;
        sp[l] = 0.0;
        ss[l] = 0.0;
        xg[i] = 0.0;
    }
    cl.sync();
    int it = 0;
    bool first = true;
    while (true) {
        double ga = 0.0, de = 0.0;
        for (int l = t; l < nl; l += B) {
            const int i = r0 + l;
            const int len = __ldg(alen + i);
            double acc = 0.0;
            for (int k = 0; k < len; ++k) {
                const int j = __ldg(acol + (size_t)k * ld + i);
                const int owner = j / L;
                acc += __ldg(aval + (size_t)k * ld + i) * ur[owner][j - owner * L];
            }
            const double ri = sr[l], ui = su[l];
            const double wi = ri + c * acc;
            sw[l] = wi;
            ga += ri * ui;
            de += wi * ui;
        }
        reduce2(ga, de, [&](double g, double d) {
            if (first) cg_first(S, g, d, P.rtol);
            else cg_next(S, g, d);
        });
        first = false;
        if (S.state != 0) break;
        if (it >= P.maxit) {
            if (rank == 0 && t == 0) raise_error(P.err, SDC_E_CG_NOCONV);
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
            su[l] = r * si[l];
        }
        cl.sync();   // u of every CTA is final before the gathers
    }
    if (S.state == 2) {
        if (rank == 0 && t == 0) raise_error(P.err, SDC_E_NONFINITE);
    } else {
        if (rank == 0 && t == 0) {
            *P.iters_out = it;
            *P.relres_out = cg_relres(S);
        }
        if (P.epi_lo < P.epi_hi) {
            cl.sync();   // every CTA's x is final (cluster-scope ordering covers global memory)
            for (int l = t; l < nl; l += B) {
                const int i = r0 + l;
                const int len = __ldg(alen + i);
                const double xi = __ldcg(xg + i);
                double acc = 0.0;
                for (int k = 0; k < len; ++k)
                    acc += __ldg(aval + (size_t)k * ld + i) * __ldcg(xg + __ldg(acol + (size_t)k * ld + i));
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
                         (int)(6 * kSmemRows * sizeof(double)));
    cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int C = 16; C >= 2; C /= 2) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(C);
        lc.blockDim = dim3(block);
        lc.dynamicSmemBytes = (size_t)6 * kSmemRows * sizeof(double);
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
    P.u = B.u;
    P.p = B.p;
    P.s = B.s;
    P.w = B.w;
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
    P.u = B.u;
    P.p = B.p;
    P.s = B.s;
    P.w = B.w;
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
                                 (int)(6 * kSmemRows * sizeof(double)));
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
        lc.dynamicSmemBytes = (size_t)6 * P.L * sizeof(double);
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
        const size_t smem = (size_t)6 * P.L * sizeof(double);
        // the largest systems keep every SM's FP64 pipe busy with 32 warps;
        // smaller ones favour shorter block-level reductions
        const int blk = n >= cfg.big_rows ? 1024 : cfg.smem_block;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_pcg_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(6 * kSmemRows * sizeof(double)));
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
    P.u = B.u;
    P.p = B.p;
    P.s = B.s;
    P.w = B.w;
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
    P.u = w.u;
    P.p = w.p;
    P.s = w.s;
    P.w = w.w;
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
