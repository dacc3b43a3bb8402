// Device helpers: Aliev-Panfilov model, deterministic reductions, bounded
// grid barrier, error flag.
#pragma once

#include <cuda_runtime.h>

#include "sdc_internal.h"

namespace sdc {

// ---- Aliev-Panfilov (Sec. 5.1.1) ----------------------------------------------
// I(v, w) = ga v (v - a)(v - 1) + v w;  R(v, w) = cw (eps + mu1 w/(v + mu2)) (-w - gs v (v - a - 1))
__device__ __forceinline__ double ap_I(const Ionic& p, double v, double w) {
    return p.ga * v * (v - p.a) * (v - 1.0) + v * w;
}
// dI/dv = ga (3 v^2 - 2 (1 + a) v + a) + w
__device__ __forceinline__ double ap_dIdv(const Ionic& p, double v, double w) {
    return p.ga * (3.0 * v * v - 2.0 * (1.0 + p.a) * v + p.a) + w;
}
// R and dR/dw, sharing the two factors
__device__ __forceinline__ void ap_R_dRdw(const Ionic& p, double v, double w, double& R,
                                          double& dRdw) {
    const double inv = 1.0 / (v + p.mu2);
    const double E = p.eps + p.mu1 * w * inv;
    const double G = -w - p.gs * v * (v - p.a - 1.0);
    R = p.cw * E * G;
    dRdw = p.cw * (p.mu1 * inv * G - E);
}

// ---- P1 element geometry (Sec. 2.2) -------------------------------------------
// Gradients of the barycentric coordinates of simplex e and its measure.
// Returns false for a degenerate element.  grad[a][c], a = 0..dim.
__device__ __forceinline__ bool p1_gradients(int dim, const double* __restrict__ xyz,
                                             const int* vt, double grad[4][3], double& vol) {
    double x0[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) x0[c] = xyz[(size_t)vt[0] * dim + c];
    // edge matrix E: column c = x_{c+1} - x_0 ; gradients = rows of E^{-1}
    double E[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int c = 0; c < dim; ++c)
        for (int r = 0; r < dim; ++r) E[r][c] = xyz[(size_t)vt[c + 1] * dim + r] - x0[r];
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) grad[a][c] = 0.0;
    double det;
    if (dim == 2) {
        det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
        const double id = 1.0 / det;
        // inverse [[E11, -E01], [-E10, E00]] / det
        grad[1][0] = E[1][1] * id;  grad[1][1] = -E[0][1] * id;
        grad[2][0] = -E[1][0] * id; grad[2][1] = E[0][0] * id;
    } else {
        const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
        const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
        const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
        det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
        const double id = 1.0 / det;
        // (E^{-1})_{rc} = adj(E)_{rc} / det, adj = cofactor^T
        grad[1][0] = c00 * id;
        grad[1][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) * id;
        grad[1][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) * id;
        grad[2][0] = c01 * id;
        grad[2][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) * id;
        grad[2][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) * id;
        grad[3][0] = c02 * id;
        grad[3][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) * id;
        grad[3][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) * id;
    }
    if (det == 0.0 || !isfinite(det)) return false;
    for (int c = 0; c < dim; ++c) grad[0][c] = -(grad[1][c] + grad[2][c] + grad[3][c]);
    vol = fabs(det) / (dim == 2 ? 2.0 : 6.0);
    return true;
}

// ---- error flag: first error wins ---------------------------------------------
__device__ __forceinline__ void raise_error(int* err, int code) { atomicCAS(err, 0, code); }

// ---- bounded grid barrier for cooperative launches ----------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Called by ONE thread per block after a __syncthreads that follows the block's
// writes, and followed by a __syncthreads: arrives with a release reduction
// (cumulative over the writes the CTA barrier ordered before it) and waits with
// acquire loads until `epoch` arrivals are counted, so every thread of the
// block sees every block's writes after the closing CTA barrier.
// A wait longer than `budget` SM cycles raises SDC_E_TIMEOUT and returns 0.
__device__ __forceinline__ int barrier_arrive_wait(unsigned* bar, unsigned epoch, long long budget,
                                                   int* err) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    const long long t0 = clock64();
    while (ld_acquire_gpu(bar) < epoch) {
        if (clock64() - t0 > budget) {
            raise_error(err, SDC_E_TIMEOUT);
            return 0;
        }
    }
    return 1;
}

// ---- deterministic reductions --------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block sum in a fixed order; result valid in thread 0.  sh: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? sh[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// Grid-wide sum of one double per thread, fused with a grid barrier, for a
// part where FP64 issue slots are scarce.  Each thread stores its value in
// red[threadIdx.x]; warp 0 adds the block's values (one lane per 32-stride
// column, then a shuffle tree), lane 0 publishes the block total to
// part[blockIdx.x] and waits at the barrier, warp 0 adds the G block totals in
// index order (bitwise identical in every block), and lane 0 alone runs
// `on_total(total)`, which derives the iteration's scalars and stores them in
// shared memory.  A closing CTA barrier makes them visible to the block.
// Returns false after a barrier timeout.  red: blockDim.x doubles; flag: an
// int in shared memory.
// The participating blocks are the `nblk` blocks of a group (the whole grid,
// or one instance's share of a batched launch); `bidx` is this block's index
// in the group, part[0..nblk) its partial-sum slots and bar its counter.
template <class F>
__device__ __forceinline__ bool group_reduce(double v, double* red, double* part, unsigned* bar,
                                             int nblk, int bidx, unsigned& epoch, long long budget,
                                             int* err, int* ok_flag, F&& on_total) {
    const int lane = threadIdx.x & 31;
    red[threadIdx.x] = v;
    __syncthreads();
    epoch += nblk;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = lane; i < (int)blockDim.x; i += 32) s += red[i];
        s = warp_sum(s);
        int ok = 1;
        if (lane == 0) {
            part[bidx] = s;
            ok = barrier_arrive_wait(bar, epoch, budget, err);
        }
        __syncwarp();
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
            double t = 0.0;
            for (int i = lane; i < nblk; i += 32) t += __ldcg(part + i);
            t = warp_sum(t);
            if (lane == 0) on_total(t);
        }
        if (lane == 0) *ok_flag = ok;
    }
    __syncthreads();
    return *ok_flag != 0;
}

template <class F>
__device__ __forceinline__ bool grid_reduce(double v, double* red, double* part, unsigned* bar,
                                            unsigned& epoch, long long budget, int* err,
                                            int* ok_flag, F&& on_total) {
    return group_reduce(v, red, part, bar, (int)gridDim.x, (int)blockIdx.x, epoch, budget, err,
                        ok_flag, on_total);
}

// Plain barrier of a block group with the same conventions (flag: an int in
// shared memory).
__device__ __forceinline__ bool group_barrier(unsigned* bar, int nblk, unsigned& epoch,
                                              long long budget, int* err, int* ok_flag) {
    epoch += nblk;
    __syncthreads();
    if (threadIdx.x == 0) *ok_flag = barrier_arrive_wait(bar, epoch, budget, err);
    __syncthreads();
    return *ok_flag != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, long long budget,
                                             int* err, int* ok_flag) {
    return group_barrier(bar, (int)gridDim.x, epoch, budget, err, ok_flag);
}

}  // namespace sdc
