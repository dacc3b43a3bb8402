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

// ---- error flag: first error wins ---------------------------------------------
__device__ __forceinline__ void raise_error(int* err, int code) { atomicCAS(err, 0, code); }

// ---- bounded grid barrier for cooperative launches ----------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every block calls this the same number of times; `epoch` counts arrivals the
// caller expects (gridDim.x per call).  A wait longer than `budget` SM cycles
// raises SDC_E_TIMEOUT and returns false in every thread of the block, so the
// kernel can leave without touching further memory.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned& epoch, long long budget,
                                          int* err) {
    epoch += gridDim.x;
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        while (ld_acquire_gpu(bar) < epoch) {
            if (clock64() - t0 > budget) {
                raise_error(err, SDC_E_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
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

// Sum of the G per-block partials written before the last grid barrier.  Every
// warp computes the same value in the same order (bitwise identical in every
// block), read through L2 so no stale L1 line is used.
__device__ __forceinline__ double sum_partials(const double* part, int G) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < G; i += 32) s += __ldcg(part + i);
    return warp_sum(s);
}

}  // namespace sdc
