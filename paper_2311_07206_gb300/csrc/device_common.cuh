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
__device__ __forceinline__ void ap_R_dRdw_inv(const Ionic& p, double v, double w, double inv,
                                              double& R, double& dRdw) {
    const double E = p.eps + p.mu1 * w * inv;
    const double G = -w - p.gs * v * (v - p.a - 1.0);
    R = p.cw * E * G;
    dRdw = p.cw * (p.mu1 * inv * G - E);
}
__device__ __forceinline__ void ap_R_dRdw(const Ionic& p, double v, double w, double& R,
                                          double& dRdw) {
    ap_R_dRdw_inv(p, v, w, 1.0 / (v + p.mu2), R, dRdw);
}

// Reciprocals of x[0..N-1] with one division (Montgomery's simultaneous inversion:
// prefix products, one reciprocal of the full product, then back-substitution),
// 3 (N - 1) multiplications instead of N - 1 further divisions.  For positive x of
// moderate range (no overflow or underflow of the product); each result within a
// few ulps of 1 / x[k].
template <int N>
__device__ __forceinline__ void batch_reciprocal(const double* x, double* inv) {
    double pre[N];
    pre[0] = x[0];
#pragma unroll
    for (int k = 1; k < N; ++k) pre[k] = pre[k - 1] * x[k];
    double a = 1.0 / pre[N - 1];
#pragma unroll
    for (int k = N - 1; k > 0; --k) {
        inv[k] = a * pre[k - 1];
        a *= x[k];
    }
    inv[0] = a;
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

// ---- checked builds -------------------------------------------------------------
// Built with SDC_CHECKED=1 (libsdc_gb300_checked.so), every gathered index of the
// kernels goes through sdc_idx(j, bound, site): an index outside [0, bound) is recorded
// in this translation unit's check words (the check site and the index of the first
// failure, and a count) and replaced by 0, an in-bounds index, so the kernel runs on to
// its end over bounded loops; the library's entry points turn a record into
// SDC_E_INVALID after the call.  Without the flag sdc_idx returns j unchanged and the
// check compiles away.
#if SDC_CHECKED
static __device__ unsigned long long g_check_first;   // (site << 32) | index, 0: none
static __device__ unsigned int g_check_count;
#endif
__device__ __forceinline__ int sdc_idx(int j, int bound, int site) {
#if SDC_CHECKED
    if ((unsigned)j >= (unsigned)bound) {
        atomicCAS(&g_check_first, 0ull, ((unsigned long long)(unsigned)site << 32) | (unsigned)j);
        atomicAdd(&g_check_count, 1u);
        return 0;
    }
#else
    (void)bound;
    (void)site;
#endif
    return j;
}

// Host side: read and clear this translation unit's check words after the work on
// `stream`; returns the first failure record (0: none) and sets *count.
#if SDC_CHECKED
#define SDC_CHECK_READER(fn)                                                               \
    unsigned long long fn(void* stream, unsigned* count) {                                  \
        unsigned long long first = 0, zero = 0;                                             \
        unsigned cnt = 0, zc = 0;                                                           \
        cudaStream_t s = (cudaStream_t)stream;                                              \
        cudaMemcpyFromSymbolAsync(&first, g_check_first, sizeof first, 0,                   \
                                  cudaMemcpyDeviceToHost, s);                               \
        cudaMemcpyFromSymbolAsync(&cnt, g_check_count, sizeof cnt, 0, cudaMemcpyDeviceToHost, \
                                  s);                                                       \
        cudaStreamSynchronize(s);                                                           \
        if (first || cnt) {                                                                 \
            cudaMemcpyToSymbolAsync(g_check_first, &zero, sizeof zero, 0,                   \
                                    cudaMemcpyHostToDevice, s);                             \
            cudaMemcpyToSymbolAsync(g_check_count, &zc, sizeof zc, 0, cudaMemcpyHostToDevice, \
                                    s);                                                     \
            cudaStreamSynchronize(s);                                                       \
        }                                                                                   \
        if (count) *count = cnt;                                                            \
        return first;                                                                       \
    }
#else
#define SDC_CHECK_READER(fn)                                \
    unsigned long long fn(void*, unsigned* count) {          \
        if (count) *count = 0;                               \
        return 0;                                            \
    }
#endif

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

// ---- exact sums on the integer pipes -----------------------------------------
// FP64 is the scarce unit on this part (a warp FP64 instruction occupies a
// sub-partition's FP64 unit for ~76 cycles whatever the number of active
// lanes), so the dot-product reductions of the CG run in exact fixed point on
// the integer units instead.  A set of doubles is summed at a common binary
// scale: with F the largest biased exponent field of the set, value
// v = +-M 2^(f - 1075) (M the 53-bit significand, f >= 1) becomes the integer
// q = +-trunc(M 2^(f - F + 48)), i.e. v = q 2^(F - 1123) up to a truncation
// below 2^(F - 1123), 2^-101 of the largest term.  |q| < 2^101, so sums of up
// to 2^26 terms fit a signed 128-bit integer.  Integer addition is exact and
// associative: a sum does not depend on its order or grouping.  A field of
// 2047 (Inf or NaN) makes the sum NaN.

// biased exponent field (denormals and zero count as 1)
__device__ __forceinline__ int xs_field(double v) {
    const int f = (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff;
    return f < 1 ? 1 : f;
}

// 128-bit integers are handled as two 64-bit halves: variable shifts and the
// final rounding run as a few 64-bit integer instructions, and nothing here
// issues on the FP64 pipe, which the product warps keep busy meanwhile.
__device__ __forceinline__ __int128 xs_make(unsigned long long hi, unsigned long long lo) {
    return (__int128)(((unsigned __int128)hi << 64) | lo);
}

// q >> d (arithmetic), 0 <= d <= 126
__device__ __forceinline__ __int128 xs_sar(__int128 q, int d) {
    const long long hi = (long long)((unsigned __int128)q >> 64);
    const unsigned long long lo = (unsigned long long)q;
    if (d == 0) return q;
    if (d < 64)
        return xs_make((unsigned long long)(hi >> d), (lo >> d) | ((unsigned long long)hi << (64 - d)));
    return xs_make((unsigned long long)(hi >> 63), (unsigned long long)(hi >> (d - 64)));
}

// v as a signed fixed-point integer at the scale of field F (F >= field of v)
__device__ __forceinline__ __int128 xs_fixed(double v, int F) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int f = (int)(bits >> 52) & 0x7ff;
    const unsigned long long mant = (bits & 0xfffffffffffffull) | (f > 0 ? (1ull << 52) : 0ull);
    const int sh = 48 - (F - (f < 1 ? 1 : f));
    unsigned long long hi = 0, lo;
    if (sh >= 0) {          // sh <= 48: mant << sh spans both halves
        lo = mant << sh;
        hi = sh > 0 ? mant >> (64 - sh) : 0ull;
    } else {
        lo = -sh >= 53 ? 0ull : mant >> -sh;
    }
    if (bits >> 63) {       // two's complement negation
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    return xs_make(hi, lo);
}

// exact warp sum of a signed 128-bit value (full warp): seven limbs summed
// with the integer warp reduction, the top limb signed
__device__ __forceinline__ __int128 xs_warp_sum(__int128 q) {
    const unsigned __int128 u = (unsigned __int128)q;
    unsigned __int128 tot = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const unsigned limb = (unsigned)(u >> (20 * k)) & 0xfffffu;
        tot += (unsigned __int128)__reduce_add_sync(0xffffffffu, limb) << (20 * k);
    }
    const int top = (int)(q >> 120);
    tot += (unsigned __int128)(__int128)__reduce_add_sync(0xffffffffu, top) << 120;
    return (__int128)tot;
}

// q 2^(F - 1123) rounded to the nearest double (ties to even).  A normal
// result is assembled from its bits with integer instructions; subnormal and
// overflowing results take ldexp.
__device__ __forceinline__ double xs_to_double(__int128 q, int F) {
    if (F >= 2047) return __longlong_as_double(0x7ff8000000000000ll);
    if (q == 0) return 0.0;
    const bool neg = q < 0;
    unsigned long long hi = (unsigned long long)((unsigned __int128)q >> 64);
    unsigned long long lo = (unsigned long long)q;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const int L = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long mant;
    int e = F - 1123;
    if (L <= 52) {
        mant = lo;
    } else {
        const int sh = L - 52;     // 1 .. 75: drop sh bits, round to nearest even
        bool up;
        if (sh < 64) {
            mant = (lo >> sh) | (hi << (64 - sh));
            const unsigned long long r = lo & ((1ull << sh) - 1ull), h = 1ull << (sh - 1);
            up = r > h || (r == h && (mant & 1ull));
        } else {
            mant = hi >> (sh - 64);
            const unsigned long long rh = hi & ((1ull << (sh - 64)) - 1ull), rl = lo;
            const unsigned long long hh = sh == 64 ? 0ull : 1ull << (sh - 65);
            const unsigned long long hl = sh == 64 ? 1ull << 63 : 0ull;
            const bool gt = rh > hh || (rh == hh && rl > hl);
            const bool eq = rh == hh && rl == hl;
            up = gt || (eq && (mant & 1ull));
        }
        if (up) ++mant;
        e += sh;
    }
    const int lead = 63 - __clzll((long long)mant);     // mant <= 2^53
    const int biased = lead + e + 1023;
    if (biased >= 1 && biased <= 2046) {
        const unsigned long long frac =
            (lead <= 52 ? mant << (52 - lead) : mant >> (lead - 52)) & 0xfffffffffffffull;
        return __longlong_as_double(
            (long long)(((unsigned long long)biased << 52) | frac | (neg ? 1ull << 63 : 0ull)));
    }
    const double d = ldexp((double)mant, e);
    return neg ? -d : d;
}

// Exact sum of two values per thread over the block.  Every thread gets the
// block's exponent fields Fa, Fb; warp 0 gets the block sums qa, qb (at those
// scales) in all its lanes.  scratch: >= 2 * 32 ints and 2 * 32 int128.
struct XsScratch {
    int fmax[64];
    __int128 q[64];
};
__device__ __forceinline__ void xs_block_sum2(double a, double b, XsScratch& X, int& Fa, int& Fb,
                                              __int128& qa, __int128& qb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int fa = __reduce_max_sync(0xffffffffu, xs_field(a));
    int fb = __reduce_max_sync(0xffffffffu, xs_field(b));
    if (lane == 0) {
        X.fmax[wid] = fa;
        X.fmax[32 + wid] = fb;
    }
    __syncthreads();
    fa = __reduce_max_sync(0xffffffffu, lane < nw ? X.fmax[lane] : 1);
    fb = __reduce_max_sync(0xffffffffu, lane < nw ? X.fmax[32 + lane] : 1);
    const __int128 sa = xs_warp_sum(xs_fixed(a, fa));
    const __int128 sb = xs_warp_sum(xs_fixed(b, fb));
    if (lane == 0) {
        X.q[wid] = sa;
        X.q[32 + wid] = sb;
    }
    __syncthreads();
    Fa = fa;
    Fb = fb;
    qa = qb = 0;
    if (wid == 0) {
        qa = xs_warp_sum(lane < nw ? X.q[lane] : (__int128)0);
        qb = xs_warp_sum(lane < nw ? X.q[32 + lane] : (__int128)0);
    }
}

// Record of one block's exact partial sums, as published for a group sum
// (48 bytes, 16-byte aligned).
struct __align__(16) XsRecord {
    unsigned long long alo, ahi, blo, bhi;
    int fa, fb, pad0, pad1;
};
__device__ __forceinline__ XsRecord xs_load_cg(const XsRecord* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 a = __ldcg(q), b = __ldcg(q + 1);
    const int4 c = __ldcg(reinterpret_cast<const int4*>(q + 2));
    XsRecord r;
    r.alo = a.x; r.ahi = a.y; r.blo = b.x; r.bhi = b.y;
    r.fa = c.x; r.fb = c.y; r.pad0 = 0; r.pad1 = 0;
    return r;
}
__device__ __forceinline__ void xs_store(XsRecord* r, int fa, int fb, __int128 qa, __int128 qb) {
    r->alo = (unsigned long long)qa;
    r->ahi = (unsigned long long)((unsigned __int128)qa >> 64);
    r->blo = (unsigned long long)qb;
    r->bhi = (unsigned long long)((unsigned __int128)qb >> 64);
    r->fa = fa;
    r->fb = fb;
}

// Exact totals of n records, computed by warps 0 and 1 together (all 64
// threads call it; all get the result).  The common field is the largest block
// field; block sums are aligned by an arithmetic right shift (truncation below
// 2^-101 of the largest term) and added.  Thread t takes records t, t + 64, ...:
// up to 64 * kXsInFlight records are loaded once, every load issued before the
// first is used, and reduced from registers (one memory round trip, not one per
// record and pass); larger groups take two passes.  The two warps exchange their
// largest fields and partial sums through X and a 64-thread named barrier.
// Integer addition is exact, so the totals do not depend on the split.
constexpr int kXsInFlight = 3;

__device__ __forceinline__ void xs_pair_barrier() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

__device__ __forceinline__ void xs_accumulate(const XsRecord& r, int fa, int fb, __int128& sa,
                                              __int128& sb) {
    const __int128 qa = xs_make(r.ahi, r.alo);
    const __int128 qb = xs_make(r.bhi, r.blo);
    const int da = fa - r.fa, db = fb - r.fb;
    sa += da >= 127 ? (qa < 0 ? (__int128)-1 : (__int128)0) : xs_sar(qa, da);
    sb += db >= 127 ? (qb < 0 ? (__int128)-1 : (__int128)0) : xs_sar(qb, db);
}

template <class Load>
__device__ __forceinline__ void xs_group_total(int n, Load&& load, XsScratch& X, double& ta,
                                               double& tb) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int fa = 1, fb = 1;
    __int128 sa = 0, sb = 0;
    auto exchange_fields = [&]() {
        fa = __reduce_max_sync(0xffffffffu, fa);
        fb = __reduce_max_sync(0xffffffffu, fb);
        if (lane == 0) {
            X.fmax[w] = fa;
            X.fmax[2 + w] = fb;
        }
        xs_pair_barrier();
        fa = max(X.fmax[0], X.fmax[1]);
        fb = max(X.fmax[2], X.fmax[3]);
    };
    if (n <= 64 * kXsInFlight) {
        XsRecord r[kXsInFlight];
#pragma unroll
        for (int k = 0; k < kXsInFlight; ++k) {
            if (t + 64 * k < n) {
                r[k] = load(t + 64 * k);
            } else {
                r[k].alo = r[k].ahi = r[k].blo = r[k].bhi = 0ull;
                r[k].fa = r[k].fb = 1;
            }
        }
#pragma unroll
        for (int k = 0; k < kXsInFlight; ++k) {
            fa = max(fa, r[k].fa);
            fb = max(fb, r[k].fb);
        }
        exchange_fields();
#pragma unroll
        for (int k = 0; k < kXsInFlight; ++k) xs_accumulate(r[k], fa, fb, sa, sb);
    } else {
        for (int i = t; i < n; i += 64) {
            const XsRecord r = load(i);
            fa = max(fa, r.fa);
            fb = max(fb, r.fb);
        }
        exchange_fields();
        for (int i = t; i < n; i += 64) xs_accumulate(load(i), fa, fb, sa, sb);
    }
    sa = xs_warp_sum(sa);
    sb = xs_warp_sum(sb);
    if (lane == 0) {
        X.q[w] = sa;
        X.q[2 + w] = sb;
    }
    xs_pair_barrier();
    ta = xs_to_double(X.q[0] + X.q[1], fa);
    tb = xs_to_double(X.q[2] + X.q[3], fb);
}

}  // namespace sdc
