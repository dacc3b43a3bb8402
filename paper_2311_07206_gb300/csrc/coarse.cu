// Two-level preconditioner of the cell-by-cell node solves (Sec. 6 proposes block
// preconditioning, with a selection of the blocks, for EMI systems).
//
// The caller labels every dof with a block (each cell, and pieces of the
// extracellular space).  For a node system A restricted to the active set I, the
// coarse space Z holds the indicator vectors of the blocks with active dofs (the
// block selection: a block without active dofs contributes nothing), E = Z' A Z, and
// the preconditioner is the additive two-level one
//     z = D^-1 r + Z E^-1 Z' r.
// The Jacobi part alone leaves the near-constant modes of the floating cells and the
// long-wavelength modes of the extracellular space to CG; the coarse part takes them.
//
// Work per sweep (the active set is fixed over the M node solves of a sweep):
//   - lab_c: the block of each compact row;
//   - crow: the compact rows sorted by (block, row), a stable compaction of the dofs
//     sorted by (block, dof) (set up once) by the active flag; boff: block ranges;
//   - the rows of the CG launch: the positions of crow in tiles of kCoarseTile, tile j
//     on CTA j mod G (the whole grid sweeps one window of the vectors at a time, as the
//     Jacobi kernels do); each tile cut at the block boundaries into pieces, numbered
//     in position order, so that the pieces of a block are contiguous (host).
// Work per node solve:
//   - E = Z' A Z accumulated in 64-bit fixed point (terms rounded at 2^-41 of the
//     largest diagonal entry; integer sums are exact, so E does not depend on the
//     order of the atomic additions), then converted;
//   - E^-1 by Gauss-Jordan elimination (E is symmetric positive definite: no
//     pivoting), kInvPanel pivots per step and one grid barrier per step, in one
//     cooperative launch.
// The CG itself is k_pcgcs_coarse (step.cu).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "sdc_internal.h"

namespace sdc {
namespace {

constexpr int kChunk = 1024;    // dofs per compaction chunk (= threads per block)
constexpr int kFracBits = 40;   // fixed-point fraction bits below the largest diagonal

inline int nb(int n, int b) { return (n + b - 1) / b; }

// lab_c[p] = lab[act[p]]
__global__ void k_coarse_labels(int n, const int* __restrict__ act, const int* __restrict__ lab,
                                int N, int* __restrict__ lab_c) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) lab_c[p] = lab[act ? sdc_idx(act[p], N, 80) : p];
}

// active dofs per chunk of gperm
__global__ void k_coarse_count(int N, const int* __restrict__ gperm, const int* __restrict__ pos,
                               int* __restrict__ cnt) {
    const int k = blockIdx.x * kChunk + threadIdx.x;
    const int on = k < N && pos[sdc_idx(gperm[k], N, 81)] >= 0;
    const int c = __syncthreads_count(on);
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// exclusive scan of the chunk counts (one block)
__global__ void k_coarse_scan(int nc, const int* __restrict__ cnt, int* __restrict__ off) {
    __shared__ int ssum[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (nc + T - 1) / T;
    const int c0 = t * per, c1 = min(nc, c0 + per);
    int local = 0;
    for (int c = c0; c < c1; ++c) local += cnt[c];
    ssum[t] = local;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const int v = t >= o ? ssum[t - o] : 0;
        __syncthreads();
        ssum[t] += v;
        __syncthreads();
    }
    int run = ssum[t] - local;
    for (int c = c0; c < c1; ++c) {
        off[c] = run;
        run += cnt[c];
    }
}

// crow[off + rank] = compact row of each active dof of gperm, in gperm order
__global__ void k_coarse_scatter(int N, const int* __restrict__ gperm, const int* __restrict__ pos,
                                 const int* __restrict__ off, int n, int* __restrict__ crow) {
    __shared__ int woff[32];
    const int k = blockIdx.x * kChunk + threadIdx.x;
    const int g = k < N ? sdc_idx(gperm[k], N, 82) : 0;
    const int p = k < N ? pos[g] : -1;
    const int on = p >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) woff[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        const int c = woff[lane];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        woff[lane] = incl - c;
    }
    __syncthreads();
    if (on) {
        const int at = off[blockIdx.x] + woff[wid] + __popc(bal & ((1u << lane) - 1u));
        crow[sdc_idx(at, n, 83)] = p;
    }
}

// boff[a] = first position k with lab_c[crow[k]] >= a (crow sorted by block)
__global__ void k_coarse_bounds(int q, int n, const int* __restrict__ crow,
                                const int* __restrict__ lab_c, int* __restrict__ boff) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a > q) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lab_c[crow[mid]] < a) lo = mid + 1; else hi = mid;
    }
    boff[a] = lo;
}

// largest diagonal entry of the node operator (positive: compared as bit patterns)
__global__ void k_coarse_dmax(int n, const double* __restrict__ mc, const double* __restrict__ J,
                              const double* __restrict__ kdc, double c,
                              unsigned long long* __restrict__ dmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
        const double d = mc[i] * (1.0 + c * J[i]) + c * kdc[i];
        if (d > 0.0 && isfinite(d)) v = (unsigned long long)__double_as_longlong(d);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v) atomicMax(dmax, v);
}

// 2^(kFracBits - e) for the largest diagonal 2^e <= dmax < 2^(e + 1)
__device__ __forceinline__ double fixed_scale(unsigned long long dmax_bits) {
    const int e = (int)((dmax_bits >> 52) & 0x7ff) - 1023;
    return ldexp(1.0, kFracBits - e);
}

__device__ __forceinline__ void fx_add(unsigned long long* p, double v, double scale) {
    const long long q = llrint(v * scale);
    if (q) atomicAdd(p, (unsigned long long)q);
}

// E = Z' A Z: per active row i of block a, (a, a) += d_i + c sum of its same-block
// off-diagonals; (a, b) += c a_ij for a slot whose column lies in block b != a
__global__ void k_coarse_E(int n, int q, const int* __restrict__ lab_c, const double* __restrict__ aval,
                           const int* __restrict__ acol, const int* __restrict__ alen, int ld,
                           const double* __restrict__ mc, const double* __restrict__ J,
                           const double* __restrict__ kdc, double c,
                           const unsigned long long* __restrict__ dmax,
                           unsigned long long* __restrict__ Eacc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = fixed_scale(*dmax);
    const int a = sdc_idx(lab_c[i], q, 84);
    double same = mc[i] * (1.0 + c * J[i]) + c * kdc[i];
    const int len = alen[i];
    for (int t = 0; t < len; ++t) {
        const size_t s = (size_t)t * ld + i;
        const int b = sdc_idx(lab_c[sdc_idx(acol[s], n, 85)], q, 86);
        const double v = c * aval[s];
        if (b == a) same += v;
        else fx_add(Eacc + (size_t)a * q + b, v, scale);
    }
    fx_add(Eacc + (size_t)a * q + a, same, scale);
}

// E from fixed point; a block without active rows gets a unit diagonal (decoupled)
__global__ void k_coarse_convert(int q, const unsigned long long* __restrict__ Eacc,
                                 const unsigned long long* __restrict__ dmax,
                                 const int* __restrict__ boff, double* __restrict__ E) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= q * q) return;
    const int a = k / q, b = k - a * q;
    const double inv = 1.0 / fixed_scale(*dmax);
    double v = (double)(long long)Eacc[k] * inv;
    if (boff[a + 1] == boff[a] || boff[b + 1] == boff[b]) v = a == b ? 1.0 : 0.0;
    E[k] = v;
}

// In-place Gauss-Jordan inversion of the q x q matrix E (row-major, symmetric positive
// definite: no pivoting), a panel of kInvPanel pivots at a time, rows owned cyclically
// by the CTAs.  Step K (pivot rows and columns K = [kb, kb + bk)), with P = E_KK^-1:
//     rows i outside K:  E_iJ <- E_iJ - E_iK P E_KJ   (J outside K),   E_iK <- -E_iK P;
//     rows of K:         E_KJ <- P E_KJ,   E_KK <- P.
// Every CTA forms P itself (scalar Gauss-Jordan on the bk x bk block in shared memory).
// The rows of K are read by every CTA during the step, so their owners write the new
// rows to T (two buffers, by step parity) and copy them back at the next step: one
// grid barrier per step.
constexpr int kInvPanel = 16;
constexpr int kInvThreads = 256;   // >= kInvPanel^2: one element of P per thread

__global__ void __launch_bounds__(kInvThreads) k_coarse_invert(int q, double* __restrict__ E,
                                                               double* __restrict__ T,
                                                               unsigned* bar, long long budget,
                                                               int* err) {
    __shared__ int ok;
    __shared__ double Pm[kInvPanel][kInvPanel + 1];
    __shared__ double piv;
    __shared__ double fv[kInvPanel];
    __shared__ double gv[kInvPanel];
    const int G = gridDim.x, c = blockIdx.x, t = threadIdx.x, NT = blockDim.x;
    unsigned epoch = 0;
    int pkb = 0, pbk = 0;    // the previous step's panel (pbk = 0: none)
    // the new values of the previous panel's row i (owned by this CTA) from T
    auto restore = [&](int i, const double* Tp) {
        const double* src = Tp + (size_t)(i - pkb) * q;
        double* row = E + (size_t)i * q;
        for (int j = t; j < q; j += NT) row[j] = __ldcg(src + j);
    };
    for (int kb = 0, step = 0; kb < q; kb += kInvPanel, ++step) {
        const int bk = min(kInvPanel, q - kb);
        const double* Tp = T + (size_t)((step + 1) & 1) * kInvPanel * q;
        double* Tc = T + (size_t)(step & 1) * kInvPanel * q;
        // P = E_KK^-1
        const int pi = t / bk, pj = t - pi * bk;
        const bool mine = t < bk * bk;
        if (mine) Pm[pi][pj] = __ldcg(E + (size_t)(kb + pi) * q + kb + pj);
        __syncthreads();
        for (int k = 0; k < bk; ++k) {
            if (t == 0) piv = 1.0 / Pm[k][k];
            __syncthreads();
            const double p = piv;
            double v = 0.0;
            if (mine) {
                if (pi == k) v = pj == k ? p : Pm[k][pj] * p;
                else v = pj == k ? -Pm[pi][k] * p : Pm[pi][pj] - Pm[pi][k] * (Pm[k][pj] * p);
            }
            __syncthreads();
            if (mine) Pm[pi][pj] = v;
            __syncthreads();
        }
        for (int i = c; i < q; i += G) {
            if (pbk && i >= pkb && i < pkb + pbk) {
                restore(i, Tp);
                __syncthreads();
            }
            double* row = E + (size_t)i * q;
            if (i >= kb && i < kb + bk) {
                // pivot row: (P E_K*)_r to T
                const int r = i - kb;
                double* dst = Tc + (size_t)r * q;
                for (int j = t; j < q; j += NT) {
                    double v;
                    if (j >= kb && j < kb + bk) {
                        v = Pm[r][j - kb];
                    } else {
                        v = 0.0;
                        for (int m = 0; m < bk; ++m) v += Pm[r][m] * __ldcg(E + (size_t)(kb + m) * q + j);
                    }
                    dst[j] = v;
                }
            } else {
                // g = -E_iK P, then E_iJ += g E_KJ
                if (t < bk) fv[t] = __ldcg(row + kb + t);
                __syncthreads();
                if (t < bk) {
                    double sum = 0.0;
                    for (int m = 0; m < bk; ++m) sum += fv[m] * Pm[m][t];
                    gv[t] = -sum;
                }
                __syncthreads();
                for (int j = t; j < q; j += NT) {
                    if (j >= kb && j < kb + bk) {
                        row[j] = gv[j - kb];
                    } else {
                        double v = __ldcg(row + j);
                        for (int m = 0; m < bk; ++m) v += gv[m] * __ldcg(E + (size_t)(kb + m) * q + j);
                        row[j] = v;
                    }
                }
            }
            __syncthreads();
        }
        pkb = kb;
        pbk = bk;
        if (!group_barrier(bar, G, epoch, budget, err, &ok)) return;
        if (kb + kInvPanel >= q) {
            // the last panel's rows
            const double* Tl = T + (size_t)(step & 1) * kInvPanel * q;
            for (int i = c; i < q; i += G)
                if (i >= pkb && i < pkb + pbk) restore(i, Tl);
        }
    }
}

}  // namespace

int coarse_setup(CoarseDev& C, const int* h_lab, int N, int q, int ld, int* err, cudaStream_t s,
                 std::string& why) {
    coarse_free(C);
    if (!h_lab || q < 1 || q > kMaxCoarseBlocks) {
        why = "coarse blocks: n_blocks must lie in [1, " + std::to_string(kMaxCoarseBlocks) + "]";
        return SDC_E_INVALID;
    }
    std::vector<int> cnt(q + 1, 0);
    for (int i = 0; i < N; ++i) {
        if (h_lab[i] < 0 || h_lab[i] >= q) {
            why = "coarse blocks: label of dof " + std::to_string(i) + " outside [0, n_blocks)";
            return SDC_E_INVALID;
        }
        ++cnt[h_lab[i] + 1];
    }
    // dofs sorted by (block, dof): a stable counting sort
    std::partial_sum(cnt.begin(), cnt.end(), cnt.begin());
    std::vector<int> gperm(N);
    for (int i = 0; i < N; ++i) gperm[cnt[h_lab[i]]++] = i;
    const int nc = nb(N, kChunk);
    const int G = pcg_sm_count();
    const int P = (ld + kCoarseTile - 1) / kCoarseTile + q;   // pieces: tiles + block boundaries
    auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 8)); };
    if (al((void**)&C.lab, (size_t)N * 4) || al((void**)&C.gperm, (size_t)N * 4) ||
        al((void**)&C.lab_c, (size_t)ld * 4) || al((void**)&C.crow, (size_t)ld * 4) ||
        al((void**)&C.boff, (size_t)(q + 1) * 4) || al((void**)&C.chunk_cnt, (size_t)nc * 4) ||
        al((void**)&C.chunk_off, (size_t)nc * 4) ||
        al((void**)&C.tp, (size_t)((ld + kCoarseTile - 1) / kCoarseTile + 1) * 4) ||
        al((void**)&C.nzb, (size_t)q * 4) || al((void**)&C.piece, (size_t)3 * P * 4) ||
        al((void**)&C.blk_ptr, (size_t)(q + 1) * 4) || al((void**)&C.tpiece, (size_t)P * 8) ||
        al((void**)&C.Eacc, (size_t)q * q * 8) ||
        al((void**)&C.Einv, (size_t)q * q * 8) || al((void**)&C.piv, (size_t)2 * kInvPanel * q * 8) ||
        al((void**)&C.dmax, 8) || al((void**)&C.bar, 8)) {
        coarse_free(C);
        why = "coarse blocks: device allocation failed";
        return SDC_E_NOMEM;
    }
    cudaMemcpyAsync(C.lab, h_lab, (size_t)N * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(C.gperm, gperm.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        coarse_free(C);
        why = "coarse blocks: upload failed";
        return SDC_E_CUDA;
    }
    C.q = q;
    C.N = N;
    C.Gmax = G;
    C.G = G;
    C.err = err;
    return SDC_OK;
}

void coarse_free(CoarseDev& C) {
    for (void* p : {(void*)C.lab, (void*)C.gperm, (void*)C.lab_c, (void*)C.crow, (void*)C.boff,
                    (void*)C.chunk_cnt, (void*)C.chunk_off, (void*)C.tp, (void*)C.piece,
                    (void*)C.blk_ptr, (void*)C.tpiece, (void*)C.nzb,
                    (void*)C.Eacc, (void*)C.Einv, (void*)C.piv, (void*)C.dmax,
                    (void*)C.bar})
        if (p) cudaFree(p);
    C = CoarseDev{};
}

int coarse_sweep(CoarseDev& C, int n, const int* act, const int* pos, int G, cudaStream_t s) {
    const int N = C.N, q = C.q, nc = nb(N, kChunk);
    if (n < 1) return SDC_OK;
    const int T = kCoarseTile, ntiles = nb(n, T);
    G = std::max(1, std::min({G, C.Gmax, ntiles}));
    k_coarse_labels<<<nb(n, 256), 256, 0, s>>>(n, act, C.lab, N, C.lab_c);
    k_coarse_count<<<nc, kChunk, 0, s>>>(N, C.gperm, pos, C.chunk_cnt);
    k_coarse_scan<<<1, 1024, 0, s>>>(nc, C.chunk_cnt, C.chunk_off);
    k_coarse_scatter<<<nc, kChunk, 0, s>>>(N, C.gperm, pos, C.chunk_off, n, C.crow);
    k_coarse_bounds<<<nb(q + 1, 256), 256, 0, s>>>(q, n, C.crow, C.lab_c, C.boff);
    C.h_boff.resize(q + 1);
    cudaMemcpyAsync(C.h_boff.data(), C.boff, (size_t)(q + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SDC_E_CUDA;
    if (C.h_boff[q] != n) return SDC_E_INVALID;   // every active row carries a block
    // pieces: the tiles cut at the block boundaries, in position order (so in block
    // order too, crow being sorted by block)
    C.h_tp.assign(ntiles + 1, 0);
    C.h_piece.clear();
    C.h_blk_ptr.assign(q + 1, 0);
    int a = 0;
    for (int j = 0; j < ntiles; ++j) {
        const int k0 = j * T, k1 = std::min(n, k0 + T);
        for (int k = k0; k < k1;) {
            while (C.h_boff[a + 1] <= k) ++a;
            const int e = std::min(k1, C.h_boff[a + 1]);
            C.h_piece.insert(C.h_piece.end(), {a, k, e});
            ++C.h_blk_ptr[a + 1];
            k = e;
        }
        C.h_tp[j + 1] = (int)(C.h_piece.size() / 3);
    }
    int pmax = 0;
    for (int b = 0; b < G; ++b) {
        int np = 0;
        for (int j = b; j < ntiles; j += G) np += C.h_tp[j + 1] - C.h_tp[j];
        pmax = std::max(pmax, np);
    }
    C.h_nzb.clear();
    for (int b = 0; b < q; ++b)
        if (C.h_blk_ptr[b + 1]) C.h_nzb.push_back(b);
    std::partial_sum(C.h_blk_ptr.begin(), C.h_blk_ptr.end(), C.h_blk_ptr.begin());
    cudaMemcpyAsync(C.tp, C.h_tp.data(), (size_t)(ntiles + 1) * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(C.blk_ptr, C.h_blk_ptr.data(), (size_t)(q + 1) * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(C.piece, C.h_piece.data(), C.h_piece.size() * 4, cudaMemcpyHostToDevice, s);
    if (!C.h_nzb.empty())
        cudaMemcpyAsync(C.nzb, C.h_nzb.data(), C.h_nzb.size() * 4, cudaMemcpyHostToDevice, s);
    C.G = G;
    C.ntiles = ntiles;
    C.tmax = nb(ntiles, G);
    C.qn = (int)C.h_nzb.size();
    C.pmax = pmax;
    C.ptot = (int)(C.h_piece.size() / 3);
    // the host vectors must outlive the copies
    return cudaStreamSynchronize(s) == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

int coarse_factor(CoarseDev& C, int n, const Ell& A, const double* mc, const double* J,
                  const double* kdc, double c, long long budget, cudaStream_t s) {
    const int q = C.q;
    cudaMemsetAsync(C.dmax, 0, 8, s);
    cudaMemsetAsync(C.Eacc, 0, (size_t)q * q * 8, s);
    k_coarse_dmax<<<nb(n, 256), 256, 0, s>>>(n, mc, J, kdc, c, C.dmax);
    k_coarse_E<<<nb(n, 128), 128, 0, s>>>(n, q, C.lab_c, A.val, A.col, A.len, A.ld, mc, J, kdc, c,
                                          C.dmax, C.Eacc);
    k_coarse_convert<<<nb(q * q, 256), 256, 0, s>>>(q, C.Eacc, C.dmax, C.boff, C.Einv);
    cudaMemsetAsync(C.bar, 0, sizeof(unsigned), s);
    const int G = std::max(1, std::min(q, pcg_sm_count()));
    int nq = q;
    double* E = C.Einv;
    double* piv = C.piv;
    unsigned* bar = C.bar;
    int* err = C.err;
    void* args[] = {&nq, &E, &piv, &bar, &budget, &err};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_coarse_invert, dim3(G),
                                                      dim3(kInvThreads), args, 0, s);
    return e == cudaSuccess ? SDC_OK : SDC_E_CUDA;
}

SDC_CHECK_READER(check_take_coarse)

}  // namespace sdc
