// P1 finite-element assembly on the device (Sec. 2.2, eq. abstract monodomain):
//   K = sum_e sbar_e |e| G_e^T D_e G_e,   m_i = sum_{e containing i} |e| / (d + 1).
//
// The host builds the integer structure (node-to-element lists and the CSR
// pattern of K).  One device thread per row then accumulates that row's values
// over the elements containing the node, in ascending element order, so the
// result is deterministic.  A second pass drops off-diagonal entries that are
// rounding residue of cancelling element terms (|K_ij| <= drop_rel sqrt(K_ii K_jj);
// on Kuhn and right-triangle meshes with a diagonal tensor these couplings are
// exactly zero in exact arithmetic) and packs the off-diagonals into
// column-major ELL slots, the diagonal into its own vector.

#include <algorithm>
#include <cstdio>
#include <numeric>

#include "device_common.cuh"
#include "sdc_internal.h"

namespace sdc {
namespace {

__global__ void k_assemble_rows(int N, int dim, const double* __restrict__ xyz,
                                const int* __restrict__ elem, const int* __restrict__ n2e_ptr,
                                const int* __restrict__ n2e, const int* __restrict__ n2e_loc,
                                const double* __restrict__ sigma9,
                                const double* __restrict__ esig9,
                                const double* __restrict__ scale, const int* __restrict__ rp,
                                const int* __restrict__ ci, double* __restrict__ val,
                                double* __restrict__ mass, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int nv = dim + 1;
    const int r0 = rp[i], r1 = rp[i + 1];
    for (int k = r0; k < r1; ++k) val[k] = 0.0;
    double msum = 0.0;
    for (int k = n2e_ptr[i]; k < n2e_ptr[i + 1]; ++k) {
        const int e = n2e[k];
        const int a = n2e_loc[k];
        const int* vt = elem + (size_t)e * nv;
#if SDC_CHECKED
        bool bad = false;
        for (int b = 0; b < nv; ++b) bad |= sdc_idx(vt[b], N, 301) != vt[b];
        if (bad) return;
#endif
        double grad[4][3];
        double vol;
        if (!p1_gradients(dim, xyz, vt, grad, vol)) {
            raise_error(err, SDC_E_INVALID);
            return;
        }
        const double* D = esig9 ? esig9 + (size_t)e * 9 : sigma9;
        double sbar = 1.0;
        if (scale) {
            double s = 0.0;
            for (int b = 0; b < nv; ++b) s += scale[vt[b]];
            sbar = s / nv;
        }
        msum += vol / nv;
        // D grad_a (the row's own basis function)
        double Dg[3] = {0, 0, 0};
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) Dg[c] += grad[a][r] * D[r * 3 + c];
        const double w = sbar * vol;
        for (int b = 0; b < nv; ++b) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += Dg[c] * grad[b][c];
            const int j = vt[b];
            // binary search of column j in the row's sorted pattern
            int lo = r0, hi = r1 - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ci[mid] < j) lo = mid + 1; else hi = mid;
            }
            val[lo] += w * s;
        }
    }
    mass[i] = msum;
}

__global__ void k_diag(int N, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ val, double* __restrict__ kdiag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) d = val[k];
    kdiag[i] = d;
}

__device__ __forceinline__ bool keep_entry(double v, double di, double dj, double drop_rel) {
    return fabs(v) > drop_rel * sqrt(fabs(di * dj));
}

__global__ void k_ell_count(int N, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ val, const double* __restrict__ kdiag,
                            double drop_rel, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (j != i && keep_entry(val[k], kdiag[i], kdiag[j], drop_rel)) ++c;
    }
    cnt[i] = c;
}

__global__ void k_ell_fill(int N, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ val, const double* __restrict__ kdiag,
                           double drop_rel, int ld, double* __restrict__ ev,
                           int* __restrict__ ec, int* __restrict__ el) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int t = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (j != i && keep_entry(val[k], kdiag[i], kdiag[j], drop_rel)) {
            ev[(size_t)t * ld + i] = val[k];
            ec[(size_t)t * ld + i] = j;
            ++t;
        }
    }
    el[i] = t;
}

template <class T>
int upload(T** d, const std::vector<T>& h, cudaStream_t s) {
    if (cudaMalloc((void**)d, std::max<size_t>(1, h.size()) * sizeof(T)) != cudaSuccess)
        return SDC_E_NOMEM;
    if (!h.empty() &&
        cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SDC_E_CUDA;
    return SDC_OK;
}

}  // namespace

int assemble_device(const sdc_mesh& mesh, double drop_rel, cudaStream_t s, AssemblyOut& out,
                    std::string& why) {
    const int N = mesh.n_nodes, dim = mesh.dim, nv = dim + 1, NE = mesh.n_elems;
    // --- host: flattened connectivity and node -> element lists (ascending e)
    std::vector<int> elem((size_t)NE * nv);
    for (int e = 0; e < NE; ++e)
        for (int a = 0; a < nv; ++a) elem[(size_t)e * nv + a] = mesh.elem_node[mesh.elem_ptr[e] + a];
    std::vector<int> n2e_ptr(N + 1, 0);
    for (int v : elem) n2e_ptr[v + 1]++;
    for (int i = 0; i < N; ++i) n2e_ptr[i + 1] += n2e_ptr[i];
    std::vector<int> fill(n2e_ptr.begin(), n2e_ptr.end() - 1), n2e(elem.size()), n2e_loc(elem.size());
    for (int e = 0; e < NE; ++e)
        for (int a = 0; a < nv; ++a) {
            const int v = elem[(size_t)e * nv + a];
            n2e[fill[v]] = e;
            n2e_loc[fill[v]] = a;
            fill[v]++;
        }
    // --- host: CSR pattern (sorted unique neighbours incl. the node itself)
    std::vector<int> rp(N + 1, 0), ci;
    ci.reserve((size_t)N * (dim == 3 ? 15 : 7));
    std::vector<int> nb;
    for (int i = 0; i < N; ++i) {
        nb.clear();
        for (int k = n2e_ptr[i]; k < n2e_ptr[i + 1]; ++k) {
            const int e = n2e[k];
            for (int b = 0; b < nv; ++b) nb.push_back(elem[(size_t)e * nv + b]);
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        if (nb.empty()) {
            why = "node " + std::to_string(i) + " belongs to no element";
            return SDC_E_INVALID;
        }
        ci.insert(ci.end(), nb.begin(), nb.end());
        rp[i + 1] = (int)ci.size();
    }
    const long long nnz = (long long)ci.size();

    // --- device buffers
    double *d_xyz = nullptr, *d_sig = nullptr, *d_esig = nullptr, *d_scale = nullptr,
           *d_val = nullptr;
    int *d_elem = nullptr, *d_n2e_ptr = nullptr, *d_n2e = nullptr, *d_n2e_loc = nullptr,
        *d_rp = nullptr, *d_ci = nullptr, *d_err = nullptr, *d_cnt = nullptr;
    int rc = SDC_OK;
    auto chk = [&](int r) { if (rc == SDC_OK && r != SDC_OK) rc = r; };
    chk(upload(&d_xyz, std::vector<double>(mesh.xyz, mesh.xyz + (size_t)N * dim), s));
    std::vector<double> sig9(9, 0.0);
    if (mesh.sigma) std::copy(mesh.sigma, mesh.sigma + 9, sig9.begin());
    chk(upload(&d_sig, sig9, s));
    if (mesh.elem_sigma)
        chk(upload(&d_esig, std::vector<double>(mesh.elem_sigma, mesh.elem_sigma + (size_t)NE * 9), s));
    if (mesh.dof_scale)
        chk(upload(&d_scale, std::vector<double>(mesh.dof_scale, mesh.dof_scale + N), s));
    chk(upload(&d_elem, elem, s));
    chk(upload(&d_n2e_ptr, n2e_ptr, s));
    chk(upload(&d_n2e, n2e, s));
    chk(upload(&d_n2e_loc, n2e_loc, s));
    chk(upload(&d_rp, rp, s));
    chk(upload(&d_ci, ci, s));
    if (rc == SDC_OK && cudaMalloc(&d_val, nnz * sizeof(double)) != cudaSuccess) rc = SDC_E_NOMEM;
    if (rc == SDC_OK && cudaMalloc(&out.kdiag, N * sizeof(double)) != cudaSuccess) rc = SDC_E_NOMEM;
    if (rc == SDC_OK && cudaMalloc(&out.mass, N * sizeof(double)) != cudaSuccess) rc = SDC_E_NOMEM;
    if (rc == SDC_OK && cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) rc = SDC_E_NOMEM;
    if (rc == SDC_OK && cudaMalloc(&d_cnt, N * sizeof(int)) != cudaSuccess) rc = SDC_E_NOMEM;
    int maxw = 0;
    if (rc == SDC_OK) {
        cudaMemsetAsync(d_err, 0, sizeof(int), s);
        const int bs = 128, gs = (N + bs - 1) / bs;
        k_assemble_rows<<<gs, bs, 0, s>>>(N, dim, d_xyz, d_elem, d_n2e_ptr, d_n2e, d_n2e_loc,
                                          d_sig, d_esig, d_scale, d_rp, d_ci, d_val, out.mass, d_err);
        k_diag<<<gs, bs, 0, s>>>(N, d_rp, d_ci, d_val, out.kdiag);
        k_ell_count<<<gs, bs, 0, s>>>(N, d_rp, d_ci, d_val, out.kdiag, drop_rel, d_cnt);
        std::vector<int> cnt(N);
        int herr = 0;
        cudaMemcpyAsync(cnt.data(), d_cnt, N * sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            rc = SDC_E_CUDA;
            why = std::string("assembly: ") + cudaGetErrorString(cudaGetLastError());
        } else if (herr != 0) {
            rc = SDC_E_INVALID;
            why = "assembly: degenerate element (zero or non-finite Jacobian determinant)";
        } else {
            long long kept = 0;
            for (int c : cnt) { maxw = std::max(maxw, c); kept += c; }
            out.nnz = kept + N;
            Ell& K = out.K;
            K.ld = (N + 31) / 32 * 32;
            K.width = std::max(maxw, 1);
            if (cudaMalloc(&K.val, (size_t)K.width * K.ld * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&K.col, (size_t)K.width * K.ld * sizeof(int)) != cudaSuccess ||
                cudaMalloc(&K.len, (size_t)K.ld * sizeof(int)) != cudaSuccess) {
                rc = SDC_E_NOMEM;
            } else {
                cudaMemsetAsync(K.len, 0, (size_t)K.ld * sizeof(int), s);
                k_ell_fill<<<gs, bs, 0, s>>>(N, d_rp, d_ci, d_val, out.kdiag, drop_rel, K.ld,
                                              K.val, K.col, K.len);
                // a node with no positive mass or diagonal cannot be integrated
                std::vector<double> hm(N), hd(N);
                cudaMemcpyAsync(hm.data(), out.mass, N * sizeof(double), cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(hd.data(), out.kdiag, N * sizeof(double), cudaMemcpyDeviceToHost, s);
                if (cudaStreamSynchronize(s) != cudaSuccess) {
                    rc = SDC_E_CUDA;
                    why = std::string("assembly: ") + cudaGetErrorString(cudaGetLastError());
                } else {
                    for (int i = 0; i < N && rc == SDC_OK; ++i)
                        if (!(hm[i] > 0.0) || !(hd[i] >= 0.0)) {
                            rc = SDC_E_INVALID;
                            why = "assembly: node " + std::to_string(i) +
                                  " has non-positive lumped mass or negative K_ii";
                        }
                }
            }
        }
    } else if (why.empty()) {
        why = "assembly: device allocation or copy failed";
    }
    MeshDev& md = out.mesh;
    md.dim = dim;
    md.n_nodes = N;
    md.n_elems = NE;
    md.nnz_pattern = nnz;
    md.xyz = d_xyz; md.sig = d_sig; md.esig = d_esig; md.scale = d_scale;
    md.elem = d_elem; md.n2e_ptr = d_n2e_ptr; md.n2e = d_n2e; md.n2e_loc = d_n2e_loc;
    md.rp = d_rp; md.ci = d_ci;
    if (rc != SDC_OK) free_mesh_dev(md);
    cudaFree(d_val); cudaFree(d_err); cudaFree(d_cnt);
    return rc;
}

void free_mesh_dev(MeshDev& m) {
    cudaFree(m.xyz); cudaFree(m.sig); cudaFree(m.esig); cudaFree(m.scale);
    cudaFree(m.elem); cudaFree(m.n2e_ptr); cudaFree(m.n2e); cudaFree(m.n2e_loc);
    cudaFree(m.rp); cudaFree(m.ci);
    m = MeshDev();
}

int reassemble_device(AssemblyOut& out, const double* h_scale, double drop_rel, cudaStream_t s,
                      std::string& why) {
    MeshDev& md = out.mesh;
    const int N = md.n_nodes;
    if (!md.rp) {
        why = "re-assembly: mesh not kept";
        return SDC_E_INVALID;
    }
    if (h_scale) {
        if (!md.scale && cudaMalloc(&md.scale, N * sizeof(double)) != cudaSuccess) return SDC_E_NOMEM;
        cudaMemcpyAsync(md.scale, h_scale, N * sizeof(double), cudaMemcpyHostToDevice, s);
    } else if (md.scale) {
        cudaFree(md.scale);
        md.scale = nullptr;
    }
    double* d_val = nullptr;
    int *d_err = nullptr, *d_cnt = nullptr;
    if (cudaMalloc(&d_val, md.nnz_pattern * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_cnt, N * sizeof(int)) != cudaSuccess) {
        cudaFree(d_val); cudaFree(d_err); cudaFree(d_cnt);
        return SDC_E_NOMEM;
    }
    int rc = SDC_OK;
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    const int bs = 128, gs = (N + bs - 1) / bs;
    k_assemble_rows<<<gs, bs, 0, s>>>(N, md.dim, md.xyz, md.elem, md.n2e_ptr, md.n2e, md.n2e_loc,
                                      md.sig, md.esig, md.scale, md.rp, md.ci, d_val, out.mass,
                                      d_err);
    k_diag<<<gs, bs, 0, s>>>(N, md.rp, md.ci, d_val, out.kdiag);
    k_ell_count<<<gs, bs, 0, s>>>(N, md.rp, md.ci, d_val, out.kdiag, drop_rel, d_cnt);
    std::vector<int> cnt(N);
    int herr = 0;
    cudaMemcpyAsync(cnt.data(), d_cnt, N * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        rc = SDC_E_CUDA;
        why = std::string("re-assembly: ") + cudaGetErrorString(cudaGetLastError());
    } else if (herr != 0) {
        rc = SDC_E_INVALID;
        why = "re-assembly: degenerate element";
    } else {
        long long kept = 0;
        int maxw = 0;
        for (int c : cnt) { maxw = std::max(maxw, c); kept += c; }
        if (maxw > out.K.width) {
            rc = SDC_E_INVALID;
            why = "re-assembly: the new scale stores more off-diagonals per row than the context";
        } else {
            out.nnz = kept + N;
            cudaMemsetAsync(out.K.len, 0, (size_t)out.K.ld * sizeof(int), s);
            k_ell_fill<<<gs, bs, 0, s>>>(N, md.rp, md.ci, d_val, out.kdiag, drop_rel, out.K.ld,
                                          out.K.val, out.K.col, out.K.len);
            if (cudaStreamSynchronize(s) != cudaSuccess) rc = SDC_E_CUDA;
        }
    }
    cudaFree(d_val); cudaFree(d_err); cudaFree(d_cnt);
    return rc;
}

}  // namespace sdc

namespace sdc {
SDC_CHECK_READER(check_take_assembly)
}  // namespace sdc
