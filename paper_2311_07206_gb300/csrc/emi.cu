// Cell-by-cell (EMI) operator for the SDC step (Sec. 2.1; abstract form of Sec. 3):
//   B u' = -(K + diag(robin)) u - b(u, w),   w_p' = R(u_k - u_l, w_p) on cell-bath pairs,
//   B = sum_p area_p Cm (e_k - e_l)(e_k - e_l)^T,
//   b = sum_p area_p I_p(u_k - u_l, w_p) (e_k - e_l),  I_p = I_ion (membrane) or g_gap v (gap).
// The sweep is the monodomain one with B in place of the lumped mass and the
// pair Jacobian D = sum_p area_p dI_p/dv (e_k - e_l)(e_k - e_l)^T in place of
// the lumped ionic Jacobian.  For each node solve the restricted operator
//   B + c (K + D_m)  on I_k
// is written as one ELL matrix (K's restricted slots plus one slot per pair
// whose other end is active), so the same PCG kernels solve it.

#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "sdc_internal.h"

namespace sdc {
namespace {

inline int nbk(int n, int b) { return (n + b - 1) / b; }

// x[M] per entry <- x0 (the initial guess of every collocation node)
template <int M>
__global__ void k_emi_spread(int n, const double* __restrict__ x0, double* __restrict__ X) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
#pragma unroll
    for (int m = 0; m < M; ++m) X[(size_t)p * M + m] = x0[p];
}

// x <- value at the last node (tau_M = 1)
template <int M>
__global__ void k_emi_final(int n, const double* __restrict__ X, double* __restrict__ x) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    x[p] = X[(size_t)p * M + M - 1];
}

// node-interleaved [n][M] -> node-major [m][n]
template <int M>
__global__ void k_emi_nodes_out(int n, const double* __restrict__ X, double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
#pragma unroll
    for (int m = 0; m < M; ++m) out[(size_t)m * n + p] = X[(size_t)p * M + m];
}

// pair currents and their voltage derivatives at every collocation node
template <int M>
__global__ void k_emi_pair_eval(int NP, const int* __restrict__ pk, const int* __restrict__ pl,
                                const int* __restrict__ pkind, const double* __restrict__ V,
                                const double* __restrict__ Wp, Ionic ion, double g_gap,
                                int reaction_implicit, double* __restrict__ Ip,
                                double* __restrict__ Jp, int N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const int k = sdc_idx(pk[p], N, 101), l = sdc_idx(pl[p], N, 102), kind = pkind[p];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const double v = V[(size_t)k * M + m] - V[(size_t)l * M + m];
        double I, J;
        if (kind == 0) {
            const double w = Wp[(size_t)p * M + m];
            I = ap_I(ion, v, w);
            J = ap_dIdv(ion, v, w);
        } else {
            I = g_gap * v;
            J = g_gap;
        }
        Ip[(size_t)m * NP + p] = I;
        Jp[(size_t)m * NP + p] = reaction_implicit ? J : 0.0;
    }
}

template <int M>
__global__ void k_emi_residual(int n, const int* __restrict__ act, const double* __restrict__ kval,
                               const int* __restrict__ kcol, const int* __restrict__ klen, int ldk,
                               const double* __restrict__ kdiag, const double* __restrict__ robin,
                               const int* __restrict__ np_ptr,
                               const int* __restrict__ np_pid, const int* __restrict__ np_part,
                               const int* __restrict__ np_sign, const double* __restrict__ parea,
                               const double* __restrict__ Ip, int NP, const double* __restrict__ V,
                               const double* __restrict__ u0, double Cm, double dt, Coll co,
                               int ld, double* __restrict__ R, double* __restrict__ J,
                               double* __restrict__ kdc, int N) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int g = act ? sdc_idx(act[q], N, 103) : q;
    const double kd = kdiag[g] + (robin ? robin[g] : 0.0);
    double f[M], bt[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        f[m] = -kd * V[(size_t)g * M + m];
        bt[m] = 0.0;
    }
    const int len = klen[g];
    for (int t = 0; t < len; ++t) {
        const double a = kval[(size_t)t * ldk + g];
        const int j = sdc_idx(kcol[(size_t)t * ldk + g], N, 104);
#pragma unroll
        for (int m = 0; m < M; ++m) f[m] -= a * V[(size_t)j * M + m];
    }
    const double u0g = u0[g];
    for (int e = np_ptr[g]; e < np_ptr[g + 1]; ++e) {
        const int pid = sdc_idx(np_pid[e], NP, 105), j = sdc_idx(np_part[e], N, 106);
        const double A = parea[pid], s = (double)np_sign[e];
        const double du0 = u0g - u0[j];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            f[m] -= s * A * Ip[(size_t)m * NP + pid];
            bt[m] += A * Cm * (du0 - (V[(size_t)g * M + m] - V[(size_t)j * M + m]));
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        double qs = 0.0;
#pragma unroll
        for (int j = 0; j < M; ++j) qs += co.Q[m * kMaxM + j] * f[j];
        R[(size_t)m * ld + q] = bt[m] + dt * qs;
        J[(size_t)m * ld + q] = 0.0;
    }
    kdc[q] = kd;
}

// ELL of B + c (K + D_m) restricted to the active rows: K's restricted slots,
// then a slot -area (Cm + c J_p)/c for every pair whose other end is active;
// the pair part of the diagonal goes to mc (the PCG forms mc + c K_ii).
__global__ void k_emi_build(int n, const int* __restrict__ act, const double* __restrict__ aval,
                            const int* __restrict__ acol, const int* __restrict__ alen, int lda,
                            int ld,
                            const int* __restrict__ np_ptr, const int* __restrict__ np_pid,
                            const int* __restrict__ np_part, const double* __restrict__ parea,
                            const double* __restrict__ Jpm, const int* __restrict__ pos,
                            double Cm, double c, double* __restrict__ eval,
                            int* __restrict__ ecol, int* __restrict__ elen,
                            double* __restrict__ mc, unsigned long long* __restrict__ slots,
                            int N) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    int added = 0;
    if (q < n) {
    const int g = act ? sdc_idx(act[q], N, 107) : q;
    int cnt = alen[q];
    for (int t = 0; t < cnt; ++t) {
        eval[(size_t)t * ld + q] = aval[(size_t)t * lda + q];
        ecol[(size_t)t * ld + q] = sdc_idx(acol[(size_t)t * lda + q], n, 108);
    }
    double pd = 0.0;
    for (int e = np_ptr[g]; e < np_ptr[g + 1]; ++e) {
        const int pid = np_pid[e];
        const double coef = parea[pid] * (Cm + c * Jpm[pid]);
        pd += coef;
        const int jq = pos[sdc_idx(np_part[e], N, 109)];
        if (jq >= 0) {
            eval[(size_t)cnt * ld + q] = -coef / c;
            ecol[(size_t)cnt * ld + q] = jq;
            ++cnt;
            ++added;
        }
    }
    elen[q] = cnt;
    mc[q] = pd;
    }
    // pair slots stored (statistics): one atomic per warp
    if (slots) {
        const int tot = __reduce_add_sync(0xffffffffu, added);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(slots, (unsigned long long)tot);
    }
}

// b_m' -= dt Qhat_m'm ((K + D_m) dv_m) for the later nodes m' > m
__global__ void k_emi_couple(int n, const int* __restrict__ act, int m, int M,
                             const double* __restrict__ aval, const int* __restrict__ acol,
                             const int* __restrict__ alen, int lda, int ld,
                             const double* __restrict__ kdc,
                             const int* __restrict__ np_ptr, const int* __restrict__ np_pid,
                             const int* __restrict__ np_part, const double* __restrict__ parea,
                             const double* __restrict__ Jpm, const int* __restrict__ pos,
                             const double* __restrict__ x, double dt, Coll co,
                             double* __restrict__ R, int N) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int g = act ? sdc_idx(act[q], N, 110) : q;
    const double xq = x[q];
    double acc = kdc[q] * xq;
    const int len = alen[q];
    for (int t = 0; t < len; ++t)
        acc += aval[(size_t)t * lda + q] * x[sdc_idx(acol[(size_t)t * lda + q], n, 111)];
    for (int e = np_ptr[g]; e < np_ptr[g + 1]; ++e) {
        const int pid = np_pid[e];
        const int jq = pos[sdc_idx(np_part[e], N, 112)];
        acc += parea[pid] * Jpm[pid] * (xq - (jq >= 0 ? x[sdc_idx(jq, n, 113)] : 0.0));
    }
    for (int mm = m + 1; mm < M; ++mm) R[(size_t)mm * ld + q] -= dt * co.Qh[mm * kMaxM + m] * acc;
}

// gating sweep of the cell-bath pairs with an active end (LU-trick recursion
// of the w equation with the updated potentials)
template <int M>
__global__ void k_emi_wsweep(int NP, const int* __restrict__ pk, const int* __restrict__ pl,
                             const int* __restrict__ pkind, const int* __restrict__ pos,
                             const double* __restrict__ V, double* __restrict__ Wp,
                             const double* __restrict__ w0, double dt, Ionic ion, Coll co,
                             int* __restrict__ err, int N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const int k = sdc_idx(pk[p], N, 114), l = sdc_idx(pl[p], N, 115);
    if (pkind[p] != 0 || (pos[k] < 0 && pos[l] < 0)) return;
    double wm[M], gR[M], dR[M], e[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const double v = V[(size_t)k * M + m] - V[(size_t)l * M + m];
        wm[m] = Wp[(size_t)p * M + m];
        if (!(v + ion.mu2 > 0.0)) raise_error(err, SDC_E_DOMAIN);
        ap_R_dRdw(ion, v, wm[m], gR[m], dR[m]);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        double q = 0.0;
#pragma unroll
        for (int j = 0; j < M; ++j) q += co.Q[m * kMaxM + j] * gR[j];
        double acc = w0[p] + dt * q - wm[m];
#pragma unroll
        for (int j = 0; j < m; ++j) acc += dt * co.Qh[m * kMaxM + j] * dR[j] * e[j];
        const double den = 1.0 - dt * co.Qh[m * kMaxM + m] * dR[m];
        if (!(den > 0.0)) raise_error(err, SDC_E_DOMAIN);
        e[m] = acc / den;
    }
#pragma unroll
    for (int m = 0; m < M; ++m) Wp[(size_t)p * M + m] = wm[m] + e[m];
}

__global__ void k_pos_identity(int n, int* __restrict__ pos, int reset) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[i] = reset ? -1 : i;
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


template <class T>
bool dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) == cudaSuccess;
}

template <class T>
bool upload(T** p, const T* h, size_t count, cudaStream_t s) {
    return dalloc(p, count) &&
           cudaMemcpyAsync(*p, h, count * sizeof(T), cudaMemcpyHostToDevice, s) == cudaSuccess;
}

}  // namespace

int emi_setup(const sdc_emi& e, int N, int M, int k_width, int ld, cudaStream_t s, EmiDev& E,
              std::string& why) {
    const int NP = e.n_pairs;
    E.np = NP;
    E.Cm = e.Cm;
    E.g_gap = e.g_gap;
    // dof -> incident pairs, each dof's pairs in ascending pair order
    std::vector<int> ptr(N + 1, 0);
    for (int p = 0; p < NP; ++p) {
        ++ptr[e.pair_k[p] + 1];
        ++ptr[e.pair_l[p] + 1];
    }
    for (int i = 0; i < N; ++i) {
        E.max_inc = std::max(E.max_inc, ptr[i + 1]);
        ptr[i + 1] += ptr[i];
    }
    std::vector<int> fill(ptr.begin(), ptr.end() - 1), pid(2 * (size_t)NP), part(2 * (size_t)NP),
        sign(2 * (size_t)NP);
    for (int p = 0; p < NP; ++p) {
        const int k = e.pair_k[p], l = e.pair_l[p];
        int at = fill[k]++;
        pid[at] = p;
        part[at] = l;
        sign[at] = 1;
        at = fill[l]++;
        pid[at] = p;
        part[at] = k;
        sign[at] = -1;
    }
    const size_t width = (size_t)k_width + E.max_inc;
    bool ok = upload(&E.pk, e.pair_k, NP, s) && upload(&E.pl, e.pair_l, NP, s) &&
              upload(&E.pkind, e.pair_kind, NP, s) && upload(&E.parea, e.pair_area, NP, s) &&
              upload(&E.np_ptr, ptr.data(), N + 1, s) && upload(&E.np_pid, pid.data(), pid.size(), s) &&
              upload(&E.np_part, part.data(), part.size(), s) &&
              upload(&E.np_sign, sign.data(), sign.size(), s) &&
              dalloc(&E.Wp, (size_t)NP * M) && dalloc(&E.Ip, (size_t)NP * M) &&
              dalloc(&E.Jp, (size_t)NP * M) && dalloc(&E.A.val, width * ld) &&
              dalloc(&E.A.col, width * ld) && dalloc(&E.A.len, ld) && dalloc(&E.pos, N) &&
              dalloc(&E.wstage, NP) && dalloc(&E.slots, 1);
    if (ok && e.robin) ok = upload(&E.robin, e.robin, N, s);
    if (!ok) {
        why = "EMI buffer allocation failed";
        return SDC_E_NOMEM;
    }
    E.A.ld = ld;
    E.A.width = (int)width;
    cudaMemsetAsync(E.pos, 0xff, (size_t)N * sizeof(int), s);   // all -1
    // the host vectors above are pageable: finish the copies before they go
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        why = std::string("EMI setup: ") + cudaGetErrorString(cudaGetLastError());
        return SDC_E_CUDA;
    }
    return SDC_OK;
}

void emi_free(EmiDev& E) {
    int* ip[] = {E.pk, E.pl, E.pkind, E.np_ptr, E.np_pid, E.np_part, E.np_sign, E.A.col, E.A.len,
                 E.pos};
    for (int* p : ip) cudaFree(p);
    double* dp[] = {E.parea, E.robin, E.Wp, E.Ip, E.Jp, E.A.val, E.wstage};
    for (double* p : dp) cudaFree(p);
    cudaFree(E.slots);
    E = EmiDev();
}

void emi_nodes_out(const EmiDev& E, int N, int M, const double* V, double* d_V, double* d_W,
                   cudaStream_t s) {
    dispatch_M(M, [&](auto mc) {
        constexpr int MM = decltype(mc)::value;
        k_emi_nodes_out<MM><<<nbk(N, 256), 256, 0, s>>>(N, V, d_V);
        k_emi_nodes_out<MM><<<nbk(E.np, 256), 256, 0, s>>>(E.np, E.Wp, d_W);
    });
}

// One SDC step of the EMI system: the sweep structure of the monodomain step
// (residual, M node solves with LU-trick coupling, update, selection,
// restricted extraction) with the pair terms of Sec. 2.1.
int emi_step(const EmiStepArgs& a, double* d_u, double* d_w, double dt, int sweeps, double TOL,
             sdc_stats* stats) {
    StepBuffers& B = *a.B;
    EmiDev& E = *a.E;
    const int N = a.N, M = a.M, NP = E.np;
    const Coll& co = *a.co;
    cudaStream_t s = a.s;
    const double tol_drop = a.opt->alpha * TOL;
    // the a priori drop tolerance (drop rule 1) lives on the device from the first sweep on
    const double* drop_dev = a.opt->drop_rule && TOL > 0.0 ? &B.sc->tol_drop : nullptr;
    // the classical CG arrangement unless the pipelined one is asked for explicitly
    PcgConfig pcg = *a.pcg;
    pcg.pipelined = a.opt->cg_pipelined == 1;
    auto fail = [&](int st, const std::string& msg) {
        *a.err = msg;
        return st;
    };
    // kernel phases: launch counts always, device time with the profile option
    const bool prof = a.opt->profile != 0 && a.events;
    struct Mark { int phase, ea, eb, k, m; };
    std::vector<Mark> marks;
    int ev_used = 0, launches[SDC_N_PHASES] = {0, 0, 0, 0, 0};
    int cur_k = -1, cur_m = -1;
    auto next_event = [&]() -> int {
        if (ev_used == (int)a.events->size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            a.events->push_back(e);
        }
        return ev_used++;
    };
    auto run = [&](int phase, int nk, auto&& fn) {
        int ea = -1;
        if (prof) {
            ea = next_event();
            cudaEventRecord((*a.events)[ea], s);
        }
        fn();
        if (prof) {
            const int eb = next_event();
            cudaEventRecord((*a.events)[eb], s);
            marks.push_back({phase, ea, eb, cur_k, cur_m});
        }
        launches[phase] += nk;
    };

    cudaMemsetAsync(B.sc, 0, sizeof(DevScalars), s);
    const double big = 1.7976931348623157e308;
    cudaMemcpyAsync(&B.sc->margin, &big, sizeof(double), cudaMemcpyHostToDevice, s);
    run(SDC_PHASE_RESIDUAL, 2, [&] {
        dispatch_M(M, [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            k_emi_spread<MM><<<nbk(N, 256), 256, 0, s>>>(N, d_u, B.V);
            k_emi_spread<MM><<<nbk(NP, 256), 256, 0, s>>>(NP, d_w, E.Wp);
        });
    });

    int n = N;
    const int* act = nullptr;
    const Ell* A = &a.K->K;
    long long nnz = a.K->nnz - N;
    int cur = 0, status = SDC_OK;
    const bool estop = a.opt->energy_stop != 0;
    double energy_prev = 0.0;
    int k = 0;
    for (k = 0; k < sweeps; ++k) {
        (*a.n_act)[k] = n;
        if (stats) {
            stats->n_active[k] = n;
            stats->nnz_active[k] = nnz;
            stats->sweeps_run = k + 1;
        }
        if (n == 0) continue;
        cur_k = k;
        cur_m = -1;
        // compact positions of the current list (partners outside it read -1)
        run(SDC_PHASE_SELECT, 1, [&] {
            if (act) launch_pos_set(n, act, E.pos, 0, B.N, s);
            else k_pos_identity<<<nbk(N, 256), 256, 0, s>>>(N, E.pos, 0);
        });
        // the two-level preconditioner on this sweep's solves (enough active rows)
        CoarseDev* const coarse = a.coarse && n >= a.opt->coarse_min_rows ? a.coarse : nullptr;
        if (coarse) {
            // the blocks of this sweep's active set: rows by block, CTA ownership
            int rc = SDC_OK;
            run(SDC_PHASE_SELECT, 5, [&] { rc = coarse_sweep(*coarse, n, act, E.pos,
                                                             a.pcg->sms, s); });
            if (rc != SDC_OK) {
                status = fail(rc, "two-level preconditioner: block ordering failed");
                break;
            }
        }
        run(SDC_PHASE_RESIDUAL, 2, [&] {
            dispatch_M(M, [&](auto mc) {
                constexpr int MM = decltype(mc)::value;
                k_emi_pair_eval<MM><<<nbk(NP, 256), 256, 0, s>>>(
                    NP, E.pk, E.pl, E.pkind, B.V, E.Wp, *a.ion, E.g_gap, a.opt->reaction_implicit,
                    E.Ip, E.Jp, B.N);
                k_emi_residual<MM><<<nbk(n, 128), 128, 0, s>>>(
                    n, act, a.K->K.val, a.K->K.col, a.K->K.len, a.K->K.ld, a.K->kdiag, E.robin,
                    E.np_ptr, E.np_pid, E.np_part, E.np_sign, E.parea, E.Ip, NP, B.V, d_u, E.Cm,
                    dt, co, B.ld, B.R, B.J, B.kdc, B.N);
            });
        });
        cudaMemsetAsync(E.slots, 0, sizeof(unsigned long long), s);
        for (int m = 0; m < M && status == SDC_OK; ++m) {
            cur_m = m;
            const double c = dt * co.Qh[m * kMaxM + m];
            const double* Jm = E.Jp + (size_t)m * NP;
            run(SDC_PHASE_EXTRACT, 1, [&] {
                k_emi_build<<<nbk(n, 128), 128, 0, s>>>(
                    n, act, A->val, A->col, A->len, A->ld, B.ld, E.np_ptr, E.np_pid, E.np_part,
                    E.parea, Jm, E.pos, E.Cm, c, E.A.val, E.A.col, E.A.len, B.mc,
                    m == 0 ? E.slots : nullptr, B.N);
            });
            PcgRole role{};
            role.b = B.R + (size_t)m * B.ld;
            role.x = B.D + (size_t)m * B.ld;
            role.J = B.J + (size_t)m * B.ld;   // zero: the pair Jacobian is in mc and the slots
            role.Jall = B.J;
            role.R = B.R;
            role.epi_lo = role.epi_hi = 0;
            role.epi_target_J = 0;
            role.c = c;
            role.iters_out = &B.sc->cg_iters[k * kMaxM + m];
            role.relres_out = &B.sc->cg_relres[k * kMaxM + m];
            role.energy_out = &B.sc->cg_energy[k * kMaxM + m];
            if (coarse) {
                run(SDC_PHASE_EXTRACT, 4, [&] {
                    if (coarse_factor(*coarse, n, E.A, B.mc, role.J, B.kdc, c, pcg.budget, s) !=
                        SDC_OK)
                        status = fail(SDC_E_CUDA, std::string("coarse factorisation launch: ") +
                                                      cudaGetErrorString(cudaGetLastError()));
                });
                if (status != SDC_OK) break;
            }
            run(SDC_PHASE_PCG, 1, [&] {
                const int rc = coarse ? launch_pcg_coarse(n, E.A, role, a.opt->cg_rtol,
                                                          a.opt->cg_maxit, *coarse, pcg, B, s)
                                        : launch_pcg_role(n, E.A, role, dt, M, a.opt->cg_rtol,
                                                          a.opt->cg_maxit, pcg, B, s);
                if (rc != SDC_OK)
                    status = fail(rc == SDC_E_INVALID ? SDC_E_INVALID : SDC_E_CUDA,
                                  std::string("cooperative CG launch: ") +
                                      cudaGetErrorString(cudaGetLastError()));
            });
            if (status == SDC_OK && m + 1 < M) {
                cur_m = -1;
                run(SDC_PHASE_UPDATE, 1, [&] {
                    k_emi_couple<<<nbk(n, 128), 128, 0, s>>>(
                        n, act, m, M, A->val, A->col, A->len, A->ld, B.ld, B.kdc, E.np_ptr,
                        E.np_pid, E.np_part, E.parea, Jm, E.pos, B.D + (size_t)m * B.ld, dt, co,
                        B.R, B.N);
                });
            }
        }
        if (status != SDC_OK) break;
        cur_m = -1;
        if (k == 0 && drop_dev)
            run(SDC_PHASE_SELECT, 2, [&] {
                // eta from the pair Jacobians (membrane and gap junction) over C_m
                launch_drop_rule(n, M, B.D, B.ld, NP, E.Jp, NP, E.Cm, a.opt->sdc_rho, TOL, dt, B,
                                 s);
            });
        run(SDC_PHASE_UPDATE, a.opt->w_frozen ? 1 : 2, [&] {
            // u update and selection flags (no node gating: w_frozen), then the pair gating
            launch_update(M, n, act, nullptr, dt, *a.ion, co, tol_drop, 1, B, s, drop_dev);
            if (!a.opt->w_frozen)
                dispatch_M(M, [&](auto mc) {
                    constexpr int MM = decltype(mc)::value;
                    k_emi_wsweep<MM><<<nbk(NP, 256), 256, 0, s>>>(
                        NP, E.pk, E.pl, E.pkind, E.pos, B.V, E.Wp, d_w, dt, *a.ion, co,
                        &B.sc->err, B.N);
                });
        });
        int* next = (k + 1 < sweeps) ? (*a.act)[k + 1] : (*a.act)[0];
        run(SDC_PHASE_SELECT, 3, [&] {
            if (act) launch_pos_set(n, act, E.pos, 1, B.N, s);
            else k_pos_identity<<<nbk(N, 256), 256, 0, s>>>(N, E.pos, 1);
            launch_select(n, act, next, B, s);
        });
        unsigned long long slots = 0;
        cudaMemcpyAsync(&a.h_pin[0], &B.sc->count, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&a.h_pin[1], &B.sc->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&slots, E.slots, sizeof(slots), cudaMemcpyDeviceToHost, s);
        if (estop)
            cudaMemcpyAsync(reinterpret_cast<char*>(a.h_pin) + 16, &B.sc->cg_energy[k * kMaxM],
                            M * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            status = fail(SDC_E_CUDA, std::string("sweep: ") +
                                          cudaGetErrorString(cudaGetLastError()));
            break;
        }
        if (stats) stats->nnz_active[k] = nnz + (long long)slots;
        const int n_next = a.h_pin[0];
        if (a.h_pin[1] != SDC_OK) {
            status = fail(a.h_pin[1], "sweep " + std::to_string(k) + ": " +
                                          sdc_status_string(a.h_pin[1]));
            break;
        }
        if (estop) {
            // Sec. 3.2: the geometric series bounds the remaining energy-norm error
            const double* he = reinterpret_cast<const double*>(reinterpret_cast<char*>(a.h_pin) + 16);
            double En = 0.0;
            for (int m = 0; m < M; ++m) En += he[m];
            double rho = a.opt->sdc_rho;
            if (!(rho > 0.0)) rho = k > 0 && energy_prev > 0.0 ? std::sqrt(En / energy_prev) : 0.0;
            energy_prev = En;
            if (rho > 0.0 && rho < 1.0) {
                const double lim = (1.0 - rho) / rho * TOL;
                if (En <= lim * lim) {
                    ++k;
                    break;
                }
            }
        }
        if (k + 1 < sweeps && n_next > 0) {
            Ell& An = B.A[cur];
            run(SDC_PHASE_EXTRACT, 1, [&] { launch_extract(n, *A, B.map, An, B, s); });
            unsigned long long hn = 0;
            cudaMemcpyAsync(&hn, &B.sc->nnz, sizeof(hn), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                status = fail(SDC_E_CUDA, "extract");
                break;
            }
            nnz = (long long)hn;
            A = &An;
            cur ^= 1;
        }
        act = (k + 1 < sweeps) ? (*a.act)[k + 1] : nullptr;
        n = n_next;
    }
    if (status == SDC_OK) {
        cur_k = cur_m = -1;
        run(SDC_PHASE_RESIDUAL, 2, [&] {
            dispatch_M(M, [&](auto mc) {
                constexpr int MM = decltype(mc)::value;
                k_emi_final<MM><<<nbk(N, 256), 256, 0, s>>>(N, B.V, d_u);
                k_emi_final<MM><<<nbk(NP, 256), 256, 0, s>>>(NP, E.Wp, d_w);
            });
        });
        if (cudaStreamSynchronize(s) != cudaSuccess)
            status = fail(SDC_E_CUDA, std::string("EMI step: ") +
                                          cudaGetErrorString(cudaGetLastError()));
    }
    if (a.sweeps_done) *a.sweeps_done = status == SDC_OK ? std::min(k, sweeps) : sweeps;
    if (stats) {
        std::vector<int> it(SDC_MAX_SWEEPS * kMaxM);
        std::vector<double> rr(SDC_MAX_SWEEPS * kMaxM), en(SDC_MAX_SWEEPS * kMaxM);
        double mg = 0.0;
        cudaMemcpyAsync(it.data(), B.sc->cg_iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(rr.data(), B.sc->cg_relres, rr.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(en.data(), B.sc->cg_energy, en.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&mg, &B.sc->margin, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        for (int kk = 0; kk < stats->sweeps_run; ++kk) {
            double En = 0.0;
            for (int m = 0; m < M; ++m) En += en[kk * kMaxM + m];
            stats->energy[kk] = En;
        }
        stats->tol_drop = tol_drop;
        if (drop_dev) {
            cudaMemcpyAsync(&stats->tol_drop, drop_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
        }
        for (int kk = 0; kk < sweeps; ++kk)
            for (int m = 0; m < M; ++m) {
                stats->cg_iters[kk][m] = it[kk * kMaxM + m];
                stats->cg_relres_max = std::max(stats->cg_relres_max, rr[kk * kMaxM + m]);
            }
        stats->min_margin = mg >= big ? INFINITY : mg;
        stats->kernel_launches = 0;
        for (int ph = 0; ph < SDC_N_PHASES; ++ph) {
            stats->phase_launches[ph] = launches[ph];
            stats->kernel_launches += launches[ph];
            stats->phase_ms[ph] = 0.0;
        }
        for (const Mark& mk : marks) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, (*a.events)[mk.ea], (*a.events)[mk.eb]) == cudaSuccess) {
                stats->phase_ms[mk.phase] += ms;
                if (mk.phase == SDC_PHASE_PCG) stats->cg_ms[mk.k][mk.m] = ms;
            }
        }
    }
    return status;
}

}  // namespace sdc

namespace sdc {
SDC_CHECK_READER(check_take_emi)
}  // namespace sdc
