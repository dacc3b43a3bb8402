// sdc_pcg_solve_noalloc: the node-system solve of sdc_pcg_solve for callers
// that must not allocate device memory themselves or through this library.
//
// Typical such callers: a host application or simulation framework that owns
// every byte of device memory through its own pool and forbids raw cudaMalloc
// (it would bypass the pool's budget or fragment it), and time-critical loops
// in which cudaMalloc/cudaFree may block or synchronise the device.  They pass
// inputs and outputs as usual; the solver's workspace (ten vectors, per-block
// partial sums, the barrier counter and status words) lives in the file-scope
// array below instead of a per-call allocation.
//
// Costs and limits of that choice:
//   * every GPU that loads the library reserves the array (about 5.6 MB) until
//     the process exits;
//   * n is limited to SDC_PCG_NOALLOC_MAX_ROWS rows;
//   * all calls on a device share the one array and it keeps the last call's
//     contents, so calls that overlap on the GPU (two streams, two host
//     threads) race and corrupt each other; serialise them;
//   * host code cannot use the array's name as a device address, so the first
//     call on each device looks the address up (cudaGetSymbolAddress, with that
//     device current) and caches it; make that first call before any stream
//     capture is started on the device.  The cache is keyed by the device's
//     context as well: after cudaDeviceReset the array lives at a new address
//     in the new context, and the first call there looks it up again.

#include <cstdio>
#include <mutex>

#include "sdc_internal.h"

namespace {

constexpr int kMaxRows = SDC_PCG_NOALLOC_MAX_ROWS;
constexpr int kMaxBlocks = 4096;   // blocks with partial-sum records (48 bytes, two buffers)
constexpr size_t kVecDoubles = 10 * (size_t)kMaxRows;
constexpr size_t kScalarDoubles = 4;   // relres, then barrier counter, error, iterations
constexpr size_t kScratchDoubles = kVecDoubles + 12 * (size_t)kMaxBlocks + kScalarDoubles;

static __device__ __align__(256) double g_pcg_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context id the address belongs to

// Unique id of the calling thread's current context (cuCtxGetId through the
// runtime's driver entry point, so the library needs no link to libcuda);
// 0 when there is none yet or the query is unavailable.
unsigned long long current_context_id() {
    using GetId = int (*)(void*, unsigned long long*);
    static GetId fn = []() -> GetId {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (GetId)p;
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}

sdc_status reject(sdc_status st, const char* msg) {
    sdc::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" sdc_status sdc_pcg_solve_noalloc(int n, const double* d_val, const int* d_col,
                                            const int* d_len, int ld, int width,
                                            const double* d_kdiag, const double* d_mass,
                                            const double* d_J, double c, const double* d_b,
                                            double* d_x, double rtol, int maxit, int* iters,
                                            double* relres, void* stream) {
    sdc::set_thread_error("");
    if (n > kMaxRows) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "sdc_pcg_solve_noalloc: n = %d exceeds the static workspace of %d rows", n,
                 kMaxRows);
        return reject(SDC_E_INVALID, buf);
    }
    // the published m takes two buffers ld apart after the eight other vectors
    if (n > 0 && ld > 0 && 9 * (size_t)n + (size_t)ld > kVecDoubles) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "sdc_pcg_solve_noalloc: ld = %d too large for n = %d in the static workspace "
                 "(9 n + ld must not exceed %zu)", ld, n, kVecDoubles);
        return reject(SDC_E_INVALID, buf);
    }
    if (n < 1 || ld < n || width < 0 || !d_len || !d_kdiag || !d_mass || !d_J || !d_b || !d_x ||
        (width > 0 && (!d_val || !d_col)) || !(rtol > 0.0) || maxit < 1 || !(c - c == 0.0))
        return reject(SDC_E_INVALID, "sdc_pcg_solve_noalloc: invalid arguments");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return reject(SDC_E_CUDA, "sdc_pcg_solve_noalloc: no current device");
    if (dev < 0 || dev >= kMaxDevices)
        return reject(SDC_E_INVALID, "sdc_pcg_solve_noalloc: device ordinal out of range");
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long ctx_id = current_context_id();
        if (!g_scratch_addr[dev] || ctx_id == 0 || ctx_id != g_scratch_ctx[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
            if (e != cudaSuccess || !p) {
                char buf[200];
                snprintf(buf, sizeof buf,
                         "sdc_pcg_solve_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return reject(SDC_E_CUDA, buf);
            }
            g_scratch_addr[dev] = (double*)p;
            // the lookup made the device's context current if it was not yet
            g_scratch_ctx[dev] = current_context_id();
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    sdc::PcgScratch w;
    w.r = base;
    w.u = base + (size_t)n;
    w.p = base + 2 * (size_t)n;
    w.s = base + 3 * (size_t)n;
    w.w = base + 4 * (size_t)n;
    w.idA = base + 5 * (size_t)n;
    w.z = base + 6 * (size_t)n;
    w.nv = base + 7 * (size_t)n;
    w.m = base + 8 * (size_t)n;
    w.part = base + kVecDoubles;
    w.max_blocks = kMaxBlocks;
    w.relres = base + kVecDoubles + 12 * (size_t)kMaxBlocks;
    unsigned* sc = (unsigned*)(w.relres + 1);
    w.bar = sc;
    w.err = (int*)(sc + 1);
    w.iters = (int*)(sc + 2);
    sdc::Ell A;
    A.val = const_cast<double*>(d_val);
    A.col = const_cast<int*>(d_col);
    A.len = const_cast<int*>(d_len);
    A.ld = ld;
    A.width = width;
    // the barrier counter, error word and outputs must start at zero on every call
    if (cudaMemsetAsync(w.relres, 0, kScalarDoubles * sizeof(double), s) != cudaSuccess)
        return reject(SDC_E_CUDA, "sdc_pcg_solve_noalloc: clearing the status words failed");
    if (sdc::launch_pcg_standalone(n, A, d_kdiag, d_mass, d_J, c, d_b, d_x, rtol, maxit,
                                   4000000000LL, 256, w, s) != SDC_OK)
        return reject(SDC_E_CUDA, "sdc_pcg_solve_noalloc: launch failed");
    int h[3] = {0, 0, 0};
    double hr = 0.0;
    if (cudaMemcpyAsync(h, sc, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hr, w.relres, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return reject(SDC_E_CUDA, "sdc_pcg_solve_noalloc: reading the status failed");
    if (iters) *iters = h[2];
    if (relres) *relres = hr;
    {
        // checked builds: an index outside its bound is reported before any CG status
        const sdc_status chk = sdc::check_outcome(nullptr, s, SDC_OK);
        if (chk != SDC_OK) return chk;
    }
    if (h[1] != 0) {
        char buf[120];
        snprintf(buf, sizeof buf, "sdc_pcg_solve_noalloc: %s", sdc_status_string(h[1]));
        return reject((sdc_status)h[1], buf);
    }
    return SDC_OK;
}
