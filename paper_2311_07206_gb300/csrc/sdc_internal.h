// Internal declarations shared by the library's translation units (host side).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/sdc.h"

namespace sdc {

constexpr int kMaxM = SDC_MAX_M;
constexpr int kUpdateBlock = 256;   // block size of the update / scatter kernels

// Aliev-Panfilov parameters as passed to kernels (Sec. 5.1.1).
struct Ionic {
    double ga, gs, a, eps, mu1, mu2, cw;
};

// Collocation matrices, fixed stride kMaxM, passed by value to kernels.
struct Coll {
    int M;
    double Q[kMaxM * kMaxM];
    double Qh[kMaxM * kMaxM];
};

// Device scalars of one context (one allocation).
struct DevScalars {
    int count;                 // |I_{k+1}| written by the scan kernel
    int err;                   // first error code raised by any kernel (0 = none)
    unsigned bar;              // grid-barrier arrival counter of the running CG launch
    int pad;
    unsigned long long nnz;    // stored off-diagonals of the newest restricted matrix
    double margin;             // min |max_m |dv| - TOL_drop| of the newest selection
    int cg_iters[SDC_MAX_SWEEPS * kMaxM];
    double cg_relres[SDC_MAX_SWEEPS * kMaxM];
    double cg_energy[SDC_MAX_SWEEPS * kMaxM];   // dv_m' A~_m dv_m per node solve
    unsigned long long drop_c;     // bits of max |dv| of the first sweep (drop rule 1)
    unsigned long long drop_eta;   // bits of max(0, -dI/dv) of the first sweep
    double tol_drop;               // the a priori drop tolerance of the step (drop rule 1)
    unsigned long long nnz_k[SDC_MAX_SWEEPS];   // stored off-diagonals of K[I_k, I_k], k >= 1
};

// ELL-R matrix in column-major slots: entry t of row i at [t * ld + i],
// row i holds len[i] entries.  Used for off-diagonal parts only.
struct Ell {
    double* val = nullptr;
    int* col = nullptr;
    int* len = nullptr;
    int ld = 0;
    int width = 0;
};

// ---- collocation (radau.cpp) ----
bool radau_collocation(int M, double* tau, double* Q, double* Qhat);

// ---- assembly (assembly.cu) ----
// The mesh as kept on the device (re-assembly, conductivity gradients).
struct MeshDev {
    int dim = 0, n_nodes = 0, n_elems = 0;
    long long nnz_pattern = 0;
    double* xyz = nullptr;     // n_nodes * dim
    double* sig = nullptr;     // 9, global tensor
    double* esig = nullptr;    // n_elems * 9 or null
    double* scale = nullptr;   // n_nodes or null (all ones)
    int* elem = nullptr;       // n_elems * (dim + 1)
    int* n2e_ptr = nullptr;    // node -> element lists, ascending element order
    int* n2e = nullptr;
    int* n2e_loc = nullptr;    // the node's local index in that element
    int* rp = nullptr;         // CSR pattern of K
    int* ci = nullptr;
};
struct AssemblyOut {
    Ell K;                 // off-diagonal part of K (device)
    double* kdiag = nullptr;
    double* mass = nullptr;
    long long nnz = 0;     // stored entries including the diagonal
    MeshDev mesh;
};
int assemble_device(const sdc_mesh& mesh, double drop_rel, cudaStream_t s, AssemblyOut& out,
                    std::string& why);
// Recompute K's values for a new per-node conductivity scale (host array, or
// null for all ones) on the kept pattern; fails if the stored width would grow.
int reassemble_device(AssemblyOut& out, const double* h_scale, double drop_rel, cudaStream_t s,
                      std::string& why);
void free_mesh_dev(MeshDev& m);

// ---- step kernels (step.cu) ----
// SDC_CHECKED=1 builds the checked library (index checks in every kernel gather).
#ifndef SDC_CHECKED
#define SDC_CHECKED 0
#endif

// Check words of the checked build (SDC_CHECKED=1), one reader per translation unit
// that runs kernels: read and clear after the work on `stream`; the first failure
// record is (check site << 32) | index, 0 when none (always 0 in normal builds).
unsigned long long check_take_step(void* stream, unsigned* count);
unsigned long long check_take_emi(void* stream, unsigned* count);
unsigned long long check_take_adjoint(void* stream, unsigned* count);
unsigned long long check_take_assembly(void* stream, unsigned* count);
unsigned long long check_take_coarse(void* stream, unsigned* count);
// The status of a call after its device work on `stream`: in checked builds an index
// recorded outside its bound turns it into SDC_E_INVALID (message on ctx, or on the
// calling thread when ctx is NULL); otherwise st unchanged.
sdc_status check_outcome(sdc_ctx* ctx, void* stream, sdc_status st);

struct StepBuffers {
    int N = 0, M = 0, ld = 0;
    double* V = nullptr;      // [N][M] node-interleaved collocation iterates of v
    double* W = nullptr;      // [N][M] same for w
    double* R = nullptr;      // [M][ld] residual / right-hand sides (compact rows)
    double* J = nullptr;      // [M][ld] dI/dv at the iterate
    double* D = nullptr;      // [M][ld] corrections dv
    double* mc = nullptr;     // [ld] lumped mass of the active rows
    double* kdc = nullptr;    // [ld] K_ii of the active rows
    double* r = nullptr;      // CG vectors [ld]: residual, u = D^-1 r, w = A u, direction p,
    double* u = nullptr;      // s = A p, z = A D^-1 s, nv = A m, reciprocal diagonal;
    double* p = nullptr;      // m = D^-1 w [2 ld] (two buffers)
    double* s = nullptr;
    double* w = nullptr;
    double* z = nullptr;
    double* nv = nullptr;
    double* m = nullptr;
    double* idA = nullptr;
    double* part = nullptr;   // 12 * max_blocks: one 48-byte exact-sum record per block, two buffers
    double* sv = nullptr;     // [ld] diag^-1/2 of the scaled solve
    double* sval = nullptr;   // [sval_width][ld] scaled off-diagonal values of the scaled solve
    int sval_width = 0;
    int max_blocks = 0;
    int* flag = nullptr;      // [ld]
    int* map = nullptr;       // [ld] old compact row -> new compact row or -1
    int* blockcnt = nullptr;  // per update block
    int* blockoff = nullptr;
    double* blockmarg = nullptr;
    Ell A[2];                 // restricted off-diagonal matrices (ping-pong)
    DevScalars* sc = nullptr;
    double* vtmp = nullptr;   // host-call staging [N]
    double* wtmp = nullptr;
    // batched contexts: nseg instances, contiguous in the dof numbering
    int nseg = 0;
    int* inst_off = nullptr;      // [nseg + 1] first dof of each instance
    int* bounds = nullptr;        // [nseg + 1] instance boundaries in the current active list
    int* segtab = nullptr;        // per-block group table of the batched PCG launch
    int segtab_cap = 0;           // blocks the group table holds
    int* plan = nullptr;          // [2 nseg] blocks and first block per instance (planned launch)
    int* nk = nullptr;            // [SDC_MAX_SWEEPS + 1] |I_k| of a captured step
    int* bounds_k = nullptr;      // [(SDC_MAX_SWEEPS + 1) (nseg + 1)] boundaries per sweep
    unsigned* bars = nullptr;     // [nseg] barrier counters
    int* seg_iters = nullptr;     // [SDC_MAX_SWEEPS * kMaxM * nseg]
    double* seg_relres = nullptr; // same shape
};

void launch_spread(int N, int M, const double* v0, const double* w0, double* V, double* W,
                   cudaStream_t s);
void launch_final(int N, int M, const double* V, const double* W, double* v, double* w,
                  cudaStream_t s);
void launch_nodes_out(int N, int M, const double* V, const double* W, double* Vout, double* Wout,
                      cudaStream_t s);
void launch_residual(int M, int n, const int* act, const Ell& K, const double* kdiag,
                     const double* mass, const double* stim, double stim_on, const double* V,
                     const double* W, const double* v0, double dt, const Ionic& ion,
                     const Coll& co, int reaction_implicit, StepBuffers& B, cudaStream_t s,
                     const int* n_dev = nullptr);
// Launch configuration of the restricted PCG solves.
constexpr int kSmemVectorsS = 6;    // the same for the symmetrically scaled variant
constexpr int kSmemVectorsCS = 4;   // the scaled classical shared-memory variant (kSmemRowsC rows)
constexpr int kSmemRowsS = 4800;    // rows per block of the symmetrically scaled variant
constexpr int kSmemVectors = 8;     // per-row doubles in shared memory, shared-memory variant
constexpr int kSmemRows = 3584;     // rows per block of the shared-memory variant
// target rows per block of the shared-memory variants below their capacity: one row
// per product thread of a 512-thread block, spread over up to one block per SM
constexpr int kSmemRowsDefault = 256;
constexpr int kClusterVectors = 10; // per-row doubles in shared memory, cluster variant
constexpr int kClusterRows = 2848;  // rows per CTA of the cluster variant
constexpr int kSmemVectorsC = 6;    // classical arrangement, shared-memory form
constexpr int kSmemRowsC = 4768;
struct PcgConfig {
    int block = 256;                // block size of the general variant
    int max_blocks_general = 0;     // cooperative grid limit of the general variant
    int smem_block = 1024;          // block size of the shared-memory variant
    int sms = 0;                    // SM count (one shared-memory block per SM at most)
    int max_blocks = 0;             // user limit on the shared-memory grid (0 = none)
    int rows_per_block = 0;         // target rows per shared-memory block (0 = default)
    int variant = 0;                // 0 auto, 1 general only, 2 shared memory when it fits
    int cluster = 0;                // CTAs of the cluster variant (0 = unavailable)
    int cluster_rows = 0;           // use the cluster variant for n <= cluster_rows
    int cluster_rows_per_cta = 64;  // rows per CTA below which fewer CTAs are used
    int big_rows = 300000;          // shared-memory variant uses 1024 threads from here on
    int max_blocks_batch = 0;       // cooperative grid limit of the batched variant
    int batch_block = 256;          // block size of the batched variant
    int batch_pipelined = 0;        // arrangement of the batched variant
    int batch_rows_per_block = 1024;
    int inject_fault = 0;
    int pipelined = 1;              // 1: pipelined CG; 0: classical arrangement
    int scaled = 1;                 // pipelined shared-memory solves in the scaled form
    int general_classical = 0;      // pipelined contexts: classical arrangement for the
                                    // global-vector variant (automatic choice)
    long long budget = 0;
};
int launch_pcg(int n, const Ell& A, int m, double dt, const Coll& co, double rtol, int maxit,
               int sweep, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s);
int pcg_sm_count();
// dof permutation (perm[new] = old): dst[i] = src[perm[i]] / dst[perm[i]] = src[i]
void launch_perm_gather(int N, const int* perm, const double* src, double* dst, cudaStream_t s);
void launch_perm_scatter(int N, const int* perm, const double* src, double* dst, cudaStream_t s);
// node values [new][M] -> [m][old]
void launch_nodes_out_perm(int N, int M, const int* perm, const double* X, double* out,
                           cudaStream_t s);
// Message returned by sdc_last_error(NULL) on the calling thread.
void set_thread_error(const char* msg);

// One node solve with caller-chosen right-hand side, solution, J and
// coupling targets (the reverse sweep of the adjoint uses it).
struct PcgRole {
    const double* b;
    double* x;
    const double* J;        // J of the solved node, compact
    const double* Jall;     // [M][ld] J of every node (targets use their own)
    double* R;              // [M][ld] coupling targets
    int epi_lo, epi_hi, epi_target_J;
    double qh[kMaxM];
    double c;               // dt * Qhat_mm of the solved node
    int* iters_out;
    double* relres_out;
    double* energy_out;     // may be null
};
int launch_pcg_role(int n, const Ell& A, const PcgRole& role, double dt, int M, double rtol,
                    int maxit, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s);

// ---- two-level preconditioner of the cell-by-cell node solves (Sec. 6) ----------
// Blocks (labels per dof, every dof in one block) give the coarse space Z of the
// additive two-level preconditioner z = D^-1 r + Z E^-1 Z' r, E = Z' A Z, over the
// blocks that hold active dofs.
constexpr int kMaxCoarseBlocks = SDC_MAX_COARSE_BLOCKS;
constexpr int kCoarseTile = 1024;   // positions per tile of the two-level CG (its block size)
struct CoarseDev {
    int q = 0;                           // blocks
    int N = 0;
    int* lab = nullptr;                  // [N] block of each dof
    int* gperm = nullptr;                // [N] dofs sorted by (block, dof)
    int* lab_c = nullptr;                // [ld] block of each compact row of the sweep
    int* crow = nullptr;                 // [ld] compact rows sorted by (block, row)
    int* boff = nullptr;                 // [q + 1] first position of each block in crow
    int* chunk_cnt = nullptr;            // compaction scratch: per-chunk counts and offsets
    int* chunk_off = nullptr;
    // rows of the CG launch: the positions of crow in tiles of kCoarseTile, tile j on CTA
    // j mod G; each tile cut at block boundaries into pieces, numbered in position order
    int* tp = nullptr;                   // [ntiles + 1] pieces of each tile
    int* piece = nullptr;                // [3 P]: block, first and end position
    int* blk_ptr = nullptr;              // [q + 1] pieces of each block (contiguous)
    int* nzb = nullptr;                  // [q] the blocks with active rows, ascending
    double* tpiece = nullptr;            // [P] partial coarse sums of each piece
    unsigned long long* Eacc = nullptr;  // [q * q] E in 64-bit fixed point
    double* Einv = nullptr;              // [q * q] E^-1, row-major
    double* piv = nullptr;               // new pivot rows of the inversion (two panels)
    unsigned long long* dmax = nullptr;  // largest diagonal of the node operator (bits)
    unsigned* bar = nullptr;             // grid barrier counter of the inversion
    int* err = nullptr;                  // shared with the step's error word
    std::vector<int> h_boff, h_tp, h_piece, h_blk_ptr, h_nzb;
    int Gmax = 0;                        // CTAs of a full-size coarse CG launch (the SMs)
    int G = 0;                           // CTAs of this sweep's coarse CG launch
    int qn = 0;                          // blocks with active rows
    int pmax = 0;                        // most pieces of one CTA
    int ptot = 0;                        // pieces of the sweep
    int ntiles = 0;                      // tiles of the sweep
    int tmax = 0;                        // most tiles of one CTA
};
// labels: host, N entries in [0, q).  Allocates and uploads; returns an sdc_status.
int coarse_setup(CoarseDev& C, const int* h_lab, int N, int q, int ld, int* err, cudaStream_t s,
                 std::string& why);
void coarse_free(CoarseDev& C);
// Per sweep: block of each compact row, rows sorted by block, block ranges and the
// pieces of the CG launch (tiles of kCoarseTile positions, round robin over the CTAs,
// cut at blocks).  pos: dof -> compact row (-1 outside the active set).  Synchronises
// the stream (reads the block ranges).
int coarse_sweep(CoarseDev& C, int n, const int* act, const int* pos, int G, cudaStream_t s);
// Per node solve: E = Z' A Z of the operator diag(mc (1 + c J) + c kdc) + c A_off on the
// active rows (exact fixed-point accumulation) and its inverse.
int coarse_factor(CoarseDev& C, int n, const Ell& A, const double* mc, const double* J,
                  const double* kdc, double c, long long budget, cudaStream_t s);
// The node solve with the two-level preconditioner (classical scaled arrangement).
int launch_pcg_coarse(int n, const Ell& A, const PcgRole& role, double rtol, int maxit,
                      const CoarseDev& C, const PcgConfig& cfg, StepBuffers& B, cudaStream_t s);

// Batched PCG: independent solves of the instances whose compact rows are
// [bounds[s], bounds[s+1]); empty instances are skipped.
int launch_pcg_batch(int n, const Ell& A, int m, double dt, const Coll& co, double rtol,
                     int maxit, int sweep, const PcgConfig& cfg, const std::vector<int>& bounds,
                     StepBuffers& B, cudaStream_t s);
void launch_seg_bounds(const int* act, const int* count, StepBuffers& B, cudaStream_t s,
                       int* bounds_out = nullptr);
// Device-planned form for captured steps: a single-block kernel apportions the fixed
// cooperative grid (max_blocks_batch blocks) to the instances from the device boundaries
// bounds_dev (plan = true: rebuild the table, once per sweep), blocks without a group
// leave at once.  Needs nseg <= max_blocks_batch.
void launch_graph_init(StepBuffers& B, cudaStream_t s);
int launch_pcg_batch_planned(const Ell& A, int m, double dt, const Coll& co, double rtol,
                             int maxit, int sweep, const PcgConfig& cfg, const int* bounds_dev,
                             bool plan, StepBuffers& B, cudaStream_t s);
int pcg_batch_max_blocks(int block);

// ---- adjoint (adjoint.cu) ----
struct AdjointArgs {
    const MeshDev* mesh;
    const Ell* K;
    const double* kdiag;
    const double* mass;
    const double* lam_v;   // adjoints of the step's outputs
    const double* lam_w;
    double* lam_v0;        // adjoints of the step's inputs (written)
    double* lam_w0;
    const double* v0;      // the step's inputs
    const double* w0;
    double* grad_scale;    // += dL/ds per node, or null
    const double* tape_V;  // [sweeps][N * M] state after each sweep
    const double* tape_W;
    const int* tape_act;   // [sweeps][N] active list of sweep k (k >= 1)
    const int* n_active;   // host [sweeps]
    int sweeps;
    double dt;
    Ionic ion;
    Coll co;
    int reaction_implicit, w_frozen;
    double rtol;
    int maxit;
    const PcgConfig* cfg;
};
struct AdjointBuffers {
    double *Vb = nullptr, *Wb = nullptr, *V0 = nullptr, *W0 = nullptr;
    double *X = nullptr, *Jb = nullptr;                       // [M][ld]
    double *bfull = nullptr, *vkfull = nullptr, *ffull = nullptr;   // [M][N]
    double *ge = nullptr;                                     // [n_elems]
    double *part3 = nullptr, *iacc = nullptr;                 // block partials, 3 accumulators
    int* pos = nullptr;                                       // [N], -1 outside a list
    int* iters = nullptr;                                     // [SDC_MAX_SWEEPS * kMaxM]
    double* relres = nullptr;
};
int adjoint_step(const AdjointArgs& a, StepBuffers& B, AdjointBuffers& W, cudaStream_t s);
void launch_pos_set(int n, const int* act, int* pos, int reset, int N, cudaStream_t s);
void launch_extract_global(int n, const int* act, const int* pos, const Ell& K, Ell& out, int N,
                           cudaStream_t s);
void launch_replay_map(int n_old, const int* act_old, const int* pos, int* map, int N,
                       cudaStream_t s);

// Workspace of one standalone PCG solve (caller-provided device memory).
// r, u, w, p, s, z, nv, idA: n doubles each; m: 2 n doubles;
// part: 12 * max_blocks doubles (16-byte aligned);
// bar, err, iters, relres: one value each, bar and err zero before the launch.
struct PcgScratch {
    double *r, *u, *w, *p, *s, *z, *nv, *m, *idA, *part;
    int max_blocks;
    unsigned* bar;
    int* err;
    int* iters;
    double* relres;
};
// Jacobi-PCG on (diag(mass (1 + c J)) + c K)[n x n] with the off-diagonal part
// of K in A (ELL-R) and its diagonal in kdiag, using the global-vector kernel.
int launch_pcg_standalone(int n, const Ell& A, const double* kdiag, const double* mass,
                          const double* J, double c, const double* b, double* x, double rtol,
                          int maxit, long long budget, int block, const PcgScratch& w,
                          cudaStream_t s);
int pcg_cluster_size(int block);
// tol_drop_dev: when set, the selection reads TOL_drop there instead of tol_drop
void launch_update(int M, int n, const int* act, const double* w0, double dt, const Ionic& ion,
                   const Coll& co, double tol_drop, int w_frozen, StepBuffers& B, cudaStream_t s,
                   const double* tol_drop_dev = nullptr, const int* n_dev = nullptr);
// A priori drop tolerance of Sec. 4.1 into B.sc->tol_drop, from the first sweep's
// corrections (n rows of D, M nodes) and Jacobians (nj entries per node at stride ldj).
void launch_drop_rule(int n, int M, const double* D, int ld, int nj, const double* J, int ldj,
                      double Cm, double rho, double TOL, double dt, StepBuffers& B,
                      cudaStream_t s);
// n_dev: when set, |I_k| is read on the device and n only sizes the grid (captured steps)
void launch_select(int n, const int* act, int* act_next, StepBuffers& B, cudaStream_t s,
                   const int* n_dev = nullptr);
void launch_extract(int n_old, const Ell& Aold, const int* map, Ell& Anew, StepBuffers& B,
                    cudaStream_t s, const int* n_dev = nullptr);
int pcg_max_blocks(int block);

// ---- cell-by-cell (EMI) model (emi.cu) ----
struct EmiDev {
    int np = 0;                 // pairs
    int max_inc = 0;            // most pairs at one dof
    double Cm = 1.0, g_gap = 0.0;
    int *pk = nullptr, *pl = nullptr, *pkind = nullptr;
    double* parea = nullptr;
    double* robin = nullptr;    // [N] or null
    int *np_ptr = nullptr, *np_pid = nullptr, *np_part = nullptr, *np_sign = nullptr;  // dof -> pairs
    double *Wp = nullptr;       // [np][M] gating at the collocation nodes
    double *Ip = nullptr, *Jp = nullptr;   // [M][np] pair current and its dI/dv
    Ell A;                      // node-solve operator B + c (K + D_m) restricted (ld = B.ld)
    int* pos = nullptr;         // [N] compact row of a dof in the current list, -1 outside
    double* wstage = nullptr;   // [np] host-call staging
    unsigned long long* slots = nullptr;   // pair slots stored by the last build (statistics)
};
// Copies the pair data (host arrays validated by the caller) and allocates
// the EMI buffers.
int emi_setup(const sdc_emi& emi, int N, int M, int k_width, int ld, cudaStream_t s, EmiDev& E,
              std::string& why);
void emi_free(EmiDev& E);
struct EmiStepArgs {
    int N, M;
    cudaStream_t s;
    const AssemblyOut* K;
    StepBuffers* B;
    EmiDev* E;
    std::vector<int*>* act;     // device lists, act[k] for sweep k >= 1, act[0] scratch
    std::vector<int>* n_act;
    const PcgConfig* pcg;
    const sdc_options* opt;
    const Coll* co;
    const Ionic* ion;
    int* h_pin;                 // pinned: [0] count, [1] err, node energies from byte 16
    std::string* err;
    std::vector<cudaEvent_t>* events;   // profiling event pool (profile option)
    int* sweeps_done;           // out: sweeps run (fewer after an energy-norm stop)
    CoarseDev* coarse;          // two-level preconditioner blocks, or null (Jacobi)
};
int emi_step(const EmiStepArgs& a, double* d_u, double* d_w, double dt, int sweeps, double TOL,
             sdc_stats* stats);
void emi_nodes_out(const EmiDev& E, int N, int M, const double* V, double* d_V, double* d_W,
                   cudaStream_t s);

}  // namespace sdc
