/*
 * sdc.h - C ABI of the GB300 (sm_103a) adaptive spectral deferred correction
 * library for P1 finite-element monodomain reaction-diffusion systems with
 * Aliev-Panfilov kinetics.
 *
 * The problem (Sec. 2.2, eq. abstract monodomain; Sec. 3, eq. abstract ODE):
 *     m .* v' = -K v - m .* (I_ion(v, w) - I_stim),     w' = R(v, w)
 * with K the P1 stiffness matrix of div(sigma grad v) under homogeneous
 * Neumann conditions and m the lumped mass.  One time step is a Radau-IIA
 * collocation step (Sec. 3.1) approximated by LU-trick SDC sweeps with the
 * v-then-w operator splitting of eq. final-sdc (Sec. 3.2).  After each sweep
 * only the dofs whose voltage correction reaches TOL_drop = alpha * TOL stay
 * active; later sweeps solve the restricted systems on those nested index sets
 * with Jacobi-preconditioned CG, holding the dropped dofs fixed (Sec. 4.2).
 *
 * Conventions for every call:
 *   - Host arrays passed to sdc_create / sdc_set_stimulus are copied; the caller
 *     keeps ownership and may free them on return.
 *   - Device arrays (prefix d_) are caller-owned FP64 device memory on the
 *     context's device; the library never frees them.
 *   - All device work is issued on the stream given to sdc_create.  Calls that
 *     read results back (sdc_step, sdc_step_host) synchronise that stream before
 *     they return.
 *   - Every call returns an sdc_status.  On failure no output is guaranteed to
 *     be meaningful and sdc_last_error(ctx) gives a one-line reason.  Invalid
 *     arguments are rejected with SDC_E_INVALID before any device work starts.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef SDC_GB300_H
#define SDC_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDC_MAX_M 8        /* collocation nodes per step */
#define SDC_MAX_SWEEPS 64  /* SDC sweeps per step */

/* Kernel phases of a step, as reported in sdc_stats. */
#define SDC_PHASE_RESIDUAL 0  /* spread, collocation residual + ionic model, final copy */
#define SDC_PHASE_PCG 1       /* restricted Jacobi-PCG solves (one launch per node)    */
#define SDC_PHASE_UPDATE 2    /* v update, w sweep, selection flags                    */
#define SDC_PHASE_SELECT 3    /* stable compaction of the next active set              */
#define SDC_PHASE_EXTRACT 4   /* restricted submatrix extraction                       */
#define SDC_N_PHASES 5

typedef struct sdc_ctx sdc_ctx;

typedef enum {
    SDC_OK = 0,
    SDC_E_INVALID = -1,   /* bad argument; nothing was launched */
    SDC_E_CUDA = -2,      /* a CUDA runtime call failed */
    SDC_E_NOMEM = -3,     /* device allocation failed */
    SDC_E_CG_NOCONV = -4, /* CG reached cg_maxit without meeting cg_rtol */
    SDC_E_TIMEOUT = -5,   /* a device-side wait exceeded its spin budget */
    SDC_E_NONFINITE = -6, /* NaN or Inf in a residual or correction */
    SDC_E_DOMAIN = -7     /* gating rate pole v + mu2 <= 0, or a non-positive pivot */
} sdc_status;

/* P1 simplex mesh (Sec. 2.2).  Host arrays, copied at sdc_create.
 *   dim        2 (triangles) or 3 (tetrahedra)
 *   xyz        n_nodes * dim coordinates, node-major
 *   elem_ptr   n_elems + 1 offsets into elem_node; every element must list
 *              exactly dim + 1 distinct nodes
 *   sigma      global conductivity tensor, 9 doubles row-major (the leading
 *              dim x dim block is used); ignored where elem_sigma is given
 *   elem_sigma NULL or n_elems * 9 per-element tensors
 *   dof_scale  NULL or n_nodes per-node conductivity scale s; element e uses
 *              the mean of s over its vertices                                 */
typedef struct {
    int dim;
    int n_nodes;
    const double* xyz;
    int n_elems;
    const int* elem_ptr;
    const int* elem_node;
    const double* sigma;
    const double* elem_sigma;
    const double* dof_scale;
} sdc_mesh;

/* Aliev-Panfilov model (Sec. 5.1.1):
 *   I_ion(v, w) = ga v (v - a)(v - 1) + v w
 *   R(v, w)     = cw (eps + mu1 w / (v + mu2)) (-w - gs v (v - a - 1))
 * The paper's values use cw = 1/4; the standard 1996 form uses cw = 1.         */
typedef struct {
    double ga, gs, a, eps, mu1, mu2, cw;
} sdc_ionic;

typedef struct {
    double alpha;          /* TOL_drop = alpha * TOL (Sec. 4.2); default 0.1                  */
    double cg_rtol;        /* stop when sqrt(r'z) <= cg_rtol sqrt(r0'z0); default 1e-10        */
    int cg_maxit;          /* default 2000                                                    */
    int reaction_implicit; /* 1: lumped dI/dv on the diagonal of every node system (Sec. 3.2) */
    int w_frozen;          /* 1: w is held at its initial value (no gating dynamics)          */
    double drop_rel;       /* assembly: off-diagonal K_ij with |K_ij| <= drop_rel sqrt(K_ii K_jj)
                              are rounding residue of cancelling element terms and are not
                              stored; default 1e-12, 0 keeps every structural entry           */
    long long spin_budget; /* SM clock cycles a device-side barrier may wait; default 4e9     */
    int cg_block_size;     /* threads per block of the global-vector CG (64..1024, multiple
                              of 32); default 1024.  Batches use min(this, 256)               */
    int cg_smem_block_size;/* threads per block of the shared-memory and cluster CG; default 512 */
    int cg_cluster_max;    /* largest cluster (CTAs) for the cluster CG, 1..16; default 16      */
    int cg_max_blocks;     /* 0: no limit on the cooperative CG grid                          */
    int cg_variant;        /* 0: automatic; 1: vectors in global memory; 2: per-block vectors
                              in shared memory whenever they fit (3584 rows per SM for the
                              pipelined, 4768 for the classical arrangement)                 */
    int cg_rows_per_block; /* shared-memory variant: target rows per block (0 = 256)          */
    int cg_cluster_rows;   /* solves with |I_k| <= this run on one thread-block cluster
                              (16 CTAs, distributed shared memory); default 10000, 0 = never */
    int profile;           /* 1: bracket every kernel launch with CUDA events on the context's
                              stream and report device time per phase in sdc_stats; default 0 */
    int inject_fault;      /* testing hook, default 0.  1: in every CG launch the last block
                              leaves without arriving at the first grid barrier, so the other
                              blocks' bounded waits run out and the step returns SDC_E_TIMEOUT */
    int cg_pipelined;      /* arrangement of the CG iteration (the same iterates in exact
                              arithmetic): 1 pipelined (one grid synchronisation per iteration,
                              the sums overlapped with the product); 0 classical (two); -1
                              automatic: for monodomain contexts pipelined where the solve's
                              vectors fit on chip and classical above (its lighter vector
                              traffic wins there); classical for cell-by-cell contexts, whose
                              long ill-conditioned solves need its smaller rounding error, and
                              for batches, whose many small groups favour its lighter rows;
                              default -1                                                       */
    int energy_stop;       /* 1: end the sweeps of a step once the energy norm of the sweep's
                              corrections, E_k = sum_m dv_m' A~_m dv_m with A~_m the node system
                              matrix, is at most ((1 - rho) / rho * TOL)^2 (Sec. 3.2); `sweeps`
                              is then the largest number of sweeps.  Monodomain and
                              cell-by-cell contexts (there A~_m = B + c_m (A + sum over pairs of
                              the pair Jacobian)); not with a tape or in a batch; default 0   */
    double sdc_rho;        /* SDC contraction rho for energy_stop, in [0, 1); 0: estimated after
                              each sweep as sqrt(E_k / E_{k-1}) (so no stop after the first
                              sweep); default 0                                               */
    int sdc_qhat;          /* lower-triangular preconditioner of the sweeps (Sec. 3.1):
                              0 LU trick, Qhat = U^T with Q^T = L U (default); 1 implicit Euler,
                              the right-looking rectangle rule, Qhat_mj = tau_j - tau_{j-1} for
                              j <= m (tau_0 = 0)                                              */
    int reorder;           /* 1: number the dofs internally in Morton (Z-curve) order of their
                              coordinates, so that the rows a block owns and the neighbours it
                              gathers lie close in memory (randomly numbered unstructured
                              meshes); states, stimuli, scales, active lists, node values and
                              the matrix stay in the caller's numbering.  Not with tapes or the
                              adjoint, in batches or EMI contexts; default 0                  */
    int drop_rule;         /* drop tolerance of the selections: 0 TOL_drop = alpha TOL (default);
                              1 the a priori tolerance of Sec. 4.1 (Eq. drop-tolerance):
                              TOL_drop = exp(-eta dt) (1 - rho) / (r + 1) TOL with rho = sdc_rho
                              (required in (0, 1)), c = max |dv| of the step's first sweep, r
                              the least integer >= 0 with c rho^r <= (1 - rho) TOL, and eta =
                              max(0, -min dI/dv) / C_m over the first sweep's linearisation
                              (zero with reaction_implicit = 0); computed on the device once
                              per step, reported in sdc_stats.tol_drop.  Not in batches      */
    int cg_scaled;         /* 1: the node solves (shared-memory, global-vector and batched
                              variants; the cluster variant keeps the Jacobi form) run in the
                              symmetrically scaled form, CG on diag^-1/2 A diag^-1/2: the same
                              iterates as Jacobi-PCG with fewer FP64 operations per row and
                              fewer vectors on chip; 0: the Jacobi form; default 1          */
    int batch_graph;       /* batches: 1 runs each step with device-driven sweeps (|I_k| read on
                              the device, the batched solves' block plan built on the device)
                              captured once per (state arrays, dt, sweeps, TOL, stimulus on or
                              off) as one CUDA graph and replayed, one host synchronisation per
                              step; 0 host-driven sweeps.  Bitwise the same results.
                              Default 1                                                      */
    int coarse_min_rows;   /* cell-by-cell contexts with coarse blocks (sdc_set_coarse_blocks):
                              node solves of sweeps with fewer active rows than this use Jacobi
                              alone (small sets converge in few iterations, where the coarse
                              space's set-up and per-iteration cost do not pay); default 0:
                              every solve uses the two-level preconditioner                 */
} sdc_options;

/* Per-step statistics (valid when sdc_step returns).                              */
typedef struct {
    int sweeps_run;
    int n_active[SDC_MAX_SWEEPS];          /* |I_k| for k = 0 .. sweeps_run-1              */
    long long nnz_active[SDC_MAX_SWEEPS];  /* stored off-diagonal entries of K[I_k, I_k]   */
    int cg_iters[SDC_MAX_SWEEPS][SDC_MAX_M];
    double cg_relres_max;                  /* max final sqrt(r'z / r0'z0) over all solves */
    double min_margin;                     /* min over selections of |max_m|dv| - TOL_drop| */
    int kernel_launches;                   /* kernels this step launched                    */
    /* per phase SDC_PHASE_*: launches, and device ms when the profile option is set */
    int phase_launches[SDC_N_PHASES];
    double phase_ms[SDC_N_PHASES];
    double cg_ms[SDC_MAX_SWEEPS][SDC_MAX_M];  /* device ms per node solve (profile option) */
    double energy[SDC_MAX_SWEEPS];         /* E_k = sum_m dv_m' A~_m dv_m of sweep k, from the CG
                                              scalars (sum of alpha gamma over each solve)    */
    double tol_drop;                       /* the drop tolerance the step's selections used   */
    int captured;                          /* 1: the step ran as a replayed CUDA graph        */
} sdc_stats;

/* Fill defaults (values above). */
void sdc_default_options(sdc_options* opt);
/* Standard Aliev-Panfilov parameters: ga = gs = 8, a = 0.15, eps = 0.002,
 * mu1 = 0.2, mu2 = 0.3, cw = 1. */
void sdc_default_ionic(sdc_ionic* ion);

/* Radau-IIA collocation data (Sec. 3.1): right Radau nodes tau[M] on [0, 1]
 * with tau[M-1] = 1; cumulative quadrature Q[m*M + j] = integral over
 * [0, tau_m] of the Lagrange polynomial l_j on tau_1..tau_M; LU-trick
 * preconditioner Qhat = U^T where Q^T = L U (Doolittle), lower triangular
 * (Sec. 3.1, after eq. SDC).  Host-only; 1 <= M <= 8. */
sdc_status sdc_radau(int M, double* tau, double* Q, double* Qhat);

/* Create a context: copies the mesh, assembles K and m on the device
 * (Sec. 2.2), and allocates every device buffer a step needs for up to
 * n_nodes active dofs.  stream: a cudaStream_t (NULL = legacy default stream)
 * of the current device.  Returns SDC_E_INVALID for a malformed mesh or
 * M outside [1, 8]; SDC_E_NOMEM when device memory is short.
 * On failure *out is NULL. */
sdc_status sdc_create(sdc_ctx** out, const sdc_mesh* mesh, const sdc_ionic* ionic, int M,
                      const sdc_options* opt, void* stream);

/* Stimulus current I_stim = amp on the listed nodes for every step whose start
 * time t satisfies t_on <= t < t_off (constant over the step).  nodes: host,
 * n entries in [0, n_nodes).  Replaces any previous stimulus; n = 0 clears. */
sdc_status sdc_set_stimulus(sdc_ctx* ctx, const int* nodes, int n, double amp, double t_on,
                            double t_off);

/* One SDC time step [t, t + dt] (Sec. 3.2 eq. final-sdc with the nested
 * index sets of Sec. 4.2).
 *   d_v, d_w  device, n_nodes doubles each: the state at t on entry, the state
 *             at t + dt (last Radau node) on return; updated in place
 *   sweeps    number of sweeps K (1 .. 64); the first sweep uses every dof
 *   TOL       SDC tolerance >= 0; TOL_drop = alpha * TOL, TOL = 0 is plain SDC
 *   stats     NULL or filled on return
 * Synchronises the context's stream.  Errors: SDC_E_CG_NOCONV, SDC_E_TIMEOUT,
 * SDC_E_NONFINITE, SDC_E_DOMAIN (the state is then partially updated). */
sdc_status sdc_step(sdc_ctx* ctx, double* d_v, double* d_w, double t, double dt, int sweeps,
                    double TOL, sdc_stats* stats);

/* sdc_step on HOST arrays h_v, h_w (n_nodes doubles each, preferably pinned):
 * copies them to context-owned device buffers, steps, and copies the result
 * back before returning. */
sdc_status sdc_step_host(sdc_ctx* ctx, double* h_v, double* h_w, double t, double dt, int sweeps,
                         double TOL, sdc_stats* stats);

/* Collocation-node values of the last step, d_V and d_W device arrays of
 * M * n_nodes doubles laid out [m][node]. */
sdc_status sdc_get_nodes(const sdc_ctx* ctx, double* d_V, double* d_W);

/* Active index list I_k of sweep k of the last step, ascending, copied to the
 * host array h_idx (capacity n_nodes).  *n receives |I_k|. */
sdc_status sdc_get_active(const sdc_ctx* ctx, int sweep, int* h_idx, int* n);

/* Sizes of the assembled system: node count and stored entries of K
 * (diagonal included, after the drop_rel filter). */
sdc_status sdc_get_info(const sdc_ctx* ctx, int* n_nodes, long long* nnz, int* max_row_offdiag);

/* The assembled K as host CSR (rows ascending, columns ascending, diagonal
 * included) and the lumped mass m; arrays sized by sdc_get_info. */
sdc_status sdc_get_matrix(const sdc_ctx* ctx, int* row_ptr, int* col, double* val, double* mass);

/* One node system of eq. final-sdc solved on its own (Sec. 3.2; Jacobi-PCG as
 * in Sec. 4.2):
 *     (diag(mass .* (1 + c J)) + c K) x = b,
 * by preconditioned CG from x = 0 with the diagonal preconditioner, stopping
 * when sqrt(r'z) <= rtol sqrt(r0'z0).  K is given by its diagonal d_kdiag[n]
 * and its off-diagonal part in column-major ELL slots: row i holds
 * d_len[i] <= width entries, entry t at d_val[t * ld + i], column
 * d_col[t * ld + i] in [0, n); ld >= n.  Every array is caller-owned device
 * memory of the current device; d_x receives the solution.  The workspace
 * (8 n + 2 ld doubles plus a few per SM) is allocated and freed inside the call, which
 * synchronises `stream` (a cudaStream_t, NULL = legacy default).  iters and
 * relres (host, may be NULL) receive the iteration count and the final
 * sqrt(r'z / r0'z0).  Errors: SDC_E_INVALID (nothing launched),
 * SDC_E_NOMEM, SDC_E_CG_NOCONV, SDC_E_NONFINITE, SDC_E_DOMAIN (a non-positive
 * diagonal); details from sdc_last_error(NULL) on the calling thread. */
sdc_status sdc_pcg_solve(int n, const double* d_val, const int* d_col, const int* d_len, int ld,
                         int width, const double* d_kdiag, const double* d_mass, const double* d_J,
                         double c, const double* d_b, double* d_x, double rtol, int maxit,
                         int* iters, double* relres, void* stream);

/* ---- Differentiation: tape, replay and the discrete adjoint of a step ----
 *
 * With the nested index sets of a step held fixed, the step is a smooth map
 * (v0, w0; s, ga, gs, a) -> (v, w) once every node solve is read as the exact
 * solution of its linear system.  A tape records what the reverse pass needs:
 * the collocation-node values after every sweep and the active lists. */
#define SDC_TAPE_OFF 0
#define SDC_TAPE_RECORD 1   /* sdc_step_taped fills the tape                     */
#define SDC_TAPE_REPLAY 2   /* sdc_step_taped takes its active sets from the tape */

typedef struct {
    int mode;
    int sweeps;                      /* sweeps recorded (set by RECORD)                     */
    double* d_V;                     /* device, sweeps * n_nodes * M doubles (caller-owned) */
    double* d_W;                     /* same                                                */
    int* d_act;                      /* device, sweeps * n_nodes ints: list of sweep k >= 1 */
    int n_active[SDC_MAX_SWEEPS];    /* |I_k|, host                                         */
} sdc_tape;

/* Bytes of device memory a tape of `sweeps` sweeps needs (d_V + d_W + d_act). */
size_t sdc_tape_bytes(const sdc_ctx* ctx, int sweeps);

/* sdc_step with a tape: RECORD stores the state after each sweep and the active
 * lists; REPLAY runs the step with the recorded active sets instead of
 * selecting new ones (the tape's sweeps must equal `sweeps`); TOL then only
 * matters for the statistics.  A NULL tape or mode OFF is sdc_step. */
sdc_status sdc_step_taped(sdc_ctx* ctx, double* d_v, double* d_w, double t, double dt, int sweeps,
                          double TOL, sdc_stats* stats, sdc_tape* tape);

/* Discrete adjoint of the step recorded on `tape` (Sec. 3.2 eq. final-sdc,
 * Sec. 4.2, active sets fixed).  Given the adjoints d_lam_v, d_lam_w of the
 * step's outputs, writes the adjoints d_lam_v0, d_lam_w0 of its inputs d_v0,
 * d_w0 (the state the recorded step started from, device), adds dL/ds to
 * d_grad_scale (device, n_nodes; may be NULL), s being the per-node
 * conductivity scale, and adds dL/d(ga, gs, a) to grad_ionic[3] (host; may be
 * NULL).  The reverse node solves use the forward's Jacobi-PCG with the
 * context's cg_rtol.  Synchronises the stream.  Not available for batches. */
sdc_status sdc_step_adjoint(sdc_ctx* ctx, const sdc_tape* tape, const double* d_v0,
                            const double* d_w0, double dt, const double* d_lam_v,
                            const double* d_lam_w, double* d_lam_v0, double* d_lam_w0,
                            double* d_grad_scale, double* grad_ionic);

/* Re-assemble K for a new per-node conductivity scale (host, n_nodes positive
 * values; NULL = all ones) on the context's mesh. */
sdc_status sdc_set_dof_scale(sdc_ctx* ctx, const double* h_scale);

/* Replace the ionic parameters of a context. */
sdc_status sdc_set_ionic(sdc_ctx* ctx, const sdc_ionic* ionic);

/* ---- Batches: many independent instances advanced by the same launches ----
 *
 * A batch stacks instances (meshes of the same dimension, each with its own
 * conductivity, stimulus and size) as disjoint diagonal blocks of one system.
 * Every kernel of the step runs once for the whole batch; the node solves run
 * one independent Jacobi-PCG per instance inside one cooperative launch (own
 * reductions, own stopping test, own iteration count), so each instance
 * follows the same iteration as a solo context up to the rounding order of
 * its dot products.  All instances share M, the ionic parameters, the options,
 * dt, the number of sweeps, TOL and one stimulus window. */
typedef struct sdc_batch sdc_batch;

/* meshes: n_instances meshes (host, copied).  Instance b owns the dofs
 * offsets[b] .. offsets[b+1]-1 of the batch state (see sdc_batch_info), in its
 * own node order. */
sdc_status sdc_batch_create(sdc_batch** out, const sdc_mesh* meshes, int n_instances,
                            const sdc_ionic* ionic, int M, const sdc_options* opt, void* stream);

/* n_instances and offsets[n_instances + 1] (host; either may be NULL). */
sdc_status sdc_batch_info(const sdc_batch* batch, int* n_instances, int* offsets);

/* Stimulus amp on the listed nodes (instance-local numbering) of one
 * instance; every instance must use the same window [t_on, t_off). */
sdc_status sdc_batch_set_stimulus(sdc_batch* batch, int instance, const int* nodes, int n,
                                  double amp, double t_on, double t_off);

/* One step of every instance: d_v, d_w hold the concatenated states
 * (offsets[n_instances] doubles each).  stats aggregates the batch
 * (n_active summed, cg_iters the maximum over instances). */
sdc_status sdc_batch_step(sdc_batch* batch, double* d_v, double* d_w, double t, double dt,
                          int sweeps, double TOL, sdc_stats* stats);

/* Per-instance statistics of sweep `sweep` of the last step: n_active[n_instances]
 * and cg_iters[M][n_instances] (host; either may be NULL). */
sdc_status sdc_batch_instance_stats(const sdc_batch* batch, int sweep, int* n_active,
                                    int* cg_iters);

/* The batch's underlying context (for sdc_get_nodes, sdc_get_active,
 * sdc_get_matrix on the stacked system); owned by the batch. */
sdc_ctx* sdc_batch_context(sdc_batch* batch);

/* ---- launch-shape autotuner --------------------------------------------------
 * The node solves (Sec. 3.2, eq. final-sdc) dominate a step, and their best launch
 * shape depends on the mesh, the active-set sizes the adaptivity produces and the
 * part.  sdc_autotune times `trial_steps` steps (1..100) from the state (d_v, d_w)
 * at (t, dt, sweeps, TOL) under candidate configurations, one knob at a time in
 * the order below (coordinate descent, each value tried with the others at their
 * best so far), and keeps the fastest; a value must beat the incumbent by 3 % to
 * be adopted (each configuration is timed twice from the restored state, the
 * better run counting).  The state arrays are restored bitwise before returning.  Every
 * configuration computes the same iteration (results differ by rounding only).
 *   single context: cg_pipelined {1, 0}; cg_scaled {1, 0}; shared-memory block
 *     size {512, 1024}; rows from which the shared-memory variants use 1024
 *     threads {0, 100000, 300000, never}; general-variant block size {256, 512,
 *     1024}; cluster_rows {0, 2000, 5000, 10000, 20000 (within the cluster's
 *     capacity)};
 *   batch: arrangement {classical, pipelined}; cg_scaled {1, 0}; block size
 *     {256, 512, 1024}; target active rows per block {256, 512, 1024, 2048, 4096}.
 * Candidates whose cooperative grid would exceed the context's reserved
 * per-block workspace are skipped.  Device time is measured with CUDA events on
 * the context's stream.  Errors of a trial step are returned (the state is
 * restored and the incumbent configuration kept).  out may be NULL. */
typedef struct {
    int trials;                 /* configurations timed, the starting one included   */
    double base_ms;             /* ms per step of the starting configuration          */
    double best_ms;             /* ms per step of the chosen configuration            */
    int cg_pipelined, cg_scaled, smem_block, big_rows, general_block, cluster_rows;
    int batch_pipelined, batch_block, batch_rows_per_block;   /* chosen values */
} sdc_tune_report;

sdc_status sdc_autotune(sdc_ctx* ctx, double* d_v, double* d_w, double t, double dt, int sweeps,
                        double TOL, int trial_steps, sdc_tune_report* out);
sdc_status sdc_batch_autotune(sdc_batch* batch, double* d_v, double* d_w, double t, double dt,
                              int sweeps, double TOL, int trial_steps, sdc_tune_report* out);

void sdc_batch_destroy(sdc_batch* batch);

/* ---- Cell-by-cell (EMI) model: membranes resolved between subdomains ----
 *
 * Sec. 2.1 (eqs. of the cell-by-cell model) in the abstract form of Sec. 3:
 *     B u' = -(K + diag(robin)) u - b(u, w),     w_p' = R(u_k - u_l, w_p)
 * with one potential dof per (mesh vertex, subdomain), K the P1 stiffness of
 * every subdomain (the mesh's elements carry their subdomain's conductivity
 * and use the dofs of that subdomain), and the membranes lumped onto dof
 * pairs p = (k, l) of area A_p:
 *     B = sum_p A_p Cm (e_k - e_l)(e_k - e_l)^T,
 *     b = sum_p A_p I_p(u_k - u_l, w_p) (e_k - e_l),
 *     I_p = I_ion of the Aliev-Panfilov model (kind 0, cell-bath membrane, k
 *           on the cell side) or g_gap v (kind 1, gap junction between cells).
 * The step is the SDC sweep of sdc_step with B in place of the lumped mass
 * and sum_p A_p dI_p/dv (e_k - e_l)(e_k - e_l)^T in place of the lumped
 * ionic Jacobian; the gating sweep runs over the kind-0 pairs with at least
 * one active end.  Host arrays, copied at sdc_create_emi:
 *   n_pairs              number of pairs (>= 1)
 *   pair_k, pair_l       dofs of each pair, distinct, in [0, n_nodes)
 *   pair_area            lumped membrane measure A_p > 0
 *   pair_kind            0 or 1
 *   robin                NULL or n_nodes values >= 0 (Robin coefficient times
 *                        the lumped boundary measure of each dof)
 *   Cm > 0, g_gap >= 0                                                           */
typedef struct {
    int n_pairs;
    const int* pair_k;
    const int* pair_l;
    const double* pair_area;
    const int* pair_kind;
    const double* robin;
    double Cm;
    double g_gap;
} sdc_emi;

/* Create a context for the cell-by-cell model.  mesh as for sdc_create
 * (elem_sigma normally per element); its lumped mass is not used.  On such a
 * context sdc_step and sdc_step_host take d_v = the n_nodes potentials u and
 * d_w = the n_pairs gating values (entries of kind-1 pairs are left as
 * given); sdc_get_nodes writes M * n_nodes potentials and M * n_pairs gating
 * values, both [m][index].  In sdc_stats, nnz_active[k] counts the stored
 * off-diagonal entries of the node-solve operator: those of K[I_k, I_k] plus
 * one per pair end whose other end is also active; the operator is built per
 * node (phase EXTRACT), the coupling into the later nodes' right-hand sides
 * runs after each solve (phase UPDATE).  Not available on such a context:
 * tapes, the adjoint, stimuli, sdc_set_dof_scale (SDC_E_INVALID). */
sdc_status sdc_create_emi(sdc_ctx** out, const sdc_mesh* mesh, const sdc_emi* emi,
                          const sdc_ionic* ionic, int M, const sdc_options* opt, void* stream);

/* Two-level preconditioner of the node solves of a cell-by-cell context.  Sec. 6
 * proposes block preconditioners with a selection of the blocks for EMI systems,
 * whose Jacobi-preconditioned solves run for hundreds to thousands of iterations:
 * their slow modes are nearly constant on each floating cell and vary slowly over
 * the extracellular space.  Given blocks (every dof in one block: each cell, and
 * pieces of the extracellular space), each node system A (Sec. 3.2, restricted to
 * the active set I_k) is solved by CG preconditioned with
 *     z = D^-1 r + Z E^-1 Z' r,    E = Z' A Z,
 * Z the indicator vectors of the blocks that hold active dofs (the block selection);
 * D^-1 alone is the default Jacobi preconditioner.  E is formed per node solve in
 * exact 64-bit fixed point (terms rounded at 2^-41 of the largest diagonal entry) and
 * inverted by Gauss-Jordan elimination on the device; results stay bitwise
 * reproducible.
 *   block_of_dof  host, n_nodes labels in [0, n_blocks) (copied)
 *   n_blocks      1 .. SDC_MAX_COARSE_BLOCKS; block_of_dof NULL or n_blocks 0
 *                 switches the two-level preconditioner off
 * Cell-by-cell contexts only (else SDC_E_INVALID); SDC_E_NOMEM when device memory
 * is short.  A CG iteration keeps the Jacobi solve's two grid synchronisations (the
 * block sums of Y'r travel with the dot products); each solve adds the set-up of E
 * and its inverse (one grid barrier per 16 blocks).  The solve's rows run in tiles
 * of the active rows sorted by block: numbering the dofs block by block keeps each
 * tile contiguous in memory.  A step returns SDC_E_INVALID if one CTA's share of the
 * pieces (tile/block intersections) and the pieces' sums exceed the launch's shared
 * memory (about 13 M active rows and more). */
#define SDC_MAX_COARSE_BLOCKS 1024
sdc_status sdc_set_coarse_blocks(sdc_ctx* ctx, const int* block_of_dof, int n_blocks);

/* Largest n accepted by sdc_pcg_solve_noalloc. */
#define SDC_PCG_NOALLOC_MAX_ROWS 65536

/* sdc_pcg_solve for callers that cannot allocate device memory (the paper has
 * no counterpart; this is a service of the library).  Same arguments, results
 * and errors as sdc_pcg_solve, but no device memory is allocated or freed:
 * the workspace is a static array of the library, reserved (about 5.6 MB) on
 * every GPU that loads the library until the process exits.
 *   - n <= SDC_PCG_NOALLOC_MAX_ROWS and 9 n + ld <= 10 SDC_PCG_NOALLOC_MAX_ROWS, else
 *     SDC_E_INVALID with a message from sdc_last_error(NULL), and nothing is launched.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture starts on the device.  After cudaDeviceReset the next
 *     call looks the address up again in the device's new context.
 *   - Every call on a device uses the same array; calls that overlap on the GPU
 *     (other streams, other host threads) race.  Serialise them.
 * Meant for host frameworks that hand out all device memory from their own
 * pool, and for time-critical loops where cudaMalloc/cudaFree may block. */
sdc_status sdc_pcg_solve_noalloc(int n, const double* d_val, const int* d_col, const int* d_len,
                                 int ld, int width, const double* d_kdiag, const double* d_mass,
                                 const double* d_J, double c, const double* d_b, double* d_x,
                                 double rtol, int maxit, int* iters, double* relres, void* stream);

/* One-line description of the last failure on ctx (never NULL). */
const char* sdc_last_error(const sdc_ctx* ctx);
const char* sdc_status_string(int status);

/* Free every device and host resource of ctx (NULL is ignored). */
void sdc_destroy(sdc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SDC_GB300_H */
