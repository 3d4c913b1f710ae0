/*
 * rs.h — C ABI of the GB300 preconditioned Krylov library.
 *
 * The calls follow the paper's statement of the problem (Liu & Chen,
 * "Scalable linear solvers for sparse linear systems from large-scale
 * numerical simulations"): vectors (Sec. 2.2, Figs. 6-13), matrices and
 * matrix-vector products (Sec. 2.3, Figs. 15-21), preconditioners with
 * setup / apply / destroy (Sec. 3, Fig. 29; Sec. 4), and solvers returning
 * an iteration count and a residual (Sec. 3, Fig. 22, Alg. 1).
 *
 * General rules
 *  - Every call returns an rs_status (0 = success); nothing asserts or exits.
 *  - All work is ordered on the stream given to rs_init.  Calls that return
 *    a host scalar (rs_vec_dot, rs_vec_norm2), copy to host (rs_vec_get with
 *    RS_MEM_HOST) or solve (rs_solve_*) synchronise that stream before they
 *    return; all other calls only enqueue work.
 *  - Handles are created by *_create / *_setup, owned by the caller and
 *    released with the matching *_destroy(&h), which sets *h to NULL.
 *    A matrix or vector must outlive every preconditioner built from it.
 *  - Creation calls copy the caller's arrays (host or device, per `mem`);
 *    the caller keeps ownership of what it passed in.
 *  - Indices are int32, 0-based.  CSR/BSR rows must list their columns in
 *    strictly ascending order and hold the diagonal; violations return
 *    RS_ERR_BAD_PATTERN.
 *  - Every device-side wait is bounded; a wait that runs out makes the call
 *    return RS_ERR_DEVICE_TIMEOUT and leaves the context usable.
 */
#ifndef RS_H
#define RS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_ctx rs_ctx;
typedef struct rs_mat rs_mat;
typedef struct rs_vec rs_vec;
typedef struct rs_pc rs_pc;
typedef struct rs_net rs_net;

typedef enum {
    RS_OK = 0,
    RS_NOT_CONVERGED = 1,        /* maxit reached; x holds the last iterate   */
    RS_ERR_INVALID_ARG = -1,
    RS_ERR_BAD_PATTERN = -2,     /* unsorted / missing diagonal / out of range */
    RS_ERR_ZERO_PIVOT = -3,      /* zero or non-finite pivot (row in info)    */
    RS_ERR_BREAKDOWN = -4,       /* BiCGSTAB rho or (rhat, v) vanished        */
    RS_ERR_DEVICE_TIMEOUT = -5,  /* a bounded device-side wait expired        */
    RS_ERR_CUDA = -6,
    RS_ERR_OOM = -7,
    RS_ERR_SIZE_MISMATCH = -8
} rs_status;

typedef enum { RS_MEM_HOST = 0, RS_MEM_DEVICE = 1 } rs_mem;

typedef enum {
    RS_PC_NONE = 0,
    RS_PC_ILU0 = 1,       /* ILU(0) of a CSR matrix (Sec. 4.1, Eq. 3)        */
    RS_PC_BILU0 = 2,      /* block ILU(0) of a BSR matrix                     */
    RS_PC_CPR = 3,        /* two-stage CPR, pressure stage ILU(0) (Alg. 6)    */
    RS_PC_CPR_LEARNED = 4, /* two-stage CPR, pressure stage = learned network */
    RS_PC_RAS = 5,        /* restricted additive Schwarz, ILU(k) local solver
                             (Sec. 4.1)                                        */
    RS_PC_AMG = 6         /* algebraic multigrid V-cycle (Sec. 4.2, Algs. 3-4) */
} rs_pc_type;

typedef enum {
    RS_FP64 = 0,          /* factors and applies in FP64                      */
    RS_MIXED = 1          /* FP32 factors and applies, FP64 Krylov outer loop */
} rs_prec;

/* Order of the stages of a CPR-like preconditioner (Sec. 4.3): F = the block
 * ILU(0) of the full system, R(A)^{-1}; P = the pressure correction
 * Pi_p M_p^{-1} Pi_r.  The first stage maps f to x; each later stage forms
 * r = f - A x and adds its correction to x. */
typedef enum {
    RS_CPR_PF = 0,        /* Alg. 6, read as x = P f; r = f - A x; x += F r   */
    RS_CPR_FP = 1,        /* Alg. 5                                           */
    RS_CPR_FPF = 2,       /* Alg. 7                                           */
    RS_CPR_FFPF = 3       /* Alg. 8                                           */
} rs_cpr_form;

typedef struct {
    int32_t prec;         /* rs_prec                                          */
    int32_t nx, ny, nz;   /* grid of the pressure unknowns (learned stage)    */
    const rs_net *net;    /* trained network (RS_PC_CPR_LEARNED)              */
    const double *log_perm; /* device pointer, nx*ny*nz log-permeabilities    */
    int32_t cpr_form;     /* rs_cpr_form (RS_PC_CPR, RS_PC_CPR_LEARNED); 0 = PF */
    /* RS_PC_RAS (Sec. 4.1, Figs. 30-31).  A zeroed field takes the value
     * in brackets. */
    int32_t ras_nparts;   /* subdomains, >= 1 [1]                               */
    int32_t ras_overlap;  /* layers of the graph of A added to each, >= 0 [0]   */
    int32_t ilu_level;    /* k of the local ILU(k), 0..8 [0]                    */
    const int32_t *ras_part; /* host array: subdomain of each (block) row, in
                                [0, ras_nparts); NULL = contiguous ranges of
                                rows, row i in floor(i nparts / n), like the
                                paper's row distribution (Sec. 2.1, Eq. 1) */
    /* RS_PC_AMG, and the AMG pressure stage of CPR (Sec. 4.2, Fig. 34).  A
     * zeroed field takes the value in brackets. */
    double amg_theta;       /* strength threshold, 0 < theta <= 1 [0.5]      */
    int32_t amg_max_levels; /* 1..16 [16]                                     */
    int32_t amg_max_coarse; /* rows at which coarsening stops, >= 1 [256]     */
    int32_t amg_nu;         /* smoothing sweeps before and after, >= 1 [2]    */
    int32_t cpr_pstage;     /* RS_PC_CPR pressure stage: 0 ILU(0) of the
                               decoupled matrix, 1 one AMG V-cycle on it     */
    /* RAS local solver (Fig. 31): 0 ILU(ilu_level), 1 ILUT(ilut_p, ilut_tol)
     * (scalar matrices), factorised on the GPU one subdomain per warp, since
     * its pattern depends on the values.  ILUT drops entries below
     * ilut_tol * ||a_i||_2 and keeps
     * the ilut_p largest of each part of a row (negative: as many as the
     * row of A has there).  Zeroed fields take the paper's defaults: p = -1,
     * tol = 1e-3. */
    int32_t ras_local;
    int32_t ilut_p;
    double ilut_tol;
    /* AMG smoother: 0 l1-Jacobi, x <- x + (b - A x) / d with d_i the row's
     * absolute sum [0]; 1 hybrid Gauss-Seidel (Fig. 34's relaxation), read
     * as Gauss-Seidel inside chunks of 32 consecutive rows and Jacobi between
     * chunks, forward before the coarse correction and backward after it;
     * it needs a nonzero diagonal on every level (else RS_ERR_ZERO_PIVOT). */
    int32_t amg_smoother;
    /* Triangular sweeps of every ILU(0) / block ILU(0) factor of this
     * preconditioner (Eq. 3).  0 [0]: the library's choice, at present the
     * same as 2 (measured faster than the segment sweeps on every grid
     * workload); 1: the segment sweeps; 2: the wavefront sweeps, taken when
     * the pattern is (a subset of) the 7-point stencil of a structured grid
     * in natural order (x fastest; the grid is read off the pattern), else
     * the segment sweeps.  RAS local factors always take the segment
     * sweeps. */
    int32_t sweep;
    /* Segment sweeps: the longest run of segments one warp carries, > 0 (1:
     * no runs).  0 [0]: no limit for FP64 scalar factors, no runs for FP32
     * and block factors (runs serve scalar factors only). */
    int32_t sweep_run_cap;
} rs_pc_opts;

typedef struct {
    int32_t iters;            /* inner iterations (Arnoldi steps / BiCGSTAB loops) */
    int32_t restarts;         /* completed GMRES cycles                       */
    int32_t status;           /* rs_status of the solve                       */
    int32_t bad_row;          /* row of a zero pivot, else -1                 */
    double true_rel_res;      /* ||b - A x||_2 / ||b||_2, recomputed in FP64  */
    double implicit_rel_res;  /* the solver's own residual estimate / ||b||   */
    double solve_s;           /* wall time of the solve call                  */
} rs_solve_info;

/* ---- context --------------------------------------------------------- */

/* Binds the library to CUDA device `device` and the caller's stream
 * (a cudaStream_t passed as void*; NULL = the legacy default stream). */
int rs_init(rs_ctx **ctx, int device, void *cuda_stream);
int rs_finalize(rs_ctx **ctx);
/* Waits for all work enqueued on the context's stream. */
int rs_sync(rs_ctx *ctx);
/* Residual history of the solves (a diagnostic; the paper's solver reports
 * only the final residual and the iteration count, Sec. 2.4).  While hist is
 * set, every solve on this context writes, for each of its inner iterations
 * k = 1, 2, ... up to len, the solver's own relative residual estimate after
 * iteration k into hist[k-1]:
 *   GMRES / FGMRES / LGMRES: |g_{k+1}| / ||b||, the residual of the rotated
 *     least-squares problem of Alg. 1 (Givens rotations);
 *   BiCGSTAB: ||r|| / ||b|| after the full loop, or ||s|| / ||b|| on a
 *     half-step exit;
 *   CG (Alg. 2): ||r|| / ||b|| of the recursive residual.
 * hist is host memory of at least len doubles, owned by the caller and
 * written when the solve returns; entries past the solve's iteration count
 * are left as they were.  hist = NULL or len = 0 stops the recording;
 * len < 0 is RS_ERR_INVALID_ARG.  Recording costs one device array of len
 * doubles per solve and one copy at its end. */
int rs_set_history(rs_ctx *ctx, double *hist, int32_t len);
/* Every device-side wait of the library (a kernel polling for a value, a
 * level or a copy) gives up after this many clock cycles, records
 * RS_ERR_DEVICE_TIMEOUT in the context's device error word and returns; the
 * context stays usable.  cycles = 0 restores the default (about two
 * seconds); negative is RS_ERR_INVALID_ARG. */
int rs_set_spin_limit(rs_ctx *ctx, int64_t cycles);
/* Synchronises the stream, then reads and clears the device error word:
 * RS_OK, RS_ERR_DEVICE_TIMEOUT (a bounded wait gave up since the last
 * check), RS_ERR_ZERO_PIVOT or RS_ERR_CUDA.  The solvers check it
 * themselves; a caller of the preconditioner applies alone uses this. */
int rs_check_device(rs_ctx *ctx);
const char *rs_status_str(int status);
/* Number of kernels this library has launched on the context so far. */
int64_t rs_launch_count(const rs_ctx *ctx);

/* Optional profiler: when enabled, every kernel the library launches is
 * bracketed by CUDA events on the context's stream and its device time is
 * added to its class.  Classes, in order: SpMV, L sweep, U sweep, CGS dots,
 * CGS update+dots, CGS update+norm, BLAS-1, other preconditioner kernels,
 * factorisation, solver scalar kernels, network, block L sweep, block U
 * sweep, CPR pressure-column residual.  nkinds >= 14. */
int rs_prof_enable(rs_ctx *ctx, int on);
/* Reads (and with reset != 0 clears) the accumulated milliseconds and launch
 * counts per class; synchronises the stream. */
int rs_prof_read(rs_ctx *ctx, double *ms, int64_t *launches, int32_t nkinds, int reset);

/* ---- vectors (Sec. 2.2) ----------------------------------------------- */

/* VecCreate (Fig. 7): an owned FP64 device vector of n entries, zeroed. */
int rs_vec_create(rs_ctx *ctx, int32_t n, rs_vec **v);
/* A non-owning view of n FP64 values at device address `dev` (e.g. memory
 * allocated by PyTorch).  The memory must stay valid while the view lives. */
int rs_vec_wrap(rs_ctx *ctx, int32_t n, double *dev, rs_vec **v);
int rs_vec_destroy(rs_vec **v);
int32_t rs_vec_size(const rs_vec *v);
double *rs_vec_data(rs_vec *v);
/* Copy n values in from / out to host or device memory. */
int rs_vec_set(rs_vec *v, const double *src, int mem);
int rs_vec_get(const rs_vec *v, double *dst, int mem);
/* VecSetValue (Fig. 13): x_i = a. */
int rs_vec_set_value(rs_vec *x, double a);
/* VecAXPBY (Fig. 10): y = a x + b y. */
int rs_vec_axpby(double a, const rs_vec *x, double b, rs_vec *y);
/* VecAXPBYZ (Fig. 11): z = a x + b y. */
int rs_vec_axpbyz(double a, const rs_vec *x, double b, const rs_vec *y, rs_vec *z);
/* VecDot (Fig. 12): *out = <x, y> (deterministic tree reduction). */
int rs_vec_dot(const rs_vec *x, const rs_vec *y, double *out);
/* *out = ||x||_2. */
int rs_vec_norm2(const rs_vec *x, double *out);

/* h[j] = <V_j, w> for the k columns V_j (column j at V + j*ld, n entries
 * each), like the first pass of the CGS2 step, but without allocating any
 * device memory: for callers that cannot call cudaMalloc (work recorded
 * while a stream is captured into a graph, hosts that own all device
 * memory).  The paper has no counterpart; this is a service of the library.
 * All pointers are device pointers; the call is ordered on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream) and does not synchronise.
 * Its scratch is a fixed static device array (512 KB per GPU that loads the
 * library, held until exit), shared by every call: calls that overlap on the
 * GPU race.  1 <= k <= 64 (larger k returns RS_ERR_INVALID_ARG); ld >= n.
 * The call runs on the device the stream belongs to (the current device for
 * the default streams).  The first call on a device looks up the array's
 * device address and keeps it for the life of the process; make it before
 * any stream capture.  A reset of the device (cudaDeviceReset) makes that
 * address stale: restart the process before calling again. */
int rs_vec_mdot_noalloc(const double *V, int32_t ld, int32_t n, int32_t k, const double *w,
                        double *h, void *cuda_stream);

/* ---- matrices (Sec. 2.3) ---------------------------------------------- */

/* MatCreate/MatAssemble (Figs. 16-19) for an n x n CSR matrix:
 * rowptr[n+1], col[nnz], val[nnz] (FP64), host or device per `mem`. */
int rs_mat_create_csr(rs_ctx *ctx, int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, int mem, rs_mat **A);
/* A block matrix of nb x nb blocks of size bs x bs (bs = 3 for the
 * black-oil systems of Eq. 9, one block per cell): browptr[nb+1],
 * bcol[nnzb], bval[nnzb*bs*bs] with each block row-major. */
int rs_mat_create_bsr(rs_ctx *ctx, int32_t nb, int32_t bs, const int32_t *browptr,
                      const int32_t *bcol, const double *bval, int mem, rs_mat **A);
int rs_mat_destroy(rs_mat **A);
/* Scalar dimension (n for CSR, nb*bs for BSR). */
int32_t rs_mat_size(const rs_mat *A);
/* MatVecMXY (Fig. 20): y = A x. */
int rs_mat_spmv(const rs_mat *A, const rs_vec *x, rs_vec *y);
/* MatVecAMXPBY (Fig. 21): y = a A x + b y (b = 0 ignores y's contents). */
int rs_mat_amxpby(double a, const rs_mat *A, const rs_vec *x, double b, rs_vec *y);

/* ---- preconditioners (Sec. 3 Fig. 29, Sec. 4) -------------------------- */

/* Builds M for A.  RS_PC_ILU0 needs a CSR matrix; RS_PC_BILU0 a BSR matrix;
 * RS_PC_AMG needs a CSR matrix (setup of the hierarchy and the V-cycle on
 * the GPU: classical strength, PMIS coarsening with SplitMix64 weights keyed
 * by level and row, direct interpolation, Galerkin products; RS_ERR_INVALID_ARG
 * when coarsening stalls above 4096 rows, a Galerkin row has more than 2048
 * candidate terms, or an option is out of range);
 * RS_PC_RAS either (on a BSR matrix the subdomains hold block rows and the
 * local solver is block ILU(k)), set by the opts->ras_* fields and
 * opts->ilu_level (RS_ERR_INVALID_ARG when out of range);
 * RS_PC_CPR a BSR matrix (quasi-IMPES pressure restriction, ILU(0) of the
 * decoupled pressure matrix, block ILU(0) of A) or a CSR matrix (pressure
 * stage on A itself, second stage ILU(0)); opts->cpr_form picks the order
 * of the stages (Algs. 5-8), opts->cpr_pstage the pressure stage, and
 * opts->ras_nparts > 1 (or ras_part) makes the F stage R(A)^{-1} restricted
 * additive Schwarz over those (block) subdomains instead of block ILU(0).  opts may be NULL (FP64, CPR-PF).
 * Returns RS_ERR_ZERO_PIVOT when a factorisation meets a zero pivot and
 * RS_ERR_INVALID_ARG for an unknown cpr_form. */
int rs_precond_setup(rs_ctx *ctx, const rs_mat *A, int type, const rs_pc_opts *opts,
                     rs_pc **M);
/* z = M^{-1} r. */
int rs_precond_apply(rs_pc *M, const rs_vec *r, rs_vec *z);
/* Copies the ILU(0) factor values (FP64, in the pattern of the factored
 * matrix: strict lower part of L, then U with its diagonal) to host memory.
 * For RS_PC_CPR the factored matrix is the decoupled pressure matrix. */
int rs_precond_get_ilu(const rs_pc *M, double *lu_host, int32_t nnz);
/* Block ILU(0) factors: lu_host[nnzb*bs*bs] and the inverted diagonal
 * blocks dinv_host[nb*bs*bs]. */
int rs_precond_get_bilu(const rs_pc *M, double *lu_host, double *dinv_host);
/* CPR on a block matrix: quasi-IMPES weights w_host[nb*(bs-1)] and the
 * decoupled pressure matrix values app_host[nnzb] (block pattern of A).
 * Either pointer may be NULL. */
int rs_precond_get_cpr(const rs_pc *M, double *w_host, double *app_host);
/* Row of the last zero pivot met by setup, or -1. */
int32_t rs_precond_bad_row(const rs_pc *M);
/* RS_PC_AMG (or RS_PC_CPR with cpr_pstage = 1): number of levels of the
 * hierarchy; sizes of level l: rows of A_l, stored entries of A_l and of the
 * interpolation P_l (0 on the coarsest level). */
int rs_precond_amg_levels(const rs_pc *M, int32_t *nlevels);
int rs_precond_amg_level_sizes(const rs_pc *M, int32_t l, int32_t *n, int64_t *nnz_a, int64_t *nnz_p);
/* Level l to host memory: A_l (aptr[n+1], acol, aval), P_l (pptr[n+1],
 * pcol, pval; n x n_{l+1}) and cidx[n], the coarse index of each point
 * (-1 for F points); P_l and cidx only below the coarsest level.  Any
 * pointer may be NULL. */
int rs_precond_get_amg_level(const rs_pc *M, int32_t l, int32_t *aptr, int32_t *acol, double *aval,
                             int32_t *pptr, int32_t *pcol, double *pval, int32_t *cidx);
/* RS_PC_RAS: the extended subdomains are stacked, subdomain after
 * subdomain, into one block-diagonal matrix (rows of a subdomain in
 * ascending global order).  *next = its (block) rows, *nnz = its stored
 * (block) entries: A's entries inside each extended set plus the ILU(k)
 * fill. */
int rs_precond_ras_info(const rs_pc *M, int32_t *next, int64_t *nnz);
/* RS_PC_RAS: that matrix to host memory: gidx[next] = global (block) row of
 * each stacked row; ptr[next+1], col[nnz] its pattern (stacked numbering);
 * lu[nnz*bs*bs] the FP64 factor in that pattern (strict lower part of L,
 * then U with its diagonal).  Any pointer may be NULL. */
int rs_precond_get_ras(const rs_pc *M, int32_t *gidx, int32_t *ptr, int32_t *col, double *lu);
/* Critical-path length of the triangular sweeps of the full-system factor
 * (ILU(0), block ILU(0), or the second stage of CPR), L and U.  Segment
 * sweeps: the number of segment levels, where a segment is a run of at most
 * 32 consecutive (block) rows solved by one warp and a segment's level is
 * one more than the highest level of the segments it reads (Eq. 3 solved
 * row by row in dependency order).  Wavefront sweeps (a structured 7-point
 * pattern on an nx x ny x nz grid): the cells on the longest dependency
 * chain, nx + ny + nz - 2, each one step of the wavefront.  Which sweeps a
 * factor takes: rs_precond_sweep_kind.  RS_ERR_INVALID_ARG for RS_PC_NONE
 * or NULL arguments. */
int rs_precond_sweep_levels(const rs_pc *M, int32_t *levels_l, int32_t *levels_u);
/* The sweeps the full-system factor takes: *kind = 0 segment sweeps, 1
 * wavefront sweeps; for wavefronts (nx, ny, nz) is the grid read off the
 * pattern (else 0, 0, 0).  Any output but kind may be NULL. */
int rs_precond_sweep_kind(const rs_pc *M, int32_t *kind, int32_t *nx, int32_t *ny, int32_t *nz);
/* Runs of the same sweeps: a run is a sequence of segments that one warp
 * solves in turn, each segment reading the one before it from the warp's
 * registers (scalar factors only; block factors have one segment per run).
 * runs_l / runs_u: the number of runs of the L / U sweep, i.e. the tickets
 * the warps take; longest_l / longest_u: the segments of the longest run.
 * The number of runs never exceeds the number of segments.  Runs change the
 * schedule, not the arithmetic: results are those of one segment per run.
 * RS_ERR_INVALID_ARG for RS_PC_NONE or NULL arguments. */
int rs_precond_sweep_runs(const rs_pc *M, int32_t *runs_l, int32_t *runs_u, int32_t *longest_l,
                          int32_t *longest_u);
/* The schedule of one triangular sweep of a pattern, computed on the host
 * only (no device, no context): the analysis rs_precond_setup runs for the
 * sweeps of an ILU(0) factor in FP64.  ptr[nrows+1], col[ptr[nrows]]: a
 * square CSR pattern, columns strictly increasing within a row, every row
 * with its diagonal (else RS_ERR_BAD_PATTERN).  lower: 1 for the L sweep
 * (rows in increasing order, reading the strictly lower entries), 0 for the
 * U sweep.  run_cap: the longest run allowed (1: no runs); run_slots: the
 * most runs kept (a layout with more, or whose runs would not halve the
 * segments, takes one segment per run).  Outputs: nseg segments of up to 32
 * consecutive rows, seg_row0[nseg+1] their first rows (a caller array of
 * nrows+1), seg_level[nseg] their levels (a segment's level is one more than
 * the highest level of the segments it reads; array of nrows), nlevels,
 * and nrun runs in the order their tickets are taken, runs[nrun][5] = first
 * segment, segments, segment stride, row stride, entry stride (array of
 * 5 nrows).  The output arrays may be NULL. */
int rs_sweep_schedule(int32_t nrows, const int32_t *ptr, const int32_t *col, int32_t lower, int32_t run_cap,
                      int64_t run_slots, int32_t *nseg, int32_t *nlevels, int32_t *nrun, int32_t *seg_row0,
                      int32_t *seg_level, int32_t *runs);
int rs_precond_destroy(rs_pc **M);

/* ---- Krylov solvers (Sec. 3, Alg. 1) ----------------------------------- */
/* x holds the initial guess on entry and the solution on exit.  Converged
 * means ||b - A x||_2 <= rtol ||b||_2 for the recomputed FP64 residual.
 * maxit counts inner iterations.  M may be NULL (no preconditioner).
 * Right preconditioning throughout; orthogonalisation by classical
 * Gram-Schmidt with one reorthogonalisation pass (CGS2).  1 <= restart <= 64.
 * Returns RS_OK, RS_NOT_CONVERGED (info filled, x = last iterate) or an
 * error; info->status repeats the return value. */
int rs_solve_gmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart,
                   double rtol, int32_t maxit, rs_solve_info *info);
/* Flexible GMRES: keeps z_i = M^{-1} v_i, so M may change between steps
 * (the learned pressure stage). */
int rs_solve_fgmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart,
                    double rtol, int32_t maxit, rs_solve_info *info);
/* LGMRES(restart, aug_k): flexible GMRES whose cycle space is extended by
 * the normalised corrections x_new - x_old of the last aug_k cycles, newest
 * first (the `aug_k` of the paper's solver settings, Sec. 3; Baker, Jessup
 * and Manteuffel 2005).  A cycle takes `restart` preconditioned Arnoldi
 * steps plus one step per stored correction; an iteration is one Arnoldi
 * step.  aug_k = 0 is FGMRES.  1 <= restart, 0 <= aug_k,
 * restart + aug_k <= 64. */
int rs_solve_lgmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart, int32_t aug_k,
                    double rtol, int32_t maxit, rs_solve_info *info);
/* BiCGSTAB (named in Sec. 3; used in Examples 2, 4, 5). */
int rs_solve_bicgstab(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, double rtol,
                      int32_t maxit, rs_solve_info *info);
/* Preconditioned conjugate gradient (Alg. 2) for symmetric positive
 * definite A and M (e.g. the pressure matrix with ILU(0), whose factors are
 * then L D L^T).  One iteration is one pass of Alg. 2's loop; the stopping
 * test on the recursive residual is confirmed on the true residual, from
 * which the method restarts if it has drifted.  (p, A p) <= 0 or (r, z) = 0
 * returns RS_ERR_BREAKDOWN. */
int rs_solve_cg(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, double rtol, int32_t maxit,
                rs_solve_info *info);

/* ---- learned pressure stage ------------------------------------------- */
/* A 3-D U-Net (4 levels, 16 channels, 3x3x3 convolutions, ReLU, 2x2x2
 * average pooling, nearest x2 upsampling with skip concatenation, 1x1x1
 * head) with bfloat16 weights and activations and FP32 accumulation; not in
 * the paper, it replaces the pressure stage of the CPR preconditioner
 * (RS_PC_CPR_LEARNED).  Input channels: r / rms(r) and log-permeability;
 * output: net * rms(r) * out_scale, an approximation of A^{-1} r.
 * Parameters (FP32, host) are laid out layer by layer (e0a, e0b, e1a, e1b,
 * e2a, e2b, e3a, e3b, d2a, d2b, d1a, d1b, d0a, d0b): weights
 * [dz][dy][dx][cout][cin] then bias [cout]; then the head's 16 weights and
 * its bias.  Grid dimensions must be multiples of 8. */
int64_t rs_net_num_params(void);
int rs_net_create(rs_ctx *ctx, const float *params, int64_t nparams, float out_scale, rs_net **net);
int rs_net_destroy(rs_net **net);
int rs_net_get_params(const rs_net *net, float *params_host, int64_t n);
int rs_net_get_grads(const rs_net *net, float *grads_host, int64_t n);
int rs_net_zero_grads(rs_net *net);
/* out = network(r, logk) on an nx x ny x nz grid (device pointers, FP64,
 * x fastest). */
int rs_net_forward(rs_net *net, int32_t nx, int32_t ny, int32_t nz, const double *r, const double *logk,
                   double *out);
/* One training sample: forward, loss ||out - e||^2 / ||e||^2, backward;
 * adds weight * dloss/dparams to the gradient; *loss_host (optional,
 * synchronises) receives the loss. */
int rs_net_accumulate(rs_net *net, int32_t nx, int32_t ny, int32_t nz, const double *r, const double *logk,
                      const double *e, double weight, double *loss_host);
/* Adam step on the accumulated gradient, which it then clears. */
int rs_net_adam(rs_net *net, float lr, float beta1, float beta2, float eps);
/* Checkpoint: parameters, Adam moments, step count and output scale. */
int rs_net_save(const rs_net *net, const char *path);
int rs_net_load(rs_ctx *ctx, const char *path, rs_net **net);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
