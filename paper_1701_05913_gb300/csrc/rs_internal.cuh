// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rs.h"

#define RS_MAX_RESTART 64
#define RS_RED_THREADS 256

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
#define RS_CUDA_TRY(expr)                                                     \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) {                                              \
            rs_set_last_cuda_error(_e);                                       \
            return _e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA; \
        }                                                                     \
    } while (0)

#define RS_TRY(expr)                    \
    do {                                \
        int _s = (expr);                \
        if (_s != RS_OK) return _s;     \
    } while (0)

void rs_set_last_cuda_error(cudaError_t e);

// device error word bits
#define RS_DEVERR_TIMEOUT 1
#define RS_DEVERR_PIVOT 2

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
// kernel classes timed by the optional event profiler
enum RsProfKind {
    RS_PROF_SPMV = 0,
    RS_PROF_LSWEEP,
    RS_PROF_USWEEP,
    RS_PROF_CGS_DOTS,
    RS_PROF_CGS_UPDATE_DOTS,
    RS_PROF_CGS_UPDATE_NORM,
    RS_PROF_BLAS1,
    RS_PROF_PRECOND_OTHER,
    RS_PROF_FACTOR,
    RS_PROF_SOLVER_SCALAR,
    RS_PROF_NET,
    RS_PROF_BLSWEEP,
    RS_PROF_BUSWEEP,
    RS_PROF_CPR_RESID,
    RS_PROF_NKINDS
};

struct RsProfRec {
    int kind;
    cudaEvent_t ev0, ev1;
};

struct rs_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    int red_blocks;          // fixed grid of the reduction kernels
    double *red_partials;    // red_blocks * (RS_MAX_RESTART + 8) doubles
    unsigned *red_ticket;    // last-block ticket of the reduction kernels
    double *d_scalars;       // small device scalar area (64 doubles)
    int *d_err;              // device error word
    int *d_bad_row;          // smallest row with a bad pivot
    double *h_pinned;        // pinned host staging (64 doubles)
    long long launches;
    long long spin_limit;    // clock cycles a device-side wait may take
    int sweep_blocks;        // resident blocks of the persistent triangular sweeps (at least)
    unsigned sleep_cap_ns;   // longest back-off of a polling warp (0: none)
    // residual history of the solves (rs_set_history): caller's host array
    double *hist_host = nullptr;
    int hist_len = 0;
    // event profiler (off unless rs_prof_enable)
    int prof_on;
    std::vector<RsProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[RS_PROF_NKINDS];
    long long prof_count[RS_PROF_NKINDS];
    // handles (vectors, matrices, preconditioners, networks) alive on this
    // context: rs_finalize releases the context when the last one goes, so
    // handles and context may be destroyed in any order
    int live = 0;
    bool closing = false;
};

// Records an event pair around the launches in its scope when profiling is on.
struct RsProfScope {
    rs_ctx *ctx;
    int kind;
    cudaEvent_t ev1;
    RsProfScope(rs_ctx *c, int k);
    ~RsProfScope();
};

struct rs_mat {
    rs_ctx *ctx;
    int bs;                  // 1 = CSR
    int nrows;               // block rows
    int n;                   // scalar rows
    int64_t nnzb;            // stored blocks (scalars for CSR)
    int *ptr, *col;
    double *val;
    std::vector<int> h_ptr, h_col;   // host copy of the pattern (analysis)
    int lanes;               // SpMV lanes per row (CSR; 1 = the pipelined row-per-thread kernel)
};

struct rs_vec {
    rs_ctx *ctx;
    int n;
    double *d;
    int owns;
};

// state of one sync-free sweep: work ticket, finished-block count, epoch
struct SweepState {
    unsigned ticket;
    unsigned done;
    int epoch;
    int pad;
};

// Row-level schedule of the ILU(0) factorisation: rows in level order of the
// dependency graph of L, each level padded to a multiple of 32 positions.
struct TriLayout {
    int npad = 0;                // positions
    int nlevels = 0;
    int nwarps = 0;
    int *pos = nullptr;          // [npad] row at each position or -1
    int *warp_level = nullptr;   // [nwarps] level of each warp of positions
    int *level_nwarps = nullptr; // [nlevels] warps per level
    int *level_count = nullptr;  // [nlevels] arrival counters (self-resetting)
    int *level_done = nullptr;   // [nlevels] epoch of the sweep that last completed the level
};

// Segment layout of one triangular factor: segments of at most 32
// consecutive rows (one warp each), ordered by their level in the segment
// dependency graph, entries stored as sliced ELL per segment.
struct SegLayout {
    int nseg = 0;
    int nlevels = 0;
    int64_t nent = 0;
    int nrun = 0;                  // runs: segments one warp takes in turn
    int max_run = 0;               // segments of the longest run
    int *runs = nullptr;           // [nrun][5] first segment, count, segment / row / entry strides
    int *sptr = nullptr;           // [nseg+1] first entry of each segment (by id)
    int *col = nullptr;            // [nent] column or -1
    int *src = nullptr;            // [nent] index of the entry in the CSR value array or -1
    unsigned char *kind = nullptr; // [nseg] 1: the only in-segment dependency is the adjacent row
    int *row0 = nullptr;           // [nseg+1] first row of each segment
    void *val = nullptr;           // [bs*bs][nent] factor values (float or double); U: D_i U_ij
    void *rdiag = nullptr;         // [bs*bs][nseg*32] U: 1 / u_ii or inv(U_II) by row
    int *adjsrc = nullptr;         // [nrows] index of the in-segment adjacent entry or -1
    void *mul = nullptr;           // [nseg][5][bs*bs][32] multipliers of the scan steps
    int grid = 0;                  // sweep blocks: follows the segments per level
};

// ILU(0) / block ILU(0) of one matrix pattern.
// Wavefront sweeps (rs_wave.cu) of a factor whose pattern is the 7-point
// stencil of an nx x ny x nz grid.  A unit (one warp) is a tile of a y-lines
// x b z-planes (a b = 32) over all x; its cells are stored by step, 32 per
// step (one per lane), npad steps per unit, units in ticket order.
struct WaveLayout {
    int on = 0;
    int nx = 0, ny = 0, nz = 0;
    int la = 0;                           // log2 a: lanes along y (a), along z (b = 32 / a)
    int nyt = 0, nzt = 0, nunits = 0;     // tiles along y and z, and in all
    int npad = 0;                         // steps stored per unit (a multiple of the chunk)
    int64_t ncell = 0;                    // stored cells: nunits npad 32
    void *lrec = nullptr, *urec = nullptr;  // L and U records in wave order (apply precision)
    void *rw = nullptr;                   // right-hand side in wave order
    void *yw = nullptr, *zw = nullptr;    // values of the L and U sweeps (sentinel protocol)
};

struct IluFactor {
    rs_ctx *ctx = nullptr;
    int bs = 1;
    int nrows = 0;
    int64_t nnzb = 0;
    int fp32 = 0;            // apply precision
    int run_warps = 1;       // warps per block of the sweeps with runs
    const int *ptr = nullptr, *col = nullptr;  // pattern (device, borrowed)
    int *diagpos = nullptr;  // [nrows]
    double *lu = nullptr;    // [nnzb*bs*bs] FP64 factors in the matrix pattern
    double *dinv = nullptr;  // [nrows*bs*bs] inverted diagonal blocks (bs > 1)
    TriLayout L;             // row-level schedule of the factorisation
    SegLayout SL, SU;        // segment layouts of the sweeps (when W is off)
    WaveLayout W;            // wavefront layout (structured 7-point patterns)
    SweepState *state = nullptr;
    void *ywork = nullptr;   // [nrows*bs] intermediate of the L sweep
    void *zwork = nullptr;   // [nrows*bs] values of the U sweep
};

// Restricted additive Schwarz (rs_ras.cu): the extended subdomains stacked
// into one block-diagonal matrix with its ILU(level) factor.
#define RS_RAS_MAX_LEVEL 8
struct RasData {
    rs_ctx *ctx = nullptr;
    int bs = 1, nrows = 0;       // block size, block rows of A
    int next = 0;                // block rows of the stacked matrix
    int64_t nnz = 0;             // its stored blocks
    int nparts = 0, overlap = 0, level = 0;
    int *ptr = nullptr, *col = nullptr;   // stacked pattern (device)
    int *src = nullptr;          // [nnz] block of A behind each entry, -1 at fill
    int *gidx = nullptr;         // [next] global block row of each stacked row
    int *own = nullptr;          // [nrows] stacked row that owns each block row
    double *val = nullptr;       // [nnz*bs*bs] stacked values
    double *rhat = nullptr, *zhat = nullptr;   // [next*bs] work vectors
    std::vector<int> h_gidx;
    IluFactor *f = nullptr;
};

// Algebraic multigrid (rs_amg.cu): operators of every level as rs_mat,
// reciprocals of the l1-Jacobi diagonals (d), work vectors, dense inverse of
// the coarsest matrix.
#define RS_AMG_MAXLEV 16
#define RS_AMG_MAX_DENSE 4096
// one captured V-cycle: its input, output and skip flag addresses, the
// executable graph and the number of kernels it launches
struct AmgGraph {
    const double *r;
    double *z;
    const int *skip;
    long long limit;         // the spin limit its kernels were captured with
    cudaGraphExec_t exec;
    long long nlaunch;
};
#define RS_AMG_MAX_GRAPHS 64
struct AmgData {
    rs_ctx *ctx = nullptr;
    int nlev = 0, nu = 2;
    int smoother = 0;            // 0 l1-Jacobi, 1 hybrid Gauss-Seidel over 32-row chunks
    bool own0 = false;           // level-0 matrix built here (not the caller's)
    rs_mat *A[RS_AMG_MAXLEV] = {}, *P[RS_AMG_MAXLEV] = {}, *R[RS_AMG_MAXLEV] = {};
    double *d[RS_AMG_MAXLEV] = {}, *b[RS_AMG_MAXLEV] = {}, *x[RS_AMG_MAXLEV] = {}, *t[RS_AMG_MAXLEV] = {};
    double *y[RS_AMG_MAXLEV] = {};   // second smoothing buffer (level 0 uses x[0])
    double *cinv = nullptr;
    int *cidx[RS_AMG_MAXLEV] = {};   // coarse index of every point of level l (-1: F), device
    std::vector<AmgGraph> graphs;
    cudaStream_t capture = nullptr;   // private stream for stream capture
    long long applies = 0;
    bool nograph = false;        // a capture failed: launch directly from then on
};

struct rs_pc {
    rs_ctx *ctx;
    int type;
    int prec;
    const rs_mat *A;
    IluFactor *ilu;          // ILU0, or pressure stage of CPR
    IluFactor *bilu;         // BILU0, or second stage of CPR
    // CPR
    int *app_ptr_unused;
    double *app_val;         // decoupled pressure matrix values (block pattern)
    double *w;               // quasi-IMPES weights [nb*(bs-1)]
    int *diagA;              // diagonal block positions of A (CPR with a RAS F stage)
    double *rp, *zp;         // pressure-stage vectors [nb]
    double *t1, *t2;         // full-size work vectors [n]
    double *pcol;            // PF form on blocks: column 0 of every block of A [nnzb*bs]
    // learned pressure stage
    const rs_net *net;
    const double *log_perm;
    int nx, ny, nz;
    int bad_row;
    int form;                // rs_cpr_form: order of the CPR stages
    RasData *ras;            // RS_PC_RAS
    AmgData *amg;            // RS_PC_AMG, or the pressure stage of CPR
    // CUDA graphs of whole CPR applies, one per (r, z, skip) address triple;
    // gen is the network workspace's generation at capture
    struct Graph {
        const double *r;
        double *z;
        const int *skip;
        unsigned gen;
        long long limit;     // the spin limit its kernels were captured with
        cudaGraphExec_t exec;
        long long nlaunch;
    };
    std::vector<Graph> graphs;
    cudaStream_t capture;
    int applies;
    bool nograph;
};

// ---------------------------------------------------------------------------
// internal entry points shared across translation units
// ---------------------------------------------------------------------------
int rs_count_launch(rs_ctx *ctx);
void rs_ctx_retain(rs_ctx *ctx);
void rs_ctx_release(rs_ctx *ctx);
int rs_check_launch(rs_ctx *ctx);
int rs_alloc(rs_ctx *ctx, void **p, size_t bytes);
void rs_free(rs_ctx *ctx, void *p);

// an nrows x ncols CSR operator from host arrays (no diagonal required)
int rs_mat_create_rect_dev(rs_ctx *ctx, int nrows, int ncols, const int32_t *ptr, const int32_t *col,
                           const double *val, rs_mat **A);
int rs_mat_create_rect(rs_ctx *ctx, int nrows, int ncols, const int32_t *ptr, const int32_t *col,
                       const double *val, rs_mat **A);

// y = alpha * A x + beta * y (beta == 0: y not read).  Kernels given a
// non-null `skip` return at once when *skip != 0 (a device flag).
int rs_spmv_launch(const rs_mat *A, const double *x, double alpha, double beta, double *y,
                   const int *skip);
// one sweep xnew = x + (b - A x) dinv, fused into the SpMV (CSR; xnew must
// not alias x)
int rs_jacobi_launch(const rs_mat *A, const double *b, const double *x, const double *dinv, double *xnew,
                     const int *skip);
// r = b - A x and, if norm2_out != nullptr, *norm2_out (device) = ||r||^2
int rs_residual_launch(const rs_mat *A, const double *b, const double *x, double *r,
                       double *norm2_out, const int *skip);
// device-scalar BLAS-1
int rs_axpby_launch(rs_ctx *ctx, int n, double a, const double *x, double b, double *y);
int rs_dot_launch(rs_ctx *ctx, int n, const double *x, const double *y, double *out_dev);

// ILU
// sweep_mode: 0 the library's choice (the wavefront sweeps when the pattern
// is a structured 7-point grid, else segments), 1 the segment sweeps, 2 the
// wavefront sweeps when the pattern is a structured 7-point grid (else
// segments).  run_cap: the longest run of segments a warp carries (0: the
// default; scalar only).
int rs_ilu_create(rs_ctx *ctx, int bs, int nrows, int64_t nnzb, const int *d_ptr,
                  const int *d_col, const std::vector<int> &h_ptr,
                  const std::vector<int> &h_col, int fp32, int sweep_mode, int run_cap,
                  IluFactor **out, int *bad_row);
int rs_ilu_factor(IluFactor *f, const double *d_val, int *bad_row);
int rs_ilu_apply(IluFactor *f, const double *r, double *z, const double *scale_dev,
                 const int *skip);
void rs_ilu_destroy(IluFactor *f);
int rs_ilu_set_factors(IluFactor *f, const double *d_lu, int *bad_row);
// wavefront sweeps (rs_wave.cu)
bool rs_wave_detect(int n, const std::vector<int> &ptr, const std::vector<int> &col, int *nx, int *ny, int *nz);
int rs_wave_create(IluFactor *f, int nx, int ny, int nz);
int rs_wave_gather(IluFactor *f);
int rs_wave_apply(IluFactor *f, const double *r, double *z, const double *scale, const int *skip);
void rs_wave_free(IluFactor *f);
// local: 0 = ILU(level), 1 = ILUT(ilut_p, ilut_tol) (scalar matrices)
int rs_ras_create(rs_ctx *ctx, const rs_mat *A, int nparts, const int32_t *part, int overlap, int level, int local,
                  int ilut_p, double ilut_tol, int fp32, RasData **out, int *bad_row);
int rs_ras_apply(RasData *R, const double *r, double *z, const int *skip);
void rs_ras_destroy(RasData *R);
// A0: the level-0 matrix when the caller has one as an rs_mat (else built
// from the host pattern and the device values d_val)
int rs_amg_create(rs_ctx *ctx, int n, const int *d_ptr, const int *d_col, const double *d_val, const rs_mat *A0,
                  double theta, int max_levels, int max_coarse, int nu, int smoother, AmgData **out);
// the hierarchy of Alg. 3 on the device (rs_amg_setup.cu): from M->A[0]
int rs_amg_setup_device(AmgData *M, double theta, int max_levels, int max_coarse);
int rs_amg_apply(AmgData *M, const double *r, double *z, const int *skip);
void rs_amg_destroy(AmgData *M);
int rs_amg_level_sizes(const AmgData *M, int l, int32_t *n, int64_t *nnz_a, int64_t *nnz_p);
int rs_amg_get_level(const AmgData *M, int l, int32_t *aptr, int32_t *acol, double *aval, int32_t *pptr,
                     int32_t *pcol, double *pval, int32_t *cidx);

// CPR / learned pressure stage
int rs_pc_apply_dev(rs_pc *M, const double *r, double *z, const int *skip);
int rs_net_apply_pressure(rs_pc *M, const double *rp, double *zp, const int *skip);
// the learned stage's workspace for M's grid, allocated if needed; gen
// changes whenever the workspace is reallocated; same_ctx: the network runs
// on M's context (and stream)
int rs_net_prepare(rs_pc *M, unsigned *gen, bool *same_ctx);

// reads back and clears the device error word; maps it to a status
int rs_collect_device_error(rs_ctx *ctx, int *bad_row);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Waits until flag >= epoch (wrap-safe) or the clock budget runs out.
// Returns false on timeout.
__device__ __forceinline__ bool wait_epoch(const int *flag, int epoch, long long limit)
{
    int v = ld_acquire(flag);
    if (v - epoch >= 0) return true;
    const long long t0 = clock64();
    unsigned ns = 8;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_acquire(flag);
        if (v - epoch >= 0) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// ---------------------------------------------------------------------------
// triangular sweeps: the value is its own ready flag (shared by the segment
// sweeps of rs_ilu.cu and the wavefront sweeps of rs_wave.cu)
// ---------------------------------------------------------------------------
// Before a sweep every entry of its work vector holds a signalling-NaN bit
// pattern that arithmetic never produces; a warp polls the entries it depends
// on until they change, and publishes each value with one plain 8-byte (or
// 4-byte) store, which is single-copy atomic.
template <typename T> struct Sentinel;
template <> struct Sentinel<double> {
    typedef unsigned long long bits_t;
    static constexpr bits_t bits = 0xFFF5A5A5A5A5A5A5ull;
};
template <> struct Sentinel<float> {
    typedef unsigned int bits_t;
    static constexpr bits_t bits = 0xFFB5A5A5u;
};

__device__ __forceinline__ unsigned long long ld_relaxed_bits(const double *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_relaxed_bits(const float *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(double *p, double v)
{
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ double bits_to(double, unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ float bits_to(float, unsigned int b) { return __uint_as_float(b); }

template <typename T>
__global__ void k_fill_sentinel(int64_t n, T *v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = bits_to(T(), Sentinel<T>::bits);
}

// Arithmetic of the sweeps.  FP64 uses fused multiply-adds (FP64
// instructions are scarce on this GPU and sit on the critical path); FP32
// (the mixed-precision apply) rounds the product and the difference
// separately, in ascending column order.
__device__ __forceinline__ double msub(double acc, double a, double b) { return fma(-a, b, acc); }
__device__ __forceinline__ float msub(float acc, float a, float b) { return __fsub_rn(acc, __fmul_rn(a, b)); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (TMA, 1-D) helpers shared by the streaming kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity to complete; gives up after `limit`
// clock cycles, setting the timeout bit of the device error word.
__device__ __forceinline__ void mbar_wait(unsigned long long *b, unsigned parity, long long limit, int *err)
{
    if (mbar_try_wait(b, parity)) return;
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity)) {
        if (clock64() - t0 > limit) {
            atomicOr(err, RS_DEVERR_TIMEOUT);
            return;
        }
    }
}
// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}


#endif
