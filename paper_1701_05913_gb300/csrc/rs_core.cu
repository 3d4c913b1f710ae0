// Context, vectors, matrices, BLAS-1 and SpMV kernels.
//
// Vectors: Sec. 2.2 (VEC, Figs. 6-13).  Matrices and products: Sec. 2.3
// (MAT, Figs. 15-21).  One process owns the whole matrix, so the halo
// exchange of MatVecMXY and the all-reduce of VecDot have no counterpart:
// dot products are deterministic two-level tree reductions on the device.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;
void rs_set_last_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

int rs_count_launch(rs_ctx *ctx)
{
    ctx->launches++;
    return RS_OK;
}

int rs_check_launch(rs_ctx *ctx)
{
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        rs_set_last_cuda_error(e);
        return RS_ERR_CUDA;
    }
    return RS_OK;
}

int rs_alloc(rs_ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        rs_set_last_cuda_error(e);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA;
    }
    return RS_OK;
}

void rs_free(rs_ctx *ctx, void *p)
{
    if (p) cudaFreeAsync(p, ctx->stream);
}

extern "C" const char *rs_status_str(int s)
{
    switch (s) {
    case RS_OK: return "ok";
    case RS_NOT_CONVERGED: return "not converged within maxit";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_BAD_PATTERN: return "bad sparsity pattern (unsorted, missing diagonal or out of range)";
    case RS_ERR_ZERO_PIVOT: return "zero or non-finite pivot";
    case RS_ERR_BREAKDOWN: return "Krylov breakdown";
    case RS_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case RS_ERR_CUDA: return cudaGetErrorString(g_last_cuda_error);
    case RS_ERR_OOM: return "out of device memory";
    case RS_ERR_SIZE_MISMATCH: return "size mismatch";
    default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int rs_init(rs_ctx **out, int device, void *stream)
{
    if (!out) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    RS_CUDA_TRY(cudaSetDevice(device));
    rs_ctx *c = new rs_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->red_blocks = 2 * c->num_sms;
    c->launches = 0;
    c->prof_on = 0;
    for (int k = 0; k < RS_PROF_NKINDS; ++k) { c->prof_ms[k] = 0.0; c->prof_count[k] = 0; }
    int clock_khz = 2000000;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
    c->spin_limit = (long long)clock_khz * 1000LL * 2;   // about two seconds
    c->sweep_blocks = 4 * c->num_sms;
    c->sleep_cap_ns = 0;   // spin: a polling warp reissues its loads as soon as they return
    // the stream-ordered pool keeps freed blocks for reuse
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    int st = RS_OK;
    st = st ? st : rs_alloc(c, (void **)&c->red_partials,
                            sizeof(double) * (size_t)c->red_blocks * (RS_MAX_RESTART + 8));
    st = st ? st : rs_alloc(c, (void **)&c->red_ticket, sizeof(unsigned) * 8);
    st = st ? st : rs_alloc(c, (void **)&c->d_scalars, sizeof(double) * 64);
    st = st ? st : rs_alloc(c, (void **)&c->d_err, sizeof(int) * 2);
    if (st) { delete c; return st; }
    c->d_bad_row = c->d_err + 1;
    cudaMemsetAsync(c->red_ticket, 0, sizeof(unsigned) * 8, c->stream);
    cudaMemsetAsync(c->d_scalars, 0, sizeof(double) * 64, c->stream);
    int init[2] = {0, 0x7fffffff};
    cudaMemcpyAsync(c->d_err, init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
    if (cudaMallocHost((void **)&c->h_pinned, sizeof(double) * 64) != cudaSuccess) {
        delete c;
        return RS_ERR_OOM;
    }
    RS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = c;
    return RS_OK;
}

static void ctx_free(rs_ctx *c)
{
    cudaStreamSynchronize(c->stream);
    rs_free(c, c->red_partials);
    rs_free(c, c->red_ticket);
    rs_free(c, c->d_scalars);
    rs_free(c, c->d_err);
    cudaStreamSynchronize(c->stream);
    cudaFreeHost(c->h_pinned);
    for (const RsProfRec &r : c->prof_pending) { cudaEventDestroy(r.ev0); cudaEventDestroy(r.ev1); }
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    delete c;
}

void rs_ctx_retain(rs_ctx *c) { ++c->live; }

void rs_ctx_release(rs_ctx *c)
{
    if (--c->live == 0 && c->closing) ctx_free(c);
}

extern "C" int rs_finalize(rs_ctx **pc)
{
    if (!pc || !*pc) return RS_OK;
    rs_ctx *c = *pc;
    *pc = nullptr;
    if (c->live > 0) {
        c->closing = true;      // released with the last handle
        cudaStreamSynchronize(c->stream);
        return RS_OK;
    }
    ctx_free(c);
    return RS_OK;
}

extern "C" int rs_set_history(rs_ctx *ctx, double *hist, int32_t len)
{
    if (!ctx || len < 0) return RS_ERR_INVALID_ARG;
    ctx->hist_host = len > 0 ? hist : nullptr;
    ctx->hist_len = hist ? len : 0;
    return RS_OK;
}

extern "C" int rs_set_spin_limit(rs_ctx *ctx, int64_t cycles)
{
    if (!ctx || cycles < 0) return RS_ERR_INVALID_ARG;
    if (cycles > 0) {
        ctx->spin_limit = cycles;
    } else {
        int clock_khz = 2000000;
        cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, ctx->device);
        ctx->spin_limit = (long long)clock_khz * 1000LL * 2;
    }
    return RS_OK;
}

extern "C" int rs_check_device(rs_ctx *ctx)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    return rs_collect_device_error(ctx, nullptr);
}

extern "C" int rs_sync(rs_ctx *ctx)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return RS_OK;
}

extern "C" int64_t rs_launch_count(const rs_ctx *ctx) { return ctx ? ctx->launches : -1; }

// ---------------------------------------------------------------------------
// event profiler
// ---------------------------------------------------------------------------
static cudaEvent_t prof_event(rs_ctx *c)
{
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

RsProfScope::RsProfScope(rs_ctx *c, int k) : ctx(c), kind(k), ev1(nullptr)
{
    if (!ctx || !ctx->prof_on) return;
    RsProfRec r;
    r.kind = kind;
    r.ev0 = prof_event(ctx);
    r.ev1 = prof_event(ctx);
    cudaEventRecord(r.ev0, ctx->stream);
    ev1 = r.ev1;
    ctx->prof_pending.push_back(r);
}

RsProfScope::~RsProfScope()
{
    if (ev1) cudaEventRecord(ev1, ctx->stream);
}

static void prof_resolve(rs_ctx *c)
{
    if (c->prof_pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (const RsProfRec &r : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev0, r.ev1) == cudaSuccess) {
            c->prof_ms[r.kind] += ms;
            c->prof_count[r.kind] += 1;
        }
        c->prof_pool.push_back(r.ev0);
        c->prof_pool.push_back(r.ev1);
    }
    c->prof_pending.clear();
}

extern "C" int rs_prof_enable(rs_ctx *ctx, int on)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    prof_resolve(ctx);
    ctx->prof_on = on ? 1 : 0;
    return RS_OK;
}

extern "C" int rs_prof_read(rs_ctx *ctx, double *ms, int64_t *launches, int32_t nkinds, int reset)
{
    if (!ctx || !ms || !launches || nkinds < RS_PROF_NKINDS) return RS_ERR_INVALID_ARG;
    prof_resolve(ctx);
    for (int k = 0; k < RS_PROF_NKINDS; ++k) {
        ms[k] = ctx->prof_ms[k];
        launches[k] = ctx->prof_count[k];
        if (reset) {
            ctx->prof_ms[k] = 0.0;
            ctx->prof_count[k] = 0;
        }
    }
    return RS_OK;
}

int rs_collect_device_error(rs_ctx *ctx, int *bad_row)
{
    int h[2];
    RS_CUDA_TRY(cudaMemcpyAsync(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (h[0] == 0) return RS_OK;
    int init[2] = {0, 0x7fffffff};
    RS_CUDA_TRY(cudaMemcpyAsync(ctx->d_err, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (bad_row) *bad_row = h[1] == 0x7fffffff ? -1 : h[1];
    if (h[0] & RS_DEVERR_TIMEOUT) return RS_ERR_DEVICE_TIMEOUT;
    if (h[0] & RS_DEVERR_PIVOT) return RS_ERR_ZERO_PIVOT;
    return RS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// BLAS-1 kernels (Figs. 10-13)
// ---------------------------------------------------------------------------
static int blas_grid(rs_ctx *ctx, int n)
{
    int g = (n + 255) / 256;
    int cap = ctx->num_sms * 8;
    return std::max(1, std::min(g, cap));
}

__global__ void k_set(int n, double a, double *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = a;
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, double *y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);
}

__global__ void k_axpbyz(int n, double a, const double *__restrict__ x, double b,
                         const double *__restrict__ y, double *__restrict__ z)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        z[i] = fma(a, x[i], b * y[i]);
}

// Two-level deterministic dot product: fixed grid, per-block partial sums,
// the last block to finish adds the partials in block order.
__global__ void __launch_bounds__(RS_RED_THREADS)
k_dot(int n, const double *__restrict__ x, const double *__restrict__ y, double *partials,
      unsigned *ticket, double *out, int sqrt_out)
{
    __shared__ double sm[RS_RED_THREADS / 32];
    __shared__ bool last;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        a0 += x[i] * y[i];
        a1 += x[i + stride] * y[i + stride];
        a2 += x[i + 2 * stride] * y[i + 2 * stride];
        a3 += x[i + 3 * stride] * y[i + 3 * stride];
    }
    for (; i < n; i += stride) a0 += x[i] * y[i];
    double a = warp_sum((a0 + a1) + (a2 + a3));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < RS_RED_THREADS / 32; ++w) s += sm[w];
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        double s = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(partials + b);
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            *out = sqrt_out ? sqrt(s) : s;
            *ticket = 0;
        }
    }
}

int rs_axpby_launch(rs_ctx *ctx, int n, double a, const double *x, double b, double *y)
{
    if (n <= 0) return RS_OK;
    RsProfScope prof(ctx, RS_PROF_BLAS1);
    k_axpby<<<blas_grid(ctx, n), 256, 0, ctx->stream>>>(n, a, x, b, y);
    return rs_check_launch(ctx);
}

int rs_dot_launch(rs_ctx *ctx, int n, const double *x, const double *y, double *out_dev)
{
    if (n <= 0) {
        RS_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(double), ctx->stream));
        return RS_OK;
    }
    RsProfScope prof(ctx, RS_PROF_BLAS1);
    k_dot<<<ctx->red_blocks, RS_RED_THREADS, 0, ctx->stream>>>(n, x, y, ctx->red_partials,
                                                               ctx->red_ticket, out_dev, 0);
    return rs_check_launch(ctx);
}

// ---------------------------------------------------------------------------
// vectors
// ---------------------------------------------------------------------------
extern "C" int rs_vec_create(rs_ctx *ctx, int32_t n, rs_vec **v)
{
    if (!ctx || !v || n < 0) return RS_ERR_INVALID_ARG;
    rs_vec *x = new rs_vec();
    x->ctx = ctx;
    x->n = n;
    x->owns = 1;
    int st = rs_alloc(ctx, (void **)&x->d, sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (st) { delete x; return st; }
    cudaMemsetAsync(x->d, 0, sizeof(double) * (size_t)n, ctx->stream);
    rs_ctx_retain(ctx);
    *v = x;
    return RS_OK;
}

extern "C" int rs_vec_wrap(rs_ctx *ctx, int32_t n, double *dev, rs_vec **v)
{
    if (!ctx || !v || n < 0 || (!dev && n > 0)) return RS_ERR_INVALID_ARG;
    rs_vec *x = new rs_vec();
    x->ctx = ctx;
    x->n = n;
    x->d = dev;
    x->owns = 0;
    rs_ctx_retain(ctx);
    *v = x;
    return RS_OK;
}

extern "C" int rs_vec_destroy(rs_vec **v)
{
    if (!v || !*v) return RS_OK;
    rs_ctx *ctx = (*v)->ctx;
    if ((*v)->owns) rs_free(ctx, (*v)->d);
    delete *v;
    *v = nullptr;
    rs_ctx_release(ctx);
    return RS_OK;
}

extern "C" int32_t rs_vec_size(const rs_vec *v) { return v ? v->n : -1; }
extern "C" double *rs_vec_data(rs_vec *v) { return v ? v->d : nullptr; }

extern "C" int rs_vec_set(rs_vec *v, const double *src, int mem)
{
    if (!v || (!src && v->n > 0)) return RS_ERR_INVALID_ARG;
    if (v->n == 0) return RS_OK;
    RS_CUDA_TRY(cudaMemcpyAsync(v->d, src, sizeof(double) * (size_t)v->n,
                                mem == RS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                v->ctx->stream));
    if (mem == RS_MEM_HOST) RS_CUDA_TRY(cudaStreamSynchronize(v->ctx->stream));
    return RS_OK;
}

extern "C" int rs_vec_get(const rs_vec *v, double *dst, int mem)
{
    if (!v || (!dst && v->n > 0)) return RS_ERR_INVALID_ARG;
    if (v->n == 0) return RS_OK;
    RS_CUDA_TRY(cudaMemcpyAsync(dst, v->d, sizeof(double) * (size_t)v->n,
                                mem == RS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                v->ctx->stream));
    if (mem == RS_MEM_HOST) RS_CUDA_TRY(cudaStreamSynchronize(v->ctx->stream));
    return RS_OK;
}

extern "C" int rs_vec_set_value(rs_vec *x, double a)
{
    if (!x) return RS_ERR_INVALID_ARG;
    if (x->n == 0) return RS_OK;
    k_set<<<blas_grid(x->ctx, x->n), 256, 0, x->ctx->stream>>>(x->n, a, x->d);
    return rs_check_launch(x->ctx);
}

extern "C" int rs_vec_axpby(double a, const rs_vec *x, double b, rs_vec *y)
{
    if (!x || !y) return RS_ERR_INVALID_ARG;
    if (x->n != y->n) return RS_ERR_SIZE_MISMATCH;
    return rs_axpby_launch(y->ctx, y->n, a, x->d, b, y->d);
}

extern "C" int rs_vec_axpbyz(double a, const rs_vec *x, double b, const rs_vec *y, rs_vec *z)
{
    if (!x || !y || !z) return RS_ERR_INVALID_ARG;
    if (x->n != y->n || x->n != z->n) return RS_ERR_SIZE_MISMATCH;
    if (z->n == 0) return RS_OK;
    k_axpbyz<<<blas_grid(z->ctx, z->n), 256, 0, z->ctx->stream>>>(z->n, a, x->d, b, y->d, z->d);
    return rs_check_launch(z->ctx);
}

static int dot_to_host(rs_ctx *ctx, int n, const double *x, const double *y, int sq, double *out)
{
    if (n == 0) { *out = 0.0; return RS_OK; }
    k_dot<<<ctx->red_blocks, RS_RED_THREADS, 0, ctx->stream>>>(n, x, y, ctx->red_partials,
                                                               ctx->red_ticket, ctx->d_scalars, sq);
    RS_TRY(rs_check_launch(ctx));
    RS_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalars, sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = ctx->h_pinned[0];
    return RS_OK;
}

extern "C" int rs_vec_dot(const rs_vec *x, const rs_vec *y, double *out)
{
    if (!x || !y || !out) return RS_ERR_INVALID_ARG;
    if (x->n != y->n) return RS_ERR_SIZE_MISMATCH;
    return dot_to_host(x->ctx, x->n, x->d, y->d, 0, out);
}

extern "C" int rs_vec_norm2(const rs_vec *x, double *out)
{
    if (!x || !out) return RS_ERR_INVALID_ARG;
    return dot_to_host(x->ctx, x->n, x->d, x->d, 1, out);
}

// ---------------------------------------------------------------------------
// SpMV kernels (Figs. 20-21)
// ---------------------------------------------------------------------------
// CSR: L lanes per row; each lane strides over the row's nonzeros, the group
// adds its lanes with shuffles.  mode 0: y = alpha*Ax + beta*y;
// mode 1: y = b - Ax (residual, b passed in `bvec`).
// CSR, medium and long rows: L lanes per row, each lane taking 4 entries
// per round with all their loads issued before the multiply-adds, so that a
// row of up to 4 L entries needs one round of memory latency.
template <int L>
__global__ void __launch_bounds__(256)
k_spmv_csr(int n, const int *__restrict__ ptr, const int *__restrict__ col,
           const double *__restrict__ val, const double *__restrict__ x, double alpha, double beta,
           const double *__restrict__ bvec, double *__restrict__ y, const int *skip,
           const double *__restrict__ dinv)
{
    if (skip && *(volatile const int *)skip) return;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gid / L;
    const int lane = gid % L;
    const bool active = row < n;
    double acc = 0.0;
    if (active) {
        const int s = ptr[row], e = ptr[row + 1];
        for (int p0 = s + lane; p0 < e; p0 += 4 * L) {
            int c[4];
            double v[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * L;
                c[u] = p < e ? col[p] : -1;
                v[u] = p < e ? val[p] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) acc = fma(v[u], xv[u], acc);
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
    if (active && lane == 0) {
        if (dinv) y[row] = fma(__dsub_rn(bvec[row], acc), dinv[row], x[row]);   // Jacobi-type sweep
        else if (bvec) y[row] = __dsub_rn(bvec[row], acc);
        else if (beta == 0.0) y[row] = alpha == 1.0 ? acc : __dmul_rn(alpha, acc);
        else y[row] = fma(alpha, acc, beta * y[row]);
    }
}

// CSR, short rows: persistent and pipelined.  A block owns every G-th tile
// of RS_SPMV_TILE consecutive rows.  One producer thread copies a tile's row
// pointers, values and column indices into a ring of RS_SPMV_S shared-memory
// stages with bulk copies (ranges widened to 16-byte boundaries; the
// library's copies of the arrays carry a few padding elements so the widened
// ranges stay inside them), RS_SPMV_S - 1 tiles ahead of the consumers; each
// consumer thread forms one row of a tile: gathers of x (the first 8 entries
// at once), sum in column order, epilogue y = alpha A x (+ beta y) or
// y = b - A x.  Three blocks fit on an SM.  A tile holding more than
// RS_SPMV_TNNZ nonzeros is read straight from global memory.
#define RS_MAT_PAD 8
#define RS_SPMV_TILE 256
#define RS_SPMV_TNNZ 1984
#define RS_SPMV_S 3
#define RS_SPMV_THREADS (RS_SPMV_TILE + 32)
struct SpmvStage {
    double val[RS_SPMV_TNNZ + 8];   // first: 16-byte aligned
    int col[RS_SPMV_TNNZ + 8];
    int ptr[RS_SPMV_TILE + 8];
};
static_assert(sizeof(SpmvStage) % 16 == 0, "stages stay 16-byte aligned");
#define RS_SPMV_SMEM (RS_SPMV_S * sizeof(SpmvStage))

__global__ void __launch_bounds__(RS_SPMV_THREADS)
k_spmv_csr_pipe(int n, const int *__restrict__ ptr, const int *__restrict__ col, const double *__restrict__ val,
                const double *__restrict__ x, double alpha, double beta, const double *__restrict__ bvec,
                double *__restrict__ y, const int *skip, int *err, long long limit,
                const double *__restrict__ dinv)
{
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ __align__(128) unsigned char spmv_smem[];
    SpmvStage *stg = (SpmvStage *)spmv_smem;
    __shared__ unsigned long long full[RS_SPMV_S], empty[RS_SPMV_S];
    __shared__ int meta[RS_SPMV_S][4];   // first copied index of ptr, val, col; direct flag
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < RS_SPMV_S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], RS_SPMV_TILE / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ntiles = (n + RS_SPMV_TILE - 1) / RS_SPMV_TILE;
    if (warp == RS_SPMV_TILE / 32) {
        if (lane != 0) return;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % RS_SPMV_S;
            if (it >= RS_SPMV_S) mbar_wait(&empty[s], (unsigned)((it / RS_SPMV_S - 1) & 1), limit, err);
            const int r0 = tile * RS_SPMV_TILE, r1 = min(r0 + RS_SPMV_TILE, n);
            const int p0 = ptr[r0], p1 = ptr[r1];
            const int pa = r0 & ~3, pcnt = (r1 + 1 - pa + 3) & ~3;
            const int direct = p1 - p0 > RS_SPMV_TNNZ;
            const int va = p0 & ~1, vcnt = (p1 - va + 1) & ~1;
            const int ca = p0 & ~3, ccnt = (p1 - ca + 3) & ~3;
            meta[s][0] = pa;
            meta[s][1] = va;
            meta[s][2] = ca;
            meta[s][3] = direct;
            const unsigned bytes = (unsigned)pcnt * 4u + (direct ? 0u : (unsigned)vcnt * 8u + (unsigned)ccnt * 4u);
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s(stg[s].ptr, ptr + pa, (unsigned)pcnt * 4u, &full[s]);
            if (!direct && vcnt > 0) bulk_g2s(stg[s].val, val + va, (unsigned)vcnt * 8u, &full[s]);
            if (!direct && ccnt > 0) bulk_g2s(stg[s].col, col + ca, (unsigned)ccnt * 4u, &full[s]);
        }
        return;
    }
    // consumers: the gathers of x for tile k+1 are issued before the sums of
    // tile k, so each warp keeps two tiles of gathers in flight
    struct Row {
        int a, b;          // entry range of the row (global indices)
        double xv[8];      // x at its first 8 entries
    };
    auto gather = [&](int it, int tile, Row &R) {
        const int s = it % RS_SPMV_S;
        mbar_wait(&full[s], (unsigned)((it / RS_SPMV_S) & 1), limit, err);
        const SpmvStage &st = stg[s];
        const int r = tile * RS_SPMV_TILE + threadIdx.x;
        R.a = R.b = 0;
        if (r < n) {
            const int pa = meta[s][0], ca = meta[s][2], direct = meta[s][3];
            R.a = st.ptr[r - pa];
            R.b = st.ptr[r + 1 - pa];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                R.xv[q] = R.a + q < R.b ? __ldg(x + (direct ? col[R.a + q] : st.col[R.a + q - ca])) : 0.0;
        }
    };
    auto finish = [&](int it, int tile, const Row &R) {
        const int s = it % RS_SPMV_S;
        const SpmvStage &st = stg[s];
        const int r = tile * RS_SPMV_TILE + threadIdx.x;
        if (r < n) {
            const int va = meta[s][1], ca = meta[s][2], direct = meta[s][3];
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (R.a + q < R.b) acc = fma(direct ? val[R.a + q] : st.val[R.a + q - va], R.xv[q], acc);
            for (int p = R.a + 8; p < R.b; ++p)   // rows longer than 8
                acc = fma(direct ? val[p] : st.val[p - va], __ldg(x + (direct ? col[p] : st.col[p - ca])), acc);
            if (dinv) y[r] = fma(__dsub_rn(bvec[r], acc), dinv[r], x[r]);   // Jacobi-type sweep
            else if (bvec) y[r] = __dsub_rn(bvec[r], acc);
            else if (beta == 0.0) y[r] = alpha == 1.0 ? acc : __dmul_rn(alpha, acc);
            else y[r] = fma(alpha, acc, beta * y[r]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    };
    Row R0, R1;
    int it = 0, tile = blockIdx.x;
    if (tile < ntiles) gather(0, tile, R0);
    while (tile < ntiles) {
        const int t1 = tile + gridDim.x;
        if (t1 < ntiles) gather(it + 1, t1, R1);
        finish(it, tile, R0);
        tile = t1;
        ++it;
        if (tile >= ntiles) break;
        const int t2 = tile + gridDim.x;
        if (t2 < ntiles) gather(it + 1, t2, R0);
        finish(it, tile, R1);
        tile = t2;
        ++it;
    }
}

// BSR: one thread per scalar row (block row I, component r).
template <int BS>
__global__ void __launch_bounds__(256)
k_spmv_bsr(int nb, int bsr, const int *__restrict__ ptr, const int *__restrict__ col,
           const double *__restrict__ val, const double *__restrict__ x, double alpha, double beta,
           const double *__restrict__ bvec, double *__restrict__ y, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    const int bs = BS > 0 ? BS : bsr;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb * bs) return;
    const int I = (int)(t / bs), r = (int)(t % bs);
    double acc = 0.0;
    for (int p = ptr[I]; p < ptr[I + 1]; ++p) {
        const double *blk = val + (size_t)p * bs * bs + (size_t)r * bs;
        const double *xs = x + (size_t)col[p] * bs;
        if (BS > 0) {
#pragma unroll
            for (int c = 0; c < (BS > 0 ? BS : 1); ++c) acc = fma(blk[c], __ldg(xs + c), acc);
        } else {
            for (int c = 0; c < bs; ++c) acc = fma(blk[c], __ldg(xs + c), acc);
        }
    }
    if (bvec) y[t] = __dsub_rn(bvec[t], acc);
    else if (beta == 0.0) y[t] = alpha == 1.0 ? acc : __dmul_rn(alpha, acc);
    else y[t] = fma(alpha, acc, beta * y[t]);
}

// y = alpha A x + beta y, y = b - A x (bvec), or with dinv the sweep
// y = x + (b - A x) dinv (y must not alias x)
static int spmv_dispatch(const rs_mat *A, const double *x, double alpha, double beta,
                         const double *bvec, double *y, const int *skip, const double *dinv = nullptr)
{
    rs_ctx *ctx = A->ctx;
    if (A->n == 0) return RS_OK;
    RsProfScope prof(ctx, RS_PROF_SPMV);
    if (A->bs == 1 && A->lanes == 1) {
        static unsigned long long raised = 0;   // devices whose shared-memory limit was raised
        const unsigned long long bit = 1ull << (ctx->device & 63);
        if (!(raised & bit)) {
            RS_CUDA_TRY(cudaFuncSetAttribute(k_spmv_csr_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RS_SPMV_SMEM));
            raised |= bit;
        }
        const int tiles = (A->n + RS_SPMV_TILE - 1) / RS_SPMV_TILE;
        const int grid = std::max(1, std::min(tiles, 3 * ctx->num_sms));
        k_spmv_csr_pipe<<<grid, RS_SPMV_THREADS, RS_SPMV_SMEM, ctx->stream>>>(
            A->n, A->ptr, A->col, A->val, x, alpha, beta, bvec, y, skip, ctx->d_err, ctx->spin_limit, dinv);
    } else if (A->bs == 1) {
        const int L = A->lanes;
        const int64_t threads = (int64_t)A->n * L;
        const int grid = (int)((threads + 255) / 256);
        switch (L) {
#define RS_SPMV_CASE(LL)                                                                    \
    case LL:                                                                                \
        k_spmv_csr<LL><<<grid, 256, 0, ctx->stream>>>(A->n, A->ptr, A->col, A->val, x, alpha, \
                                                      beta, bvec, y, skip, dinv);           \
        break;
            RS_SPMV_CASE(1)
            RS_SPMV_CASE(2)
            RS_SPMV_CASE(4)
            RS_SPMV_CASE(8)
            RS_SPMV_CASE(16)
            RS_SPMV_CASE(32)
#undef RS_SPMV_CASE
        default: return RS_ERR_INVALID_ARG;
        }
    } else {
        const int64_t threads = (int64_t)A->nrows * A->bs;
        const int grid = (int)((threads + 255) / 256);
        if (A->bs == 3)
            k_spmv_bsr<3><<<grid, 256, 0, ctx->stream>>>(A->nrows, 3, A->ptr, A->col, A->val, x,
                                                         alpha, beta, bvec, y, skip);
        else if (A->bs == 2)
            k_spmv_bsr<2><<<grid, 256, 0, ctx->stream>>>(A->nrows, 2, A->ptr, A->col, A->val, x,
                                                         alpha, beta, bvec, y, skip);
        else
            k_spmv_bsr<0><<<grid, 256, 0, ctx->stream>>>(A->nrows, A->bs, A->ptr, A->col, A->val,
                                                         x, alpha, beta, bvec, y, skip);
    }
    return rs_check_launch(ctx);
}

int rs_spmv_launch(const rs_mat *A, const double *x, double alpha, double beta, double *y,
                   const int *skip)
{
    return spmv_dispatch(A, x, alpha, beta, nullptr, y, skip);
}

int rs_jacobi_launch(const rs_mat *A, const double *b, const double *x, const double *dinv, double *xnew,
                     const int *skip)
{
    if (A->bs != 1) return RS_ERR_INVALID_ARG;
    return spmv_dispatch(A, x, 1.0, 0.0, b, xnew, skip, dinv);
}

int rs_residual_launch(const rs_mat *A, const double *b, const double *x, double *r,
                       double *norm2_out, const int *skip)
{
    RS_TRY(spmv_dispatch(A, x, -1.0, 0.0, b, r, skip));
    if (norm2_out) RS_TRY(rs_dot_launch(A->ctx, A->n, r, r, norm2_out));
    return RS_OK;
}

// ---------------------------------------------------------------------------
// matrices
// ---------------------------------------------------------------------------
static int validate_pattern(int nrows, int ncols, const std::vector<int> &ptr,
                            const std::vector<int> &col, bool need_diag = true)
{
    if ((int)ptr.size() != nrows + 1 || ptr[0] != 0) return RS_ERR_BAD_PATTERN;
    for (int i = 0; i < nrows; ++i) {
        if (ptr[i + 1] < ptr[i]) return RS_ERR_BAD_PATTERN;
        bool diag = false;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int c = col[p];
            if (c < 0 || c >= ncols) return RS_ERR_BAD_PATTERN;
            if (p > ptr[i] && col[p - 1] >= c) return RS_ERR_BAD_PATTERN;
            if (c == i) diag = true;
        }
        if (!diag && need_diag) return RS_ERR_BAD_PATTERN;
    }
    if ((size_t)ptr[nrows] != col.size()) return RS_ERR_BAD_PATTERN;
    return RS_OK;
}

static int mat_create(rs_ctx *ctx, int nrows, int bs, const int32_t *ptr, const int32_t *col,
                      const double *val, int mem, rs_mat **out, int ncols = -1)
{
    if (!ctx || !out || nrows < 0 || bs < 1 || bs > 8 || !ptr) return RS_ERR_INVALID_ARG;
    if ((int64_t)nrows * bs > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    const cudaMemcpyKind h2d = mem == RS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind d2h = mem == RS_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    rs_mat *A = new rs_mat();
    A->ctx = ctx;
    A->bs = bs;
    A->nrows = nrows;
    A->n = nrows * bs;
    A->h_ptr.resize(nrows + 1);
    RS_CUDA_TRY(cudaMemcpyAsync(A->h_ptr.data(), ptr, sizeof(int) * (nrows + 1), d2h, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    const int64_t nnzb = A->h_ptr[nrows];
    if (nnzb < 0 || (!col && nnzb > 0) || (!val && nnzb > 0) ||
        nnzb * bs * bs > 0x7fffffffLL) {
        delete A;
        return RS_ERR_INVALID_ARG;
    }
    A->nnzb = nnzb;
    A->h_col.resize(nnzb);
    if (nnzb) {
        RS_CUDA_TRY(cudaMemcpyAsync(A->h_col.data(), col, sizeof(int) * nnzb, d2h, ctx->stream));
        RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    // square matrices need every diagonal entry; rectangular operators
    // (interpolation, restriction) only sorted, in-range columns
    int st = validate_pattern(nrows, ncols < 0 ? nrows : ncols, A->h_ptr, A->h_col, ncols < 0);
    if (st) { delete A; return st; }
    // RS_MAT_PAD zeroed elements after each array: the SpMV's bulk copies
    // widen their ranges to 16-byte boundaries
    st = rs_alloc(ctx, (void **)&A->ptr, sizeof(int) * (nrows + 1 + RS_MAT_PAD));
    st = st ? st : rs_alloc(ctx, (void **)&A->col, sizeof(int) * (nnzb + RS_MAT_PAD));
    st = st ? st : rs_alloc(ctx, (void **)&A->val, sizeof(double) * (nnzb * bs * bs + RS_MAT_PAD));
    if (st) { rs_free(ctx, A->ptr); rs_free(ctx, A->col); delete A; return st; }
    RS_CUDA_TRY(cudaMemsetAsync(A->ptr + nrows + 1, 0, sizeof(int) * RS_MAT_PAD, ctx->stream));
    RS_CUDA_TRY(cudaMemsetAsync(A->col + nnzb, 0, sizeof(int) * RS_MAT_PAD, ctx->stream));
    RS_CUDA_TRY(cudaMemsetAsync(A->val + nnzb * bs * bs, 0, sizeof(double) * RS_MAT_PAD, ctx->stream));
    RS_CUDA_TRY(cudaMemcpyAsync(A->ptr, ptr, sizeof(int) * (nrows + 1), h2d, ctx->stream));
    if (nnzb) {
        RS_CUDA_TRY(cudaMemcpyAsync(A->col, col, sizeof(int) * nnzb, h2d, ctx->stream));
        RS_CUDA_TRY(cudaMemcpyAsync(A->val, val, sizeof(double) * nnzb * bs * bs, h2d, ctx->stream));
    }
    if (mem == RS_MEM_HOST) RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    // rows of at most 12 entries on average go to the pipelined row-per-thread
    // kernel (lanes = 1); longer ones to the lane kernel with the smallest
    // power of two L for which 4 L entries cover the mean row
    const double mean = nrows ? (double)nnzb / nrows : 1.0;
    int L = 1;
    if (mean > 12.0)
        while (L < 32 && 4.0 * L < mean) L <<= 1;
    A->lanes = L;
    rs_ctx_retain(ctx);
    *out = A;
    return RS_OK;
}

extern "C" int rs_mat_create_csr(rs_ctx *ctx, int32_t n, const int32_t *rowptr,
                                 const int32_t *col, const double *val, int mem, rs_mat **A)
{
    return mat_create(ctx, n, 1, rowptr, col, val, mem, A);
}

int rs_mat_create_rect(rs_ctx *ctx, int nrows, int ncols, const int32_t *ptr, const int32_t *col,
                       const double *val, rs_mat **A)
{
    if (ncols < 0) return RS_ERR_INVALID_ARG;
    return mat_create(ctx, nrows, 1, ptr, col, val, RS_MEM_HOST, A, ncols);
}

// from device arrays (copied); ncols < 0: square, every diagonal entry present
int rs_mat_create_rect_dev(rs_ctx *ctx, int nrows, int ncols, const int32_t *ptr, const int32_t *col,
                           const double *val, rs_mat **A)
{
    return mat_create(ctx, nrows, 1, ptr, col, val, RS_MEM_DEVICE, A, ncols);
}

extern "C" int rs_mat_create_bsr(rs_ctx *ctx, int32_t nb, int32_t bs, const int32_t *browptr,
                                 const int32_t *bcol, const double *bval, int mem, rs_mat **A)
{
    return mat_create(ctx, nb, bs, browptr, bcol, bval, mem, A);
}

extern "C" int rs_mat_destroy(rs_mat **pA)
{
    if (!pA || !*pA) return RS_OK;
    rs_mat *A = *pA;
    rs_ctx *ctx = A->ctx;
    rs_free(ctx, A->ptr);
    rs_free(ctx, A->col);
    rs_free(ctx, A->val);
    delete A;
    *pA = nullptr;
    rs_ctx_release(ctx);
    return RS_OK;
}

extern "C" int32_t rs_mat_size(const rs_mat *A) { return A ? A->n : -1; }

extern "C" int rs_mat_spmv(const rs_mat *A, const rs_vec *x, rs_vec *y)
{
    if (!A || !x || !y) return RS_ERR_INVALID_ARG;
    if (x->n != A->n || y->n != A->n) return RS_ERR_SIZE_MISMATCH;
    if (x->d == y->d && A->n > 0) return RS_ERR_INVALID_ARG;
    return rs_spmv_launch(A, x->d, 1.0, 0.0, y->d, nullptr);
}

extern "C" int rs_mat_amxpby(double a, const rs_mat *A, const rs_vec *x, double b, rs_vec *y)
{
    if (!A || !x || !y) return RS_ERR_INVALID_ARG;
    if (x->n != A->n || y->n != A->n) return RS_ERR_SIZE_MISMATCH;
    if (x->d == y->d && A->n > 0) return RS_ERR_INVALID_ARG;
    return rs_spmv_launch(A, x->d, a, b, y->d, nullptr);
}
