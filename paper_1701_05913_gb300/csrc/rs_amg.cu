// Algebraic multigrid preconditioner (Sec. 4.2: Alg. 3 setup, Alg. 4
// V-cycle, Eq. 4).
//
// Setup (once per matrix, on the GPU: rs_amg_setup.cu), level by level in
// Alg. 3's order: classical strength (theta = 0.5 by default, Fig. 34), PMIS
// coarsening, direct interpolation, R = P^T, A_{l+1} = R A_l P (Eq. 4), the
// l1-Jacobi smoother's diagonal d_i = sum_j |a_ij|.  Levels stop at
// max_coarse rows, max_levels, or when coarsening stalls; the coarsest
// matrix is inverted densely.
//
// Apply (on the GPU): one V-cycle from x = 0 (Alg. 4): nu sweeps, residual,
// restriction, the next level, prolongation and correction, nu sweeps;
// the coarsest level is one dense matrix-vector product.  Every operator is
// an rs_mat, so the products run in the library's SpMV kernels; a smoothing
// sweep is one SpMV whose epilogue forms x + (b - A x) / d into a second
// buffer.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rs_internal.cuh"

// The smoother multiplies by dinv = 1/d, formed once at setup: a divide on
// every sweep would cost this GPU's FP64 pipe about ten times as much.
// first sweep from x = 0:  x_i = b_i / d_i
__global__ void k_amg_first(int n, const double *__restrict__ b, const double *__restrict__ dinv,
                            double *__restrict__ x, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = b[i] * dinv[i];
}

__global__ void k_amg_copy(int n, const double *__restrict__ a, double *__restrict__ x, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = a[i];
}

// One hybrid Gauss-Seidel sweep (Fig. 34's relaxation): a warp per chunk of
// 32 consecutive rows.  Each lane subtracts from b_i the terms its row takes
// from xold (null: zero), i.e. columns outside the chunk (Jacobi between
// chunks) and those of the chunk that the sweep reaches later, keeps its
// couplings to the chunk's earlier rows in registers (up to RS_HGS_REG; a
// row with more rescans the rest) and inverts its diagonal.  A chunk whose
// rows couple only to their predecessor is solved by a warp scan; otherwise
// the lanes finish in sweep order (increasing rows, BACKWARD: decreasing),
// each from the new values before it, kept in shared memory.
#define RS_HGS_WARPS 8
#define RS_HGS_REG 8
template <bool BACKWARD>
__global__ void __launch_bounds__(32 * RS_HGS_WARPS)
k_amg_hgs(int n, const int *__restrict__ ptr, const int *__restrict__ col, const double *__restrict__ val,
          const double *__restrict__ b, const double *__restrict__ xold, double *__restrict__ xnew, const int *skip)
{
    __shared__ double xs[RS_HGS_WARPS][32];
    if (skip && *(volatile const int *)skip) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nchunk = (n + 31) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunk; c += (gridDim.x * blockDim.x) >> 5) {
        const int c0 = c << 5, c1 = min(c0 + 32, n), i = c0 + lane;
        const bool active = i < c1;
        double s = 0.0, d = 1.0;
        int ej[RS_HGS_REG];
        double ev[RS_HGS_REG];
        int ne = 0;
        bool over = false;
#pragma unroll
        for (int q = 0; q < RS_HGS_REG; ++q) {
            ej[q] = 0;
            ev[q] = 0.0;
        }
        const int p0 = active ? ptr[i] : 0, p1 = active ? ptr[i + 1] : 0;
        if (active) {
            s = b[i];
            for (int p = p0; p < p1; ++p) {
                const int j = col[p];
                const double v = val[p];
                if (j == i) {
                    d = v;
                } else if (j >= c0 && j < c1 && (BACKWARD ? j > i : j < i)) {
                    if (ne < RS_HGS_REG) {
#pragma unroll
                        for (int q = 0; q < RS_HGS_REG; ++q)
                            if (q == ne) {
                                ej[q] = j - c0;
                                ev[q] = v;
                            }
                        ++ne;
                    } else {
                        over = true;
                    }
                } else if (xold) {
                    s = fma(-v, xold[j], s);
                }
            }
        }
        const double rd = 1.0 / d;
        // a chunk whose rows couple at most to the row before them in sweep
        // order (a grid line in natural order) is a first-order recurrence
        // x_i = c_i + m_i x_{i-/+1}: five steps of a warp scan of affine maps
        const bool chain_lane = !over && (ne == 0 || (ne == 1 && ej[0] == (BACKWARD ? lane + 1 : lane - 1)));
        if (__all_sync(0xffffffffu, chain_lane)) {
            double m = ne == 1 ? -ev[0] * rd : 0.0, cc = s * rd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double mp = BACKWARD ? __shfl_down_sync(0xffffffffu, m, o) : __shfl_up_sync(0xffffffffu, m, o);
                const double cp = BACKWARD ? __shfl_down_sync(0xffffffffu, cc, o) : __shfl_up_sync(0xffffffffu, cc, o);
                if (BACKWARD ? lane + o < 32 : lane >= o) {
                    cc = fma(m, cp, cc);
                    m *= mp;
                }
            }
            if (active) xnew[i] = cc;
            continue;
        }
        for (int t = 0; t < 32; ++t) {
            const int k = BACKWARD ? 31 - t : t;
            if (lane == k && active) {
#pragma unroll
                for (int q = 0; q < RS_HGS_REG; ++q)
                    if (q < ne) s = fma(-ev[q], xs[w][ej[q]], s);
                if (over) {   // couplings past the first RS_HGS_REG, in row order
                    int seen = 0;
                    for (int p = p0; p < p1; ++p) {
                        const int j = col[p];
                        if (j >= c0 && j < c1 && (BACKWARD ? j > i : j < i) && seen++ >= RS_HGS_REG)
                            s = fma(-val[p], xs[w][j - c0], s);
                    }
                }
                xs[w][lane] = s * rd;
            }
            __syncwarp();
        }
        if (active) xnew[i] = xs[w][lane];
        __syncwarp();
    }
}

// coarsest level: x = Ainv b, one warp per row
__global__ void k_amg_dense(int n, const double *__restrict__ inv, const double *__restrict__ b,
                            double *__restrict__ x, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s = fma(inv[(size_t)i * n + j], b[j], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = s;
    }
}

static int amg_grid(rs_ctx *ctx, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

void rs_amg_destroy(AmgData *M)
{
    if (!M) return;
    rs_ctx *ctx = M->ctx;
    for (int l = 0; l < RS_AMG_MAXLEV; ++l) {           // also the levels of a setup that failed
        if (l > 0 || M->own0) rs_mat_destroy(&M->A[l]);   // level 0 may be the caller's matrix
        rs_mat_destroy(&M->P[l]);
        rs_mat_destroy(&M->R[l]);
        rs_free(ctx, M->d[l]);
        rs_free(ctx, M->b[l]);
        rs_free(ctx, M->x[l]);
        rs_free(ctx, M->t[l]);
        rs_free(ctx, M->y[l]);
    }
    rs_free(ctx, M->cinv);
    for (int l = 0; l < RS_AMG_MAXLEV; ++l) rs_free(ctx, M->cidx[l]);
    for (const AmgGraph &g : M->graphs) cudaGraphExecDestroy(g.exec);
    if (M->capture) cudaStreamDestroy(M->capture);
    delete M;
}

int rs_amg_create(rs_ctx *ctx, int n, const int *d_ptr, const int *d_col, const double *d_val, const rs_mat *A0,
                  double theta, int max_levels, int max_coarse, int nu, int smoother, AmgData **out)
{
    *out = nullptr;
    if (n < 1 || max_levels < 1 || max_levels > RS_AMG_MAXLEV || max_coarse < 1 || nu < 1 || !(theta >= 0.0) ||
        smoother < 0 || smoother > 1)
        return RS_ERR_INVALID_ARG;
    AmgData *M = new AmgData();
    M->ctx = ctx;
    M->nu = nu;
    M->smoother = smoother;
    int st = RS_OK;
    if (A0) {
        M->A[0] = const_cast<rs_mat *>(A0);
    } else {
        M->own0 = true;
        st = rs_mat_create_rect_dev(ctx, n, -1, d_ptr, d_col, d_val, &M->A[0]);
    }
    // the hierarchy (Alg. 3), smoother diagonals and the coarsest inverse
    if (!st) st = rs_amg_setup_device(M, theta, max_levels, max_coarse);
    // work vectors
    for (int l = 0; l < M->nlev && !st; ++l) {
        const int nl = M->A[l]->n;
        st = rs_alloc(ctx, (void **)&M->b[l], sizeof(double) * nl);
        if (!st) st = rs_alloc(ctx, (void **)&M->x[l], sizeof(double) * nl);
        if (!st) st = rs_alloc(ctx, (void **)&M->t[l], sizeof(double) * nl);
        if (!st && l > 0) st = rs_alloc(ctx, (void **)&M->y[l], sizeof(double) * nl);
    }
    if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = RS_ERR_CUDA;
    if (st) {
        rs_amg_destroy(M);
        return st;
    }
    *out = M;
    return RS_OK;
}

// one V-cycle on level l: x_l = B_l b_l (Alg. 4 from x = 0)
static int vcycle(AmgData *M, int l, const double *b, double *x, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    const rs_mat *A = M->A[l];
    const int n = A->n;
    if (l == M->nlev - 1) {
        RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
        k_amg_dense<<<std::max(1, std::min((n + 7) / 8, ctx->num_sms * 4)), 256, 0, ctx->stream>>>(n, M->cinv, b, x,
                                                                                                  skip);
        return rs_check_launch(ctx);
    }
    const int g = amg_grid(ctx, n);
    const int nu = M->nu;
    double *t = M->t[l];
    // sweeps alternate between x and a second buffer; the first sweep (from
    // x = 0) is placed so that the last pre-smoothing sweep lands in x
    double *X = x, *Y = l == 0 ? M->x[0] : M->y[l];
    double *cur = (nu - 1) % 2 == 0 ? X : Y, *oth = cur == X ? Y : X;
    const int gh = std::max(1, std::min((n + 32 * RS_HGS_WARPS - 1) / (32 * RS_HGS_WARPS), ctx->num_sms * 16));
    if (M->smoother == 1) {
        {
            RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
            k_amg_hgs<false><<<gh, 32 * RS_HGS_WARPS, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, b, nullptr, cur, skip);
        }
        RS_TRY(rs_check_launch(ctx));
        for (int s = 1; s < nu; ++s) {
            {
                RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
                k_amg_hgs<false><<<gh, 32 * RS_HGS_WARPS, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, b, cur, oth, skip);
            }
            RS_TRY(rs_check_launch(ctx));
            std::swap(cur, oth);
        }
    } else {
        {
            RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
            k_amg_first<<<g, 256, 0, ctx->stream>>>(n, b, M->d[l], cur, skip);
        }
        RS_TRY(rs_check_launch(ctx));
        for (int s = 1; s < nu; ++s) {
            RS_TRY(rs_jacobi_launch(A, b, cur, M->d[l], oth, skip));
            std::swap(cur, oth);
        }
    }
    RS_TRY(rs_residual_launch(A, b, X, t, nullptr, skip));
    RS_TRY(rs_spmv_launch(M->R[l], t, 1.0, 0.0, M->b[l + 1], skip));
    RS_TRY(vcycle(M, l + 1, M->b[l + 1], M->x[l + 1], skip));
    RS_TRY(rs_spmv_launch(M->P[l], M->x[l + 1], 1.0, 1.0, X, skip));
    cur = X;
    oth = Y;
    for (int s = 0; s < nu; ++s) {
        if (M->smoother == 1) {   // backward sweeps: the adjoint of the forward ones
            {
                RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
                k_amg_hgs<true><<<gh, 32 * RS_HGS_WARPS, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, b, cur, oth, skip);
            }
            RS_TRY(rs_check_launch(ctx));
        } else {
            RS_TRY(rs_jacobi_launch(A, b, cur, M->d[l], oth, skip));
        }
        std::swap(cur, oth);
    }
    if (cur != X) {       // an odd number of post-smoothing sweeps
        {
            RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
            k_amg_copy<<<g, 256, 0, ctx->stream>>>(n, cur, X, skip);
        }
        RS_TRY(rs_check_launch(ctx));
    }
    return RS_OK;
}

// A V-cycle is some 60 small launches on its coarse levels; after the first
// apply, each (r, z, skip) address triple is captured once into a CUDA
// graph and replayed.  Capture runs on a private stream (the caller's may be
// the legacy default stream, which cannot be captured); replays go to the
// caller's stream.  With the profiler on, or if a capture fails, the
// V-cycle is launched kernel by kernel.
int rs_amg_apply(AmgData *M, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (ctx->prof_on || M->nograph || cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return vcycle(M, 0, r, z, skip);
    for (size_t i = 0; i < M->graphs.size(); ++i) {
        const AmgGraph &g = M->graphs[i];
        if (g.r != r || g.z != z || g.skip != skip) continue;
        if (g.limit == ctx->spin_limit) {
            if (cudaGraphLaunch(g.exec, ctx->stream) != cudaSuccess) return RS_ERR_CUDA;
            ctx->launches += g.nlaunch;
            return RS_OK;
        }
        // captured with another device-wait limit (rs_set_spin_limit since)
        cudaGraphExecDestroy(g.exec);
        M->graphs.erase(M->graphs.begin() + i);
        break;
    }
    if (M->applies++ == 0 || (int)M->graphs.size() >= RS_AMG_MAX_GRAPHS) return vcycle(M, 0, r, z, skip);
    if (!M->capture && cudaStreamCreateWithFlags(&M->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        M->nograph = true;
        return vcycle(M, 0, r, z, skip);
    }
    const long long l0 = ctx->launches;
    cudaStream_t user = ctx->stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int st = RS_ERR_CUDA;
    if (cudaStreamBeginCapture(M->capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        ctx->stream = M->capture;
        st = vcycle(M, 0, r, z, skip);
        ctx->stream = user;
        const cudaError_t e = cudaStreamEndCapture(M->capture, &graph);
        if (e != cudaSuccess) st = RS_ERR_CUDA;
    }
    if (!st && (!graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)) st = RS_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (st) {
        cudaGetLastError();
        M->nograph = true;
        ctx->launches = l0;
        return vcycle(M, 0, r, z, skip);
    }
    M->graphs.push_back({r, z, skip, ctx->spin_limit, exec, ctx->launches - l0});
    // the capture has counted the graph's launches once; this is their run
    return cudaGraphLaunch(exec, user) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

int rs_amg_level_sizes(const AmgData *M, int l, int32_t *n, int64_t *nnz_a, int64_t *nnz_p)
{
    if (l < 0 || l >= M->nlev) return RS_ERR_INVALID_ARG;
    *n = M->A[l]->n;
    *nnz_a = M->A[l]->nnzb;
    *nnz_p = l + 1 < M->nlev ? M->P[l]->nnzb : 0;
    return RS_OK;
}

int rs_amg_get_level(const AmgData *M, int l, int32_t *aptr, int32_t *acol, double *aval, int32_t *pptr,
                     int32_t *pcol, double *pval, int32_t *cidx)
{
    if (l < 0 || l >= M->nlev) return RS_ERR_INVALID_ARG;
    rs_ctx *ctx = M->ctx;
    const cudaStream_t s = ctx->stream;
    auto get = [&](void *dst, const void *src, size_t bytes) -> int {
        if (!dst || !bytes) return RS_OK;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
    };
    const rs_mat *A = M->A[l];
    RS_TRY(get(aptr, A->ptr, sizeof(int) * (A->n + 1)));
    RS_TRY(get(acol, A->col, sizeof(int) * A->nnzb));
    RS_TRY(get(aval, A->val, sizeof(double) * A->nnzb));
    if (l + 1 < M->nlev) {
        const rs_mat *P = M->P[l];
        RS_TRY(get(pptr, P->ptr, sizeof(int) * (P->n + 1)));
        RS_TRY(get(pcol, P->col, sizeof(int) * P->nnzb));
        RS_TRY(get(pval, P->val, sizeof(double) * P->nnzb));
        RS_TRY(get(cidx, M->cidx[l], sizeof(int) * A->n));
    }
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    return RS_OK;
}

