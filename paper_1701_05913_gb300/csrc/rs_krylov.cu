// Krylov solvers: restarted GMRES(m) (Sec. 3, Alg. 1), flexible GMRES and
// BiCGSTAB (named in Sec. 3), right-preconditioned, FP64.
//
// Device-resident design: the Hessenberg matrix, the Givens rotations, the
// rotated residual and every BiCGSTAB scalar live in device memory and are
// updated by the last block of the reduction that produces them, so a whole
// GMRES cycle (or a batch of BiCGSTAB iterations) is enqueued without waiting
// for the host.  Once a cycle has converged, a device flag makes every later
// kernel of the cycle return at once.  The host reads the state back twice
// per GMRES cycle and once per batch of BiCGSTAB iterations.
//
// Orthogonalisation is classical Gram-Schmidt with one full
// reorthogonalisation pass (CGS2) instead of the modified Gram-Schmidt loop
// printed in Alg. 1: the 2(i+1) dot products of step i become three fused
// passes over the basis V (dots; update + dots; update + norm), each a
// tall-skinny product computed row-wise with per-block partial sums.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "rs_internal.cuh"

#define RS_PSTRIDE (RS_MAX_RESTART + 8)   // partials per block in ctx->red_partials

struct GmresDev {
    double H[(RS_MAX_RESTART + 1) * RS_MAX_RESTART];   // column-major, ld = m+1
    double cs[RS_MAX_RESTART], sn[RS_MAX_RESTART];
    double g[RS_MAX_RESTART + 1], y[RS_MAX_RESTART + 1];
    double h1[RS_MAX_RESTART + 2], h2[RS_MAX_RESTART + 2];
    double bnorm, tol, beta, hdiv, w0sq, implicit, r2;
    int iters, k, cycle_done, converged, maxit, m, noupd, status;
    double augn2;           // ||Z y||^2 of the last cycle (LGMRES)
    double *hist;           // residual history (device), hist_len entries
    int hist_len, pad_;
};

// The solver's relative residual estimate after iteration it (from 1) into
// the history, when one is recorded.
__device__ __forceinline__ void record_hist(double *hist, int hist_len, int it, double res, double bnorm)
{
    if (hist && it >= 1 && it - 1 < hist_len) hist[it - 1] = res / bnorm;
}

// A device array for the residual history of one solve, when the context
// records one (rs_set_history); null otherwise.
static int hist_begin(rs_ctx *ctx, double **dh, int *len)
{
    *dh = nullptr;
    *len = ctx->hist_host ? ctx->hist_len : 0;
    if (*len == 0) return RS_OK;
    return rs_alloc(ctx, (void **)dh, sizeof(double) * (size_t)*len);
}

// Copies the first min(len, iters) entries back to the caller's array and
// frees the device array.
static int hist_end(rs_ctx *ctx, double *dh, int len, int iters)
{
    int st = RS_OK;
    const int k = std::min(len, iters);
    if (dh && k > 0) {
        if (cudaMemcpyAsync(ctx->hist_host, dh, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            st = RS_ERR_CUDA;
    }
    rs_free(ctx, dh);
    return st;
}

// ---------------------------------------------------------------------------
// block reduction of up to NC+1 per-thread sums with a last-block finish
// ---------------------------------------------------------------------------
template <int NV, int NW = RS_RED_THREADS / 32>
__device__ __forceinline__ bool reduce_partials(double (&acc)[NV], int nv, double *partials,
                                                unsigned *ticket, double *out)
{
    __shared__ double sm[NW][NV];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k < nv) {
            const double v = warp_sum(acc[k]);
            if (lane == 0) sm[warp][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += sm[w][k];
        partials[(size_t)blockIdx.x * RS_PSTRIDE + k] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int k = warp; k < nv; k += NW) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partials + (size_t)b * RS_PSTRIDE + k);
        s = warp_sum(s);
        if (lane == 0) out[k] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
    __syncthreads();
    return true;
}

// Warp reduce-scatter of NC per-lane values (NC a power of two): after
// log2(NC) exchange-and-add steps lane l holds complete sums of columns
// [l*NC/32, (l+1)*NC/32) (NC >= 32) or of column l/(32/NC) (NC < 32), for
// about NC FP64 additions per lane instead of 5 per column.  Each step is a
// template instance, so every index is a compile-time constant and the
// values stay in registers.
template <int NC, int W, int M>
struct ReduceScatter {
    static __device__ __forceinline__ void run(double (&v)[NC], int lane)
    {
        if constexpr (M >= 1) {
            if constexpr (W > 1) {
                // split: keep one half of the live values, send the other to lane ^ M
                const bool up = lane & M;
#pragma unroll
                for (int j = 0; j < W / 2; ++j) {
                    const double send = up ? v[j] : v[j + W / 2];
                    const double keep = up ? v[j + W / 2] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, M);
                }
                ReduceScatter<NC, W / 2, M / 2>::run(v, lane);
            } else {
                v[0] += __shfl_xor_sync(0xffffffffu, v[0], M);
                ReduceScatter<NC, 1, M / 2>::run(v, lane);
            }
        }
    }
};

template <int NC>
__device__ __forceinline__ void warp_reduce_scatter(double (&v)[NC], int lane)
{
    ReduceScatter<NC, NC, 16>::run(v, lane);
}

// Block reduction of NC per-thread column sums (and one extra scalar) with a
// last-block finish: out[k] for k < nc, out[nc] = the extra scalar's sum.
template <int NC, int NW = RS_RED_THREADS / 32>
__device__ __forceinline__ bool reduce_columns(double (&acc)[NC], double extra, bool has_extra, int nc,
                                               double *partials, unsigned *ticket, double *out)
{
    __shared__ double sm[NW][NC + 1];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    warp_reduce_scatter<NC>(acc, lane);
    if (NC >= 32) {
#pragma unroll
        for (int j = 0; j < NC / 32; ++j) sm[warp][lane * (NC / 32) + j] = acc[j];
    } else {
        constexpr int G = NC < 32 ? 32 / NC : 1;   // lanes sharing one column
        if (lane % G == 0) sm[warp][lane / G] = acc[0];
    }
    if (has_extra) {
        const double e = warp_sum(extra);
        if (lane == 0) sm[warp][NC] = e;
    }
    __syncthreads();
    const int nv = nc + (has_extra ? 1 : 0);
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const int src = k < nc ? k : NC;
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += sm[w][src];
        partials[(size_t)blockIdx.x * RS_PSTRIDE + k] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int k = warp; k < nv; k += NW) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(partials + (size_t)b * RS_PSTRIDE + k);
        t = warp_sum(t);
        if (lane == 0) out[k] = t;
    }
    if (threadIdx.x == 0) *ticket = 0;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// CGS2 passes for Arnoldi step i (nc = i+1 basis vectors, w in V[:, i+1])
// ---------------------------------------------------------------------------
// The passes are FP64-bound (one to two multiply-adds per 8 bytes read, on a
// GPU with about two FP64 lanes per clock per SM), so the loads are taken off
// the FP64 warps: one producer thread streams tiles of TILE rows of the nc
// basis vectors and of w into a shared-memory ring of 3 to 8 stages with bulk copies
// (completion counted by an mbarrier per stage), and the consumer warps,
// one row per thread, run only shared-memory loads and multiply-adds.
//   pass 1 (CGS_DOTS):        h1 = V^T w, and ||w||^2 for the breakdown test
//   pass 2 (CGS_UPDATE_DOTS): w -= V h1; h2 = V^T w; H[:, i] = h1 + h2
//   pass 3 (CGS_UPDATE_NORM): w -= V h2; h_{i+1,i} = ||w||; Givens update
// A block's consumer thread adds its rows in tile order and the block sums go
// through the fixed last-block reduction, so the results are deterministic.
enum { CGS_DOTS = 0, CGS_UPDATE_DOTS = 1, CGS_UPDATE_NORM = 2 };

template <int NC>
struct CgsCfg {
    static constexpr int CW = NC <= 32 ? 4 : 2;        // consumer warps
    static constexpr int NW = CW + 1;                   // + the producer warp
    static constexpr int THREADS = 32 * NW;
    static constexpr int TILE = 32 * CW;                // rows per tile, one per consumer thread
    static constexpr int STAGE = (NC + 1) * TILE;       // doubles per stage: NC columns, then w
    // stages: about 100 KB of ring per block (two blocks per SM), so that a
    // narrow basis still keeps enough bytes in flight to feed the FP64 pipe
    static constexpr int S = 100 * 1024 / (STAGE * 8) < 3 ? 3 : (100 * 1024 / (STAGE * 8) > 8 ? 8 : 100 * 1024 / (STAGE * 8));
    static constexpr size_t SMEM = (size_t)S * STAGE * sizeof(double) + 2 * S * sizeof(unsigned long long);
};

// NC: columns of the ring and of the reduction (a power of two); NCC: the
// unrolled bound of the multiply-add loops (nc rounded down to 4); the last
// nc - NCC (0 to 3) columns take a warp-uniform branch, so that no FP64
// multiply-add is issued for a column that does not exist (predicated-off
// FP64 instructions still occupy the FP64 pipe on this GPU).
template <int NC, int NCC, int MODE>
__global__ void __launch_bounds__(CgsCfg<NC>::THREADS)
k_cgs_pass(int n, int ld, int nc, const double *__restrict__ V, double *w, double *partials, unsigned *ticket,
           GmresDev *d, int *err, long long limit)
{
    typedef CgsCfg<NC> C;
    if (*(volatile int *)&d->cycle_done) return;
    extern __shared__ __align__(128) unsigned char cgs_smem[];
    double *ring = (double *)cgs_smem;
    unsigned long long *full = (unsigned long long *)(ring + C::S * C::STAGE);
    unsigned long long *empty = full + C::S;
    __shared__ double hs[NC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (MODE != CGS_DOTS)
        for (int k = threadIdx.x; k < nc; k += blockDim.x) hs[k] = MODE == CGS_UPDATE_DOTS ? d->h1[k] : d->h2[k];
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C::CW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ntiles = (n + C::TILE - 1) / C::TILE;
    double acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.0;
    double extra = 0.0;
    if (warp == C::CW) {
        if (lane == 0) {
            // producer: whole tiles, the last one rounded up to an even row
            // count (inside the column padding: ld is a multiple of 32)
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int s = it % C::S;
                if (it >= C::S) mbar_wait(&empty[s], (unsigned)((it / C::S - 1) & 1), limit, err);
                const int r0 = tile * C::TILE;
                const int rows = min(C::TILE, n - r0);
                const unsigned bytes = (unsigned)((rows + 1) & ~1) * 8u;
                double *st = ring + s * C::STAGE;
                mbar_arrive_expect_tx(&full[s], bytes * (unsigned)(nc + 1));
                for (int k = 0; k < nc; ++k) bulk_g2s(st + k * C::TILE, V + (size_t)k * ld + r0, bytes, &full[s]);
                bulk_g2s(st + NC * C::TILE, w + r0, bytes, &full[s]);
            }
        }
    } else {
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % C::S;
            mbar_wait(&full[s], (unsigned)((it / C::S) & 1), limit, err);
            const double *st = ring + s * C::STAGE + threadIdx.x;
            const int r = tile * C::TILE + threadIdx.x;
            if (r < n) {
                const double wr = st[NC * C::TILE];
                const int rem = nc - NCC;   // 0..3, the same for the whole grid
                if (MODE == CGS_DOTS) {
#pragma unroll
                    for (int k = 0; k < NCC; ++k) acc[k] = fma(st[k * C::TILE], wr, acc[k]);
#pragma unroll
                    for (int k = NCC; k < NCC + 3 && k < NC; ++k)
                        if (k - NCC < rem) acc[k] = fma(st[k * C::TILE], wr, acc[k]);
                    extra = fma(wr, wr, extra);
                } else {
                    double s0 = 0.0, s1 = 0.0;
#pragma unroll
                    for (int k = 0; k < NCC; ++k) {
                        if (k & 1) s1 = fma(st[k * C::TILE], hs[k], s1);
                        else s0 = fma(st[k * C::TILE], hs[k], s0);
                    }
#pragma unroll
                    for (int k = NCC; k < NCC + 3 && k < NC; ++k) {
                        if (k - NCC < rem) {
                            if (k & 1) s1 = fma(st[k * C::TILE], hs[k], s1);
                            else s0 = fma(st[k * C::TILE], hs[k], s0);
                        }
                    }
                    const double w1 = wr - (s0 + s1);
                    w[r] = w1;
                    if (MODE == CGS_UPDATE_DOTS) {
#pragma unroll
                        for (int k = 0; k < NCC; ++k) acc[k] = fma(st[k * C::TILE], w1, acc[k]);
#pragma unroll
                        for (int k = NCC; k < NCC + 3 && k < NC; ++k)
                            if (k - NCC < rem) acc[k] = fma(st[k * C::TILE], w1, acc[k]);
                    } else {
                        extra = fma(w1, w1, extra);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    if (MODE == CGS_DOTS) {
        if (reduce_columns<NC, C::NW>(acc, extra, true, nc, partials, ticket, d->h1)) {
            if (threadIdx.x == 0) d->w0sq = d->h1[nc];
        }
    } else if (MODE == CGS_UPDATE_DOTS) {
        if (reduce_columns<NC, C::NW>(acc, 0.0, false, nc, partials, ticket, d->h2)) {
            const int i = nc - 1, m1 = d->m + 1;
            for (int k = threadIdx.x; k < nc; k += blockDim.x) d->H[(size_t)i * m1 + k] = hs[k] + d->h2[k];
        }
    } else {
        double a1[1] = {extra};
        if (reduce_partials<1, C::NW>(a1, 1, partials, ticket, &d->r2)) {
            if (threadIdx.x == 0) {
                const int i = nc - 1, m1 = d->m + 1;
                double *h = d->H + (size_t)i * m1;
                const double hnext = sqrt(d->r2);
                for (int k = 0; k < i; ++k) {
                    const double a = h[k], b = h[k + 1];
                    h[k] = __dadd_rn(__dmul_rn(d->cs[k], a), __dmul_rn(d->sn[k], b));
                    h[k + 1] = __dadd_rn(__dmul_rn(-d->sn[k], a), __dmul_rn(d->cs[k], b));
                }
                const double rho = hypot(h[i], hnext);
                d->cs[i] = __ddiv_rn(h[i], rho);
                d->sn[i] = __ddiv_rn(hnext, rho);
                h[i] = rho;
                h[i + 1] = 0.0;
                d->g[i + 1] = __dmul_rn(-d->sn[i], d->g[i]);
                d->g[i] = __dmul_rn(d->cs[i], d->g[i]);
                d->iters += 1;
                d->k = i + 1;
                d->implicit = fabs(d->g[i + 1]);
                record_hist(d->hist, d->hist_len, d->iters, d->implicit, d->bnorm);
                const bool happy = hnext <= 1e-14 * sqrt(d->w0sq);
                if (d->implicit <= d->tol || d->iters >= d->maxit || happy || i == d->m - 1)
                    d->cycle_done = 1;
                d->hdiv = 1.0 / hnext;     // v_{i+1} = w / h_{i+1,i}
            }
        }
    }
}

// x[r] (or u[r]) = sum_j B[j][r] y[j] for j < k; add = 1 accumulates into x
__global__ void k_basis_combine(int n, int ld, const double *__restrict__ B, const GmresDev *d,
                                double *__restrict__ x, int add)
{
    if (*(volatile const int *)&d->noupd) return;
    __shared__ double ys[RS_MAX_RESTART];
    const int k = d->k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = d->y[j];
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(B[(size_t)j * ld + r], ys[j], s);
        x[r] = add ? __dadd_rn(x[r], s) : s;
    }
}

// v = s * r with s a device scalar (the reciprocal of the normalising norm)
__global__ void k_scale_dev(int n, const double *__restrict__ r, const double *__restrict__ s,
                            double *__restrict__ v, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    const double a = *s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = r[i] * a;
}

// y = x / sqrt(*n2) (0 when *n2 = 0): the normalised LGMRES correction
__global__ void k_scale_rsqrt(int n, const double *__restrict__ x, const double *__restrict__ n2,
                              double *__restrict__ y, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    const double s = *n2;
    const double a = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i] * a;
}

__global__ void k_axpy_skip(int n, const double *__restrict__ x, double *__restrict__ y, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] += x[i];
}

// cycle start: beta = ||r||, convergence test on the true residual
__global__ void k_gmres_start(GmresDev *d, const double *r2, double rtol, int first)
{
    if (threadIdx.x != 0) return;
    const double beta = sqrt(*r2);
    if (first) {
        d->tol = rtol * d->bnorm;
    }
    d->beta = beta;
    d->implicit = beta;
    d->converged = beta <= d->tol;
    d->cycle_done = d->converged || d->iters >= d->maxit;
    d->g[0] = beta;
    for (int j = 1; j <= d->m; ++j) d->g[j] = 0.0;
    d->k = 0;
    d->noupd = 1;
    d->hdiv = 1.0 / beta;      // v_1 = r / beta
}

// y = H(0:k,0:k)^{-1} g(0:k) by back-substitution
__global__ void k_gmres_backsolve(GmresDev *d)
{
    if (threadIdx.x != 0) return;
    const int k = d->k, m1 = d->m + 1;
    for (int j = k - 1; j >= 0; --j) {
        double s = d->g[j];
        for (int l = j + 1; l < k; ++l) s = fma(-d->H[(size_t)l * m1 + j], d->y[l], s);
        d->y[j] = __ddiv_rn(s, d->H[(size_t)j * m1 + j]);
    }
    d->noupd = k == 0;
}

static int red_grid(rs_ctx *ctx) { return ctx->red_blocks; }

static int blas_grid(rs_ctx *ctx, int n)
{
    return std::max(1, std::min((n + 255) / 256, ctx->num_sms * 8));
}

template <int NC, int NCC, int MODE>
static int launch_cgs_pass(rs_ctx *ctx, int n, int ld, int nc, double *V, GmresDev *d)
{
    typedef CgsCfg<NC> C;
    static unsigned long long raised = 0;   // devices whose shared-memory limit was raised
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (C::SMEM > 48 * 1024 && !(raised & bit)) {
        RS_CUDA_TRY(cudaFuncSetAttribute(k_cgs_pass<NC, NCC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM));
        raised |= bit;
    }
    RsProfScope prof(ctx, MODE == CGS_DOTS ? RS_PROF_CGS_DOTS
                          : MODE == CGS_UPDATE_DOTS ? RS_PROF_CGS_UPDATE_DOTS : RS_PROF_CGS_UPDATE_NORM);
    k_cgs_pass<NC, NCC, MODE><<<red_grid(ctx), C::THREADS, C::SMEM, ctx->stream>>>(
        n, ld, nc, V, V + (size_t)nc * ld, ctx->red_partials, ctx->red_ticket, d, ctx->d_err, ctx->spin_limit);
    ctx->launches++;
    return rs_check_launch(ctx);
}

// NCC = nc rounded down to 4; the reduction and ring width NC (a power of
// two) holds the up to 3 columns past it
template <int NCC>
static int launch_cgs(rs_ctx *ctx, int n, int ld, int nc, double *V, GmresDev *d)
{
    constexpr int NC = NCC + 3 <= 8 ? 8 : NCC + 3 <= 16 ? 16 : NCC + 3 <= 32 ? 32 : 64;
    int st = launch_cgs_pass<NC, NCC, CGS_DOTS>(ctx, n, ld, nc, V, d);
    if (!st) st = launch_cgs_pass<NC, NCC, CGS_UPDATE_DOTS>(ctx, n, ld, nc, V, d);
    if (!st) st = launch_cgs_pass<NC, NCC, CGS_UPDATE_NORM>(ctx, n, ld, nc, V, d);
    return st;
}

static int cgs_step(rs_ctx *ctx, int n, int ld, int nc, double *V, GmresDev *d)
{
    switch (nc / 4) {
    case 0: return launch_cgs<0>(ctx, n, ld, nc, V, d);
    case 1: return launch_cgs<4>(ctx, n, ld, nc, V, d);
    case 2: return launch_cgs<8>(ctx, n, ld, nc, V, d);
    case 3: return launch_cgs<12>(ctx, n, ld, nc, V, d);
    case 4: return launch_cgs<16>(ctx, n, ld, nc, V, d);
    case 5: return launch_cgs<20>(ctx, n, ld, nc, V, d);
    case 6: return launch_cgs<24>(ctx, n, ld, nc, V, d);
    case 7: return launch_cgs<28>(ctx, n, ld, nc, V, d);
    case 8: return launch_cgs<32>(ctx, n, ld, nc, V, d);
    case 9: return launch_cgs<36>(ctx, n, ld, nc, V, d);
    case 10: return launch_cgs<40>(ctx, n, ld, nc, V, d);
    case 11: return launch_cgs<44>(ctx, n, ld, nc, V, d);
    case 12: return launch_cgs<48>(ctx, n, ld, nc, V, d);
    case 13: return launch_cgs<52>(ctx, n, ld, nc, V, d);
    case 14: return launch_cgs<56>(ctx, n, ld, nc, V, d);
    case 15: return launch_cgs<60>(ctx, n, ld, nc, V, d);
    default: return nc <= 64 ? launch_cgs<64 - 3>(ctx, n, ld, nc, V, d) : RS_ERR_INVALID_ARG;
    }
}

static int finish_info(rs_ctx *ctx, const rs_mat *A, const double *b, const double *x, double *r,
                       double bnorm, rs_solve_info *info)
{
    RS_TRY(rs_residual_launch(A, b, x, r, ctx->d_scalars + 1, nullptr));
    RS_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_scalars + 1, sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    info->true_rel_res = bnorm > 0 ? sqrt(ctx->h_pinned[1]) / bnorm : 0.0;
    return RS_OK;
}

// GMRES(m) (Alg. 1 with right preconditioning and CGS2), FGMRES(m), and
// with aug_k > 0 (flexible only) LGMRES(m, aug_k): each cycle then adds one
// Arnoldi step per stored correction of the last aug_k cycles (newest
// first, held in a ring), and the cycle's correction Z y, normalised, joins
// the ring.
static int gmres_impl(const rs_mat *A, rs_pc *M, const rs_vec *bv, rs_vec *xv, int m, int aug_k, double rtol,
                      int maxit, int flexible, rs_solve_info *info)
{
    if (!A || !bv || !xv || !info) return RS_ERR_INVALID_ARG;
    if (m < 1 || aug_k < 0 || m + aug_k > RS_MAX_RESTART || (aug_k > 0 && !flexible) || maxit < 0 || !(rtol >= 0))
        return RS_ERR_INVALID_ARG;
    if (bv->n != A->n || xv->n != A->n) return RS_ERR_SIZE_MISMATCH;
    if (M && M->A->n != A->n) return RS_ERR_SIZE_MISMATCH;
    memset(info, 0, sizeof(*info));
    info->bad_row = -1;
    rs_ctx *ctx = A->ctx;
    const auto t0 = std::chrono::steady_clock::now();
    const int n = A->n;
    const int ld = (n + 31) / 32 * 32;
    double *V = nullptr, *Z = nullptr, *r = nullptr, *t = nullptr, *Aug = nullptr;
    GmresDev *d = nullptr;
    double *dhist = nullptr;
    int hlen = 0;
    int naug = 0, head = 0;      // stored corrections; the next ring slot
    int st = rs_alloc(ctx, (void **)&V, sizeof(double) * (size_t)ld * (m + aug_k + 1));
    if (!st && flexible) st = rs_alloc(ctx, (void **)&Z, sizeof(double) * (size_t)ld * (m + aug_k));
    if (!st && aug_k > 0) st = rs_alloc(ctx, (void **)&Aug, sizeof(double) * (size_t)ld * aug_k);
    if (!st) st = rs_alloc(ctx, (void **)&r, sizeof(double) * ld);
    if (!st) st = rs_alloc(ctx, (void **)&t, sizeof(double) * ld);
    if (!st) st = rs_alloc(ctx, (void **)&d, sizeof(GmresDev));
    if (!st) st = hist_begin(ctx, &dhist, &hlen);
    int status = RS_NOT_CONVERGED;
    double bnorm = 0.0;
    const double *b = bv->d;
    double *x = xv->d;
    if (st) goto out;
    {
        GmresDev h0;
        memset(&h0, 0, sizeof(h0));
        h0.m = m;
        h0.maxit = maxit;
        h0.noupd = 1;
        h0.hist = dhist;
        h0.hist_len = hlen;
        // ||b||
        st = rs_dot_launch(ctx, n, b, b, ctx->d_scalars);
        if (st) goto out;
        if (cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalars, sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            st = RS_ERR_CUDA;
            goto out;
        }
        bnorm = sqrt(ctx->h_pinned[0]);
        if (bnorm == 0.0) {
            cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream);
            status = RS_OK;
            goto done;
        }
        h0.bnorm = bnorm;
        cudaMemcpyAsync(d, &h0, sizeof(h0), cudaMemcpyHostToDevice, ctx->stream);
        const int gb = blas_grid(ctx, n);
        int *cycle_done = &d->cycle_done;
        int *noupd = &d->noupd;
        int first = 1;
        for (;;) {
            // this cycle's Arnoldi dimension: m, plus the stored corrections
            const int dim = m + naug;
            if (aug_k > 0 &&
                cudaMemcpyAsync(&d->m, &dim, sizeof(int), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
                st = RS_ERR_CUDA;
                goto out;
            }
            // true residual and cycle start
            st = rs_residual_launch(A, b, x, r, &d->r2, nullptr);
            if (st) goto out;
            k_gmres_start<<<1, 32, 0, ctx->stream>>>(d, &d->r2, rtol, first);
            first = 0;
            ctx->launches++;
            int hs[4];
            if (cudaMemcpyAsync(hs, &d->iters, sizeof(int) * 4, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                st = RS_ERR_CUDA;
                goto out;
            }
            // hs: iters, k, cycle_done, converged
            info->iters = hs[0];
            if (hs[3]) { status = RS_OK; break; }
            if (hs[2]) { status = RS_NOT_CONVERGED; break; }
            k_scale_dev<<<gb, 256, 0, ctx->stream>>>(n, r, &d->hdiv, V, nullptr);
            ctx->launches++;
            for (int i = 0; i < dim; ++i) {
                double *vi = V + (size_t)i * ld;
                double *zi = flexible ? Z + (size_t)i * ld : t;
                double *w = V + (size_t)(i + 1) * ld;
                if (i >= m) {
                    // augmented step: the (i - m)-th newest stored correction
                    const int slot = ((head - 1 - (i - m)) % aug_k + aug_k) % aug_k;
                    if (cudaMemcpyAsync(zi, Aug + (size_t)slot * ld, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                        ctx->stream) != cudaSuccess)
                        st = RS_ERR_CUDA;
                } else if (M) {
                    st = rs_pc_apply_dev(M, vi, zi, cycle_done);
                } else if (flexible) {
                    if (cudaMemcpyAsync(zi, vi, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream) !=
                        cudaSuccess)
                        st = RS_ERR_CUDA;
                } else {
                    zi = vi;
                }
                if (!st) st = rs_spmv_launch(A, zi, 1.0, 0.0, w, cycle_done);
                if (!st) st = cgs_step(ctx, n, ld, i + 1, V, d);
                if (st) goto out;
                if (i + 1 < dim) {
                    k_scale_dev<<<gb, 256, 0, ctx->stream>>>(n, w, &d->hdiv, w, cycle_done);
                    ctx->launches++;
                }
            }
            k_gmres_backsolve<<<1, 32, 0, ctx->stream>>>(d);
            ctx->launches++;
            if (flexible && aug_k > 0) {
                // the correction t = Z y; x += t; t / ||t|| joins the ring
                k_basis_combine<<<gb, 256, 0, ctx->stream>>>(n, ld, Z, d, t, 0);
                k_axpy_skip<<<gb, 256, 0, ctx->stream>>>(n, t, x, noupd);
                ctx->launches += 2;
                st = rs_dot_launch(ctx, n, t, t, &d->augn2);
                if (st) goto out;
                k_scale_rsqrt<<<gb, 256, 0, ctx->stream>>>(n, t, &d->augn2, Aug + (size_t)head * ld, noupd);
                ctx->launches++;
                head = (head + 1) % aug_k;
                naug = std::min(naug + 1, aug_k);
            } else if (flexible) {
                k_basis_combine<<<gb, 256, 0, ctx->stream>>>(n, ld, Z, d, x, 1);
                ctx->launches++;
            } else {
                k_basis_combine<<<gb, 256, 0, ctx->stream>>>(n, ld, V, d, r, 0);
                ctx->launches++;
                if (M) {
                    st = rs_pc_apply_dev(M, r, t, noupd);
                    if (st) goto out;
                    k_axpy_skip<<<gb, 256, 0, ctx->stream>>>(n, t, x, noupd);
                } else {
                    k_axpy_skip<<<gb, 256, 0, ctx->stream>>>(n, r, x, noupd);
                }
                ctx->launches++;
            }
            info->restarts++;
            if (cudaGetLastError() != cudaSuccess) { st = RS_ERR_CUDA; goto out; }
        }
        GmresDev hf;
        cudaMemcpyAsync(&hf, d, sizeof(hf), cudaMemcpyDeviceToHost, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        info->iters = hf.iters;
        info->implicit_rel_res = hf.implicit / bnorm;
    }
done:
    st = rs_collect_device_error(ctx, &info->bad_row);
    if (st) goto out;
    st = finish_info(ctx, A, b, x, r ? r : t, bnorm, info);
    if (st) goto out;
    if (status == RS_OK && info->true_rel_res > rtol && bnorm > 0) status = RS_NOT_CONVERGED;
out:
    {
        const int hs = hist_end(ctx, dhist, hlen, info->iters);
        if (!st) st = hs;
    }
    rs_free(ctx, V);
    rs_free(ctx, Z);
    rs_free(ctx, Aug);
    rs_free(ctx, r);
    rs_free(ctx, t);
    rs_free(ctx, d);
    info->status = st ? st : status;
    info->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return info->status;
}

extern "C" int rs_solve_gmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart,
                              double rtol, int32_t maxit, rs_solve_info *info)
{
    return gmres_impl(A, M, b, x, restart, 0, rtol, maxit, 0, info);
}

extern "C" int rs_solve_fgmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart,
                               double rtol, int32_t maxit, rs_solve_info *info)
{
    return gmres_impl(A, M, b, x, restart, 0, rtol, maxit, 1, info);
}

extern "C" int rs_solve_lgmres(const rs_mat *A, rs_pc *M, const rs_vec *b, rs_vec *x, int32_t restart,
                               int32_t aug_k, double rtol, int32_t maxit, rs_solve_info *info)
{
    return gmres_impl(A, M, b, x, restart, aug_k, rtol, maxit, 1, info);
}

// ---------------------------------------------------------------------------
// BiCGSTAB
// ---------------------------------------------------------------------------
struct BicgDev {
    double red[8];          // reduction outputs
    double rho, rho0, alpha, omega, beta, tol, bnorm, implicit;
    int iters, done, half, fresh, breakdown, maxit, status, pad;
    double *hist;           // residual history (device), hist_len entries
    int hist_len, pad_;
};

// generic fused row kernel with up to 3 dot products and a scalar epilogue
//  op 0: p = r + beta (p - omega v)                             (no dots)
//  op 1: s = r - alpha v;  red = {||s||^2}                       -> half-step test
//  op 2: x += alpha ph + omega sh; r = s - omega t; red = {(rh,r), ||r||^2}
//  op 3: red = {(rh, v)}                                        -> alpha
//  op 4: red = {(t, s), (t, t)}                                 -> omega
//  op 5: x += alpha ph (half-step exit)
__global__ void __launch_bounds__(RS_RED_THREADS)
k_bicg(int op, int n, double *p, double *r, const double *__restrict__ v, double *s,
       const double *__restrict__ t, double *x, const double *__restrict__ ph,
       const double *__restrict__ sh, const double *__restrict__ rh, double *partials,
       unsigned *ticket, BicgDev *d)
{
    if (op != 5 && (*(volatile int *)&d->done || *(volatile int *)&d->half)) return;
    if (op == 5 && !*(volatile int *)&d->half) return;
    const double alpha = d->alpha, omega = d->omega, beta = d->beta;
    double acc[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        switch (op) {
        case 0: p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]); break;
        case 1: {
            const double si = fma(-alpha, v[i], r[i]);
            s[i] = si;
            acc[0] = fma(si, si, acc[0]);
            break;
        }
        case 2: {
            x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
            const double ri = fma(-omega, t[i], s[i]);
            r[i] = ri;
            acc[0] = fma(rh[i], ri, acc[0]);
            acc[1] = fma(ri, ri, acc[1]);
            break;
        }
        case 3: acc[0] = fma(rh[i], v[i], acc[0]); break;
        case 4:
            acc[0] = fma(t[i], s[i], acc[0]);
            acc[1] = fma(t[i], t[i], acc[1]);
            break;
        case 5: x[i] = fma(alpha, ph[i], x[i]); break;
        }
    }
    if (op == 0) return;
    if (op == 5) {
        // the half-step update runs once: the last block to finish clears the flag
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
                d->half = 0;
                *ticket = 0;
                __threadfence();
            }
        }
        return;
    }
    const int nv = (op == 2 || op == 4) ? 2 : 1;
    if (!reduce_partials<2>(acc, nv, partials, ticket, d->red)) return;
    if (threadIdx.x != 0) return;
    switch (op) {
    case 1: {
        d->iters += 1;
        const double sn = sqrt(d->red[0]);
        if (sn <= d->tol) {
            d->half = 1; d->implicit = sn; d->done = 1; d->fresh = 1;
            record_hist(d->hist, d->hist_len, d->iters, sn, d->bnorm);
        }
        break;
    }
    case 2: {
        const double rho = d->red[0];
        const double rn = sqrt(d->red[1]);
        d->implicit = rn;
        record_hist(d->hist, d->hist_len, d->iters, rn, d->bnorm);
        d->rho0 = d->rho;
        if (rn <= d->tol) { d->done = 1; d->fresh = 1; break; }
        if (!(d->omega != 0.0) || !isfinite(d->omega)) { d->breakdown = 1; d->done = 1; break; }
        if (!(fabs(rho) > 0.0) || !isfinite(rho)) { d->breakdown = 1; d->done = 1; break; }
        d->beta = (rho / d->rho0) * (d->alpha / d->omega);
        d->rho = rho;
        if (d->iters >= d->maxit) d->done = 1;
        break;
    }
    case 3: {
        const double rv = d->red[0];
        if (!(fabs(rv) > 0.0) || !isfinite(rv)) { d->breakdown = 1; d->done = 1; break; }
        d->alpha = d->rho / rv;
        break;
    }
    case 4: {
        const double ts = d->red[0], tt = d->red[1];
        d->omega = tt > 0.0 ? ts / tt : 0.0;
        break;
    }
    }
}

// restart from the true residual r = b - A x (already in r, ||r||^2 in red[1])
__global__ void k_bicg_restart(int n, const double *__restrict__ r, double *rh, double *p, double *v,
                               BicgDev *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        rh[i] = r[i];
        p[i] = 0.0;
        v[i] = 0.0;
    }
}

__global__ void k_bicg_restart_scalars(BicgDev *d, const double *r2)
{
    if (threadIdx.x) return;
    const double rn = sqrt(*r2);
    d->implicit = rn;
    d->fresh = 0;
    d->half = 0;
    d->done = 0;
    if (rn <= d->tol) { d->done = 1; d->status = 1; return; }   // status 1: converged
    if (d->iters >= d->maxit) { d->done = 1; return; }
    // rho = (rh, r) = ||r||^2 with rh = r; beta multiplies p = 0, so its value is irrelevant
    d->rho0 = 1.0;
    d->alpha = 1.0;
    d->omega = 1.0;
    d->rho = *r2;
    d->beta = 0.0;
    if (!(d->rho > 0.0) || !isfinite(d->rho)) { d->breakdown = 1; d->done = 1; }
}

extern "C" int rs_solve_bicgstab(const rs_mat *A, rs_pc *M, const rs_vec *bv, rs_vec *xv, double rtol,
                                 int32_t maxit, rs_solve_info *info)
{
    if (!A || !bv || !xv || !info) return RS_ERR_INVALID_ARG;
    if (maxit < 0 || !(rtol >= 0)) return RS_ERR_INVALID_ARG;
    if (bv->n != A->n || xv->n != A->n) return RS_ERR_SIZE_MISMATCH;
    memset(info, 0, sizeof(*info));
    info->bad_row = -1;
    rs_ctx *ctx = A->ctx;
    const auto t0 = std::chrono::steady_clock::now();
    const int n = A->n;
    const int ld = (n + 31) / 32 * 32;
    double *buf = nullptr;
    BicgDev *d = nullptr;
    double *dhist = nullptr;
    int hlen = 0;
    int st = rs_alloc(ctx, (void **)&buf, sizeof(double) * (size_t)ld * 8);
    if (!st) st = rs_alloc(ctx, (void **)&d, sizeof(BicgDev));
    if (!st) st = hist_begin(ctx, &dhist, &hlen);
    int status = RS_NOT_CONVERGED;
    double bnorm = 0.0;
    const double *b = bv->d;
    double *x = xv->d;
    double *r = buf, *rh = buf + ld, *p = buf + 2 * (size_t)ld, *v = buf + 3 * (size_t)ld;
    double *s = buf + 4 * (size_t)ld, *t = buf + 5 * (size_t)ld, *ph = buf + 6 * (size_t)ld;
    double *sh = buf + 7 * (size_t)ld;
    if (!M) {            // no preconditioner: M^{-1} p = p, M^{-1} s = s
        ph = p;
        sh = s;
    }
    if (st) goto out;
    {
        st = rs_dot_launch(ctx, n, b, b, ctx->d_scalars);
        if (st) goto out;
        cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { st = RS_ERR_CUDA; goto out; }
        bnorm = sqrt(ctx->h_pinned[0]);
        if (bnorm == 0.0) {
            cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream);
            status = RS_OK;
            goto done;
        }
        BicgDev h0;
        memset(&h0, 0, sizeof(h0));
        h0.tol = rtol * bnorm;
        h0.bnorm = bnorm;
        h0.maxit = maxit;
        h0.hist = dhist;
        h0.hist_len = hlen;
        cudaMemcpyAsync(d, &h0, sizeof(h0), cudaMemcpyHostToDevice, ctx->stream);
        const int gr = red_grid(ctx), gb = blas_grid(ctx, n);
        int *halt = &d->done;
        const int batch = 8;
        for (;;) {
            // (re)start from the true residual
            st = rs_residual_launch(A, b, x, r, &d->red[1], nullptr);
            if (st) goto out;
            k_bicg_restart<<<gb, 256, 0, ctx->stream>>>(n, r, rh, p, v, d);
            k_bicg_restart_scalars<<<1, 32, 0, ctx->stream>>>(d, &d->red[1]);
            ctx->launches += 2;
            bool restart = false;
            while (!restart) {
                for (int it = 0; it < batch; ++it) {
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(0, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    ctx->launches++;
                    if (M) st = rs_pc_apply_dev(M, p, ph, halt);
                    if (st) goto out;
                    st = rs_spmv_launch(A, ph, 1.0, 0.0, v, halt);
                    if (st) goto out;
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(3, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(1, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(5, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    ctx->launches += 3;
                    if (M) st = rs_pc_apply_dev(M, s, sh, halt);
                    if (st) goto out;
                    st = rs_spmv_launch(A, sh, 1.0, 0.0, t, halt);
                    if (st) goto out;
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(4, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_bicg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(2, n, p, r, v, s, t, x, ph, sh, rh,
                                                                       ctx->red_partials, ctx->red_ticket, d);
                    }
                    ctx->launches += 2;
                }
                BicgDev hd;
                if (cudaMemcpyAsync(&hd, d, sizeof(hd), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                    cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                    st = RS_ERR_CUDA;
                    goto out;
                }
                info->iters = hd.iters;
                info->implicit_rel_res = hd.implicit / bnorm;
                if (hd.status == 1) { status = RS_OK; goto done; }
                if (hd.breakdown) { status = RS_ERR_BREAKDOWN; goto done; }
                if (hd.fresh) { restart = true; break; }       // confirm with the true residual
                if (hd.done || hd.iters >= maxit) { status = RS_NOT_CONVERGED; goto done; }
            }
        }
    }
done:
    st = rs_collect_device_error(ctx, &info->bad_row);
    if (st) goto out;
    st = finish_info(ctx, A, b, x, r, bnorm, info);
    if (st) goto out;
    if (status == RS_OK && info->true_rel_res > rtol && bnorm > 0) status = RS_NOT_CONVERGED;
    if (status == RS_NOT_CONVERGED && info->true_rel_res <= rtol && bnorm > 0) status = RS_OK;
out:
    {
        const int hs = hist_end(ctx, dhist, hlen, info->iters);
        if (!st) st = hs;
    }
    rs_free(ctx, buf);
    rs_free(ctx, d);
    info->status = st ? st : status;
    info->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return info->status;
}

// ---------------------------------------------------------------------------
// Preconditioned conjugate gradient (Alg. 2), device-resident like BiCGSTAB:
// the scalars live in device memory and the last block of each reduction
// forms beta or alpha; the host synchronises once per batch of iterations.
// ---------------------------------------------------------------------------
struct CgDev {
    double red[2];
    double rho, rho0, alpha, beta, tol, bnorm, implicit;
    int iters, done, fresh, breakdown, maxit, status, first, pad;
    double *hist;           // residual history (device), hist_len entries
    int hist_len, pad_;
};

//  op 0: red = {(r, z)}                 -> rho, beta = rho / rho_prev (0 on the first pass)
//  op 1: p = z + beta p
//  op 2: red = {(p, q)}                 -> alpha = rho / (p, q)
//  op 3: x += alpha p; r -= alpha q; red = {||r||^2} -> convergence test
__global__ void __launch_bounds__(RS_RED_THREADS)
k_cg(int op, int n, double *x, double *r, const double *__restrict__ z, double *p,
     const double *__restrict__ q, double *partials, unsigned *ticket, CgDev *d)
{
    if (*(volatile int *)&d->done) return;
    const double alpha = d->alpha, beta = d->beta;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        switch (op) {
        case 0: acc[0] = fma(r[i], z[i], acc[0]); break;
        case 1: p[i] = fma(beta, p[i], z[i]); break;
        case 2: acc[0] = fma(p[i], q[i], acc[0]); break;
        case 3: {
            x[i] = fma(alpha, p[i], x[i]);
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            acc[0] = fma(ri, ri, acc[0]);
            break;
        }
        }
    }
    if (op == 1) return;
    if (!reduce_partials<1>(acc, 1, partials, ticket, d->red)) return;
    if (threadIdx.x != 0) return;
    switch (op) {
    case 0: {
        const double rho = d->red[0];
        if (!(rho != 0.0) || !isfinite(rho)) { d->breakdown = 1; d->done = 1; break; }
        d->beta = d->first ? 0.0 : rho / d->rho0;
        d->first = 0;
        d->rho = rho;
        break;
    }
    case 2: {
        const double pq = d->red[0];
        if (!(pq > 0.0) || !isfinite(pq)) { d->breakdown = 1; d->done = 1; break; }
        d->alpha = d->rho / pq;
        break;
    }
    case 3: {
        d->iters += 1;
        d->rho0 = d->rho;
        const double rn = sqrt(d->red[0]);
        d->implicit = rn;
        record_hist(d->hist, d->hist_len, d->iters, rn, d->bnorm);
        if (rn <= d->tol) { d->done = 1; d->fresh = 1; break; }
        if (d->iters >= d->maxit) d->done = 1;
        break;
    }
    }
}

// restart from the true residual (in r, ||r||^2 in *r2): p = 0, first pass
__global__ void k_cg_restart(int n, double *p, CgDev *d, const double *r2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0.0;
    if (blockIdx.x || threadIdx.x) return;
    const double rn = sqrt(*r2);
    d->implicit = rn;
    d->fresh = 0;
    d->done = 0;
    d->first = 1;
    d->beta = 0.0;
    if (rn <= d->tol) { d->done = 1; d->status = 1; return; }   // status 1: converged
    if (d->iters >= d->maxit) d->done = 1;
}

extern "C" int rs_solve_cg(const rs_mat *A, rs_pc *M, const rs_vec *bv, rs_vec *xv, double rtol, int32_t maxit,
                           rs_solve_info *info)
{
    if (!A || !bv || !xv || !info) return RS_ERR_INVALID_ARG;
    if (maxit < 0 || !(rtol >= 0)) return RS_ERR_INVALID_ARG;
    if (bv->n != A->n || xv->n != A->n) return RS_ERR_SIZE_MISMATCH;
    memset(info, 0, sizeof(*info));
    info->bad_row = -1;
    rs_ctx *ctx = A->ctx;
    const auto t0 = std::chrono::steady_clock::now();
    const int n = A->n;
    const int ld = (n + 31) / 32 * 32;
    double *buf = nullptr;
    CgDev *d = nullptr;
    double *dhist = nullptr;
    int hlen = 0;
    int st = rs_alloc(ctx, (void **)&buf, sizeof(double) * (size_t)ld * 4);
    if (!st) st = rs_alloc(ctx, (void **)&d, sizeof(CgDev));
    if (!st) st = hist_begin(ctx, &dhist, &hlen);
    int status = RS_NOT_CONVERGED;
    double bnorm = 0.0;
    const double *b = bv->d;
    double *x = xv->d;
    double *r = buf, *z = buf + ld, *p = buf + 2 * (size_t)ld, *q = buf + 3 * (size_t)ld;
    if (!M) z = r;       // no preconditioner: z = r
    if (st) goto out;
    {
        st = rs_dot_launch(ctx, n, b, b, ctx->d_scalars);
        if (st) goto out;
        cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { st = RS_ERR_CUDA; goto out; }
        bnorm = sqrt(ctx->h_pinned[0]);
        if (bnorm == 0.0) {
            cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream);
            status = RS_OK;
            goto done;
        }
        CgDev h0;
        memset(&h0, 0, sizeof(h0));
        h0.tol = rtol * bnorm;
        h0.bnorm = bnorm;
        h0.maxit = maxit;
        h0.hist = dhist;
        h0.hist_len = hlen;
        cudaMemcpyAsync(d, &h0, sizeof(h0), cudaMemcpyHostToDevice, ctx->stream);
        const int gr = red_grid(ctx), gb = blas_grid(ctx, n);
        int *halt = &d->done;
        const int batch = 8;
        for (;;) {
            st = rs_residual_launch(A, b, x, r, &d->red[1], nullptr);
            if (st) goto out;
            k_cg_restart<<<gb, 256, 0, ctx->stream>>>(n, p, d, &d->red[1]);
            ctx->launches++;
            bool restart = false;
            while (!restart) {
                for (int it = 0; it < batch; ++it) {
                    if (M) st = rs_pc_apply_dev(M, r, z, halt);
                    if (st) goto out;
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_cg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(0, n, x, r, z, p, q, ctx->red_partials,
                                                                     ctx->red_ticket, d);
                    }
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_cg<<<gb, RS_RED_THREADS, 0, ctx->stream>>>(1, n, x, r, z, p, q, ctx->red_partials,
                                                                     ctx->red_ticket, d);
                    }
                    ctx->launches += 2;
                    st = rs_spmv_launch(A, p, 1.0, 0.0, q, halt);
                    if (st) goto out;
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_cg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(2, n, x, r, z, p, q, ctx->red_partials,
                                                                     ctx->red_ticket, d);
                    }
                    {
                        RsProfScope prof(ctx, RS_PROF_BLAS1);
                        k_cg<<<gr, RS_RED_THREADS, 0, ctx->stream>>>(3, n, x, r, z, p, q, ctx->red_partials,
                                                                     ctx->red_ticket, d);
                    }
                    ctx->launches += 2;
                }
                CgDev hd;
                if (cudaMemcpyAsync(&hd, d, sizeof(hd), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                    cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                    st = RS_ERR_CUDA;
                    goto out;
                }
                info->iters = hd.iters;
                info->implicit_rel_res = hd.implicit / bnorm;
                if (hd.status == 1) { status = RS_OK; goto done; }
                if (hd.breakdown) { status = RS_ERR_BREAKDOWN; goto done; }
                if (hd.fresh) { restart = true; break; }       // confirm with the true residual
                if (hd.done || hd.iters >= maxit) { status = RS_NOT_CONVERGED; goto done; }
            }
        }
    }
done:
    st = rs_collect_device_error(ctx, &info->bad_row);
    if (st) goto out;
    st = finish_info(ctx, A, b, x, r, bnorm, info);
    if (st) goto out;
    if (status == RS_OK && info->true_rel_res > rtol && bnorm > 0) status = RS_NOT_CONVERGED;
    if (status == RS_NOT_CONVERGED && info->true_rel_res <= rtol && bnorm > 0) status = RS_OK;
out:
    {
        const int hs = hist_end(ctx, dhist, hlen, info->iters);
        if (!st) st = hs;
    }
    rs_free(ctx, buf);
    rs_free(ctx, d);
    info->status = st ? st : status;
    info->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return info->status;
}
