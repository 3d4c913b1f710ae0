// ILU(0) and block ILU(0): analysis, numeric factorisation, triangular solves.
//
// The factorisation L U ~ A and the two solves L y = r, U z = y are Eq. 3
// (Sec. 4.1); the paper notes these solves run row by row and scale poorly.
// Here each row is one GPU thread and rows run as soon as the rows they depend
// on are final ("sync-free" sweeps):
//  * the host computes, once per pattern, the level of every row in the
//    dependency graph of L (and of U) and orders the rows level by level,
//    each level padded to a multiple of 32 so a warp never holds two levels;
//  * the factors are stored in that order in a sliced-ELL layout (slices of
//    32 rows, entry e of the 32 rows of a slice contiguous) so every load of
//    factor data is coalesced;
//  * blocks take consecutive work tickets from an atomic counter, so every
//    row a thread waits for belongs to a block that is already running —
//    the sweep cannot deadlock; each wait is also bounded in time and
//    reports RS_ERR_DEVICE_TIMEOUT instead of hanging;
//  * a row publishes its value with a release store of the sweep's epoch
//    into its flag, so flags never need clearing; the last block of a sweep
//    advances the epoch and resets the ticket (the sweep is self-cleaning).
// The factorisation itself uses the same schedule (the rows that row i reads
// are exactly its L-dependencies), runs the IKJ update in ascending column
// order without contracted multiply-adds, and therefore produces the same
// FP64 factors as a sequential row-by-row ILU(0).
#include <math.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

#define RS_SWEEP_THREADS 128

// ---------------------------------------------------------------------------
// host analysis
// ---------------------------------------------------------------------------
static int build_layout(rs_ctx *ctx, int nrows, const std::vector<int> &ptr,
                        const std::vector<int> &col, const std::vector<int> &diag, bool lower,
                        TriLayout &T)
{
    std::vector<int> lev(nrows, 0);
    int nlev = 0;
    if (lower) {
        for (int i = 0; i < nrows; ++i) {
            int l = 0;
            for (int q = ptr[i]; q < diag[i]; ++q) l = std::max(l, lev[col[q]] + 1);
            lev[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    } else {
        for (int i = nrows - 1; i >= 0; --i) {
            int l = 0;
            for (int q = diag[i] + 1; q < ptr[i + 1]; ++q) l = std::max(l, lev[col[q]] + 1);
            lev[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    }
    std::vector<int> cnt(nlev + 1, 0);
    for (int i = 0; i < nrows; ++i) cnt[lev[i]]++;
    std::vector<int64_t> start(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) start[l + 1] = start[l] + ((cnt[l] + 31) / 32) * 32;
    const int64_t npad = start[nlev];
    if (npad > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
    std::vector<int> pos(npad, -1);
    std::vector<int64_t> fill(start.begin(), start.end());
    if (lower) {
        for (int i = 0; i < nrows; ++i) pos[fill[lev[i]]++] = i;
    } else {
        for (int i = nrows - 1; i >= 0; --i) pos[fill[lev[i]]++] = i;
    }
    const int nslices = (int)(npad / 32);
    std::vector<int> sptr(nslices + 1, 0);
    int64_t nent = 0;
    for (int s = 0; s < nslices; ++s) {
        int w = 0;
        for (int l = 0; l < 32; ++l) {
            const int row = pos[s * 32 + l];
            if (row < 0) continue;
            const int c = lower ? diag[row] - ptr[row] : ptr[row + 1] - diag[row] - 1;
            w = std::max(w, c);
        }
        sptr[s] = (int)nent;
        nent += (int64_t)w * 32;
        if (nent > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
    }
    sptr[nslices] = (int)nent;
    std::vector<int> ecol(nent, -1), esrc(nent, -1), dsrc(npad, -1);
    for (int s = 0; s < nslices; ++s) {
        for (int l = 0; l < 32; ++l) {
            const int row = pos[s * 32 + l];
            if (row < 0) continue;
            const int q0 = lower ? ptr[row] : diag[row] + 1;
            const int q1 = lower ? diag[row] : ptr[row + 1];
            for (int q = q0; q < q1; ++q) {
                const int64_t e = sptr[s] + (int64_t)(q - q0) * 32 + l;
                ecol[e] = col[q];
                esrc[e] = q;
            }
            dsrc[s * 32 + l] = diag[row];
        }
    }
    T.npad = (int)npad;
    T.nslices = nslices;
    T.nlevels = nlev;
    T.nent = nent;
    int st = RS_OK;
    st = st ? st : rs_alloc(ctx, (void **)&T.pos, sizeof(int) * npad);
    st = st ? st : rs_alloc(ctx, (void **)&T.slice_ptr, sizeof(int) * (nslices + 1));
    st = st ? st : rs_alloc(ctx, (void **)&T.col, sizeof(int) * nent);
    st = st ? st : rs_alloc(ctx, (void **)&T.src, sizeof(int) * nent);
    st = st ? st : rs_alloc(ctx, (void **)&T.dsrc, sizeof(int) * npad);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    RS_CUDA_TRY(cudaMemcpyAsync(T.pos, pos.data(), sizeof(int) * npad, cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaMemcpyAsync(T.slice_ptr, sptr.data(), sizeof(int) * (nslices + 1),
                                cudaMemcpyHostToDevice, s));
    if (nent) {
        RS_CUDA_TRY(cudaMemcpyAsync(T.col, ecol.data(), sizeof(int) * nent, cudaMemcpyHostToDevice, s));
        RS_CUDA_TRY(cudaMemcpyAsync(T.src, esrc.data(), sizeof(int) * nent, cudaMemcpyHostToDevice, s));
    }
    RS_CUDA_TRY(cudaMemcpyAsync(T.dsrc, dsrc.data(), sizeof(int) * npad, cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));   // host vectors go out of scope
    return RS_OK;
}

static void free_layout(rs_ctx *ctx, TriLayout &T)
{
    rs_free(ctx, T.pos);
    rs_free(ctx, T.slice_ptr);
    rs_free(ctx, T.col);
    rs_free(ctx, T.src);
    rs_free(ctx, T.dsrc);
    rs_free(ctx, T.val);
    rs_free(ctx, T.diag);
    T = TriLayout();
}

// ---------------------------------------------------------------------------
// sweep bookkeeping shared by all sync-free kernels
// ---------------------------------------------------------------------------
struct SweepTicket {
    int base;
    int epoch;
};

__device__ __forceinline__ void sweep_begin(SweepState *st, int *s_base, int *s_epoch)
{
    if (threadIdx.x == 0) {
        *s_base = (int)atomicAdd(&st->ticket, 1u) * blockDim.x;
        *s_epoch = *(volatile int *)&st->epoch;
    }
    __syncthreads();
}

__device__ __forceinline__ void sweep_end(SweepState *st, int epoch)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&st->done, 1u);
        if (d == gridDim.x - 1) {
            st->ticket = 0;
            st->done = 0;
            st->epoch = epoch + 1;
            __threadfence();
        }
    }
}

__device__ __forceinline__ void report_timeout(int *err) { atomicOr(err, RS_DEVERR_TIMEOUT); }

// ---------------------------------------------------------------------------
// numeric factorisation
// ---------------------------------------------------------------------------
// Scalar ILU(0), IKJ form: for each k < i in row i (ascending): l_ik = a_ik / u_kk,
// then a_ij -= l_ik u_kj for every j > k present in both rows.
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_ilu0_factor(int npad, const int *__restrict__ pos, const int *__restrict__ ptr,
              const int *__restrict__ col, const int *__restrict__ diagpos, double *lu,
              int *flags, SweepState *st, int *err, int *bad_row, long long limit)
{
    __shared__ int s_base, s_epoch;
    sweep_begin(st, &s_base, &s_epoch);
    const int epoch = s_epoch;
    const int p = s_base + threadIdx.x;
    const int row = p < npad ? pos[p] : -1;
    if (row >= 0) {
        const int e_i = ptr[row + 1];
        const int d_i = diagpos[row];
        for (int q = ptr[row]; q < d_i; ++q) {
            const int k = col[q];
            if (!wait_epoch(flags + k, epoch, limit)) report_timeout(err);
            const int d_k = diagpos[k];
            const double lik = lu[q] / __ldcg(lu + d_k);
            lu[q] = lik;
            int qq = q + 1;
            const int e_k = ptr[k + 1];
            for (int r = d_k + 1; r < e_k; ++r) {
                const int j = col[r];
                while (qq < e_i && col[qq] < j) ++qq;
                if (qq == e_i) break;
                if (col[qq] == j) lu[qq] = __dsub_rn(lu[qq], __dmul_rn(lik, __ldcg(lu + r)));
            }
        }
        const double d = lu[d_i];
        if (!(d != 0.0) || !isfinite(d)) {
            atomicOr(err, RS_DEVERR_PIVOT);
            atomicMin(bad_row, row);
        }
        st_release(flags + row, epoch);
    }
    sweep_end(st, epoch);
}

// bs x bs block helpers (row-major, registers)
template <int BS>
__device__ __forceinline__ void blk_mul(const double *a, const double *b, double *c)
{
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < BS; ++k) s = __dadd_rn(s, __dmul_rn(a[i * BS + k], b[k * BS + j]));
            c[i * BS + j] = s;
        }
}

// inverse by Gauss-Jordan elimination with partial pivoting; false if singular
template <int BS>
__device__ bool blk_inverse(const double *a, double *inv)
{
    double m[BS * BS], e[BS * BS];
#pragma unroll
    for (int i = 0; i < BS * BS; ++i) { m[i] = a[i]; e[i] = 0.0; }
#pragma unroll
    for (int i = 0; i < BS; ++i) e[i * BS + i] = 1.0;
#pragma unroll
    for (int c = 0; c < BS; ++c) {
        int piv = c;
#pragma unroll
        for (int r = c + 1; r < BS; ++r)
            if (fabs(m[r * BS + c]) > fabs(m[piv * BS + c])) piv = r;
        // swap rows c and piv (done with selects to keep arrays in registers)
#pragma unroll
        for (int r = c + 1; r < BS; ++r) {
            if (r == piv) {
#pragma unroll
                for (int k = 0; k < BS; ++k) {
                    double t = m[c * BS + k]; m[c * BS + k] = m[r * BS + k]; m[r * BS + k] = t;
                    t = e[c * BS + k]; e[c * BS + k] = e[r * BS + k]; e[r * BS + k] = t;
                }
            }
        }
        const double d = m[c * BS + c];
        if (!(d != 0.0) || !isfinite(d)) return false;
#pragma unroll
        for (int k = 0; k < BS; ++k) { m[c * BS + k] = m[c * BS + k] / d; e[c * BS + k] = e[c * BS + k] / d; }
#pragma unroll
        for (int r = 0; r < BS; ++r) {
            if (r == c) continue;
            const double f = m[r * BS + c];
#pragma unroll
            for (int k = 0; k < BS; ++k) {
                m[r * BS + k] = __dsub_rn(m[r * BS + k], __dmul_rn(f, m[c * BS + k]));
                e[r * BS + k] = __dsub_rn(e[r * BS + k], __dmul_rn(f, e[c * BS + k]));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < BS * BS; ++i) inv[i] = e[i];
    return true;
}

// Block ILU(0): L_IK = A_IK inv(U_KK); A_IJ -= L_IK U_KJ; dinv_I = inv(U_II).
template <int BS>
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_bilu0_factor(int npad, const int *__restrict__ pos, const int *__restrict__ ptr,
               const int *__restrict__ col, const int *__restrict__ diagpos, double *lu,
               double *dinv, int *flags, SweepState *st, int *err, int *bad_row, long long limit)
{
    constexpr int B2 = BS * BS;
    __shared__ int s_base, s_epoch;
    sweep_begin(st, &s_base, &s_epoch);
    const int epoch = s_epoch;
    const int p = s_base + threadIdx.x;
    const int row = p < npad ? pos[p] : -1;
    if (row >= 0) {
        const int e_i = ptr[row + 1];
        const int d_i = diagpos[row];
        double a[B2], t[B2], u[B2], c[B2];
        for (int q = ptr[row]; q < d_i; ++q) {
            const int k = col[q];
            if (!wait_epoch(flags + k, epoch, limit)) report_timeout(err);
#pragma unroll
            for (int x = 0; x < B2; ++x) { a[x] = lu[(size_t)q * B2 + x]; t[x] = __ldcg(dinv + (size_t)k * B2 + x); }
            blk_mul<BS>(a, t, c);                      // L_IK
#pragma unroll
            for (int x = 0; x < B2; ++x) lu[(size_t)q * B2 + x] = c[x];
            int qq = q + 1;
            const int e_k = ptr[k + 1];
            for (int r = diagpos[k] + 1; r < e_k; ++r) {
                const int j = col[r];
                while (qq < e_i && col[qq] < j) ++qq;
                if (qq == e_i) break;
                if (col[qq] == j) {
#pragma unroll
                    for (int x = 0; x < B2; ++x) t[x] = __ldcg(lu + (size_t)r * B2 + x);
                    blk_mul<BS>(c, t, u);
#pragma unroll
                    for (int x = 0; x < B2; ++x)
                        lu[(size_t)qq * B2 + x] = __dsub_rn(lu[(size_t)qq * B2 + x], u[x]);
                }
            }
        }
#pragma unroll
        for (int x = 0; x < B2; ++x) a[x] = lu[(size_t)d_i * B2 + x];
        if (!blk_inverse<BS>(a, t)) {
            atomicOr(err, RS_DEVERR_PIVOT);
            atomicMin(bad_row, row);
#pragma unroll
            for (int x = 0; x < B2; ++x) t[x] = 0.0;
        }
#pragma unroll
        for (int x = 0; x < B2; ++x) dinv[(size_t)row * B2 + x] = t[x];
        st_release(flags + row, epoch);
    }
    sweep_end(st, epoch);
}

// Gather the factor values of one triangle into its sliced-ELL arrays
// (plane-major for blocks: value x of entry e at [x * nent + e]).
template <typename T>
__global__ void k_gather_tri(int64_t nent, int b2, const int *__restrict__ src,
                             const double *__restrict__ lu, T *__restrict__ val)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nent;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = src[e];
        for (int x = 0; x < b2; ++x) val[(size_t)x * nent + e] = s >= 0 ? (T)lu[(size_t)s * b2 + x] : (T)0;
    }
}

// diagonal of U per position: u_ii (scalar) or inv(U_II) (blocks)
template <typename T>
__global__ void k_gather_diag(int npad, int b2, const int *__restrict__ pos, const int *__restrict__ dsrc,
                              const double *__restrict__ lu, const double *__restrict__ dinv,
                              T *__restrict__ diag)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npad; p += gridDim.x * blockDim.x) {
        const int row = pos[p];
        for (int x = 0; x < b2; ++x) {
            double v = 1.0;
            if (row >= 0) v = b2 == 1 ? lu[dsrc[p]] : dinv[(size_t)row * b2 + x];
            diag[(size_t)x * npad + p] = (T)v;
        }
    }
}

// ---------------------------------------------------------------------------
// triangular sweeps
// ---------------------------------------------------------------------------
// L y = r (unit lower).  TI: type of r; T: working type.  scale (device,
// optional) multiplies r on load.
template <int BS, typename T, typename TI>
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_lsolve(int npad, int64_t nent, const int *__restrict__ pos, const int *__restrict__ sptr,
         const int *__restrict__ ecol, const T *__restrict__ val, const TI *__restrict__ r,
         const double *__restrict__ scale, T *y, int *flags, SweepState *st, int *err,
         long long limit, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;   // uniform over the grid
    __shared__ int s_base, s_epoch;
    sweep_begin(st, &s_base, &s_epoch);
    const int epoch = s_epoch;
    const int p = s_base + threadIdx.x;
    const int row = p < npad ? pos[p] : -1;
    if (row >= 0) {
        const double sc = scale ? *scale : 1.0;
        T acc[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) acc[k] = (T)(sc == 1.0 ? (double)r[(size_t)row * BS + k]
                                                            : (double)r[(size_t)row * BS + k] * sc);
        const int s = p >> 5, lane = p & 31;
        const int off = sptr[s];
        const int w = (sptr[s + 1] - off) >> 5;
        for (int e = 0; e < w; ++e) {
            const int idx = off + e * 32 + lane;
            const int c = ecol[idx];
            if (c < 0) continue;
            if (!wait_epoch(flags + c, epoch, limit)) report_timeout(err);
            T yc[BS];
#pragma unroll
            for (int k = 0; k < BS; ++k) yc[k] = __ldcg(y + (size_t)c * BS + k);
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int k = 0; k < BS; ++k) acc[i] -= val[(size_t)(i * BS + k) * nent + idx] * yc[k];
        }
#pragma unroll
        for (int k = 0; k < BS; ++k) y[(size_t)row * BS + k] = acc[k];
        st_release(flags + row, epoch);
    }
    sweep_end(st, epoch);
}

// U z = y.  z (type T) carries values between rows; out (FP64, optional)
// receives a widened copy.
template <int BS, typename T>
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_usolve(int npad, int64_t nent, const int *__restrict__ pos, const int *__restrict__ sptr,
         const int *__restrict__ ecol, const T *__restrict__ val, const T *__restrict__ diag,
         const T *__restrict__ y, T *z, double *__restrict__ out, int *flags, SweepState *st,
         int *err, long long limit, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;   // uniform over the grid
    __shared__ int s_base, s_epoch;
    sweep_begin(st, &s_base, &s_epoch);
    const int epoch = s_epoch;
    const int p = s_base + threadIdx.x;
    const int row = p < npad ? pos[p] : -1;
    if (row >= 0) {
        T acc[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) acc[k] = y[(size_t)row * BS + k];
        const int s = p >> 5, lane = p & 31;
        const int off = sptr[s];
        const int w = (sptr[s + 1] - off) >> 5;
        for (int e = 0; e < w; ++e) {
            const int idx = off + e * 32 + lane;
            const int c = ecol[idx];
            if (c < 0) continue;
            if (!wait_epoch(flags + c, epoch, limit)) report_timeout(err);
            T zc[BS];
#pragma unroll
            for (int k = 0; k < BS; ++k) zc[k] = __ldcg(z + (size_t)c * BS + k);
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int k = 0; k < BS; ++k) acc[i] -= val[(size_t)(i * BS + k) * nent + idx] * zc[k];
        }
        T res[BS];
        if (BS == 1) {
            res[0] = acc[0] / diag[p];
        } else {
#pragma unroll
            for (int i = 0; i < BS; ++i) {
                T sum = 0;
#pragma unroll
                for (int k = 0; k < BS; ++k) sum += diag[(size_t)(i * BS + k) * npad + p] * acc[k];
                res[i] = sum;
            }
        }
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            z[(size_t)row * BS + k] = res[k];
            if (out) out[(size_t)row * BS + k] = (double)res[k];
        }
        st_release(flags + row, epoch);
    }
    sweep_end(st, epoch);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int rs_ilu_create(rs_ctx *ctx, int bs, int nrows, int64_t nnzb, const int *d_ptr, const int *d_col,
                  const std::vector<int> &h_ptr, const std::vector<int> &h_col, int fp32,
                  IluFactor **out, int *bad_row)
{
    (void)bad_row;
    if (bs != 1 && bs != 2 && bs != 3 && bs != 4) return RS_ERR_INVALID_ARG;
    IluFactor *f = new IluFactor();
    f->ctx = ctx;
    f->bs = bs;
    f->nrows = nrows;
    f->nnzb = nnzb;
    f->fp32 = fp32;
    f->ptr = d_ptr;
    f->col = d_col;
    std::vector<int> diag(nrows, -1);
    for (int i = 0; i < nrows; ++i)
        for (int q = h_ptr[i]; q < h_ptr[i + 1]; ++q)
            if (h_col[q] == i) diag[i] = q;
    const size_t b2 = (size_t)bs * bs;
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    int st = build_layout(ctx, nrows, h_ptr, h_col, diag, true, f->L);
    st = st ? st : build_layout(ctx, nrows, h_ptr, h_col, diag, false, f->U);
    st = st ? st : rs_alloc(ctx, (void **)&f->diagpos, sizeof(int) * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->lu, sizeof(double) * b2 * (nnzb > 0 ? nnzb : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->dinv, sizeof(double) * b2 * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, &f->L.val, esz * b2 * (f->L.nent > 0 ? f->L.nent : 1));
    st = st ? st : rs_alloc(ctx, &f->U.val, esz * b2 * (f->U.nent > 0 ? f->U.nent : 1));
    st = st ? st : rs_alloc(ctx, &f->U.diag, esz * b2 * (f->U.npad > 0 ? f->U.npad : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->flags, sizeof(int) * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->state, sizeof(SweepState));
    st = st ? st : rs_alloc(ctx, &f->ywork, esz * bs * (nrows > 0 ? nrows : 1));
    if (!st && fp32) st = rs_alloc(ctx, &f->zwork, esz * bs * (nrows > 0 ? nrows : 1));
    if (st) { rs_ilu_destroy(f); return st; }
    SweepState s0 = {0u, 0u, 1, 0};
    RS_CUDA_TRY(cudaMemsetAsync(f->flags, 0, sizeof(int) * (nrows > 0 ? nrows : 1), ctx->stream));
    RS_CUDA_TRY(cudaMemcpyAsync(f->state, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->stream));
    RS_CUDA_TRY(cudaMemcpyAsync(f->diagpos, diag.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice,
                                ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = f;
    return RS_OK;
}

void rs_ilu_destroy(IluFactor *f)
{
    if (!f) return;
    rs_ctx *ctx = f->ctx;
    free_layout(ctx, f->L);
    free_layout(ctx, f->U);
    rs_free(ctx, f->diagpos);
    rs_free(ctx, f->lu);
    rs_free(ctx, f->dinv);
    rs_free(ctx, f->flags);
    rs_free(ctx, f->state);
    rs_free(ctx, f->ywork);
    rs_free(ctx, f->zwork);
    delete f;
}

static int sweep_grid(int npad) { return (npad + RS_SWEEP_THREADS - 1) / RS_SWEEP_THREADS; }

int rs_ilu_factor(IluFactor *f, const double *d_val, int *bad_row)
{
    rs_ctx *ctx = f->ctx;
    const size_t b2 = (size_t)f->bs * f->bs;
    if (bad_row) *bad_row = -1;
    if (f->nrows == 0) return RS_OK;
    RS_CUDA_TRY(cudaMemcpyAsync(f->lu, d_val, sizeof(double) * b2 * f->nnzb, cudaMemcpyDeviceToDevice,
                                ctx->stream));
    const int g = sweep_grid(f->L.npad);
    switch (f->bs) {
    case 1:
        k_ilu0_factor<<<g, RS_SWEEP_THREADS, 0, ctx->stream>>>(f->L.npad, f->L.pos, f->ptr, f->col,
                                                              f->diagpos, f->lu, f->flags, f->state,
                                                              ctx->d_err, ctx->d_bad_row, ctx->spin_limit);
        break;
#define RS_BF(BB)                                                                              \
    case BB:                                                                                   \
        k_bilu0_factor<BB><<<g, RS_SWEEP_THREADS, 0, ctx->stream>>>(                           \
            f->L.npad, f->L.pos, f->ptr, f->col, f->diagpos, f->lu, f->dinv, f->flags, f->state, \
            ctx->d_err, ctx->d_bad_row, ctx->spin_limit);                                      \
        break;
        RS_BF(2)
        RS_BF(3)
        RS_BF(4)
#undef RS_BF
    default: return RS_ERR_INVALID_ARG;
    }
    RS_TRY(rs_check_launch(ctx));
    const int ge = (int)std::min<int64_t>(std::max<int64_t>((f->L.nent + 255) / 256, 1), 4096);
    const int gu = (int)std::min<int64_t>(std::max<int64_t>((f->U.nent + 255) / 256, 1), 4096);
    const int gd = std::max(1, std::min((f->U.npad + 255) / 256, 4096));
    if (f->fp32) {
        k_gather_tri<float><<<ge, 256, 0, ctx->stream>>>(f->L.nent, (int)b2, f->L.src, f->lu, (float *)f->L.val);
        k_gather_tri<float><<<gu, 256, 0, ctx->stream>>>(f->U.nent, (int)b2, f->U.src, f->lu, (float *)f->U.val);
        k_gather_diag<float><<<gd, 256, 0, ctx->stream>>>(f->U.npad, (int)b2, f->U.pos, f->U.dsrc, f->lu,
                                                          f->dinv, (float *)f->U.diag);
    } else {
        k_gather_tri<double><<<ge, 256, 0, ctx->stream>>>(f->L.nent, (int)b2, f->L.src, f->lu, (double *)f->L.val);
        k_gather_tri<double><<<gu, 256, 0, ctx->stream>>>(f->U.nent, (int)b2, f->U.src, f->lu, (double *)f->U.val);
        k_gather_diag<double><<<gd, 256, 0, ctx->stream>>>(f->U.npad, (int)b2, f->U.pos, f->U.dsrc, f->lu,
                                                           f->dinv, (double *)f->U.diag);
    }
    RS_TRY(rs_check_launch(ctx));
    ctx->launches += 2;
    return rs_collect_device_error(ctx, bad_row);
}

template <int BS, typename T>
static int apply_typed(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    rs_ctx *ctx = f->ctx;
    T *y = (T *)f->ywork;
    k_lsolve<BS, T, double><<<sweep_grid(f->L.npad), RS_SWEEP_THREADS, 0, ctx->stream>>>(
        f->L.npad, f->L.nent, f->L.pos, f->L.slice_ptr, f->L.col, (const T *)f->L.val, r, scale, y,
        f->flags, f->state, ctx->d_err, ctx->spin_limit, skip);
    RS_TRY(rs_check_launch(ctx));
    T *zt = sizeof(T) == sizeof(double) ? (T *)z : (T *)f->zwork;
    double *out = sizeof(T) == sizeof(double) ? nullptr : z;
    k_usolve<BS, T><<<sweep_grid(f->U.npad), RS_SWEEP_THREADS, 0, ctx->stream>>>(
        f->U.npad, f->U.nent, f->U.pos, f->U.slice_ptr, f->U.col, (const T *)f->U.val,
        (const T *)f->U.diag, y, zt, out, f->flags, f->state, ctx->d_err, ctx->spin_limit, skip);
    return rs_check_launch(ctx);
}

int rs_ilu_apply(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    if (f->nrows == 0) return RS_OK;
    switch (f->bs) {
    case 1: return f->fp32 ? apply_typed<1, float>(f, r, z, scale, skip) : apply_typed<1, double>(f, r, z, scale, skip);
    case 2: return f->fp32 ? apply_typed<2, float>(f, r, z, scale, skip) : apply_typed<2, double>(f, r, z, scale, skip);
    case 3: return f->fp32 ? apply_typed<3, float>(f, r, z, scale, skip) : apply_typed<3, double>(f, r, z, scale, skip);
    case 4: return f->fp32 ? apply_typed<4, float>(f, r, z, scale, skip) : apply_typed<4, double>(f, r, z, scale, skip);
    default: return RS_ERR_INVALID_ARG;
    }
}
