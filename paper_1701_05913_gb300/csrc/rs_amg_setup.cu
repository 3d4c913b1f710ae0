// The AMG setup (Alg. 3) on the GPU, level by level:
//   1. strength: j strongly influences i when j != i and
//      -a_ij >= theta max_{k != i} (-a_ik), and its transpose;
//   2. C/F splitting by PMIS (De Sterck, Yang and Heys 2006, one of the
//      coarsenings Sec. 4.2 names): lambda_i = |S_i^T| + w_i with w_i from a
//      counter-based SplitMix64 keyed by (level, i); points that influence no
//      point are F; then in rounds every undecided point whose measure exceeds
//      that of every undecided point of S_i and S_i^T becomes C and every
//      undecided point that strongly depends on a C point becomes F;
//   3. direct interpolation (as in Sec. 4.2's classical AMG);
//   4. R = P^T;  5. A_{l+1} = R (A_l P) (Eq. 4);
// then the smoother's diagonal and the coarsest level's dense inverse.
//
// Arithmetic follows the definitions term by term in the same order as a
// sequential reading, each product and sum rounded once (no contraction):
// the strength, splitting and patterns are exact, and a Galerkin entry is the
// sum of its products in the order (row entry of the left factor, row entry
// of the right factor), so the coarse matrices come out bit for bit the same
// as a sequential row-by-row product.  Host work is sizes and allocation.
#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

namespace {

constexpr int SG_CAP = 2048;     // candidate terms of one row of a product
constexpr int SG_WARPS = 4;      // rows (warps) per block of the product

// ---------------------------------------------------------------------------
// exclusive prefix sums of int counts (out[n] = total)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int before = wid ? sh[wid - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(int n, const int *__restrict__ in, int *__restrict__ out,
                                                        int *__restrict__ bsum)
{
    __shared__ int sh[32];
    const int i = blockIdx.x * SCAN_T + threadIdx.x;
    int tot;
    const int e = block_excl_scan(i < n ? in[i] : 0, sh, &tot);
    if (i < n) out[i] = e;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: the block sums in place, exclusive; *total at the end
__global__ void __launch_bounds__(SCAN_T) k_scan_top(int nb, int *__restrict__ bsum, int *__restrict__ total)
{
    __shared__ int sh[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int i = b0 + threadIdx.x;
        int tot;
        const int v = i < nb ? bsum[i] : 0;
        const int e = block_excl_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(int n, int *__restrict__ out, const int *__restrict__ bsum,
                                                     const int *__restrict__ total)
{
    const int i = blockIdx.x * SCAN_T + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
    if (i == 0) out[n] = *total;
}

// ---------------------------------------------------------------------------
// 1. strength and its transpose
// ---------------------------------------------------------------------------
// count pass (sptr == nullptr): cnt[i] = |S_i|; fill pass: scol
__global__ void k_strength(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                           const double *__restrict__ val, double theta, const int *__restrict__ sptr,
                           int *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double mx = 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p)
            if (col[p] != i && -val[p] > mx) mx = -val[p];
        int k = sptr ? sptr[i] : 0;
        if (mx > 0.0) {
            const double th = __dmul_rn(theta, mx);
            for (int p = ptr[i]; p < ptr[i + 1]; ++p)
                if (col[p] != i && -val[p] >= th) {
                    if (sptr) out[k] = col[p];
                    ++k;
                }
        }
        if (!sptr) out[i] = k;
    }
}

__global__ void k_count_cols(int64_t nnz, const int *__restrict__ col, int *__restrict__ cnt)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1);
}

// transpose fill: entries land at an atomic slot of their column; values
// optional; rows of the transpose are sorted afterwards where order matters
__global__ void k_transpose_fill(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                                 const double *__restrict__ val, int *__restrict__ fill, int *__restrict__ tcol,
                                 double *__restrict__ tval)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int q = atomicAdd(&fill[col[p]], 1);
            tcol[q] = i;
            if (tval) tval[q] = val[p];
        }
}

// insertion sort of every row by column (rows of a transpose are short)
__global__ void k_sort_rows(int n, const int *__restrict__ ptr, int *__restrict__ col, double *__restrict__ val)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = ptr[i], e = ptr[i + 1];
        for (int a = s + 1; a < e; ++a) {
            const int c = col[a];
            const double v = val ? val[a] : 0.0;
            int b = a - 1;
            while (b >= s && col[b] > c) {
                col[b + 1] = col[b];
                if (val) val[b + 1] = val[b];
                --b;
            }
            col[b + 1] = c;
            if (val) val[b + 1] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// 2. PMIS
// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood 2014), counter-based: the k-th output of
// the generator started from state 0
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long k)
{
    unsigned long long z = (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_pmis_init(int n, const int *__restrict__ tptr, int level, double *__restrict__ lam,
                            char *__restrict__ st, int *__restrict__ und)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = tptr[i + 1] - tptr[i];
        const unsigned long long k = ((unsigned long long)(unsigned)level << 32) | (unsigned)i;
        const double w = (double)(splitmix64(k) >> 11) * 0x1.0p-53;
        lam[i] = __dadd_rn((double)t, w);
        st[i] = t == 0 ? 2 : 0;
        if (t != 0) atomicAdd(und, 1);
    }
}

// undecided points that are the strict maximum of their undecided
// neighbourhood (states of the round's start: old) become C
__global__ void k_pmis_select(int n, const int *__restrict__ sptr, const int *__restrict__ scol,
                              const int *__restrict__ tptr, const int *__restrict__ tcol,
                              const double *__restrict__ lam, const char *__restrict__ old, char *__restrict__ st)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (old[i] != 0) continue;
        const double li = lam[i];
        bool top = true;
        for (int q = sptr[i]; q < sptr[i + 1] && top; ++q)
            if (old[scol[q]] == 0 && !(li > lam[scol[q]])) top = false;
        for (int q = tptr[i]; q < tptr[i + 1] && top; ++q)
            if (old[tcol[q]] == 0 && !(li > lam[tcol[q]])) top = false;
        if (top) st[i] = 1;
    }
}

// undecided points that depend strongly on a C point become F; count the rest
__global__ void k_pmis_f(int n, const int *__restrict__ sptr, const int *__restrict__ scol, char *__restrict__ st,
                         int *__restrict__ und)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (st[j] != 0) continue;
        bool f = false;
        for (int q = sptr[j]; q < sptr[j + 1] && !f; ++q) f = st[scol[q]] == 1;
        if (f) st[j] = 2;
        else atomicAdd(und, 1);
    }
}

__global__ void k_cflag(int n, const char *__restrict__ st, int *__restrict__ flag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flag[i] = st[i] == 1;
}

__global__ void k_cidx(int n, const char *__restrict__ st, const int *__restrict__ scan, int *__restrict__ cidx)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cidx[i] = st[i] == 1 ? scan[i] : -1;
}

// ---------------------------------------------------------------------------
// 3. direct interpolation: C points inject; an F point interpolates from
// its strong C neighbours k with w_ik = -alpha a_ik / d (a_ik < 0) or
// -beta a_ik / d (a_ik > 0), alpha (beta) = the row's sum of negative
// (positive) off-diagonal entries over that of its strong C neighbours,
// d = a_ii, plus the positive couplings when no strong C coupling is positive
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_row(const int *__restrict__ sc, int s, int e, int k)
{
    for (int r = s; r < e; ++r)
        if (sc[r] == k) return true;
    return false;
}

// count pass (pptr == nullptr): cnt[i]; fill pass: pcol, pval
__global__ void k_interp(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                         const double *__restrict__ val, const int *__restrict__ sptr, const int *__restrict__ scol,
                         const int *__restrict__ cidx, const int *__restrict__ pptr, int *__restrict__ out,
                         double *__restrict__ pval)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (cidx[i] >= 0) {
            if (pptr) {
                out[pptr[i]] = cidx[i];
                pval[pptr[i]] = 1.0;
            } else {
                out[i] = 1;
            }
            continue;
        }
        const int s0 = sptr[i], s1 = sptr[i + 1];
        if (!pptr) {
            int k = 0;
            for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
                const int c = col[p];
                if (c != i && cidx[c] >= 0 && in_row(scol, s0, s1, c)) ++k;
            }
            out[i] = k;
            continue;
        }
        double aii = 0.0, neg = 0.0, pos = 0.0, negc = 0.0, posc = 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const double v = val[p];
            if (col[p] == i) aii = v;
            else if (v < 0.0) neg = __dadd_rn(neg, v);
            else pos = __dadd_rn(pos, v);
        }
        // the strong C neighbours' couplings, in column order
        for (int r = s0; r < s1; ++r) {
            const int c = scol[r];
            if (cidx[c] < 0) continue;
            for (int p = ptr[i]; p < ptr[i + 1]; ++p)
                if (col[p] == c) {
                    if (val[p] < 0.0) negc = __dadd_rn(negc, val[p]);
                    else posc = __dadd_rn(posc, val[p]);
                }
        }
        double diag = aii, beta = 0.0;
        if (posc == 0.0) diag = __dadd_rn(diag, pos);
        else beta = __ddiv_rn(pos, posc);
        const double alpha = negc != 0.0 ? __ddiv_rn(neg, negc) : 0.0;
        int k = pptr[i];
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int c = col[p];
            if (c == i || cidx[c] < 0 || !in_row(scol, s0, s1, c)) continue;
            out[k] = cidx[c];
            pval[k] = __ddiv_rn(__dmul_rn(-(val[p] < 0.0 ? alpha : beta), val[p]), diag);
            ++k;
        }
    }
}

// ---------------------------------------------------------------------------
// 5. sparse products C = A B, a warp per row.  The row's candidate terms
// (entry p of A's row, entry q of B's row p), numbered in that order, are
// sorted by (column, number); a column's terms are then summed in number
// order.  Count pass (cptr == nullptr): the distinct columns; fill pass:
// columns and sums.  A row with more than SG_CAP terms sets *err.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void __launch_bounds__(32 * SG_WARPS)
k_spgemm(int n, const int *__restrict__ aptr, const int *__restrict__ acol, const double *__restrict__ aval,
         const int *__restrict__ bptr, const int *__restrict__ bcol, const double *__restrict__ bval,
         const int *__restrict__ cptr, int *__restrict__ out, double *__restrict__ cval, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char sg_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *key = (unsigned long long *)sg_smem + (size_t)wid * SG_CAP;
    double *tv = (double *)(sg_smem + (size_t)SG_WARPS * SG_CAP * sizeof(unsigned long long)) + (size_t)wid * SG_CAP;
    const int stride = gridDim.x * SG_WARPS;
    for (int i = blockIdx.x * SG_WARPS + wid; i < n; i += stride) {
        // the row's terms
        int len = 0;
        for (int p = aptr[i]; p < aptr[i + 1]; ++p) len += bptr[acol[p] + 1] - bptr[acol[p]];
        if (len > SG_CAP) {
            if (lane == 0) {
                atomicOr(err, 1);
                if (!FILL) out[i] = 0;
            }
            continue;
        }
        int base = 0;
        for (int p = aptr[i]; p < aptr[i + 1]; ++p) {
            const int j = acol[p];
            const double a = aval[p];
            const int q0 = bptr[j], m = bptr[j + 1] - q0;
            for (int q = lane; q < m; q += 32) {
                const int t = base + q;
                key[t] = ((unsigned long long)(unsigned)bcol[q0 + q] << 32) | (unsigned)t;
                if (FILL) tv[t] = __dmul_rn(a, bval[q0 + q]);
            }
            base += m;
        }
        int sz = 1;
        while (sz < len) sz <<= 1;
        for (int t = len + lane; t < sz; t += 32) key[t] = ~0ull;
        __syncwarp();
        // bitonic sort of (key, term) over sz entries
        for (int k = 2; k <= sz; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < sz; t += 32) {
                    const int u = t ^ j;
                    if (u > t) {
                        const bool up = (t & k) == 0;
                        const unsigned long long kt = key[t], ku = key[u];
                        if ((kt > ku) == up) {
                            key[t] = ku;
                            key[u] = kt;
                            if (FILL) {
                                const double x = tv[t];
                                tv[t] = tv[u];
                                tv[u] = x;
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        // distinct columns: the first term of each column starts a segment
        int nseg = 0;
        const int o0 = FILL ? cptr[i] : 0;
        for (int t0 = 0; t0 < len; t0 += 32) {
            const int t = t0 + lane;
            const bool first = t < len && (t == 0 || (key[t] >> 32) != (key[t - 1] >> 32));
            const unsigned m = __ballot_sync(0xffffffffu, first);
            if (FILL && first) {
                const int o = o0 + nseg + __popc(m & ((1u << lane) - 1));
                const unsigned c = (unsigned)(key[t] >> 32);
                double s = 0.0;
                for (int e = t; e < len && (unsigned)(key[e] >> 32) == c; ++e) s = __dadd_rn(s, tv[e]);
                out[o] = (int)c;
                cval[o] = s;
            }
            nseg += __popc(m);
        }
        if (!FILL && lane == 0) out[i] = nseg;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// smoother diagonal, zero-diagonal check, coarsest dense inverse
// ---------------------------------------------------------------------------
// dinv_i = 1 / sum_j |a_ij|; *bad |= 1 when a diagonal entry is 0 (needed by
// hybrid Gauss-Seidel)
__global__ void k_amg_l1(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                         const double *__restrict__ val, double *__restrict__ dinv, int *__restrict__ bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0, dg = 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            s = __dadd_rn(s, fabs(val[p]));
            if (col[p] == i) dg = val[p];
        }
        dinv[i] = __ddiv_rn(1.0, s);
        if (dg == 0.0) atomicOr(bad, 1);
    }
}

// the coarsest matrix into [A | I] (n x 2n, row-major)
__global__ void k_dense_aug(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                            const double *__restrict__ val, double *__restrict__ m)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * 2 * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / (2 * n)), c = (int)(e - (int64_t)r * 2 * n);
        m[e] = c >= n ? (c - n == r ? 1.0 : 0.0) : 0.0;
    }
}
__global__ void k_dense_scatter(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                                const double *__restrict__ val, double *__restrict__ m)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) m[(size_t)i * 2 * n + col[p]] = val[p];
}

// Gauss-Jordan with partial pivoting, column c: one block finds the pivot
// (largest |m_rc|, r >= c, lowest row on ties), swaps it into row c and
// divides row c by it; *bad |= 1 on a zero or non-finite pivot
__global__ void __launch_bounds__(256) k_gj_pivot(int n, int c, double *__restrict__ m, int *__restrict__ bad)
{
    __shared__ double bv[256];
    __shared__ int br[256];
    const int w = 2 * n;
    double best = -1.0;
    int row = c;
    for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
        const double a = fabs(m[(size_t)r * w + c]);
        if (a > best) {
            best = a;
            row = r;
        }
    }
    bv[threadIdx.x] = best;
    br[threadIdx.x] = row;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = bv[threadIdx.x + s];
            const int orow = br[threadIdx.x + s];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && orow < br[threadIdx.x])) {
                bv[threadIdx.x] = o;
                br[threadIdx.x] = orow;
            }
        }
        __syncthreads();
    }
    const int p = br[0];
    const double piv = m[(size_t)p * w + c];
    __syncthreads();         // every thread has the pivot before row p changes
    if (!(piv != 0.0) || !isfinite(piv)) {
        if (threadIdx.x == 0) atomicOr(bad, 1);
        return;
    }
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double a = m[(size_t)p * w + j], b = m[(size_t)c * w + j];
        m[(size_t)c * w + j] = __ddiv_rn(a, piv);
        if (p != c) m[(size_t)p * w + j] = b;
    }
}

// rows r != c: m_r -= m_rc m_c (m_rc read before the row changes)
__global__ void k_gj_elim(int n, int c, double *__restrict__ m, const int *__restrict__ bad)
{
    if (*bad) return;
    const int w = 2 * n;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        if (r == c) continue;
        const double f = m[(size_t)r * w + c];
        __syncthreads();
        if (f != 0.0)
            for (int j = threadIdx.x; j < w; j += blockDim.x)
                m[(size_t)r * w + j] = __dsub_rn(m[(size_t)r * w + j], __dmul_rn(f, m[(size_t)c * w + j]));
        __syncthreads();
    }
}

// the right half of [I | inv] into inv (n x n)
__global__ void k_dense_take(int n, const double *__restrict__ m, double *__restrict__ inv)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
        inv[e] = m[(size_t)r * 2 * n + n + c];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Dev {
    rs_ctx *ctx;
    std::vector<void *> tmp;
    explicit Dev(rs_ctx *c) : ctx(c) {}
    ~Dev()
    {
        for (void *p : tmp) rs_free(ctx, p);
    }
    template <typename T>
    int alloc(T **p, size_t count)
    {
        *p = nullptr;
        int st = rs_alloc(ctx, (void **)p, sizeof(T) * std::max<size_t>(count, 1));
        if (!st) tmp.push_back(*p);
        return st;
    }
};

int grid_for(rs_ctx *ctx, int64_t n, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)ctx->num_sms * 8));
}

// exclusive scan of n counts into out[0..n]; *total on the host
int scan(rs_ctx *ctx, Dev &D, const int *in, int *out, int n, int *total)
{
    const int nb = std::max(1, (n + SCAN_T - 1) / SCAN_T);
    int *bsum, *dt;
    RS_TRY(D.alloc(&bsum, nb));
    RS_TRY(D.alloc(&dt, 1));
    k_scan_blocks<<<nb, SCAN_T, 0, ctx->stream>>>(n, in, out, bsum);
    k_scan_top<<<1, SCAN_T, 0, ctx->stream>>>(nb, bsum, dt);
    k_scan_add<<<nb, SCAN_T, 0, ctx->stream>>>(n, out, bsum, dt);
    ctx->launches += 2;
    RS_TRY(rs_check_launch(ctx));
    RS_CUDA_TRY(cudaMemcpyAsync(total, dt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return RS_OK;
}

int read_flag(rs_ctx *ctx, const int *d, int *h)
{
    RS_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return RS_OK;
}

// transpose (values optional) with sorted rows
int transpose(rs_ctx *ctx, Dev &D, int n, int m, int64_t nnz, const int *ptr, const int *col, const double *val,
              int **tptr, int **tcol, double **tval)
{
    int *cnt, *fill, tot = 0;
    RS_TRY(D.alloc(&cnt, m));
    RS_TRY(D.alloc(tptr, m + 1));
    RS_TRY(D.alloc(tcol, nnz));
    if (tval) RS_TRY(D.alloc(tval, nnz));
    RS_TRY(D.alloc(&fill, m));
    RS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max(m, 1), ctx->stream));
    k_count_cols<<<grid_for(ctx, nnz, 256), 256, 0, ctx->stream>>>(nnz, col, cnt);
    RS_TRY(rs_check_launch(ctx));
    RS_TRY(scan(ctx, D, cnt, *tptr, m, &tot));
    RS_CUDA_TRY(cudaMemcpyAsync(fill, *tptr, sizeof(int) * std::max(m, 1), cudaMemcpyDeviceToDevice, ctx->stream));
    k_transpose_fill<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(n, ptr, col, val, fill, *tcol,
                                                                     tval ? *tval : nullptr);
    k_sort_rows<<<grid_for(ctx, m, 128), 128, 0, ctx->stream>>>(m, *tptr, *tcol, tval ? *tval : nullptr);
    ctx->launches += 1;
    return rs_check_launch(ctx);
}

// C = A B (n x k by k x m) into freshly allocated device arrays
int spgemm(rs_ctx *ctx, Dev &D, int n, const int *aptr, const int *acol, const double *aval, const int *bptr,
           const int *bcol, const double *bval, int **cptr, int **ccol, double **cval, int64_t *cnnz)
{
    int *cnt, *err, tot = 0, herr = 0;
    RS_TRY(D.alloc(&cnt, n));
    RS_TRY(D.alloc(cptr, n + 1));
    RS_TRY(D.alloc(&err, 1));
    RS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    const size_t smem = (size_t)SG_WARPS * SG_CAP * (sizeof(unsigned long long) + sizeof(double));
    static unsigned long long raised = 0;      // one bit per device
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(raised & bit)) {
        RS_CUDA_TRY(cudaFuncSetAttribute(k_spgemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RS_CUDA_TRY(cudaFuncSetAttribute(k_spgemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        raised |= bit;
    }
    const int gb = std::max(1, std::min((n + SG_WARPS - 1) / SG_WARPS, ctx->num_sms * 2));
    k_spgemm<false><<<gb, 32 * SG_WARPS, smem, ctx->stream>>>(n, aptr, acol, aval, bptr, bcol, bval, nullptr, cnt,
                                                               nullptr, err);
    RS_TRY(rs_check_launch(ctx));
    RS_TRY(read_flag(ctx, err, &herr));
    if (herr) return RS_ERR_INVALID_ARG;     // a row of the product has more than SG_CAP terms
    RS_TRY(scan(ctx, D, cnt, *cptr, n, &tot));
    *cnnz = tot;
    RS_TRY(D.alloc(ccol, tot));
    RS_TRY(D.alloc(cval, tot));
    k_spgemm<true><<<gb, 32 * SG_WARPS, smem, ctx->stream>>>(n, aptr, acol, aval, bptr, bcol, bval, *cptr, *ccol,
                                                              *cval, err);
    return rs_check_launch(ctx);
}

}  // namespace

// The hierarchy of Alg. 3 on the device: M->A[0] is given; builds M->P, M->R,
// M->A[1..], M->cidx, M->d and the coarsest inverse M->cinv; sets M->nlev.
int rs_amg_setup_device(AmgData *M, double theta, int max_levels, int max_coarse)
{
    rs_ctx *ctx = M->ctx;
    int l = 0;
    for (;; ++l) {
        const rs_mat *A = M->A[l];
        const int n = A->n;
        if (n <= max_coarse || l + 1 >= max_levels) break;
        Dev D(ctx);
        const int g = grid_for(ctx, n, 128);
        // 1. strength S and its transpose
        int *scnt, *sptr, *scol, *tptr, *tcol, ns = 0;
        RS_TRY(D.alloc(&scnt, n));
        RS_TRY(D.alloc(&sptr, n + 1));
        k_strength<<<g, 128, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, theta, nullptr, scnt);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(scan(ctx, D, scnt, sptr, n, &ns));
        RS_TRY(D.alloc(&scol, ns));
        k_strength<<<g, 128, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, theta, sptr, scol);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(transpose(ctx, D, n, n, ns, sptr, scol, nullptr, &tptr, &tcol, nullptr));
        // 2. PMIS
        double *lam;
        char *st, *old;
        int *und, *flag, *cscan, *cidx, hund = 0, nc = 0;
        RS_TRY(D.alloc(&lam, n));
        RS_TRY(D.alloc(&st, n));
        RS_TRY(D.alloc(&old, n));
        RS_TRY(D.alloc(&und, 1));
        RS_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(int), ctx->stream));
        k_pmis_init<<<g, 128, 0, ctx->stream>>>(n, tptr, l, lam, st, und);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(read_flag(ctx, und, &hund));
        for (int round = 0; hund > 0; ++round) {
            if (round > n) return RS_ERR_INVALID_ARG;          // cannot happen: every round decides a point
            RS_CUDA_TRY(cudaMemcpyAsync(old, st, n, cudaMemcpyDeviceToDevice, ctx->stream));
            RS_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(int), ctx->stream));
            k_pmis_select<<<g, 128, 0, ctx->stream>>>(n, sptr, scol, tptr, tcol, lam, old, st);
            k_pmis_f<<<g, 128, 0, ctx->stream>>>(n, sptr, scol, st, und);
            ctx->launches += 1;
            RS_TRY(rs_check_launch(ctx));
            RS_TRY(read_flag(ctx, und, &hund));
        }
        RS_TRY(D.alloc(&flag, n));
        RS_TRY(D.alloc(&cscan, n + 1));
        k_cflag<<<g, 128, 0, ctx->stream>>>(n, st, flag);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(scan(ctx, D, flag, cscan, n, &nc));
        if (nc == 0 || nc >= n) break;
        RS_TRY(rs_alloc(ctx, (void **)&cidx, sizeof(int) * n));
        M->cidx[l] = cidx;
        k_cidx<<<g, 128, 0, ctx->stream>>>(n, st, cscan, cidx);
        RS_TRY(rs_check_launch(ctx));
        // 3. direct interpolation P (n x nc)
        int *pcnt, *pptr, *pcol, np = 0;
        double *pval;
        RS_TRY(D.alloc(&pcnt, n));
        RS_TRY(D.alloc(&pptr, n + 1));
        k_interp<<<g, 128, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, sptr, scol, cidx, nullptr, pcnt, nullptr);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(scan(ctx, D, pcnt, pptr, n, &np));
        RS_TRY(D.alloc(&pcol, np));
        RS_TRY(D.alloc(&pval, np));
        k_interp<<<g, 128, 0, ctx->stream>>>(n, A->ptr, A->col, A->val, sptr, scol, cidx, pptr, pcol, pval);
        RS_TRY(rs_check_launch(ctx));
        // 4. R = P^T (nc x n)
        int *rptr, *rcol;
        double *rval;
        RS_TRY(transpose(ctx, D, n, nc, np, pptr, pcol, pval, &rptr, &rcol, &rval));
        // 5. A_{l+1} = R (A P)
        int *xptr, *xcol, *cptr, *ccol;
        double *xval, *cval;
        int64_t nx = 0, ncn = 0;
        RS_TRY(spgemm(ctx, D, n, A->ptr, A->col, A->val, pptr, pcol, pval, &xptr, &xcol, &xval, &nx));
        RS_TRY(spgemm(ctx, D, nc, rptr, rcol, rval, xptr, xcol, xval, &cptr, &ccol, &cval, &ncn));
        RS_TRY(rs_mat_create_rect_dev(ctx, n, nc, pptr, pcol, pval, &M->P[l]));
        RS_TRY(rs_mat_create_rect_dev(ctx, nc, n, rptr, rcol, rval, &M->R[l]));
        RS_TRY(rs_mat_create_rect_dev(ctx, nc, -1, cptr, ccol, cval, &M->A[l + 1]));
    }
    M->nlev = l + 1;
    const int ncoarse = M->A[l]->n;
    if (ncoarse > RS_AMG_MAX_DENSE) return RS_ERR_INVALID_ARG;   // coarsening stalled: no small coarsest level
    // smoother diagonals, the zero-diagonal check of hybrid Gauss-Seidel
    Dev D(ctx);
    int *bad, hbad = 0;
    RS_TRY(D.alloc(&bad, 1));
    for (int k = 0; k < M->nlev; ++k) {
        const rs_mat *A = M->A[k];
        RS_TRY(rs_alloc(ctx, (void **)&M->d[k], sizeof(double) * A->n));
        RS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
        k_amg_l1<<<grid_for(ctx, A->n, 128), 128, 0, ctx->stream>>>(A->n, A->ptr, A->col, A->val, M->d[k], bad);
        RS_TRY(rs_check_launch(ctx));
        RS_TRY(read_flag(ctx, bad, &hbad));
        if (hbad && M->smoother == 1 && k + 1 < M->nlev) return RS_ERR_ZERO_PIVOT;
    }
    // the coarsest matrix's dense inverse
    double *aug;
    RS_TRY(D.alloc(&aug, (size_t)ncoarse * 2 * ncoarse));
    RS_TRY(rs_alloc(ctx, (void **)&M->cinv, sizeof(double) * (size_t)ncoarse * ncoarse));
    const rs_mat *Cm = M->A[l];
    RS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    k_dense_aug<<<grid_for(ctx, (int64_t)ncoarse * 2 * ncoarse, 256), 256, 0, ctx->stream>>>(ncoarse, Cm->ptr,
                                                                                          Cm->col, Cm->val, aug);
    k_dense_scatter<<<grid_for(ctx, ncoarse, 128), 128, 0, ctx->stream>>>(ncoarse, Cm->ptr, Cm->col, Cm->val, aug);
    ctx->launches += 1;
    RS_TRY(rs_check_launch(ctx));
    const int ge = std::max(1, std::min(ncoarse, ctx->num_sms * 4));
    for (int c = 0; c < ncoarse; ++c) {
        k_gj_pivot<<<1, 256, 0, ctx->stream>>>(ncoarse, c, aug, bad);
        k_gj_elim<<<ge, 256, 0, ctx->stream>>>(ncoarse, c, aug, bad);
        ctx->launches += 1;
    }
    RS_TRY(rs_check_launch(ctx));
    RS_TRY(read_flag(ctx, bad, &hbad));
    if (hbad) return RS_ERR_ZERO_PIVOT;
    k_dense_take<<<grid_for(ctx, (int64_t)ncoarse * ncoarse, 256), 256, 0, ctx->stream>>>(ncoarse, aug, M->cinv);
    RS_TRY(rs_check_launch(ctx));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return RS_OK;
}
