// Restricted additive Schwarz on one GPU (Sec. 4.1, after Cai and Sarkis).
//
// The (block) rows are split into subdomains by a partition; subdomain s is
// extended by `overlap` layers of the graph of A (the next layer is the set
// of columns of the rows of the current one).  The local matrices A_s (the
// entries of A whose row and column both lie in the extended set, rows in
// ascending global order) are stacked, subdomain after subdomain, into one
// block-diagonal matrix.  Its factor is ILU(level) of every block: ILU(0) on
// the level-of-fill pattern, with zeros at the new positions.  The factor
// and its triangular sweeps are the ones of rs_ilu.cu.  No block reads
// another, so the sweeps' dependency chains are those of a single
// subdomain and all subdomains advance together: the parallelism the paper
// gets from RAS across processes comes here from the warps of one GPU.
//
// Apply:  r_hat = r gathered to the stacked rows;  z_hat = (L U)^{-1} r_hat;
//         z_i = z_hat[own(i)], the copy of row i in the subdomain that owns
//         it (the restricted prolongation).
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "rs_internal.cuh"

// values of the stacked matrix: the entry src[q] of A, or zero at fill
__global__ void k_ras_values(int64_t nnz, int b2, const int *__restrict__ src, const double *__restrict__ a,
                             double *__restrict__ v)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz * b2;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / b2;
        const int s = src[q];
        v[e] = s >= 0 ? a[(int64_t)s * b2 + (e - q * b2)] : 0.0;
    }
}

// r_hat[j] = r[gidx[j]] (bs values per block row)
__global__ void k_ras_gather(int next, int bs, const int *__restrict__ gidx, const double *__restrict__ r,
                             double *__restrict__ rh, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)next * bs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / bs;
        rh[e] = r[(int64_t)gidx[j] * bs + (e - j * bs)];
    }
}

// z[i] = z_hat[own[i]]
__global__ void k_ras_scatter(int nrows, int bs, const int *__restrict__ own, const double *__restrict__ zh,
                              double *__restrict__ z, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nrows * bs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / bs;
        z[e] = zh[(int64_t)own[i] * bs + (e - i * bs)];
    }
}

static int ras_grid(rs_ctx *ctx, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

// Level-of-fill pattern of one local matrix (rows 0..n-1, sorted columns):
// entries of the matrix have level 0; pivot row k turns (i, j), j > k, into
// an entry of level lev(i,k) + lev(k,j) + 1 (the smallest such level is
// kept); entries of level <= p stay.  Appends the rows to (optr, ocol, osrc)
// with osrc = the entry's index in A for original entries, -1 for fill.
static void iluk_rows(int n, const std::vector<int> &lptr, const std::vector<int> &lcol, const std::vector<int> &lsrc,
                      int p, int base, std::vector<int> &optr, std::vector<int> &ocol, std::vector<int> &osrc)
{
    std::vector<int> rowstart(n + 1);          // kept pattern of the local rows, for later pivots
    std::vector<int> kcol, klev;
    std::vector<int> lev(n, -1), srcof(n, -1);
    std::vector<int> cols;
    for (int i = 0; i < n; ++i) {
        cols.assign(lcol.begin() + lptr[i], lcol.begin() + lptr[i + 1]);
        for (int q = lptr[i]; q < lptr[i + 1]; ++q) {
            lev[lcol[q]] = 0;
            srcof[lcol[q]] = lsrc[q];
        }
        for (size_t t = 0; t < cols.size() && cols[t] < i; ++t) {
            const int k = cols[t];
            for (int q = rowstart[k]; q < rowstart[k + 1]; ++q) {
                const int j = kcol[q];
                if (j <= k) continue;
                const int l = lev[k] + klev[q] + 1;
                if (l > p) continue;
                if (lev[j] >= 0) {
                    lev[j] = std::min(lev[j], l);
                } else {
                    lev[j] = l;
                    srcof[j] = -1;
                    cols.insert(std::lower_bound(cols.begin() + t + 1, cols.end(), j), j);
                }
            }
        }
        rowstart[i] = (int)kcol.size();
        for (int c : cols) {
            kcol.push_back(c);
            klev.push_back(lev[c]);
            ocol.push_back(base + c);
            osrc.push_back(srcof[c]);
            lev[c] = -1;
            srcof[c] = -1;
        }
        rowstart[i + 1] = (int)kcol.size();
        optr.push_back((int)ocol.size());
    }
}

// ILUT(p, tol) of the stacked local matrices on the GPU, one thread per
// subdomain (the subdomains are independent; a subdomain's rows depend on
// each other, in order), Saad's algorithm row by row as the sequential
// reading has it: the row in a dense work array w; its lower entries
// eliminated in ascending order, fill included, each multiplier
// w_k = w_k / u_kk dropped below tau = tol ||a_i||_2, else
// w_j -= w_k u_kj over the stored U row k; then off-diagonal entries below
// tau dropped and the p largest kept in each part (ties to the lower
// column; p < 0: as many as row i has there).  Every product and sum is
// rounded once, in the sequential order, so the dropping decisions (and the
// pattern) are those of a sequential run.
//
// Subdomain s owns stacked rows [sb[s], sb[s+1]) and, in the scratch arrays
// indexed by stacked row, its w, flags and lists; its factor rows go to
// [cap[s], cap[s+1]) of ocol/oval, row r at [rs[r], re[r]) with its diagonal
// at rd[r].  st[s]: -1 done, >= 0 the local row of a zero pivot, -2 the
// output region overflowed.
__device__ __forceinline__ bool ilut_larger(int ca, double va, int cb, double vb)
{
    const double x = fabs(va), y = fabs(vb);
    return x != y ? x > y : ca < cb;
}

__global__ void k_ilut(int nparts, const int *__restrict__ sb, const int *__restrict__ lptr,
                       const int *__restrict__ lcol, const double *__restrict__ lval, int p, double tol,
                       const int64_t *__restrict__ cap, int *__restrict__ ocol, double *__restrict__ oval,
                       int64_t *__restrict__ rs_, int64_t *__restrict__ rd, int64_t *__restrict__ re,
                       double *__restrict__ w_, char *__restrict__ in_, int *__restrict__ touched_,
                       int *__restrict__ lower_, int *__restrict__ cc_, double *__restrict__ cv_, int *__restrict__ st)
{
    // one subdomain per warp, on its first lane: the rows are sequential and
    // the subdomains' control flow diverges, so a warp each keeps them apart
    const int s = blockIdx.x;
    if (s >= nparts || threadIdx.x != 0) return;
    const int b0 = sb[s], n = sb[s + 1] - b0;
    double *w = w_ + b0;
    char *in = in_ + b0;
    int *touched = touched_ + b0, *lower = lower_ + b0, *cc = cc_ + b0;
    double *cv = cv_ + b0;
    int64_t o = cap[s];
    const int64_t oend = cap[s + 1];
    for (int i = 0; i < n; ++i) {
        const int r = b0 + i;
        int nt = 0, nlow = 0, pl = 0, pu = 0;
        double sq = 0.0;
        for (int q = lptr[r]; q < lptr[r + 1]; ++q) {
            const int c = lcol[q];
            w[c] = lval[q];
            in[c] = 1;
            touched[nt++] = c;
            sq = __dadd_rn(sq, __dmul_rn(lval[q], lval[q]));
            if (c < i) {
                ++pl;
                lower[nlow++] = c;
            } else if (c > i) {
                ++pu;
            }
        }
        const double tau = __dmul_rn(tol, __dsqrt_rn(sq));
        if (p >= 0) pl = pu = p;
        for (int t = 0; t < nlow; ++t) {
            const int k = lower[t];
            if (w[k] == 0.0) continue;
            w[k] = __ddiv_rn(w[k], oval[rd[b0 + k]]);
            if (fabs(w[k]) < tau) {
                w[k] = 0.0;
                continue;
            }
            const double wk = w[k];
            for (int64_t q = rd[b0 + k] + 1; q < re[b0 + k]; ++q) {
                const int j = ocol[q];
                if (!in[j]) {
                    in[j] = 1;
                    w[j] = 0.0;
                    touched[nt++] = j;
                    if (j < i) {            // a new lower entry, in sorted position behind t
                        int a = nlow++;
                        while (a > t + 1 && lower[a - 1] > j) {
                            lower[a] = lower[a - 1];
                            --a;
                        }
                        lower[a] = j;
                    }
                }
                w[j] = __dsub_rn(w[j], __dmul_rn(wk, oval[q]));
            }
        }
        // the surviving off-diagonal entries: lower ones at the front of the
        // candidate buffer, upper ones at its back
        int nl = 0, nu = 0;
        double diag = 0.0;
        for (int a = 0; a < nt; ++a) {
            const int c = touched[a];
            if (c == i) {
                diag = w[c];
            } else if (w[c] != 0.0 && fabs(w[c]) >= tau) {
                const int at = c < i ? nl++ : n - 1 - nu++;
                cc[at] = c;
                cv[at] = w[c];
            }
            w[c] = 0.0;
            in[c] = 0;
        }
        if (!(diag != 0.0) || !isfinite(diag)) {
            st[s] = i;
            return;
        }
        // each part: the p largest (insertion sort by magnitude), then by column
        const int ulo = n - nu;                 // first upper candidate
        for (int part = 0; part < 2; ++part) {
            const int lo = part ? ulo : 0, len = part ? nu : nl, lim = part ? pu : pl;
            for (int a = lo + 1; a < lo + len; ++a) {
                const int c = cc[a];
                const double v = cv[a];
                int b = a - 1;
                while (b >= lo && ilut_larger(c, v, cc[b], cv[b])) {
                    cc[b + 1] = cc[b];
                    cv[b + 1] = cv[b];
                    --b;
                }
                cc[b + 1] = c;
                cv[b + 1] = v;
            }
            const int keep = len < lim ? len : lim;
            for (int a = lo + 1; a < lo + keep; ++a) {
                const int c = cc[a];
                const double v = cv[a];
                int b = a - 1;
                while (b >= lo && cc[b] > c) {
                    cc[b + 1] = cc[b];
                    cv[b + 1] = cv[b];
                    --b;
                }
                cc[b + 1] = c;
                cv[b + 1] = v;
            }
            if (part) nu = keep;
            else nl = keep;
        }
        if (o + nl + 1 + nu > oend) {
            st[s] = -2;
            return;
        }
        rs_[r] = o;
        for (int a = 0; a < nl; ++a, ++o) {
            ocol[o] = cc[a];
            oval[o] = cv[a];
        }
        rd[r] = o;
        ocol[o] = i;
        oval[o] = diag;
        ++o;
        for (int a = 0; a < nu; ++a, ++o) {
            ocol[o] = cc[ulo + a];
            oval[o] = cv[ulo + a];
        }
        re[r] = o;
    }
    st[s] = -1;
}

// the factor rows, from their places in the scratch into the stacked CSR
// (columns offset by the subdomain's first stacked row)
__global__ void k_ilut_compact(int nx, const int64_t *__restrict__ rs_, const int64_t *__restrict__ re,
                               const int *__restrict__ hptr, const int *__restrict__ rbase,
                               const int *__restrict__ ocol, const double *__restrict__ oval, int *__restrict__ col,
                               double *__restrict__ val)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nx; r += gridDim.x * blockDim.x) {
        int d = hptr[r];
        for (int64_t q = rs_[r]; q < re[r]; ++q, ++d) {
            col[d] = ocol[q] + rbase[r];
            val[d] = oval[q];
        }
    }
}

// ILUT of the stacked local matrices on the GPU (k_ilut): xptr/xcol the
// stacked local pattern (local columns), xsrc the positions of its values in
// A, sbase the subdomains' first stacked rows, rbase every stacked row's.
// Fills hptr/hcol (host, stacked columns) and *val (device).  The output
// regions start at 8 entries per local entry plus 2 per row and double
// while a subdomain overflows its region.  RS_ERR_ZERO_PIVOT: *bad = the
// stacked row of the first zero pivot (lowest subdomain).
static int ilut_device(rs_ctx *ctx, const rs_mat *A, int nparts, const std::vector<int> &sbase,
                       const std::vector<int> &xptr, const std::vector<int> &xcol, const std::vector<int> &xsrc,
                       const std::vector<int> &rbase, int p, double tol, std::vector<int> &hptr,
                       std::vector<int> &hcol, double **val, int *bad)
{
    const cudaStream_t sm = ctx->stream;
    const int nx = (int)rbase.size();
    const int64_t nnz = (int64_t)xcol.size();
    std::vector<void *> tmp;
    auto alloc = [&](void **ptr, size_t bytes) -> int {
        *ptr = nullptr;
        const int st = rs_alloc(ctx, ptr, std::max<size_t>(bytes, 16));
        if (!st) tmp.push_back(*ptr);
        return st;
    };
    auto up = [&](void *dst, const void *src, size_t bytes) -> int {
        return !bytes || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, sm) == cudaSuccess ? RS_OK
                                                                                                     : RS_ERR_CUDA;
    };
    int st = RS_OK;
    int *d_sb, *d_ptr, *d_col, *d_src, *d_st, *d_touch, *d_low, *d_cc, *d_rbase;
    double *d_val, *d_w, *d_cv;
    char *d_in;
    int64_t *d_rs, *d_rd, *d_re;
    st = st ? st : alloc((void **)&d_sb, sizeof(int) * (nparts + 1));
    st = st ? st : alloc((void **)&d_ptr, sizeof(int) * (nx + 1));
    st = st ? st : alloc((void **)&d_col, sizeof(int) * nnz);
    st = st ? st : alloc((void **)&d_src, sizeof(int) * nnz);
    st = st ? st : alloc((void **)&d_val, sizeof(double) * nnz);
    st = st ? st : alloc((void **)&d_st, sizeof(int) * nparts);
    st = st ? st : alloc((void **)&d_w, sizeof(double) * nx);
    st = st ? st : alloc((void **)&d_in, (size_t)nx);
    st = st ? st : alloc((void **)&d_touch, sizeof(int) * nx);
    st = st ? st : alloc((void **)&d_low, sizeof(int) * nx);
    st = st ? st : alloc((void **)&d_cc, sizeof(int) * nx);
    st = st ? st : alloc((void **)&d_cv, sizeof(double) * nx);
    st = st ? st : alloc((void **)&d_rs, sizeof(int64_t) * nx);
    st = st ? st : alloc((void **)&d_rd, sizeof(int64_t) * nx);
    st = st ? st : alloc((void **)&d_re, sizeof(int64_t) * nx);
    st = st ? st : alloc((void **)&d_rbase, sizeof(int) * nx);
    st = st ? st : up(d_sb, sbase.data(), sizeof(int) * (nparts + 1));
    st = st ? st : up(d_ptr, xptr.data(), sizeof(int) * (nx + 1));
    st = st ? st : up(d_col, xcol.data(), sizeof(int) * nnz);
    st = st ? st : up(d_src, xsrc.data(), sizeof(int) * nnz);
    st = st ? st : up(d_rbase, rbase.data(), sizeof(int) * nx);
    if (!st && nnz > 0) {
        // the local values, gathered from A
        k_ras_values<<<ras_grid(ctx, nnz), 256, 0, sm>>>(nnz, 1, d_src, A->val, d_val);
        st = rs_check_launch(ctx);
    }
    if (!st && cudaMemsetAsync(d_w, 0, sizeof(double) * nx, sm) != cudaSuccess) st = RS_ERR_CUDA;
    if (!st && cudaMemsetAsync(d_in, 0, (size_t)nx, sm) != cudaSuccess) st = RS_ERR_CUDA;
    // output regions
    std::vector<int64_t> mult(nparts, 1), cap(nparts + 1);
    std::vector<int> hst(nparts, -1);
    int *d_ocol = nullptr;
    double *d_oval = nullptr;
    int64_t *d_cap = nullptr;
    for (int attempt = 0; !st; ++attempt) {
        cap[0] = 0;
        for (int s = 0; s < nparts; ++s) {
            const int64_t ns = sbase[s + 1] - sbase[s];
            const int64_t ln = xptr[sbase[s + 1]] - xptr[sbase[s]];
            cap[s + 1] = cap[s] + std::min<int64_t>((8 * ln + 2 * ns) * mult[s], ns * ns + ns);
        }
        if (d_ocol) { rs_free(ctx, d_ocol); rs_free(ctx, d_oval); rs_free(ctx, d_cap); }
        st = rs_alloc(ctx, (void **)&d_ocol, sizeof(int) * std::max<int64_t>(cap[nparts], 1));
        st = st ? st : rs_alloc(ctx, (void **)&d_oval, sizeof(double) * std::max<int64_t>(cap[nparts], 1));
        st = st ? st : rs_alloc(ctx, (void **)&d_cap, sizeof(int64_t) * (nparts + 1));
        st = st ? st : up(d_cap, cap.data(), sizeof(int64_t) * (nparts + 1));
        if (st) break;
        k_ilut<<<nparts, 32, 0, sm>>>(nparts, d_sb, d_ptr, d_col, d_val, p, tol, d_cap, d_ocol, d_oval,
                                                  d_rs, d_rd, d_re, d_w, d_in, d_touch, d_low, d_cc, d_cv, d_st);
        st = rs_check_launch(ctx);
        if (!st && (cudaMemcpyAsync(hst.data(), d_st, sizeof(int) * nparts, cudaMemcpyDeviceToHost, sm) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(sm) != cudaSuccess))
            st = RS_ERR_CUDA;
        if (st) break;
        bool over = false;
        for (int s = 0; s < nparts && !st; ++s) {
            if (hst[s] >= 0) {
                *bad = sbase[s] + hst[s];
                st = RS_ERR_ZERO_PIVOT;
            } else if (hst[s] == -2) {
                over = true;
                mult[s] *= 2;
            }
        }
        if (st || !over) break;
        // an overflow leaves w and the flags as they were: clear them
        if (cudaMemsetAsync(d_w, 0, sizeof(double) * nx, sm) != cudaSuccess ||
            cudaMemsetAsync(d_in, 0, (size_t)nx, sm) != cudaSuccess)
            st = RS_ERR_CUDA;
        if (attempt > 40) st = RS_ERR_INVALID_ARG;
    }
    // the stacked pattern: row lengths on the host, the rows compacted on the GPU
    if (!st) {
        std::vector<int64_t> hrs(nx), hre(nx);
        if (nx > 0 &&
            (cudaMemcpyAsync(hrs.data(), d_rs, sizeof(int64_t) * nx, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
             cudaMemcpyAsync(hre.data(), d_re, sizeof(int64_t) * nx, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
             cudaStreamSynchronize(sm) != cudaSuccess))
            st = RS_ERR_CUDA;
        hptr.assign(1, 0);
        for (int r = 0; r < nx && !st; ++r) {
            if ((int64_t)hptr.back() + (hre[r] - hrs[r]) > INT_MAX) st = RS_ERR_INVALID_ARG;
            else hptr.push_back(hptr.back() + (int)(hre[r] - hrs[r]));
        }
    }
    int *d_hptr = nullptr, *d_fcol = nullptr;
    const int64_t fnnz = st ? 0 : hptr.back();
    if (!st) st = alloc((void **)&d_hptr, sizeof(int) * (nx + 1));
    if (!st) st = alloc((void **)&d_fcol, sizeof(int) * fnnz);
    if (!st) st = rs_alloc(ctx, (void **)val, sizeof(double) * std::max<int64_t>(fnnz, 1));
    if (!st) st = up(d_hptr, hptr.data(), sizeof(int) * (nx + 1));
    if (!st && nx > 0) {
        k_ilut_compact<<<ras_grid(ctx, nx), 256, 0, sm>>>(nx, d_rs, d_re, d_hptr, d_rbase, d_ocol, d_oval, d_fcol,
                                                          *val);
        st = rs_check_launch(ctx);
    }
    if (!st) {
        hcol.resize(fnnz);
        if (fnnz > 0 &&
            (cudaMemcpyAsync(hcol.data(), d_fcol, sizeof(int) * fnnz, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
             cudaStreamSynchronize(sm) != cudaSuccess))
            st = RS_ERR_CUDA;
    }
    if (d_ocol) { rs_free(ctx, d_ocol); rs_free(ctx, d_oval); rs_free(ctx, d_cap); }
    for (void *q : tmp) rs_free(ctx, q);
    if (st && *val) {
        rs_free(ctx, *val);
        *val = nullptr;
    }
    return st;
}

int rs_ras_create(rs_ctx *ctx, const rs_mat *A, int nparts, const int32_t *part, int overlap, int level, int local,
                  int ilut_p, double ilut_tol, int fp32, RasData **out, int *bad_row)
{
    *out = nullptr;
    if (bad_row) *bad_row = -1;
    const int n = A->nrows, bs = A->bs;
    if (nparts < 1 || overlap < 0 || level < 0 || level > RS_RAS_MAX_LEVEL) return RS_ERR_INVALID_ARG;
    if (local != 0 && (local != 1 || bs != 1 || !(ilut_tol >= 0.0))) return RS_ERR_INVALID_ARG;
    // subdomain of each block row: the caller's, or contiguous ranges of rows
    std::vector<int> pt(n);
    for (int i = 0; i < n; ++i) {
        pt[i] = part ? part[i] : (int)((int64_t)i * nparts / std::max(n, 1));
        if (pt[i] < 0 || pt[i] >= nparts) return RS_ERR_INVALID_ARG;
    }
    const std::vector<int> &ap = A->h_ptr, &ac = A->h_col;
    // ILUT: the stacked local matrices (pattern, and the positions of their
    // values in A), factorised on the GPU after the loop
    std::vector<int> sbase(1, 0), xptr(1, 0), xcol, xsrc, rbase;
    // rows of each subdomain, ascending
    std::vector<int> pstart(nparts + 1, 0), prow(n);
    for (int i = 0; i < n; ++i) ++pstart[pt[i] + 1];
    for (int s = 0; s < nparts; ++s) pstart[s + 1] += pstart[s];
    {
        std::vector<int> fillp(pstart.begin(), pstart.end() - 1);
        for (int i = 0; i < n; ++i) prow[fillp[pt[i]]++] = i;
    }
    std::vector<int> gidx, own(n, -1), hptr(1, 0), hcol, hsrc;
    std::vector<int> mark(n, -1), loc(n, 0), set, frontier, next;
    std::vector<int> lptr, lcol, lsrc;
    int64_t total_nnz = 0;
    for (int s = 0; s < nparts; ++s) {
        set.assign(prow.begin() + pstart[s], prow.begin() + pstart[s + 1]);
        for (int g : set) mark[g] = s;
        frontier = set;
        for (int m = 0; m < overlap && !frontier.empty(); ++m) {
            next.clear();
            for (int g : frontier)
                for (int q = ap[g]; q < ap[g + 1]; ++q)
                    if (mark[ac[q]] != s) {
                        mark[ac[q]] = s;
                        next.push_back(ac[q]);
                    }
            set.insert(set.end(), next.begin(), next.end());
            frontier.swap(next);
        }
        std::sort(set.begin(), set.end());
        const int ns = (int)set.size();
        if ((int64_t)gidx.size() + ns > INT_MAX) return RS_ERR_INVALID_ARG;
        const int base = (int)gidx.size();
        for (int a = 0; a < ns; ++a) loc[set[a]] = a;
        lptr.assign(1, 0);
        lcol.clear();
        lsrc.clear();
        for (int a = 0; a < ns; ++a) {
            const int g = set[a];
            for (int q = ap[g]; q < ap[g + 1]; ++q)
                if (mark[ac[q]] == s) {
                    lcol.push_back(loc[ac[q]]);
                    lsrc.push_back(q);
                }
            lptr.push_back((int)lcol.size());
        }
        if (local == 1) {
            for (int a = 0; a < ns; ++a) {
                for (int q = lptr[a]; q < lptr[a + 1]; ++q) {
                    xcol.push_back(lcol[q]);
                    xsrc.push_back(lsrc[q]);
                }
                xptr.push_back((int)xcol.size());
                rbase.push_back(base);
            }
            sbase.push_back(base + ns);
            if ((int64_t)xcol.size() > INT_MAX) return RS_ERR_INVALID_ARG;
        } else if (level == 0) {
            for (int a = 0; a < ns; ++a) {
                for (int q = lptr[a]; q < lptr[a + 1]; ++q) {
                    hcol.push_back(base + lcol[q]);
                    hsrc.push_back(lsrc[q]);
                }
                hptr.push_back((int)hcol.size());
            }
        } else {
            iluk_rows(ns, lptr, lcol, lsrc, level, base, hptr, hcol, hsrc);
        }
        total_nnz = (int64_t)hcol.size();
        if (total_nnz > INT_MAX) return RS_ERR_INVALID_ARG;
        gidx.insert(gidx.end(), set.begin(), set.end());
        for (int r = pstart[s]; r < pstart[s + 1]; ++r) own[prow[r]] = base + loc[prow[r]];
    }
    const int nx = (int)gidx.size();
    double *ilut_val = nullptr;                // ILUT: the stacked factor's values (device)
    if (local == 1) {
        int bad = -1;
        const int st0 = ilut_device(ctx, A, nparts, sbase, xptr, xcol, xsrc, rbase, ilut_p, ilut_tol, hptr, hcol,
                                    &ilut_val, &bad);
        if (st0 == RS_ERR_ZERO_PIVOT && bad_row) *bad_row = gidx[bad];
        if (st0) return st0;
        hsrc.assign(hcol.size(), -1);
        total_nnz = (int64_t)hcol.size();
    }
    RasData *R = new RasData();
    R->ctx = ctx;
    R->bs = bs;
    R->nrows = n;
    R->next = nx;
    R->nnz = total_nnz;
    R->nparts = nparts;
    R->overlap = overlap;
    R->level = level;
    R->h_gidx = gidx;
    const size_t b2 = (size_t)bs * bs;
    int st = rs_alloc(ctx, (void **)&R->ptr, sizeof(int) * (nx + 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->col, sizeof(int) * std::max<int64_t>(total_nnz, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->src, sizeof(int) * std::max<int64_t>(total_nnz, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->gidx, sizeof(int) * std::max(nx, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->own, sizeof(int) * std::max(n, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->val, sizeof(double) * b2 * std::max<int64_t>(total_nnz, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->rhat, sizeof(double) * bs * std::max(nx, 1));
    st = st ? st : rs_alloc(ctx, (void **)&R->zhat, sizeof(double) * bs * std::max(nx, 1));
    if (st) {
        rs_ras_destroy(R);
        return st;
    }
    cudaStream_t sm = ctx->stream;
    if (cudaMemcpyAsync(R->ptr, hptr.data(), sizeof(int) * (nx + 1), cudaMemcpyHostToDevice, sm) != cudaSuccess ||
        (total_nnz > 0 &&
         (cudaMemcpyAsync(R->col, hcol.data(), sizeof(int) * total_nnz, cudaMemcpyHostToDevice, sm) != cudaSuccess ||
          cudaMemcpyAsync(R->src, hsrc.data(), sizeof(int) * total_nnz, cudaMemcpyHostToDevice, sm) !=
              cudaSuccess)) ||
        (nx > 0 && cudaMemcpyAsync(R->gidx, gidx.data(), sizeof(int) * nx, cudaMemcpyHostToDevice, sm) != cudaSuccess) ||
        (n > 0 && cudaMemcpyAsync(R->own, own.data(), sizeof(int) * n, cudaMemcpyHostToDevice, sm) != cudaSuccess)) {
        rs_ras_destroy(R);
        return RS_ERR_CUDA;
    }
    if (local == 1) {
        // the factor formed on the GPU (ilut_device)
        if (total_nnz > 0 && cudaMemcpyAsync(R->val, ilut_val, sizeof(double) * total_nnz, cudaMemcpyDeviceToDevice,
                                             sm) != cudaSuccess)
            st = RS_ERR_CUDA;
        rs_free(ctx, ilut_val);
    } else if (total_nnz > 0) {
        k_ras_values<<<ras_grid(ctx, total_nnz * (int64_t)b2), 256, 0, sm>>>(total_nnz, (int)b2, R->src, A->val, R->val);
        st = rs_check_launch(ctx);
    }
    // the stacked pattern's host copy is only needed by the analysis below
    int bad = -1;
    st = st ? st : rs_ilu_create(ctx, bs, nx, total_nnz, R->ptr, R->col, hptr, hcol, fp32, 1, 0, &R->f, &bad);
    if (local == 1) st = st ? st : rs_ilu_set_factors(R->f, R->val, &bad);
    else st = st ? st : rs_ilu_factor(R->f, R->val, &bad);
    if (bad >= 0 && bad < nx && bad_row) *bad_row = gidx[bad];
    if (st == RS_ERR_ZERO_PIVOT) {
        *out = R;            // the caller keeps the object to report the row
        return st;
    }
    if (st) {
        rs_ras_destroy(R);
        return st;
    }
    *out = R;
    return RS_OK;
}

int rs_ras_apply(RasData *R, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = R->ctx;
    if (R->nrows == 0) return RS_OK;
    {
        RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
        k_ras_gather<<<ras_grid(ctx, (int64_t)R->next * R->bs), 256, 0, ctx->stream>>>(R->next, R->bs, R->gidx, r,
                                                                                      R->rhat, skip);
    }
    RS_TRY(rs_check_launch(ctx));
    RS_TRY(rs_ilu_apply(R->f, R->rhat, R->zhat, nullptr, skip));
    RsProfScope prof(ctx, RS_PROF_PRECOND_OTHER);
    k_ras_scatter<<<ras_grid(ctx, (int64_t)R->nrows * R->bs), 256, 0, ctx->stream>>>(R->nrows, R->bs, R->own,
                                                                                    R->zhat, z, skip);
    return rs_check_launch(ctx);
}

void rs_ras_destroy(RasData *R)
{
    if (!R) return;
    rs_ctx *ctx = R->ctx;
    if (R->f) rs_ilu_destroy(R->f);     // borrows ptr / col: released first
    rs_free(ctx, R->ptr);
    rs_free(ctx, R->col);
    rs_free(ctx, R->src);
    rs_free(ctx, R->gidx);
    rs_free(ctx, R->own);
    rs_free(ctx, R->val);
    rs_free(ctx, R->rhat);
    rs_free(ctx, R->zhat);
    delete R;
}
