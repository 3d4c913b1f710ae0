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

// ILUT(p, tol) of one local matrix (rows 0..n-1, sorted columns, values
// lval), Saad's algorithm row by row: the row in a dense work array; its
// lower entries eliminated in ascending order (fill included), each
// multiplier w_k = w_k / u_kk dropped below tau = tol ||a_i||_2, else
// w_j -= w_k u_kj over the stored U row k; then off-diagonal entries below
// tau dropped and the p largest kept in each part (ties to the lower
// column; p < 0: as many as row i has there).  Appends the factor rows
// (strict L, then U with its diagonal, columns + base) to optr/ocol/olu.
// Returns the local row of a zero pivot, or -1.
static int ilut_rows(int n, const std::vector<int> &lptr, const std::vector<int> &lcol, const std::vector<double> &lval,
                     int p, double tol, int base, std::vector<int> &optr, std::vector<int> &ocol,
                     std::vector<double> &olu)
{
    std::vector<int> up(n + 1), uc;          // U rows kept so far (diagonal first)
    std::vector<double> uv;
    std::vector<double> w(n, 0.0);
    std::vector<char> in(n, 0);
    std::vector<int> touched, lower;
    std::vector<std::pair<int, double>> lo, hi;
    auto larger = [](const std::pair<int, double> &a, const std::pair<int, double> &b) {
        const double x = std::fabs(a.second), y = std::fabs(b.second);
        return x != y ? x > y : a.first < b.first;
    };
    for (int i = 0; i < n; ++i) {
        touched.clear();
        lower.clear();
        int pl = 0, pu = 0;
        double sq = 0.0;
        for (int q = lptr[i]; q < lptr[i + 1]; ++q) {
            const int c = lcol[q];
            w[c] = lval[q];
            in[c] = 1;
            touched.push_back(c);
            sq += lval[q] * lval[q];
            if (c < i) { ++pl; lower.push_back(c); }
            else if (c > i) ++pu;
        }
        const double tau = tol * std::sqrt(sq);
        if (p >= 0) pl = pu = p;
        for (size_t t = 0; t < lower.size(); ++t) {
            const int k = lower[t];
            if (w[k] == 0.0) continue;
            w[k] = w[k] / uv[up[k]];
            if (std::fabs(w[k]) < tau) { w[k] = 0.0; continue; }
            for (int q = up[k] + 1; q < up[k + 1]; ++q) {
                const int j = uc[q];
                if (!in[j]) {
                    in[j] = 1;
                    w[j] = 0.0;
                    touched.push_back(j);
                    if (j < i) lower.insert(std::upper_bound(lower.begin() + t + 1, lower.end(), j), j);
                }
                w[j] = w[j] - w[k] * uv[q];
            }
        }
        lo.clear();
        hi.clear();
        double diag = 0.0;
        for (int c : touched) {
            if (c == i) diag = w[c];
            else if (w[c] != 0.0 && std::fabs(w[c]) >= tau) (c < i ? lo : hi).push_back({c, w[c]});
            w[c] = 0.0;
            in[c] = 0;
        }
        if (!(diag != 0.0) || !std::isfinite(diag)) return i;
        std::sort(lo.begin(), lo.end(), larger);
        std::sort(hi.begin(), hi.end(), larger);
        if ((int)lo.size() > pl) lo.resize(pl);
        if ((int)hi.size() > pu) hi.resize(pu);
        std::sort(lo.begin(), lo.end());
        std::sort(hi.begin(), hi.end());
        for (const auto &e : lo) { ocol.push_back(base + e.first); olu.push_back(e.second); }
        ocol.push_back(base + i);
        olu.push_back(diag);
        up[i] = (int)uc.size();
        uc.push_back(i);
        uv.push_back(diag);
        for (const auto &e : hi) {
            ocol.push_back(base + e.first);
            olu.push_back(e.second);
            uc.push_back(e.first);
            uv.push_back(e.second);
        }
        up[i + 1] = (int)uc.size();
        optr.push_back((int)ocol.size());
    }
    return -1;
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
    std::vector<double> av;                    // A's values, for ILUT on the host
    if (local == 1 && !ac.empty()) {
        av.resize(ac.size());
        if (cudaMemcpyAsync(av.data(), A->val, sizeof(double) * ac.size(), cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    std::vector<double> hlu;                   // ILUT: the stacked factor
    int ilut_bad = -1;
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
            std::vector<double> lval(lsrc.size());
            for (size_t q = 0; q < lsrc.size(); ++q) lval[q] = av[lsrc[q]];
            const int b = ilut_rows(ns, lptr, lcol, lval, ilut_p, ilut_tol, base, hptr, hcol, hlu);
            if (b >= 0) {
                ilut_bad = set[b];
                break;
            }
            hsrc.resize(hcol.size(), -1);
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
    if (ilut_bad >= 0) {
        if (bad_row) *bad_row = ilut_bad;
        return RS_ERR_ZERO_PIVOT;
    }
    const int nx = (int)gidx.size();
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
        // the factor itself was formed on the host
        if (total_nnz > 0 &&
            cudaMemcpyAsync(R->val, hlu.data(), sizeof(double) * total_nnz, cudaMemcpyHostToDevice, sm) != cudaSuccess)
            st = RS_ERR_CUDA;
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
