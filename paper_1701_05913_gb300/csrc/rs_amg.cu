// Algebraic multigrid preconditioner (Sec. 4.2: Alg. 3 setup, Alg. 4
// V-cycle, Eq. 4).
//
// Setup (once per matrix, on the host, like the setup phase of the AMG
// package the paper calls), level by level in Alg. 3's order:
//   1. strength: j strongly influences i when j != i and
//      -a_ij >= theta max_{k != i} (-a_ik) (theta = 0.5 by default, Fig. 34);
//   2. coarse points: the Ruge-Stueben first pass.  The measure of a point
//      is the number of undecided points it strongly influences plus twice
//      the number of F points it strongly influences; the undecided point
//      of largest measure (lowest index on ties) becomes C and the
//      undecided points it strongly influences become F.  Points with no
//      strong connection in either direction are F from the start;
//   3. direct interpolation: C points inject; an F point i interpolates from
//      its strong C neighbours k with w_ik = -alpha a_ik / a_ii (a_ik < 0) or
//      -beta a_ik / a_ii (a_ik > 0), alpha (beta) = the row's sum of negative
//      (positive) off-diagonal entries over that of its strong C neighbours;
//      with no positive strong C coupling the positive couplings join a_ii;
//   4. R = P^T;  5. A_{l+1} = R A_l P (Eq. 4);
//   6. smoother: l1-Jacobi, x <- x + (b - A x) / d, d_i = sum_j |a_ij|.
// Levels stop at max_coarse rows, max_levels, or when coarsening stalls;
// the coarsest matrix is inverted densely.
//
// Apply (on the GPU): one V-cycle from x = 0 (Alg. 4): nu sweeps, residual,
// restriction, the next level, prolongation and correction, nu sweeps;
// the coarsest level is one dense matrix-vector product.  Every operator is
// an rs_mat, so the products run in the library's SpMV kernels; a smoothing
// sweep is one SpMV whose epilogue forms x + (b - A x) / d into a second
// buffer.
#include <algorithm>
#include <cmath>
#include <queue>
#include <vector>

#include "rs_internal.cuh"

namespace {

struct HCsr {
    int n = 0, m = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};

// strong influences of every row: S[i] = { j : j strongly influences i }
void strength(const HCsr &A, double theta, std::vector<int> &sp, std::vector<int> &sc)
{
    sp.assign(A.n + 1, 0);
    sc.clear();
    for (int i = 0; i < A.n; ++i) {
        double mx = 0.0;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
            if (A.col[p] != i) mx = std::max(mx, -A.val[p]);
        if (mx > 0.0)
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
                if (A.col[p] != i && -A.val[p] >= theta * mx) sc.push_back(A.col[p]);
        sp[i + 1] = (int)sc.size();
    }
}

// coarse index of every point (-1 = F) by the Ruge-Stueben first pass
int first_pass(int n, const std::vector<int> &sp, const std::vector<int> &sc, std::vector<int> &cidx)
{
    // transpose of S: the points each point strongly influences
    std::vector<int> tp(n + 1, 0), tc(sc.size());
    for (int c : sc) ++tp[c + 1];
    for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
    {
        std::vector<int> f(tp.begin(), tp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int q = sp[i]; q < sp[i + 1]; ++q) tc[f[sc[q]]++] = i;
    }
    enum : char { UND = 0, CP = 1, FP = 2 };
    std::vector<char> st(n, UND);
    std::vector<int> lam(n);
    // max-heap on (measure, -index); stale entries are skipped when popped
    std::priority_queue<std::pair<int, int>> heap;
    for (int i = 0; i < n; ++i) {
        lam[i] = tp[i + 1] - tp[i];
        if (lam[i] == 0 && sp[i + 1] == sp[i]) st[i] = FP;
        else heap.push({lam[i], -i});
    }
    while (!heap.empty()) {
        const auto e = heap.top();
        heap.pop();
        const int i = -e.second;
        if (st[i] != UND || e.first != lam[i]) continue;
        st[i] = CP;
        for (int q = tp[i]; q < tp[i + 1]; ++q) {
            const int j = tc[q];
            if (st[j] != UND) continue;
            st[j] = FP;
            for (int r = sp[j]; r < sp[j + 1]; ++r) {
                const int k = sc[r];
                if (st[k] == UND) heap.push({++lam[k], -k});
            }
        }
        for (int r = sp[i]; r < sp[i + 1]; ++r) {
            const int k = sc[r];
            if (st[k] == UND) heap.push({--lam[k], -k});
        }
    }
    cidx.assign(n, -1);
    int nc = 0;
    for (int i = 0; i < n; ++i)
        if (st[i] == CP) cidx[i] = nc++;
    return nc;
}

void direct_interpolation(const HCsr &A, const std::vector<int> &sp, const std::vector<int> &sc,
                          const std::vector<int> &cidx, int nc, HCsr &P)
{
    P.n = A.n;
    P.m = nc;
    P.ptr.assign(1, 0);
    P.col.clear();
    P.val.clear();
    std::vector<char> strongc(A.n, 0);
    for (int i = 0; i < A.n; ++i) {
        if (cidx[i] >= 0) {
            P.col.push_back(cidx[i]);
            P.val.push_back(1.0);
        } else {
            for (int r = sp[i]; r < sp[i + 1]; ++r)
                if (cidx[sc[r]] >= 0) strongc[sc[r]] = 1;
            double aii = 0.0, neg = 0.0, pos = 0.0, negc = 0.0, posc = 0.0;
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                const int j = A.col[p];
                const double v = A.val[p];
                if (j == i) { aii = v; continue; }
                (v < 0.0 ? neg : pos) += v;
                if (strongc[j]) (v < 0.0 ? negc : posc) += v;
            }
            double diag = aii, beta = 0.0;
            if (posc == 0.0) diag += pos;
            else beta = pos / posc;
            const double alpha = negc != 0.0 ? neg / negc : 0.0;
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                const int k = A.col[p];
                if (k == i || !strongc[k]) continue;
                P.col.push_back(cidx[k]);
                P.val.push_back(-(A.val[p] < 0.0 ? alpha : beta) * A.val[p] / diag);
            }
            for (int r = sp[i]; r < sp[i + 1]; ++r) strongc[sc[r]] = 0;
        }
        P.ptr.push_back((int)P.col.size());
    }
}

void transpose(const HCsr &A, HCsr &T)
{
    T.n = A.m;
    T.m = A.n;
    T.ptr.assign(A.m + 1, 0);
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    for (int c : A.col) ++T.ptr[c + 1];
    for (int c = 0; c < A.m; ++c) T.ptr[c + 1] += T.ptr[c];
    std::vector<int> f(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n; ++i)
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int q = f[A.col[p]]++;
            T.col[q] = i;
            T.val[q] = A.val[p];
        }
}

// C = A B by rows (Gustavson), columns sorted
void multiply(const HCsr &A, const HCsr &B, HCsr &C)
{
    C.n = A.n;
    C.m = B.m;
    C.ptr.assign(1, 0);
    C.col.clear();
    C.val.clear();
    std::vector<int> mark(B.m, -1), cols;
    std::vector<double> acc(B.m, 0.0);
    for (int i = 0; i < A.n; ++i) {
        cols.clear();
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int j = A.col[p];
            const double a = A.val[p];
            for (int q = B.ptr[j]; q < B.ptr[j + 1]; ++q) {
                const int c = B.col[q];
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols.push_back(c);
                }
                acc[c] += a * B.val[q];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int c : cols) {
            C.col.push_back(c);
            C.val.push_back(acc[c]);
        }
        C.ptr.push_back((int)C.col.size());
    }
}

// dense inverse by Gauss-Jordan elimination with partial pivoting
bool invert(int n, std::vector<double> a, std::vector<double> &inv)
{
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
        const double piv = a[(size_t)p * n + c];
        if (!(piv != 0.0) || !std::isfinite(piv)) return false;
        if (p != c)
            for (int j = 0; j < n; ++j) {
                std::swap(a[(size_t)c * n + j], a[(size_t)p * n + j]);
                std::swap(inv[(size_t)c * n + j], inv[(size_t)p * n + j]);
            }
        for (int j = 0; j < n; ++j) {
            a[(size_t)c * n + j] /= piv;
            inv[(size_t)c * n + j] /= piv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[(size_t)r * n + j] -= f * a[(size_t)c * n + j];
                inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
            }
        }
    }
    return true;
}

}  // namespace

// the host hierarchy, kept for export
struct AmgHost {
    std::vector<HCsr> A, P;
    std::vector<std::vector<int>> cidx;
};

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
    for (int l = 0; l < M->nlev; ++l) {
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
    for (const AmgGraph &g : M->graphs) cudaGraphExecDestroy(g.exec);
    if (M->capture) cudaStreamDestroy(M->capture);
    delete M->host;
    delete M;
}

int rs_amg_create(rs_ctx *ctx, int n, const std::vector<int> &hptr, const std::vector<int> &hcol,
                  const double *d_val, const rs_mat *A0, double theta, int max_levels, int max_coarse, int nu,
                  int smoother, AmgData **out)
{
    *out = nullptr;
    if (n < 1 || max_levels < 1 || max_levels > RS_AMG_MAXLEV || max_coarse < 1 || nu < 1 || !(theta >= 0.0) ||
        smoother < 0 || smoother > 1)
        return RS_ERR_INVALID_ARG;
    AmgData *M = new AmgData();
    M->ctx = ctx;
    M->nu = nu;
    M->smoother = smoother;
    M->host = new AmgHost();
    AmgHost &H = *M->host;
    H.A.emplace_back();
    HCsr &F = H.A[0];
    F.n = F.m = n;
    F.ptr = hptr;
    F.col = hcol;
    F.val.resize(hcol.size());
    if (!hcol.empty()) {
        RS_CUDA_TRY(cudaMemcpyAsync(F.val.data(), d_val, sizeof(double) * hcol.size(), cudaMemcpyDeviceToHost,
                                    ctx->stream));
        RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    // the hierarchy (Alg. 3)
    std::vector<int> sp, sc;
    for (int l = 0;; ++l) {
        if (H.A[l].n <= max_coarse || l + 1 >= max_levels) break;
        strength(H.A[l], theta, sp, sc);
        std::vector<int> cidx;
        const int nc = first_pass(H.A[l].n, sp, sc, cidx);
        if (nc == 0 || nc >= H.A[l].n) break;
        HCsr P, R, AP, Ac;
        direct_interpolation(H.A[l], sp, sc, cidx, nc, P);
        transpose(P, R);
        multiply(H.A[l], P, AP);
        multiply(R, AP, Ac);
        H.P.push_back(std::move(P));
        H.cidx.push_back(std::move(cidx));
        H.A.push_back(std::move(Ac));
    }
    M->nlev = (int)H.A.size();
    if (H.A.back().n > RS_AMG_MAX_DENSE) {     // coarsening stalled: no small coarsest level
        rs_amg_destroy(M);
        return RS_ERR_INVALID_ARG;
    }
    if (smoother == 1) {   // Gauss-Seidel divides by a_ii on every smoothed level
        for (int l = 0; l + 1 < M->nlev; ++l) {
            const HCsr &A = H.A[l];
            for (int i = 0; i < A.n; ++i) {
                double dg = 0.0;
                for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
                    if (A.col[p] == i) dg = A.val[p];
                if (dg == 0.0) {
                    rs_amg_destroy(M);
                    return RS_ERR_ZERO_PIVOT;
                }
            }
        }
    }
    std::vector<double> inv;
    {
        const HCsr &C = H.A.back();
        std::vector<double> dense((size_t)C.n * C.n, 0.0);
        for (int i = 0; i < C.n; ++i)
            for (int p = C.ptr[i]; p < C.ptr[i + 1]; ++p) dense[(size_t)i * C.n + C.col[p]] = C.val[p];
        if (!invert(C.n, std::move(dense), inv)) {
            rs_amg_destroy(M);
            return RS_ERR_ZERO_PIVOT;
        }
    }
    // device objects
    int st = RS_OK;
    for (int l = 0; l < M->nlev && !st; ++l) {
        const HCsr &A = H.A[l];
        if (l == 0 && A0) {
            M->A[0] = const_cast<rs_mat *>(A0);
        } else {
            M->own0 = M->own0 || l == 0;
            st = rs_mat_create_rect(ctx, A.n, A.n, A.ptr.data(), A.col.data(), A.val.data(), &M->A[l]);
            if (st) break;
        }
        if (l + 1 < M->nlev) {
            HCsr R;
            transpose(H.P[l], R);
            st = rs_mat_create_rect(ctx, H.P[l].n, H.P[l].m, H.P[l].ptr.data(), H.P[l].col.data(),
                                    H.P[l].val.data(), &M->P[l]);
            if (!st) st = rs_mat_create_rect(ctx, R.n, R.m, R.ptr.data(), R.col.data(), R.val.data(), &M->R[l]);
            if (st) break;
        }
        std::vector<double> d(A.n);      // 1 / d_i, d_i = sum_j |a_ij|
        for (int i = 0; i < A.n; ++i) {
            double s = 0.0;
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) s += std::fabs(A.val[p]);
            d[i] = 1.0 / s;
        }
        st = rs_alloc(ctx, (void **)&M->d[l], sizeof(double) * A.n);
        if (!st) st = rs_alloc(ctx, (void **)&M->b[l], sizeof(double) * A.n);
        if (!st) st = rs_alloc(ctx, (void **)&M->x[l], sizeof(double) * A.n);
        if (!st) st = rs_alloc(ctx, (void **)&M->t[l], sizeof(double) * A.n);
        if (!st && l > 0) st = rs_alloc(ctx, (void **)&M->y[l], sizeof(double) * A.n);
        if (!st && cudaMemcpyAsync(M->d[l], d.data(), sizeof(double) * A.n, cudaMemcpyHostToDevice, ctx->stream) !=
                       cudaSuccess)
            st = RS_ERR_CUDA;
    }
    const int nc = H.A.back().n;
    if (!st) st = rs_alloc(ctx, (void **)&M->cinv, sizeof(double) * (size_t)nc * nc);
    if (!st && cudaMemcpyAsync(M->cinv, inv.data(), sizeof(double) * (size_t)nc * nc, cudaMemcpyHostToDevice,
                               ctx->stream) != cudaSuccess)
        st = RS_ERR_CUDA;
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
    const AmgHost &H = *M->host;
    *n = H.A[l].n;
    *nnz_a = (int64_t)H.A[l].col.size();
    *nnz_p = l + 1 < M->nlev ? (int64_t)H.P[l].col.size() : 0;
    return RS_OK;
}

int rs_amg_get_level(const AmgData *M, int l, int32_t *aptr, int32_t *acol, double *aval, int32_t *pptr,
                     int32_t *pcol, double *pval, int32_t *cidx)
{
    if (l < 0 || l >= M->nlev) return RS_ERR_INVALID_ARG;
    const AmgHost &H = *M->host;
    const HCsr &A = H.A[l];
    if (aptr) std::copy(A.ptr.begin(), A.ptr.end(), aptr);
    if (acol) std::copy(A.col.begin(), A.col.end(), acol);
    if (aval) std::copy(A.val.begin(), A.val.end(), aval);
    if (l + 1 < M->nlev) {
        const HCsr &P = H.P[l];
        if (pptr) std::copy(P.ptr.begin(), P.ptr.end(), pptr);
        if (pcol) std::copy(P.col.begin(), P.col.end(), pcol);
        if (pval) std::copy(P.val.begin(), P.val.end(), pval);
        if (cidx) std::copy(H.cidx[l].begin(), H.cidx[l].end(), cidx);
    }
    return RS_OK;
}
