/*
 * Plain, slow, single-threaded FP64 CPU oracle of the preconditioned Krylov
 * path (Liu & Chen, "Scalable linear solvers for sparse linear systems from
 * large-scale numerical simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the arrays produced by the seeded input generators.
 *
 * Conventions: every summation runs in ascending column order, one row at a
 * time; no blocking, reordering or fusion.  Build with -ffp-contract=off so
 * that no multiply-add is contracted (results are then the same on x86-64
 * and AArch64).
 *
 * Parity status of each function is listed where it is defined; all of them
 * are pinned by tests/test_oracle_pins.py except the learned stage, which
 * lives in oracle/convnet.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_INVALID (-1)
#define OR_ZERO_PIVOT (-3)
#define OR_BREAKDOWN (-4)

/* ------------------------------------------------------------------------ */
/* Matrix: CSR (bs = 1) or BSR with bs x bs row-major blocks.                */
/* Sec. 2.3, Fig. 15 (MAT: per-row column indices and values).               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t bs;          /* 1 => CSR; > 1 => BSR */
    int32_t nrows;       /* block rows */
    const int32_t *ptr;  /* nrows + 1 */
    const int32_t *col;  /* block column of each stored block */
    const double *val;   /* bs*bs values per stored block, row-major */
} or_mat;

/* y = A x.  Sec. 2.3, Fig. 20 (MatVecMXY): y_i = sum_j a_ij x_j. */
void or_spmv(const or_mat *A, const double *x, double *y)
{
    const int32_t bs = A->bs;
    for (int32_t I = 0; I < A->nrows; ++I) {
        for (int32_t r = 0; r < bs; ++r) {
            double acc = 0.0;
            for (int32_t p = A->ptr[I]; p < A->ptr[I + 1]; ++p) {
                const double *blk = A->val + (size_t)p * bs * bs + (size_t)r * bs;
                for (int32_t c = 0; c < bs; ++c)
                    acc += blk[c] * x[(size_t)A->col[p] * bs + c];
            }
            y[(size_t)I * bs + r] = acc;
        }
    }
}

/* y = a*(A x) + b*y.  Sec. 2.3, Fig. 21 (MatVecAMXPBY). */
void or_amxpby(double a, const or_mat *A, const double *x, double b, double *y)
{
    const int32_t bs = A->bs;
    for (int32_t I = 0; I < A->nrows; ++I) {
        for (int32_t r = 0; r < bs; ++r) {
            double acc = 0.0;
            for (int32_t p = A->ptr[I]; p < A->ptr[I + 1]; ++p) {
                const double *blk = A->val + (size_t)p * bs * bs + (size_t)r * bs;
                for (int32_t c = 0; c < bs; ++c)
                    acc += blk[c] * x[(size_t)A->col[p] * bs + c];
            }
            const size_t i = (size_t)I * bs + r;
            y[i] = a * acc + b * y[i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* BLAS-1.  Sec. 2.2, Figs. 10-13.                                            */
/* ------------------------------------------------------------------------ */
/* y = a x + b y (Fig. 10, VecAXPBY) */
void or_axpby(int64_t n, double a, const double *x, double b, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = a * x[i] + b * y[i];
}

/* z = a x + b y (Fig. 11, VecAXPBYZ) */
void or_axpbyz(int64_t n, double a, const double *x, double b, const double *y, double *z)
{
    for (int64_t i = 0; i < n; ++i) z[i] = a * x[i] + b * y[i];
}

/* <x, y> (Fig. 12, VecDot; one process, so no reduction across ranks) */
double or_dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

double or_norm2(int64_t n, const double *x) { return sqrt(or_dot(n, x, x)); }

/* x_i = v (Fig. 13, VecSetValue) */
void or_set(int64_t n, double v, double *x)
{
    for (int64_t i = 0; i < n; ++i) x[i] = v;
}

/* ------------------------------------------------------------------------ */
/* ILU(0).  Sec. 4.1, Eq. 3 names the factorisation L U and its two          */
/* triangular solves; ILU(0) keeps exactly the pattern of A (Saad,           */
/* "Iterative methods for sparse linear systems", the IKJ variant).          */
/* Result: lu holds the strictly lower part of L (unit diagonal implied)     */
/* and the upper part of U including its diagonal, in A's pattern.           */
/* Requires sorted columns and a stored diagonal in every row.               */
/* ------------------------------------------------------------------------ */
static int32_t find_diag(const int32_t *ptr, const int32_t *col, int32_t i)
{
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p)
        if (col[p] == i) return p;
    return -1;
}

int or_ilu0(int32_t n, const int32_t *ptr, const int32_t *col, const double *a,
            double *lu, int32_t *bad_row)
{
    memcpy(lu, a, sizeof(double) * (size_t)ptr[n]);
    *bad_row = -1;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t di = find_diag(ptr, col, i);
        if (di < 0) { *bad_row = i; return OR_INVALID; }
        for (int32_t p = ptr[i]; p < di; ++p) {
            const int32_t k = col[p];
            const int32_t dk = find_diag(ptr, col, k);
            const double piv = lu[dk];
            lu[p] = lu[p] / piv;
            /* a_ij -= a_ik * a_kj for j > k in pat(i) and pat(k) */
            int32_t q = p + 1;
            for (int32_t r = dk + 1; r < ptr[k + 1]; ++r) {
                const int32_t j = col[r];
                while (q < ptr[i + 1] && col[q] < j) ++q;
                if (q == ptr[i + 1]) break;
                if (col[q] == j) lu[q] = lu[q] - lu[p] * lu[r];
            }
        }
        if (!(lu[di] != 0.0) || !isfinite(lu[di])) { *bad_row = i; return OR_ZERO_PIVOT; }
    }
    return OR_OK;
}

/* z = U^{-1} L^{-1} r (Eq. 3: L y = r, then U z = y). */
void or_ilu0_solve(int32_t n, const int32_t *ptr, const int32_t *col, const double *lu,
                   const double *r, double *z)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) {
        double acc = r[i];
        for (int32_t p = ptr[i]; p < ptr[i + 1] && col[p] < i; ++p) acc -= lu[p] * y[col[p]];
        y[i] = acc;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        const int32_t di = find_diag(ptr, col, i);
        double acc = y[i];
        for (int32_t p = di + 1; p < ptr[i + 1]; ++p) acc -= lu[p] * z[col[p]];
        z[i] = acc / lu[di];
    }
    free(y);
}

/* Same solve with FP32 factors and FP32 arithmetic (the mixed-precision
 * preconditioner apply): r is rounded to FP32 on entry, z widened on exit. */
void or_ilu0_solve_f32(int32_t n, const int32_t *ptr, const int32_t *col, const float *lu,
                       const double *r, double *z)
{
    float *y = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float *w = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) {
        float acc = (float)r[i];
        for (int32_t p = ptr[i]; p < ptr[i + 1] && col[p] < i; ++p) acc -= lu[p] * y[col[p]];
        y[i] = acc;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        const int32_t di = find_diag(ptr, col, i);
        float acc = y[i];
        for (int32_t p = di + 1; p < ptr[i + 1]; ++p) acc -= lu[p] * w[col[p]];
        w[i] = acc / lu[di];
    }
    for (int32_t i = 0; i < n; ++i) z[i] = (double)w[i];
    free(y);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Block ILU(0) with bs x bs blocks (not in the paper, which cites block-    */
/* wise ILU as related work in Sec. 1): ILU(0) over the block pattern, with  */
/* L_IK = A_IK inv(U_KK) and A_IJ -= L_IK U_KJ.  dinv holds inv(U_II).        */
/* ------------------------------------------------------------------------ */

/* inverse of a bs x bs row-major block by Gauss-Jordan elimination with
 * partial pivoting; returns 0 when a pivot is zero or non-finite. */
static int block_inverse(int32_t bs, const double *a, double *inv)
{
    double m[64], e[64];
    if (bs > 8) return 0;
    for (int32_t i = 0; i < bs * bs; ++i) { m[i] = a[i]; e[i] = 0.0; }
    for (int32_t i = 0; i < bs; ++i) e[i * bs + i] = 1.0;
    for (int32_t c = 0; c < bs; ++c) {
        int32_t piv = c;
        for (int32_t r = c + 1; r < bs; ++r)
            if (fabs(m[r * bs + c]) > fabs(m[piv * bs + c])) piv = r;
        if (!(m[piv * bs + c] != 0.0) || !isfinite(m[piv * bs + c])) return 0;
        if (piv != c) {
            for (int32_t k = 0; k < bs; ++k) {
                double t = m[c * bs + k]; m[c * bs + k] = m[piv * bs + k]; m[piv * bs + k] = t;
                t = e[c * bs + k]; e[c * bs + k] = e[piv * bs + k]; e[piv * bs + k] = t;
            }
        }
        const double d = m[c * bs + c];
        for (int32_t k = 0; k < bs; ++k) { m[c * bs + k] /= d; e[c * bs + k] /= d; }
        for (int32_t r = 0; r < bs; ++r) {
            if (r == c) continue;
            const double f = m[r * bs + c];
            for (int32_t k = 0; k < bs; ++k) {
                m[r * bs + k] -= f * m[c * bs + k];
                e[r * bs + k] -= f * e[c * bs + k];
            }
        }
    }
    for (int32_t i = 0; i < bs * bs; ++i) inv[i] = e[i];
    return 1;
}

/* c = a b for bs x bs row-major blocks */
static void block_mul(int32_t bs, const double *a, const double *b, double *c)
{
    for (int32_t i = 0; i < bs; ++i)
        for (int32_t j = 0; j < bs; ++j) {
            double s = 0.0;
            for (int32_t k = 0; k < bs; ++k) s += a[i * bs + k] * b[k * bs + j];
            c[i * bs + j] = s;
        }
}

int or_bilu0(int32_t nb, int32_t bs, const int32_t *ptr, const int32_t *col, const double *a,
             double *lu, double *dinv, int32_t *bad_row)
{
    const size_t b2 = (size_t)bs * bs;
    double t[64], u[64];
    if (bs < 1 || bs > 8) return OR_INVALID;
    memcpy(lu, a, sizeof(double) * b2 * (size_t)ptr[nb]);
    *bad_row = -1;
    for (int32_t I = 0; I < nb; ++I) {
        const int32_t dI = find_diag(ptr, col, I);
        if (dI < 0) { *bad_row = I; return OR_INVALID; }
        for (int32_t p = ptr[I]; p < dI; ++p) {
            const int32_t K = col[p];
            const int32_t dK = find_diag(ptr, col, K);
            block_mul(bs, lu + p * b2, dinv + (size_t)K * b2, t);
            memcpy(lu + p * b2, t, sizeof(double) * b2);
            int32_t q = p + 1;
            for (int32_t r = dK + 1; r < ptr[K + 1]; ++r) {
                const int32_t J = col[r];
                while (q < ptr[I + 1] && col[q] < J) ++q;
                if (q == ptr[I + 1]) break;
                if (col[q] == J) {
                    block_mul(bs, lu + p * b2, lu + r * b2, u);
                    for (size_t e = 0; e < b2; ++e) lu[q * b2 + e] = lu[q * b2 + e] - u[e];
                }
            }
        }
        if (!block_inverse(bs, lu + dI * b2, dinv + (size_t)I * b2)) { *bad_row = I; return OR_ZERO_PIVOT; }
    }
    return OR_OK;
}

/* z = U^{-1} L^{-1} r over blocks: y_I = r_I - sum_{J<I} L_IJ y_J;
 * z_I = inv(U_II) (y_I - sum_{J>I} U_IJ z_J). */
void or_bilu0_solve(int32_t nb, int32_t bs, const int32_t *ptr, const int32_t *col,
                    const double *lu, const double *dinv, const double *r, double *z)
{
    const size_t b2 = (size_t)bs * bs;
    double *y = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1) * bs);
    double acc[8];
    for (int32_t I = 0; I < nb; ++I) {
        for (int32_t k = 0; k < bs; ++k) acc[k] = r[(size_t)I * bs + k];
        for (int32_t p = ptr[I]; p < ptr[I + 1] && col[p] < I; ++p)
            for (int32_t k = 0; k < bs; ++k)
                for (int32_t c = 0; c < bs; ++c)
                    acc[k] -= lu[p * b2 + k * bs + c] * y[(size_t)col[p] * bs + c];
        for (int32_t k = 0; k < bs; ++k) y[(size_t)I * bs + k] = acc[k];
    }
    for (int32_t I = nb - 1; I >= 0; --I) {
        const int32_t dI = find_diag(ptr, col, I);
        for (int32_t k = 0; k < bs; ++k) acc[k] = y[(size_t)I * bs + k];
        for (int32_t p = dI + 1; p < ptr[I + 1]; ++p)
            for (int32_t k = 0; k < bs; ++k)
                for (int32_t c = 0; c < bs; ++c)
                    acc[k] -= lu[p * b2 + k * bs + c] * z[(size_t)col[p] * bs + c];
        for (int32_t k = 0; k < bs; ++k) {
            double s = 0.0;
            for (int32_t c = 0; c < bs; ++c) s += dinv[(size_t)I * b2 + k * bs + c] * acc[c];
            z[(size_t)I * bs + k] = s;
        }
    }
    free(y);
}

/* FP32 factors and arithmetic (mixed-precision apply). */
void or_bilu0_solve_f32(int32_t nb, int32_t bs, const int32_t *ptr, const int32_t *col,
                        const float *lu, const float *dinv, const double *r, double *z)
{
    const size_t b2 = (size_t)bs * bs;
    float *y = (float *)malloc(sizeof(float) * (size_t)(nb > 0 ? nb : 1) * bs);
    float *w = (float *)malloc(sizeof(float) * (size_t)(nb > 0 ? nb : 1) * bs);
    float acc[8];
    for (int32_t I = 0; I < nb; ++I) {
        for (int32_t k = 0; k < bs; ++k) acc[k] = (float)r[(size_t)I * bs + k];
        for (int32_t p = ptr[I]; p < ptr[I + 1] && col[p] < I; ++p)
            for (int32_t k = 0; k < bs; ++k)
                for (int32_t c = 0; c < bs; ++c)
                    acc[k] -= lu[p * b2 + k * bs + c] * y[(size_t)col[p] * bs + c];
        for (int32_t k = 0; k < bs; ++k) y[(size_t)I * bs + k] = acc[k];
    }
    for (int32_t I = nb - 1; I >= 0; --I) {
        const int32_t dI = find_diag(ptr, col, I);
        for (int32_t k = 0; k < bs; ++k) acc[k] = y[(size_t)I * bs + k];
        for (int32_t p = dI + 1; p < ptr[I + 1]; ++p)
            for (int32_t k = 0; k < bs; ++k)
                for (int32_t c = 0; c < bs; ++c)
                    acc[k] -= lu[p * b2 + k * bs + c] * w[(size_t)col[p] * bs + c];
        for (int32_t k = 0; k < bs; ++k) {
            float s = 0.0f;
            for (int32_t c = 0; c < bs; ++c) s += dinv[(size_t)I * b2 + k * bs + c] * acc[c];
            w[(size_t)I * bs + k] = s;
        }
    }
    for (size_t i = 0; i < (size_t)nb * bs; ++i) z[i] = (double)w[i];
    free(y);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Quasi-IMPES decoupling and the CPR restriction / prolongation.            */
/* Sec. 4.3, Eqs. 5-9: Pi_r picks the pressure unknowns, Pi_p injects a      */
/* pressure vector with zero saturations.  Quasi-IMPES (named in Example 2)  */
/* left-scales each cell's equations: weight w_Ik = -D_I[0][k] / D_I[k][k]   */
/* with D_I the diagonal block, so the decoupled pressure row is             */
/* row 0 + sum_k w_Ik row k of block row I.                                  */
/* ------------------------------------------------------------------------ */
void or_qimpes_weights(const or_mat *A, double *w)
{
    const int32_t bs = A->bs;
    const size_t b2 = (size_t)bs * bs;
    for (int32_t I = 0; I < A->nrows; ++I) {
        const int32_t dI = find_diag(A->ptr, A->col, I);
        const double *D = A->val + (size_t)dI * b2;
        for (int32_t k = 1; k < bs; ++k)
            w[(size_t)I * (bs - 1) + (k - 1)] = -D[k] / D[k * bs + k];
    }
}

/* App' in the block pattern of A: pressure-column entry of the decoupled
 * pressure row, A_IJ[0][0] + sum_k w_Ik A_IJ[k][0]. */
void or_qimpes_app(const or_mat *A, const double *w, double *app)
{
    const int32_t bs = A->bs;
    const size_t b2 = (size_t)bs * bs;
    for (int32_t I = 0; I < A->nrows; ++I)
        for (int32_t p = A->ptr[I]; p < A->ptr[I + 1]; ++p) {
            const double *B = A->val + (size_t)p * b2;
            double s = B[0];
            for (int32_t k = 1; k < bs; ++k) s += w[(size_t)I * (bs - 1) + (k - 1)] * B[k * bs];
            app[p] = s;
        }
}

/* rp_I = f_{I,0} + sum_k w_Ik f_{I,k}  (Pi_r after the decoupling) */
void or_qimpes_restrict(int32_t nb, int32_t bs, const double *w, const double *f, double *rp)
{
    for (int32_t I = 0; I < nb; ++I) {
        double s = f[(size_t)I * bs];
        for (int32_t k = 1; k < bs; ++k) s += w[(size_t)I * (bs - 1) + (k - 1)] * f[(size_t)I * bs + k];
        rp[I] = s;
    }
}

/* Pi_p (Eq. 8): z_{I,0} = p_I, z_{I,k} = 0 */
void or_prolong(int32_t nb, int32_t bs, const double *p, double *z)
{
    for (int32_t I = 0; I < nb; ++I) {
        z[(size_t)I * bs] = p[I];
        for (int32_t k = 1; k < bs; ++k) z[(size_t)I * bs + k] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* ILU(k) pattern by level of fill (Sec. 4.1 names ILU(k) as the default     */
/* local solver of RAS; the rule is the textbook one, Saad, "Iterative       */
/* methods for sparse linear systems", Sec. 10.3.3): entries of A have       */
/* level 0; eliminating with pivot row k produces (i, j), j > k, at level    */
/* lev(i,k) + lev(k,j) + 1, keeping the smallest level met; entries whose    */
/* level is at most p are kept.  The numeric ILU(k) is then ILU(0) on this   */
/* pattern with zeros at the new positions.                                  */
/* On return *optr (n+1) and *ocol (sorted rows) are malloc'ed.               */
/* ------------------------------------------------------------------------ */
int or_iluk_symbolic(int32_t n, const int32_t *ptr, const int32_t *col, int32_t p,
                     int32_t **optr, int32_t **ocol)
{
    const int32_t NONE = -1;
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t cap = ptr[n] > 16 ? 2 * (int64_t)ptr[n] : 32, len = 0;
    int32_t *rc = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *rl = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);   /* level of each kept entry */
    int32_t *lev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < n; ++j) lev[j] = NONE;
    rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        /* the row as a sorted linked list: head, nxt[], ending at NONE */
        int32_t head = NONE, tail = NONE;
        for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
            const int32_t c = col[q];
            lev[c] = 0;
            nxt[c] = NONE;
            if (tail == NONE) head = c; else nxt[tail] = c;
            tail = c;
        }
        for (int32_t k = head; k != NONE && k < i; k = nxt[k]) {
            /* the upper part of the kept row k */
            for (int64_t q = rp[k]; q < rp[k + 1]; ++q) {
                const int32_t j = rc[q];
                if (j <= k) continue;
                const int32_t l = lev[k] + rl[q] + 1;
                if (l > p) continue;
                if (lev[j] != NONE) {
                    if (l < lev[j]) lev[j] = l;
                    continue;
                }
                /* insert j after the last entry below it, searching from k */
                int32_t a = k;
                while (nxt[a] != NONE && nxt[a] < j) a = nxt[a];
                nxt[j] = nxt[a];
                nxt[a] = j;
                lev[j] = l;
            }
        }
        for (int32_t c = head; c != NONE; c = nxt[c]) {
            if (len == cap) {
                cap *= 2;
                rc = (int32_t *)realloc(rc, sizeof(int32_t) * (size_t)cap);
                rl = (int32_t *)realloc(rl, sizeof(int32_t) * (size_t)cap);
            }
            rc[len] = c;
            rl[len] = lev[c];
            ++len;
        }
        for (int32_t c = head; c != NONE; c = nxt[c]) lev[c] = NONE;
        rp[i + 1] = (int32_t)len;
    }
    free(rl);
    free(lev);
    free(nxt);
    *optr = rp;
    *ocol = rc;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* ILUT(p, tol), a local solver of RAS (Sec. 4.1, Fig. 31: default p = -1,   */
/* tol = 1e-3), as in Saad's book (the ILUT algorithm).  Row i:              */
/*   w = a_i*;  tau = tol * ||a_i*||_2;                                     */
/*   for k < i with w_k != 0, ascending: w_k = w_k / u_kk; if |w_k| < tau    */
/*     drop it, else w_j -= w_k u_kj for the entries j > k of U row k;       */
/*   drop the off-diagonal w_j with |w_j| < tau; keep the p largest of the   */
/*   L part and of the U part (ties to the lower column), and the diagonal.  */
/* p < 0: p_L and p_U are the numbers of entries row i of A has in each part.*/
/* The factor is returned in its own pattern (sorted rows): strict lower     */
/* part of L (unit diagonal implied), then U with its diagonal.              */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t c; double v; } or_cv;
static int cv_by_magnitude(const void *a, const void *b)
{
    const or_cv *x = (const or_cv *)a, *y = (const or_cv *)b;
    const double ax = fabs(x->v), ay = fabs(y->v);
    if (ax != ay) return ax > ay ? -1 : 1;
    return x->c < y->c ? -1 : (x->c > y->c);
}
static int cv_by_column(const void *a, const void *b)
{
    const or_cv *x = (const or_cv *)a, *y = (const or_cv *)b;
    return x->c < y->c ? -1 : (x->c > y->c);
}

int or_ilut(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, int32_t p, double tol,
            int32_t **optr, int32_t **ocol, double **olu, int32_t *bad_row)
{
    *bad_row = -1;
    int64_t cap = ptr[n] > 16 ? 2 * (int64_t)ptr[n] : 32, len = 0;
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *rc = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *rv = (double *)malloc(sizeof(double) * (size_t)cap);
    int32_t *udiag = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));   /* position of u_kk */
    double *w = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    char *nz = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_cv *buf = (or_cv *)malloc(sizeof(or_cv) * (size_t)(n > 0 ? n : 1));
    int32_t *lowers = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));   /* sorted */
    int st = OR_OK;
    rp[0] = 0;
    for (int32_t i = 0; i < n && st == OR_OK; ++i) {
        int32_t cnt = 0, plo = 0, pup = 0, nlow = 0;
        double nrm = 0.0;
        for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
            const int32_t c = col[q];
            w[c] = val[q];
            nz[c] = 1;
            list[cnt++] = c;
            nrm += val[q] * val[q];
            if (c < i) ++plo, lowers[nlow++] = c;
            else if (c > i) ++pup;
        }
        nrm = sqrt(nrm);
        const double tau = tol * nrm;
        if (p >= 0) plo = pup = p;
        /* elimination in ascending k over the row's lower entries, fill included:
         * a new lower entry j > k is inserted behind k in sorted position */
        for (int32_t t = 0; t < nlow; ++t) {
            const int32_t k = lowers[t];
            if (w[k] == 0.0) continue;
            w[k] = w[k] / rv[udiag[k]];
            if (fabs(w[k]) < tau) { w[k] = 0.0; continue; }
            for (int32_t q = udiag[k] + 1; q < rp[k + 1]; ++q) {
                const int32_t j = rc[q];
                if (!nz[j]) {
                    nz[j] = 1;
                    w[j] = 0.0;
                    list[cnt++] = j;
                    if (j < i) {
                        int32_t a = nlow++;
                        while (lowers[a - 1] > j) { lowers[a] = lowers[a - 1]; --a; }
                        lowers[a] = j;
                    }
                }
                w[j] = w[j] - w[k] * rv[q];
            }
        }
        /* dropping: the surviving lower entries go to buf[0 .. nl), the upper
         * ones to buf[n - nu .. n) */
        int32_t nl = 0, nu = 0;
        double diag = 0.0;
        for (int32_t a = 0; a < cnt; ++a) {
            const int32_t c = list[a];
            if (c == i) diag = w[c];
            else if (w[c] != 0.0 && fabs(w[c]) >= tau) {
                if (c < i) buf[nl++] = (or_cv){c, w[c]};
                else buf[n - 1 - nu++] = (or_cv){c, w[c]};
            }
        }
        /* the p largest of each part (ties to the lower column) */
        qsort(buf, (size_t)nl, sizeof(or_cv), cv_by_magnitude);
        qsort(buf + (n - nu), (size_t)nu, sizeof(or_cv), cv_by_magnitude);
        const int32_t ul = n - nu;              /* first upper entry */
        if (nl > plo) nl = plo;
        if (nu > pup) nu = pup;
        for (int32_t a = 0; a < nu; ++a) buf[nl + a] = buf[ul + a];   /* nl + a <= ul + a */
        for (int32_t a = 0; a < cnt; ++a) { w[list[a]] = 0.0; nz[list[a]] = 0; }
        if (!(diag != 0.0) || !isfinite(diag)) { *bad_row = i; st = OR_ZERO_PIVOT; break; }
        while (len + nl + nu + 1 > cap) {
            cap *= 2;
            rc = (int32_t *)realloc(rc, sizeof(int32_t) * (size_t)cap);
            rv = (double *)realloc(rv, sizeof(double) * (size_t)cap);
        }
        qsort(buf, (size_t)nl, sizeof(or_cv), cv_by_column);
        for (int32_t a = 0; a < nl; ++a) { rc[len] = buf[a].c; rv[len] = buf[a].v; ++len; }
        udiag[i] = (int32_t)len;
        rc[len] = i;
        rv[len] = diag;
        ++len;
        /* the kept upper entries, by column */
        qsort(buf + nl, (size_t)nu, sizeof(or_cv), cv_by_column);
        for (int32_t a = 0; a < nu; ++a) { rc[len] = buf[nl + a].c; rv[len] = buf[nl + a].v; ++len; }
        rp[i + 1] = (int32_t)len;
    }
    free(w); free(nz); free(list); free(buf); free(udiag); free(lowers);
    if (st != OR_OK) { free(rp); free(rc); free(rv); return st; }
    *optr = rp;
    *ocol = rc;
    *olu = rv;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Restricted additive Schwarz (Sec. 4.1, after Cai and Sarkis).             */
/* On a block matrix (bs > 1) rows are block rows and the local solver is    */
/* block ILU(level) (block ILU(0) on the level-of-fill block pattern).       */
/* part[i] in [0, nsub) assigns row i to a subdomain.  Subdomain s is        */
/* extended by `overlap` layers of the graph of A (layer m+1 = the columns   */
/* of the rows of layer m); its local matrix A_s keeps the entries of A      */
/* whose row and column both lie in the extended set, in ascending global    */
/* order; the local solver is ILU(level) of A_s.  Apply:                     */
/*   z_i = ( ILU(A_s)^{-1} r|ext(s) )_i  for s = part[i],                    */
/* i.e. every subdomain solves on its extended rows and only the rows it     */
/* owns are written (the restricted prolongation).                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n, nsub, bs;
    int32_t *part;           /* copy of the partition */
    int32_t *ext_ptr;        /* nsub + 1 offsets into ext */
    int32_t *ext;            /* extended rows of each subdomain, ascending */
    int32_t **lptr, **lcol;  /* local ILU(k) pattern per subdomain */
    double **llu;            /* local factors */
    double **ldinv;          /* inverted diagonal blocks (bs > 1) */
} or_ras;

void or_ras_free(or_ras *R)
{
    if (!R) return;
    for (int32_t s = 0; s < R->nsub; ++s) {
        free(R->lptr[s]);
        free(R->lcol[s]);
        free(R->llu[s]);
        free(R->ldinv[s]);
    }
    free(R->lptr);
    free(R->lcol);
    free(R->llu);
    free(R->ldinv);
    free(R->part);
    free(R->ext_ptr);
    free(R->ext);
    free(R);
}

/* local = 0: ILU(level) local solvers; local = 1: ILUT(ilut_p, ilut_tol)
 * (scalar matrices only) */
int or_ras_setup(int32_t n, int32_t bs, const int32_t *ptr, const int32_t *col, const double *val, int32_t nsub,
                 const int32_t *part, int32_t overlap, int32_t level, int32_t local, int32_t ilut_p,
                 double ilut_tol, or_ras **out, int32_t *bad_row)
{
    *out = NULL;
    *bad_row = -1;
    if (nsub < 1 || overlap < 0 || level < 0 || bs < 1 || bs > 8) return OR_INVALID;
    if (local != 0 && (local != 1 || bs != 1 || !(ilut_tol >= 0.0))) return OR_INVALID;
    const size_t b2 = (size_t)bs * bs;
    for (int32_t i = 0; i < n; ++i)
        if (part[i] < 0 || part[i] >= nsub) return OR_INVALID;
    or_ras *R = (or_ras *)calloc(1, sizeof(or_ras));
    R->n = n;
    R->nsub = nsub;
    R->bs = bs;
    R->part = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    memcpy(R->part, part, sizeof(int32_t) * (size_t)n);
    R->ext_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsub + 1));
    R->lptr = (int32_t **)calloc((size_t)nsub, sizeof(int32_t *));
    R->lcol = (int32_t **)calloc((size_t)nsub, sizeof(int32_t *));
    R->llu = (double **)calloc((size_t)nsub, sizeof(double *));
    R->ldinv = (double **)calloc((size_t)nsub, sizeof(double *));
    int64_t cap = n > 0 ? n : 1, len = 0;
    R->ext = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    char *in = (char *)malloc((size_t)(n > 0 ? n : 1));
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int st = OR_OK;
    R->ext_ptr[0] = 0;
    for (int32_t s = 0; s < nsub && st == OR_OK; ++s) {
        /* the extended set, by `overlap` rounds over the whole set */
        for (int32_t i = 0; i < n; ++i) in[i] = part[i] == s;
        for (int32_t m = 0; m < overlap; ++m) {
            char *add = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
            for (int32_t i = 0; i < n; ++i)
                if (in[i])
                    for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) add[col[q]] = 1;
            for (int32_t i = 0; i < n; ++i) in[i] = in[i] | add[i];
            free(add);
        }
        int32_t ns = 0;
        for (int32_t i = 0; i < n; ++i)
            if (in[i]) {
                if (len == cap) {
                    cap *= 2;
                    R->ext = (int32_t *)realloc(R->ext, sizeof(int32_t) * (size_t)cap);
                }
                loc[i] = ns++;
                R->ext[len++] = i;
            }
        R->ext_ptr[s + 1] = (int32_t)len;
        const int32_t *er = R->ext + R->ext_ptr[s];
        /* local matrix A_s */
        int32_t *ap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns + 1));
        int64_t nz = 0;
        for (int32_t a = 0; a < ns; ++a)
            for (int32_t q = ptr[er[a]]; q < ptr[er[a] + 1]; ++q) nz += in[col[q]] ? 1 : 0;
        int32_t *ac = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nz > 0 ? nz : 1));
        double *av = (double *)malloc(sizeof(double) * b2 * (size_t)(nz > 0 ? nz : 1));
        ap[0] = 0;
        nz = 0;
        for (int32_t a = 0; a < ns; ++a) {
            for (int32_t q = ptr[er[a]]; q < ptr[er[a] + 1]; ++q)
                if (in[col[q]]) {
                    ac[nz] = loc[col[q]];
                    memcpy(av + (size_t)nz * b2, val + (size_t)q * b2, sizeof(double) * b2);
                    ++nz;
                }
            ap[a + 1] = (int32_t)nz;
        }
        if (local == 1) {
            /* ILUT: the factor and its pattern come from the values */
            int32_t bad = -1;
            st = or_ilut(ns, ap, ac, av, ilut_p, ilut_tol, &R->lptr[s], &R->lcol[s], &R->llu[s], &bad);
            if (st != OR_OK) *bad_row = bad >= 0 ? er[bad] : -1;
            free(ap);
            free(ac);
            free(av);
            continue;
        }
        /* the ILU(level) pattern of A_s, with A_s's values and zeros at fill */
        int32_t *kp, *kc;
        or_iluk_symbolic(ns, ap, ac, level, &kp, &kc);
        double *kv = (double *)malloc(sizeof(double) * b2 * (size_t)(kp[ns] > 0 ? kp[ns] : 1));
        for (int32_t a = 0; a < ns; ++a) {
            int32_t q = ap[a];
            for (int32_t t = kp[a]; t < kp[a + 1]; ++t) {
                while (q < ap[a + 1] && ac[q] < kc[t]) ++q;
                const int hit = q < ap[a + 1] && ac[q] == kc[t];
                for (size_t e = 0; e < b2; ++e) kv[(size_t)t * b2 + e] = hit ? av[(size_t)q * b2 + e] : 0.0;
            }
        }
        double *lu = (double *)malloc(sizeof(double) * b2 * (size_t)(kp[ns] > 0 ? kp[ns] : 1));
        int32_t bad = -1;
        if (bs == 1) {
            st = or_ilu0(ns, kp, kc, kv, lu, &bad);
        } else {
            R->ldinv[s] = (double *)malloc(sizeof(double) * b2 * (size_t)(ns > 0 ? ns : 1));
            st = or_bilu0(ns, bs, kp, kc, kv, lu, R->ldinv[s], &bad);
        }
        if (st != OR_OK) *bad_row = bad >= 0 ? er[bad] : -1;
        R->lptr[s] = kp;
        R->lcol[s] = kc;
        R->llu[s] = lu;
        free(ap);
        free(ac);
        free(av);
        free(kv);
    }
    free(in);
    free(loc);
    if (st != OR_OK) {
        or_ras_free(R);
        return st;
    }
    *out = R;
    return OR_OK;
}

void or_ras_apply(const or_ras *R, const double *r, double *z)
{
    const int32_t bs = R->bs;
    for (int32_t s = 0; s < R->nsub; ++s) {
        const int32_t *er = R->ext + R->ext_ptr[s];
        const int32_t ns = R->ext_ptr[s + 1] - R->ext_ptr[s];
        double *rl = (double *)malloc(sizeof(double) * (size_t)bs * (ns > 0 ? ns : 1));
        double *zl = (double *)malloc(sizeof(double) * (size_t)bs * (ns > 0 ? ns : 1));
        for (int32_t a = 0; a < ns; ++a)
            for (int32_t c = 0; c < bs; ++c) rl[(size_t)a * bs + c] = r[(size_t)er[a] * bs + c];
        if (bs == 1) or_ilu0_solve(ns, R->lptr[s], R->lcol[s], R->llu[s], rl, zl);
        else or_bilu0_solve(ns, bs, R->lptr[s], R->lcol[s], R->llu[s], R->ldinv[s], rl, zl);
        for (int32_t a = 0; a < ns; ++a)
            if (R->part[er[a]] == s)
                for (int32_t c = 0; c < bs; ++c) z[(size_t)er[a] * bs + c] = zl[(size_t)a * bs + c];
        free(rl);
        free(zl);
    }
}

/* Sizes of the block-diagonal matrix that stacks the local problems in
 * subdomain order: extended rows and stored entries. */
void or_ras_sizes(const or_ras *R, int32_t *next, int64_t *nnz)
{
    *next = R->ext_ptr[R->nsub];
    int64_t t = 0;
    for (int32_t s = 0; s < R->nsub; ++s) t += R->lptr[s][R->ext_ptr[s + 1] - R->ext_ptr[s]];
    *nnz = t;
}

/* That matrix: global row of every extended row, its pattern (columns
 * numbered in the stacked order) and the factor values. */
void or_ras_export(const or_ras *R, int32_t *gidx, int32_t *ptr, int32_t *col, double *lu)
{
    const size_t b2 = (size_t)R->bs * R->bs;
    int64_t q = 0;
    ptr[0] = 0;
    for (int32_t s = 0; s < R->nsub; ++s) {
        const int32_t base = R->ext_ptr[s], ns = R->ext_ptr[s + 1] - base;
        for (int32_t a = 0; a < ns; ++a) {
            gidx[base + a] = R->ext[base + a];
            for (int32_t t = R->lptr[s][a]; t < R->lptr[s][a + 1]; ++t, ++q) {
                col[q] = base + R->lcol[s][t];
                memcpy(lu + (size_t)q * b2, R->llu[s] + (size_t)t * b2, sizeof(double) * b2);
            }
            ptr[base + a + 1] = (int32_t)q;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Algebraic multigrid (Sec. 4.2: Alg. 3 setup, Alg. 4 V-cycle, Eq. 4).      */
/* Setup of level l, in Alg. 3's order:                                      */
/*  1. strength: j strongly influences i (j in S_i) when j != i and          */
/*     -a_ij >= theta max_{k != i} (-a_ik) (none when that max is <= 0);      */
/*  2. coarse points by the Ruge-Stueben first pass: lambda_i = number of    */
/*     points that i strongly influences; repeatedly the undecided point of  */
/*     largest lambda (ties: lowest index) becomes C, the undecided points   */
/*     that it strongly influences become F, lambda_k + 1 for the undecided  */
/*     k in S_j of each new F point j and lambda_k - 1 for the undecided k   */
/*     in S_i of the new C point i; points with neither strong connections   */
/*     nor points depending on them are F from the start;                    */
/*  3. direct interpolation: C points copy their coarse value; an F point i  */
/*     takes w_ik = -alpha_i a_ik / a_ii over its strong C neighbours k with */
/*     a_ik < 0 and -beta_i a_ik / a_ii over those with a_ik > 0, where      */
/*     alpha_i (beta_i) is the sum of all negative (positive) off-diagonal   */
/*     a_ij over the sum of those of its strong C neighbours; without a      */
/*     positive strong C coupling the positive couplings join a_ii;          */
/*  4. R = P^T;  5. A_{l+1} = R A_l P (Eq. 4);                               */
/*  6. smoother: l1-Jacobi, x <- x + (b - A x) / d with d_i = sum_j |a_ij|, */
/*     or hybrid Gauss-Seidel (Fig. 34's relaxation: Gauss-Seidel inside a  */
/*     process, Jacobi between processes), read on one device as chunks of */
/*     32 consecutive rows: forward sweeps before the coarse correction,    */
/*     backward sweeps after it, so that the V-cycle stays symmetric.       */
/* Levels stop at <= max_coarse rows, at max_levels, or when coarsening      */
/* stalls; the coarsest system is solved with a dense inverse.               */
/* V-cycle from x = 0 (Alg. 4): nu smoothing sweeps, residual, restriction,  */
/* the next level, prolongation and correction, nu smoothing sweeps.         */
/* ------------------------------------------------------------------------ */
#define OR_AMG_MAXLEV 16

typedef struct {
    int32_t n, m;            /* rows, columns */
    int32_t *ptr, *col;
    double *val;
} or_csr;

#define OR_HGS_CHUNK 32

typedef struct {
    int32_t nlev, nu, smoother;  /* smoother: 0 l1-Jacobi, 1 hybrid Gauss-Seidel */
    or_csr A[OR_AMG_MAXLEV], P[OR_AMG_MAXLEV], R[OR_AMG_MAXLEV];
    double *d[OR_AMG_MAXLEV];    /* l1-Jacobi diagonal */
    int32_t *cidx[OR_AMG_MAXLEV]; /* coarse index of each point of level l, -1 for F */
    double *cinv;                /* dense inverse of the coarsest matrix, row-major */
} or_amg;

static void csr_free(or_csr *M)
{
    free(M->ptr);
    free(M->col);
    free(M->val);
    memset(M, 0, sizeof(*M));
}

/* C = A B (both CSR, B with A.m rows), rows accumulated in a dense row of
 * B.m entries, columns then sorted. */
static void csr_mul(const or_csr *A, const or_csr *B, or_csr *C)
{
    double *acc = (double *)calloc((size_t)(B->m > 0 ? B->m : 1), sizeof(double));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(B->m > 0 ? B->m : 1));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(B->m > 0 ? B->m : 1));
    for (int32_t c = 0; c < B->m; ++c) mark[c] = -1;
    int64_t cap = 16, len = 0;
    C->n = A->n;
    C->m = B->m;
    C->ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->n + 1));
    C->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    C->val = (double *)malloc(sizeof(double) * (size_t)cap);
    C->ptr[0] = 0;
    for (int32_t i = 0; i < A->n; ++i) {
        int32_t nc = 0;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            const int32_t j = A->col[p];
            for (int32_t q = B->ptr[j]; q < B->ptr[j + 1]; ++q) {
                const int32_t c = B->col[q];
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols[nc++] = c;
                }
                acc[c] = acc[c] + A->val[p] * B->val[q];
            }
        }
        /* insertion sort of the row's columns (rows are short) */
        for (int32_t a = 1; a < nc; ++a) {
            const int32_t v = cols[a];
            int32_t b = a - 1;
            while (b >= 0 && cols[b] > v) { cols[b + 1] = cols[b]; --b; }
            cols[b + 1] = v;
        }
        while (len + nc > cap) {
            cap *= 2;
            C->col = (int32_t *)realloc(C->col, sizeof(int32_t) * (size_t)cap);
            C->val = (double *)realloc(C->val, sizeof(double) * (size_t)cap);
        }
        for (int32_t a = 0; a < nc; ++a) {
            C->col[len] = cols[a];
            C->val[len] = acc[cols[a]];
            ++len;
        }
        C->ptr[i + 1] = (int32_t)len;
    }
    free(acc);
    free(mark);
    free(cols);
}

static void csr_transpose(const or_csr *A, or_csr *T)
{
    T->n = A->m;
    T->m = A->n;
    const int64_t nnz = A->ptr[A->n];
    T->ptr = (int32_t *)calloc((size_t)(A->m + 1), sizeof(int32_t));
    T->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    T->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t p = 0; p < nnz; ++p) T->ptr[A->col[p] + 1]++;
    for (int32_t c = 0; c < A->m; ++c) T->ptr[c + 1] += T->ptr[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->m > 0 ? A->m : 1));
    memcpy(fill, T->ptr, sizeof(int32_t) * (size_t)A->m);
    for (int32_t i = 0; i < A->n; ++i)          /* rows in order: columns of T come out sorted */
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            const int32_t q = fill[A->col[p]]++;
            T->col[q] = i;
            T->val[q] = A->val[p];
        }
    free(fill);
}

/* binary max-heap of (lambda, -index) with stale entries skipped on pop */
typedef struct { int32_t lam, idx; } or_hent;
static int hent_less(or_hent a, or_hent b) { return a.lam < b.lam || (a.lam == b.lam && a.idx > b.idx); }
static void heap_push(or_hent **h, int64_t *len, int64_t *cap, or_hent e)
{
    if (*len == *cap) {
        *cap *= 2;
        *h = (or_hent *)realloc(*h, sizeof(or_hent) * (size_t)*cap);
    }
    int64_t i = (*len)++;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (!hent_less((*h)[p], e)) break;
        (*h)[i] = (*h)[p];
        i = p;
    }
    (*h)[i] = e;
}
static or_hent heap_pop(or_hent *h, int64_t *len)
{
    const or_hent top = h[0];
    const or_hent last = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *len) break;
        if (c + 1 < *len && hent_less(h[c], h[c + 1])) ++c;
        if (!hent_less(last, h[c])) break;
        h[i] = h[c];
        i = c;
    }
    if (*len > 0) h[i] = last;
    return top;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used counter-based: the
 * k-th output of the generator started from state 0, i.e. its finaliser
 * applied to (k + 1) times the golden-ratio increment. */
uint64_t or_splitmix64(uint64_t k)
{
    uint64_t z = (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* the PMIS weight of point i on level l: uniform in [0, 1), 53 bits */
static double pmis_weight(int32_t level, int32_t i)
{
    return (double)(or_splitmix64(((uint64_t)(uint32_t)level << 32) | (uint32_t)i) >> 11) * 0x1.0p-53;
}

/* PMIS coarsening (De Sterck, Yang and Heys, SIAM J. Matrix Anal. Appl.
 * 2006), one of the coarsenings Sec. 4.2 names.  S (sp, sc): the points each
 * point strongly depends on; ST (tp, tc): those it strongly influences.  The
 * measure of i is lambda_i = |S_i^T| + w_i.  Points that influence no point
 * are F from the start.  Then, in rounds until no point is undecided: every
 * undecided point whose measure exceeds that of every undecided point of
 * S_i and S_i^T (the states at the start of the round) becomes C; then every
 * undecided point that strongly depends on a C point becomes F.  st[i]:
 * 1 C, 2 F.  Returns the number of rounds. */
int32_t or_pmis(int32_t n, const int32_t *sp, const int32_t *sc, const int32_t *tp, const int32_t *tc,
                const double *w, char *st)
{
    double *lam = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    char *old = (char *)malloc((size_t)(n > 0 ? n : 1));
    int32_t und = 0;
    for (int32_t i = 0; i < n; ++i) {
        lam[i] = (double)(tp[i + 1] - tp[i]) + w[i];
        st[i] = tp[i + 1] == tp[i] ? 2 : 0;
        und += st[i] == 0;
    }
    int32_t rounds = 0;
    while (und > 0) {
        ++rounds;
        memcpy(old, st, (size_t)n);
        for (int32_t i = 0; i < n; ++i) {
            if (old[i] != 0) continue;
            int top = 1;
            for (int32_t q = sp[i]; q < sp[i + 1] && top; ++q)
                if (old[sc[q]] == 0 && !(lam[i] > lam[sc[q]])) top = 0;
            for (int32_t q = tp[i]; q < tp[i + 1] && top; ++q)
                if (old[tc[q]] == 0 && !(lam[i] > lam[tc[q]])) top = 0;
            if (top) st[i] = 1;
        }
        for (int32_t j = 0; j < n; ++j) {
            if (st[j] != 0) continue;
            for (int32_t q = sp[j]; q < sp[j + 1]; ++q)
                if (st[sc[q]] == 1) {
                    st[j] = 2;
                    break;
                }
        }
        und = 0;
        for (int32_t i = 0; i < n; ++i) und += st[i] == 0;
    }
    free(lam);
    free(old);
    return rounds;
}

/* one level of Alg. 3: P (n x nc) from A and the coarse index of every
 * point (-1 for F, into cidx_out[n]); coarsen 0: the Ruge-Stueben first
 * pass, 1: PMIS with the weights of this level; returns nc */
static int32_t amg_coarsen(const or_csr *A, double theta, int32_t coarsen, int32_t level, or_csr *P,
                           int32_t *cidx_out)
{
    const int32_t n = A->n;
    /* 1. strength */
    int32_t *sp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *sc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->ptr[n] > 0 ? A->ptr[n] : 1));
    sp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double mx = 0.0;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
            if (A->col[p] != i && -A->val[p] > mx) mx = -A->val[p];
        int32_t k = sp[i];
        if (mx > 0.0)
            for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
                if (A->col[p] != i && -A->val[p] >= theta * mx) sc[k++] = A->col[p];
        sp[i + 1] = k;
    }
    /* S^T: the points each point strongly influences */
    or_csr S = {n, n, sp, sc, NULL}, ST;
    S.val = (double *)calloc((size_t)(sp[n] > 0 ? sp[n] : 1), sizeof(double));
    csr_transpose(&S, &ST);
    /* 2. the C/F splitting */
    enum { U = 0, CPT = 1, FPT = 2 };
    int32_t *lam = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    char *st = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (coarsen == 1) {
        double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        for (int32_t i = 0; i < n; ++i) w[i] = pmis_weight(level, i);
        or_pmis(n, sp, sc, ST.ptr, ST.col, w, st);
        free(w);
    } else {
        int64_t hcap = n > 0 ? 2 * (int64_t)n : 2, hlen = 0;
        or_hent *heap = (or_hent *)malloc(sizeof(or_hent) * (size_t)hcap);
        for (int32_t i = 0; i < n; ++i) {
            lam[i] = ST.ptr[i + 1] - ST.ptr[i];
            if (lam[i] == 0 && sp[i + 1] == sp[i]) st[i] = FPT;
            else heap_push(&heap, &hlen, &hcap, (or_hent){lam[i], i});
        }
        while (hlen > 0) {
            const or_hent e = heap_pop(heap, &hlen);
            const int32_t i = e.idx;
            if (st[i] != U || e.lam != lam[i]) continue;
            st[i] = CPT;
            for (int32_t q = ST.ptr[i]; q < ST.ptr[i + 1]; ++q) {
                const int32_t j = ST.col[q];
                if (st[j] != U) continue;
                st[j] = FPT;
                for (int32_t r = sp[j]; r < sp[j + 1]; ++r) {
                    const int32_t k = sc[r];
                    if (st[k] == U) {
                        lam[k] += 1;
                        heap_push(&heap, &hlen, &hcap, (or_hent){lam[k], k});
                    }
                }
            }
            for (int32_t r = sp[i]; r < sp[i + 1]; ++r) {
                const int32_t k = sc[r];
                if (st[k] == U) {
                    lam[k] -= 1;
                    heap_push(&heap, &hlen, &hcap, (or_hent){lam[k], k});
                }
            }
        }
        free(heap);
    }
    /* coarse numbering */
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t nc = 0;
    for (int32_t i = 0; i < n; ++i) cidx[i] = st[i] == CPT ? nc++ : -1;
    /* 3. direct interpolation */
    P->n = n;
    P->m = nc;
    P->ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    P->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sp[n] + n + 1));
    P->val = (double *)malloc(sizeof(double) * (size_t)(sp[n] + n + 1));
    int64_t len = 0;
    P->ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (st[i] == CPT) {
            P->col[len] = cidx[i];
            P->val[len] = 1.0;
            ++len;
        } else {
            double aii = 0.0, neg = 0.0, pos = 0.0, negc = 0.0, posc = 0.0;
            for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                const double v = A->val[p];
                if (A->col[p] == i) aii = v;
                else if (v < 0.0) neg += v;
                else pos += v;
            }
            for (int32_t r = sp[i]; r < sp[i + 1]; ++r) {
                if (st[sc[r]] != CPT) continue;
                /* the value a_ik of this strong C neighbour */
                for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
                    if (A->col[p] == sc[r]) {
                        if (A->val[p] < 0.0) negc += A->val[p];
                        else posc += A->val[p];
                    }
            }
            double diag = aii, beta = 0.0;
            if (posc == 0.0) diag += pos;
            else beta = pos / posc;
            const double alpha = negc != 0.0 ? neg / negc : 0.0;
            /* strong C neighbours in ascending column order = ascending coarse index */
            for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                const int32_t k = A->col[p];
                if (k == i || st[k] != CPT) continue;
                int strong = 0;
                for (int32_t r = sp[i]; r < sp[i + 1]; ++r) strong |= sc[r] == k;
                if (!strong) continue;
                P->col[len] = cidx[k];
                P->val[len] = -(A->val[p] < 0.0 ? alpha : beta) * A->val[p] / diag;
                ++len;
            }
        }
        P->ptr[i + 1] = (int32_t)len;
    }
    memcpy(cidx_out, cidx, sizeof(int32_t) * (size_t)n);
    free(lam);
    free(st);
    free(cidx);
    free(S.val);
    csr_free(&ST);
    free(sp);
    free(sc);
    return nc;
}

/* inverse of a dense n x n row-major matrix by Gauss-Jordan elimination with
 * partial pivoting; returns 0 on a zero or non-finite pivot */
static int dense_inverse(int32_t n, const double *a, double *inv)
{
    double *m = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    memcpy(m, a, sizeof(double) * (size_t)n * n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) inv[(size_t)i * n + j] = i == j ? 1.0 : 0.0;
    int ok = 1;
    for (int32_t c = 0; c < n && ok; ++c) {
        int32_t p = c;
        for (int32_t r = c + 1; r < n; ++r)
            if (fabs(m[(size_t)r * n + c]) > fabs(m[(size_t)p * n + c])) p = r;
        const double piv = m[(size_t)p * n + c];
        if (!(piv != 0.0) || !isfinite(piv)) { ok = 0; break; }
        if (p != c)
            for (int32_t j = 0; j < n; ++j) {
                double t = m[(size_t)c * n + j]; m[(size_t)c * n + j] = m[(size_t)p * n + j]; m[(size_t)p * n + j] = t;
                t = inv[(size_t)c * n + j]; inv[(size_t)c * n + j] = inv[(size_t)p * n + j]; inv[(size_t)p * n + j] = t;
            }
        for (int32_t j = 0; j < n; ++j) {
            m[(size_t)c * n + j] /= piv;
            inv[(size_t)c * n + j] /= piv;
        }
        for (int32_t r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = m[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int32_t j = 0; j < n; ++j) {
                m[(size_t)r * n + j] -= f * m[(size_t)c * n + j];
                inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
            }
        }
    }
    free(m);
    return ok;
}

void or_amg_free(or_amg *M)
{
    if (!M) return;
    for (int32_t l = 0; l < M->nlev; ++l) {
        csr_free(&M->A[l]);
        csr_free(&M->P[l]);
        csr_free(&M->R[l]);
        free(M->d[l]);
        free(M->cidx[l]);
    }
    free(M->cinv);
    free(M);
}

/* One hybrid Gauss-Seidel sweep: the rows are cut into chunks of `chunk`
 * consecutive rows; inside a chunk, rows are taken in increasing order
 * (backward: decreasing) and each reads the newest values of its chunk,
 * while values of other chunks are those of x (Jacobi between chunks):
 *   out_i = (b_i - sum_{j != i} a_ij v_j) / a_ii,
 * v_j = out_j for j in i's chunk and already taken, x_j otherwise.
 * chunk = 1 is Jacobi, chunk >= n plain Gauss-Seidel.  Returns OR_ZERO_PIVOT
 * (out untouched from that row on) at a row without a nonzero diagonal. */
int or_hgs_sweep(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const double *b,
                 const double *x, int32_t chunk, int32_t backward, double *out)
{
    if (chunk < 1) return OR_INVALID;
    for (int32_t i = 0; i < n; ++i) out[i] = x[i];
    for (int32_t c0 = 0; c0 < n; c0 += chunk) {
        const int32_t c1 = c0 + chunk < n ? c0 + chunk : n;
        for (int32_t t = 0; t < c1 - c0; ++t) {
            const int32_t i = backward ? c1 - 1 - t : c0 + t;
            double s = b[i], d = 0.0;
            for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
                const int32_t j = col[p];
                if (j == i) {
                    d = val[p];
                    continue;
                }
                s -= val[p] * (j >= c0 && j < c1 ? out[j] : x[j]);
            }
            if (d == 0.0) return OR_ZERO_PIVOT;
            out[i] = s / d;
        }
    }
    return OR_OK;
}

int or_amg_setup(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, double theta,
                 int32_t max_levels, int32_t max_coarse, int32_t nu, int32_t smoother, int32_t coarsen,
                 or_amg **out)
{
    *out = NULL;
    if (n < 1 || max_levels < 1 || max_levels > OR_AMG_MAXLEV || max_coarse < 1 || nu < 1 || !(theta >= 0.0) ||
        smoother < 0 || smoother > 1 || coarsen < 0 || coarsen > 1)
        return OR_INVALID;
    or_amg *M = (or_amg *)calloc(1, sizeof(or_amg));
    M->nu = nu;
    M->smoother = smoother;
    or_csr *A0 = &M->A[0];
    A0->n = A0->m = n;
    A0->ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    A0->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ptr[n] > 0 ? ptr[n] : 1));
    A0->val = (double *)malloc(sizeof(double) * (size_t)(ptr[n] > 0 ? ptr[n] : 1));
    memcpy(A0->ptr, ptr, sizeof(int32_t) * (size_t)(n + 1));
    memcpy(A0->col, col, sizeof(int32_t) * (size_t)ptr[n]);
    memcpy(A0->val, val, sizeof(double) * (size_t)ptr[n]);
    int32_t l = 0;
    for (;;) {
        const or_csr *A = &M->A[l];
        M->d[l] = (double *)malloc(sizeof(double) * (size_t)A->n);
        int nodiag = 0;
        for (int32_t i = 0; i < A->n; ++i) {
            double s = 0.0, dg = 0.0;
            for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                s += fabs(A->val[p]);
                if (A->col[p] == i) dg = A->val[p];
            }
            M->d[l][i] = s;
            nodiag |= dg == 0.0;
        }
        if (smoother == 1 && nodiag) {   /* Gauss-Seidel divides by a_ii */
            M->nlev = l + 1;
            or_amg_free(M);
            return OR_ZERO_PIVOT;
        }
        if (A->n <= max_coarse || l + 1 >= max_levels) break;
        or_csr P;
        M->cidx[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)A->n);
        const int32_t nc = amg_coarsen(A, theta, coarsen, l, &P, M->cidx[l]);
        if (nc == 0 || nc >= A->n) {
            csr_free(&P);
            break;
        }
        M->P[l] = P;
        csr_transpose(&M->P[l], &M->R[l]);
        or_csr AP;
        csr_mul(A, &M->P[l], &AP);
        csr_mul(&M->R[l], &AP, &M->A[l + 1]);
        csr_free(&AP);
        ++l;
    }
    M->nlev = l + 1;
    /* dense inverse of the coarsest matrix */
    const or_csr *C = &M->A[l];
    double *dense = (double *)calloc((size_t)C->n * C->n, sizeof(double));
    for (int32_t i = 0; i < C->n; ++i)
        for (int32_t p = C->ptr[i]; p < C->ptr[i + 1]; ++p) dense[(size_t)i * C->n + C->col[p]] = C->val[p];
    M->cinv = (double *)malloc(sizeof(double) * (size_t)C->n * C->n);
    const int ok = dense_inverse(C->n, dense, M->cinv);
    free(dense);
    if (!ok) {
        or_amg_free(M);
        return OR_ZERO_PIVOT;
    }
    *out = M;
    return OR_OK;
}

static void csr_mv(const or_csr *A, const double *x, double *y)
{
    for (int32_t i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) s += A->val[p] * x[A->col[p]];
        y[i] = s;
    }
}

/* x <- x + (b - A x) / d (Jacobi: every row reads the old x) */
static void l1_jacobi(const or_csr *A, const double *d, const double *b, double *x, double *t)
{
    csr_mv(A, x, t);
    for (int32_t i = 0; i < A->n; ++i) t[i] = b[i] - t[i];
    for (int32_t i = 0; i < A->n; ++i) x[i] = x[i] + t[i] / d[i];
}

static void amg_vcycle(const or_amg *M, int32_t l, const double *b, double *x)
{
    const or_csr *A = &M->A[l];
    const int32_t n = A->n;
    if (l == M->nlev - 1) {
        for (int32_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int32_t j = 0; j < n; ++j) s += M->cinv[(size_t)i * n + j] * b[j];
            x[i] = s;
        }
        return;
    }
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    const int32_t nc = M->A[l + 1].n;
    double *bc = (double *)malloc(sizeof(double) * (size_t)nc);
    double *xc = (double *)malloc(sizeof(double) * (size_t)nc);
    if (M->smoother == 1) {
        /* pre-smoothing from x = 0: forward hybrid Gauss-Seidel sweeps */
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        for (int32_t s = 0; s < M->nu; ++s) {
            or_hgs_sweep(n, A->ptr, A->col, A->val, b, x, OR_HGS_CHUNK, 0, t);
            memcpy(x, t, sizeof(double) * (size_t)n);
        }
    } else {
        /* pre-smoothing from x = 0: the first sweep is x = b / d */
        for (int32_t i = 0; i < n; ++i) x[i] = b[i] / M->d[l][i];
        for (int32_t s = 1; s < M->nu; ++s) l1_jacobi(A, M->d[l], b, x, t);
    }
    csr_mv(A, x, t);
    for (int32_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
    csr_mv(&M->R[l], t, bc);
    amg_vcycle(M, l + 1, bc, xc);
    csr_mv(&M->P[l], xc, t);
    for (int32_t i = 0; i < n; ++i) x[i] = x[i] + t[i];
    for (int32_t s = 0; s < M->nu; ++s) {
        if (M->smoother == 1) {     /* backward sweeps: the adjoint of the forward ones */
            or_hgs_sweep(n, A->ptr, A->col, A->val, b, x, OR_HGS_CHUNK, 1, t);
            memcpy(x, t, sizeof(double) * (size_t)n);
        } else {
            l1_jacobi(A, M->d[l], b, x, t);
        }
    }
    free(t);
    free(bc);
    free(xc);
}

void or_amg_apply(const or_amg *M, const double *r, double *z) { amg_vcycle(M, 0, r, z); }

int32_t or_amg_nlevels(const or_amg *M) { return M->nlev; }

/* sizes of level l: rows of A_l, entries of A_l, entries of P_l (0 on the coarsest) */
void or_amg_level_sizes(const or_amg *M, int32_t l, int32_t *n, int64_t *nnz_a, int64_t *nnz_p)
{
    *n = M->A[l].n;
    *nnz_a = M->A[l].ptr[M->A[l].n];
    *nnz_p = l + 1 < M->nlev ? M->P[l].ptr[M->P[l].n] : 0;
}

/* coarse index of every point of level l (-1 for F); l below the coarsest */
void or_amg_cidx(const or_amg *M, int32_t l, int32_t *cidx)
{
    memcpy(cidx, M->cidx[l], sizeof(int32_t) * (size_t)M->A[l].n);
}

/* copies of A_l and (if l is not the coarsest) P_l; any pointer may be NULL */
void or_amg_level(const or_amg *M, int32_t l, int32_t *aptr, int32_t *acol, double *aval, int32_t *pptr,
                  int32_t *pcol, double *pval)
{
    const or_csr *A = &M->A[l];
    if (aptr) memcpy(aptr, A->ptr, sizeof(int32_t) * (size_t)(A->n + 1));
    if (acol) memcpy(acol, A->col, sizeof(int32_t) * (size_t)A->ptr[A->n]);
    if (aval) memcpy(aval, A->val, sizeof(double) * (size_t)A->ptr[A->n]);
    if (l + 1 < M->nlev) {
        const or_csr *P = &M->P[l];
        if (pptr) memcpy(pptr, P->ptr, sizeof(int32_t) * (size_t)(P->n + 1));
        if (pcol) memcpy(pcol, P->col, sizeof(int32_t) * (size_t)P->ptr[P->n]);
        if (pval) memcpy(pval, P->val, sizeof(double) * (size_t)P->ptr[P->n]);
    }
}

/* ------------------------------------------------------------------------ */
/* Preconditioner object (Sec. 3, Fig. 29: setup / solve / destroy).         */
/* ------------------------------------------------------------------------ */
typedef int (*or_apply_fn)(void *user, int64_t n, const double *r, double *z);

enum { OR_PC_NONE = 0, OR_PC_ILU0 = 1, OR_PC_BILU0 = 2, OR_PC_CPR = 3, OR_PC_CALLBACK = 4, OR_PC_RAS = 5,
       OR_PC_AMG = 6 };

typedef struct {
    int32_t type;
    int32_t mixed;              /* 1: FP32 factors and FP32 applies */
    /* scalar ILU(0): on A (type ILU0) or on App' (type CPR pressure stage) */
    int32_t n;
    const int32_t *ptr, *col;
    const double *lu;
    const float *lu32;
    /* block ILU(0) (type BILU0, and the second stage of CPR) */
    int32_t nb, bs;
    const int32_t *bptr, *bcol;
    const double *blu, *bdinv;
    const float *blu32, *bdinv32;
    /* CPR */
    const or_mat *A;
    const double *w;            /* nb x (bs-1) quasi-IMPES weights */
    or_apply_fn pstage;         /* optional pressure-stage override */
    void *pstage_user;
    /* plain callback preconditioner */
    or_apply_fn fn;
    void *user;
    /* CPR form: 0 PF (Alg. 6, read as below), 1 FP (Alg. 5), 2 FPF (Alg. 7),
     * 3 FFPF (Alg. 8) */
    int32_t form;
    /* restricted additive Schwarz (type RAS; with type CPR, the F stage) */
    const or_ras *ras;
    /* algebraic multigrid V-cycle (type AMG) */
    const or_amg *amg;
} or_pc;

/* One stage of a CPR-like preconditioner on a right-hand side v:
 * 'F' = R(A)^{-1} v (block ILU(0) of the full system),
 * 'P' = Pi_p M_p^{-1} (Pi_r v) (quasi-IMPES restriction, pressure solve by
 * ILU(0) of App' or the pstage callback, prolongation). */
static int cpr_stage(const or_pc *M, char kind, int64_t n, const double *v, double *out)
{
    const int32_t nb = M->nb, bs = M->bs;
    if (kind == 'F') {
        if (M->ras) or_ras_apply(M->ras, v, out);
        else if (M->mixed) or_bilu0_solve_f32(nb, bs, M->bptr, M->bcol, M->blu32, M->bdinv32, v, out);
        else or_bilu0_solve(nb, bs, M->bptr, M->bcol, M->blu, M->bdinv, v, out);
        return OR_OK;
    }
    double *rp = (double *)malloc(sizeof(double) * (size_t)nb);
    double *zp = (double *)malloc(sizeof(double) * (size_t)nb);
    int st = OR_OK;
    or_qimpes_restrict(nb, bs, M->w, v, rp);
    if (M->pstage) st = M->pstage(M->pstage_user, nb, rp, zp);
    else if (M->amg) or_amg_apply(M->amg, rp, zp);
    else if (M->mixed) or_ilu0_solve_f32(M->n, M->ptr, M->col, M->lu32, rp, zp);
    else or_ilu0_solve(M->n, M->ptr, M->col, M->lu, rp, zp);
    or_prolong(nb, bs, zp, out);
    (void)n;
    free(rp);
    free(zp);
    return st;
}

static int64_t pc_len(const or_pc *M, int64_t n) { (void)M; return n; }

/* z = M^{-1} r */
int or_pc_apply(const or_pc *M, int64_t n, const double *r, double *z)
{
    (void)pc_len;
    switch (M ? M->type : OR_PC_NONE) {
    case OR_PC_NONE:
        memcpy(z, r, sizeof(double) * (size_t)n);
        return OR_OK;
    case OR_PC_ILU0:
        if (M->mixed) or_ilu0_solve_f32(M->n, M->ptr, M->col, M->lu32, r, z);
        else or_ilu0_solve(M->n, M->ptr, M->col, M->lu, r, z);
        return OR_OK;
    case OR_PC_BILU0:
        if (M->mixed) or_bilu0_solve_f32(M->nb, M->bs, M->bptr, M->bcol, M->blu32, M->bdinv32, r, z);
        else or_bilu0_solve(M->nb, M->bs, M->bptr, M->bcol, M->blu, M->bdinv, r, z);
        return OR_OK;
    case OR_PC_CALLBACK:
        return M->fn(M->user, n, r, z);
    case OR_PC_RAS:
        or_ras_apply(M->ras, r, z);
        return OR_OK;
    case OR_PC_AMG:
        or_amg_apply(M->amg, r, z);
        return OR_OK;
    case OR_PC_CPR: {
        /* CPR-like preconditioners, Algs. 5-8, each step in the printed
         * order: the first stage maps f to x; every later stage forms
         * r = f - A x and adds its correction, x = x + stage(r).  Alg. 6 is
         * garbled as printed (its second step discards the first, its last
         * uses f) and is read as  x = P f;  r = f - A x;  x = x + F r. */
        static const char *forms[4] = {"PF", "FP", "FPF", "FFPF"};
        const char *seq = forms[(M->form >= 0 && M->form < 4) ? M->form : 0];
        double *res = (double *)malloc(sizeof(double) * (size_t)n);
        double *dz = (double *)malloc(sizeof(double) * (size_t)n);
        int st = cpr_stage(M, seq[0], n, r, z);
        for (int k = 1; seq[k] && st == OR_OK; ++k) {
            memcpy(res, r, sizeof(double) * (size_t)n);
            or_amxpby(-1.0, M->A, z, 1.0, res);
            st = cpr_stage(M, seq[k], n, res, dz);
            for (int64_t i = 0; i < n; ++i) z[i] = z[i] + dz[i];
        }
        free(res);
        free(dz);
        return st;
    }
    default:
        return OR_INVALID;
    }
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers.                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t iters;             /* inner iterations (Arnoldi steps / BiCGSTAB loops) */
    int32_t restarts;          /* completed GMRES cycles */
    int32_t status;
    int32_t pad;
    double true_rel_res;       /* ||b - A x|| / ||b|| at exit, recomputed */
    double implicit_rel_res;   /* the solver's own residual estimate at exit */
} or_info;

static int64_t mat_n(const or_mat *A) { return (int64_t)A->nrows * A->bs; }

/* One Arnoldi step with classical Gram-Schmidt and one full
 * reorthogonalisation pass (CGS2): orthogonalises w against the i+1 columns
 * of V (ld = n) and returns h[0..i] plus h[i+1] = ||w||.  With mgs = 1 it runs
 * modified Gram-Schmidt instead (Alg. 1, inner loop over k). */
void or_orthogonalise(int64_t n, int32_t i, const double *V, double *w, double *h, int32_t mgs)
{
    if (mgs) {
        for (int32_t k = 0; k <= i; ++k) {
            const double *v = V + (size_t)k * n;
            h[k] = or_dot(n, w, v);
            for (int64_t r = 0; r < n; ++r) w[r] = w[r] - h[k] * v[r];
        }
    } else {
        double t[512];
        for (int32_t k = 0; k <= i; ++k) h[k] = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int32_t k = 0; k <= i; ++k) t[k] = or_dot(n, V + (size_t)k * n, w);
            for (int64_t r = 0; r < n; ++r) {
                double s = 0.0;
                for (int32_t k = 0; k <= i; ++k) s += V[(size_t)k * n + r] * t[k];
                w[r] = w[r] - s;
            }
            for (int32_t k = 0; k <= i; ++k) h[k] += t[k];
        }
    }
    h[i + 1] = or_norm2(n, w);
}

/* Restarted GMRES(m) (Sec. 3, Alg. 1) and flexible GMRES.
 *  side = 0: right preconditioning, A M^{-1} u = b, x = M^{-1} u; the
 *            implicit residual is the true residual norm of the iterate.
 *  side = 1: left preconditioning exactly as Alg. 1 (M r = b - A x0,
 *            M w = A v); stopping test on the preconditioned residual.
 *  flexible = 1 (right side only): keeps z_i = M^{-1} v_i and forms
 *            x += Z y (Saad's FGMRES), so M may change between steps.
 * Orthogonalisation: CGS2 (mgs = 0) or MGS as printed in Alg. 1 (mgs = 1).
 * Givens rotations reduce the Hessenberg matrix; the least-squares problem
 * min ||s - H y|| of Alg. 1 is then a triangular back-substitution.
 * Convergence: ||b - A x|| <= rtol ||b|| checked with the true residual at
 * the end of every cycle; inside a cycle the rotated residual |g_{i+1}|
 * ends the cycle early.  maxit counts inner iterations. */
int or_gmres(const or_mat *A, const or_pc *M, const double *b, double *x,
             int32_t m, double rtol, int32_t maxit, int32_t side, int32_t flexible,
             int32_t mgs, double *hist, int32_t hist_len, or_info *info)
{
    const int64_t n = mat_n(A);
    memset(info, 0, sizeof(*info));
    if (m < 1 || m > 500 || n < 1) { info->status = OR_INVALID; return OR_INVALID; }
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (m + 1));
    double *Z = flexible ? (double *)malloc(sizeof(double) * (size_t)n * m) : NULL;
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* column-major, ld m+1 */
    double *cs = (double *)malloc(sizeof(double) * m);
    double *sn = (double *)malloc(sizeof(double) * m);
    double *g = (double *)malloc(sizeof(double) * (m + 1));
    double *y = (double *)malloc(sizeof(double) * (m + 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);

    const double bnorm = or_norm2(n, b);
    int status = OR_NOT_CONVERGED;
    int32_t iters = 0, cycles = 0;
    double implicit = 0.0;
    if (bnorm == 0.0) {
        or_set(n, 0.0, x);
        status = OR_OK;
        goto done;
    }
    double tol;
    /* reference norm for the stopping test */
    if (side == 1) {
        or_pc_apply(M, n, b, t);
        tol = rtol * or_norm2(n, t);
    } else {
        tol = rtol * bnorm;
    }
    for (;;) {
        /* r = b - A x (Fig. 21 with a = -1, b = 1) */
        memcpy(r, b, sizeof(double) * (size_t)n);
        or_amxpby(-1.0, A, x, 1.0, r);
        if (side == 1) { or_pc_apply(M, n, r, t); memcpy(r, t, sizeof(double) * (size_t)n); }
        const double beta = or_norm2(n, r);
        implicit = beta;
        if (beta <= tol) { status = OR_OK; break; }
        if (iters >= maxit) break;
        for (int64_t k = 0; k < n; ++k) V[k] = r[k] / beta;
        g[0] = beta;
        for (int32_t k = 1; k <= m; ++k) g[k] = 0.0;
        int32_t kdim = 0;
        for (int32_t i = 0; i < m; ++i) {
            double *vi = V + (size_t)i * n;
            double *zi = flexible ? Z + (size_t)i * n : t;
            if (side == 1) {
                or_spmv(A, vi, t);
                or_pc_apply(M, n, t, w);
            } else {
                or_pc_apply(M, n, vi, zi);
                or_spmv(A, zi, w);
            }
            const double w0 = or_norm2(n, w);
            double *h = H + (size_t)i * (m + 1);
            or_orthogonalise(n, i, V, w, h, mgs);
            /* apply the previous rotations to column i */
            for (int32_t k = 0; k < i; ++k) {
                const double a = h[k], c = h[k + 1];
                h[k] = cs[k] * a + sn[k] * c;
                h[k + 1] = -sn[k] * a + cs[k] * c;
            }
            const double hnext = h[i + 1];
            const double rho = hypot(h[i], hnext);
            cs[i] = h[i] / rho;
            sn[i] = hnext / rho;
            h[i] = rho;
            h[i + 1] = 0.0;
            g[i + 1] = -sn[i] * g[i];
            g[i] = cs[i] * g[i];
            ++iters;
            kdim = i + 1;
            implicit = fabs(g[i + 1]);
            if (hist && iters - 1 < hist_len) hist[iters - 1] = implicit / (side == 1 ? tol / rtol : bnorm);
            const int happy = hnext <= 1e-14 * w0;
            if (implicit <= tol || iters >= maxit || happy || i == m - 1) break;
            double *vn = V + (size_t)(i + 1) * n;
            for (int64_t k = 0; k < n; ++k) vn[k] = w[k] / hnext;
        }
        /* back-substitution H(0:k,0:k) y = g(0:k) */
        for (int32_t k = kdim - 1; k >= 0; --k) {
            double s = g[k];
            for (int32_t j = k + 1; j < kdim; ++j) s -= H[(size_t)j * (m + 1) + k] * y[j];
            y[k] = s / H[(size_t)k * (m + 1) + k];
        }
        if (flexible) {
            for (int64_t r2 = 0; r2 < n; ++r2) {
                double s = 0.0;
                for (int32_t j = 0; j < kdim; ++j) s += Z[(size_t)j * n + r2] * y[j];
                x[r2] = x[r2] + s;
            }
        } else {
            for (int64_t r2 = 0; r2 < n; ++r2) {
                double s = 0.0;
                for (int32_t j = 0; j < kdim; ++j) s += V[(size_t)j * n + r2] * y[j];
                w[r2] = s;
            }
            if (side == 1) {
                for (int64_t r2 = 0; r2 < n; ++r2) x[r2] = x[r2] + w[r2];
            } else {
                or_pc_apply(M, n, w, t);
                for (int64_t r2 = 0; r2 < n; ++r2) x[r2] = x[r2] + t[r2];
            }
        }
        ++cycles;
    }
done:
    memcpy(r, b, sizeof(double) * (size_t)n);
    or_amxpby(-1.0, A, x, 1.0, r);
    info->true_rel_res = bnorm > 0.0 ? or_norm2(n, r) / bnorm : 0.0;
    info->implicit_rel_res = bnorm > 0.0 ? implicit / (side == 1 ? tol / rtol : bnorm) : 0.0;
    if (side == 0 && status == OR_OK && info->true_rel_res > rtol) status = OR_NOT_CONVERGED;
    info->iters = iters;
    info->restarts = cycles;
    info->status = status;
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r); free(t); free(w);
    return status;
}

/* LGMRES(m, k), the augmented restarted GMRES behind the `aug_k` setting of
 * Sec. 3's solver (Baker, Jessup and Manteuffel 2005; the paper prints no
 * algorithm).  Flexible GMRES whose cycle space is extended by the
 * normalised corrections x_new - x_old of the last k cycles, newest first:
 * a cycle takes m Arnoldi steps with z_i = M^{-1} v_i and then one step per
 * stored correction with z_i = that correction; w = A z_i, CGS2, Givens
 * rotations and stopping tests as in or_gmres; x += Z y, and Z y / ||Z y||
 * joins the stored corrections.  k = 0 is FGMRES(m).  An iteration is one
 * Arnoldi step. */
int or_lgmres(const or_mat *A, const or_pc *M, const double *b, double *x, int32_t m, int32_t k,
              double rtol, int32_t maxit, or_info *info)
{
    const int64_t n = mat_n(A);
    memset(info, 0, sizeof(*info));
    if (m < 1 || k < 0 || m + k > 500 || n < 1) { info->status = OR_INVALID; return OR_INVALID; }
    const int32_t mk = m + k;
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (mk + 1));
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * mk);
    double *aug = (double *)malloc(sizeof(double) * (size_t)n * (k > 0 ? k : 1));   /* aug[0] newest */
    double *H = (double *)calloc((size_t)(mk + 1) * mk, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * mk);
    double *sn = (double *)malloc(sizeof(double) * mk);
    double *g = (double *)malloc(sizeof(double) * (mk + 1));
    double *y = (double *)malloc(sizeof(double) * (mk + 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    const double bnorm = or_norm2(n, b);
    int status = OR_NOT_CONVERGED;
    int32_t iters = 0, cycles = 0, naug = 0;
    double implicit = 0.0;
    if (bnorm == 0.0) {
        or_set(n, 0.0, x);
        status = OR_OK;
        goto done;
    }
    const double tol = rtol * bnorm;
    for (;;) {
        memcpy(r, b, sizeof(double) * (size_t)n);
        or_amxpby(-1.0, A, x, 1.0, r);
        const double beta = or_norm2(n, r);
        implicit = beta;
        if (beta <= tol) { status = OR_OK; break; }
        if (iters >= maxit) break;
        const int32_t dim = m + naug;
        for (int64_t q = 0; q < n; ++q) V[q] = r[q] / beta;
        g[0] = beta;
        for (int32_t q = 1; q <= dim; ++q) g[q] = 0.0;
        int32_t kdim = 0;
        for (int32_t i = 0; i < dim; ++i) {
            double *vi = V + (size_t)i * n;
            double *zi = Z + (size_t)i * n;
            if (i < m) or_pc_apply(M, n, vi, zi);
            else memcpy(zi, aug + (size_t)(i - m) * n, sizeof(double) * (size_t)n);
            or_spmv(A, zi, w);
            const double w0 = or_norm2(n, w);
            double *h = H + (size_t)i * (dim + 1);
            or_orthogonalise(n, i, V, w, h, 0);
            for (int32_t q = 0; q < i; ++q) {
                const double a = h[q], c = h[q + 1];
                h[q] = cs[q] * a + sn[q] * c;
                h[q + 1] = -sn[q] * a + cs[q] * c;
            }
            const double hnext = h[i + 1];
            const double rho = hypot(h[i], hnext);
            cs[i] = h[i] / rho;
            sn[i] = hnext / rho;
            h[i] = rho;
            h[i + 1] = 0.0;
            g[i + 1] = -sn[i] * g[i];
            g[i] = cs[i] * g[i];
            ++iters;
            kdim = i + 1;
            implicit = fabs(g[i + 1]);
            const int happy = hnext <= 1e-14 * w0;
            if (implicit <= tol || iters >= maxit || happy || i == dim - 1) break;
            double *vn = V + (size_t)(i + 1) * n;
            for (int64_t q = 0; q < n; ++q) vn[q] = w[q] / hnext;
        }
        for (int32_t q = kdim - 1; q >= 0; --q) {
            double s2 = g[q];
            for (int32_t j = q + 1; j < kdim; ++j) s2 -= H[(size_t)j * (dim + 1) + q] * y[j];
            y[q] = s2 / H[(size_t)q * (dim + 1) + q];
        }
        /* the correction dx = Z y (in w), then x += dx */
        for (int64_t q = 0; q < n; ++q) {
            double s2 = 0.0;
            for (int32_t j = 0; j < kdim; ++j) s2 += Z[(size_t)j * n + q] * y[j];
            w[q] = s2;
        }
        for (int64_t q = 0; q < n; ++q) x[q] = x[q] + w[q];
        if (k > 0) {
            const double nrm = or_norm2(n, w);
            if (naug == k) --naug;                 /* the oldest correction drops out */
            memmove(aug + (size_t)n, aug, sizeof(double) * (size_t)n * naug);
            for (int64_t q = 0; q < n; ++q) aug[q] = nrm > 0.0 ? w[q] / nrm : 0.0;
            ++naug;
        }
        ++cycles;
    }
done:
    memcpy(r, b, sizeof(double) * (size_t)n);
    or_amxpby(-1.0, A, x, 1.0, r);
    info->true_rel_res = bnorm > 0.0 ? or_norm2(n, r) / bnorm : 0.0;
    info->implicit_rel_res = bnorm > 0.0 ? implicit / bnorm : 0.0;
    if (status == OR_OK && info->true_rel_res > rtol) status = OR_NOT_CONVERGED;
    info->iters = iters;
    info->restarts = cycles;
    info->status = status;
    free(V); free(Z); free(aug); free(H); free(cs); free(sn); free(g); free(y); free(r); free(w);
    return status;
}

/* Right-preconditioned BiCGSTAB (named in Sec. 3 and used in Examples 2, 4
 * and 5; the paper does not print it, so this is van der Vorst's 1992
 * algorithm as given in Saad's book, with z = M^{-1} applied to p and s).
 * All scalars FP64.  One iteration = one full loop; a half-step exit on
 * ||s|| counts as one iteration.  On an implicit convergence the true
 * residual is recomputed; if it has drifted above the tolerance the method
 * restarts from the true residual. */
int or_bicgstab(const or_mat *A, const or_pc *M, const double *b, double *x,
                double rtol, int32_t maxit, double *hist, int32_t hist_len, or_info *info)
{
    const int64_t n = mat_n(A);
    memset(info, 0, sizeof(*info));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *rh = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    double *ph = (double *)malloc(sizeof(double) * (size_t)n);
    double *sh = (double *)malloc(sizeof(double) * (size_t)n);
    const double bnorm = or_norm2(n, b);
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double implicit = 0.0;
    if (bnorm == 0.0) { or_set(n, 0.0, x); status = OR_OK; goto done; }
    const double tol = rtol * bnorm;
    int fresh = 1;
    double rho0 = 1.0, alpha = 1.0, omega = 1.0;
    while (it < maxit) {
        if (fresh) {
            memcpy(r, b, sizeof(double) * (size_t)n);
            or_amxpby(-1.0, A, x, 1.0, r);
            implicit = or_norm2(n, r);
            if (implicit <= tol) { status = OR_OK; break; }
            memcpy(rh, r, sizeof(double) * (size_t)n);
            or_set(n, 0.0, p);
            or_set(n, 0.0, v);
            rho0 = alpha = omega = 1.0;
            fresh = 0;
        }
        const double rho = or_dot(n, rh, r);
        if (!(fabs(rho) > 0.0) || !isfinite(rho)) { status = OR_BREAKDOWN; break; }
        const double beta = (rho / rho0) * (alpha / omega);
        /* p = r + beta (p - omega v) */
        for (int64_t k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
        or_pc_apply(M, n, p, ph);
        or_spmv(A, ph, v);
        const double rv = or_dot(n, rh, v);
        if (!(fabs(rv) > 0.0) || !isfinite(rv)) { status = OR_BREAKDOWN; break; }
        alpha = rho / rv;
        for (int64_t k = 0; k < n; ++k) s[k] = r[k] - alpha * v[k];
        ++it;
        const double snorm = or_norm2(n, s);
        if (snorm <= tol) {
            for (int64_t k = 0; k < n; ++k) x[k] = x[k] + alpha * ph[k];
            implicit = snorm;
            if (hist && it - 1 < hist_len) hist[it - 1] = snorm / bnorm;
            fresh = 1;            /* confirm with the true residual */
            continue;
        }
        or_pc_apply(M, n, s, sh);
        or_spmv(A, sh, t);
        const double tt = or_dot(n, t, t);
        const double ts = or_dot(n, t, s);
        omega = tt > 0.0 ? ts / tt : 0.0;
        for (int64_t k = 0; k < n; ++k) x[k] = x[k] + alpha * ph[k] + omega * sh[k];
        for (int64_t k = 0; k < n; ++k) r[k] = s[k] - omega * t[k];
        rho0 = rho;
        implicit = or_norm2(n, r);
        if (hist && it - 1 < hist_len) hist[it - 1] = implicit / bnorm;
        if (implicit <= tol) { fresh = 1; continue; }
        if (!(omega != 0.0) || !isfinite(omega)) { status = OR_BREAKDOWN; break; }
    }
    if (status == OR_NOT_CONVERGED && fresh && it >= maxit) {
        /* the last loop ended on an implicit convergence: confirm it */
        memcpy(r, b, sizeof(double) * (size_t)n);
        or_amxpby(-1.0, A, x, 1.0, r);
        if (or_norm2(n, r) <= tol) status = OR_OK;
    }
done:
    memcpy(r, b, sizeof(double) * (size_t)n);
    or_amxpby(-1.0, A, x, 1.0, r);
    info->true_rel_res = bnorm > 0.0 ? or_norm2(n, r) / bnorm : 0.0;
    info->implicit_rel_res = bnorm > 0.0 ? implicit / bnorm : 0.0;
    info->iters = it;
    info->status = status;
    free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
    return status;
}

/* Preconditioned conjugate gradient, Alg. 2, for symmetric positive definite
 * A and M.  One iteration is one pass of the printed loop: z = M^{-1} r;
 * rho = (r, z); p = z (first pass) or p = z + (rho / rho_prev) p; q = A p;
 * alpha = rho / (p, q); x += alpha p; r -= alpha q; stop on ||r||.  The
 * stopping norm is the recursive residual; when it passes the tolerance the
 * true residual b - A x is recomputed, and the loop restarts from it (p
 * discarded) if it has drifted above.  (p, q) <= 0 or a non-finite rho is a
 * breakdown (A or M not positive definite). */
int or_cg(const or_mat *A, const or_pc *M, const double *b, double *x,
          double rtol, int32_t maxit, double *hist, int32_t hist_len, or_info *info)
{
    const int64_t n = mat_n(A);
    memset(info, 0, sizeof(*info));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    const double bnorm = or_norm2(n, b);
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double rn = 0.0;
    if (bnorm == 0.0) {
        or_set(n, 0.0, x);
        status = OR_OK;
        goto done;
    }
    const double tol = rtol * bnorm;
    for (;;) {
        /* r = b - A x (line 1) */
        memcpy(r, b, sizeof(double) * (size_t)n);
        or_amxpby(-1.0, A, x, 1.0, r);
        rn = or_norm2(n, r);
        if (rn <= tol) { status = OR_OK; break; }
        if (it >= maxit) break;
        double rho_prev = 0.0;
        int first = 1, converged = 0;
        while (it < maxit) {
            or_pc_apply(M, n, r, z);                               /* line 4 */
            const double rho = or_dot(n, r, z);                    /* line 5 */
            if (!isfinite(rho) || rho == 0.0) { status = OR_BREAKDOWN; goto done; }
            if (first) {                                           /* lines 6-11 */
                memcpy(p, z, sizeof(double) * (size_t)n);
            } else {
                const double beta = rho / rho_prev;
                for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            }
            first = 0;
            or_spmv(A, p, q);                                      /* line 12 */
            const double pq = or_dot(n, p, q);                     /* line 13 */
            if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; goto done; }
            const double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];   /* line 14 */
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];   /* line 15 */
            it += 1;
            rn = or_norm2(n, r);                                   /* line 16 */
            if (hist && it - 1 < hist_len) hist[it - 1] = rn / bnorm;
            rho_prev = rho;
            if (rn <= tol) { converged = 1; break; }
        }
        if (!converged) {
            /* out of iterations: the true residual decides */
            memcpy(r, b, sizeof(double) * (size_t)n);
            or_amxpby(-1.0, A, x, 1.0, r);
            if (or_norm2(n, r) <= tol) status = OR_OK;
            break;
        }
        /* recursive residual converged: confirm with the true residual */
    }
done:
    memcpy(r, b, sizeof(double) * (size_t)n);
    or_amxpby(-1.0, A, x, 1.0, r);
    info->true_rel_res = bnorm > 0.0 ? or_norm2(n, r) / bnorm : 0.0;
    info->implicit_rel_res = bnorm > 0.0 ? rn / bnorm : 0.0;
    info->iters = it;
    info->status = status;
    free(r); free(z); free(p); free(q);
    return status;
}
