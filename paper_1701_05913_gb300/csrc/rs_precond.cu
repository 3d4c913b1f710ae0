// Preconditioner objects: setup / apply / destroy (Sec. 3, Fig. 29) for
// ILU(0), block ILU(0) and the two-stage CPR preconditioner (Sec. 4.3).
//
// CPR, pressure stage first (Alg. 6, read as the standard two-stage form:
//   z1 = Pi_p M_p^{-1} Pi_r f;   t = f - A z1;   z = z1 + R(A)^{-1} t),
// where Pi_r is the quasi-IMPES-weighted restriction to the pressure
// unknowns (Eqs. 5-7), Pi_p injects pressures with zero saturations (Eq. 8),
// M_p is ILU(0) of the decoupled pressure matrix App' (or the learned
// network) and R is block ILU(0) of the full matrix.  On a CSR matrix the
// restriction is the identity and App' = A.
#include <algorithm>

#include "rs_internal.cuh"

// quasi-IMPES weights w_Ik = -D_I[0][k] / D_I[k][k] (D_I the diagonal block)
__global__ void k_qimpes_weights(int nb, int bs, const int *__restrict__ diagpos,
                                 const double *__restrict__ val, double *__restrict__ w)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nb; I += gridDim.x * blockDim.x) {
        const double *D = val + (size_t)diagpos[I] * bs * bs;
        for (int k = 1; k < bs; ++k) w[(size_t)I * (bs - 1) + k - 1] = -D[k] / D[k * bs + k];
    }
}

// App'_IJ = A_IJ[0][0] + sum_k w_Ik A_IJ[k][0]
__global__ void k_qimpes_app(int nb, int bs, const int *__restrict__ ptr, const double *__restrict__ val,
                             const double *__restrict__ w, double *__restrict__ app)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nb; I += gridDim.x * blockDim.x) {
        for (int p = ptr[I]; p < ptr[I + 1]; ++p) {
            const double *B = val + (size_t)p * bs * bs;
            double s = B[0];
            for (int k = 1; k < bs; ++k) s = __dadd_rn(s, __dmul_rn(w[(size_t)I * (bs - 1) + k - 1], B[k * bs]));
            app[p] = s;
        }
    }
}

// rp_I = f_I0 + sum_k w_Ik f_Ik
__global__ void k_qimpes_restrict(int nb, int bs, const double *__restrict__ w,
                                  const double *__restrict__ f, double *__restrict__ rp,
                                  const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nb; I += gridDim.x * blockDim.x) {
        double s = f[(size_t)I * bs];
        for (int k = 1; k < bs; ++k) s = __dadd_rn(s, __dmul_rn(w[(size_t)I * (bs - 1) + k - 1], f[(size_t)I * bs + k]));
        rp[I] = s;
    }
}

// z_I0 = p_I, z_Ik = 0 (Eq. 8)
__global__ void k_prolong(int nb, int bs, const double *__restrict__ p, double *__restrict__ z,
                          const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nb * bs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t / bs), k = (int)(t % bs);
        z[t] = k == 0 ? p[I] : 0.0;
    }
}

__global__ void k_copy_add(int64_t n, const double *__restrict__ a, double *__restrict__ z,
                           int add, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        z[i] = add ? __dadd_rn(z[i], a[i]) : a[i];
}

// pcol[p bs + r] = A_p[r][0]: the pressure column of every block, the only
// one a prolonged pressure correction (Eq. 8) meets
__global__ void k_pcol_gather(int64_t nnzb, int bs, const double *__restrict__ val, double *__restrict__ pcol)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnzb * bs;
         t += (int64_t)gridDim.x * blockDim.x)
        pcol[t] = val[t * bs];
}

// t = f - A (Pi_p p): the residual after a pressure stage.  The prolonged
// vector is zero outside the pressure unknowns, so only the pressure column
// of each block contributes; the remaining terms of the full product are
// exact zeros.  One thread per scalar row, multiply-adds in the block order
// of the BSR SpMV, so the sums are those of the full product.
template <int BS>
__global__ void __launch_bounds__(256)
k_cpr_presid(int nb, int bsr, const int *__restrict__ ptr, const int *__restrict__ col,
             const double *__restrict__ pcol, const double *__restrict__ p, const double *__restrict__ f,
             double *__restrict__ t, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    const int bs = BS > 0 ? BS : bsr;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nb * bs) return;
    const int I = (int)(i / bs), r = (int)(i % bs);
    double acc = 0.0;
    for (int q = ptr[I]; q < ptr[I + 1]; ++q) acc = fma(pcol[(size_t)q * bs + r], __ldg(p + col[q]), acc);
    t[i] = __dsub_rn(f[i], acc);
}

// z = Pi_p p + t: prolongation and the second stage's correction in one pass
__global__ void k_prolong_add(int nb, int bs, const double *__restrict__ p, const double *__restrict__ t,
                              double *__restrict__ z, const int *skip)
{
    if (skip && *(volatile const int *)skip) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)nb * bs;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(i / bs), k = (int)(i % bs);
        z[i] = k == 0 ? __dadd_rn(p[I], t[i]) : t[i];
    }
}

static int grid_for(rs_ctx *ctx, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

// One stage of a CPR-like preconditioner on v: 'F' = R(A)^{-1} v, the
// block ILU(0) of the full system; 'P' = Pi_p M_p^{-1} (Pi_r v), quasi-IMPES
// restriction (the identity on a scalar matrix), the pressure solve (ILU(0)
// of the decoupled matrix, or the network) and prolongation.
static int cpr_stage(rs_pc *M, char kind, const double *v, double *out, const int *skip, bool prolong = true)
{
    rs_ctx *ctx = M->ctx;
    const rs_mat *A = M->A;
    if (kind == 'F')
        return M->ras ? rs_ras_apply(M->ras, v, out, skip) : rs_ilu_apply(M->bilu, v, out, nullptr, skip);
    const int nb = A->nrows, bs = A->bs;
    const double *rp = v;
    if (bs > 1) {
        k_qimpes_restrict<<<grid_for(ctx, nb), 256, 0, ctx->stream>>>(nb, bs, M->w, v, M->rp, skip);
        RS_TRY(rs_check_launch(ctx));
        rp = M->rp;
    }
    double *zp = bs > 1 ? M->zp : out;
    if (M->type == RS_PC_CPR_LEARNED) RS_TRY(rs_net_apply_pressure(M, rp, zp, skip));
    else if (M->amg) RS_TRY(rs_amg_apply(M->amg, rp, zp, skip));
    else RS_TRY(rs_ilu_apply(M->ilu, rp, zp, nullptr, skip));
    if (bs > 1 && prolong) {
        k_prolong<<<grid_for(ctx, A->n), 256, 0, ctx->stream>>>(nb, bs, M->zp, out, skip);
        RS_TRY(rs_check_launch(ctx));
    }
    return RS_OK;
}

// Alg. 6 (PF) on a block matrix: z1 = Pi_p M_p^{-1} Pi_r r stays in the
// pressure vector zp; t1 = r - A z1 takes the pressure column of A only;
// z = z1 + R(A)^{-1} t1 in one pass.  Equal to the general sequence up to
// the sign of zero results.
static int cpr_apply_pf_blocks(rs_pc *M, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    const rs_mat *A = M->A;
    const int nb = A->nrows, bs = A->bs;
    RS_TRY(cpr_stage(M, 'P', r, nullptr, skip, false));
    {
        RsProfScope prof(ctx, RS_PROF_CPR_RESID);
        const int64_t threads = (int64_t)A->n;
        const int grid = (int)((threads + 255) / 256);
        if (bs == 3)
            k_cpr_presid<3><<<grid, 256, 0, ctx->stream>>>(nb, 3, A->ptr, A->col, M->pcol, M->zp, r, M->t1, skip);
        else
            k_cpr_presid<0><<<grid, 256, 0, ctx->stream>>>(nb, bs, A->ptr, A->col, M->pcol, M->zp, r, M->t1, skip);
        RS_TRY(rs_check_launch(ctx));
    }
    RS_TRY(cpr_stage(M, 'F', M->t1, M->t2, skip));
    k_prolong_add<<<grid_for(ctx, A->n), 256, 0, ctx->stream>>>(nb, bs, M->zp, M->t2, z, skip);
    return rs_check_launch(ctx);
}

// Algs. 5-8: the first stage maps f to z; every later stage forms
// t1 = f - A z and adds its correction t2 = stage(t1) to z
static int cpr_apply(rs_pc *M, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    const rs_mat *A = M->A;
    static const char *forms[4] = {"PF", "FP", "FPF", "FFPF"};
    const char *seq = forms[M->form];
    if (M->pcol) return cpr_apply_pf_blocks(M, r, z, skip);
    RS_TRY(cpr_stage(M, seq[0], r, z, skip));
    for (int k = 1; seq[k]; ++k) {
        RS_TRY(rs_residual_launch(A, r, z, M->t1, nullptr, skip));
        RS_TRY(cpr_stage(M, seq[k], M->t1, M->t2, skip));
        k_copy_add<<<grid_for(ctx, A->n), 256, 0, ctx->stream>>>(A->n, M->t2, z, 1, skip);
        RS_TRY(rs_check_launch(ctx));
    }
    return RS_OK;
}

// A CPR apply is a few dozen launches (with the learned stage, the U-Net's
// layers).  After the first apply, each (r, z, skip) address triple is
// captured once into a CUDA graph and replayed; a nested AMG V-cycle then
// runs inside the capture.  Capture runs on a private stream (the caller's
// may be the legacy default stream, which cannot be captured); replays go to
// the caller's stream.  A graph is dropped when the device-wait limit has
// changed since its capture (rs_set_spin_limit), and a graph of the learned
// stage when the network's workspace has been reallocated since (another
// grid).  With the
// profiler on, a network on another context, or if a capture fails, the
// apply is launched kernel by kernel.
static int cpr_apply_graph(rs_pc *M, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    unsigned gen = 0;
    bool same = true;
    if (M->type == RS_PC_CPR_LEARNED) RS_TRY(rs_net_prepare(M, &gen, &same));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!same || ctx->prof_on || M->nograph || cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return cpr_apply(M, r, z, skip);
    for (size_t i = 0; i < M->graphs.size(); ++i) {
        rs_pc::Graph &g = M->graphs[i];
        if (g.r != r || g.z != z || g.skip != skip) continue;
        if (g.gen == gen && g.limit == ctx->spin_limit) {
            if (cudaGraphLaunch(g.exec, ctx->stream) != cudaSuccess) return RS_ERR_CUDA;
            ctx->launches += g.nlaunch;
            return RS_OK;
        }
        cudaGraphExecDestroy(g.exec);
        M->graphs.erase(M->graphs.begin() + i);
        break;
    }
    if (M->applies++ == 0 || M->graphs.size() >= 64) return cpr_apply(M, r, z, skip);
    if (!M->capture && cudaStreamCreateWithFlags(&M->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        M->nograph = true;
        return cpr_apply(M, r, z, skip);
    }
    const long long l0 = ctx->launches;
    cudaStream_t user = ctx->stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int st = RS_ERR_CUDA;
    if (cudaStreamBeginCapture(M->capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        ctx->stream = M->capture;
        st = cpr_apply(M, r, z, skip);
        ctx->stream = user;
        if (cudaStreamEndCapture(M->capture, &graph) != cudaSuccess) st = RS_ERR_CUDA;
    }
    if (!st && (!graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)) st = RS_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (st) {
        cudaGetLastError();
        M->nograph = true;
        ctx->launches = l0;
        return cpr_apply(M, r, z, skip);
    }
    M->graphs.push_back({r, z, skip, gen, ctx->spin_limit, exec, ctx->launches - l0});
    // the capture has counted the graph's launches once; this is their run
    return cudaGraphLaunch(exec, user) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

int rs_pc_apply_dev(rs_pc *M, const double *r, double *z, const int *skip)
{
    rs_ctx *ctx = M->ctx;
    const rs_mat *A = M->A;
    switch (M->type) {
    case RS_PC_NONE:
        k_copy_add<<<grid_for(ctx, A->n), 256, 0, ctx->stream>>>(A->n, r, z, 0, skip);
        return rs_check_launch(ctx);
    case RS_PC_ILU0:
        return rs_ilu_apply(M->ilu, r, z, nullptr, skip);
    case RS_PC_BILU0:
        return rs_ilu_apply(M->bilu, r, z, nullptr, skip);
    case RS_PC_RAS:
        return rs_ras_apply(M->ras, r, z, skip);
    case RS_PC_AMG:
        if (!M->amg) return RS_ERR_INVALID_ARG;
        return rs_amg_apply(M->amg, r, z, skip);
    case RS_PC_CPR:
    case RS_PC_CPR_LEARNED:
        return cpr_apply_graph(M, r, z, skip);
    default:
        return RS_ERR_INVALID_ARG;
    }
}

static void pc_free(rs_pc *M)
{
    if (!M) return;
    rs_ctx *ctx = M->ctx;
    for (const rs_pc::Graph &g : M->graphs) cudaGraphExecDestroy(g.exec);
    if (M->capture) cudaStreamDestroy(M->capture);
    if (M->ilu && M->ilu != M->bilu) rs_ilu_destroy(M->ilu);
    if (M->bilu) rs_ilu_destroy(M->bilu);
    if (M->ras) rs_ras_destroy(M->ras);
    if (M->amg) rs_amg_destroy(M->amg);
    rs_free(ctx, M->app_val);
    rs_free(ctx, M->diagA);
    rs_free(ctx, M->w);
    rs_free(ctx, M->rp);
    rs_free(ctx, M->zp);
    rs_free(ctx, M->t1);
    rs_free(ctx, M->t2);
    rs_free(ctx, M->pcol);
    delete M;
}

// AMG options, zeroed fields taking their defaults (Fig. 34's strength 0.5
// and two relaxation sweeps; up to 16 levels down to 256 rows)
static int amg_params(const rs_pc_opts *o, double *theta, int *lev, int *coarse, int *nu, int *smoother)
{
    *theta = o && o->amg_theta != 0.0 ? o->amg_theta : 0.5;
    *lev = o && o->amg_max_levels ? o->amg_max_levels : RS_AMG_MAXLEV;
    *coarse = o && o->amg_max_coarse ? o->amg_max_coarse : 256;
    *nu = o && o->amg_nu ? o->amg_nu : 2;
    *smoother = o ? o->amg_smoother : 0;
    if (!(*theta > 0.0 && *theta <= 1.0) || *lev < 1 || *lev > RS_AMG_MAXLEV || *coarse < 1 || *nu < 1 ||
        *smoother < 0 || *smoother > 1)
        return RS_ERR_INVALID_ARG;
    return RS_OK;
}

extern "C" int rs_precond_setup(rs_ctx *ctx, const rs_mat *A, int type, const rs_pc_opts *opts,
                                rs_pc **out)
{
    if (!ctx || !A || !out) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    rs_pc *M = new rs_pc();
    M->ctx = ctx;
    M->type = type;
    M->prec = opts ? opts->prec : RS_FP64;
    M->form = opts ? opts->cpr_form : RS_CPR_PF;
    if (M->form < RS_CPR_PF || M->form > RS_CPR_FFPF) {
        delete M;
        return RS_ERR_INVALID_ARG;
    }
    M->A = A;
    M->bad_row = -1;
    const int fp32 = M->prec == RS_MIXED;
    // the ILU factors' triangular sweeps: wavefronts or segments, run length
    const int sweep = opts ? opts->sweep : 0, run_cap = opts ? opts->sweep_run_cap : 0;
    int st = RS_OK;
    int bad = -1;
    if (sweep < 0 || sweep > 2 || run_cap < 0) {
        delete M;
        return RS_ERR_INVALID_ARG;
    }
    switch (type) {
    case RS_PC_NONE:
        break;
    case RS_PC_ILU0:
        if (A->bs != 1) { st = RS_ERR_INVALID_ARG; break; }
        st = rs_ilu_create(ctx, 1, A->nrows, A->nnzb, A->ptr, A->col, A->h_ptr, A->h_col, fp32, sweep, run_cap, &M->ilu, &bad);
        if (!st) st = rs_ilu_factor(M->ilu, A->val, &bad);
        break;
    case RS_PC_BILU0:
        st = rs_ilu_create(ctx, A->bs, A->nrows, A->nnzb, A->ptr, A->col, A->h_ptr, A->h_col, fp32, sweep, run_cap, &M->bilu, &bad);
        if (!st) st = rs_ilu_factor(M->bilu, A->val, &bad);
        break;
    case RS_PC_AMG: {
        double th;
        int lev, nc, nu, sm;
        if (A->bs != 1 || (st = amg_params(opts, &th, &lev, &nc, &nu, &sm))) {
            st = RS_ERR_INVALID_ARG;
            break;
        }
        st = rs_amg_create(ctx, A->nrows, A->ptr, A->col, A->val, A, th, lev, nc, nu, sm, &M->amg);
        break;
    }
    case RS_PC_RAS: {
        const int nparts = opts && opts->ras_nparts ? opts->ras_nparts : 1;
        st = rs_ras_create(ctx, A, nparts, opts ? opts->ras_part : nullptr, opts ? opts->ras_overlap : 0,
                           opts ? opts->ilu_level : 0, opts ? opts->ras_local : 0,
                           opts && opts->ilut_p ? opts->ilut_p : -1,
                           opts && opts->ilut_tol != 0.0 ? opts->ilut_tol : 1e-3, fp32, &M->ras, &bad);
        break;
    }
    case RS_PC_CPR:
    case RS_PC_CPR_LEARNED: {
        const int nb = A->nrows, bs = A->bs;
        if (type == RS_PC_CPR_LEARNED) {
            if (!opts || !opts->net || !opts->log_perm || (int64_t)opts->nx * opts->ny * opts->nz != nb) {
                st = RS_ERR_INVALID_ARG;
                break;
            }
            M->net = opts->net;
            M->log_perm = opts->log_perm;
            M->nx = opts->nx;
            M->ny = opts->ny;
            M->nz = opts->nz;
        }
        const int pstage = opts ? opts->cpr_pstage : 0;
        double th;
        int lev, ncoarse, nu, sm;
        if (pstage < 0 || pstage > 1 || (pstage == 1 && amg_params(opts, &th, &lev, &ncoarse, &nu, &sm))) {
            st = RS_ERR_INVALID_ARG;
            break;
        }
        // the F stage R(A)^{-1}: block ILU(0) of A, or restricted additive
        // Schwarz over block subdomains when subdomains are given
        const bool fras = opts && (opts->ras_nparts > 1 || opts->ras_part);
        if (fras)
            st = rs_ras_create(ctx, A, opts->ras_nparts ? opts->ras_nparts : 1, opts->ras_part, opts->ras_overlap,
                               opts->ilu_level, opts->ras_local, opts->ilut_p ? opts->ilut_p : -1,
                               opts->ilut_tol != 0.0 ? opts->ilut_tol : 1e-3, fp32, &M->ras, &bad);
        else
            st = rs_ilu_create(ctx, bs, nb, A->nnzb, A->ptr, A->col, A->h_ptr, A->h_col, fp32, sweep, run_cap, &M->bilu, &bad);
        if (!st && !fras) st = rs_ilu_factor(M->bilu, A->val, &bad);
        if (st) break;
        st = rs_alloc(ctx, (void **)&M->t1, sizeof(double) * (A->n > 0 ? A->n : 1));
        if (!st) st = rs_alloc(ctx, (void **)&M->t2, sizeof(double) * (A->n > 0 ? A->n : 1));
        if (st) break;
        if (bs == 1) {
            // pressure stage on A itself: its ILU(0), or an AMG V-cycle
            if (pstage == 1 && type == RS_PC_CPR) {
                st = rs_amg_create(ctx, nb, A->ptr, A->col, A->val, A, th, lev, ncoarse, nu, sm, &M->amg);
            } else if (fras) {
                st = rs_ilu_create(ctx, 1, nb, A->nnzb, A->ptr, A->col, A->h_ptr, A->h_col, fp32, sweep, run_cap, &M->ilu, &bad);
                if (!st) st = rs_ilu_factor(M->ilu, A->val, &bad);
            } else {
                M->ilu = M->bilu;
            }
            break;
        }
        st = rs_alloc(ctx, (void **)&M->w, sizeof(double) * (size_t)nb * (bs - 1));
        if (!st) st = rs_alloc(ctx, (void **)&M->app_val, sizeof(double) * (A->nnzb > 0 ? A->nnzb : 1));
        if (!st) st = rs_alloc(ctx, (void **)&M->rp, sizeof(double) * (nb > 0 ? nb : 1));
        if (!st) st = rs_alloc(ctx, (void **)&M->zp, sizeof(double) * (nb > 0 ? nb : 1));
        if (!st && M->form == RS_CPR_PF) {
            st = rs_alloc(ctx, (void **)&M->pcol, sizeof(double) * bs * (A->nnzb > 0 ? A->nnzb : 1));
            if (!st && A->nnzb > 0) {
                k_pcol_gather<<<grid_for(ctx, A->nnzb * bs), 256, 0, ctx->stream>>>(A->nnzb, bs, A->val, M->pcol);
                st = rs_check_launch(ctx);
            }
        }
        if (st) break;
        if (!st && fras) {
            // positions of the diagonal blocks, for the quasi-IMPES weights
            std::vector<int> dp(nb, 0);
            for (int I = 0; I < nb; ++I)
                for (int q = A->h_ptr[I]; q < A->h_ptr[I + 1]; ++q)
                    if (A->h_col[q] == I) dp[I] = q;
            st = rs_alloc(ctx, (void **)&M->diagA, sizeof(int) * (nb > 0 ? nb : 1));
            if (!st && nb > 0 &&
                cudaMemcpyAsync(M->diagA, dp.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, ctx->stream) !=
                    cudaSuccess)
                st = RS_ERR_CUDA;
            if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = RS_ERR_CUDA;
        }
        if (st) break;
        if (nb > 0) {
            k_qimpes_weights<<<grid_for(ctx, nb), 256, 0, ctx->stream>>>(nb, bs, fras ? M->diagA : M->bilu->diagpos,
                                                                        A->val, M->w);
            k_qimpes_app<<<grid_for(ctx, nb), 256, 0, ctx->stream>>>(nb, bs, A->ptr, A->val, M->w, M->app_val);
            st = rs_check_launch(ctx);
            ctx->launches++;
        }
        if (st) break;
        if (pstage == 1 && type == RS_PC_CPR) {
            // AMG V-cycle on the decoupled pressure matrix (the paper's CPR pressure stage)
            st = rs_amg_create(ctx, nb, A->ptr, A->col, M->app_val, nullptr, th, lev, ncoarse, nu, sm, &M->amg);
            break;
        }
        st = rs_ilu_create(ctx, 1, nb, A->nnzb, A->ptr, A->col, A->h_ptr, A->h_col, fp32, sweep, run_cap, &M->ilu, &bad);
        if (!st) st = rs_ilu_factor(M->ilu, M->app_val, &bad);
        break;
    }
    default:
        st = RS_ERR_INVALID_ARG;
    }
    M->bad_row = bad;
    // a zero pivot of an ILU factor keeps the handle, so that the caller can
    // query the row; an AMG hierarchy that could not be built leaves none
    const bool amg_missing =
        !M->amg && (type == RS_PC_AMG || (type == RS_PC_CPR && opts && opts->cpr_pstage == 1));
    if (st == RS_ERR_ZERO_PIVOT && !amg_missing) {
        rs_ctx_retain(ctx);
        *out = M;
        return st;
    }
    if (st) {
        pc_free(M);
        return st;
    }
    rs_ctx_retain(ctx);
    *out = M;
    return RS_OK;
}

extern "C" int rs_precond_apply(rs_pc *M, const rs_vec *r, rs_vec *z)
{
    if (!M || !r || !z) return RS_ERR_INVALID_ARG;
    if (r->n != M->A->n || z->n != M->A->n) return RS_ERR_SIZE_MISMATCH;
    RS_TRY(rs_pc_apply_dev(M, r->d, z->d, nullptr));
    return RS_OK;
}

extern "C" int rs_precond_get_ilu(const rs_pc *M, double *lu_host, int32_t nnz)
{
    if (!M || !M->ilu || !lu_host) return RS_ERR_INVALID_ARG;
    if (nnz != M->ilu->nnzb) return RS_ERR_SIZE_MISMATCH;
    RS_CUDA_TRY(cudaMemcpyAsync(lu_host, M->ilu->lu, sizeof(double) * nnz, cudaMemcpyDeviceToHost,
                                M->ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(M->ctx->stream));
    return RS_OK;
}

extern "C" int rs_precond_get_bilu(const rs_pc *M, double *lu_host, double *dinv_host)
{
    if (!M || !M->bilu || !lu_host || !dinv_host) return RS_ERR_INVALID_ARG;
    const size_t b2 = (size_t)M->bilu->bs * M->bilu->bs;
    RS_CUDA_TRY(cudaMemcpyAsync(lu_host, M->bilu->lu, sizeof(double) * b2 * M->bilu->nnzb,
                                cudaMemcpyDeviceToHost, M->ctx->stream));
    RS_CUDA_TRY(cudaMemcpyAsync(dinv_host, M->bilu->dinv, sizeof(double) * b2 * M->bilu->nrows,
                                cudaMemcpyDeviceToHost, M->ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(M->ctx->stream));
    return RS_OK;
}

extern "C" int rs_precond_get_cpr(const rs_pc *M, double *w_host, double *app_host)
{
    if (!M || !M->w || !M->app_val) return RS_ERR_INVALID_ARG;
    const rs_mat *A = M->A;
    if (w_host)
        RS_CUDA_TRY(cudaMemcpyAsync(w_host, M->w, sizeof(double) * (size_t)A->nrows * (A->bs - 1),
                                    cudaMemcpyDeviceToHost, M->ctx->stream));
    if (app_host)
        RS_CUDA_TRY(cudaMemcpyAsync(app_host, M->app_val, sizeof(double) * A->nnzb,
                                    cudaMemcpyDeviceToHost, M->ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(M->ctx->stream));
    return RS_OK;
}

extern "C" int32_t rs_precond_bad_row(const rs_pc *M) { return M ? M->bad_row : -1; }

extern "C" int rs_precond_sweep_levels(const rs_pc *M, int32_t *levels_l, int32_t *levels_u)
{
    if (!M || !levels_l || !levels_u) return RS_ERR_INVALID_ARG;
    // the full-system factor: ILU(0) alone, the stacked RAS factor, or the
    // second stage of CPR
    const IluFactor *f = M->ras ? M->ras->f : M->bilu ? M->bilu : M->ilu;
    if (!f) return RS_ERR_INVALID_ARG;
    if (f->W.on) {
        *levels_l = *levels_u = f->W.nx + f->W.ny + f->W.nz - 2;
    } else {
        *levels_l = f->SL.nlevels;
        *levels_u = f->SU.nlevels;
    }
    return RS_OK;
}

extern "C" int rs_precond_sweep_kind(const rs_pc *M, int32_t *kind, int32_t *nx, int32_t *ny, int32_t *nz)
{
    if (!M || !kind) return RS_ERR_INVALID_ARG;
    const IluFactor *f = M->ras ? M->ras->f : M->bilu ? M->bilu : M->ilu;
    if (!f) return RS_ERR_INVALID_ARG;
    *kind = f->W.on ? 1 : 0;
    if (nx) *nx = f->W.nx;
    if (ny) *ny = f->W.ny;
    if (nz) *nz = f->W.nz;
    return RS_OK;
}

extern "C" int rs_precond_sweep_runs(const rs_pc *M, int32_t *runs_l, int32_t *runs_u, int32_t *longest_l,
                                     int32_t *longest_u)
{
    if (!M || !runs_l || !runs_u || !longest_l || !longest_u) return RS_ERR_INVALID_ARG;
    const IluFactor *f = M->ras ? M->ras->f : M->bilu ? M->bilu : M->ilu;
    if (!f) return RS_ERR_INVALID_ARG;
    *runs_l = f->SL.nrun;
    *runs_u = f->SU.nrun;
    *longest_l = f->SL.max_run;
    *longest_u = f->SU.max_run;
    return RS_OK;
}

extern "C" int rs_precond_amg_levels(const rs_pc *M, int32_t *nlevels)
{
    if (!M || !M->amg || !nlevels) return RS_ERR_INVALID_ARG;
    *nlevels = M->amg->nlev;
    return RS_OK;
}

extern "C" int rs_precond_amg_level_sizes(const rs_pc *M, int32_t l, int32_t *n, int64_t *nnz_a, int64_t *nnz_p)
{
    if (!M || !M->amg || !n || !nnz_a || !nnz_p) return RS_ERR_INVALID_ARG;
    return rs_amg_level_sizes(M->amg, l, n, nnz_a, nnz_p);
}

extern "C" int rs_precond_get_amg_level(const rs_pc *M, int32_t l, int32_t *aptr, int32_t *acol, double *aval,
                                        int32_t *pptr, int32_t *pcol, double *pval, int32_t *cidx)
{
    if (!M || !M->amg) return RS_ERR_INVALID_ARG;
    return rs_amg_get_level(M->amg, l, aptr, acol, aval, pptr, pcol, pval, cidx);
}

extern "C" int rs_precond_ras_info(const rs_pc *M, int32_t *next, int64_t *nnz)
{
    if (!M || !M->ras || !next || !nnz) return RS_ERR_INVALID_ARG;
    *next = M->ras->next;
    *nnz = M->ras->nnz;
    return RS_OK;
}

extern "C" int rs_precond_get_ras(const rs_pc *M, int32_t *gidx, int32_t *ptr, int32_t *col, double *lu)
{
    if (!M || !M->ras) return RS_ERR_INVALID_ARG;
    const RasData *R = M->ras;
    cudaStream_t sm = M->ctx->stream;
    const size_t b2 = (size_t)R->bs * R->bs;
    if (gidx && R->next > 0)
        RS_CUDA_TRY(cudaMemcpyAsync(gidx, R->gidx, sizeof(int) * R->next, cudaMemcpyDeviceToHost, sm));
    if (ptr) RS_CUDA_TRY(cudaMemcpyAsync(ptr, R->ptr, sizeof(int) * (R->next + 1), cudaMemcpyDeviceToHost, sm));
    if (col && R->nnz > 0)
        RS_CUDA_TRY(cudaMemcpyAsync(col, R->col, sizeof(int) * R->nnz, cudaMemcpyDeviceToHost, sm));
    if (lu && R->nnz > 0)
        RS_CUDA_TRY(cudaMemcpyAsync(lu, R->f->lu, sizeof(double) * b2 * R->nnz, cudaMemcpyDeviceToHost, sm));
    RS_CUDA_TRY(cudaStreamSynchronize(sm));
    return RS_OK;
}

extern "C" int rs_precond_destroy(rs_pc **M)
{
    if (!M || !*M) return RS_OK;
    rs_ctx *ctx = (*M)->ctx;
    pc_free(*M);
    *M = nullptr;
    rs_ctx_release(ctx);
    return RS_OK;
}
