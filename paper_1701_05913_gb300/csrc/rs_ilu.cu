// ILU(0) and block ILU(0): analysis, numeric factorisation, triangular solves.
//
// The factorisation L U ~ A and the two solves L y = r, U z = y are Eq. 3
// (Sec. 4.1); the paper notes these solves run row by row and scale poorly.
// Here rows run as soon as the rows they depend on are final ("sync-free"):
//  * Factorisation: the host levels the rows of the dependency graph of L
//    (each level padded to a multiple of 32 rows); persistent blocks take the
//    rows in level order from a ticket counter, one row per thread; a warp
//    waits until the previous level is complete (a per-level arrival count
//    and a completion epoch), then runs the IKJ update in ascending column
//    order without contracted multiply-adds, so the FP64 factors equal those
//    of a sequential row-by-row ILU(0).
//  * Sweeps: rows are grouped into segments of up to 32 consecutive (block)
//    rows, one warp each, taken in segment-level order; a row's value is its
//    own ready flag (a sentinel NaN pattern until written); the in-segment
//    recurrence is solved with a warp scan (details at the kernels).  In
//    FP64 scalar sweeps a warp carries a run of segments, each reading the
//    one before it from the warp's registers (details at the runs).
//  * Every wait is bounded in time and reports RS_ERR_DEVICE_TIMEOUT instead
//    of hanging; every schedule is deadlock-free because a warp only waits for
//    rows held by warps that took earlier tickets and are already running.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "rs_internal.cuh"

#define RS_SWEEP_THREADS 128
#define RS_RUN_CH 4        // widest segment (entries per row) a run continues with
#define RS_RUN_P 6                       // segments staged ahead
#define RS_RUN_SLOTS (RS_RUN_P + 1)      // the slot being read is never refilled
#define RS_RUN_WORDS (RS_RUN_CH + 5 + 2) // per lane: values, multipliers, r or y, D
#define RS_RUN_RING ((RS_RUN_SLOTS + 1) * RS_RUN_WORDS * 32)   // 8-byte words per warp, with a spare slot

// ---------------------------------------------------------------------------
// host analysis
// ---------------------------------------------------------------------------
static int build_layout(rs_ctx *ctx, int nrows, const std::vector<int> &ptr,
                        const std::vector<int> &col, const std::vector<int> &diag, TriLayout &T)
{
    // level of each row in the dependency graph of L
    std::vector<int> lev(nrows, 0);
    int nlev = 0;
    for (int i = 0; i < nrows; ++i) {
        int l = 0;
        for (int q = ptr[i]; q < diag[i]; ++q) l = std::max(l, lev[col[q]] + 1);
        lev[i] = l;
        nlev = std::max(nlev, l + 1);
    }
    std::vector<int> cnt(nlev + 1, 0);
    for (int i = 0; i < nrows; ++i) cnt[lev[i]]++;
    std::vector<int64_t> start(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) start[l + 1] = start[l] + ((cnt[l] + 31) / 32) * 32;
    const int64_t npad = start[nlev];
    if (npad > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
    std::vector<int> pos(npad, -1);
    std::vector<int64_t> fill(start.begin(), start.end());
    for (int i = 0; i < nrows; ++i) pos[fill[lev[i]]++] = i;
    const int nwarps = (int)(npad / 32);
    std::vector<int> wlev(nwarps > 0 ? nwarps : 1), lnw(nlev > 0 ? nlev : 1, 0);
    for (int l = 0; l < nlev; ++l) {
        lnw[l] = (int)((start[l + 1] - start[l]) / 32);
        for (int64_t wi = start[l] / 32; wi < start[l + 1] / 32; ++wi) wlev[wi] = l;
    }
    T.npad = (int)npad;
    T.nlevels = nlev;
    T.nwarps = nwarps;
    int st = RS_OK;
    st = st ? st : rs_alloc(ctx, (void **)&T.pos, sizeof(int) * (npad > 0 ? npad : 1));
    st = st ? st : rs_alloc(ctx, (void **)&T.warp_level, sizeof(int) * wlev.size());
    st = st ? st : rs_alloc(ctx, (void **)&T.level_nwarps, sizeof(int) * lnw.size());
    st = st ? st : rs_alloc(ctx, (void **)&T.level_count, sizeof(int) * lnw.size());
    st = st ? st : rs_alloc(ctx, (void **)&T.level_done, sizeof(int) * lnw.size());
    if (st) return st;
    cudaStream_t s = ctx->stream;
    if (npad) RS_CUDA_TRY(cudaMemcpyAsync(T.pos, pos.data(), sizeof(int) * npad, cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaMemcpyAsync(T.warp_level, wlev.data(), sizeof(int) * wlev.size(), cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaMemcpyAsync(T.level_nwarps, lnw.data(), sizeof(int) * lnw.size(), cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaMemsetAsync(T.level_count, 0, sizeof(int) * lnw.size(), s));
    RS_CUDA_TRY(cudaMemsetAsync(T.level_done, 0, sizeof(int) * lnw.size(), s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));   // host vectors go out of scope
    return RS_OK;
}

// Segment layout (scalar factors): segments are runs of at most 32
// consecutive rows.  A new segment also starts where one chain of
// consecutive dependencies ends and the next begins (row i does not read row
// i-1 while row i-1 reads row i-2; for U the mirror image), so that on
// structured grids segments never straddle grid lines whatever their
// length.  A segment's level is one more than the highest level of the
// segments holding the columns it reads outside itself.
// The host analysis of one sweep: segments, their levels and kinds, the
// entry layout, and the runs (no device work; rs_sweep_schedule exposes it)
struct SegHost {
    int nseg = 0, nlev = 0, nrun = 0, max_run = 0;
    int64_t nent = 0;
    std::vector<int> r0v, lev, order, sptr, adjsrc, ecol, esrc, rdesc;
    std::vector<unsigned char> kind;
};

static int seg_schedule(int nrows, const std::vector<int> &ptr, const std::vector<int> &col,
                        const std::vector<int> &diag, bool lower, int run_cap, int64_t run_slots, SegHost &H)
{
    // does row i read row j = i-1 (L) / i+1 (U)?  (the entry next to the diagonal)
    auto reads_prev = [&](int i) { return i > 0 && diag[i] > ptr[i] && col[diag[i] - 1] == i - 1; };
    auto reads_next = [&](int i) { return i + 1 < nrows && diag[i] + 1 < ptr[i + 1] && col[diag[i] + 1] == i + 1; };
    std::vector<int> r0v;
    r0v.reserve(nrows / 16 + 2);
    for (int i = 0; i < nrows; ++i) {
        bool start = r0v.empty() || i - r0v.back() == 32;
        if (!start && i >= 2) {
            if (lower) start = !reads_prev(i) && reads_prev(i - 1);
            else start = !reads_next(i - 1) && reads_next(i);
        }
        if (start) r0v.push_back(i);
    }
    const int nseg = (int)r0v.size();
    r0v.push_back(nrows);
    std::vector<int> seg_of(nrows);
    for (int sg = 0; sg < nseg; ++sg)
        for (int i = r0v[sg]; i < r0v[sg + 1]; ++i) seg_of[i] = sg;
    std::vector<int> lev(nseg, 0), width(nseg, 0);
    std::vector<unsigned char> kind(nseg, 1);
    int nlev = 0;
    for (int t = 0; t < nseg; ++t) {
        const int sg = lower ? t : nseg - 1 - t;
        const int r0 = r0v[sg], r1 = r0v[sg + 1];
        int l = 0, w = 0;
        for (int i = r0; i < r1; ++i) {
            const int q0 = lower ? ptr[i] : diag[i] + 1;
            const int q1 = lower ? diag[i] : ptr[i + 1];
            w = std::max(w, q1 - q0);
            for (int q = q0; q < q1; ++q) {
                const int c = col[q];
                if (c >= r0 && c < r1) {
                    if (c != (lower ? i - 1 : i + 1)) kind[sg] = 0;
                } else {
                    l = std::max(l, lev[seg_of[c]] + 1);
                }
            }
        }
        lev[sg] = l;
        width[sg] = w;
        nlev = std::max(nlev, l + 1);
    }
    std::vector<int> order(nseg);
    for (int t = 0; t < nseg; ++t) order[t] = lower ? t : nseg - 1 - t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lev[a] < lev[b]; });
    std::vector<int> sptr(nseg + 1, 0);
    int64_t nent = 0;
    for (int sg = 0; sg < nseg; ++sg) {
        sptr[sg] = (int)nent;
        nent += (int64_t)width[sg] * 32;
        if (nent > 0x7fffffffLL) return RS_ERR_INVALID_ARG;
    }
    sptr[nseg] = (int)nent;
    // the entry a row of a chain segment reads from its neighbour inside the segment
    std::vector<int> adjsrc(nrows, -1);
    for (int sg = 0; sg < nseg; ++sg) {
        const int r0 = r0v[sg], r1 = r0v[sg + 1];
        for (int i = r0; i < r1; ++i) {
            if (lower && i > r0 && reads_prev(i)) adjsrc[i] = diag[i] - 1;
            if (!lower && i + 1 < r1 && reads_next(i)) adjsrc[i] = diag[i] + 1;
        }
    }
    std::vector<int> ecol(nent, -1), esrc(nent, -1);
    for (int sg = 0; sg < nseg; ++sg) {
        const int r0 = r0v[sg], r1 = r0v[sg + 1];
        for (int i = r0; i < r1; ++i) {
            const int q0 = lower ? ptr[i] : diag[i] + 1;
            const int q1 = lower ? diag[i] : ptr[i + 1];
            for (int q = q0; q < q1; ++q) {
                const int64_t e = sptr[sg] + (int64_t)(q - q0) * 32 + (i - r0);
                ecol[e] = col[q];
                esrc[e] = q;
            }
        }
    }
    // Runs.  A warp that has finished segment p may go on with a segment s
    // of the next level that reads p, taking p's values from its registers
    // instead of from memory.  s joins p's run when
    //  * s is p shifted by a fixed number of rows (same length; from the
    //    run's second segment on also the same width and kind, every column
    //    shifted by the same amount), and the run's segment and row strides,
    //    and from the second segment on its entry stride, stay constant, so
    //    that the warp computes every later segment's addresses without
    //    loads;
    //  * every other segment s reads lies in an earlier run or earlier in
    //    this one.
    // Runs take tickets in the order they were opened, i.e. in the level
    // order of their first segments, so a warp only waits for runs held by
    // warps that took earlier tickets, as before.  Among the candidates p
    // (segments of the previous level that feed at least half of s's rows),
    // the one s reads most often comes first, then the nearest: on a grid in
    // natural order a run follows one x-segment through the y-lines of a
    // plane.
    std::vector<int> run_of(nseg, -1), rlast, rdesc;
    {
        std::vector<std::pair<int, int>> deps;   // (segment, entries of s that read it)
        for (int t = 0; t < nseg; ++t) {
            const int sg = order[t];
            const int r0 = r0v[sg], len = r0v[sg + 1] - r0;
            int R = -1;
            if (run_cap > 1 && kind[sg] && width[sg] > 0 && width[sg] <= RS_RUN_CH) {
                deps.clear();
                for (int i = r0; i < r0 + len; ++i) {
                    const int q0 = lower ? ptr[i] : diag[i] + 1;
                    const int q1 = lower ? diag[i] : ptr[i + 1];
                    for (int q = q0; q < q1; ++q) {
                        const int c = col[q];
                        if (c >= r0 && c < r0 + len) continue;
                        const int d = seg_of[c];
                        auto it = std::find_if(deps.begin(), deps.end(), [&](const std::pair<int, int> &x) { return x.first == d; });
                        if (it == deps.end()) deps.push_back({d, 1});
                        else ++it->second;
                    }
                }
                std::stable_sort(deps.begin(), deps.end(), [&](const std::pair<int, int> &a, const std::pair<int, int> &b) {
                    if (a.second != b.second) return a.second > b.second;
                    return std::abs(r0v[a.first] - r0) < std::abs(r0v[b.first] - r0);
                });
                for (const auto &cand : deps) {
                    if (2 * cand.second < len) break;   // p must feed at least half of s's rows
                    const int p = cand.first, Rp = run_of[p];
                    const int *d = &rdesc[5 * Rp];
                    if (rlast[Rp] != p || d[1] >= run_cap || lev[p] != lev[sg] - 1) continue;
                    if (r0v[p + 1] - r0v[p] != len) continue;
                    const int dseg = sg - p, drow = r0 - r0v[p], dent = sptr[sg] - sptr[p];
                    // the run's first segment takes the general path, so
                    // only its rows need to fit; the entries of the later
                    // segments shift by the row stride from the second on
                    if (d[1] >= 2 && (dseg != d[2] || drow != d[3] || !kind[p] || width[p] != width[sg])) continue;
                    if (d[1] >= 3 && dent != d[4]) continue;
                    bool ok = true;
                    for (int e = 0; d[1] >= 2 && e < width[sg] * 32 && ok; ++e) {
                        const int a = ecol[sptr[p] + e], b = ecol[sptr[sg] + e];
                        ok = (a < 0) == (b < 0) && (a < 0 || b == a + drow);
                    }
                    for (const auto &o : deps) ok = ok && (o.first == p || run_of[o.first] <= Rp);
                    if (!ok) continue;
                    R = Rp;
                    break;
                }
            }
            if (R >= 0) {
                int *d = &rdesc[5 * R];
                if (d[1] == 1) {
                    d[2] = sg - d[0];
                    d[3] = r0 - r0v[d[0]];
                } else if (d[1] == 2) {
                    d[4] = sptr[sg] - sptr[rlast[R]];
                }
                ++d[1];
                rlast[R] = sg;
                run_of[sg] = R;
            } else {
                run_of[sg] = (int)rlast.size();
                rlast.push_back(sg);
                rdesc.insert(rdesc.end(), {sg, 1, 0, 0, 0});
            }
        }
    }
    // Runs pay for their shared-memory ring (which limits a sweep block to
    // two per SM) only where they take over most of the segments and every
    // run can hold a resident warp at once (many independent chains, as in
    // the stacked subdomains of RAS, need the warps more); otherwise every
    // segment stays a run of its own.
    if (2 * (int64_t)rlast.size() > nseg || (int64_t)rlast.size() > run_slots) {
        rlast.clear();
        rdesc.clear();
        for (int t = 0; t < nseg; ++t) {
            rlast.push_back(order[t]);
            rdesc.insert(rdesc.end(), {order[t], 1, 0, 0, 0});
            run_of[order[t]] = t;
        }
    }
    const int nrun = (int)rlast.size();
    int max_run = 0;
    for (int R = 0; R < nrun; ++R) max_run = std::max(max_run, rdesc[5 * R + 1]);
    H.nseg = nseg;
    H.nlev = nlev;
    H.nent = nent;
    H.nrun = nrun;
    H.max_run = max_run;
    H.r0v.swap(r0v);
    H.lev.swap(lev);
    H.order.swap(order);
    H.sptr.swap(sptr);
    H.adjsrc.swap(adjsrc);
    H.ecol.swap(ecol);
    H.esrc.swap(esrc);
    H.rdesc.swap(rdesc);
    H.kind.swap(kind);
    return RS_OK;
}

static int build_segments(rs_ctx *ctx, int nrows, const std::vector<int> &ptr,
                          const std::vector<int> &col, const std::vector<int> &diag, bool lower,
                          int run_cap, int64_t run_slots, SegLayout &S)
{
    SegHost H;
    RS_TRY(seg_schedule(nrows, ptr, col, diag, lower, run_cap, run_slots, H));
    const int nseg = H.nseg, nrun = H.nrun;
    const int64_t nent = H.nent;
    const std::vector<int> &r0v = H.r0v, &sptr = H.sptr, &adjsrc = H.adjsrc, &ecol = H.ecol, &esrc = H.esrc,
                           &rdesc = H.rdesc;
    const std::vector<unsigned char> &kind = H.kind;
    S.nseg = nseg;
    S.nlevels = H.nlev;
    S.nent = nent;
    S.nrun = nrun;
    S.max_run = H.max_run;
    int st = RS_OK;
    st = st ? st : rs_alloc(ctx, (void **)&S.runs, sizeof(int) * 5 * (nrun > 0 ? nrun : 1));
    st = st ? st : rs_alloc(ctx, (void **)&S.sptr, sizeof(int) * (nseg + 1));
    st = st ? st : rs_alloc(ctx, (void **)&S.col, sizeof(int) * (nent > 0 ? nent : 1));
    st = st ? st : rs_alloc(ctx, (void **)&S.src, sizeof(int) * (nent > 0 ? nent : 1));
    st = st ? st : rs_alloc(ctx, (void **)&S.kind, nseg > 0 ? nseg : 1);
    st = st ? st : rs_alloc(ctx, (void **)&S.row0, sizeof(int) * (nseg + 1));
    st = st ? st : rs_alloc(ctx, (void **)&S.adjsrc, sizeof(int) * (nrows > 0 ? nrows : 1));
    if (st) return st;
    cudaStream_t sm = ctx->stream;
    if (nseg) {
        RS_CUDA_TRY(cudaMemcpyAsync(S.runs, rdesc.data(), sizeof(int) * 5 * nrun, cudaMemcpyHostToDevice, sm));
        RS_CUDA_TRY(cudaMemcpyAsync(S.kind, kind.data(), nseg, cudaMemcpyHostToDevice, sm));
    }
    RS_CUDA_TRY(cudaMemcpyAsync(S.sptr, sptr.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, sm));
    RS_CUDA_TRY(cudaMemcpyAsync(S.row0, r0v.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, sm));
    if (nrows)
        RS_CUDA_TRY(cudaMemcpyAsync(S.adjsrc, adjsrc.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice, sm));
    if (nent) {
        RS_CUDA_TRY(cudaMemcpyAsync(S.col, ecol.data(), sizeof(int) * nent, cudaMemcpyHostToDevice, sm));
        RS_CUDA_TRY(cudaMemcpyAsync(S.src, esrc.data(), sizeof(int) * nent, cudaMemcpyHostToDevice, sm));
    }
    RS_CUDA_TRY(cudaStreamSynchronize(sm));
    return RS_OK;
}

static void free_segments(rs_ctx *ctx, SegLayout &S)
{
    rs_free(ctx, S.runs);
    rs_free(ctx, S.sptr);
    rs_free(ctx, S.col);
    rs_free(ctx, S.src);
    rs_free(ctx, S.kind);
    rs_free(ctx, S.row0);
    rs_free(ctx, S.val);
    rs_free(ctx, S.rdiag);
    rs_free(ctx, S.adjsrc);
    rs_free(ctx, S.mul);
    S = SegLayout();
}

static void free_layout(rs_ctx *ctx, TriLayout &T)
{
    rs_free(ctx, T.pos);
    rs_free(ctx, T.warp_level);
    rs_free(ctx, T.level_nwarps);
    rs_free(ctx, T.level_count);
    rs_free(ctx, T.level_done);
    T = TriLayout();
}

// ---------------------------------------------------------------------------
// persistent level-chained sweep
// ---------------------------------------------------------------------------
// Positions are processed one warp (32 positions of one level) at a time.
// Blocks stay resident and take tickets of blockDim positions in order.
// A warp of level l waits until level l-1 is complete (then every level
// below it is complete too: each warp of level l-1 itself waited for l-2),
// which one lane polls.  After its rows are written the warp counts itself
// into its level; the last warp of the level resets the counter and
// publishes the level with a release store of the sweep's epoch.
struct SweepArgs {
    int npad;
    const int *pos;
    const int *wlev, *lnw;
    int *lcount, *ldone;
    SweepState *st;
    int *err;
    long long limit;
    const int *skip;
};

static SweepArgs sweep_args(rs_ctx *ctx, const TriLayout &T, SweepState *st, const int *skip)
{
    SweepArgs a;
    a.npad = T.npad;
    a.pos = T.pos;
    a.wlev = T.warp_level;
    a.lnw = T.level_nwarps;
    a.lcount = T.level_count;
    a.ldone = T.level_done;
    a.st = st;
    a.err = ctx->d_err;
    a.limit = ctx->spin_limit;
    a.skip = skip;
    return a;
}

__device__ __forceinline__ void report_timeout(int *err) { atomicOr(err, RS_DEVERR_TIMEOUT); }

template <class Body>
__device__ __forceinline__ void run_sweep(const SweepArgs &a, Body body)
{
    if (a.skip && *(volatile const int *)a.skip) return;   // uniform over the grid
    __shared__ int s_base, s_epoch;
    if (threadIdx.x == 0) s_epoch = *(volatile int *)&a.st->epoch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_base = (int)atomicAdd(&a.st->ticket, 1u) * (int)blockDim.x;
        __syncthreads();
        const int base = s_base, epoch = s_epoch;
        __syncthreads();
        if (base >= a.npad) break;
        const int w0 = base + warp * 32;
        if (w0 < a.npad) {
            const int lev = a.wlev[w0 >> 5];
            if (lev > 0) {
                if (lane == 0 && !wait_epoch(a.ldone + lev - 1, epoch, a.limit)) report_timeout(a.err);
                __syncwarp();
            }
            body(w0 + lane);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                const int old = atomicAdd(a.lcount + lev, 1);
                if (old == a.lnw[lev] - 1) {
                    a.lcount[lev] = 0;
                    st_release(a.ldone + lev, epoch);
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.st->done, 1u) == gridDim.x - 1) {
            a.st->ticket = 0;
            a.st->done = 0;
            a.st->epoch = s_epoch + 1;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// numeric factorisation (schedule of the L sweep)
// ---------------------------------------------------------------------------
// Scalar ILU(0), IKJ form: for each k < i in row i (ascending): l_ik = a_ik / u_kk,
// then a_ij -= l_ik u_kj for every j > k present in both rows.
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_ilu0_factor(SweepArgs a, const int *__restrict__ ptr, const int *__restrict__ col,
              const int *__restrict__ diagpos, double *lu, int *bad_row)
{
    run_sweep(a, [&](int p) {
        const int row = a.pos[p];
        if (row < 0) return;
        const int e_i = ptr[row + 1];
        const int d_i = diagpos[row];
        for (int q = ptr[row]; q < d_i; ++q) {
            const int k = col[q];
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
            atomicOr(a.err, RS_DEVERR_PIVOT);
            atomicMin(bad_row, row);
        }
    });
}

// bs x bs block helpers (row-major, registers)
template <int BS>
__device__ __forceinline__ void blk_mul(const double *x, const double *y, double *c)
{
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < BS; ++k) s = __dadd_rn(s, __dmul_rn(x[i * BS + k], y[k * BS + j]));
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
k_bilu0_factor(SweepArgs a, const int *__restrict__ ptr, const int *__restrict__ col,
               const int *__restrict__ diagpos, double *lu, double *dinv, int *bad_row)
{
    constexpr int B2 = BS * BS;
    run_sweep(a, [&](int p) {
        const int row = a.pos[p];
        if (row < 0) return;
        const int e_i = ptr[row + 1];
        const int d_i = diagpos[row];
        double x[B2], t[B2], u[B2], c[B2];
        for (int q = ptr[row]; q < d_i; ++q) {
            const int k = col[q];
#pragma unroll
            for (int v = 0; v < B2; ++v) { x[v] = lu[(size_t)q * B2 + v]; t[v] = __ldcg(dinv + (size_t)k * B2 + v); }
            blk_mul<BS>(x, t, c);                      // L_IK
#pragma unroll
            for (int v = 0; v < B2; ++v) lu[(size_t)q * B2 + v] = c[v];
            int qq = q + 1;
            const int e_k = ptr[k + 1];
            for (int r = diagpos[k] + 1; r < e_k; ++r) {
                const int j = col[r];
                while (qq < e_i && col[qq] < j) ++qq;
                if (qq == e_i) break;
                if (col[qq] == j) {
#pragma unroll
                    for (int v = 0; v < B2; ++v) t[v] = __ldcg(lu + (size_t)r * B2 + v);
                    blk_mul<BS>(c, t, u);
#pragma unroll
                    for (int v = 0; v < B2; ++v)
                        lu[(size_t)qq * B2 + v] = __dsub_rn(lu[(size_t)qq * B2 + v], u[v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < B2; ++v) x[v] = lu[(size_t)d_i * B2 + v];
        if (!blk_inverse<BS>(x, t)) {
            atomicOr(a.err, RS_DEVERR_PIVOT);
            atomicMin(bad_row, row);
#pragma unroll
            for (int v = 0; v < B2; ++v) t[v] = 0.0;
        }
#pragma unroll
        for (int v = 0; v < B2; ++v) dinv[(size_t)row * B2 + v] = t[v];
    });
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

// D_i (the inverse of row i's diagonal block: 1 / u_ii for scalars) of a row
template <int BS>
__device__ __forceinline__ void diag_inverse(int row, const int *__restrict__ diagpos, const double *__restrict__ lu,
                                             const double *__restrict__ dinv, double (&D)[BS * BS])
{
    if (BS == 1) {
        D[0] = 1.0 / lu[diagpos[row]];
    } else {
#pragma unroll
        for (int v = 0; v < BS * BS; ++v) D[v] = dinv[(size_t)row * BS * BS + v];
    }
}

// The U triangle premultiplied by the inverted diagonal: entry e of row i
// holds D_i U_ij, so that the U sweep reads z_i = D_i y_i - sum_j (D_i U_ij) z_j
// directly.  One warp per segment; products in FP64, rounded once to T.
template <int BS, typename T>
__global__ void k_gather_useg(int nseg, int64_t nent, const int *__restrict__ sptr, const int *__restrict__ row0,
                              const int *__restrict__ src, const int *__restrict__ diagpos,
                              const double *__restrict__ lu, const double *__restrict__ dinv, T *__restrict__ val)
{
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int seg = blockIdx.x * wpb + (threadIdx.x >> 5); seg < nseg; seg += gridDim.x * wpb) {
        const int row = row0[seg] + lane;
        const bool active = row < row0[seg + 1];
        double D[BS * BS];
#pragma unroll
        for (int v = 0; v < BS * BS; ++v) D[v] = 0.0;
        if (active) diag_inverse<BS>(row, diagpos, lu, dinv, D);
        for (int64_t e = sptr[seg] + lane; e < sptr[seg + 1]; e += 32) {
            const int q = src[e];
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int j = 0; j < BS; ++j) {
                    double t = 0.0;
                    if (q >= 0)
#pragma unroll
                        for (int k = 0; k < BS; ++k) t = fma(D[i * BS + k], lu[(size_t)q * BS * BS + k * BS + j], t);
                    val[(size_t)(i * BS + j) * nent + e] = (T)t;
                }
        }
    }
}

// Multipliers of the five steps of the segment scan.  Lane t of a chain
// segment maps its neighbour's value to its own by the affine map
// x_t = c_t + A_t x_{t-1} (L: A_t = -L_{t,t-1}) or x_t = c_t + A_t x_{t+1}
// (U: A_t = -D_t U_{t,t+1}), A_t = 0 where the neighbour lies outside the
// segment.  Step k (offset o = 2^k) composes each lane's map with the map of
// lane t -/+ o; the c parts depend on the right-hand side, the A parts do not,
// so the products A_t^{(k)} are formed here once per factorisation:
// A^{(0)} = A, A^{(k+1)}_t = A^{(k)}_t A^{(k)}_{t-/+o} (for lanes that take).
// Stored per segment as [5][bs*bs][32] in T, computed in FP64.
template <int BS, typename T, bool LOWER>
__global__ void k_scan_mul(int nseg, const int *__restrict__ row0, const int *__restrict__ adjsrc,
                           const int *__restrict__ diagpos, const double *__restrict__ lu,
                           const double *__restrict__ dinv, T *__restrict__ mul)
{
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int seg = blockIdx.x * wpb + (threadIdx.x >> 5); seg < nseg; seg += gridDim.x * wpb) {
        const int row = row0[seg] + lane;
        const int q = row < row0[seg + 1] ? adjsrc[row] : -1;
        double a[BS * BS];
#pragma unroll
        for (int v = 0; v < BS * BS; ++v) a[v] = 0.0;
        if (q >= 0) {
            if (LOWER) {
#pragma unroll
                for (int v = 0; v < BS * BS; ++v) a[v] = -lu[(size_t)q * BS * BS + v];
            } else {
                double D[BS * BS];
                diag_inverse<BS>(row, diagpos, lu, dinv, D);
#pragma unroll
                for (int i = 0; i < BS; ++i)
#pragma unroll
                    for (int j = 0; j < BS; ++j) {
                        double t = 0.0;
#pragma unroll
                        for (int k = 0; k < BS; ++k) t = fma(D[i * BS + k], lu[(size_t)q * BS * BS + k * BS + j], t);
                        a[i * BS + j] = -t;
                    }
            }
        }
        T *out = mul + (size_t)seg * 5 * BS * BS * 32;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
            for (int v = 0; v < BS * BS; ++v) out[(k * BS * BS + v) * 32 + lane] = (T)a[v];
            if (k == 4) break;
            const int o = 1 << k;
            double ap[BS * BS], na[BS * BS];
#pragma unroll
            for (int v = 0; v < BS * BS; ++v)
                ap[v] = LOWER ? __shfl_up_sync(0xffffffffu, a[v], o) : __shfl_down_sync(0xffffffffu, a[v], o);
            const bool take = LOWER ? lane >= o : lane + o < 32;
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int j = 0; j < BS; ++j) {
                    double t = 0.0;
#pragma unroll
                    for (int m = 0; m < BS; ++m) t = fma(a[i * BS + m], ap[m * BS + j], t);
                    na[i * BS + j] = t;
                }
            if (take) {
#pragma unroll
                for (int v = 0; v < BS * BS; ++v) a[v] = na[v];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// triangular sweeps: the value is its own ready flag
// ---------------------------------------------------------------------------
// Before a sweep every entry of its work vector holds a signalling-NaN bit
// pattern that arithmetic never produces; a warp polls the entries it depends
// on until they change, and publishes each value with one plain 8-byte (or
// 4-byte) store, which is single-copy atomic.  The L sweep resets the U
// sweep's work vector to the sentinel (row by row) and the U sweep resets the
// L sweep's, so no clearing pass is needed.

// ---------------------------------------------------------------------------
// segment sweeps
// ---------------------------------------------------------------------------
// One warp per segment (up to 32 consecutive rows or block rows), segments
// taken in level order from a warp-granular ticket, so every awaited segment
// is held by a warp that is already running.  Each lane subtracts the
// contributions of its row's columns outside the segment (loaded together,
// polled on the sentinel).  What remains inside the segment is, for the usual
// stencils in natural order, a first-order recurrence y_t = c_t + A_t y_{t-1}
// (L) or z_t = c_t + A_t z_{t+1} (U) with A_t a bs x bs block, solved by a
// 5-step warp scan of affine maps whose matrix parts (products of the A_t)
// are formed once per factorisation and staged into shared memory while the
// warp waits, so that after the last awaited value arrives a lane does only
// its subtractions and five multiply-adds of bs-vectors; any other
// in-segment pattern is resolved lane by lane with broadcasts.
struct SegArgs {
    int nrows, nrun;
    unsigned sleep_cap;
    const int *runs, *sptr, *ecol, *row0;
    const unsigned char *kind;
    int64_t nent;
    int npr;                 // padded row count of the diagonal arrays
    SweepState *st;
    int *err;
    long long limit;
    const int *skip;
};

static SegArgs seg_args(rs_ctx *ctx, const SegLayout &S, int nrows, SweepState *st, const int *skip)
{
    SegArgs a;
    a.nrows = nrows;
    a.nrun = S.nrun;
    a.sleep_cap = ctx->sleep_cap_ns;
    a.runs = S.runs;
    a.sptr = S.sptr;
    a.ecol = S.col;
    a.row0 = S.row0;
    a.kind = S.kind;
    a.nent = S.nent;
    a.npr = S.nseg * 32;
    a.st = st;
    a.err = ctx->d_err;
    a.limit = ctx->spin_limit;
    a.skip = skip;
    return a;
}

// acc -= sum of V_e x[c_e] over this lane's entries whose block column lies
// outside [lo, hi).  All lanes load their outside values at once; while any
// lane still sees a sentinel the whole warp sleeps once and reloads only the
// pending values.
template <int BS, typename T>
__device__ __forceinline__ void seg_external(const SegArgs &g, const T *__restrict__ val, const T *x, int off,
                                             int w, int lane, int lo, int hi, T (&acc)[BS])
{
    typedef typename Sentinel<T>::bits_t B;
    constexpr int CH = BS == 1 ? 8 : 4;
    for (int e0 = 0; e0 < w; e0 += CH) {
        int c[CH];
        T v[CH][BS * BS];
        B b[CH][BS];
        bool ext[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int64_t idx = off + (int64_t)(e0 + j) * 32 + lane;
            c[j] = e0 + j < w ? g.ecol[idx] : -1;
#pragma unroll
            for (int q = 0; q < BS * BS; ++q) v[j][q] = c[j] >= 0 ? val[q * g.nent + idx] : T(0);
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            ext[j] = c[j] >= 0 && (c[j] < lo || c[j] >= hi);
#pragma unroll
            for (int k = 0; k < BS; ++k) b[j][k] = ext[j] ? ld_relaxed_bits(x + (size_t)c[j] * BS + k) : (B)0;
        }
        // back-off: none after the first look, then 16 ns doubling up to
        // sleep_cap (0: no sleep); the time limit runs from the first look
        unsigned ns = 0;
        long long t0 = 0;
        for (bool first = true;; first = false) {
            bool pend = false;
#pragma unroll
            for (int j = 0; j < CH; ++j)
#pragma unroll
                for (int k = 0; k < BS; ++k) pend |= ext[j] && b[j][k] == Sentinel<T>::bits;
            if (!__any_sync(0xffffffffu, pend)) break;
            if (first) {
                t0 = clock64();
            } else {
                if (clock64() - t0 > g.limit) {
                    if (pend) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                    break;
                }
                if (ns) __nanosleep(ns);
            }
            ns = first ? min(16u, g.sleep_cap) : min(ns * 2, g.sleep_cap);
#pragma unroll
            for (int j = 0; j < CH; ++j)
#pragma unroll
                for (int k = 0; k < BS; ++k)
                    if (ext[j] && b[j][k] == Sentinel<T>::bits) b[j][k] = ld_relaxed_bits(x + (size_t)c[j] * BS + k);
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (!ext[j]) continue;
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int k = 0; k < BS; ++k) acc[i] = msub(acc[i], v[j][i * BS + k], bits_to(T(), b[j][k]));
        }
    }
}

// The scan multipliers of a chain segment (5 * bs*bs * 32 values, a multiple
// of 16 bytes) are copied into the warp's slot of shared memory with cp.async
// before the warp polls, and waited for after: they never sit on the path
// from the last awaited value to the stores.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int BS, typename T>
struct ScanStage {
    static constexpr int N = 5 * BS * BS * 32;                  // elements per segment
    static constexpr int PIECES = N * (int)sizeof(T) / 16;      // 16-byte pieces
    static_assert(N * sizeof(T) % 16 == 0, "stage is a multiple of 16 bytes");
};

template <int BS, typename T>
__device__ __forceinline__ void stage_mul(const T *__restrict__ mul, int seg, T *stage, int lane)
{
    const char *src = (const char *)(mul + (size_t)seg * ScanStage<BS, T>::N);
    char *dst = (char *)stage;
    __syncwarp();   // every lane is done reading the previous segment's multipliers
    for (int c = lane; c < ScanStage<BS, T>::PIECES; c += 32) cp_async16(dst + 16 * c, src + 16 * c);
}

// x_t = c_t + A_t x_{t-/+1} over the warp: five steps of
// acc_t += A^{(k)}_t acc_{t-/+o} with the staged multipliers A^{(k)}.
template <int BS, typename T, bool LOWER>
__device__ __forceinline__ void scan_staged(const T *stage, T (&acc)[BS], int lane, bool run = false)
{
    // a run keeps its RS_RUN_P staged segments in flight
    if (run) asm volatile("cp.async.wait_group %0;" ::"n"(RS_RUN_P) : "memory");
    else cp_async_wait_all();
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int o = 1 << k;
        T bp[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i)
            bp[i] = LOWER ? __shfl_up_sync(0xffffffffu, acc[i], o) : __shfl_down_sync(0xffffffffu, acc[i], o);
        if (LOWER ? lane >= o : lane + o < 32) {
#pragma unroll
            for (int i = 0; i < BS; ++i)
#pragma unroll
                for (int j = 0; j < BS; ++j) acc[i] = mad(stage[((k * BS + i) * BS + j) * 32 + lane], bp[j], acc[i]);
        }
    }
}

template <int BS, typename T>
__device__ __forceinline__ void seg_end(const SegArgs &g)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&g.st->done, 1u) == gridDim.x - 1) {
            g.st->ticket = 0;
            g.st->done = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// runs: the later segments of a run (scalar factors only)
// ---------------------------------------------------------------------------
// Segment k of a run is its first segment shifted by k row strides; from
// the second segment on, its entries and columns follow by the run's strides
// as well (the first segment, which may differ, takes the general path).  A
// warp copies the factor values, multipliers and right-hand side of segment
// k + RS_RUN_P into a ring of shared-memory slots (cp.async, one group per
// segment) after it has scanned segment k, so the HBM latency stays off the
// run's path; it takes a first look at the values segment k + 1 reads from
// other warps one segment ahead.  Entries that read segment k - 1 take its
// values from the warp's registers (a shuffle) instead of polling memory.
// The arithmetic is that of the general path, in the same order, so a run
// changes no result.

struct RunCtx {
    int seg0, dseg, drow, dent, row0, len, off1, w;
    int c1[RS_RUN_CH];   // this lane's columns in the second segment, or -1
    int sl[RS_RUN_CH];   // the lane of the previous segment holding that column
    // entries read from memory / from the previous segment: the same at
    // every step, since columns and rows shift together
    unsigned ext, prv;
    bool any_ext;        // does any lane read from memory (warp-uniform)
};

template <typename T>
struct RunLook {         // first look at the values a segment reads from memory
    typename Sentinel<T>::bits_t b[RS_RUN_CH];
};

// segment k >= 1 of a run: rows row0 + k drow, segment seg0 + k dseg,
// entries from off1 + (k - 1) dent, columns c1 + (k - 1) drow
__device__ __forceinline__ RunCtx run_ctx(const SegArgs &g, const int *rd, int row0, int len, int lane)
{
    RunCtx rc;
    rc.seg0 = rd[0];
    rc.dseg = rd[2];
    rc.drow = rd[3];
    rc.dent = rd[4];
    rc.row0 = row0;
    rc.len = len;
    const int s1 = rc.seg0 + rc.dseg;
    rc.off1 = g.sptr[s1];
    rc.w = (g.sptr[s1 + 1] - rc.off1) >> 5;
    rc.ext = 0;
    rc.prv = 0;
#pragma unroll
    for (int j = 0; j < RS_RUN_CH; ++j) {
        const int c = j < rc.w ? g.ecol[rc.off1 + j * 32 + lane] : -1;
        rc.c1[j] = c;
        rc.sl[j] = (c - row0) & 31;
        // at step k the segment is [row0 + k drow, + len) and the previous
        // one [row0 + (k - 1) drow, + len); the column is c + (k - 1) drow
        const bool own = c - row0 - rc.drow >= 0 && c - row0 - rc.drow < len;
        const bool prv = !own && c - row0 >= 0 && c - row0 < len;
        rc.ext |= (unsigned)(c >= 0 && !own && !prv) << j;
        rc.prv |= (unsigned)(c >= 0 && prv) << j;
    }
    rc.any_ext = __any_sync(0xffffffffu, rc.ext != 0);
    return rc;
}

__device__ __forceinline__ void cp_async_n(void *smem, const void *gmem, int bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// copy segment k's per-lane data into its ring slot (one cp.async group,
// committed by the caller); L: r_i and the U work vector's reset;
// U: y_i and D_i
template <typename T, bool LOWER>
__device__ __forceinline__ void run_stage(const RunCtx &rc, int k, int slot, int lane, unsigned long long *ring,
                                          const T *__restrict__ val, const T *__restrict__ mul,
                                          const double *__restrict__ r, const T *yin, T *reset,
                                          const T *__restrict__ dinv)
{
    const int row = rc.row0 + k * rc.drow + lane;
    const int64_t off = rc.off1 + (int64_t)(k - 1) * rc.dent;
    unsigned long long *sl = ring + slot * RS_RUN_WORDS * 32 + lane;
#pragma unroll
    for (int j = 0; j < RS_RUN_CH; ++j)
        if (rc.c1[j] >= 0) cp_async_n(sl + j * 32, val + off + j * 32 + lane, sizeof(T));
    const T *ms = mul + (size_t)(rc.seg0 + k * rc.dseg) * ScanStage<1, T>::N + lane;
#pragma unroll
    for (int q = 0; q < 5; ++q) cp_async_n(sl + (RS_RUN_CH + q) * 32, ms + q * 32, sizeof(T));
    if (lane < rc.len) {
        if (LOWER) {
            cp_async_n(sl + (RS_RUN_CH + 5) * 32, r + row, 8);
            reset[row] = bits_to(T(), Sentinel<T>::bits);
        } else {
            cp_async_n(sl + (RS_RUN_CH + 5) * 32, yin + row, sizeof(T));
            cp_async_n(sl + (RS_RUN_CH + 6) * 32, dinv + row, sizeof(T));
        }
    }
}

// first look at segment k's values from memory (k >= 1); x is the vector
// the sweep produces
template <typename T>
__device__ __forceinline__ void run_look(const RunCtx &rc, int k, const T *x, RunLook<T> &s)
{
#pragma unroll
    for (int j = 0; j < RS_RUN_CH; ++j)
        s.b[j] = ((rc.ext >> j) & 1u) ? ld_relaxed_bits(x + (rc.c1[j] + (k - 1) * rc.drow)) : 0;
}

// finish segment k of the run from its staged slot: wait for the values
// read from memory, subtract, scan, store; returns this lane's value (the
// next segment's prev)
template <typename T, bool LOWER>
__device__ __forceinline__ T run_finish(const SegArgs &g, const RunCtx &rc, int k, int lane,
                                        const unsigned long long *ring, RunLook<T> &s, T prev, T *x, T *yin,
                                        double *__restrict__ out, double sc, bool &late)
{
    const int r0 = rc.row0 + k * rc.drow, row = r0 + lane;
    const bool active = lane < rc.len;
    const unsigned long long *sl = ring + (k % RS_RUN_SLOTS) * RS_RUN_WORDS * 32 + lane;
    T v[RS_RUN_CH], m[5];
#pragma unroll
    for (int j = 0; j < RS_RUN_CH; ++j) v[j] = *(const T *)(sl + j * 32);
#pragma unroll
    for (int q = 0; q < 5; ++q) m[q] = *(const T *)(sl + (RS_RUN_CH + q) * 32);
    T acc = T(0);
    if (active) {
        if (LOWER) {
            const double rv = *(const double *)(sl + (RS_RUN_CH + 5) * 32);
            acc = (T)(sc == 1.0 ? rv : rv * sc);
        } else {
            const T yv = *(const T *)(sl + (RS_RUN_CH + 5) * 32);
            acc = mad(*(const T *)(sl + (RS_RUN_CH + 6) * 32), yv, T(0));
            yin[row] = bits_to(T(), Sentinel<T>::bits);   // the copy of y_i is complete
        }
    }
    unsigned ns = 0;
    long long t0 = 0;
    for (bool first = true; rc.any_ext; first = false) {
        bool pend = false;
#pragma unroll
        for (int j = 0; j < RS_RUN_CH; ++j) pend |= ((rc.ext >> j) & 1u) && s.b[j] == Sentinel<T>::bits;
        if (!__any_sync(0xffffffffu, pend)) break;
        if (first) {
            t0 = clock64();
        } else {
            // one expired wait ends the waiting for the rest of the run
            if (late || clock64() - t0 > g.limit) {
                if (pend) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                late = true;
                break;
            }
            if (ns) __nanosleep(ns);
        }
        ns = first ? min(16u, g.sleep_cap) : min(ns * 2, g.sleep_cap);
#pragma unroll
        for (int j = 0; j < RS_RUN_CH; ++j)
            if (((rc.ext >> j) & 1u) && s.b[j] == Sentinel<T>::bits) s.b[j] = ld_relaxed_bits(x + (rc.c1[j] + (k - 1) * rc.drow));
    }

#pragma unroll
    for (int j = 0; j < RS_RUN_CH; ++j) {
        if (j >= rc.w) break;
        const T xp = __shfl_sync(0xffffffffu, prev, rc.sl[j]);
        if ((rc.ext >> j) & 1u) acc = msub(acc, v[j], bits_to(T(), s.b[j]));
        else if ((rc.prv >> j) & 1u) acc = msub(acc, v[j], xp);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int o = 1 << q;
        const T bp = LOWER ? __shfl_up_sync(0xffffffffu, acc, o) : __shfl_down_sync(0xffffffffu, acc, o);
        if (LOWER ? lane >= o : lane + o < 32) acc = mad(m[q], bp, acc);
    }
    if (active) {
        st_relaxed(x + row, acc);
        if (!LOWER) out[row] = (double)acc;
    }
    return acc;
}



// L y = r (unit lower).  scale (device, optional) multiplies r on load;
// zreset is the U sweep's work vector.
template <int BS, typename T, bool RUNS>
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_lsolve_seg(SegArgs g, const T *__restrict__ val, const T *__restrict__ mul, const double *__restrict__ r,
             const double *__restrict__ scale, T *y, T *zreset)
{
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    if (g.skip && *(volatile const int *)g.skip) return;
    const int lane = threadIdx.x & 31;
    T *stage = (T *)sweep_smem + (threadIdx.x >> 5) * ScanStage<BS, T>::N;
    unsigned long long *ring = (unsigned long long *)((T *)sweep_smem + (blockDim.x >> 5) * ScanStage<BS, T>::N) +
                               (threadIdx.x >> 5) * RS_RUN_RING;
    const double sc = scale ? *scale : 1.0;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&g.st->ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= g.nrun) break;
        const int *rd = g.runs + 5 * t;
        const int seg = rd[0];
        const int count = RUNS ? rd[1] : 1;
        const int row0 = g.row0[seg], len = g.row0[seg + 1] - row0, row = row0 + lane;
        const bool active = lane < len;
        const int off = g.sptr[seg];
        const int w = (g.sptr[seg + 1] - off) >> 5;
        const bool chain = g.kind[seg];   // read before the polls, which order later loads
        if (chain) stage_mul<BS, T>(mul, seg, stage, lane);
        T acc[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            acc[k] = T(0);
            if (active) {
                acc[k] = (T)(sc == 1.0 ? r[(size_t)row * BS + k] : r[(size_t)row * BS + k] * sc);
                zreset[(size_t)row * BS + k] = bits_to(T(), Sentinel<T>::bits);
            }
        }
        RunCtx rc;
        RunLook<T> nx;
        if constexpr (RUNS) {
            if (count > 1) {
                rc = run_ctx(g, rd, row0, len, lane);
                cp_async_commit();   // the first segment's multipliers
                for (int k = 1; k <= RS_RUN_P; ++k) {
                    if (k < count) run_stage<T, true>(rc, k, k % RS_RUN_SLOTS, lane, ring, val, mul, r, nullptr, zreset, nullptr);
                    cp_async_commit();
                }
                run_look<T>(rc, 1, y, nx);
            }
        }
        seg_external<BS, T>(g, val, y, off, w, lane, row0, row0 + len, acc);
        if (chain) {
            scan_staged<BS, T, true>(stage, acc, lane, count > 1);
        } else {
            // lane k is final once lanes 0..k-1 have been applied
            for (int k = 0; k < 31; ++k) {
                T yk[BS];
#pragma unroll
                for (int i = 0; i < BS; ++i) yk[i] = __shfl_sync(0xffffffffu, acc[i], k);
                if (lane > k) {
                    for (int e = 0; e < w; ++e) {
                        const int64_t idx = off + (int64_t)e * 32 + lane;
                        if (g.ecol[idx] != row0 + k) continue;
#pragma unroll
                        for (int i = 0; i < BS; ++i)
#pragma unroll
                            for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], val[(i * BS + j) * g.nent + idx], yk[j]);
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < BS; ++k) st_relaxed(y + (size_t)row * BS + k, acc[k]);
        }
        if constexpr (RUNS) {
            T prev = acc[0];
            bool late = false;
            for (int k = 1; k < count; ++k) {
                RunLook<T> cur = nx;
                run_look<T>(rc, min(k + 1, count - 1), y, nx);
                cp_async_wait<RS_RUN_P - 1>();   // segment k's slot has arrived
                prev = run_finish<T, true>(g, rc, k, lane, ring, cur, prev, y, nullptr, nullptr, sc, late);
                // segment k + RS_RUN_P into its slot, or (past the run's end,
                // so that no branch splits this block from the scan) the last
                // segment again into the spare slot
                const bool in = k + RS_RUN_P < count;
                run_stage<T, true>(rc, in ? k + RS_RUN_P : count - 1, in ? (k + RS_RUN_P) % RS_RUN_SLOTS : RS_RUN_SLOTS,
                                   lane, ring, val, mul, r, nullptr, zreset, nullptr);
                cp_async_commit();
            }
        }
    }
    seg_end<BS, T>(g);
}

// U z = y.  val holds D_i U_ij (D_i = 1/u_ii or inv(U_II)) and dinv holds
// D_i per row, plane-major, so z_i = D_i y_i - sum_j (D_i U_ij) z_j; z carries
// values between rows and is reset to the sentinel by the next L sweep; out
// (FP64) receives the result; y is reset for the next L sweep.
template <int BS, typename T, bool RUNS>
__global__ void __launch_bounds__(RS_SWEEP_THREADS)
k_usolve_seg(SegArgs g, const T *__restrict__ val, const T *__restrict__ mul, const T *__restrict__ dinv, T *y,
             T *z, double *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    if (g.skip && *(volatile const int *)g.skip) return;
    const int lane = threadIdx.x & 31;
    T *stage = (T *)sweep_smem + (threadIdx.x >> 5) * ScanStage<BS, T>::N;
    unsigned long long *ring = (unsigned long long *)((T *)sweep_smem + (blockDim.x >> 5) * ScanStage<BS, T>::N) +
                               (threadIdx.x >> 5) * RS_RUN_RING;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&g.st->ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= g.nrun) break;
        const int *rd = g.runs + 5 * t;
        const int seg = rd[0];
        const int count = RUNS ? rd[1] : 1;
        const int row0 = g.row0[seg], len = g.row0[seg + 1] - row0, row = row0 + lane;
        const bool active = lane < len;
        const int off = g.sptr[seg];
        const int w = (g.sptr[seg + 1] - off) >> 5;
        const bool chain = g.kind[seg];   // read before the polls, which order later loads
        if (chain) stage_mul<BS, T>(mul, seg, stage, lane);
        T yv[BS], acc[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            yv[k] = T(0);
            if (active) {
                yv[k] = y[(size_t)row * BS + k];
                y[(size_t)row * BS + k] = bits_to(T(), Sentinel<T>::bits);
            }
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T sum = T(0);
#pragma unroll
            for (int k = 0; k < BS; ++k) sum = mad(active ? dinv[(size_t)(i * BS + k) * g.npr + row] : T(0), yv[k], sum);
            acc[i] = sum;
        }
        RunCtx rc;
        RunLook<T> nx;
        if constexpr (RUNS) {
            if (count > 1) {
                rc = run_ctx(g, rd, row0, len, lane);
                cp_async_commit();   // the first segment's multipliers
                for (int k = 1; k <= RS_RUN_P; ++k) {
                    if (k < count) run_stage<T, false>(rc, k, k % RS_RUN_SLOTS, lane, ring, val, mul, nullptr, y, nullptr, dinv);
                    cp_async_commit();
                }
                run_look<T>(rc, 1, z, nx);
            }
        }
        seg_external<BS, T>(g, val, z, off, w, lane, row0, row0 + len, acc);
        if (chain) {
            scan_staged<BS, T, false>(stage, acc, lane, count > 1);
        } else {
            // lane k is final once lanes k+1..31 have been applied
            for (int k = 31; k > 0; --k) {
                T zk[BS];
#pragma unroll
                for (int i = 0; i < BS; ++i) zk[i] = __shfl_sync(0xffffffffu, acc[i], k);
                if (lane < k) {
                    for (int e = 0; e < w; ++e) {
                        const int64_t idx = off + (int64_t)e * 32 + lane;
                        if (g.ecol[idx] != row0 + k) continue;
#pragma unroll
                        for (int i = 0; i < BS; ++i)
#pragma unroll
                            for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], val[(i * BS + j) * g.nent + idx], zk[j]);
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < BS; ++k) {
                st_relaxed(z + (size_t)row * BS + k, acc[k]);
                out[(size_t)row * BS + k] = (double)acc[k];
            }
        }
        if constexpr (RUNS) {
            T prev = acc[0];
            bool late = false;
            for (int k = 1; k < count; ++k) {
                RunLook<T> cur = nx;
                run_look<T>(rc, min(k + 1, count - 1), z, nx);
                cp_async_wait<RS_RUN_P - 1>();   // segment k's slot has arrived
                prev = run_finish<T, false>(g, rc, k, lane, ring, cur, prev, z, y, out, 1.0, late);
                const bool in = k + RS_RUN_P < count;
                run_stage<T, false>(rc, in ? k + RS_RUN_P : count - 1, in ? (k + RS_RUN_P) % RS_RUN_SLOTS : RS_RUN_SLOTS,
                                    lane, ring, val, mul, nullptr, y, nullptr, dinv);
                cp_async_commit();
            }
        }
    }
    seg_end<BS, T>(g);
}

// diagonal inverses per row (plane-major): 1/u_ii for scalars, inv(U_II) for blocks
template <typename T>
__global__ void k_gather_dinv(int nrows, int npr, int b2, const int *__restrict__ diagpos,
                              const double *__restrict__ lu, const double *__restrict__ dinv, T *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npr; i += gridDim.x * blockDim.x)
        for (int q = 0; q < b2; ++q) {
            double v = 0.0;
            if (i < nrows) v = b2 == 1 ? 1.0 / lu[diagpos[i]] : dinv[(size_t)i * b2 + q];
            out[(size_t)q * npr + i] = (T)v;
        }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// The sweep schedule of a pattern, host only (see rs.h).
extern "C" int rs_sweep_schedule(int32_t nrows, const int32_t *ptr, const int32_t *col, int32_t lower,
                                 int32_t run_cap, int64_t run_slots, int32_t *nseg, int32_t *nlevels,
                                 int32_t *nrun, int32_t *seg_row0, int32_t *seg_level, int32_t *runs)
{
    if (nrows < 0 || !ptr || !nseg || !nlevels || !nrun || run_cap < 1 || run_slots < 1) return RS_ERR_INVALID_ARG;
    if (ptr[0] != 0) return RS_ERR_INVALID_ARG;
    // the whole of ptr first: it must not decrease (so ptr[nrows] >= 0 and
    // no row reads past the column array) before any column is read
    for (int i = 0; i < nrows; ++i)
        if (ptr[i + 1] < ptr[i]) return RS_ERR_BAD_PATTERN;
    if (ptr[nrows] > 0 && !col) return RS_ERR_INVALID_ARG;
    std::vector<int> hp(ptr, ptr + nrows + 1), hc(col, col + ptr[nrows]), diag(nrows, -1);
    for (int i = 0; i < nrows; ++i) {
        for (int q = hp[i]; q < hp[i + 1]; ++q) {
            if (hc[q] < 0 || hc[q] >= nrows || (q > hp[i] && hc[q] <= hc[q - 1])) return RS_ERR_BAD_PATTERN;
            if (hc[q] == i) diag[i] = q;
        }
        if (diag[i] < 0) return RS_ERR_BAD_PATTERN;
    }
    SegHost H;
    RS_TRY(seg_schedule(nrows, hp, hc, diag, lower != 0, run_cap, run_slots, H));
    *nseg = H.nseg;
    *nlevels = H.nlev;
    *nrun = H.nrun;
    if (seg_row0) std::copy(H.r0v.begin(), H.r0v.end(), seg_row0);
    if (seg_level) std::copy(H.lev.begin(), H.lev.end(), seg_level);
    if (runs) std::copy(H.rdesc.begin(), H.rdesc.end(), runs);
    return RS_OK;
}

int rs_ilu_create(rs_ctx *ctx, int bs, int nrows, int64_t nnzb, const int *d_ptr, const int *d_col,
                  const std::vector<int> &h_ptr, const std::vector<int> &h_col, int fp32, int sweep_mode,
                  int run_cap, IluFactor **out, int *bad_row)
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
    // row-level schedule of the factorisation
    int st = build_layout(ctx, nrows, h_ptr, h_col, diag, f->L);
    // the sweeps: wavefronts on a structured 7-point pattern, else segments
    int gx = 0, gy = 0, gz = 0;
    const bool wave = sweep_mode != 1 && rs_wave_detect(nrows, h_ptr, h_col, &gx, &gy, &gz);
    if (!wave) {
        // runs are taken by the scalar FP64 sweeps.  In FP32 a hop between
        // warps already costs about what a step of a run does (0.8 against
        // 0.7 us at 128 x 128 x 64), and waiting inside a run adds more than
        // that saves; run_cap > 0 sets the longest run for either precision
        // (1: every segment is a run of its own).
        int cap = run_cap > 0 ? run_cap : fp32 ? 1 : 1 << 30;
        if (bs != 1) cap = 1;
        // warps resident at once in sweep blocks that carry the runs' ring
        const int64_t run_block = (int64_t)(RS_SWEEP_THREADS / 32) *
                                  (5 * 32 * (fp32 ? sizeof(float) : sizeof(double)) +
                                   RS_RUN_RING * sizeof(unsigned long long));
        const int64_t run_slots =
            std::max<int64_t>(1, (int64_t)227 * 1024 / run_block) * (RS_SWEEP_THREADS / 32) * ctx->num_sms;
        st = st ? st : build_segments(ctx, nrows, h_ptr, h_col, diag, true, cap, run_slots, f->SL);
        st = st ? st : build_segments(ctx, nrows, h_ptr, h_col, diag, false, cap, run_slots, f->SU);
        // sweep blocks: a single dependency chain (global ILU in natural
        // order) gains nothing from more warps, which only add polling; many
        // independent chains (the stacked subdomains of RAS) do.  Aim at
        // three warps per segment of a level, between 4 and 8 blocks per SM.
        for (SegLayout *S : {&f->SL, &f->SU}) {
            const int wpb = RS_SWEEP_THREADS / 32;
            const int64_t per_level = S->nlevels > 0 ? (int64_t)S->nseg / S->nlevels : 0;
            int64_t g = (3 * per_level + wpb - 1) / wpb;
            g = std::max<int64_t>(g, ctx->sweep_blocks);
            S->grid = (int)std::min<int64_t>(g, (int64_t)8 * ctx->num_sms);
        }
        st = st ? st : rs_alloc(ctx, &f->SL.val, esz * b2 * (f->SL.nent > 0 ? f->SL.nent : 1));
        st = st ? st : rs_alloc(ctx, &f->SU.val, esz * b2 * (f->SU.nent > 0 ? f->SU.nent : 1));
        st = st ? st : rs_alloc(ctx, &f->SU.rdiag, esz * b2 * ((size_t)f->SU.nseg * 32 > 0 ? (size_t)f->SU.nseg * 32 : 1));
        st = st ? st : rs_alloc(ctx, &f->SL.mul, esz * b2 * 5 * 32 * (f->SL.nseg > 0 ? (size_t)f->SL.nseg : 1));
        st = st ? st : rs_alloc(ctx, &f->SU.mul, esz * b2 * 5 * 32 * (f->SU.nseg > 0 ? (size_t)f->SU.nseg : 1));
    }
    st = st ? st : rs_alloc(ctx, (void **)&f->diagpos, sizeof(int) * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->lu, sizeof(double) * b2 * (nnzb > 0 ? nnzb : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->dinv, sizeof(double) * b2 * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, (void **)&f->state, sizeof(SweepState));
    if (wave) {
        st = st ? st : rs_wave_create(f, gx, gy, gz);
        if (st) { rs_ilu_destroy(f); return st; }
    } else {
    st = st ? st : rs_alloc(ctx, &f->ywork, esz * bs * (nrows > 0 ? nrows : 1));
    st = st ? st : rs_alloc(ctx, &f->zwork, esz * bs * (nrows > 0 ? nrows : 1));
    if (st) { rs_ilu_destroy(f); return st; }
    {
        const int64_t nv = (int64_t)bs * (nrows > 0 ? nrows : 1);
        const int g = (int)std::min<int64_t>((nv + 255) / 256, 4096);
        if (fp32) {
            k_fill_sentinel<float><<<g, 256, 0, ctx->stream>>>(nv, (float *)f->ywork);
            k_fill_sentinel<float><<<g, 256, 0, ctx->stream>>>(nv, (float *)f->zwork);
        } else {
            k_fill_sentinel<double><<<g, 256, 0, ctx->stream>>>(nv, (double *)f->ywork);
            k_fill_sentinel<double><<<g, 256, 0, ctx->stream>>>(nv, (double *)f->zwork);
        }
        RS_TRY(rs_check_launch(ctx));
        ctx->launches++;
    }
    }
    SweepState s0 = {0u, 0u, 1, 0};
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
    free_segments(ctx, f->SL);
    free_segments(ctx, f->SU);
    rs_wave_free(f);
    rs_free(ctx, f->diagpos);
    rs_free(ctx, f->lu);
    rs_free(ctx, f->dinv);
    rs_free(ctx, f->state);
    rs_free(ctx, f->ywork);
    rs_free(ctx, f->zwork);
    delete f;
}

static int sweep_grid(rs_ctx *ctx, int npad)
{
    const int need = (npad + RS_SWEEP_THREADS - 1) / RS_SWEEP_THREADS;
    return std::max(1, std::min(need, ctx->sweep_blocks));
}

// After the numeric factorisation: the sweeps' copies of the factors (L
// entries; U entries premultiplied by D_i), the diagonal inverses by row and
// the scan multipliers of both triangles, in the apply precision T.
template <int BS, typename T>
static int gather_sweep_data(IluFactor *f, int *bad_row)
{
    rs_ctx *ctx = f->ctx;
    const int b2 = BS * BS;
    const int gl = (int)std::min<int64_t>(std::max<int64_t>((f->SL.nent + 255) / 256, 1), 4096);
    const int np = f->SU.nseg * 32;
    const int gr = std::max(1, std::min((np + 255) / 256, 4096));
    const int gsl = std::max(1, std::min((f->SL.nseg + 7) / 8, 4096));
    const int gsu = std::max(1, std::min((f->SU.nseg + 7) / 8, 4096));
    k_gather_tri<T><<<gl, 256, 0, ctx->stream>>>(f->SL.nent, b2, f->SL.src, f->lu, (T *)f->SL.val);
    k_gather_useg<BS, T><<<gsu, 256, 0, ctx->stream>>>(f->SU.nseg, f->SU.nent, f->SU.sptr, f->SU.row0, f->SU.src,
                                                         f->diagpos, f->lu, f->dinv, (T *)f->SU.val);
    k_gather_dinv<T><<<gr, 256, 0, ctx->stream>>>(f->nrows, np, b2, f->diagpos, f->lu, f->dinv, (T *)f->SU.rdiag);
    k_scan_mul<BS, T, true><<<gsl, 256, 0, ctx->stream>>>(f->SL.nseg, f->SL.row0, f->SL.adjsrc, f->diagpos, f->lu,
                                                            f->dinv, (T *)f->SL.mul);
    k_scan_mul<BS, T, false><<<gsu, 256, 0, ctx->stream>>>(f->SU.nseg, f->SU.row0, f->SU.adjsrc, f->diagpos, f->lu,
                                                             f->dinv, (T *)f->SU.mul);
    RS_TRY(rs_check_launch(ctx));
    ctx->launches += 5;
    return rs_collect_device_error(ctx, bad_row);
}

int rs_ilu_factor(IluFactor *f, const double *d_val, int *bad_row)
{
    rs_ctx *ctx = f->ctx;
    const size_t b2 = (size_t)f->bs * f->bs;
    if (bad_row) *bad_row = -1;
    if (f->nrows == 0) return RS_OK;
    RS_CUDA_TRY(cudaMemcpyAsync(f->lu, d_val, sizeof(double) * b2 * f->nnzb, cudaMemcpyDeviceToDevice,
                                ctx->stream));
    const int g = sweep_grid(ctx, f->L.npad);
    const SweepArgs a = sweep_args(ctx, f->L, f->state, nullptr);
    RsProfScope prof(ctx, RS_PROF_FACTOR);
    switch (f->bs) {
    case 1:
        k_ilu0_factor<<<g, RS_SWEEP_THREADS, 0, ctx->stream>>>(a, f->ptr, f->col, f->diagpos, f->lu,
                                                              ctx->d_bad_row);
        break;
#define RS_BF(BB)                                                                          \
    case BB:                                                                               \
        k_bilu0_factor<BB><<<g, RS_SWEEP_THREADS, 0, ctx->stream>>>(a, f->ptr, f->col,     \
                                                                    f->diagpos, f->lu,    \
                                                                    f->dinv, ctx->d_bad_row); \
        break;
        RS_BF(2)
        RS_BF(3)
        RS_BF(4)
#undef RS_BF
    default: return RS_ERR_INVALID_ARG;
    }
    RS_TRY(rs_check_launch(ctx));
    if (f->W.on) {
        RS_TRY(rs_wave_gather(f));
        return rs_collect_device_error(ctx, bad_row);
    }
    switch (f->bs) {
    case 1: return f->fp32 ? gather_sweep_data<1, float>(f, bad_row) : gather_sweep_data<1, double>(f, bad_row);
    case 2: return f->fp32 ? gather_sweep_data<2, float>(f, bad_row) : gather_sweep_data<2, double>(f, bad_row);
    case 3: return f->fp32 ? gather_sweep_data<3, float>(f, bad_row) : gather_sweep_data<3, double>(f, bad_row);
    default: return f->fp32 ? gather_sweep_data<4, float>(f, bad_row) : gather_sweep_data<4, double>(f, bad_row);
    }
}

// A factor computed elsewhere (ILUT on the host), FP64 in the pattern of f:
// strict lower part of L, then U with its diagonal (scalar only).  Builds
// the sweeps' data from it, as after a factorisation.
int rs_ilu_set_factors(IluFactor *f, const double *d_lu, int *bad_row)
{
    if (f->bs != 1) return RS_ERR_INVALID_ARG;
    if (bad_row) *bad_row = -1;
    if (f->nrows == 0) return RS_OK;
    RS_CUDA_TRY(cudaMemcpyAsync(f->lu, d_lu, sizeof(double) * f->nnzb, cudaMemcpyDeviceToDevice, f->ctx->stream));
    if (f->W.on) {
        RS_TRY(rs_wave_gather(f));
        return rs_collect_device_error(f->ctx, bad_row);
    }
    return f->fp32 ? gather_sweep_data<1, float>(f, bad_row) : gather_sweep_data<1, double>(f, bad_row);
}

// Dynamic shared memory of a sweep block: one scan stage per warp.  Above the
// default 48 KB the kernel's limit is raised once per device.
template <int BS, typename T, bool RUNS, bool LOWER, class K>
static int sweep_smem(rs_ctx *ctx, K kernel, int wpb, size_t *bytes)
{
    static unsigned long long raised = 0;   // one per kernel instantiation
    const size_t per_warp = ScanStage<BS, T>::N * sizeof(T) + (RUNS ? RS_RUN_RING * sizeof(unsigned long long) : 0);
    *bytes = (size_t)wpb * per_warp;
    const size_t most = (size_t)(RS_SWEEP_THREADS / 32) * per_warp;
    if (most <= 48 * 1024) return RS_OK;
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(raised & bit)) {
        RS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
        raised |= bit;
    }
    return RS_OK;
}

template <int BS, typename T>
static int apply_seg(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    rs_ctx *ctx = f->ctx;
    T *y = (T *)f->ywork, *zt = (T *)f->zwork;
    // layouts with runs (scalar factors only) take the kernels that carry
    // the run code and the ring, in blocks of run_warps warps, one run per
    // warp; the others keep the leaner kernels, whose register count lets
    // more sweep blocks share an SM
    const bool rl = BS == 1 && f->SL.max_run > 1, ru = BS == 1 && f->SU.max_run > 1;
    const int wl = rl ? f->run_warps : RS_SWEEP_THREADS / 32, wu = ru ? f->run_warps : RS_SWEEP_THREADS / 32;
    const int gl = std::max(1, rl ? (f->SL.nrun + wl - 1) / wl : std::min((f->SL.nrun + wl - 1) / wl, f->SL.grid));
    const int gu = std::max(1, ru ? (f->SU.nrun + wu - 1) / wu : std::min((f->SU.nrun + wu - 1) / wu, f->SU.grid));
    size_t sl = 0, su = 0;
    {
        const int e1 = rl ? sweep_smem<BS, T, true, true>(ctx, k_lsolve_seg<BS, T, BS == 1>, wl, &sl)
                          : sweep_smem<BS, T, false, true>(ctx, k_lsolve_seg<BS, T, false>, wl, &sl);
        const int e2 = e1 ? e1
                          : ru ? sweep_smem<BS, T, true, false>(ctx, k_usolve_seg<BS, T, BS == 1>, wu, &su)
                               : sweep_smem<BS, T, false, false>(ctx, k_usolve_seg<BS, T, false>, wu, &su);
        if (e2) return e2;
    }
    {
        RsProfScope prof(ctx, BS == 1 ? RS_PROF_LSWEEP : RS_PROF_BLSWEEP);
        const SegArgs a = seg_args(ctx, f->SL, f->nrows, f->state, skip);
        if (rl)
            k_lsolve_seg<BS, T, BS == 1><<<gl, 32 * wl, sl, ctx->stream>>>(
                a, (const T *)f->SL.val, (const T *)f->SL.mul, r, scale, y, zt);
        else
            k_lsolve_seg<BS, T, false><<<gl, 32 * wl, sl, ctx->stream>>>(
                a, (const T *)f->SL.val, (const T *)f->SL.mul, r, scale, y, zt);
    }
    RS_TRY(rs_check_launch(ctx));
    RsProfScope prof(ctx, BS == 1 ? RS_PROF_USWEEP : RS_PROF_BUSWEEP);
    const SegArgs a = seg_args(ctx, f->SU, f->nrows, f->state, skip);
    if (ru)
        k_usolve_seg<BS, T, BS == 1><<<gu, 32 * wu, su, ctx->stream>>>(
            a, (const T *)f->SU.val, (const T *)f->SU.mul, (const T *)f->SU.rdiag, y, zt, z);
    else
        k_usolve_seg<BS, T, false><<<gu, 32 * wu, su, ctx->stream>>>(
            a, (const T *)f->SU.val, (const T *)f->SU.mul, (const T *)f->SU.rdiag, y, zt, z);
    return rs_check_launch(ctx);
}

int rs_ilu_apply(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    if (f->nrows == 0) return RS_OK;
    if (f->W.on) return rs_wave_apply(f, r, z, scale, skip);
    switch (f->bs) {
    case 1: return f->fp32 ? apply_seg<1, float>(f, r, z, scale, skip) : apply_seg<1, double>(f, r, z, scale, skip);
    case 2: return f->fp32 ? apply_seg<2, float>(f, r, z, scale, skip) : apply_seg<2, double>(f, r, z, scale, skip);
    case 3: return f->fp32 ? apply_seg<3, float>(f, r, z, scale, skip) : apply_seg<3, double>(f, r, z, scale, skip);
    case 4: return f->fp32 ? apply_seg<4, float>(f, r, z, scale, skip) : apply_seg<4, double>(f, r, z, scale, skip);
    default: return RS_ERR_INVALID_ARG;
    }
}
