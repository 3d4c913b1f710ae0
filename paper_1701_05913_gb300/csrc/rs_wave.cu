// Wavefront triangular sweeps of ILU(0) and block ILU(0) on structured grids.
//
// The solves L y = r and U z = y of Eq. 3 (Sec. 4.1), which the paper notes
// run row by row, on a matrix whose pattern is (a subset of) the 7-point
// stencil of an nx x ny x nz grid in natural order: row (x, y, z) of L reads
// only (x-1, y, z), (x, y-1, z) and (x, y, z-1), and U the mirror images.
// ILU(0) keeps that pattern, so the dependency graph of either sweep is the
// grid itself and its critical path is nx + ny + nz - 2 cells long.
//
// Schedule.  One warp takes a unit: 32 consecutive y-lines of one z-plane
// (the last unit of a plane may hold fewer).  At step t lane j solves cell
// (x = t - j, y = 32 yb + j): its x-neighbour is the lane's own value of the
// previous step, its y-neighbour the previous step's value of lane j - 1 (a
// shuffle), so a unit takes nx + 31 steps of a few dependent operations.
// The y-neighbour of lane 0 and every z-neighbour come from other units
// through L2: the value is its own ready flag (a sentinel NaN until
// written), loaded several steps ahead and checked when it is used.  Units
// are taken in order from a ticket counter (the U sweep in reverse), so a
// warp only waits for units held by warps that took earlier tickets and are
// running: the schedule cannot deadlock, and every wait is bounded in time.
//
// Layout.  Factor values, the right-hand side and the sweeps' values are
// stored in wave order: inside a unit, cell (t, j) follows all cells of the
// steps before t.  A step's cells are then contiguous, and so is a whole
// unit: a warp streams its unit's records and right-hand side through a ring
// of shared-memory slots with bulk copies (mbarrier-counted), and its z-
// neighbours sit at the same offset in the previous plane's unit.  Units are
// padded to whole chunks of the ring.  Two permutation kernels move r from
// natural into wave order (scaled, rounded to the apply precision) and the
// result back.
//
// Arithmetic.  L: y_i = r_i - L_iz y_z - L_iy y_y - L_ix y_x, in ascending
// column order (FP32: each product and difference rounded, as the
// sequential FP32 solve does; FP64: fused multiply-adds).  U is stored
// premultiplied by D_i = inv(U_ii), z_i = D_i y_i - sum_j (D_i U_ij) z_j,
// with the z-term (loaded ahead) first.  Blocks (bs x bs) take the same
// steps with block products.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

#define RS_WAVE_MAX_NX 4096
#define RS_WAVE_OFF_PAD 33   // entries per off table beyond nx (steps up to nx + 32)
#define RS_WAVE_DRAIN (1LL << 30)   // clock cycles a late bulk copy is still waited for

namespace {

constexpr int pow2_floor(int v) { return v >= 2 ? 2 * pow2_floor(v / 2) : 1; }

// Records, ring and hand-off depth per block size and apply precision.
template <int BS, typename T>
struct WaveCfg {
    static constexpr int B2 = BS * BS;
    static constexpr int VQ = 16 / (int)sizeof(T);                 // T per 16 bytes
    static constexpr int RL = (3 * B2 + VQ - 1) / VQ * VQ;           // L record: L_z, L_y, L_x
    static constexpr int RU = (4 * B2 + VQ - 1) / VQ * VQ;           // U record: U'_z, U'_x, U'_y, D
    // cells per chunk: a power of two, about 10 KB per U slot
    static constexpr int CC0 = pow2_floor(10240 / ((RU + BS) * (int)sizeof(T)));
    static constexpr int CC = CC0 < 16 ? 16 : CC0;
    static constexpr int R = 4;                                      // ring slots per warp
    // hand-off values loaded this many steps ahead (a step of a scalar FP64
    // sweep takes about 200 cycles of FP64 pipe, an FP32 one far less)
    static constexpr int HP = sizeof(T) == 8 ? (BS == 1 ? 8 : 2) : (BS == 1 ? 24 : 8);
    // warps per block: FP64 sweeps keep the SM's scarce FP64 pipes for few warps
    static constexpr int WPB = sizeof(T) == 8 ? 2 : 4;
    static constexpr int BAR_BYTES = 128;                            // WPB * R mbarriers, padded
    template <bool LOWER>
    static constexpr int slot_bytes() { return CC * ((LOWER ? RL : RU) + BS) * (int)sizeof(T); }
    template <bool LOWER>
    static constexpr int smem_bytes() { return BAR_BYTES + WPB * R * slot_bytes<LOWER>(); }
};

struct WaveArgs {
    int nx, ny, nz, nyb, nunits, lastL;
    int sfull;               // padded cells of a unit of 32 lines
    int64_t plane;           // padded cells of a plane
    const int *off;          // [2][nx + RS_WAVE_OFF_PAD]: first cell of each step (32 lines, last unit)
    SweepState *st;
    int *err;
    long long limit;
    const int *skip;
};

WaveArgs wave_args(rs_ctx *ctx, const WaveLayout &W, SweepState *st, const int *skip)
{
    WaveArgs g;
    g.nx = W.nx;
    g.ny = W.ny;
    g.nz = W.nz;
    g.nyb = W.nyb;
    g.nunits = W.nunits;
    g.lastL = W.lastL;
    g.sfull = W.sfull;
    g.plane = W.plane;
    g.off = W.off;
    g.st = st;
    g.err = ctx->d_err;
    g.limit = ctx->spin_limit;
    g.skip = skip;
    return g;
}

struct Unit {
    int z, yb, L, nsteps;
    int64_t base;            // first (padded) cell of the unit in wave order
    const int *tab;          // its off table
};

__device__ __forceinline__ Unit unit_of(const WaveArgs &g, int u)
{
    Unit U;
    U.z = u / g.nyb;
    U.yb = u - U.z * g.nyb;
    const bool last = U.yb == g.nyb - 1;
    U.L = last ? g.lastL : 32;
    U.nsteps = g.nx + U.L - 1;
    U.base = (int64_t)U.z * g.plane + (int64_t)U.yb * g.sfull;
    U.tab = g.off + (last ? g.nx + RS_WAVE_OFF_PAD : 0);
    return U;
}

// cell of lane j at step t inside a unit with off table tab
__device__ __forceinline__ int wave_cell(const int *tab, int nx, int t, int j)
{
    return __ldg(tab + t) + j - max(0, t - nx + 1);
}

// wave-order position of natural (block) row i
__device__ __forceinline__ int64_t wave_pos(const WaveArgs &g, int i)
{
    const int x = i % g.nx, rest = i / g.nx;
    const int y = rest % g.ny, z = rest / g.ny;
    const int yb = y >> 5, j = y & 31;
    const int *tab = g.off + (yb == g.nyb - 1 ? g.nx + RS_WAVE_OFF_PAD : 0);
    return (int64_t)z * g.plane + (int64_t)yb * g.sfull + wave_cell(tab, g.nx, x + j, j);
}

// RB values from 16-byte aligned shared memory, in 16-byte loads
template <int RB>
__device__ __forceinline__ void lds_rec(const float *p, float (&v)[RB])
{
    static_assert(RB % 4 == 0, "records are whole 16-byte words");
    const float4 *q = (const float4 *)p;
#pragma unroll
    for (int k = 0; k < RB / 4; ++k) {
        const float4 w = q[k];
        v[4 * k] = w.x;
        v[4 * k + 1] = w.y;
        v[4 * k + 2] = w.z;
        v[4 * k + 3] = w.w;
    }
}
template <int RB>
__device__ __forceinline__ void lds_rec(const double *p, double (&v)[RB])
{
    static_assert(RB % 2 == 0, "records are whole 16-byte words");
    const double2 *q = (const double2 *)p;
#pragma unroll
    for (int k = 0; k < RB / 2; ++k) {
        const double2 w = q[k];
        v[2 * k] = w.x;
        v[2 * k + 1] = w.y;
    }
}

__device__ __forceinline__ void wave_end(const WaveArgs &g)
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
// the sweep: L (LOWER) or U
// ---------------------------------------------------------------------------
// rec: the unit's records; rhs: r in wave order (L) or y (U); xv: the values
// this sweep produces, polled by the neighbouring units (sentinel before).
template <int BS, typename T, bool LOWER>
__global__ void __launch_bounds__(32 * WaveCfg<BS, T>::WPB)
k_wave_sweep(WaveArgs g, const T *__restrict__ rec, const T *__restrict__ rhs, T *xv)
{
    using C = WaveCfg<BS, T>;
    constexpr int B2 = C::B2;
    constexpr int RB = LOWER ? C::RL : C::RU;
    constexpr int SLOT = C::template slot_bytes<LOWER>();
    constexpr int HP = C::HP;
    constexpr unsigned FULL = 0xffffffffu;
    typedef typename Sentinel<T>::bits_t bits_t;
    constexpr bits_t SENT = Sentinel<T>::bits;
    extern __shared__ __align__(128) unsigned char wave_smem[];
    if (g.skip && *(volatile const int *)g.skip) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *bars = (unsigned long long *)wave_smem + wid * C::R;
    unsigned char *slots = wave_smem + C::BAR_BYTES + (size_t)wid * C::R * SLOT;
    if (lane == 0) {
        for (int s = 0; s < C::R; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    unsigned parity = 0;     // bit s: parity of slot s's next completion
    bool dead = false;       // a hand-off poll gave up: later polls give up at once
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = (int)atomicAdd(&g.st->ticket, 1u);
        tk = __shfl_sync(FULL, tk, 0);
        if (tk >= g.nunits) break;
        const Unit U = unit_of(g, LOWER ? tk : g.nunits - 1 - tk);
        const int nch = (U.L * g.nx + C::CC - 1) / C::CC;
        const T *grec = rec + U.base * RB;
        const T *grhs = rhs + U.base * BS;
        // neighbours in other units: z (every lane), y (lane 0 of L, lane 31 of U)
        const bool has_z = LOWER ? U.z > 0 : U.z < g.nz - 1;
        const int64_t zbase = U.base + (LOWER ? -g.plane : g.plane);
        const bool has_y = LOWER ? U.yb > 0 : U.yb < g.nyb - 1;
        const int ylane = LOWER ? 0 : 31;
        const int *ytab = LOWER ? g.off : g.off + (U.yb + 1 == g.nyb - 1 ? g.nx + RS_WAVE_OFF_PAD : 0);
        const int64_t ybase = U.base + (LOWER ? -(int64_t)g.sfull : (int64_t)g.sfull);

        // chunk q of the stream (the U sweep streams its unit backwards)
        int issued = 0, waited = 0;
        auto issue_to = [&](int upto) {
            upto = min(upto, nch);
            if (issued >= upto) return;
            __syncwarp();
            if (lane == 0) {
                // the slots' earlier contents were read through the generic proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                for (int q = issued; q < upto; ++q) {
                    const int k = LOWER ? q : nch - 1 - q;
                    const int s = q % C::R;
                    unsigned char *dst = slots + (size_t)s * SLOT;
                    mbar_arrive_expect_tx(&bars[s], SLOT);
                    bulk_g2s(dst, grec + (int64_t)k * C::CC * RB, C::CC * RB * (int)sizeof(T), &bars[s]);
                    bulk_g2s(dst + C::CC * RB * sizeof(T), grhs + (int64_t)k * C::CC * BS,
                             C::CC * BS * (int)sizeof(T), &bars[s]);
                }
            }
            issued = upto;
        };
        // A chunk wait longer than the spin limit records the timeout, then
        // still waits (up to RS_WAVE_DRAIN cycles) for the copy itself, so
        // that no copy lands in a slot after it has been reused.
        auto wait_to = [&](int upto) {
            while (waited < upto) {
                const int s = waited % C::R;
                const unsigned par = (parity >> s) & 1u;
                if (!mbar_try_wait(&bars[s], par)) {
                    const long long t0 = clock64();
                    bool late = false;
                    while (!mbar_try_wait(&bars[s], par)) {
                        const long long dt = clock64() - t0;
                        if (!late && dt > g.limit) {
                            late = true;
                            if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                        }
                        if (dt > RS_WAVE_DRAIN) break;
                    }
                }
                parity ^= 1u << s;
                ++waited;
            }
        };
        // the hand-off values of step s (raw bits; 0.0 where none is read)
        auto fetch = [&](int s, bits_t (&oz)[BS], bits_t (&oy)[BS]) {
#pragma unroll
            for (int k = 0; k < BS; ++k) oz[k] = oy[k] = 0;
            if (s >= U.nsteps) return;
            const int t = LOWER ? s : U.nsteps - 1 - s;
            const int x = t - lane;
            if (lane >= U.L || x < 0 || x >= g.nx) return;
            if (has_z) {
                const T *p = xv + (zbase + wave_cell(U.tab, g.nx, t, lane)) * BS;
#pragma unroll
                for (int k = 0; k < BS; ++k) oz[k] = ld_relaxed_bits(p + k);
            }
            if (has_y && lane == ylane) {
                // L: (x, y-1) is lane 31 of the unit before, at step t + 31;
                // U: (x, y+1) is lane 0 of the unit after, at step t - 31
                const int cy = LOWER ? wave_cell(ytab, g.nx, t + 31, 31) : wave_cell(ytab, g.nx, t - 31, 0);
                const T *p = xv + (ybase + cy) * BS;
#pragma unroll
                for (int k = 0; k < BS; ++k) oy[k] = ld_relaxed_bits(p + k);
            }
        };

        issue_to(C::R);
        bits_t hz[HP][BS], hy[HP][BS];
#pragma unroll
        for (int k = 0; k < HP; ++k) fetch(k, hz[k], hy[k]);
        T vprev[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) vprev[k] = T(0);

        for (int s0 = 0; s0 < U.nsteps; s0 += HP) {
#pragma unroll
            for (int kk = 0; kk < HP; ++kk) {
                const int s = s0 + kk;
                if (s < U.nsteps) {
                const int t = LOWER ? s : U.nsteps - 1 - s;
                const int x = t - lane;
                const bool act = lane < U.L && x >= 0 && x < g.nx;
                const int tlo = __ldg(U.tab + t), thi = __ldg(U.tab + t + 1);
                const int c = tlo + lane - max(0, t - g.nx + 1);
                // refill the slots of chunks already consumed, wait for the ones this step reads
                if (LOWER) {
                    issue_to(tlo / C::CC + C::R);
                    wait_to((thi - 1) / C::CC + 1);
                } else {
                    issue_to(nch - (thi + C::CC - 1) / C::CC + C::R);
                    wait_to(nch - tlo / C::CC);
                }
                T rv[RB], bv[BS];
                if (act) {
                    const int k = c / C::CC, o = c - k * C::CC;
                    const int q = LOWER ? k : nch - 1 - k;
                    const unsigned char *sp = slots + (size_t)(q % C::R) * SLOT;
                    lds_rec<RB>((const T *)sp + o * RB, rv);
                    const T *rp = (const T *)(sp + C::CC * RB * sizeof(T)) + o * BS;
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) bv[k2] = rp[k2];
                } else {
#pragma unroll
                    for (int k2 = 0; k2 < RB; ++k2) rv[k2] = T(0);
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) bv[k2] = T(0);
                }
                // hand-off values: loaded HP steps ago; reload while any is a sentinel
                const bool need_z = act && has_z, need_y = act && has_y && lane == ylane;
                bool pend = false;
#pragma unroll
                for (int k2 = 0; k2 < BS; ++k2)
                    pend |= (need_z && hz[kk][k2] == SENT) || (need_y && hy[kk][k2] == SENT);
                if (__any_sync(FULL, pend)) {
                    const long long t0 = clock64();
                    for (;;) {
                        if (pend) {
                            bits_t oz[BS], oy[BS];
                            fetch(s, oz, oy);
#pragma unroll
                            for (int k2 = 0; k2 < BS; ++k2) {
                                if (need_z) hz[kk][k2] = oz[k2];
                                if (need_y) hy[kk][k2] = oy[k2];
                            }
                            pend = false;
#pragma unroll
                            for (int k2 = 0; k2 < BS; ++k2)
                                pend |= (need_z && hz[kk][k2] == SENT) || (need_y && hy[kk][k2] == SENT);
                        }
                        if (!__any_sync(FULL, pend)) break;
                        if (dead || clock64() - t0 > g.limit) {
                            // give up: carry NaN on (arithmetic on the sentinel quiets it)
                            if (pend) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                            dead = true;
                            break;
                        }
                    }
                }
                T vz[BS], vy[BS];
#pragma unroll
                for (int k2 = 0; k2 < BS; ++k2) {
                    vz[k2] = need_z ? bits_to(T(), hz[kk][k2]) : T(0);
                    const T sh = LOWER ? __shfl_up_sync(FULL, vprev[k2], 1) : __shfl_down_sync(FULL, vprev[k2], 1);
                    vy[k2] = lane == ylane ? (need_y ? bits_to(T(), hy[kk][k2]) : T(0)) : sh;
                }
                // load step s + HP's hand-off values into the slot just used
                fetch(s + HP, hz[kk], hy[kk]);
                T acc[BS];
                if (LOWER) {
#pragma unroll
                    for (int i = 0; i < BS; ++i) acc[i] = bv[i];
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[i * BS + j], vz[j]);
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[B2 + i * BS + j], vy[j]);
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[2 * B2 + i * BS + j], vprev[j]);
                } else {
#pragma unroll
                    for (int i = 0; i < BS; ++i) {
                        T sum = T(0);
#pragma unroll
                        for (int j = 0; j < BS; ++j) sum = mad(rv[3 * B2 + i * BS + j], bv[j], sum);
                        acc[i] = sum;
                    }
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[i * BS + j], vz[j]);
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[B2 + i * BS + j], vprev[j]);
#pragma unroll
                    for (int i = 0; i < BS; ++i)
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc[i] = msub(acc[i], rv[2 * B2 + i * BS + j], vy[j]);
                }
#pragma unroll
                for (int i = 0; i < BS; ++i) vprev[i] = act ? acc[i] : T(0);
                if (act) {
                    T *p = xv + (U.base + c) * BS;
#pragma unroll
                    for (int i = 0; i < BS; ++i) st_relaxed(p + i, vprev[i]);
                }
                }   // s < nsteps
            }
        }
    }
    wave_end(g);
}

// r (natural order, FP64) -> wave order in the apply precision, times *scale;
// the U sweep's values back to the sentinel
template <int BS, typename T>
__global__ void k_wave_in(WaveArgs g, const double *__restrict__ r, const double *__restrict__ scale,
                          T *__restrict__ rw, T *__restrict__ zreset)
{
    if (g.skip && *(volatile const int *)g.skip) return;
    const double sc = scale ? *scale : 1.0;
    const int n = g.nx * g.ny * g.nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t w = wave_pos(g, i);
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            const double v = r[(size_t)i * BS + k];
            rw[w * BS + k] = (T)(sc == 1.0 ? v : v * sc);
            zreset[w * BS + k] = bits_to(T(), Sentinel<T>::bits);
        }
    }
}

// the U sweep's values -> natural order, FP64; the L sweep's values back to
// the sentinel
template <int BS, typename T>
__global__ void k_wave_out(WaveArgs g, const T *__restrict__ zw, T *__restrict__ yreset, double *__restrict__ out)
{
    if (g.skip && *(volatile const int *)g.skip) return;
    const int n = g.nx * g.ny * g.nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t w = wave_pos(g, i);
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            out[(size_t)i * BS + k] = (double)zw[w * BS + k];
            yreset[w * BS + k] = bits_to(T(), Sentinel<T>::bits);
        }
    }
}

// Records in wave order from the FP64 factor in the matrix pattern: L_z,
// L_y, L_x of each row; D_i U_ij for the z, x and y neighbours and D_i =
// inv(U_ii) (products in FP64, rounded once to T).  Absent entries are 0.
template <int BS, typename T>
__global__ void k_wave_gather(WaveArgs g, const int *__restrict__ ptr, const int *__restrict__ col,
                              const int *__restrict__ diagpos, const double *__restrict__ lu,
                              const double *__restrict__ dinv, T *__restrict__ lrec, T *__restrict__ urec)
{
    using C = WaveCfg<BS, T>;
    constexpr int B2 = BS * BS;
    const int n = g.nx * g.ny * g.nz;
    const int nxy = g.nx * g.ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t w = wave_pos(g, i);
        double D[B2];
        if (BS == 1) {
            D[0] = 1.0 / lu[diagpos[i]];
        } else {
#pragma unroll
            for (int e = 0; e < B2; ++e) D[e] = dinv[(size_t)i * B2 + e];
        }
        T *lr = lrec + w * C::RL, *ur = urec + w * C::RU;
        for (int e = 0; e < C::RL; ++e) lr[e] = T(0);
        for (int e = 0; e < C::RU; ++e) ur[e] = T(0);
#pragma unroll
        for (int e = 0; e < B2; ++e) ur[3 * B2 + e] = (T)D[e];
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int d = col[p] - i;
            const double *a = lu + (size_t)p * B2;
            int lslot = -1, uslot = -1;
            if (d == -nxy) lslot = 0;
            else if (d == -g.nx) lslot = 1;
            else if (d == -1) lslot = 2;
            else if (d == nxy) uslot = 0;
            else if (d == 1) uslot = 1;
            else if (d == g.nx) uslot = 2;
            if (lslot >= 0) {
#pragma unroll
                for (int e = 0; e < B2; ++e) lr[lslot * B2 + e] = (T)a[e];
            } else if (uslot >= 0) {
#pragma unroll
                for (int r2 = 0; r2 < BS; ++r2)
#pragma unroll
                    for (int c2 = 0; c2 < BS; ++c2) {
                        double s = 0.0;
#pragma unroll
                        for (int m = 0; m < BS; ++m) s = __dadd_rn(s, __dmul_rn(D[r2 * BS + m], a[m * BS + c2]));
                        ur[uslot * B2 + r2 * BS + c2] = (T)s;
                    }
            }
        }
    }
}

// The sweep's dynamic shared memory above the default 48 KB, raised once per
// device for each instantiation (L and U are separate kernels).
template <int BS, typename T, bool LOWER>
int raise_sweep_smem(rs_ctx *ctx)
{
    constexpr int bytes = WaveCfg<BS, T>::template smem_bytes<LOWER>();
    if (bytes <= 48 * 1024) return RS_OK;
    static unsigned long long raised = 0;    // one bit per device
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(raised & bit)) {
        RS_CUDA_TRY(cudaFuncSetAttribute(k_wave_sweep<BS, T, LOWER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes));
        raised |= bit;
    }
    return RS_OK;
}

template <int BS, typename T>
int wave_apply_t(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    using C = WaveCfg<BS, T>;
    rs_ctx *ctx = f->ctx;
    const WaveLayout &W = f->W;
    const WaveArgs g = wave_args(ctx, W, f->state, skip);
    const int n = f->nrows;
    const int gp = std::max(1, std::min((n + 255) / 256, 8 * ctx->num_sms));
    const int gw = std::max(1, std::min((W.nunits + C::WPB - 1) / C::WPB, ctx->num_sms));
    constexpr int sl = C::template smem_bytes<true>(), su = C::template smem_bytes<false>();
    RS_TRY((raise_sweep_smem<BS, T, true>(ctx)));
    RS_TRY((raise_sweep_smem<BS, T, false>(ctx)));
    {
        RsProfScope prof(ctx, BS == 1 ? RS_PROF_LSWEEP : RS_PROF_BLSWEEP);
        k_wave_in<BS, T><<<gp, 256, 0, ctx->stream>>>(g, r, scale, (T *)W.rw, (T *)W.zw);
        k_wave_sweep<BS, T, true><<<gw, 32 * C::WPB, sl, ctx->stream>>>(g, (const T *)W.lrec, (const T *)W.rw,
                                                                       (T *)W.yw);
    }
    RS_TRY(rs_check_launch(ctx));
    {
        RsProfScope prof(ctx, BS == 1 ? RS_PROF_USWEEP : RS_PROF_BUSWEEP);
        k_wave_sweep<BS, T, false><<<gw, 32 * C::WPB, su, ctx->stream>>>(g, (const T *)W.urec, (const T *)W.yw,
                                                                        (T *)W.zw);
        k_wave_out<BS, T><<<gp, 256, 0, ctx->stream>>>(g, (const T *)W.zw, (T *)W.yw, z);
    }
    ctx->launches += 2;   // rs_check_launch counts one per call
    RS_TRY(rs_check_launch(ctx));
    return RS_OK;
}

template <int BS, typename T>
int wave_gather_t(IluFactor *f)
{
    rs_ctx *ctx = f->ctx;
    const WaveArgs g = wave_args(ctx, f->W, f->state, nullptr);
    const int gp = std::max(1, std::min((f->nrows + 127) / 128, 8 * ctx->num_sms));
    k_wave_gather<BS, T><<<gp, 128, 0, ctx->stream>>>(g, f->ptr, f->col, f->diagpos, f->lu, f->dinv,
                                                       (T *)f->W.lrec, (T *)f->W.urec);
    return rs_check_launch(ctx);
}

int cells_per_chunk(int bs, int fp32)
{
    switch (bs) {
    case 1: return fp32 ? WaveCfg<1, float>::CC : WaveCfg<1, double>::CC;
    case 2: return fp32 ? WaveCfg<2, float>::CC : WaveCfg<2, double>::CC;
    case 3: return fp32 ? WaveCfg<3, float>::CC : WaveCfg<3, double>::CC;
    default: return fp32 ? WaveCfg<4, float>::CC : WaveCfg<4, double>::CC;
    }
}

int record_len(int bs, int fp32, bool lower)
{
    switch (bs) {
    case 1: return fp32 ? (lower ? WaveCfg<1, float>::RL : WaveCfg<1, float>::RU)
                        : (lower ? WaveCfg<1, double>::RL : WaveCfg<1, double>::RU);
    case 2: return fp32 ? (lower ? WaveCfg<2, float>::RL : WaveCfg<2, float>::RU)
                        : (lower ? WaveCfg<2, double>::RL : WaveCfg<2, double>::RU);
    case 3: return fp32 ? (lower ? WaveCfg<3, float>::RL : WaveCfg<3, float>::RU)
                        : (lower ? WaveCfg<3, double>::RL : WaveCfg<3, double>::RU);
    default: return fp32 ? (lower ? WaveCfg<4, float>::RL : WaveCfg<4, float>::RU)
                         : (lower ? WaveCfg<4, double>::RL : WaveCfg<4, double>::RU);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// The grid of a pattern whose every off-diagonal entry is a 7-point neighbour
// on an nx x ny x nz grid in natural order (x fastest): the distinct offsets
// |j - i| are a subset of {1, nx, nx ny}.  One-dimensional chains (ny nz = 1)
// and rows longer than RS_WAVE_MAX_NX are left to the segment sweeps.
bool rs_wave_detect(int n, const std::vector<int> &ptr, const std::vector<int> &col, int *gx, int *gy, int *gz)
{
    if (n < 2) return false;
    std::vector<int> offs;
    for (int i = 0; i < n; ++i)
        for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
            const int d = std::abs(col[q] - i);
            if (d == 0 || std::find(offs.begin(), offs.end(), d) != offs.end()) continue;
            offs.push_back(d);
            if (offs.size() > 3) return false;
        }
    if (offs.empty()) return false;
    std::sort(offs.begin(), offs.end());
    int nx, nxy;
    if (offs[0] == 1) {
        nx = offs.size() >= 2 ? offs[1] : n;
        nxy = offs.size() == 3 ? offs[2] : n;
    } else {
        if (offs.size() == 3) return false;
        nx = offs[0];
        nxy = offs.size() == 2 ? offs[1] : n;
    }
    if (nx < 2 || nxy % nx != 0 || n % nxy != 0) return false;
    const int ny = nxy / nx, nz = n / nxy;
    if (nx > RS_WAVE_MAX_NX || (int64_t)ny * nz < 2) return false;
    for (int i = 0; i < n; ++i) {
        const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
        for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
            const int d = col[q] - i;
            const bool ok = d == 0 || (d == -1 && x > 0) || (d == 1 && x < nx - 1) || (d == -nx && y > 0) ||
                            (d == nx && y < ny - 1) || (d == -nxy && z > 0) || (d == nxy && z < nz - 1);
            if (!ok) return false;
        }
    }
    *gx = nx;
    *gy = ny;
    *gz = nz;
    return true;
}

int rs_wave_create(IluFactor *f, int nx, int ny, int nz)
{
    rs_ctx *ctx = f->ctx;
    WaveLayout &W = f->W;
    const int bs = f->bs;
    const size_t esz = f->fp32 ? sizeof(float) : sizeof(double);
    W.nx = nx;
    W.ny = ny;
    W.nz = nz;
    W.nyb = (ny + 31) / 32;
    W.lastL = ny - 32 * (W.nyb - 1);
    W.nunits = nz * W.nyb;
    W.cc = cells_per_chunk(bs, f->fp32);
    W.sfull = (32 * nx + W.cc - 1) / W.cc * W.cc;
    const int slast = (W.lastL * nx + W.cc - 1) / W.cc * W.cc;
    W.plane = (int64_t)(W.nyb - 1) * W.sfull + slast;
    W.ncell = (int64_t)nz * W.plane;
    // first cell of every step, for units of 32 lines and for the last one
    const int stride = nx + RS_WAVE_OFF_PAD;
    std::vector<int> off(2 * (size_t)stride, 0);
    for (int b = 0; b < 2; ++b) {
        const int L = b == 0 ? 32 : W.lastL;
        int *o = off.data() + (size_t)b * stride;
        for (int t = 0; t + 1 < stride; ++t) {
            const int cnt = t < nx + L - 1 ? std::min(t, L - 1) - std::max(0, t - nx + 1) + 1 : 0;
            o[t + 1] = o[t] + cnt;
        }
    }
    const int lr = record_len(bs, f->fp32, true), ur = record_len(bs, f->fp32, false);
    int st = rs_alloc(ctx, (void **)&W.off, sizeof(int) * off.size());
    st = st ? st : rs_alloc(ctx, &W.lrec, esz * lr * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.urec, esz * ur * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.rw, esz * bs * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.yw, esz * bs * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.zw, esz * bs * (size_t)W.ncell);
    if (st) return st;
    RS_CUDA_TRY(cudaMemcpyAsync(W.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, ctx->stream));
    // padding cells are streamed but never used: keep them defined
    RS_CUDA_TRY(cudaMemsetAsync(W.lrec, 0, esz * lr * (size_t)W.ncell, ctx->stream));
    RS_CUDA_TRY(cudaMemsetAsync(W.urec, 0, esz * ur * (size_t)W.ncell, ctx->stream));
    RS_CUDA_TRY(cudaMemsetAsync(W.rw, 0, esz * bs * (size_t)W.ncell, ctx->stream));
    const int64_t nv = (int64_t)bs * W.ncell;
    const int g = (int)std::min<int64_t>((nv + 255) / 256, 4096);
    if (f->fp32) {
        k_fill_sentinel<float><<<g, 256, 0, ctx->stream>>>(nv, (float *)W.yw);
        k_fill_sentinel<float><<<g, 256, 0, ctx->stream>>>(nv, (float *)W.zw);
    } else {
        k_fill_sentinel<double><<<g, 256, 0, ctx->stream>>>(nv, (double *)W.yw);
        k_fill_sentinel<double><<<g, 256, 0, ctx->stream>>>(nv, (double *)W.zw);
    }
    ctx->launches += 1;      // and one more by rs_check_launch
    RS_TRY(rs_check_launch(ctx));
    W.on = 1;
    return RS_OK;
}

void rs_wave_free(IluFactor *f)
{
    rs_ctx *ctx = f->ctx;
    WaveLayout &W = f->W;
    rs_free(ctx, W.off);
    rs_free(ctx, W.lrec);
    rs_free(ctx, W.urec);
    rs_free(ctx, W.rw);
    rs_free(ctx, W.yw);
    rs_free(ctx, W.zw);
    W = WaveLayout();
}

int rs_wave_gather(IluFactor *f)
{
    switch (f->bs) {
    case 1: return f->fp32 ? wave_gather_t<1, float>(f) : wave_gather_t<1, double>(f);
    case 2: return f->fp32 ? wave_gather_t<2, float>(f) : wave_gather_t<2, double>(f);
    case 3: return f->fp32 ? wave_gather_t<3, float>(f) : wave_gather_t<3, double>(f);
    case 4: return f->fp32 ? wave_gather_t<4, float>(f) : wave_gather_t<4, double>(f);
    default: return RS_ERR_INVALID_ARG;
    }
}

int rs_wave_apply(IluFactor *f, const double *r, double *z, const double *scale, const int *skip)
{
    switch (f->bs) {
    case 1: return f->fp32 ? wave_apply_t<1, float>(f, r, z, scale, skip) : wave_apply_t<1, double>(f, r, z, scale, skip);
    case 2: return f->fp32 ? wave_apply_t<2, float>(f, r, z, scale, skip) : wave_apply_t<2, double>(f, r, z, scale, skip);
    case 3: return f->fp32 ? wave_apply_t<3, float>(f, r, z, scale, skip) : wave_apply_t<3, double>(f, r, z, scale, skip);
    case 4: return f->fp32 ? wave_apply_t<4, float>(f, r, z, scale, skip) : wave_apply_t<4, double>(f, r, z, scale, skip);
    default: return RS_ERR_INVALID_ARG;
    }
}
