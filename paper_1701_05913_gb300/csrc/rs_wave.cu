// Wavefront triangular sweeps of ILU(0) and block ILU(0) on structured grids.
//
// The solves L y = r and U z = y of Eq. 3 (Sec. 4.1), which the paper notes
// run row by row, on a matrix whose pattern is (a subset of) the 7-point
// stencil of an nx x ny x nz grid in natural order: row (x, y, z) of L reads
// only (x-1, y, z), (x, y-1, z) and (x, y, z-1), and U the mirror images.
// ILU(0) keeps that pattern, so the dependency graph of either sweep is the
// grid itself and its critical path is nx + ny + nz - 2 cells long.
//
// Schedule.  A block of two warps takes a unit: a tile of a y-lines by b
// z-planes (a b = 32 lanes) over all x.  In the compute warp lane (jy, jz)
// solves cell (x = t - jy - jz, y0 + jy, z0 + jz) at step t: its
// x-neighbour is the lane's own value of the step before, its y- and
// z-neighbours inside the tile the step-before values of lanes (jy-1, jz)
// and (jy, jz-1), one shuffle each.  Only the tile's faces read other units,
// through L2, with the value as its own ready flag (a sentinel NaN until
// written).  The producer warp polls those values, several steps at a time
// and continuously, so that each is seen about one L2 round trip after it is
// written, and hands them to the compute warp through a shared-memory ring
// with a step counter; it also streams the unit's records and right-hand
// side into the compute warp's ring of bulk-copy slots.  The compute warp
// thus runs only the step's arithmetic.  A unit takes nx + a + b - 2 steps;
// the units on the critical path number ceil(ny/a) + ceil(nz/b) - 1, so a
// and b are chosen to minimise it.  Units are taken in order from a ticket
// counter (the U sweep in reverse), so a block only waits for units held by
// blocks that took earlier tickets and are running: the schedule cannot
// deadlock, and every wait is bounded in time.
//
// Layout.  Every unit stores its cells by step, 32 per step (lane order,
// zeros where a lane is idle), so a step's values, records and right-hand
// side are contiguous and every address is the unit's base plus 32 t plus
// the lane.  The records and right-hand side stream through a ring of
// shared-memory slots of G steps each, filled by bulk copies
// (mbarrier-counted).  Two permutation kernels move r from natural into wave
// order (scaled, rounded to the apply precision) and the result back.
//
// Arithmetic.  L: y_i = r_i - L_iz y_z - L_iy y_y - L_ix y_x, in ascending
// column order (FP32: each product and difference rounded, as the
// sequential FP32 solve does; FP64: fused multiply-adds).  U is stored
// premultiplied by D_i = inv(U_ii), z_i = D_i y_i - sum_j (D_i U_ij) z_j.
// Blocks (bs x bs) take the same steps with block products.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

#define RS_WAVE_MAX_NX 4096
#define RS_WAVE_DRAIN (1LL << 30)   // clock cycles a late bulk copy is still waited for

namespace {

// Records, rings and hand-off depth per block size and apply precision.
template <int BS, typename T>
struct WaveCfg {
    static constexpr int B2 = BS * BS;
    static constexpr int VQ = 16 / (int)sizeof(T);                 // T per 16 bytes
    static constexpr int RL = (3 * B2 + VQ - 1) / VQ * VQ;           // L record: L_z, L_y, L_x
    static constexpr int RU = (4 * B2 + VQ - 1) / VQ * VQ;           // U record: U'_z, U'_x, U'_y, D
    // steps per bulk-copy slot: about 10 KB per U slot (20 KB for FP64
    // blocks, so that a slot holds two steps)
    static constexpr int G0 = ((BS > 1 && sizeof(T) == 8) ? 20480 : 10240) / (32 * (RU + BS) * (int)sizeof(T));
    static constexpr int G = G0 >= 16 ? 16 : G0 >= 8 ? 8 : G0 >= 4 ? 4 : G0 >= 2 ? 2 : 1;
    static constexpr int R = 4;                                      // bulk-copy slots (WaveHdr::bar)
    // steps of hand-off values the producer polls at once: enough to keep
    // ahead of the compute warp's pace over one L2 round trip, few enough
    // that the round trip stays short (block records: 4 steps measured
    // faster than 8)
    static constexpr int K = BS == 1 ? (sizeof(T) == 4 ? 16 : 8) : (sizeof(T) == 4 ? 4 : 2);
    // (step, position) pairs of a polling round per producer lane
    static constexpr int JP = 4;
    // hand-off ring (steps), a power of two
    static constexpr int HR = 2 * K < 16 ? 16 : 2 * K;
    static constexpr int HDR_BYTES = 128;                            // R mbarriers, ticket, counters
    static_assert((G & (G - 1)) == 0 && (HR & (HR - 1)) == 0 && HR % G == 0, "rings are powers of two, chunks fit the hand-off ring");
    template <bool LOWER>
    static constexpr int slot_bytes() { return G * 32 * ((LOWER ? RL : RU) + BS) * (int)sizeof(T); }
    static constexpr int ring_bytes() { return HR * 2 * 32 * BS * (int)sizeof(T); }
    // FP64 block records: the components of a step are computed by BS warps,
    // one component each (a warp's FP64 multiply-adds share one FP64 unit, so
    // one warp doing all BS^2 per block is bound by that unit), exchanged
    // through shared memory; one warp otherwise
    static constexpr int NCW = (BS > 1 && sizeof(T) == 8) ? BS : 1;
    static constexpr int THREADS = 32 * (NCW + 1);                   // + the producer warp
    static constexpr int xbuf_bytes() { return NCW > 1 ? 2 * NCW * 32 * (int)sizeof(T) : 0; }
    template <bool LOWER>
    static constexpr int smem_bytes() { return HDR_BYTES + R * slot_bytes<LOWER>() + ring_bytes() + xbuf_bytes(); }
};

// the block's shared header
struct WaveHdr {
    unsigned long long bar[4];    // bulk-copy slots' mbarriers
    int tk;                       // the unit's ticket
    unsigned prod;                // steps whose hand-off values are in the ring
    unsigned cons;                // steps the compute warp has finished with
};

struct WaveArgs {
    int nx, ny, nz, la;
    int nyt, nzt, nunits, npad;
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
    g.la = W.la;
    g.nyt = W.nyt;
    g.nzt = W.nzt;
    g.nunits = W.nunits;
    g.npad = W.npad;
    g.st = st;
    g.err = ctx->d_err;
    g.limit = ctx->spin_limit;
    g.skip = skip;
    return g;
}

// Loads and stores of the hand-off values, relaxed at GPU scope (single-copy
// atomic, seen across SMs), written without a compiler memory clobber so
// that they do not pin the step's other memory operations in place: the
// protocol needs no ordering between different addresses.
__device__ __forceinline__ unsigned long long ld_poll(const double *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned int ld_poll(const float *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_poll(double *p, double v)
{
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void st_poll(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

// wave-order position (cell index) of natural (block) row i
__device__ __forceinline__ int64_t wave_pos(const WaveArgs &g, int i)
{
    const int x = i % g.nx, rest = i / g.nx;
    const int y = rest % g.ny, z = rest / g.ny;
    const int a = 1 << g.la, b = 32 >> g.la;
    const int jy = y & (a - 1), jz = z % b;
    const int u = (z / b) * g.nyt + (y >> g.la);
    return ((int64_t)u * g.npad + x + jy + jz) * 32 + jy + (jz << g.la);
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
// shared-memory counters between the two warps of a block
__device__ __forceinline__ unsigned ld_acq_cta(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)));
    return v;
}
__device__ __forceinline__ void st_rel_cta(unsigned *p, unsigned v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
// The compute warp's progress.  A plain store: the slots it frees were read
// by loads whose values the warp has already used (they fed the step
// before's arithmetic, which fed this step's shuffles), so the loads are
// complete when the store issues, and a release (which would wait for the
// warp's outstanding global stores) is not needed.
__device__ __forceinline__ void st_cons(unsigned *p, unsigned v)
{
    asm volatile("st.volatile.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v));
}
// hand-off values from the ring, after the acquire of the step counter (kept
// in program order with it: both are volatile asm)
__device__ __forceinline__ double lds_ho(const double *p)
{
    double v;
    asm volatile("ld.shared::cta.f64 %0, [%1];" : "=d"(v) : "r"(smem_addr(p)));
    return v;
}
__device__ __forceinline__ float lds_ho(const float *p)
{
    float v;
    asm volatile("ld.shared::cta.f32 %0, [%1];" : "=f"(v) : "r"(smem_addr(p)));
    return v;
}

// rec: the units' records; rhs: r in wave order (L) or y (U); xv: the values
// this sweep produces, polled by the neighbouring units (sentinel before).
// Warp 0 computes, warp 1 produces.  Waits inside the block (for a bulk
// copy, for the ring) record a timeout after the spin limit and give up
// after four limits plus RS_WAVE_DRAIN cycles; a poll of another unit's
// value records it after the limit and carries the sentinel on from then.
template <int BS, typename T, bool LOWER>
__global__ void __launch_bounds__(WaveCfg<BS, T>::THREADS)
k_wave_sweep(WaveArgs g, const T *__restrict__ rec, const T *__restrict__ rhs, T *xv)
{
    using C = WaveCfg<BS, T>;
    constexpr int B2 = C::B2;
    constexpr int RB = LOWER ? C::RL : C::RU;
    constexpr int G = C::G;
    constexpr int R = C::R;
    constexpr int K = C::K;
    constexpr int HR = C::HR;
    constexpr int JP = C::JP;
    constexpr int SLOT = C::template slot_bytes<LOWER>();
    constexpr unsigned FULL = 0xffffffffu;
    typedef typename Sentinel<T>::bits_t bits_t;
    constexpr bits_t SENT = Sentinel<T>::bits;
    extern __shared__ __align__(128) unsigned char wave_smem[];
    if (g.skip && *(volatile const int *)g.skip) return;
    constexpr int NCW = C::NCW;
    const int lane = threadIdx.x & 31;
    const int cw = threadIdx.x >> 5;          // compute warp (its component when NCW > 1)
    const bool producer = cw == NCW;
    WaveHdr *hd = (WaveHdr *)wave_smem;
    unsigned char *slots = wave_smem + C::HDR_BYTES;
    T *ring = (T *)(slots + R * SLOT);       // [HR steps][z, y][32 lanes][BS]
    T *xbuf = ring + (size_t)HR * 2 * 32 * BS;   // NCW > 1: [2 parities][NCW components][32 lanes]
    if (producer && lane == 0) {
        for (int q = 0; q < R; ++q) mbar_init(&hd->bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int a = 1 << g.la, b = 32 >> g.la;
    const int jy = lane & (a - 1), jz = lane >> g.la;
    const int nch = g.npad / G;               // chunks per unit
    const int64_t ucells = (int64_t)g.npad * 32;
    const long long giveup = 4 * g.limit + RS_WAVE_DRAIN;
    unsigned parity = 0;     // compute warp, bit q: parity of slot q's next completion
    bool dead = false;       // producer: a poll gave up; later polls give up at once
    for (;;) {
        __syncthreads();     // both warps are done with the unit before
        if (producer && lane == 0) {
            hd->tk = (int)atomicAdd(&g.st->ticket, 1u);
            hd->prod = 0;
            hd->cons = 0;
        }
        __syncthreads();
        const int tk = *(volatile int *)&hd->tk;
        if (tk >= g.nunits) break;
        const int u = LOWER ? tk : g.nunits - 1 - tk;
        const int zt = u / g.nyt, yt = u - zt * g.nyt;
        const int64_t base = (int64_t)u * ucells;

        if (producer) {
            // ---------------------------------------------------------------
            // producer: bulk copies of chunk q (steps [q G, (q+1) G); the U
            // sweep streams its unit backwards: chunk q is stored chunk
            // nch - 1 - q) into slot q % R once the compute warp has left
            // chunk q - R; hand-off values of step s into ring slot s % HR
            // once it has left step s - HR
            // ---------------------------------------------------------------
            const T *grec = rec + base * RB;
            const T *grhs = rhs + base * BS;
            int qb = 0;                           // next chunk to copy
            auto cons_now = [&]() -> int {
                unsigned c = 0;
                if (lane == 0) c = ld_acq_cta(&hd->cons);
                return (int)__shfl_sync(FULL, c, 0);
            };
            auto issue_ready = [&](int c) {
                while (qb < nch && (qb < R || c >= (qb - R + 1) * G)) {
                    if (lane == 0) {
                        const int k = LOWER ? qb : nch - 1 - qb;
                        const int sl = qb % R;
                        unsigned char *dst = slots + (size_t)sl * SLOT;
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        mbar_arrive_expect_tx(&hd->bar[sl], SLOT);
                        bulk_g2s(dst, grec + (int64_t)k * G * 32 * RB, G * 32 * RB * (int)sizeof(T), &hd->bar[sl]);
                        bulk_g2s(dst + G * 32 * RB * sizeof(T), grhs + (int64_t)k * G * 32 * BS,
                                 G * 32 * BS * (int)sizeof(T), &hd->bar[sl]);
                    }
                    ++qb;
                }
            };
            // The unit's hand-off positions: p < a on the z face (the
            // consumer lane with jy = p on the face row), p >= a on the y face
            // (jz = p - a).  The pairs (step k of the round, position p) are
            // spread over the lanes, JP per lane, so that a round of polls
            // takes few load instructions.
            const int F = a + b;
            const int KE = min(K, (32 * JP) / F);        // steps per round, >= 1
            int jk[JP], jring[JP], jskew[JP];
            int64_t jsrc[JP];
            bool jin[JP], jok[JP];
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                const int idx = lane + 32 * j;
                const int k = idx / F, p = idx - k * F;
                const bool zf = p < a;
                const int cy = zf ? p : (LOWER ? 0 : a - 1);           // consumer lane (cy, cz)
                const int cz = zf ? (LOWER ? 0 : b - 1) : p - a;
                const bool has = zf ? (LOWER ? zt > 0 : zt < g.nzt - 1) : (LOWER ? yt > 0 : yt < g.nyt - 1);
                const bool c_ok = (yt << g.la) + cy < g.ny && zt * b + cz < g.nz;
                // the upstream unit's cell: same x, one step of the skew away
                const int64_t uu = zf ? (LOWER ? (int64_t)u - g.nyt : (int64_t)u + g.nyt) : (LOWER ? u - 1 : u + 1);
                const int sl = zf ? (LOWER ? cy + ((b - 1) << g.la) : cy) : (LOWER ? (a - 1) + (cz << g.la) : (cz << g.la));
                const int so = zf ? (LOWER ? b - 1 : -(b - 1)) : (LOWER ? a - 1 : -(a - 1));
                jin[j] = k < KE;
                jok[j] = jin[j] && has && c_ok;
                jk[j] = k;
                jring[j] = ((zf ? 0 : 1) * 32 + cy + (cz << g.la)) * BS;
                jskew[j] = cy + cz;
                jsrc[j] = jok[j] ? uu * ucells + 32 * so + sl : 0;
            }
            int sp = 0;                           // next step to hand over
            long long tl = clock64();             // last progress
            bool late = false;
            while (sp < g.npad) {
                const int c = cons_now();
                issue_ready(c);
                const int room = min(g.npad, c + HR) - sp;
                if (room <= 0) {
                    // the ring is full: wait for the compute warp
                    const long long dt = clock64() - tl;
                    if (!late && dt > g.limit) {
                        late = true;
                        if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                    }
                    if (dt > giveup) break;
                    continue;
                }
                bits_t v[JP][BS];
                unsigned miss = 0;
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    const int s = sp + jk[j];
                    const int t = LOWER ? s : g.npad - 1 - s;
                    const bool act = jok[j] && jk[j] < room && (unsigned)(t - jskew[j]) < (unsigned)g.nx;
                    const T *src = xv + (jsrc[j] + 32 * (int64_t)t) * BS;
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) v[j][k2] = act ? ld_poll(src + k2) : bits_t(0);
                }
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    bool p = false;
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) p |= v[j][k2] == SENT;
                    if (p) miss |= 1u << jk[j];
                }
                miss = __reduce_or_sync(FULL, miss);
                int ready = min(room, KE);
                if (miss && !dead) ready = min(ready, __ffs(miss) - 1);
                // every position of the steps handed over is written: the
                // value, or 0 where no value is read
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    if (jin[j] && jk[j] < ready) {
                        T *hp = ring + (size_t)((sp + jk[j]) & (HR - 1)) * 2 * 32 * BS + jring[j];
#pragma unroll
                        for (int k2 = 0; k2 < BS; ++k2) hp[k2] = bits_to(T(), v[j][k2]);
                    }
                }
                if (ready > 0) {
                    __syncwarp();
                    sp += ready;
                    if (lane == 0) st_rel_cta(&hd->prod, (unsigned)sp);
                    tl = clock64();
                } else if (clock64() - tl > g.limit) {
                    // give up: carry the sentinel on (arithmetic on it gives NaN)
                    if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                    dead = true;
                }
            }
            // the last chunks, as the compute warp frees their slots
            tl = clock64();
            while (qb < nch) {
                issue_ready(cons_now());
                if (qb < nch && clock64() - tl > giveup) {
                    if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                    break;
                }
            }
            continue;
        }

        // -------------------------------------------------------------------
        // compute warp
        // -------------------------------------------------------------------
        // waits for chunk q's bulk copies; past the limit it records the
        // timeout, then still waits (up to the give-up bound) so that no copy
        // lands in a slot after it has been reused
        auto wait = [&](int q) {
            const int sl = q % R;
            const unsigned par = (parity >> sl) & 1u;
            if (!mbar_try_wait(&hd->bar[sl], par)) {
                const long long t0 = clock64();
                bool late = false;
                while (!mbar_try_wait(&hd->bar[sl], par)) {
                    const long long dt = clock64() - t0;
                    if (!late && dt > g.limit) {
                        late = true;
                        if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                    }
                    if (dt > giveup) break;
                }
            }
            parity ^= 1u << sl;
        };
        // the producer's step counter, until it passes step s
        auto wait_prod = [&](int s) -> unsigned {
            unsigned v = __shfl_sync(FULL, ld_acq_cta(&hd->prod), 0);
            if (v > (unsigned)s) return v;
            const long long t0 = clock64();
            bool late = false;
            for (;;) {
                v = __shfl_sync(FULL, ld_acq_cta(&hd->prod), 0);
                if (v > (unsigned)s) return v;
                const long long dt = clock64() - t0;
                if (!late && dt > g.limit) {
                    late = true;
                    if (lane == 0) atomicOr(g.err, RS_DEVERR_TIMEOUT);
                }
                if (dt > giveup) return (unsigned)g.npad;
            }
        };
        // The step is branch-free but for the hand-off counter: idle lanes
        // (outside the grid, or x outside [0, nx)) read the zero records and
        // right-hand side of the padding and zero hand-off values (the
        // producer writes 0 where no value is read), so they compute 0 from
        // finite inputs and store it into their own padding cells, which no
        // lane reads; an active lane reads only active cells (its in-tile
        // neighbours at the same x are active, and its hand-offs are the
        // upstream unit's active face cells).
        const bool yin = LOWER ? jy > 0 : jy < a - 1;
        const bool zin = LOWER ? jz > 0 : jz < b - 1;
        T *xout = xv + (base + lane) * BS;
        unsigned avail = 0;
        T vprev[BS];
#pragma unroll
        for (int k = 0; k < BS; ++k) vprev[k] = T(0);
        if constexpr (NCW == 1) {
        for (int s0 = 0; s0 < g.npad; s0 += G) {
            wait(s0 / G);
            const unsigned char *sp = slots + (size_t)((s0 / G) % R) * SLOT;
            const T *hring = ring + ((size_t)((s0 & (HR - 1)) * 2) * 32 + lane) * BS;
#pragma unroll
            for (int kk = 0; kk < G; ++kk) {
                const int s = s0 + kk;
                const int t = LOWER ? s : g.npad - 1 - s;
                // this step's record and right-hand side: step t % G of the slot
                const int pos = LOWER ? kk : G - 1 - kk;
                T rv[RB], bv[BS];
                lds_rec<RB>((const T *)sp + (pos * 32 + lane) * RB, rv);
                {
                    const T *rp = (const T *)(sp + G * 32 * RB * sizeof(T)) + (pos * 32 + lane) * BS;
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) bv[k2] = rp[k2];
                }
                // neighbours inside the tile: one shuffle each
                T sy[BS], sz[BS];
#pragma unroll
                for (int k2 = 0; k2 < BS; ++k2) {
                    sy[k2] = LOWER ? __shfl_up_sync(FULL, vprev[k2], 1) : __shfl_down_sync(FULL, vprev[k2], 1);
                    sz[k2] = LOWER ? __shfl_up_sync(FULL, vprev[k2], a) : __shfl_down_sync(FULL, vprev[k2], a);
                }
                // steps before s are done with (every lane stores the same value)
                st_cons(&hd->cons, (unsigned)s);
                // hand-off values from other units (0 where none is read)
                if (avail <= (unsigned)s) avail = wait_prod(s);
                T vz[BS], vy[BS];
#pragma unroll
                for (int k2 = 0; k2 < BS; ++k2) {
                    const T *hp = hring + (size_t)kk * 2 * 32 * BS;
                    const T hz = lds_ho(hp + k2), hy = lds_ho(hp + 32 * BS + k2);
                    vy[k2] = yin ? sy[k2] : hy;
                    vz[k2] = zin ? sz[k2] : hz;
                }
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
                for (int i = 0; i < BS; ++i) {
                    vprev[i] = acc[i];
                    st_poll(xout + (int64_t)32 * BS * t + i, acc[i]);
                }
            }
        }
        } else {
            // NCW = BS warps: warp cw computes component cw of every cell of
            // the step, in the single warp's order (so the values are the
            // same), then the components meet in xbuf; one barrier per step
            // (double-buffered by the step's parity)
            const int ci = cw;
            for (int s0 = 0; s0 < g.npad; s0 += G) {
                wait(s0 / G);
                const unsigned char *sp = slots + (size_t)((s0 / G) % R) * SLOT;
                const T *hring = ring + ((size_t)((s0 & (HR - 1)) * 2) * 32 + lane) * BS;
#pragma unroll
                for (int kk = 0; kk < G; ++kk) {
                    const int s = s0 + kk;
                    const int t = LOWER ? s : g.npad - 1 - s;
                    const int pos = LOWER ? kk : G - 1 - kk;
                    // row ci of each of the record's blocks, and the right-hand side
                    constexpr int NB = LOWER ? 3 : 4;
                    T rv[NB * BS], bv[BS], bci;
                    {
                        const T *rp0 = (const T *)sp + (pos * 32 + lane) * RB + ci * BS;
#pragma unroll
                        for (int q = 0; q < NB; ++q)
#pragma unroll
                            for (int j = 0; j < BS; ++j) rv[q * BS + j] = rp0[q * B2 + j];
                        const T *rp = (const T *)(sp + G * 32 * RB * sizeof(T)) + (pos * 32 + lane) * BS;
#pragma unroll
                        for (int k2 = 0; k2 < BS; ++k2) bv[k2] = rp[k2];
                        bci = rp[ci];
                    }
                    T sy[BS], sz[BS];
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) {
                        sy[k2] = LOWER ? __shfl_up_sync(FULL, vprev[k2], 1) : __shfl_down_sync(FULL, vprev[k2], 1);
                        sz[k2] = LOWER ? __shfl_up_sync(FULL, vprev[k2], a) : __shfl_down_sync(FULL, vprev[k2], a);
                    }
                    // steps before s are done with by every compute warp (the
                    // barrier of step s - 1 is behind all of them)
                    if (cw == 0) st_cons(&hd->cons, (unsigned)s);
                    if (avail <= (unsigned)s) avail = wait_prod(s);
                    T vz[BS], vy[BS];
#pragma unroll
                    for (int k2 = 0; k2 < BS; ++k2) {
                        const T *hp = hring + (size_t)kk * 2 * 32 * BS;
                        const T hz = lds_ho(hp + k2), hy = lds_ho(hp + 32 * BS + k2);
                        vy[k2] = yin ? sy[k2] : hy;
                        vz[k2] = zin ? sz[k2] : hz;
                    }
                    T acc;
                    if (LOWER) {
                        acc = bci;
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[j], vz[j]);
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[BS + j], vy[j]);
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[2 * BS + j], vprev[j]);
                    } else {
                        T sum = T(0);
#pragma unroll
                        for (int j = 0; j < BS; ++j) sum = mad(rv[3 * BS + j], bv[j], sum);
                        acc = sum;
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[j], vz[j]);
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[BS + j], vprev[j]);
#pragma unroll
                        for (int j = 0; j < BS; ++j) acc = msub(acc, rv[2 * BS + j], vy[j]);
                    }
                    st_poll(xout + (int64_t)32 * BS * t + ci, acc);
                    T *xb = xbuf + (size_t)(s & 1) * NCW * 32;
                    xb[ci * 32 + lane] = acc;
                    asm volatile("bar.sync 1, %0;" ::"r"(NCW * 32) : "memory");
#pragma unroll
                    for (int j = 0; j < BS; ++j) vprev[j] = xb[j * 32 + lane];
                }
            }
        }
        // every chunk was waited for at its first step: none is in flight
    }
    wave_end(g);
}

// Permutations between natural order and wave order.  A block takes 32
// steps of one unit: the 32 lanes' x-line segments (x = t - jy - jz for the
// block's steps, contiguous in natural order) and the unit's 32 x 32 wave
// cells of those steps (contiguous in wave order) go through a
// shared-memory tile, so both sides are read and written in whole lines.
constexpr int WAVE_PERM_THREADS = 256;

// x of lane l's cell at step t0 + i, and whether the cell exists
__device__ __forceinline__ bool perm_cell(const WaveArgs &g, int yt, int zt, int l, int t, int *x, int64_t *line)
{
    const int a = 1 << g.la, b = 32 >> g.la;
    const int jy = l & (a - 1), jz = l >> g.la;
    const int y = (yt << g.la) + jy, z = zt * b + jz;
    *x = t - jy - jz;
    *line = ((int64_t)z * g.ny + y) * g.nx;
    return y < g.ny && z < g.nz && *x >= 0 && *x < g.nx && t < g.npad;
}

// r (natural order, FP64) -> wave order in the apply precision, times *scale;
// the U sweep's values back to the sentinel
template <int BS, typename T>
__global__ void __launch_bounds__(WAVE_PERM_THREADS)
k_wave_in(WaveArgs g, const double *__restrict__ r, const double *__restrict__ scale, T *__restrict__ rw,
          T *__restrict__ zreset)
{
    constexpr int W = 32 * BS + 1;                 // tile row: one lane's 32 cells, padded
    __shared__ double tile[32 * W];
    if (g.skip && *(volatile const int *)g.skip) return;
    const double sc = scale ? *scale : 1.0;
    const int nb = (g.npad + 31) / 32;
    const int u = blockIdx.x / nb, t0 = (blockIdx.x - u * nb) * 32;
    const int zt = u / g.nyt, yt = u - zt * g.nyt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the lanes' line segments, one warp per line
    for (int l = wid; l < 32; l += WAVE_PERM_THREADS / 32) {
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            const int e = lane + 32 * k, i = e / BS, c = e - i * BS;
            int x;
            int64_t line;
            if (perm_cell(g, yt, zt, l, t0 + i, &x, &line)) tile[l * W + e] = r[(line + x) * BS + c];
        }
    }
    __syncthreads();
    // the wave cells of the block's steps, contiguous
    const int64_t wbase = ((int64_t)u * g.npad + t0) * 32 * BS;
    for (int e = threadIdx.x; e < 32 * 32 * BS; e += WAVE_PERM_THREADS) {
        const int i = e / (32 * BS), rem = e - i * 32 * BS;
        const int l = rem / BS, c = rem - l * BS;
        int x;
        int64_t line;
        if (perm_cell(g, yt, zt, l, t0 + i, &x, &line)) {
            const double v = tile[l * W + i * BS + c];
            rw[wbase + e] = (T)(sc == 1.0 ? v : v * sc);
            zreset[wbase + e] = bits_to(T(), Sentinel<T>::bits);
        }
    }
}

// the U sweep's values -> natural order, FP64; the L sweep's values back to
// the sentinel
template <int BS, typename T>
__global__ void __launch_bounds__(WAVE_PERM_THREADS)
k_wave_out(WaveArgs g, const T *__restrict__ zw, T *__restrict__ yreset, double *__restrict__ out)
{
    constexpr int W = 32 * BS + 1;
    __shared__ double tile[32 * W];
    if (g.skip && *(volatile const int *)g.skip) return;
    const int nb = (g.npad + 31) / 32;
    const int u = blockIdx.x / nb, t0 = (blockIdx.x - u * nb) * 32;
    const int zt = u / g.nyt, yt = u - zt * g.nyt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t wbase = ((int64_t)u * g.npad + t0) * 32 * BS;
    for (int e = threadIdx.x; e < 32 * 32 * BS; e += WAVE_PERM_THREADS) {
        const int i = e / (32 * BS), rem = e - i * 32 * BS;
        const int l = rem / BS, c = rem - l * BS;
        int x;
        int64_t line;
        if (perm_cell(g, yt, zt, l, t0 + i, &x, &line)) {
            tile[l * W + i * BS + c] = (double)zw[wbase + e];
            yreset[wbase + e] = bits_to(T(), Sentinel<T>::bits);
        }
    }
    __syncthreads();
    for (int l = wid; l < 32; l += WAVE_PERM_THREADS / 32) {
#pragma unroll
        for (int k = 0; k < BS; ++k) {
            const int e = lane + 32 * k, i = e / BS, c = e - i * BS;
            int x;
            int64_t line;
            if (perm_cell(g, yt, zt, l, t0 + i, &x, &line)) out[(line + x) * BS + c] = tile[l * W + e];
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
            const double *av = lu + (size_t)p * B2;
            int lslot = -1, uslot = -1;
            if (d == -nxy) lslot = 0;
            else if (d == -g.nx) lslot = 1;
            else if (d == -1) lslot = 2;
            else if (d == nxy) uslot = 0;
            else if (d == 1) uslot = 1;
            else if (d == g.nx) uslot = 2;
            if (lslot >= 0) {
#pragma unroll
                for (int e = 0; e < B2; ++e) lr[lslot * B2 + e] = (T)av[e];
            } else if (uslot >= 0) {
#pragma unroll
                for (int r2 = 0; r2 < BS; ++r2)
#pragma unroll
                    for (int c2 = 0; c2 < BS; ++c2) {
                        double s = 0.0;
#pragma unroll
                        for (int m = 0; m < BS; ++m) s = __dadd_rn(s, __dmul_rn(D[r2 * BS + m], av[m * BS + c2]));
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
    const int gp = W.nunits * ((W.npad + 31) / 32);
    // one unit per block at a time; up to about 200 KB of blocks per SM (at
    // 128^3 the FP32 block sweeps were 2 % slower with four blocks per SM than
    // with three), and as many of the large FP64-block blocks as fit in the
    // SM's 228 KB (1 KB of it reserved per block)
    const int per_sm = std::max(1, std::min(8, C::NCW > 1 ? (228 * 1024) / (C::template smem_bytes<false>() + 1024)
                                                          : (200 * 1024) / C::template smem_bytes<false>()));
    const int gw = std::max(1, std::min(W.nunits, per_sm * ctx->num_sms));
    constexpr int sl = C::template smem_bytes<true>(), su = C::template smem_bytes<false>();
    RS_TRY((raise_sweep_smem<BS, T, true>(ctx)));
    RS_TRY((raise_sweep_smem<BS, T, false>(ctx)));
    {
        RsProfScope prof(ctx, BS == 1 ? RS_PROF_LSWEEP : RS_PROF_BLSWEEP);
        k_wave_in<BS, T><<<gp, WAVE_PERM_THREADS, 0, ctx->stream>>>(g, r, scale, (T *)W.rw, (T *)W.zw);
        k_wave_sweep<BS, T, true><<<gw, C::THREADS, sl, ctx->stream>>>(g, (const T *)W.lrec, (const T *)W.rw,
                                                                       (T *)W.yw);
    }
    RS_TRY(rs_check_launch(ctx));
    {
        RsProfScope prof(ctx, BS == 1 ? RS_PROF_USWEEP : RS_PROF_BUSWEEP);
        k_wave_sweep<BS, T, false><<<gw, C::THREADS, su, ctx->stream>>>(g, (const T *)W.urec, (const T *)W.yw,
                                                                        (T *)W.zw);
        k_wave_out<BS, T><<<gp, WAVE_PERM_THREADS, 0, ctx->stream>>>(g, (const T *)W.zw, (T *)W.yw, z);
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

template <int BS>
void cfg_of(int fp32, int *G, int *rl, int *ru)
{
    if (fp32) {
        *G = WaveCfg<BS, float>::G;
        *rl = WaveCfg<BS, float>::RL;
        *ru = WaveCfg<BS, float>::RU;
    } else {
        *G = WaveCfg<BS, double>::G;
        *rl = WaveCfg<BS, double>::RL;
        *ru = WaveCfg<BS, double>::RU;
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

// Tile shape: a lanes along y, 32 / a along z, minimising the units on the
// critical path (ceil(ny/a) + ceil(nz/b)), then the idle lanes.
static int tile_log2a(int ny, int nz)
{
    int best = 5;
    int64_t bh = -1, bi = -1;
    for (int la = 0; la <= 5; ++la) {
        const int a = 1 << la, b = 32 >> la;
        const int64_t nyt = (ny + a - 1) / a, nzt = (nz + b - 1) / b;
        const int64_t hops = nyt + nzt, idle = nyt * nzt * 32 - (int64_t)ny * nz;
        if (bh < 0 || hops < bh || (hops == bh && idle < bi)) {
            best = la;
            bh = hops;
            bi = idle;
        }
    }
    return best;
}

int rs_wave_create(IluFactor *f, int nx, int ny, int nz)
{
    rs_ctx *ctx = f->ctx;
    WaveLayout &W = f->W;
    const int bs = f->bs;
    const size_t esz = f->fp32 ? sizeof(float) : sizeof(double);
    int G = 1, rl = 0, ru = 0;
    switch (bs) {
    case 1: cfg_of<1>(f->fp32, &G, &rl, &ru); break;
    case 2: cfg_of<2>(f->fp32, &G, &rl, &ru); break;
    case 3: cfg_of<3>(f->fp32, &G, &rl, &ru); break;
    default: cfg_of<4>(f->fp32, &G, &rl, &ru); break;
    }
    W.nx = nx;
    W.ny = ny;
    W.nz = nz;
    W.la = tile_log2a(ny, nz);
    const int a = 1 << W.la, b = 32 >> W.la;
    W.nyt = (ny + a - 1) / a;
    W.nzt = (nz + b - 1) / b;
    W.nunits = W.nyt * W.nzt;
    const int nsteps = nx + a + b - 2;
    W.npad = (nsteps + G - 1) / G * G;       // whole chunks
    W.ncell = (int64_t)W.nunits * W.npad * 32;
    int st = rs_alloc(ctx, &W.lrec, esz * rl * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.urec, esz * ru * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.rw, esz * bs * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.yw, esz * bs * (size_t)W.ncell);
    st = st ? st : rs_alloc(ctx, &W.zw, esz * bs * (size_t)W.ncell);
    if (st) return st;
    // idle cells are streamed but never used: keep them defined
    RS_CUDA_TRY(cudaMemsetAsync(W.lrec, 0, esz * rl * (size_t)W.ncell, ctx->stream));
    RS_CUDA_TRY(cudaMemsetAsync(W.urec, 0, esz * ru * (size_t)W.ncell, ctx->stream));
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
