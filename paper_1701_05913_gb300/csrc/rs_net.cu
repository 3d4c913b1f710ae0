// Learned pressure stage: a 3-D U-Net (4 levels, 16 channels, 3x3x3
// convolutions, ReLU, 2x2x2 average pooling, nearest x2 upsampling with skip
// concatenation, 1x1x1 head) evaluated and trained with BF16 tensor-core
// kernels and FP32 accumulation.  The paper has no learned component; the
// stage replaces the pressure solve M_p^{-1} of the two-stage CPR
// preconditioner (Alg. 6 as read in rs_precond.cu) inside FGMRES.
//
// Activations are NDHWC bfloat16 (16 channels, 32 bytes per voxel).  Every
// 3x3x3 convolution is an implicit GEMM: a block stages a 16x4x4 output
// brick's 18x6x6 input halo and the 27 weight taps in shared memory, and each
// warp multiplies 16-voxel x-rows (M) by 16 output channels (N) over
// K = 27 taps x channels with mma.m16n8k16 (bf16 in, f32 accumulate),
// fragments loaded with ldmatrix.  The data gradient is the same kernel with
// flipped, transposed weights; the weight gradient multiplies the output
// gradient (transposed with ldmatrix.trans) by the shifted input per tap.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

typedef __nv_bfloat16 bf16;

#define NET_CH 16
#define NET_LEVELS 4
#define NET_NLAYERS 14
#define TX 16
#define TY 4
#define TZ 4
#define TVOX (TX * TY * TZ)
#define HX (TX + 2)
#define HY (TY + 2)
#define HZ (TZ + 2)
#define HVOX (HX * HY * HZ)
#define CONV_THREADS 256
#define NET_MAGIC 0x52534e31u   // file tag of saved networks

enum { IN_PLAIN = 0, IN_CATUP = 1, IN_FIRST = 2 };

// layer table: cin (real), kind of input, level
struct LayerDef {
    int cin;
    int mode;
    int level;
};
static const LayerDef kLayers[NET_NLAYERS] = {
    {2, IN_FIRST, 0},  {16, IN_PLAIN, 0},   // e0a e0b
    {16, IN_PLAIN, 1}, {16, IN_PLAIN, 1},   // e1a e1b
    {16, IN_PLAIN, 2}, {16, IN_PLAIN, 2},   // e2a e2b
    {16, IN_PLAIN, 3}, {16, IN_PLAIN, 3},   // e3a e3b
    {32, IN_CATUP, 2}, {16, IN_PLAIN, 2},   // d2a d2b
    {32, IN_CATUP, 1}, {16, IN_PLAIN, 1},   // d1a d1b
    {32, IN_CATUP, 0}, {16, IN_PLAIN, 0},   // d0a d0b
};
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, D0A, D0B };

static int cin_pad(int l) { return kLayers[l].cin < 16 ? 16 : kLayers[l].cin; }

struct Level {
    int nx, ny, nz;
    int64_t nvox;
};

struct rs_net {
    rs_ctx *ctx;
    float out_scale;
    int64_t nparams;
    int64_t woff[NET_NLAYERS], boff[NET_NLAYERS], hoff;   // offsets in the flat parameter vector
    float *p, *g, *m, *v;                                   // FP32 master, gradient, Adam moments
    int step;
    bf16 *wf[NET_NLAYERS];   // forward weights [27][16][cinp]
    bf16 *wb[NET_NLAYERS];   // data-gradient weights [27][cin][16] (flipped taps)
    // workspace for the current grid
    int nx, ny, nz;
    Level lv[NET_LEVELS];
    bf16 *act[NET_NLAYERS];                 // layer outputs
    bf16 *up0;                              // a decoder's coarse input, upsampled to its level
    // tensor maps of the tcgen05 convolutions' inputs, encoded once per workspace
    struct TmapEntry {
        const void *base;
        int dims[3];
        int box[3];
        CUtensorMap m;
    } tmaps[16];
    int ntmaps;
    bf16 *pool[NET_LEVELS];                 // pooled inputs of e1a, e2a, e3a
    bf16 *g16a[NET_LEVELS], *g16b[NET_LEVELS], *g32[NET_LEVELS];
    float *partials;                        // weight-gradient partials
    int64_t partials_len;
    double *scal;                           // [0] rms, [1] 1/rms, [2] loss, [3..] reduction scratch
    double *red;                            // per-block reduction partials
    unsigned *ticket;
    int *flag;                              // non-finite output flag
    unsigned gen;                           // workspace generation: bumped on every (re)allocation
    double *gout;                           // dL/d(output) (per voxel)
    double *outb;                           // network output during training
    float *headpart;                        // head gradient partials
};

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ bool skipped(const int *skip) { return skip && *(volatile const int *)skip; }

// ---------------------------------------------------------------------------
// halo loader shared by the convolution kernels
// ---------------------------------------------------------------------------
// Loads the 18x6x6 input halo of the brick at (tx0, ty0, tz0) into sx
// (stride SIN bf16 per voxel), zero outside the grid.
template <int CIN, int MODE>
__device__ __forceinline__ void load_halo(bf16 *sx, int SIN, int D, int H, int W, int tx0, int ty0, int tz0,
                                          const bf16 *X, const bf16 *U, const double *r, const double *logk,
                                          const double *rscale)
{
    constexpr int CH8 = CIN / 8;
    for (int i = threadIdx.x; i < HVOX * CH8; i += blockDim.x) {
        const int hv = i / CH8, ch = i % CH8;
        const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
        const int gx = tx0 + hx - 1, gy = ty0 + hy - 1, gz = tz0 + hz - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D) {
            const int64_t vi = ((int64_t)gz * H + gy) * W + gx;
            if (MODE == IN_PLAIN) {
                val = *(const uint4 *)(X + vi * CIN + ch * 8);
            } else if (MODE == IN_CATUP) {
                if (ch < 2) {
                    const int W2 = W >> 1, H2 = H >> 1;
                    const int64_t ci = ((int64_t)(gz >> 1) * H2 + (gy >> 1)) * W2 + (gx >> 1);
                    val = *(const uint4 *)(U + ci * 16 + ch * 8);
                } else {
                    val = *(const uint4 *)(X + vi * 16 + (ch - 2) * 8);
                }
            } else {   // IN_FIRST: channels (r * rscale, logk, 0, ...)
                if (ch == 0) {
                    __nv_bfloat162 p0 = __floats2bfloat162_rn((float)(r[vi] * *rscale), (float)logk[vi]);
                    val.x = *(unsigned *)&p0;
                }
            }
        }
        *(uint4 *)(sx + hv * SIN + ch * 8) = val;
    }
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution (forward, and data gradient with flipped weights)
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(CONV_THREADS)
k_conv3(int D, int H, int W, const bf16 *__restrict__ X, const bf16 *__restrict__ U,
        const double *__restrict__ r, const double *__restrict__ logk, const double *__restrict__ rscale,
        const bf16 *__restrict__ Wp, const float *__restrict__ bias, int relu, bf16 *__restrict__ Y,
        const int *skip)
{
    if (skipped(skip)) return;
    constexpr int SIN = CIN + 8, SW = CIN + 8;
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16 *sx = (bf16 *)smraw;
    bf16 *sw = sx + HVOX * SIN;
    const int ntx = (W + TX - 1) / TX, nty = (H + TY - 1) / TY;
    int b = blockIdx.x;
    const int tx0 = (b % ntx) * TX;
    b /= ntx;
    const int ty0 = (b % nty) * TY, tz0 = (b / nty) * TZ;
    constexpr int WCH = CIN / 8;
    for (int i = threadIdx.x; i < 27 * COUT * WCH; i += blockDim.x) {
        const int row = i / WCH, ch = i % WCH;
        *(uint4 *)(sw + row * SW + ch * 8) = *(const uint4 *)(Wp + (size_t)row * CIN + ch * 8);
    }
    load_halo<CIN, MODE>(sx, SIN, D, H, W, tx0, ty0, tz0, X, U, r, logk, rscale);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, rr = lane & 7;
    constexpr int NT = COUT / 8;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][n][j] = 0.f;

    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            unsigned bfr[NT][2];
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                const bf16 *pb = sw + (t * COUT + (np * 2 + (q >> 1)) * 8 + rr) * SW + kc * 16 + (q & 1) * 8;
                ldsm_x4(bfr[np * 2][0], bfr[np * 2][1], bfr[np * 2 + 1][0], bfr[np * 2 + 1][1], pb);
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int row = warp * 2 + m;
                const int ly = row % TY, lz = row / TY;
                const int lx = rr + (q & 1) * 8;
                const int hv = ((lz + dz) * HY + (ly + dy)) * HX + lx + dx;
                unsigned a0, a1, a2, a3;
                ldsm_x4(a0, a1, a2, a3, sx + hv * SIN + kc * 16 + (q >> 1) * 8);
#pragma unroll
                for (int n = 0; n < NT; ++n) mma_bf16(acc[m][n], a0, a1, a2, a3, bfr[n][0], bfr[n][1]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int row = warp * 2 + m;
        const int gy = ty0 + row % TY, gz = tz0 + row / TY;
        if (gy >= H || gz >= D) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int gx = tx0 + (lane >> 2) + half * 8;
            if (gx >= W) continue;
            const int64_t vi = ((int64_t)gz * H + gy) * W + gx;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = n * 8 + (lane & 3) * 2;
                float v0 = acc[m][n][half * 2], v1 = acc[m][n][half * 2 + 1];
                if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                *(__nv_bfloat162 *)(Y + vi * COUT + co) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// first layer: 2 input channels (r / rms(r) and log k), packed per voxel as
// a pair of bfloat16.  The 27 taps x 2 channels form the K dimension of the
// implicit GEMM (k = 2 t + c: 54, padded to 64), so the tensor cores see 4
// k-steps per voxel row instead of 27 taps padded to 16 channels each; a k
// pair (2t, 2t+1) is the packed word of the voxel at tap t, so the A
// fragments are read from the halo directly.  Persistent blocks: the
// weights are staged once, and the next brick's halo is loaded into
// registers while the current one is computed.
// ---------------------------------------------------------------------------
#define FK 64            // packed K: k = 2 t + c
#define FKS (FK + 8)     // shared-memory row stride (bf16) of the weight tile
#define FHR ((HVOX + CONV_THREADS - 1) / CONV_THREADS)   // halo words per thread

// halo words of brick b for this thread: hc[u] packs (hx, hy, hz) of its
// element u (0xFFFFFFFF past the halo)
__device__ __forceinline__ void first_halo(unsigned (&h)[FHR], const unsigned (&hc)[FHR], int b, int nbricks, int D,
                                           int H, int W, int ntx, int nty, const double *__restrict__ r,
                                           const double *__restrict__ logk, double rsc)
{
    const int tx0 = (b % ntx) * TX - 1, ty0 = ((b / ntx) % nty) * TY - 1, tz0 = (b / (ntx * nty)) * TZ - 1;
    double a[FHR], c[FHR];
    bool in[FHR];
#pragma unroll
    for (int u = 0; u < FHR; ++u) {
        const int gx = tx0 + (int)(hc[u] & 0xFF), gy = ty0 + (int)((hc[u] >> 8) & 0xFF),
                  gz = tz0 + (int)((hc[u] >> 16) & 0xFF);
        in[u] = b < nbricks && hc[u] != 0xFFFFFFFFu && (unsigned)gx < (unsigned)W && (unsigned)gy < (unsigned)H &&
                (unsigned)gz < (unsigned)D;
        const int64_t vi = in[u] ? ((int64_t)gz * H + gy) * W + gx : 0;
        a[u] = in[u] ? r[vi] : 0.0;
        c[u] = in[u] ? logk[vi] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < FHR; ++u) {
        __nv_bfloat162 pr = __floats2bfloat162_rn((float)(a[u] * rsc), (float)c[u]);
        h[u] = in[u] ? *(unsigned *)&pr : 0u;
    }
}

// zero words behind the halo: a padding tap (t >= 27) reads at FPAD past a
// voxel's tap-0 index, which always lands there
#define FPAD HVOX
#define FSH (((TZ - 1) * HY + TY - 1) * HX + 15 + FPAD + 1)

__global__ void __launch_bounds__(CONV_THREADS, 4)
k_conv3_first(int D, int H, int W, const double *__restrict__ r, const double *__restrict__ logk,
              const double *__restrict__ rscale, const bf16 *__restrict__ Wp, const float *__restrict__ bias,
              bf16 *__restrict__ Y, const int *skip)
{
    if (skipped(skip)) return;
    __shared__ __align__(16) bf16 sb[16 * FKS];
    __shared__ unsigned sh[FSH];            // the halo, then zeros for the padding taps
    __shared__ __align__(16) bf16 so[TVOX * 16];   // the output brick, [row][x][channel]
    __shared__ float sbias[16];
    const int ntx = (W + TX - 1) / TX, nty = (H + TY - 1) / TY;
    const int nbricks = ntx * nty * ((D + TZ - 1) / TZ);
    // weights: sb[co][2 t + c] = W[t][co][c] (forward layout [27][16][16], c < 2)
    {
        bf16 wv[16 * FK / CONV_THREADS];
#pragma unroll
        for (int u = 0; u < 16 * FK / CONV_THREADS; ++u) {
            const int i = threadIdx.x + u * CONV_THREADS, co = i / FK, k = i % FK;
            wv[u] = k < 54 ? Wp[((k >> 1) * 16 + co) * 16 + (k & 1)] : __float2bfloat16_rn(0.f);
        }
#pragma unroll
        for (int u = 0; u < 16 * FK / CONV_THREADS; ++u) {
            const int i = threadIdx.x + u * CONV_THREADS;
            sb[(i / FK) * FKS + i % FK] = wv[u];
        }
    }
    if (threadIdx.x < 16) sbias[threadIdx.x] = bias[threadIdx.x];
    for (int i = HVOX + threadIdx.x; i < FSH; i += blockDim.x) sh[i] = 0u;
    const double rsc = *rscale;
    // brick-invariant: this thread's halo elements and fragment offsets
    unsigned hc[FHR];
#pragma unroll
    for (int u = 0; u < FHR; ++u) {
        const int hv = threadIdx.x + u * CONV_THREADS;
        hc[u] = hv < HVOX ? (unsigned)(hv % HX) | ((unsigned)((hv / HX) % HY) << 8) | ((unsigned)(hv / (HX * HY)) << 16)
                          : 0xFFFFFFFFu;
    }
    unsigned hreg[FHR];
    first_halo(hreg, hc, blockIdx.x, nbricks, D, H, W, ntx, nty, r, logk, rsc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, rr = lane & 7;
    const int g = lane >> 2, tq = lane & 3;
    // tap offsets of this thread's k pairs, per k-step and half (padding taps: FPAD)
    int toff[FK / 16][2];
#pragma unroll
    for (int kc = 0; kc < FK / 16; ++kc)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 8 * kc + tq + 4 * h;
            toff[kc][h] = t < 27 ? ((t / 9) * HY + (t / 3) % 3) * HX + t % 3 : FPAD;
        }
    int vbase[2];                            // halo index of voxel x = g at tap 0, per M tile
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int row = warp * 2 + m;
        vbase[m] = ((row / TY) * HY + row % TY) * HX + g;
    }
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x) {
        const int tx0 = (b % ntx) * TX, ty0 = ((b / ntx) % nty) * TY, tz0 = (b / (ntx * nty)) * TZ;
        __syncthreads();                     // the previous brick's reads of sh and so are done
#pragma unroll
        for (int u = 0; u < FHR; ++u) {
            const int hv = threadIdx.x + u * CONV_THREADS;
            if (hv < HVOX) sh[hv] = hreg[u];
        }
        __syncthreads();
        first_halo(hreg, hc, b + gridDim.x, nbricks, D, H, W, ntx, nty, r, logk, rsc);   // in flight during the MMAs

        float acc[2][2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[m][n][j] = 0.f;
#pragma unroll
        for (int kc = 0; kc < FK / 16; ++kc) {
            unsigned b00, b01, b10, b11;
            ldsm_x4(b00, b01, b10, b11, sb + ((q >> 1) * 8 + rr) * FKS + kc * 16 + (q & 1) * 8);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                // A fragment: rows g and g + 8 (x), k pairs 2 tq and 2 tq + 8
                const unsigned *p0 = sh + vbase[m] + toff[kc][0], *p1 = sh + vbase[m] + toff[kc][1];
                mma_bf16(acc[m][0], p0[0], p0[8], p1[0], p1[8], b00, b01);
                mma_bf16(acc[m][1], p0[0], p0[8], p1[0], p1[8], b10, b11);
            }
        }
        // bias and ReLU into the staged brick, then 16-byte stores: a row of
        // 16 x is 512 contiguous bytes of Y
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int row = warp * 2 + m;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int lx = (lane >> 2) + half * 8;
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    const int co = n * 8 + (lane & 3) * 2;
                    float v0 = acc[m][n][half * 2] + sbias[co], v1 = acc[m][n][half * 2 + 1] + sbias[co + 1];
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                    *(__nv_bfloat162 *)(so + (row * TX + lx) * 16 + co) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TVOX * 2 / CONV_THREADS; ++u) {
            const int c = threadIdx.x + u * CONV_THREADS;
            const int v = c >> 1, row = v / TX, lx = v % TX;
            const int gx = tx0 + lx, gy = ty0 + row % TY, gz = tz0 + row / TY;
            if (gx < W && gy < H && gz < D)
                *(uint4 *)(Y + (((int64_t)gz * H + gy) * W + gx) * 16 + (c & 1) * 8) = *(const uint4 *)(so + c * 8);
        }
    }
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution on the tcgen05 tensor cores (16 output channels), used
// for the finest level.
//
// Implicit GEMM: D[voxel][co] = sum over taps t and input channels ci of
// X[voxel + off_t][ci] W[t][co][ci].  A brick is 8 x 16 y BZ z output voxels;
// per (tap, 16-channel chunk, z-plane) one tcgen05.mma with M = 128 (the
// 8 x 16 voxels of a plane), N = 16, K = 16 accumulates in tensor memory.
//
// Operands sit in shared memory in the canonical no-swizzle K-major layout
// (core matrix: 8 rows of 16 bytes).  The brick's input halo (10 x, 18 y,
// BZ + 2 z) is one TMA box per 8-channel plane, stored [z][y][x][8 channels]:
// a core matrix is 8 consecutive x of one y row (128 contiguous bytes), the
// next core matrix along M is the next y row (160 bytes on) and the next 8
// channels are the next plane.  A tap only moves the start address (by
// 16 dx + 160 dy + one z slab dz), so one copy of the halo serves all 27.
//
// The tensor pipe takes an M = 128, K = 16 MMA about every 42 cycles per SM
// for N up to 32, so N = 16 caps the rate at a quarter of the dense peak.
// The N dimension therefore stacks the brick's two z-planes: a halo plane hz
// at tap (dy, dx) meets the weights of tap dz = hz - z for output plane z, so
// one MMA with B = [W(hz) | W(hz - 1)] (zero blocks where dz is out of
// range) serves both planes: 36 MMAs with N = 32 per brick and 16-channel
// chunk instead of 54 with N = 16.  A single thread issues one MMA every
// ~150 cycles, so four warps issue.  Warp roles, coupled only by mbarriers:
//   warps 0-3   MMA issue (lane 0).  Warp w owns accumulator w of each TMEM
//               set: halo plane w, both output planes; the four partial sums
//               meet in the epilogue.
//   warps 4-11  epilogue: tcgen05.ld of the partials, bias, ReLU, bf16 stores;
//               a warp reads TMEM lanes 32 (warp mod 4) + 0..31.
//   warp 12     producer (lane 0): TMA box loads into an NBUF-slot ring.
// Barriers: full[slot] (TMA bytes), empty[slot] (the four issuers' MMAs
// that read the slot completed), tfull[set] (accumulators ready), tempty[set]
// (the epilogue has read them).  Every wait is bounded.
// ---------------------------------------------------------------------------
template <int CIN>
struct TcCfg {
    static constexpr int BX = 8, BY = 16, BZ = 2;
    static constexpr int HXb = BX + 2, HYb = BY + 2, HZb = BZ + 2;
    static constexpr int RS = HXb * 16;                      // bytes of one halo row (10 x, 8 channels)
    static constexpr int BOX = HZb * HYb * RS;               // bytes of one plane's TMA box
    static constexpr int PB = (BOX + 127) / 128 * 128;      // plane stride in shared memory
    static constexpr int NP = CIN / 8, KC = CIN / 16;
    static constexpr int SLOT = NP * PB;
    static constexpr int NBUF = CIN == 16 ? 6 : 3;
    // weights: [hz][dy dx][kc][k half][n = 16 z + co][8 channels], 1 KB a block
    static constexpr int WB = 4 * 9 * KC * 1024;
    static constexpr int SMEM = NBUF * SLOT + WB;
    static constexpr int ACC_COLS = 32;                     // one issuer's accumulator (N = 32)
    static constexpr int NSET = 4, SET_COLS = 4 * ACC_COLS, TMEM_COLS = NSET * SET_COLS;
    static_assert(TMEM_COLS <= 512, "one CTA per SM holds all of TMEM at most");
    static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
    static constexpr int THREADS = 13 * 32;
};

__device__ __forceinline__ uint64_t tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    // shared-memory matrix descriptor: start, leading (K) and stride (M/N)
    // byte offsets in 16-byte units; descriptor version 1; no swizzle
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: F32 accumulate, BF16 A and B, both K-major, M = 128
#define TC_IDESC(N) ((1u << 4) | (1u << 7) | (1u << 10) | (((unsigned)(N) >> 3) << 17) | ((128u >> 4) << 24))

// TMA: one box of a 4-D tensor map (coordinates innermost first) into shared memory
__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
                 "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
                 : "memory");
}

template <int N>
__device__ __forceinline__ void tc_mma(uint32_t tacc, uint64_t da, uint64_t db, unsigned accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tacc),
                 "l"(da), "l"(db), "r"(TC_IDESC(N)), "r"(accumulate)
                 : "memory");
}

// the MMAs of issuer WI for one brick: halo plane WI at the nine (dy, dx) and
// each 16-channel chunk, N = 32 (both output planes).  With one chunk the
// loop is unrolled (each descriptor is the slot's base plus a constant);
// with two it is not, which keeps the descriptors out of registers.
template <int CIN, int WI>
__device__ __forceinline__ void tc_issue(uint32_t tacc, uint64_t dA0, uint64_t dB0)
{
    typedef TcCfg<CIN> C;
#pragma unroll(C::KC == 1 ? 9 : 1)
    for (int j = 0; j < 9; ++j) {
        const int dy = j / 3, dx = j % 3;
#pragma unroll
        for (int kc = 0; kc < C::KC; ++kc) {
            const uint64_t da = dA0 + (uint64_t)((2 * kc * C::PB + (WI * C::HYb + dy) * C::RS + dx * 16) >> 4);
            const uint64_t db = dB0 + (uint64_t)((((WI * 9 + j) * C::KC + kc) * 1024) >> 4);
            tc_mma<32>(tacc, da, db, (j | kc) ? 1u : 0u);
        }
    }
}

template <int CIN>
__global__ void __launch_bounds__(TcCfg<CIN>::THREADS, 1)
k_conv3_tc(int D, int H, int W, const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap umap,
           const bf16 *__restrict__ Wp, const float *__restrict__ bias, bf16 *__restrict__ Y, int *err,
           long long limit, const int *skip, const float *__restrict__ wh, const double *__restrict__ scal,
           float out_scale, double *__restrict__ out, int *flag)
{
    typedef TcCfg<CIN> C;
    if (skipped(skip)) return;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *bufs = tc_smem;                         // NBUF x SLOT
    unsigned char *wts = tc_smem + C::NBUF * C::SLOT;      // WB
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long full[C::NBUF], empty[C::NBUF], tfull[C::NSET], tempty[C::NSET];
    __shared__ float sbias[16], swh[17];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // with wh (16 input channels only) the output head is applied in the
    // epilogue and out written instead of Y: out[v] = (sum_c wh[c] y[v][c] +
    // wh[16]) rms s, summed in channel order, non-finite values flagged
    const bool head = CIN == 16 && wh != nullptr;
    const int nbx = (W + C::BX - 1) / C::BX, nby = (H + C::BY - 1) / C::BY, nbz = (D + C::BZ - 1) / C::BZ;
    const int nbricks = nbx * nby * nbz;
    const int nmine = blockIdx.x < nbricks ? (nbricks - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // block (hz, dy dx, kc), column n = 16 z + co: W[dz = hz - z][dy][dx][co], zero for dz outside 0..2
    for (int i = tid; i < 36 * C::KC * 32 * 2; i += blockDim.x) {
        const int blk = i / 64, n = (i / 2) % 32, kh = i % 2;
        const int kc = blk % C::KC, hz = blk / (9 * C::KC), j = (blk / C::KC) % 9, z = n >> 4, co = n & 15,
                  dz = hz - z;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (dz >= 0 && dz <= 2)
            v = *(const uint4 *)(Wp + ((size_t)(dz * 9 + j) * 16 + co) * CIN + kc * 16 + kh * 8);
        *(uint4 *)(wts + blk * 1024 + kh * 512 + (n >> 3) * 128 + (n & 7) * 16) = v;
    }
    if (tid < 16) sbias[tid] = bias[tid];
    if (head && tid < 17) swh[tid] = wh[tid];
    if (tid == 0) {
        for (int k = 0; k < C::NBUF; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 4);
        }
        for (int k = 0; k < C::NSET; ++k) {
            mbar_init(&tfull[k], 4);
            mbar_init(&tempty[k], 256);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the weights, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp == 12) {
        // producer
        if (lane == 0) {
            for (int k = 0; k < nmine; ++k) {
                const int slot = k % C::NBUF, b = blockIdx.x + k * gridDim.x;
                if (k >= C::NBUF) mbar_wait(&empty[slot], (unsigned)((k / C::NBUF - 1) & 1), limit, err);
                const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
                mbar_arrive_expect_tx(&full[slot], (unsigned)(C::NP * C::BOX));
#pragma unroll
                for (int pl = 0; pl < C::NP; ++pl) {
                    // 16 input channels: both planes from X; 32: planes 0, 1 from the
                    // upsampled coarse tensor, 2, 3 from X (the skip connection)
                    const CUtensorMap *map = (CIN == 32 && pl < 2) ? &umap : &xmap;
                    tma_load4(bufs + slot * C::SLOT + pl * C::PB, map, (pl & 1) * 8, bx * C::BX - 1, by * C::BY - 1,
                              bz * C::BZ - 1, &full[slot]);
                }
            }
            // the copies of the last bricks have landed before this block can end
            for (int k = nmine > C::NBUF ? nmine - C::NBUF : 0; k < nmine; ++k)
                mbar_wait(&full[k % C::NBUF], (unsigned)((k / C::NBUF) & 1), limit, err);
        }
    } else if (warp < 4) {
        // MMA issue
        if (lane == 0) {
            // B: the k halves of a block are 512 bytes apart, 8-column groups 128
            const uint64_t dB0 = tc_desc(smem_u32(wts), 512, 128);
            for (int k = 0; k < nmine; ++k) {
                const int slot = k % C::NBUF, set = k % C::NSET;
                mbar_wait(&full[slot], (unsigned)((k / C::NBUF) & 1), limit, err);
                if (k >= C::NSET) mbar_wait(&tempty[set], (unsigned)((k / C::NSET - 1) & 1), limit, err);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tacc = tmem_base + set * C::SET_COLS + warp * C::ACC_COLS;
                const uint64_t dA0 = tc_desc(smem_u32(bufs + slot * C::SLOT), C::PB, C::RS);
                switch (warp) {
                case 0: tc_issue<CIN, 0>(tacc, dA0, dB0); break;
                case 1: tc_issue<CIN, 1>(tacc, dA0, dB0); break;
                case 2: tc_issue<CIN, 2>(tacc, dA0, dB0); break;
                default: tc_issue<CIN, 3>(tacc, dA0, dB0); break;
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[slot]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&tfull[set]))
                             : "memory");
            }
            // this issuer's last MMAs have completed before TMEM is released
            if (nmine > 0)
                mbar_wait(&tfull[(nmine - 1) % C::NSET], (unsigned)(((nmine - 1) / C::NSET) & 1), limit, err);
        }
    } else {
        // epilogue: warps 4..11
        const int e = warp - 4, q = warp & 3;
        const int row = q * 32 + lane;                      // M row = TMEM lane
        const int x = row & 7, y = row >> 3;
        const int z = C::BZ == 2 ? (e >> 2) : 0;
        const int c0 = C::BZ == 2 ? 0 : (e >> 2) * 8;      // 32 input channels: two warps per quadrant
        constexpr int NCOL = C::BZ == 2 ? 16 : 8;
        for (int k = 0; k < nmine; ++k) {
            const int set = k % C::NSET, b = blockIdx.x + k * gridDim.x;
            mbar_wait(&tfull[set], (unsigned)((k / C::NSET) & 1), limit, err);
            __syncwarp();   // the TMEM loads below are warp-collective
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float f[NCOL];
#pragma unroll
            for (int j = 0; j < NCOL; ++j) f[j] = sbias[c0 + j];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                // issuer g's partial: plane z of its N = 32 accumulator, or its 16 columns
                const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + set * C::SET_COLS +
                                    g * C::ACC_COLS + z * 16;
                uint32_t v[16];
                if constexpr (NCOL == 16) {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                                 : "r"(ta));
                } else {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                                   "=r"(v[6]), "=r"(v[7])
                                 : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < NCOL; ++j) f[j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty[set]);
            const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
            const int gx = bx * C::BX + x, gy = by * C::BY + y, gz = bz * C::BZ + z;
            if (gx < W && gy < H && gz < D) {
                const int64_t vi = ((int64_t)gz * H + gy) * W + gx;
                unsigned packed[NCOL / 2];
#pragma unroll
                for (int j = 0; j < NCOL / 2; ++j) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(f[2 * j], 0.f), fmaxf(f[2 * j + 1], 0.f));
                    packed[j] = *(unsigned *)&h;
                }
                if constexpr (NCOL == 16) {
                    if (head) {
                        float hs = swh[16];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const __nv_bfloat162 h = *(const __nv_bfloat162 *)&packed[j];
                            hs = fmaf(swh[2 * j], __low2float(h), hs);
                            hs = fmaf(swh[2 * j + 1], __high2float(h), hs);
                        }
                        const double o = (double)hs * (scal[0] * (double)out_scale);
                        out[vi] = o;
                        if (!isfinite(o)) atomicOr(flag, 1);
                        continue;
                    }
                }
                uint4 *dst = (uint4 *)(Y + vi * 16 + c0);
                dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                if constexpr (NCOL == 16) dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS));
    }
}

// nearest-neighbour x2 upsampling of a 16-channel tensor: Uf[z][y][x] = Uc[z/2][y/2][x/2]
__global__ void k_upsample2(int D, int H, int W, const bf16 *__restrict__ Uc, bf16 *__restrict__ Uf, const int *skip)
{
    if (skipped(skip)) return;
    const int64_t n = (int64_t)D * H * W;
    const int W2 = W >> 1, H2 = H >> 1;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        const int64_t c = ((int64_t)(z >> 1) * H2 + (y >> 1)) * W2 + (x >> 1);
        const uint4 *s = (const uint4 *)(Uc + c * 16);
        uint4 *d = (uint4 *)(Uf + v * 16);
        d[0] = s[0];
        d[1] = s[1];
    }
}

// ---------------------------------------------------------------------------
// weight gradient: partial[blk][t][co][ci] = sum over the brick of
// G[v][co] * X[v + off_t][ci];  partial[blk][27*16*CIN + co] = sum_v G[v][co]
// ---------------------------------------------------------------------------
template <int CIN, int MODE>
__global__ void __launch_bounds__(CONV_THREADS)
k_conv3_dw(int D, int H, int W, const bf16 *__restrict__ X, const bf16 *__restrict__ U,
           const double *__restrict__ r, const double *__restrict__ logk, const double *__restrict__ rscale,
           const bf16 *__restrict__ G, float *__restrict__ partial)
{
    constexpr int SIN = CIN + 8, SG = 24;
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16 *sx = (bf16 *)smraw;
    bf16 *sg = sx + HVOX * SIN;
    const int ntx = (W + TX - 1) / TX, nty = (H + TY - 1) / TY;
    int b = blockIdx.x;
    const int tx0 = (b % ntx) * TX;
    b /= ntx;
    const int ty0 = (b % nty) * TY, tz0 = (b / nty) * TZ;
    load_halo<CIN, MODE>(sx, SIN, D, H, W, tx0, ty0, tz0, X, U, r, logk, rscale);
    for (int i = threadIdx.x; i < TVOX * 2; i += blockDim.x) {
        const int tv = i >> 1, ch = i & 1;
        const int lx = tv % TX, ly = (tv / TX) % TY, lz = tv / (TX * TY);
        const int gx = tx0 + lx, gy = ty0 + ly, gz = tz0 + lz;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gx < W && gy < H && gz < D) val = *(const uint4 *)(G + (((int64_t)gz * H + gy) * W + gx) * 16 + ch * 8);
        *(uint4 *)(sg + tv * SG + ch * 8) = val;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, rr = lane & 7;
    constexpr int NT = CIN / 8;
    float acc[4][NT][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[a][n][j] = 0.f;
    for (int row = 0; row < TY * TZ; ++row) {
        const int ly = row % TY, lz = row / TY;
        unsigned a0, a1, a2, a3;
        // A = G^T: rows co, columns = the 16 voxels of this x-row
        ldsm_x4_t(a0, a1, a2, a3, sg + (row * TX + (q >> 1) * 8 + rr) * SG + (q & 1) * 8);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int t = warp + 8 * s;
            if (t >= 27) continue;
            const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
            const int lx = (q & 1) * 8 + rr;
            const int hv = ((lz + dz) * HY + (ly + dy)) * HX + lx + dx;
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                unsigned b0, b1, b2, b3;
                ldsm_x4_t(b0, b1, b2, b3, sx + hv * SIN + np * 16 + (q >> 1) * 8);
                mma_bf16(acc[s][np * 2], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[s][np * 2 + 1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    float *out = partial + (size_t)blockIdx.x * (27 * 16 * CIN + 16);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int t = warp + 8 * s;
        if (t >= 27) continue;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = lane >> 2, ci = n * 8 + (lane & 3) * 2;
            out[(t * 16 + co) * CIN + ci] = acc[s][n][0];
            out[(t * 16 + co) * CIN + ci + 1] = acc[s][n][1];
            out[(t * 16 + co + 8) * CIN + ci] = acc[s][n][2];
            out[(t * 16 + co + 8) * CIN + ci + 1] = acc[s][n][3];
        }
    }
    // bias gradient: sum of G over the brick
    if (threadIdx.x < 16) {
        float sum = 0.f;
        for (int tv = 0; tv < TVOX; ++tv) sum += __bfloat162float(sg[tv * SG + threadIdx.x]);
        out[27 * 16 * CIN + threadIdx.x] = sum;
    }
}

// grad[woff + (t*16+co)*cin + ci] += w * sum_b partial[b][(t*16+co)*cinp + ci]; bias likewise
__global__ void k_dw_reduce(int nblocks, int cin, int cinp, const float *__restrict__ partial, float *grad,
                            int64_t woff, int64_t boff, float wscale)
{
    const int stride = 27 * 16 * cinp + 16;
    const int nw = 27 * 16 * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + 16; i += gridDim.x * blockDim.x) {
        int src;
        int64_t dst;
        if (i < nw) {
            const int tc = i / cin, ci = i % cin;
            src = tc * cinp + ci;
            dst = woff + i;
        } else {
            src = 27 * 16 * cinp + (i - nw);
            dst = boff + (i - nw);
        }
        float s = 0.f;
        for (int bk = 0; bk < nblocks; ++bk) s += partial[(size_t)bk * stride + src];
        grad[dst] += wscale * s;
    }
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------
// 2x2x2 average pooling of a 16-channel tensor: a thread per coarse voxel and
// 8-channel half, 16-byte loads; per channel the eight inputs are summed in
// FP32 in (dz, dy, dx) order
__global__ void k_avgpool(int Dc, int Hc, int Wc, const bf16 *__restrict__ X, bf16 *__restrict__ Y, const int *skip)
{
    if (skipped(skip)) return;
    const int64_t n = (int64_t)Dc * Hc * Wc * 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(i & 1);
        const int64_t vc = i >> 1;
        const int x = (int)(vc % Wc), y = (int)((vc / Wc) % Hc), z = (int)(vc / ((int64_t)Wc * Hc));
        const int W = Wc * 2, H = Hc * 2;
        uint4 in[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t vf = ((int64_t)(2 * z + (k >> 2)) * H + (2 * y + ((k >> 1) & 1))) * W + 2 * x + (k & 1);
            in[k] = *(const uint4 *)(X + vf * 16 + h * 8);
        }
        unsigned outw[4];
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const bf16 *e = (const bf16 *)&in[k];
                s0 += __bfloat162float(e[c]);
                s1 += __bfloat162float(e[c + 1]);
            }
            __nv_bfloat162 pr = __floats2bfloat162_rn(s0 * 0.125f, s1 * 0.125f);
            outw[c >> 1] = *(unsigned *)&pr;
        }
        *(uint4 *)(Y + vc * 16 + h * 8) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
    }
}

// g_pre = g * (y > 0)
__global__ void k_relu_mask(int64_t n, const bf16 *__restrict__ g, const bf16 *__restrict__ y, bf16 *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(y[i]) > 0.f ? g[i] : __float2bfloat16_rn(0.f);
}

// coarse gradient of a nearest-upsampled input: sum over the 8 children of
// channels 0..15 of a 32-channel fine gradient
__global__ void k_up_backward(int Dc, int Hc, int Wc, const bf16 *__restrict__ gcat, bf16 *__restrict__ gc)
{
    const int64_t n = (int64_t)Dc * Hc * Wc * 16;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % 16);
        const int64_t vc = i / 16;
        const int x = (int)(vc % Wc), y = (int)((vc / Wc) % Hc), z = (int)(vc / ((int64_t)Wc * Hc));
        const int W = Wc * 2, H = Hc * 2;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t vf = ((int64_t)(2 * z + (k >> 2)) * H + (2 * y + ((k >> 1) & 1))) * W + 2 * x + (k & 1);
            s += __bfloat162float(gcat[vf * 32 + c]);
        }
        gc[i] = __float2bfloat16_rn(s);
    }
}

// gradient of a skip tensor: skip part of the decoder's gradient (channels
// 16..31 of gcat) plus the average-pooling adjoint of the coarse gradient
__global__ void k_pool_backward_add(int D, int H, int W, const bf16 *__restrict__ gcoarse,
                                    const bf16 *__restrict__ gcat, bf16 *__restrict__ out)
{
    const int64_t n = (int64_t)D * H * W * 16;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % 16);
        const int64_t v = i / 16;
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        const int64_t vc = ((int64_t)(z >> 1) * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1);
        const float s = __bfloat162float(gcat[v * 32 + 16 + c]) + 0.125f * __bfloat162float(gcoarse[vc * 16 + c]);
        out[i] = __float2bfloat16_rn(s);
    }
}

// sum of squares of r (FP64) with a last-block finish: scal[0] = rms, scal[1] = 1/rms
__global__ void __launch_bounds__(256)
k_rms(int64_t n, const double *__restrict__ r, double *red, unsigned *ticket, double *scal, const int *skip)
{
    if (skipped(skip)) return;
    __shared__ double sm[8];
    __shared__ bool last;
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (((uintptr_t)r & 15) == 0) {
        // four 16-byte loads in flight per thread (n is even: the grid's
        // sides are multiples of 8)
        const int64_t n2 = n / 2;
        const double2 *r2 = (const double2 *)r;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 4 * stride) {
            double2 a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = i + u * stride < n2 ? r2[i + u * stride] : make_double2(0.0, 0.0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s = fma(a[u].x, a[u].x, s);
                s = fma(a[u].y, a[u].y, s);
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s = fma(r[i], r[i], s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        red[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(red + b);
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        double rms = sqrt(t / (double)n);
        if (!(rms > 0.0) || !isfinite(rms)) rms = 1.0;
        scal[0] = rms;
        scal[1] = 1.0 / rms;
        *ticket = 0;
    }
}

// head: out[v] = (sum_c wh[c] x[v][c] + bh) * rms * s; flags non-finite output
__global__ void k_head(int64_t n, const bf16 *__restrict__ x, const float *__restrict__ wh, const double *__restrict__ scal,
                       float out_scale, double *__restrict__ out, int *flag, const int *skip)
{
    if (skipped(skip)) return;
    const double sc = scal[0] * (double)out_scale;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint4 *p = (const uint4 *)(x + v * 16);
        const uint4 a = p[0], b = p[1];
        const bf16 *e0 = (const bf16 *)&a, *e1 = (const bf16 *)&b;
        float s = wh[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(wh[c], __bfloat162float(e0[c]), s);
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(wh[8 + c], __bfloat162float(e1[c]), s);
        const double o = (double)s * sc;
        out[v] = o;
        if (flag && !isfinite(o)) atomicOr(flag, 1);
    }
}

// loss = sum (o - e)^2 / sum e^2 (two sums with a last-block finish), and
// gout = w * 2 (o - e) / sum e^2 computed after the sums by k_loss_grad
__global__ void __launch_bounds__(256)
k_loss_sums(int64_t n, const double *__restrict__ o, const double *__restrict__ e, double *red, unsigned *ticket,
            double *scal)
{
    __shared__ double sm[2][8];
    __shared__ bool last;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = o[i] - e[i];
        s0 = fma(d, d, s0);
        s1 = fma(e[i], e[i], s1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = s0; sm[1][threadIdx.x >> 5] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += sm[0][w]; b += sm[1][w]; }
        red[2 * blockIdx.x] = a;
        red[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int bk = threadIdx.x; bk < (int)gridDim.x; bk += 32) { a += __ldcg(red + 2 * bk); b += __ldcg(red + 2 * bk + 1); }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
        scal[2] = b > 0.0 ? a / b : 0.0;
        scal[3] = b;
        *ticket = 0;
    }
}

__global__ void k_loss_grad(int64_t n, const double *__restrict__ o, const double *__restrict__ e,
                            const double *__restrict__ scal, double w, double *__restrict__ g)
{
    const double den = scal[3] > 0.0 ? scal[3] : 1.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = w * 2.0 * (o[i] - e[i]) / den;
}

// head backward: ge = g * rms * s; dx[v][c] = ge * wh[c]; per-block partial
// sums of ge * x[v][c] (16) and ge (1) into hp[block][17]
__global__ void __launch_bounds__(256)
k_head_backward(int64_t n, const bf16 *__restrict__ x, const float *__restrict__ wh, const double *__restrict__ scal,
                float out_scale, const double *__restrict__ g, bf16 *__restrict__ dx, float *__restrict__ hp)
{
    __shared__ float sm[8][17];
    const double sc = scal[0] * (double)out_scale;
    float acc[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) acc[c] = 0.f;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const float ge = (float)(g[v] * sc);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            acc[c] = fmaf(ge, __bfloat162float(x[v * 16 + c]), acc[c]);
            dx[v * 16 + c] = __float2bfloat16_rn(ge * wh[c]);
        }
        acc[16] += ge;
    }
#pragma unroll
    for (int c = 0; c < 17; ++c) {
        float s = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += sm[w][threadIdx.x];
        hp[blockIdx.x * 17 + threadIdx.x] = s;
    }
}

__global__ void k_head_reduce(int nblocks, const float *__restrict__ hp, float *grad, int64_t hoff)
{
    const int c = threadIdx.x;
    if (c >= 17) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += hp[b * 17 + c];
    grad[hoff + c] += s;
}

// FP32 master -> bf16 forward [27][16][cinp] and data-gradient [27][cin][16] weights
__global__ void k_pack_weights(int cin, int cinp, const float *__restrict__ w, bf16 *__restrict__ wf, bf16 *__restrict__ wb)
{
    const int n = 27 * 16 * cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cinp, co = (i / cinp) % 16, t = i / (16 * cinp);
        const float v = ci < cin ? w[(t * 16 + co) * cin + ci] : 0.f;
        wf[i] = __float2bfloat16_rn(v);
        if (wb && ci < cin) wb[((26 - t) * cin + ci) * 16 + co] = __float2bfloat16_rn(v);
    }
}

__global__ void k_adam(int64_t n, float *p, float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int conv_smem(int cin, int cout) { return (HVOX * (cin + 8) + 27 * cout * (cin + 8)) * 2; }
static int dw_smem(int cin) { return (HVOX * (cin + 8) + TVOX * 24) * 2; }

static int64_t nbricks(const Level &L)
{
    return (int64_t)((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY) * ((L.nz + TZ - 1) / TZ);
}

static int ew_grid(rs_ctx *ctx, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

static bool g_attrs_set = false;

template <int CIN, int COUT, int MODE>
static void set_attr()
{
    cudaFuncSetAttribute(k_conv3<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem(CIN, COUT));
}

template <int CIN, int MODE>
static void set_attr_dw()
{
    cudaFuncSetAttribute(k_conv3_dw<CIN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, dw_smem(CIN));
}

static void ensure_attrs()
{
    if (g_attrs_set) return;
    set_attr<16, 16, IN_PLAIN>();
    set_attr<16, 16, IN_FIRST>();
    set_attr<32, 16, IN_CATUP>();
    set_attr<16, 32, IN_PLAIN>();
    set_attr_dw<16, IN_PLAIN>();
    set_attr_dw<16, IN_FIRST>();
    set_attr_dw<32, IN_CATUP>();
    cudaFuncSetAttribute(k_conv3_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<16>::SMEM);
    cudaFuncSetAttribute(k_conv3_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<32>::SMEM);
    g_attrs_set = true;
}

// TMA tensor map of an NDHWC bf16 tensor [D][H][W][C]: boxes of 8 channels
// x bx x by y x bz z, zero fill outside; the encoder comes from the driver
// through the runtime's versioned entry-point query
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static int make_tmap(CUtensorMap *m, const bf16 *base, int C, int W, int H, int D, int bx, int by, int bz)
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return RS_ERR_CUDA;
        fn = (EncodeTiledFn)p;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? RS_OK : RS_ERR_CUDA;
}

// the tensor map of a workspace buffer, encoded on first use (the buffers
// live as long as the workspace, which clears the cache)
static int cached_tmap(rs_net *net, const CUtensorMap **out, const bf16 *base, int W, int H, int D, int bx, int by,
                       int bz)
{
    for (int k = 0; k < net->ntmaps; ++k) {
        const rs_net::TmapEntry &e = net->tmaps[k];
        if (e.base == base && e.dims[0] == W && e.dims[1] == H && e.dims[2] == D && e.box[0] == bx &&
            e.box[1] == by && e.box[2] == bz) {
            *out = &e.m;
            return RS_OK;
        }
    }
    if (net->ntmaps == 16) net->ntmaps = 0;      // more maps than expected: start over
    rs_net::TmapEntry &e = net->tmaps[net->ntmaps];
    RS_TRY(make_tmap(&e.m, base, 16, W, H, D, bx, by, bz));
    e.base = base;
    e.dims[0] = W;
    e.dims[1] = H;
    e.dims[2] = D;
    e.box[0] = bx;
    e.box[1] = by;
    e.box[2] = bz;
    ++net->ntmaps;
    *out = &e.m;
    return RS_OK;
}

static void free_workspace(rs_net *net)
{
    rs_ctx *c = net->ctx;
    net->ntmaps = 0;
    for (int l = 0; l < NET_NLAYERS; ++l) { rs_free(c, net->act[l]); net->act[l] = nullptr; }
    rs_free(c, net->up0);
    net->up0 = nullptr;
    for (int l = 0; l < NET_LEVELS; ++l) {
        rs_free(c, net->pool[l]);
        rs_free(c, net->g16a[l]);
        rs_free(c, net->g16b[l]);
        rs_free(c, net->g32[l]);
        net->pool[l] = net->g16a[l] = net->g16b[l] = net->g32[l] = nullptr;
    }
    rs_free(c, net->partials);
    rs_free(c, net->gout);
    rs_free(c, net->outb);
    rs_free(c, net->headpart);
    net->partials = nullptr;
    net->gout = nullptr;
    net->outb = nullptr;
    net->headpart = nullptr;
    net->nx = net->ny = net->nz = 0;
}

static int ensure_workspace(rs_net *net, int nx, int ny, int nz)
{
    if (net->nx == nx && net->ny == ny && net->nz == nz) return RS_OK;
    if (nx % 8 || ny % 8 || nz % 8 || nx < 8 || ny < 8 || nz < 8) return RS_ERR_INVALID_ARG;
    free_workspace(net);
    rs_ctx *c = net->ctx;
    for (int l = 0; l < NET_LEVELS; ++l) {
        net->lv[l].nx = nx >> l;
        net->lv[l].ny = ny >> l;
        net->lv[l].nz = nz >> l;
        net->lv[l].nvox = (int64_t)net->lv[l].nx * net->lv[l].ny * net->lv[l].nz;
    }
    int st = RS_OK;
    for (int l = 0; l < NET_NLAYERS && !st; ++l)
        st = rs_alloc(c, (void **)&net->act[l], sizeof(bf16) * 16 * net->lv[kLayers[l].level].nvox);
    if (!st) st = rs_alloc(c, (void **)&net->up0, sizeof(bf16) * 16 * net->lv[0].nvox);
    int64_t maxp = 0;
    for (int l = 0; l < NET_LEVELS && !st; ++l) {
        const int64_t nv = net->lv[l].nvox;
        st = rs_alloc(c, (void **)&net->pool[l], sizeof(bf16) * 16 * nv);
        if (!st) st = rs_alloc(c, (void **)&net->g16a[l], sizeof(bf16) * 16 * nv);
        if (!st) st = rs_alloc(c, (void **)&net->g16b[l], sizeof(bf16) * 16 * nv);
        if (!st) st = rs_alloc(c, (void **)&net->g32[l], sizeof(bf16) * 32 * nv);
        maxp = std::max(maxp, nbricks(net->lv[l]) * (27 * 16 * 32 + 16));
    }
    if (!st) st = rs_alloc(c, (void **)&net->partials, sizeof(float) * maxp);
    if (!st) st = rs_alloc(c, (void **)&net->gout, sizeof(double) * net->lv[0].nvox);
    if (!st) st = rs_alloc(c, (void **)&net->outb, sizeof(double) * net->lv[0].nvox);
    if (!st) st = rs_alloc(c, (void **)&net->headpart, sizeof(float) * 17 * c->num_sms * 8);
    if (st) { free_workspace(net); return st; }
    net->partials_len = maxp;
    net->nx = nx;
    net->ny = ny;
    net->nz = nz;
    ++net->gen;
    return RS_OK;
}

static int pack_all(rs_net *net)
{
    rs_ctx *c = net->ctx;
    for (int l = 0; l < NET_NLAYERS; ++l) {
        const int cin = kLayers[l].cin, cinp = cin_pad(l);
        k_pack_weights<<<ew_grid(c, 27 * 16 * cinp), 256, 0, c->stream>>>(cin, cinp, net->p + net->woff[l], net->wf[l],
                                                                         l == E0A ? nullptr : net->wb[l]);
    }
    c->launches += NET_NLAYERS - 1;
    return rs_check_launch(c);
}

// launches one forward convolution of layer l
// The finest level's forward convolutions run on tcgen05, and so do a
// coarser level's when it has at least two of the kernel's bricks (8 x 16 x 2
// voxels) per SM: with fewer, the persistent pipeline's prologue (weights,
// TMEM allocation, first copies) is not amortised and mma.sync is as fast.
static bool use_tc(const rs_net *net, int level)
{
    const Level &L = net->lv[level];
    const int64_t bricks = (int64_t)((L.nx + 7) / 8) * ((L.ny + 15) / 16) * ((L.nz + 1) / 2);
    return level == 0 || bricks >= 2 * (int64_t)net->ctx->num_sms;
}

// hout: the last layer applies the output head in its epilogue and writes
// the network output there instead of Y (finest level, tcgen05 kernel only)
static int conv_forward(rs_net *net, int l, const bf16 *X, const bf16 *U, const double *r, const double *logk,
                        bf16 *Y, const int *skip, double *hout = nullptr)
{
    rs_ctx *c = net->ctx;
    const Level &L = net->lv[kLayers[l].level];
    const int grid = (int)nbricks(L);
    const float *bias = net->p + net->boff[l];
    if (use_tc(net, kLayers[l].level) && kLayers[l].mode != IN_FIRST) {
        const CUtensorMap *xmap, *umap;
        if (kLayers[l].mode == IN_CATUP) {
            // the coarse input, upsampled to this level, is the first half of the concatenation
            typedef TcCfg<32> TC;
            RS_TRY(cached_tmap(net, &umap, net->up0, L.nx, L.ny, L.nz, TC::HXb, TC::HYb, TC::HZb));
            RS_TRY(cached_tmap(net, &xmap, X, L.nx, L.ny, L.nz, TC::HXb, TC::HYb, TC::HZb));
            k_upsample2<<<ew_grid(c, L.nvox), 256, 0, c->stream>>>(L.nz, L.ny, L.nx, U, net->up0, skip);
            RS_TRY(rs_check_launch(c));
            const int nb = ((L.nx + TC::BX - 1) / TC::BX) * ((L.ny + TC::BY - 1) / TC::BY) * ((L.nz + TC::BZ - 1) / TC::BZ);
            k_conv3_tc<32><<<std::min(nb, c->num_sms), TC::THREADS, TC::SMEM, c->stream>>>(
                L.nz, L.ny, L.nx, *xmap, *umap, net->wf[l], bias, Y, c->d_err, c->spin_limit, skip, nullptr,
                nullptr, 0.f, nullptr, nullptr);
        } else {
            typedef TcCfg<16> TC;
            RS_TRY(cached_tmap(net, &xmap, X, L.nx, L.ny, L.nz, TC::HXb, TC::HYb, TC::HZb));
            const int nb = ((L.nx + TC::BX - 1) / TC::BX) * ((L.ny + TC::BY - 1) / TC::BY) * ((L.nz + TC::BZ - 1) / TC::BZ);
            k_conv3_tc<16><<<std::min(nb, c->num_sms), TC::THREADS, TC::SMEM, c->stream>>>(
                L.nz, L.ny, L.nx, *xmap, *xmap, net->wf[l], bias, Y, c->d_err, c->spin_limit, skip,
                hout ? net->p + net->hoff : nullptr, net->scal, net->out_scale, hout, net->flag);
        }
        return rs_check_launch(c);
    }
    if (hout) return RS_ERR_INVALID_ARG;        // the head is fused on the tcgen05 path only
    switch (kLayers[l].mode) {
    case IN_FIRST:
        k_conv3_first<<<std::min(grid, c->num_sms * 4), CONV_THREADS, 0, c->stream>>>(
            L.nz, L.ny, L.nx, r, logk, net->scal + 1, net->wf[l], bias, Y, skip);
        break;
    case IN_CATUP:
        k_conv3<32, 16, IN_CATUP><<<grid, CONV_THREADS, conv_smem(32, 16), c->stream>>>(
            L.nz, L.ny, L.nx, X, U, nullptr, nullptr, nullptr, net->wf[l], bias, 1, Y, skip);
        break;
    default:
        k_conv3<16, 16, IN_PLAIN><<<grid, CONV_THREADS, conv_smem(16, 16), c->stream>>>(
            L.nz, L.ny, L.nx, X, nullptr, nullptr, nullptr, nullptr, net->wf[l], bias, 1, Y, skip);
    }
    return rs_check_launch(c);
}

static int pool_forward(rs_net *net, int lvl, const bf16 *X, bf16 *Y, const int *skip)
{
    rs_ctx *c = net->ctx;
    const Level &L = net->lv[lvl];
    k_avgpool<<<ew_grid(c, L.nvox * 2), 256, 0, c->stream>>>(L.nz, L.ny, L.nx, X, Y, skip);
    return rs_check_launch(c);
}

// forward pass; out (FP64, nvox) = network(r, logk) * rms * out_scale.
// keep: the last layer's activations are kept for a backward pass; else the
// output head runs in the last convolution's epilogue
static int net_forward(rs_net *net, const double *r, const double *logk, double *out, const int *skip,
                       bool keep = false)
{
    rs_ctx *c = net->ctx;
    const int64_t n0 = net->lv[0].nvox;
    // one profiler interval over the whole pass: the kernels, without the
    // host work between their launches
    RsProfScope prof(c, RS_PROF_NET);
    k_rms<<<c->red_blocks, 256, 0, c->stream>>>(n0, r, net->red, net->ticket, net->scal, skip);
    RS_TRY(rs_check_launch(c));
    bf16 **A = net->act;
    RS_TRY(conv_forward(net, E0A, nullptr, nullptr, r, logk, A[E0A], skip));
    RS_TRY(conv_forward(net, E0B, A[E0A], nullptr, nullptr, nullptr, A[E0B], skip));
    RS_TRY(pool_forward(net, 1, A[E0B], net->pool[1], skip));
    RS_TRY(conv_forward(net, E1A, net->pool[1], nullptr, nullptr, nullptr, A[E1A], skip));
    RS_TRY(conv_forward(net, E1B, A[E1A], nullptr, nullptr, nullptr, A[E1B], skip));
    RS_TRY(pool_forward(net, 2, A[E1B], net->pool[2], skip));
    RS_TRY(conv_forward(net, E2A, net->pool[2], nullptr, nullptr, nullptr, A[E2A], skip));
    RS_TRY(conv_forward(net, E2B, A[E2A], nullptr, nullptr, nullptr, A[E2B], skip));
    RS_TRY(pool_forward(net, 3, A[E2B], net->pool[3], skip));
    RS_TRY(conv_forward(net, E3A, net->pool[3], nullptr, nullptr, nullptr, A[E3A], skip));
    RS_TRY(conv_forward(net, E3B, A[E3A], nullptr, nullptr, nullptr, A[E3B], skip));
    RS_TRY(conv_forward(net, D2A, A[E2B], A[E3B], nullptr, nullptr, A[D2A], skip));
    RS_TRY(conv_forward(net, D2B, A[D2A], nullptr, nullptr, nullptr, A[D2B], skip));
    RS_TRY(conv_forward(net, D1A, A[E1B], A[D2B], nullptr, nullptr, A[D1A], skip));
    RS_TRY(conv_forward(net, D1B, A[D1A], nullptr, nullptr, nullptr, A[D1B], skip));
    RS_TRY(conv_forward(net, D0A, A[E0B], A[D1B], nullptr, nullptr, A[D0A], skip));
    if (!keep) return conv_forward(net, D0B, A[D0A], nullptr, nullptr, nullptr, A[D0B], skip, out);
    RS_TRY(conv_forward(net, D0B, A[D0A], nullptr, nullptr, nullptr, A[D0B], skip));
    k_head<<<ew_grid(c, n0), 256, 0, c->stream>>>(n0, A[D0B], net->p + net->hoff, net->scal, net->out_scale, out,
                                                 net->flag, skip);
    return rs_check_launch(c);
}

// weight gradient of layer l for output gradient G (pre-activation), input as in the forward pass
static int conv_dw(rs_net *net, int l, const bf16 *X, const bf16 *U, const double *r, const double *logk,
                   const bf16 *G, float wscale)
{
    rs_ctx *c = net->ctx;
    const Level &L = net->lv[kLayers[l].level];
    const int grid = (int)nbricks(L);
    RsProfScope prof(c, RS_PROF_NET);
    switch (kLayers[l].mode) {
    case IN_FIRST:
        k_conv3_dw<16, IN_FIRST><<<grid, CONV_THREADS, dw_smem(16), c->stream>>>(L.nz, L.ny, L.nx, nullptr, nullptr, r,
                                                                                logk, net->scal + 1, G, net->partials);
        break;
    case IN_CATUP:
        k_conv3_dw<32, IN_CATUP><<<grid, CONV_THREADS, dw_smem(32), c->stream>>>(L.nz, L.ny, L.nx, X, U, nullptr,
                                                                                nullptr, nullptr, G, net->partials);
        break;
    default:
        k_conv3_dw<16, IN_PLAIN><<<grid, CONV_THREADS, dw_smem(16), c->stream>>>(L.nz, L.ny, L.nx, X, nullptr, nullptr,
                                                                                nullptr, nullptr, G, net->partials);
    }
    RS_TRY(rs_check_launch(c));
    const int cin = kLayers[l].cin, cinp = cin_pad(l);
    k_dw_reduce<<<ew_grid(c, 27 * 16 * cin + 16), 256, 0, c->stream>>>(grid, cin, cinp, net->partials, net->g,
                                                                        net->woff[l], net->boff[l], wscale);
    return rs_check_launch(c);
}

// data gradient: dX = conv(G, flipped transposed weights)
static int conv_dx(rs_net *net, int l, const bf16 *G, bf16 *dX)
{
    rs_ctx *c = net->ctx;
    const Level &L = net->lv[kLayers[l].level];
    const int grid = (int)nbricks(L);
    RsProfScope prof(c, RS_PROF_NET);
    if (kLayers[l].cin == 32)
        k_conv3<16, 32, IN_PLAIN><<<grid, CONV_THREADS, conv_smem(16, 32), c->stream>>>(
            L.nz, L.ny, L.nx, G, nullptr, nullptr, nullptr, nullptr, net->wb[l], nullptr, 0, dX, nullptr);
    else
        k_conv3<16, 16, IN_PLAIN><<<grid, CONV_THREADS, conv_smem(16, 16), c->stream>>>(
            L.nz, L.ny, L.nx, G, nullptr, nullptr, nullptr, nullptr, net->wb[l], nullptr, 0, dX, nullptr);
    return rs_check_launch(c);
}

static int relu_mask(rs_net *net, int lvl, const bf16 *g, const bf16 *y, bf16 *out)
{
    rs_ctx *c = net->ctx;
    const int64_t n = net->lv[lvl].nvox * 16;
    k_relu_mask<<<ew_grid(c, n), 256, 0, c->stream>>>(n, g, y, out);
    return rs_check_launch(c);
}

// backward of one conv+ReLU layer: g_post (gradient of the layer output) ->
// weight gradients and, if dX != null, the input gradient
static int layer_backward(rs_net *net, int l, const bf16 *g_post, bf16 *gpre, const bf16 *X, const bf16 *U,
                          const double *r, const double *logk, bf16 *dX, float wscale)
{
    const int lvl = kLayers[l].level;
    RS_TRY(relu_mask(net, lvl, g_post, net->act[l], gpre));
    RS_TRY(conv_dw(net, l, X, U, r, logk, gpre, wscale));
    if (dX) RS_TRY(conv_dx(net, l, gpre, dX));
    return RS_OK;
}

static int net_backward(rs_net *net, const double *r, const double *logk, float wscale)
{
    rs_ctx *c = net->ctx;
    bf16 **A = net->act;
    const int64_t n0 = net->lv[0].nvox;
    {
        RsProfScope prof(c, RS_PROF_NET);
        const int hb = std::min<int64_t>((n0 + 255) / 256, (int64_t)c->num_sms * 8);
        k_head_backward<<<hb, 256, 0, c->stream>>>(n0, A[D0B], net->p + net->hoff, net->scal, net->out_scale,
                                                   net->gout, net->g16a[0], net->headpart);
        k_head_reduce<<<1, 32, 0, c->stream>>>(hb, net->headpart, net->g, net->hoff);
        c->launches++;
        RS_TRY(rs_check_launch(c));
    }
    // decoder, fine to coarse
    const int dec_b[3] = {D0B, D1B, D2B}, dec_a[3] = {D0A, D1A, D2A};
    const int skip_src[3] = {E0B, E1B, E2B}, up_src[3] = {D1B, D2B, E3B};
    for (int lvl = 0; lvl < 3; ++lvl) {
        const int lb = dec_b[lvl], la = dec_a[lvl];
        RS_TRY(layer_backward(net, lb, net->g16a[lvl], net->g16b[lvl], A[la], nullptr, nullptr, nullptr,
                              net->g16a[lvl], wscale));
        RS_TRY(layer_backward(net, la, net->g16a[lvl], net->g16b[lvl], A[skip_src[lvl]], A[up_src[lvl]], nullptr,
                              nullptr, net->g32[lvl], wscale));
        const Level &C = net->lv[lvl + 1];
        k_up_backward<<<ew_grid(c, C.nvox * 16), 256, 0, c->stream>>>(C.nz, C.ny, C.nx, net->g32[lvl], net->g16a[lvl + 1]);
        RS_TRY(rs_check_launch(c));
    }
    // encoder, coarse to fine
    const int enc_b[4] = {E0B, E1B, E2B, E3B}, enc_a[4] = {E0A, E1A, E2A, E3A};
    for (int lvl = 3; lvl >= 0; --lvl) {
        const int lb = enc_b[lvl], la = enc_a[lvl];
        RS_TRY(layer_backward(net, lb, net->g16a[lvl], net->g16b[lvl], A[la], nullptr, nullptr, nullptr,
                              net->g16a[lvl], wscale));
        if (lvl == 0) {
            RS_TRY(layer_backward(net, la, net->g16a[0], net->g16b[0], nullptr, nullptr, r, logk, nullptr, wscale));
        } else {
            RS_TRY(layer_backward(net, la, net->g16a[lvl], net->g16b[lvl], net->pool[lvl], nullptr, nullptr, nullptr,
                                  net->g16a[lvl], wscale));
            const Level &F = net->lv[lvl - 1];
            k_pool_backward_add<<<ew_grid(c, F.nvox * 16), 256, 0, c->stream>>>(F.nz, F.ny, F.nx, net->g16a[lvl],
                                                                                 net->g32[lvl - 1], net->g16a[lvl - 1]);
            RS_TRY(rs_check_launch(c));
        }
    }
    return RS_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static int64_t layout(rs_net *net)
{
    int64_t off = 0;
    for (int l = 0; l < NET_NLAYERS; ++l) {
        net->woff[l] = off;
        off += 27 * 16 * kLayers[l].cin;
        net->boff[l] = off;
        off += 16;
    }
    net->hoff = off;
    return off + 17;
}

extern "C" int64_t rs_net_num_params(void)
{
    rs_net tmp;
    return layout(&tmp);
}

static void net_free(rs_net *net)
{
    if (!net) return;
    rs_ctx *c = net->ctx;
    free_workspace(net);
    rs_free(c, net->p);
    rs_free(c, net->g);
    rs_free(c, net->m);
    rs_free(c, net->v);
    for (int l = 0; l < NET_NLAYERS; ++l) { rs_free(c, net->wf[l]); rs_free(c, net->wb[l]); }
    rs_free(c, net->scal);
    rs_free(c, net->red);
    rs_free(c, net->ticket);
    rs_free(c, net->flag);
    delete net;
}

extern "C" int rs_net_create(rs_ctx *ctx, const float *params, int64_t nparams, float out_scale, rs_net **out)
{
    if (!ctx || !params || !out) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    rs_net *net = new rs_net();
    memset((void *)net, 0, sizeof(rs_net));
    net->ctx = ctx;
    net->out_scale = out_scale;
    net->nparams = layout(net);
    if (nparams != net->nparams) { delete net; return RS_ERR_SIZE_MISMATCH; }
    ensure_attrs();
    int st = RS_OK;
    const size_t pb = sizeof(float) * nparams;
    st = st ? st : rs_alloc(ctx, (void **)&net->p, pb);
    st = st ? st : rs_alloc(ctx, (void **)&net->g, pb);
    st = st ? st : rs_alloc(ctx, (void **)&net->m, pb);
    st = st ? st : rs_alloc(ctx, (void **)&net->v, pb);
    for (int l = 0; l < NET_NLAYERS && !st; ++l) {
        st = rs_alloc(ctx, (void **)&net->wf[l], sizeof(bf16) * 27 * 16 * cin_pad(l));
        if (!st) st = rs_alloc(ctx, (void **)&net->wb[l], sizeof(bf16) * 27 * 16 * cin_pad(l));
    }
    st = st ? st : rs_alloc(ctx, (void **)&net->scal, sizeof(double) * 16);
    st = st ? st : rs_alloc(ctx, (void **)&net->red, sizeof(double) * 2 * ctx->red_blocks);
    st = st ? st : rs_alloc(ctx, (void **)&net->ticket, sizeof(unsigned) * 4);
    st = st ? st : rs_alloc(ctx, (void **)&net->flag, sizeof(int) * 4);
    if (st) { net_free(net); return st; }
    cudaStream_t s = ctx->stream;
    RS_CUDA_TRY(cudaMemcpyAsync(net->p, params, pb, cudaMemcpyHostToDevice, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->g, 0, pb, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->m, 0, pb, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->v, 0, pb, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->scal, 0, sizeof(double) * 16, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->ticket, 0, sizeof(unsigned) * 4, s));
    RS_CUDA_TRY(cudaMemsetAsync(net->flag, 0, sizeof(int) * 4, s));
    st = pack_all(net);
    if (st) { net_free(net); return st; }
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    rs_ctx_retain(ctx);
    *out = net;
    return RS_OK;
}

extern "C" int rs_net_destroy(rs_net **net)
{
    if (!net || !*net) return RS_OK;
    rs_ctx *ctx = (*net)->ctx;
    cudaStreamSynchronize(ctx->stream);
    net_free(*net);
    *net = nullptr;
    rs_ctx_release(ctx);
    return RS_OK;
}

extern "C" int rs_net_get_params(const rs_net *net, float *out, int64_t n)
{
    if (!net || !out) return RS_ERR_INVALID_ARG;
    if (n != net->nparams) return RS_ERR_SIZE_MISMATCH;
    RS_CUDA_TRY(cudaMemcpyAsync(out, net->p, sizeof(float) * n, cudaMemcpyDeviceToHost, net->ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(net->ctx->stream));
    return RS_OK;
}

extern "C" int rs_net_get_grads(const rs_net *net, float *out, int64_t n)
{
    if (!net || !out) return RS_ERR_INVALID_ARG;
    if (n != net->nparams) return RS_ERR_SIZE_MISMATCH;
    RS_CUDA_TRY(cudaMemcpyAsync(out, net->g, sizeof(float) * n, cudaMemcpyDeviceToHost, net->ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(net->ctx->stream));
    return RS_OK;
}

extern "C" int rs_net_zero_grads(rs_net *net)
{
    if (!net) return RS_ERR_INVALID_ARG;
    RS_CUDA_TRY(cudaMemsetAsync(net->g, 0, sizeof(float) * net->nparams, net->ctx->stream));
    return RS_OK;
}

extern "C" int rs_net_forward(rs_net *net, int32_t nx, int32_t ny, int32_t nz, const double *r, const double *logk,
                              double *out)
{
    if (!net || !r || !logk || !out) return RS_ERR_INVALID_ARG;
    RS_TRY(ensure_workspace(net, nx, ny, nz));
    return net_forward(net, r, logk, out, nullptr);
}

extern "C" int rs_net_accumulate(rs_net *net, int32_t nx, int32_t ny, int32_t nz, const double *r, const double *logk,
                                 const double *e, double weight, double *loss_host)
{
    if (!net || !r || !logk || !e) return RS_ERR_INVALID_ARG;
    RS_TRY(ensure_workspace(net, nx, ny, nz));
    rs_ctx *c = net->ctx;
    const int64_t n0 = net->lv[0].nvox;
    RS_TRY(net_forward(net, r, logk, net->outb, nullptr, true));
    k_loss_sums<<<c->red_blocks, 256, 0, c->stream>>>(n0, net->outb, e, net->red, net->ticket, net->scal);
    k_loss_grad<<<ew_grid(c, n0), 256, 0, c->stream>>>(n0, net->outb, e, net->scal, weight, net->gout);
    c->launches++;
    RS_TRY(rs_check_launch(c));
    RS_TRY(net_backward(net, r, logk, 1.0f));
    if (loss_host) {
        RS_CUDA_TRY(cudaMemcpyAsync(c->h_pinned + 8, net->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        RS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        *loss_host = c->h_pinned[8];
    }
    return RS_OK;
}

extern "C" int rs_net_adam(rs_net *net, float lr, float beta1, float beta2, float eps)
{
    if (!net) return RS_ERR_INVALID_ARG;
    rs_ctx *c = net->ctx;
    net->step += 1;
    const float c1 = 1.f - powf(beta1, (float)net->step), c2 = 1.f - powf(beta2, (float)net->step);
    k_adam<<<ew_grid(c, net->nparams), 256, 0, c->stream>>>(net->nparams, net->p, net->g, net->m, net->v, lr, beta1,
                                                            beta2, eps, c1, c2);
    RS_TRY(rs_check_launch(c));
    return pack_all(net);
}

struct NetFileHeader {
    unsigned magic;
    int version;
    int64_t nparams;
    float out_scale;
    int step;
};

extern "C" int rs_net_save(const rs_net *net, const char *path)
{
    if (!net || !path) return RS_ERR_INVALID_ARG;
    std::vector<float> buf(3 * net->nparams);
    cudaStream_t s = net->ctx->stream;
    RS_CUDA_TRY(cudaMemcpyAsync(buf.data(), net->p, sizeof(float) * net->nparams, cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaMemcpyAsync(buf.data() + net->nparams, net->m, sizeof(float) * net->nparams, cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaMemcpyAsync(buf.data() + 2 * net->nparams, net->v, sizeof(float) * net->nparams, cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    FILE *f = fopen(path, "wb");
    if (!f) return RS_ERR_INVALID_ARG;
    NetFileHeader h = {NET_MAGIC, 1, net->nparams, net->out_scale, net->step};
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    return ok ? RS_OK : RS_ERR_INVALID_ARG;
}

extern "C" int rs_net_load(rs_ctx *ctx, const char *path, rs_net **out)
{
    if (!ctx || !path || !out) return RS_ERR_INVALID_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return RS_ERR_INVALID_ARG;
    NetFileHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || h.magic != NET_MAGIC || h.version != 1 || h.nparams != rs_net_num_params()) {
        fclose(f);
        return RS_ERR_INVALID_ARG;
    }
    std::vector<float> buf(3 * h.nparams);
    const bool ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return RS_ERR_INVALID_ARG;
    RS_TRY(rs_net_create(ctx, buf.data(), h.nparams, h.out_scale, out));
    rs_net *net = *out;
    RS_CUDA_TRY(cudaMemcpyAsync(net->m, buf.data() + h.nparams, sizeof(float) * h.nparams, cudaMemcpyHostToDevice, ctx->stream));
    RS_CUDA_TRY(cudaMemcpyAsync(net->v, buf.data() + 2 * h.nparams, sizeof(float) * h.nparams, cudaMemcpyHostToDevice, ctx->stream));
    RS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    net->step = h.step;
    return RS_OK;
}

// flag[1] = 1 (skip the fallback sweeps) unless the cycle runs and the
// network output had a non-finite value (flag[0])
__global__ void k_fallback_flag(int *flag, const int *skip)
{
    flag[1] = (skip && *(volatile const int *)skip) || flag[0] == 0;
}

static int rs_ilu_fallback(rs_pc *M, const double *rp, double *zp, int *flag, const int *skip)
{
    rs_ctx *c = M->ctx;
    k_fallback_flag<<<1, 1, 0, c->stream>>>(flag, skip);
    RS_TRY(rs_check_launch(c));
    return rs_ilu_apply(M->ilu, rp, zp, nullptr, flag + 1);
}

int rs_net_prepare(rs_pc *M, unsigned *gen, bool *same_ctx)
{
    rs_net *net = const_cast<rs_net *>(M->net);
    RS_TRY(ensure_workspace(net, M->nx, M->ny, M->nz));
    *gen = net->gen;
    *same_ctx = net->ctx == M->ctx;
    return RS_OK;
}

// pressure stage of the learned CPR preconditioner: zp = net(rp, log k); if
// any output is not finite, ILU(0) of the pressure matrix is applied instead
int rs_net_apply_pressure(rs_pc *M, const double *rp, double *zp, const int *skip)
{
    rs_net *net = const_cast<rs_net *>(M->net);
    rs_ctx *c = net->ctx;
    RS_TRY(ensure_workspace(net, M->nx, M->ny, M->nz));
    RS_CUDA_TRY(cudaMemsetAsync(net->flag, 0, sizeof(int), c->stream));
    RS_TRY(net_forward(net, rp, M->log_perm, zp, skip));
    // fallback: the ILU(0) sweeps run only when the flag is set; the flag is
    // inverted into net->flag[1] (1 = network output usable, skip the sweeps)
    RS_TRY(rs_ilu_fallback(M, rp, zp, net->flag, skip));
    return RS_OK;
}
