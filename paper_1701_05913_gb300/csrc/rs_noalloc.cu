// A multi-dot product h = V^T w that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, callers that hand the library memory from their own pools
// and forbid further device allocations, or embedded hosts with a fixed
// device-memory budget.  This entry point serves them: its scratch (the
// per-block partial sums of the two-level reduction and the last-block
// ticket) lives in a file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits.
//
// Limits: at most RS_NOALLOC_MAX_COLS columns (larger k is rejected), and
// at most RS_NOALLOC_MAX_BLOCKS blocks in the reduction grid.
//
// The array is shared by every call: calls that overlap on the GPU (on two
// streams, or from two host threads) race on it.  The ticket is cleared with
// a memset on the caller's stream before every launch, so a call never
// depends on what an earlier call left behind.
//
// In host code the name of a __device__ array is only a host-side stand-in;
// the kernel must be given the device address, which cudaGetSymbolAddress
// returns.  The first call on each device looks that address up (with that
// device current) and caches it for the life of the process; make that
// first call before capturing a stream into a graph.  The device is the one
// the caller's stream belongs to.  A reset of that device (cudaDeviceReset)
// unloads the array, so the cached address is stale afterwards: restart the
// process before calling again.
#include <mutex>

#include "rs_internal.cuh"

#define RS_NOALLOC_MAX_COLS 64
#define RS_NOALLOC_MAX_BLOCKS 1024
#define RS_NOALLOC_THREADS 256
#define RS_NOALLOC_MAX_DEVICES 64
#define RS_NOALLOC_CHUNK 8

static __device__ __align__(256) double g_noalloc_partials[RS_NOALLOC_MAX_BLOCKS * RS_NOALLOC_MAX_COLS];
static __device__ __align__(256) unsigned g_noalloc_ticket[64];

struct NoallocSlot {
    bool ready;
    double *partials;
    unsigned *ticket;
    int blocks;
};

static NoallocSlot g_slots[RS_NOALLOC_MAX_DEVICES];
static std::mutex g_slots_mu;

// Looks up the device addresses of the scratch arrays for device dev (the
// current device).
static int noalloc_setup(int dev, NoallocSlot **out)
{
    if (dev < 0 || dev >= RS_NOALLOC_MAX_DEVICES) return RS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_slots_mu);
    NoallocSlot &s = g_slots[dev];
    if (!s.ready) {
        void *p = nullptr, *t = nullptr;
        RS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partials));
        RS_CUDA_TRY(cudaGetSymbolAddress(&t, g_noalloc_ticket));
        int sms = 0;
        RS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        s.partials = (double *)p;
        s.ticket = (unsigned *)t;
        s.blocks = sms * 2 < RS_NOALLOC_MAX_BLOCKS ? sms * 2 : RS_NOALLOC_MAX_BLOCKS;
        s.ready = true;
    }
    *out = &s;
    return RS_OK;
}

// Each block forms partial sums of k dot products over a grid-strided set of
// rows (columns in chunks of 8 held in registers), writes them to the
// scratch, and the last block to finish adds the partials in block order.
__global__ void __launch_bounds__(RS_NOALLOC_THREADS)
k_mdot_noalloc(int n, int ld, int k, const double *__restrict__ V, const double *__restrict__ w,
               double *__restrict__ partials, unsigned *ticket, double *__restrict__ h)
{
    __shared__ double sm[RS_NOALLOC_THREADS / 32][RS_NOALLOC_CHUNK];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < k; j0 += RS_NOALLOC_CHUNK) {
        double acc[RS_NOALLOC_CHUNK];
#pragma unroll
        for (int j = 0; j < RS_NOALLOC_CHUNK; ++j) acc[j] = 0.0;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            const double wr = w[r];
#pragma unroll
            for (int j = 0; j < RS_NOALLOC_CHUNK; ++j)
                if (j0 + j < k) acc[j] = fma(V[(size_t)(j0 + j) * ld + r], wr, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < RS_NOALLOC_CHUNK; ++j) {
            const double v = warp_sum(acc[j]);
            if (lane == 0) sm[warp][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < RS_NOALLOC_CHUNK && j0 + threadIdx.x < k) {
            double s = 0.0;
            for (int q = 0; q < RS_NOALLOC_THREADS / 32; ++q) s += sm[q][threadIdx.x];
            partials[(size_t)blockIdx.x * RS_NOALLOC_MAX_COLS + j0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = warp; j < k; j += RS_NOALLOC_THREADS / 32) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partials + (size_t)b * RS_NOALLOC_MAX_COLS + j);
        s = warp_sum(s);
        if (lane == 0) h[j] = s;
    }
}

extern "C" int rs_vec_mdot_noalloc(const double *V, int32_t ld, int32_t n, int32_t k, const double *w,
                                   double *h, void *cuda_stream)
{
    if (k < 1 || k > RS_NOALLOC_MAX_COLS) return RS_ERR_INVALID_ARG;
    if (n < 0 || ld < n || (n > 0 && (!V || !w)) || !h) return RS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the device of the caller's stream (the current device for the
    // default streams), made current for the call
    int dev = 0, cur = 0;
    RS_CUDA_TRY(cudaGetDevice(&cur));
    RS_CUDA_TRY(cudaStreamGetDevice(st, &dev));
    if (dev != cur) RS_CUDA_TRY(cudaSetDevice(dev));
    NoallocSlot *s = nullptr;
    int rc = noalloc_setup(dev, &s);
    if (rc == RS_OK) {
        int blocks = (n + RS_NOALLOC_THREADS - 1) / RS_NOALLOC_THREADS;
        if (blocks > s->blocks) blocks = s->blocks;
        if (blocks < 1) blocks = 1;
        if (cudaMemsetAsync(s->ticket, 0, sizeof(unsigned), st) != cudaSuccess) {
            rc = RS_ERR_CUDA;
        } else {
            k_mdot_noalloc<<<blocks, RS_NOALLOC_THREADS, 0, st>>>(n, ld, k, V, w, s->partials, s->ticket, h);
            if (cudaGetLastError() != cudaSuccess) rc = RS_ERR_CUDA;
        }
    }
    if (dev != cur) cudaSetDevice(cur);
    return rc;
}
