// Device-wide scans of int32 arrays (sum or max), reduce-then-scan: block
// reductions, one block scanning the block totals, then block scans with the
// carried-in total. No kernel waits on another block.
#include "internal.cuh"

namespace gbd {

namespace {

constexpr int THREADS = 256;
constexpr int ITEMS = 16;
constexpr int CHUNK = THREADS * ITEMS;

__device__ __forceinline__ int32_t op_apply(int32_t a, int32_t b, int op) { return op == SCAN_ADD ? a + b : max(a, b); }
__device__ __forceinline__ int32_t op_identity(int op) { return op == SCAN_ADD ? 0 : INT32_MIN; }
__device__ __forceinline__ int pad(int j) { return j + (j >> 5); }

// inclusive block scan of one value per thread; returns inclusive, *total = block total
__device__ __forceinline__ int32_t block_scan_incl(int32_t x, int op, int32_t* s_warp, int32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc = op_apply(y, inc, op);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < THREADS / 32 ? s_warp[lane] : op_identity(op);
        int32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi = op_apply(y, wi, op);
        }
        if (lane < THREADS / 32) s_warp[lane] = wi;  // inclusive over warps
    }
    __syncthreads();
    int32_t r = warp > 0 ? op_apply(s_warp[warp - 1], inc, op) : inc;
    *total = s_warp[THREADS / 32 - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(THREADS) k_reduce(const int32_t* __restrict__ in, int64_t n, int op,
                                                    int32_t* __restrict__ partial)
{
    __shared__ int32_t s_warp[THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    int32_t acc = op_identity(op);
    for (int i = 0; i < ITEMS; ++i) {
        int64_t idx = base + i * THREADS + threadIdx.x;
        if (idx < n) acc = op_apply(acc, in[idx], op);
    }
    int32_t total;
    block_scan_incl(acc, op, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// exclusive scan of the block totals in place (one block, loops over chunks)
__global__ void __launch_bounds__(THREADS) k_scan_partials(int32_t* partial, int64_t nb, int op)
{
    __shared__ int32_t s_warp[THREADS / 32];
    __shared__ int32_t s_inc[THREADS];
    int32_t carry = op_identity(op);
    for (int64_t b = 0; b < nb; b += THREADS) {
        const int64_t idx = b + threadIdx.x;
        const int32_t x = idx < nb ? partial[idx] : op_identity(op);
        int32_t total;
        const int32_t inc = block_scan_incl(x, op, s_warp, &total);
        s_inc[threadIdx.x] = inc;
        __syncthreads();
        const int32_t ex = threadIdx.x > 0 ? s_inc[threadIdx.x - 1] : op_identity(op);
        if (idx < nb) partial[idx] = op_apply(carry, ex, op);
        carry = op_apply(carry, total, op);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(THREADS) k_scan_apply(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                        int64_t n, int op, int inclusive,
                                                        const int32_t* __restrict__ partial)
{
    // padded by one word per 32 so that per-thread runs of ITEMS words do not
    // fall into the same banks
    __shared__ int32_t s_data[CHUNK + CHUNK / 32];
    __shared__ int32_t s_warp[THREADS / 32];
    __shared__ int32_t s_inc[THREADS];
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    // coalesced load into shared memory
    for (int i = 0; i < ITEMS; ++i) {
        const int64_t idx = base + i * THREADS + threadIdx.x;
        s_data[pad(i * THREADS + threadIdx.x)] = idx < n ? in[idx] : op_identity(op);
    }
    __syncthreads();
    // each thread owns ITEMS consecutive values
    int32_t v[ITEMS];
    int32_t acc = op_identity(op);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        v[i] = s_data[pad(threadIdx.x * ITEMS + i)];
        acc = op_apply(acc, v[i], op);
    }
    int32_t total;
    const int32_t inc = block_scan_incl(acc, op, s_warp, &total);
    s_inc[threadIdx.x] = inc;
    __syncthreads();
    const int32_t prev = threadIdx.x > 0 ? s_inc[threadIdx.x - 1] : op_identity(op);
    int32_t x = op_apply(partial[blockIdx.x], prev, op);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int32_t nx = op_apply(x, v[i], op);
        s_data[pad(threadIdx.x * ITEMS + i)] = inclusive ? nx : x;
        x = nx;
    }
    __syncthreads();
    for (int i = 0; i < ITEMS; ++i) {
        const int64_t idx = base + i * THREADS + threadIdx.x;
        if (idx < n) out[idx] = s_data[pad(i * THREADS + threadIdx.x)];
    }
}

}  // namespace

size_t scan_temp_words(int64_t n) { return (size_t)((n + CHUNK - 1) / CHUNK) + 1; }

cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t n, ScanOp op, bool inclusive, int32_t* temp,
                     cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + CHUNK - 1) / CHUNK;
    k_reduce<<<(unsigned)nb, THREADS, 0, s>>>(in, n, (int)op, temp);
    k_scan_partials<<<1, THREADS, 0, s>>>(temp, nb, (int)op);
    k_scan_apply<<<(unsigned)nb, THREADS, 0, s>>>(in, out, n, (int)op, inclusive ? 1 : 0, temp);
    note_launches(3);
    return cudaGetLastError();
}

}  // namespace gbd
