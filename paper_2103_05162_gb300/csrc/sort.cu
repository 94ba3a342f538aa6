// Stable LSD radix sort of (key, value) pairs, onesweep style: one kernel
// builds the digit histograms of every pass in a single read of the keys;
// then each pass (one SORT_DIGIT_BITS-bit digit) is a single kernel in which a tile ranks its keys in
// shared memory, publishes its per-digit counts, finds its global offsets by
// decoupled look-back over the tiles before it, and scatters.
//
// Forward progress: tiles take their index from an atomic counter when they
// start, so a tile only ever waits for tiles that are already running. Every
// wait is bounded (SPIN_LIMIT spins, or the test hook's limit); a tile whose
// wait runs out sets ERR_SORT_TIMEOUT in the device error word, publishes no
// prefix and scatters nothing (its output slots keep what they held), so a
// timed-out sort never writes outside its buffers; later stages of the
// pipeline read the error word and stop.
//
// This orders Morton codes / grid-cell keys (the space-filling-curve order of
// Sec. 4.1 and the cell grouping of Sec. 4.2). A keys-only form sorts 64-bit
// words that carry the key above the point's index (key << b | index) on
// bits [b, b + key bits): a third less traffic per pass than separate
// 64-bit keys and 32-bit values, in the same stable order.
#include <atomic>

#include "internal.cuh"

namespace gbd {

namespace {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int DIGIT_BITS = SORT_DIGIT_BITS;
constexpr int RADIX = SORT_RADIX;
constexpr uint32_t DMASK = RADIX - 1;
// digits per thread in the per-digit steps: thread t owns digits
// [t * DPT, t * DPT + DPT), whose status words it publishes in one store
constexpr int DPT = RADIX / THREADS;
static_assert(DPT == 1 || DPT == 2, "one or two digits per thread");
constexpr int ITEMS = 16;  // keys per thread (8 was measured slower despite 3 blocks per SM)
constexpr int TILE_ITEMS = THREADS * ITEMS;
static_assert(TILE_ITEMS == SORT_TILE_KEYS, "tile size shared with the static-scratch entry point");
constexpr uint32_t FLAG_AGG = 1u << 30;
constexpr uint32_t FLAG_PRE = 2u << 30;
constexpr uint32_t VAL_MASK = (1u << 30) - 1;

// The passes a launch of the sort takes part in, decided once per block (a
// word another block sets during the launch must not split the block):
// 0 if the sort is gated off or aborted, else the passes the keys need.
__device__ __forceinline__ int sort_block_passes(const SortCtl& c, int host_passes, int* s_dec)
{
    if (threadIdx.x == 0) {
        int p = host_passes;
        if (c.gate && ld_relaxed(c.gate) != c.gate_val) p = 0;
        if (c.abort && ld_relaxed(c.abort) != 0) p = 0;
        if (p && c.key_bits) {
            const int d = sort_passes((int)ld_relaxed(c.key_bits));
            p = d < 1 ? 1 : (d < host_passes ? d : host_passes);
        }
        *s_dec = p;
    }
    __syncthreads();
    return *s_dec;
}

template <typename K>
__global__ void __launch_bounds__(THREADS) k_hist(const K* __restrict__ k0, const K* __restrict__ k1, int64_t n,
                                                  int shift0, int passes, SortCtl ctl, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t sh[SORT_MAX_PASSES * RADIX];
    __shared__ int s_dec;
    const int pd = sort_block_passes(ctl, passes, &s_dec);
    if (pd == 0) return;
    const K* __restrict__ keys = sort_dev_input_alt(passes, pd) ? k1 : k0;
    for (int i = threadIdx.x; i < pd * RADIX; i += THREADS) sh[i] = 0;
    __syncthreads();
    // four keys per step: four independent loads in flight per thread
    const int64_t stride = (int64_t)gridDim.x * THREADS;
    int64_t i = blockIdx.x * (int64_t)THREADS + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        K k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = keys[i + u * stride];
        for (int p = 0; p < pd; ++p) {
            const int sh_p = shift0 + DIGIT_BITS * p;
#pragma unroll
            for (int u = 0; u < 4; ++u) atomicAdd(&sh[p * RADIX + (uint32_t)((k[u] >> sh_p) & DMASK)], 1u);
        }
    }
    for (; i < n; i += stride) {
        const K k = keys[i];
        for (int p = 0; p < pd; ++p) atomicAdd(&sh[p * RADIX + (uint32_t)((k >> (shift0 + DIGIT_BITS * p)) & DMASK)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pd * RADIX; i += THREADS) {
        uint32_t v = sh[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// exclusive scan of one value per thread over the 256 threads of the block
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < WARPS ? s_warp[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < WARPS) s_warp[lane] = wi - w;
    }
    __syncthreads();
    uint32_t r = inc - x + s_warp[warp];
    __syncthreads();
    return r;
}

// A tile's status for the DPT digits of one thread: one relaxed store or
// load (both halves of a 64-bit word always carry the same flag).
__device__ __forceinline__ void st_status(uint32_t* p, const uint32_t (&w)[DPT])
{
    if constexpr (DPT == 1) st_relaxed(p, w[0]);
    else st_relaxed64(reinterpret_cast<uint64_t*>(p), (uint64_t)w[0] | ((uint64_t)w[DPT - 1] << 32));
}
__device__ __forceinline__ void ld_status(const uint32_t* p, uint32_t (&w)[DPT])
{
    if constexpr (DPT == 1) {
        w[0] = ld_relaxed(p);
    } else {
        const uint64_t v = ld_relaxed64(reinterpret_cast<const uint64_t*>(p));
        w[0] = (uint32_t)v;
        w[DPT - 1] = (uint32_t)(v >> 32);
    }
}

// (three blocks per SM with values: the compiler then keeps every key, value
// and rank in 80 registers without spilling, instead of taking 128 and
// fitting two; four for keys only)
//
// Pass `pass` of `passes`: reads buffer 0 and writes buffer 1 on even passes
// (the reverse on odd ones), or, under device control, as the passes the keys
// need decide (sort_dev_input_alt); passes beyond those do nothing.
template <typename K, bool VALS>
__global__ void __launch_bounds__(THREADS, VALS ? 3 : 4)
    k_onesweep(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, int shift0, int pass, int passes, SortCtl ctl,
               const uint32_t* __restrict__ hist, uint32_t* __restrict__ status, uint32_t* tile_counter,
               uint32_t* err, int wait_limit, int stall_first_tile)
{
    extern __shared__ __align__(16) unsigned char smem[];
    K* keys_s = reinterpret_cast<K*>(smem);
    uint32_t* vals_s = reinterpret_cast<uint32_t*>(smem + TILE_ITEMS * sizeof(K));
    uint32_t* whist = reinterpret_cast<uint32_t*>(smem);  // [WARPS][RADIX], aliases keys_s
    __shared__ uint32_t s_tile;
    __shared__ __align__(8) uint32_t s_excl[RADIX];
    __shared__ uint32_t s_gofs[RADIX];
    __shared__ uint32_t s_warp[WARPS];
    __shared__ int s_dec;

    const int pd = sort_block_passes(ctl, passes, &s_dec);
    if (pass >= pd) return;
    const int sel = (sort_dev_input_alt(passes, pd) ? 1 : 0) ^ (pass & 1);
    const K* __restrict__ kin = sel ? k1 : k0;
    const uint32_t* __restrict__ vin = sel ? v1 : v0;
    K* __restrict__ kout = sel ? k0 : k1;
    uint32_t* __restrict__ vout = sel ? v0 : v1;
    const int shift = shift0 + DIGIT_BITS * pass;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < WARPS * RADIX; i += THREADS) whist[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * TILE_ITEMS;
    const int64_t wbase = base + warp * (32 * ITEMS);

    K k[ITEMS];
    uint32_t v[ITEMS];
    uint32_t r[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            k[i] = kin[idx];
            v[i] = VALS ? vin[idx] : 0u;
        } else {
            k[i] = ~K(0);
            v[i] = 0;
        }
    }
    // rank each key among equal digits of its warp, in input order
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool valid = (wbase + i * 32 + lane) < n;
        const uint32_t d = (uint32_t)(k[i] >> shift) & DMASK;
        uint32_t peers = __ballot_sync(FULL, valid);
#pragma unroll
        for (int b = 0; b < DIGIT_BITS; ++b) {
            const uint32_t bit = (d >> b) & 1u;
            const uint32_t m = __ballot_sync(FULL, bit);
            peers &= bit ? m : ~m;
        }
        uint32_t* h = &whist[warp * RADIX + d];
        const uint32_t prior = valid ? *h : 0u;
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) *h = prior + __popc(peers);
        __syncwarp();
        r[i] = prior + __popc(peers & lt);
    }
    __syncthreads();

    // thread tid owns digits tid * DPT + q: per-warp exclusive offsets and
    // the tile counts
    uint32_t total[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int dg = tid * DPT + q;
        uint32_t t = 0;
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = whist[w * RADIX + dg];
            whist[w * RADIX + dg] = t;
            t += c;
        }
        total[q] = t;
    }
    uint32_t* st = status + (size_t)tile * RADIX + tid * DPT;
    const bool withhold = stall_first_tile && tile == 0;  // test hook: nothing published
    uint32_t word[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) word[q] = (tile == 0 ? FLAG_PRE : FLAG_AGG) | total[q];
    if (!withhold) st_status(st, word);

    // exclusive scans over the digits in order: the tile's own offsets and
    // the pass's digit bases
    uint32_t tsum = 0, hsum = 0, hv[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        hv[q] = hist[tid * DPT + q];
        tsum += total[q];
        hsum += hv[q];
    }
    uint32_t excl = block_excl_scan(tsum, s_warp);
    uint32_t dbase = block_excl_scan(hsum, s_warp);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        s_excl[tid * DPT + q] = excl;
        excl += total[q];
    }

    uint32_t prefix[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) prefix[q] = 0;
    bool gave_up = false;
    if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        int spins = 0;
        while (j >= 0) {
            uint32_t sw[DPT];
            ld_status(status + (size_t)j * RADIX + tid * DPT, sw);
            const uint32_t flag = sw[0] & ~VAL_MASK;
            if (flag == 0u) {
                if (++spins > wait_limit) {
                    atomicOr(err, ERR_SORT_TIMEOUT);
                    gave_up = true;
                    break;
                }
                __nanosleep(32);
                continue;
            }
#pragma unroll
            for (int q = 0; q < DPT; ++q) prefix[q] += sw[q] & VAL_MASK;
            if (flag == FLAG_PRE) break;
            --j;
        }
        // a tile whose wait ran out publishes no prefix: later tiles look
        // past it to the aggregates before it (or run out themselves)
        if (!gave_up) {
#pragma unroll
            for (int q = 0; q < DPT; ++q) word[q] = FLAG_PRE | ((prefix[q] + total[q]) & VAL_MASK);
            st_status(st, word);
        }
    }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        s_gofs[tid * DPT + q] = dbase + prefix[q];
        dbase += hv[q];
    }
    // any digit without its offset: the tile's positions are unknown, so it
    // writes nothing
    if (__syncthreads_or(gave_up)) return;

    // tile-local positions (sorted by digit, stable), then stage in shared memory
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = (uint32_t)(k[i] >> shift) & DMASK;
        r[i] += s_excl[d] + whist[warp * RADIX + d];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if ((wbase + i * 32 + lane) < n) {
            keys_s[r[i]] = k[i];
            if (VALS) vals_s[r[i]] = v[i];
        }
    }
    __syncthreads();
    const int64_t rem = n - base;
    const int cnt = rem < TILE_ITEMS ? (int)rem : TILE_ITEMS;
    for (int j = tid; j < cnt; j += THREADS) {
        const K kk = keys_s[j];
        const uint32_t d = (uint32_t)(kk >> shift) & DMASK;
        const uint32_t o = s_gofs[d] + (uint32_t)j - s_excl[d];
        kout[o] = kk;
        if (VALS) vout[o] = vals_s[j];
    }
}

std::atomic<int> g_wait_limit{SPIN_LIMIT};
std::atomic<int> g_stall_first_tile{0};

// sorts by bits [shift0, shift0 + bits) of the keys; vals null: keys only.
// Under device control (sb.ctl.key_bits) `bits` is an upper bound and the
// keys must have been written to the buffer sort_dev_input_alt names; the
// result lands where `bits` would leave it either way (*in_alt).
template <typename K>
cudaError_t sort_pairs(K* keys, uint32_t* vals, int64_t n, int shift0, int bits, const SortBuffers& sb,
                       cudaStream_t s, bool* in_alt)
{
    *in_alt = false;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int passes = sort_passes(bits);
    const int64_t tiles = (n + TILE_ITEMS - 1) / TILE_ITEMS;
    cudaError_t e;
    if ((e = cudaMemsetAsync(sb.hist, 0, sizeof(uint32_t) * RADIX * passes, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sb.counters, 0, sizeof(uint32_t) * passes, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sb.status, 0, sizeof(uint32_t) * RADIX * (size_t)tiles * passes, s)) != cudaSuccess)
        return e;
    K* k_alt = static_cast<K*>(sb.keys_alt);
    // once a wait has run out, no later pass may run: its input holds slots
    // the timed-out tiles never wrote, and ranks computed from them could
    // point past the end of the output
    SortCtl ctl = sb.ctl;
    if (!ctl.abort) ctl.abort = sb.err;
    const int hist_blocks = (int)(tiles < 1216 ? tiles : 1216);
    k_hist<K><<<hist_blocks, THREADS, 0, s>>>(keys, k_alt, n, shift0, passes, ctl, sb.hist);
    note_launches(1);
    const bool with_vals = vals != nullptr;
    const size_t smem = TILE_ITEMS * (sizeof(K) + (with_vals ? sizeof(uint32_t) : 0));
    static_assert(TILE_ITEMS * sizeof(uint32_t) >= WARPS * RADIX * sizeof(uint32_t), "histograms alias keys");
    if ((e = cudaFuncSetAttribute(with_vals ? k_onesweep<K, true> : k_onesweep<K, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    const int limit = g_wait_limit.load(std::memory_order_relaxed);
    const int stall = g_stall_first_tile.load(std::memory_order_relaxed);
    for (int p = 0; p < passes; ++p) {
        if (with_vals)
            k_onesweep<K, true><<<(unsigned)tiles, THREADS, smem, s>>>(
                keys, vals, k_alt, sb.vals_alt, n, shift0, p, passes, ctl, sb.hist + RADIX * p,
                sb.status + (size_t)RADIX * tiles * p, sb.counters + p, sb.err, limit, stall);
        else
            k_onesweep<K, false><<<(unsigned)tiles, THREADS, smem, s>>>(
                keys, nullptr, k_alt, nullptr, n, shift0, p, passes, ctl, sb.hist + RADIX * p,
                sb.status + (size_t)RADIX * tiles * p, sb.counters + p, sb.err, limit, stall);
        note_launches(1);
    }
    *in_alt = (passes & 1) != 0;
    return cudaGetLastError();
}

}  // namespace

int64_t sort_tiles(int64_t n, int key_bytes)
{
    (void)key_bytes;
    return (n + TILE_ITEMS - 1) / TILE_ITEMS;
}

size_t sort_status_words(int64_t n, int key_bytes, int bits)
{
    const int passes = sort_passes(bits);
    return (size_t)RADIX * (size_t)sort_tiles(n, key_bytes) * (size_t)(passes > 0 ? passes : 1);
}

void sort_set_test_hooks(int64_t wait_limit, int stall_first_tile)
{
    g_wait_limit.store(wait_limit < 0 ? SPIN_LIMIT : (int)(wait_limit > SPIN_LIMIT ? SPIN_LIMIT : wait_limit),
                       std::memory_order_relaxed);
    g_stall_first_tile.store(stall_first_tile ? 1 : 0, std::memory_order_relaxed);
}

cudaError_t sort_pairs_u32(uint32_t* keys, uint32_t* vals, int64_t n, int bits, const SortBuffers& sb,
                           cudaStream_t s, bool* in_alt)
{
    return sort_pairs<uint32_t>(keys, vals, n, 0, bits, sb, s, in_alt);
}

cudaError_t sort_pairs_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, const SortBuffers& sb,
                           cudaStream_t s, bool* in_alt)
{
    return sort_pairs<uint64_t>(keys, vals, n, 0, bits, sb, s, in_alt);
}

cudaError_t sort_keys_u64(uint64_t* keys, int64_t n, int shift0, int bits, const SortBuffers& sb, cudaStream_t s,
                          bool* in_alt)
{
    return sort_pairs<uint64_t>(keys, nullptr, n, shift0, bits, sb, s, in_alt);
}

}  // namespace gbd
