// dbscan_sort_pairs_u64_noalloc: the radix sort entry point for callers that
// must not allocate device memory -- code running while a CUDA graph is being
// captured, real-time loops where a cudaMalloc could stall or fail at the
// wrong moment, and applications whose device memory is owned by a
// framework-level pool. Its scratch (the alternate key/value buffers, the
// digit histograms, the tile counters and the look-back status words) lives in
// one file-scope __device__ array instead of a workspace from cudaMalloc.
//
// Costs and rules of use:
//  * Every GPU that loads this library holds the array (NOALLOC_SCRATCH_BYTES,
//    about 14 MB) until the process exits.
//  * All calls on a device share the array and it keeps the last call's
//    contents; the call clears what must start at zero (histograms, tile
//    counters, status words, the error word) before sorting. Calls that
//    overlap on the GPU (different streams, or different host threads) race
//    on the array and give wrong results: serialise them.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current); make that first call
//    before any stream capture.
#include <mutex>

#include "capi_internal.h"
#include "internal.cuh"

namespace gbd {
namespace {

constexpr int64_t NOALLOC_MAX_PAIRS = DBSCAN_SORT_NOALLOC_MAX_PAIRS;
constexpr int64_t NOALLOC_TILE_KEYS = SORT_TILE_KEYS;  // keys per look-back tile of the onesweep kernel
constexpr int64_t NOALLOC_TILES = (NOALLOC_MAX_PAIRS + NOALLOC_TILE_KEYS - 1) / NOALLOC_TILE_KEYS;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_VALS = OFF_KEYS + align256(sizeof(uint64_t) * NOALLOC_MAX_PAIRS);
constexpr size_t OFF_HIST = OFF_VALS + align256(sizeof(uint32_t) * NOALLOC_MAX_PAIRS);
constexpr size_t OFF_COUNTERS = OFF_HIST + align256(sizeof(uint32_t) * 8 * 256);
constexpr size_t OFF_ERR = OFF_COUNTERS + align256(sizeof(uint32_t) * 8);
constexpr size_t OFF_STATUS = OFF_ERR + 256;
constexpr size_t STATUS_WORDS = (size_t)256 * NOALLOC_TILES * 8;  // 256 digits x tiles x 8 passes
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_STATUS + align256(sizeof(uint32_t) * STATUS_WORDS);

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gbd

using namespace gbd;

extern "C" dbscan_status dbscan_sort_pairs_u64_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                                       dbscan_stream stream)
{
    if (n < 0 || n > NOALLOC_MAX_PAIRS)
        return set_error(DBSCAN_ERR_INVALID_ARG, "n = %lld is outside [0, %lld], the capacity of the static scratch",
                         (long long)n, (long long)NOALLOC_MAX_PAIRS);
    if (key_bits < 0 || key_bits > 64) return set_error(DBSCAN_ERR_INVALID_ARG, "key_bits must be in [0, 64]");
    if (n > 0 && (!keys || !values)) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    if (n <= 1 || key_bits == 0) return DBSCAN_OK;
    if (sort_status_words(n, 8, key_bits) > STATUS_WORDS)
        return set_error(DBSCAN_ERR_INVALID_ARG, "sort status does not fit the static scratch");
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static sort scratch)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SortBuffers sb;
    sb.keys_alt = base + OFF_KEYS;
    sb.vals_alt = reinterpret_cast<uint32_t*>(base + OFF_VALS);
    sb.hist = reinterpret_cast<uint32_t*>(base + OFF_HIST);
    sb.counters = reinterpret_cast<uint32_t*>(base + OFF_COUNTERS);
    sb.err = reinterpret_cast<uint32_t*>(base + OFF_ERR);
    sb.status = reinterpret_cast<uint32_t*>(base + OFF_STATUS);
    // histograms, counters and status words are cleared by the sort itself
    if ((e = cudaMemsetAsync(sb.err, 0, sizeof(uint32_t), s)) != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    bool in_alt = false;
    if ((e = sort_pairs_u64(keys, values, n, key_bits, sb, s, &in_alt)) != cudaSuccess)
        return cuda_error(e, "radix sort");
    if (in_alt) {
        if ((e = cudaMemcpyAsync(keys, sb.keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
        if ((e = cudaMemcpyAsync(values, sb.vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
    }
    uint32_t err = 0;
    if ((e = cudaMemcpyAsync(&err, sb.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_error(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    if (err) return set_error(DBSCAN_ERR_DEVICE_TIMEOUT, "radix sort look-back gave up (bits 0x%x)", err);
    return DBSCAN_OK;
}
