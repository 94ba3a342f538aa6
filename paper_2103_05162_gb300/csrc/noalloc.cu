// dbscan_sort_pairs_u64_noalloc: the radix sort entry point for callers that
// must not allocate device memory -- real-time loops, where a cudaMalloc can
// synchronise the device or fail at a moment the loop cannot absorb, and
// applications whose device memory is handed to a framework-level pool or
// budget that an allocation behind its back would overrun. Its scratch (the
// alternate key/value buffers, the digit histograms, the tile counters and
// the look-back status words) lives in one file-scope __device__ array
// instead of a workspace from cudaMalloc.
//
// Costs and rules of use:
//  * Every GPU that loads this library holds the array (NOALLOC_SCRATCH_BYTES,
//    about 14 MB) until the process exits.
//  * All calls on a device share the array and it keeps the last call's
//    contents; the call clears what must start at zero (histograms, tile
//    counters, status words, the error word) before sorting. Calls that
//    overlap on the GPU (different streams, or different host threads) race
//    on the array and give wrong results: serialise them.
//  * In host code the array's name stands for a host-side shadow, not for
//    device memory: the kernels get the device address, which the first call
//    in each CUDA context looks up with cudaGetSymbolAddress (with that
//    device current) and keeps for that context; make that first call before
//    any stream capture.
#include <cuda.h>

#include <map>
#include <mutex>
#include <utility>

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
constexpr size_t OFF_COUNTERS = OFF_HIST + align256(sizeof(uint32_t) * SORT_MAX_PASSES * SORT_RADIX);
constexpr size_t OFF_ERR = OFF_COUNTERS + align256(sizeof(uint32_t) * SORT_MAX_PASSES);
constexpr size_t OFF_STATUS = OFF_ERR + 256;
constexpr size_t STATUS_WORDS = (size_t)SORT_RADIX * NOALLOC_TILES * SORT_MAX_PASSES;  // digits x tiles x passes
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_STATUS + align256(sizeof(uint32_t) * STATUS_WORDS);

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
// device address of the array per (device, context id): a context created
// after cudaDeviceReset loads the module anew, possibly elsewhere, and has a
// new id, so a stale address is never reused
std::map<std::pair<int, unsigned long long>, unsigned char*> g_scratch_addr;

// the unique id of the calling thread's current context (0: none current, or
// the driver lacks cuCtxGetId); taken through the runtime's driver entry
// points, so the library needs no link to libcuda
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// device address of the scratch array in the current device's context
// (looked up once per context; looked up on every call if the context cannot
// be identified)
cudaError_t scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_mu);
    unsigned long long id = current_context_id();
    if (id != 0) {
        auto it = g_scratch_addr.find(std::make_pair(dev, id));
        if (it != g_scratch_addr.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's primary context current if needed
    if (e != cudaSuccess) return e;
    id = current_context_id();
    if (id != 0) g_scratch_addr[std::make_pair(dev, id)] = static_cast<unsigned char*>(p);
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace gbd

using namespace gbd;

extern "C" dbscan_status dbscan_sort_pairs_u64_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                                       dbscan_stream stream)
{
    clear_error();
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
