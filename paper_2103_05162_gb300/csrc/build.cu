// Index construction: bounds, space-filling-curve keys, gather into sorted
// order, DenseBox cell classification and leaf layout, Karras LBVH topology
// and the atomic bottom-up refit (Sec. 4.1, 4.2).
#include "build.cuh"

namespace gbd {

// ---------------------------------------------------------------------------
// K1: exact fp32 bounding box of the points, plus a flag for NaN/Inf.
// Each thread strides over the flat coordinate array with a stride that is a
// multiple of D, so it always sees the same axis.
// ---------------------------------------------------------------------------
template <int D, int BT = bounds_threads<D>()>
__global__ void __launch_bounds__(BT) k_bounds(const float* __restrict__ pts, int64_t n,
                                               uint32_t* __restrict__ ctrl)
{
    __shared__ uint32_t s_lo[D], s_hi[D];
    __shared__ int s_bad;
    if (threadIdx.x < D) { s_lo[threadIdx.x] = 0xffffffffu; s_hi[threadIdx.x] = 0u; }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const int64_t total = n * D;
    const int64_t stride = (int64_t)gridDim.x * BT;
    const int axis = threadIdx.x % D;
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < total; i += stride) {
        float v = __ldcs(pts + i);
        bad |= !isfinite(v);
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    if (lo <= hi) {
        atomicMin(&s_lo[axis], f2ord(lo));
        atomicMax(&s_hi[axis], f2ord(hi));
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (threadIdx.x < D) {
        atomicMin(&ctrl[CTRL_LO + threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&ctrl[CTRL_HI + threadIdx.x], s_hi[threadIdx.x]);
    }
    if (threadIdx.x == 0 && s_bad) atomicOr(&ctrl[CTRL_ABORT], ERR_NONFINITE);
}

// the run's first kernel (see launch_run_begin)
__global__ void k_run_begin(uint32_t* ctrl, int algo)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const uint32_t a = ctrl[CTRL_ABORT];
        if (a) ctrl[CTRL_ERR] |= a;
        ctrl[CTRL_ABORT] = 0u;
        ctrl[CTRL_ALGO] = (uint32_t)algo;
    }
}

// DenseBox grid (Sec. 4.2) from the bounds on the device, in double
// precision: cell side h = f * eps / sqrt(D), enlarged when the widest axis
// would need more than 2^max_axis_bits - 2 cells (the per-cell guard keeps
// the result exact for any cell size, reading of Sec. 4.2); cmax_k = the
// cell index of hi_k (plus one spare cell for rounding at the top); the key
// interleaves `bits` bits per axis, enough for every cmax_k.
template <int D>
__global__ void k_grid(uint32_t* ctrl, float eps, float factor, int max_axis_bits, GridParams* gp)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GridParams g{};
    double h = (double)factor * (double)eps / sqrt((double)D);
    const double maxcells = ldexp(1.0, max_axis_bits);
    float lo[D], hi[D];
    double ext_max = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        lo[k] = ord2f(ctrl[CTRL_LO + k]);
        hi[k] = ord2f(ctrl[CTRL_HI + k]);
        ext_max = fmax(ext_max, (double)hi[k] - (double)lo[k]);
    }
    if (!(ext_max >= 0.0) || isinf(ext_max)) ext_max = 0.0;  // non-finite input: the run is aborted anyway
    if (ext_max / h >= maxcells - 2.0) h = ext_max / (maxcells - 2.0);
    const float inv_h = (float)(1.0 / h);
    int bits = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        g.lo[k] = lo[k];
        double c = floor(((double)hi[k] - (double)lo[k]) * (double)inv_h) + 1.0;
        if (!(c >= 1.0)) c = 1.0;
        if (c > maxcells - 1.0) c = maxcells - 1.0;
        g.cmax[k] = (uint32_t)c;
        while (bits < max_axis_bits && (ldexp(1.0, bits) - 1.0) < (double)g.cmax[k]) ++bits;
    }
    g.inv_h = inv_h;
    g.bits = bits;
    g.morton = 1;
    *gp = g;
    ctrl[CTRL_KEYBITS] = (uint32_t)(bits * D);
}

// ---------------------------------------------------------------------------
// K2: keys. Bit interleaving with axis 0 in the lowest bit.
// ---------------------------------------------------------------------------
// Morton code of each point on a 2^bits grid over the (device-side) bounds;
// u32 keys (FDBSCAN ordering). values = input index.
template <int D>
__global__ void k_morton32(const float* __restrict__ pts, int64_t n, const uint32_t* __restrict__ ctrl, int bits,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    if (!stage_on(ctrl, DBSCAN_ALGO_FDBSCAN)) return;
    float lo[D], scale[D];
    const float cells = (float)(1u << bits);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        lo[k] = ord2f(ctrl[CTRL_LO + k]);
        const float ext = __fsub_rn(ord2f(ctrl[CTRL_HI + k]), lo[k]);
        scale[k] = ext > 0.0f ? __fdiv_rn(cells, ext) : 0.0f;
    }
    const uint32_t cmax = (1u << bits) - 1u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            c[k] = cell_index(floorf(__fmul_rn(__fsub_rn(pts[i * D + k], lo[k]), scale[k])), cmax);
        }
        keys[i] = (uint32_t)interleave<D>(c);
        vals[i] = (uint32_t)i;
    }
}

// The same with 64-bit keys (FDBSCAN ordering above 3D).
template <int D>
__global__ void k_morton64(const float* __restrict__ pts, int64_t n, const uint32_t* __restrict__ ctrl, int bits,
                           uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    if (!stage_on(ctrl, DBSCAN_ALGO_FDBSCAN)) return;
    float lo[D], scale[D];
    const float cells = (float)(1u << bits);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        lo[k] = ord2f(ctrl[CTRL_LO + k]);
        const float ext = __fsub_rn(ord2f(ctrl[CTRL_HI + k]), lo[k]);
        scale[k] = ext > 0.0f ? __fdiv_rn(cells, ext) : 0.0f;
    }
    const uint32_t cmax = (1u << bits) - 1u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            c[k] = cell_index(floorf(__fmul_rn(__fsub_rn(pts[i * D + k], lo[k]), scale[k])), cmax);
        }
        keys[i] = interleave<D>(c);
        vals[i] = (uint32_t)i;
    }
}

// Grid-cell key of each point (DenseBox, Sec. 4.2): cell index
// floor((x_k - lo_k) * inv_h) clamped to [0, cmax_k], Morton-interleaved (or
// packed axis by axis when `morton` is 0). values = input index.
template <int D>
__device__ __forceinline__ uint64_t cell_key(const float* __restrict__ p, const GridParams& g)
{
    uint32_t c[D];
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = cell_index(floorf(__fmul_rn(__fsub_rn(p[k], g.lo[k]), g.inv_h)), g.cmax[k]);
    uint64_t key;
    if (g.morton) {
        key = interleave<D>(c);
    } else {
        key = 0;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) key = (key << g.bits) | c[k];
    }
    return key;
}

// Packed for a keys-only sort: key << idx_bits | i in one word (the host
// caps the grid so that key bits + idx_bits <= 64, and n <= 2^idx_bits). The
// words go to the buffer the sort takes its input from (sort_dev_input_alt).
template <int D>
__global__ void k_cellkey_packed(const float* __restrict__ pts, int64_t n, const GridParams* __restrict__ gp,
                                 const uint32_t* __restrict__ ctrl, int idx_bits, int host_passes,
                                 uint64_t* __restrict__ words0, uint64_t* __restrict__ words1)
{
    if (!stage_on(ctrl, DBSCAN_ALGO_DENSEBOX)) return;
    const GridParams g = *gp;
    // (host_passes 0: no sort runs, n <= 1, and the words stay in words0)
    uint64_t* __restrict__ words =
        host_passes > 0 && sort_dev_input_alt(host_passes, sort_passes((int)ctrl[CTRL_KEYBITS])) ? words1 : words0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        words[i] = (cell_key<D>(pts + i * D, g) << idx_bits) | (uint64_t)i;
}

// ---------------------------------------------------------------------------
// Density estimate for the automatic FDbscan / DenseBox choice: the share of
// points that lie in DenseBox cells holding at least minPts points, from
// EST_SAMPLES strided sample points. Their cells go into an open-addressing
// table; one pass over all points counts the points of each sampled cell
// (per-block shared counters, flushed once); the estimate is the share of
// samples whose cell reaches minPts. Above 2^22 points the counting pass
// reads every stride-th point only and scales its counts by the stride (an
// estimate either way). Keys use at most 63 bits, so the all-ones word marks
// an empty slot.
// ---------------------------------------------------------------------------
constexpr unsigned long long EST_EMPTY = ~0ull;

__device__ __forceinline__ uint32_t est_hash(uint64_t k)
{
    return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 52);  // 12 bits: EST_SLOTS = 4096
}

template <int D>
__global__ void k_est_insert(const float* __restrict__ pts, int64_t n, int s, const GridParams* __restrict__ gp,
                             const uint32_t* __restrict__ ctrl, unsigned long long* __restrict__ table,
                             int32_t* __restrict__ slot)
{
    if (!stage_on(ctrl, -1)) return;
    const GridParams g = *gp;
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const int64_t i = (int64_t)j * n / s;
        const unsigned long long key = cell_key<D>(pts + i * D, g);
        uint32_t h = est_hash(key);
        slot[j] = -1;
        for (int probe = 0; probe < EST_SLOTS; ++probe) {  // load <= 1/2: a slot is always found
            const unsigned long long prev = atomicCAS(&table[h], EST_EMPTY, key);
            if (prev == EST_EMPTY || prev == key) {
                slot[j] = (int32_t)h;
                break;
            }
            h = (h + 1) & (EST_SLOTS - 1);
        }
    }
}

template <int D>
__global__ void k_est_count(const float* __restrict__ pts, int64_t n, int64_t stride,
                            const GridParams* __restrict__ gp, const uint32_t* __restrict__ ctrl,
                            const unsigned long long* __restrict__ table, uint32_t* __restrict__ counts)
{
    if (!stage_on(ctrl, -1)) return;
    const GridParams g = *gp;
    __shared__ uint32_t sc[EST_SLOTS];
    for (int t = threadIdx.x; t < EST_SLOTS; t += blockDim.x) sc[t] = 0;
    __syncthreads();
    const int64_t nc = (n + stride - 1) / stride;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc; j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = cell_key<D>(pts + j * stride * D, g);
        uint32_t h = est_hash(key);
        for (int probe = 0; probe < EST_SLOTS; ++probe) {
            const unsigned long long k = __ldg(&table[h]);
            if (k == key) {
                atomicAdd(&sc[h], 1u);
                break;
            }
            if (k == EST_EMPTY) break;
            h = (h + 1) & (EST_SLOTS - 1);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < EST_SLOTS; t += blockDim.x)
        if (sc[t]) atomicAdd(&counts[t], sc[t]);
}

// out[0] = samples whose cell holds >= min_pts points; out[2..3] = the sum
// over the samples of their cell's point count (64-bit, low word first);
// then the choice: DenseBox if the dense share reaches auto_fraction or the
// mean occupancy auto_occupancy, else FDbscan (CTRL_ALGO, estimates in
// CTRL_EST_FRAC / CTRL_EST_OCC). One block.
__global__ void k_est_result(const int32_t* __restrict__ slot, int s, const uint32_t* __restrict__ counts,
                             int64_t n, int64_t stride, int min_pts, float auto_fraction, float auto_occupancy,
                             uint32_t* __restrict__ out, uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;
    uint32_t c = 0;
    unsigned long long occ = 0;
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        if (slot[j] < 0) continue;
        // the sample itself once, the other counted points of its cell scaled
        // by the stride (the sample is among the counted points iff its index
        // is a multiple of the stride)
        const int64_t i = (int64_t)j * n / s;
        const unsigned long long self = (i % stride == 0) ? 1ull : 0ull;
        const unsigned long long others = (unsigned long long)counts[slot[j]] - self;
        const unsigned long long k = 1ull + others * (unsigned long long)stride;
        if (k >= (unsigned long long)min_pts) ++c;
        occ += k;
    }
    atomicAdd(out, c);
    atomicAdd(reinterpret_cast<unsigned long long*>(out + 2), occ);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence_block();
        const uint32_t dense = *(volatile uint32_t*)out;
        const unsigned long long occ_sum = *(volatile unsigned long long*)(out + 2);
        const float frac = (float)dense / (float)s;
        const float mean_occ = (float)((double)occ_sum / (double)s);
        ctrl[CTRL_EST_FRAC] = __float_as_uint(frac);
        ctrl[CTRL_EST_OCC] = __float_as_uint(mean_occ);
        ctrl[CTRL_ALGO] = (frac >= auto_fraction || mean_occ >= auto_occupancy) ? (uint32_t)DBSCAN_ALGO_DENSEBOX
                                                                               : (uint32_t)DBSCAN_ALGO_FDBSCAN;
    }
}

// generic Morton codes with host-side bounds (component entry point)
template <int D>
__global__ void k_morton_generic(const float* __restrict__ pts, int64_t n, GridParams g, uint64_t* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            c[k] = cell_index(floorf(__fmul_rn(__fsub_rn(pts[i * D + k], g.lo[k]), g.scale[k])), g.cmax[k]);
        }
        uint64_t key = 0;
        for (int b = 0; b < g.bits; ++b)
            for (int k = 0; k < D; ++k) key |= (uint64_t)((c[k] >> b) & 1u) << (b * D + k);
        out[i] = key;
    }
}

// ---------------------------------------------------------------------------
// K4: gather the points into sorted order (structure of points, one 16-byte
// (3D) or 8-byte (2D) record per point).
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_gather(const float* __restrict__ pts, const uint32_t* __restrict__ perm, int64_t n,
                         typename Traits<D>::Point* __restrict__ sp, const uint32_t* __restrict__ ctrl, int algo)
{
    // a sort that gave up leaves stale words in perm: never index with them
    if (!stage_on(ctrl, algo)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sp[i] = Traits<D>::load_point(pts, perm[i]);
}

// A 3D input point (12 bytes at float index 3j) read in aligned pieces: the
// 16-byte block that holds it when it lies in one (one load), else an 8-byte
// and a 4-byte piece (two loads), never past the end of the array (n points).
// The input must be 16-byte aligned.
__device__ __forceinline__ float4 load_point3_aligned(const float* __restrict__ pts, uint32_t j, int64_t n)
{
    const int64_t f = 3 * (int64_t)j;
    const int64_t b = f & ~(int64_t)3;
    const int o = (int)(f - b);
    if (o == 1 || (o == 0 && b + 4 <= 3 * n)) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(pts + b));
        return o == 0 ? make_float4(v.x, v.y, v.z, 0.0f) : make_float4(v.y, v.z, v.w, 0.0f);
    }
    if (o == 3) {
        const float2 yz = __ldg(reinterpret_cast<const float2*>(pts + f + 1));
        return make_float4(__ldg(pts + f), yz.x, yz.y, 0.0f);
    }
    // o == 2, or the last point of the array at o == 0
    const float2 xy = __ldg(reinterpret_cast<const float2*>(pts + f));
    return make_float4(xy.x, xy.y, __ldg(pts + f + 2), 0.0f);
}

template <int D, bool A16>
__device__ __forceinline__ typename Traits<D>::Point gather_point(const float* __restrict__ pts, uint32_t j, int64_t n)
{
    if constexpr (D == 3 && A16) return load_point3_aligned(pts, j, n);
    else return Traits<D>::load_point(pts, j);
}

// The same from sorted packed words, which it splits into the permutation
// and the sorted keys: two sorted positions per thread and step, so that two
// independent input reads are in flight (the words, keys and permutation are
// 16- and 8-byte aligned workspace arrays).
template <int D, bool A16>
__global__ void k_gather_packed(const float* __restrict__ pts, const uint64_t* __restrict__ words, int64_t n,
                                int idx_bits, typename Traits<D>::Point* __restrict__ sp,
                                uint32_t* __restrict__ perm, uint64_t* __restrict__ keys,
                                const uint32_t* __restrict__ ctrl)
{
    using P = typename Traits<D>::Point;
    if (!stage_on(ctrl, DBSCAN_ALGO_DENSEBOX)) return;  // (a sort that gave up: stale index bits)
    const uint64_t mask = (1ull << idx_bits) - 1ull;
    const int64_t pairs = n >> 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pairs; t += stride) {
        // the words are read once and the permutation is next read by the
        // last stages: both stream through L2 with evict-first priority, so
        // that more of the randomly read input points stay cached
        const ulonglong2 w = __ldcs(reinterpret_cast<const ulonglong2*>(words) + t);
        const uint32_t j0 = (uint32_t)(w.x & mask), j1 = (uint32_t)(w.y & mask);
        const P p0 = gather_point<D, A16>(pts, j0, n);
        const P p1 = gather_point<D, A16>(pts, j1, n);
        __stcs(reinterpret_cast<uint2*>(perm) + t, make_uint2(j0, j1));
        reinterpret_cast<ulonglong2*>(keys)[t] = make_ulonglong2(w.x >> idx_bits, w.y >> idx_bits);
        sp[2 * t] = p0;
        sp[2 * t + 1] = p1;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t i = n - 1;
        const uint64_t w = words[i];
        const uint32_t j = (uint32_t)(w & mask);
        perm[i] = j;
        keys[i] = w >> idx_bits;
        sp[i] = gather_point<D, A16>(pts, j, n);
    }
}

// ---------------------------------------------------------------------------
// K5/K6: DenseBox classification. Cells are runs of equal keys in sorted
// order. A cell is dense iff it holds at least minPts points AND the squared
// distance between the corners of the exact bounding box of its points passes
// the eps test: by monotone rounding every pair inside then passes too, so
// "all points core and in one cluster" (Sec. 4.2) holds exactly, whatever
// rounding the grid arithmetic suffered (the precision hazard of Sec. 4.2 is
// turned into a per-cell check instead of an abort).
//
// One pass: the thread at the first point of a run checks with one load
// whether the run reaches minPts points; only those runs are then walked, by
// the whole warp, for the box and the guard, and their points marked 1
// (dense, fits in a tile) or 2 (dense, larger than a tile: a leaf of its
// own), with the run's first point. pdense must be zero on entry.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_dense_classify(const uint64_t* __restrict__ keys, const typename Traits<D>::Point* __restrict__ sp,
                                 int64_t n, int min_pts, float e2, uint8_t* __restrict__ pdense,
                                 int32_t* __restrict__ dstart, uint32_t* __restrict__ ctrl)
{
    using T = Traits<D>;
    if (!stage_on(ctrl, DBSCAN_ALGO_DENSEBOX)) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together so that the cell walks below are cooperative
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; base < n; base += stride) {
        const int64_t i = base + lane;
        bool cand = false;
        if (i < n) {
            const uint64_t k = keys[i];
            const int64_t j = i + min_pts - 1;
            cand = (i == 0 || keys[i - 1] != k) && j < n && keys[j] == k;
        }
        unsigned cm = __ballot_sync(FULL, cand);
        while (cm) {
            const int src = __ffs(cm) - 1;
            cm &= cm - 1;
            const int64_t c0 = __shfl_sync(FULL, i, src);
            const uint64_t k = keys[c0];
            // walk the run with the whole warp: extent and exact box
            typename T::Box b = T::empty_box();
            int64_t e = c0;
            for (;;) {
                const int64_t t = e + lane;
                const bool in = t < n && keys[t] == k;
                if (in) T::grow(b, sp[t]);
                const unsigned im = __ballot_sync(FULL, in);
                e += __popc(im);
                if (im != FULL) break;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) T::merge(b, T::shfl_xor(b, o));
            if (T::diag2(b) > e2) continue;  // the guard: not provably one clique
            const uint8_t f = (e - c0 > TILE) ? 2 : 1;
            for (int64_t t = c0 + lane; t < e; t += 32) {
                pdense[t] = f;
                dstart[t] = (int32_t)c0;
            }
            if (lane == 0) atomicAdd(&ctrl[CTRL_NCELLS], 1u);
        }
    }
}

// Common-prefix length of the sorted keys a (at position pa) and b (at
// position pb, -1 outside [0, n)), equal keys told apart by position: the
// delta of Karras (2012).
template <typename K>
__device__ __forceinline__ int key_delta(K a, int64_t pa, K b, int64_t pb, int64_t n)
{
    constexpr int KB = 8 * (int)sizeof(K);
    if (pb < 0 || pb >= n) return -1;
    if (a != b) return sizeof(K) == 8 ? __clzll((long long)(a ^ b)) : __clz((int)(a ^ b));
    return KB + __clz((int)((uint32_t)pa ^ (uint32_t)pb));
}

template <typename K>
__device__ __forceinline__ K shfl_key(K v, int src)
{
    if constexpr (sizeof(K) == 8) {
        const uint32_t lo = __shfl_sync(FULL, (uint32_t)v, src), hi = __shfl_sync(FULL, (uint32_t)(v >> 32), src);
        return (K)(((uint64_t)hi << 32) | lo);
    } else {
        return (K)__shfl_sync(FULL, (uint32_t)v, src);
    }
}

// Leaf starts. A new leaf starts at point i where the node of the points'
// radix tree (Karras: keys with position tie-break) that splits i - 1 from i
// covers more than TILE points -- tiles are then the maximal subtrees of at
// most TILE points, spatially compact unlike fixed runs in Morton order; and
// at the first point of every dense cell larger than a tile, after such a
// cell, and (batches) where the instance changes.
// The node splitting g and g + 1 has prefix length d = delta(g, g + 1) and
// covers the run around them of keys sharing d bits with key g; delta(g, j)
// only falls as j moves away from g. A warp holds the keys of the 96
// positions around its 32 points in registers (three coalesced loads per
// lane), so four probes per point, taken by shuffles, decide most splits:
// delta(g, g - 31) >= d or delta(g, g + 32) >= d means more than 32 points;
// delta(g, g - 15) < d and delta(g, g + 16) < d means at most 30. For the
// points left undecided the warp ballots, per point, which adjacent prefix
// lengths of the window reach its d (the common prefix of sorted keys a < b
// is the smallest adjacent one between them), and the run lengths to the
// left and right follow from bit scans.
constexpr int LEAF_T = TILE;
static_assert(LEAF_T == 32, "the window holds 32 points on each side");

template <typename K>
__global__ void k_leaf_flags(const K* __restrict__ keys, const int32_t* __restrict__ dstart,
                             const uint8_t* __restrict__ pdense, int64_t n, int id_shift, uint32_t* __restrict__ lfw,
                             int32_t* __restrict__ lfc, const uint32_t* __restrict__ ctrl, int algo)
{
    if (!stage_on(ctrl, algo)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int prev = (lane + 31) & 31;
    for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {  // whole warps iterate together
        // window: positions base - 32 + lane, base + lane, base + 32 + lane
        const int64_t p0 = base - 32 + lane, p1 = base + lane, p2 = base + 32 + lane;
        const K k0 = p0 >= 0 ? keys[p0] : K(0);  // (p0 < base < n)
        const K k1 = p1 < n ? keys[p1] : K(0);
        const K k2 = p2 < n ? keys[p2] : K(0);
        // this lane's point i = p1 and split g = i - 1 (all lanes take part in
        // every shuffle; lane-dependent sources pick the window segment)
        const int64_t i = p1, g = i - 1;
        K kg = shfl_key(k1, prev);
        const K kg_first = shfl_key(k0, 31);
        if (lane == 0) kg = kg_first;
        const K kr_a = shfl_key(k2, prev), kr_b = shfl_key(k1, 31);      // g + 32
        const K kl_a = shfl_key(k0, (lane + 16) & 31), kl_b = shfl_key(k1, (lane + 16) & 31);  // g - 15
        const K km_a = shfl_key(k1, (lane + 15) & 31), km_b = shfl_key(k2, (lane + 15) & 31);  // g + 16
        const K k_right32 = lane == 0 ? kr_b : kr_a;
        const K k_left15 = lane < 16 ? kl_a : kl_b;
        const K k_right16 = lane <= 16 ? km_a : km_b;
        const bool generic = i < n && i > 0;
        int d = -1;
        int state = 0;  // 1 exceeds, 2 does not, 0 undecided
        if (generic) {
            d = key_delta(kg, g, k1, i, n);
            if (key_delta(kg, g, k0, g - 31, n) >= d || key_delta(kg, g, k_right32, g + 32, n) >= d)
                state = 1;
            else if (key_delta(kg, g, k_left15, g - 15, n) < d && key_delta(kg, g, k_right16, g + 16, n) < d)
                state = 2;
        } else {
            state = 2;
        }
        unsigned und = __ballot_sync(FULL, state == 0);
        if (und) {
            // adjacent prefix lengths of the window; -1 outside [0, n)
            K n0 = shfl_key(k0, (lane + 1) & 31), n1 = shfl_key(k1, (lane + 1) & 31),
              n2 = shfl_key(k2, (lane + 1) & 31);
            const K f1 = shfl_key(k1, 0), f2 = shfl_key(k2, 0);
            if (lane == 31) {
                n0 = f1;
                n1 = f2;
                n2 = base + 64 < n ? keys[base + 64] : K(0);
            }
            const int w0 = p0 >= 0 ? key_delta(k0, p0, n0, p0 + 1, n) : -1;
            const int w1 = p1 < n ? key_delta(k1, p1, n1, p1 + 1, n) : -1;
            const int w2 = p2 < n ? key_delta(k2, p2, n2, p2 + 1, n) : -1;
            uint32_t m0 = 0, m1 = 0, m2 = 0;
            while (und) {
                const int src = __ffs(und) - 1;
                und &= und - 1;
                const int ds = __shfl_sync(FULL, d, src);
                const uint32_t b0 = __ballot_sync(FULL, w0 >= ds);
                const uint32_t b1 = __ballot_sync(FULL, w1 >= ds);
                const uint32_t b2 = __ballot_sync(FULL, w2 >= ds);
                if (lane == src) {
                    m0 = b0;
                    m1 = b1;
                    m2 = b2;
                }
            }
            if (state == 0) {
                // window index of g is lane + 31
                const uint64_t lo = (uint64_t)m0 | ((uint64_t)m1 << 32), hi = m2;
                const int pg = lane + 31;
                const uint64_t below = ~lo & ((1ull << pg) - 1ull);
                const int r_left = below ? pg - 1 - (63 - __clzll((long long)below)) : pg;
                const uint64_t y = (lo >> (pg + 1)) | (hi << (63 - pg));
                const int r_right = ~y ? __ffsll((long long)~y) - 1 : 64;
                state = (r_left + r_right + 2) > LEAF_T ? 1 : 2;
            }
        }
        bool f = false;
        if (i >= n) f = false;
        else if (i == 0) f = true;
        else if (id_shift < 64 && ((uint64_t)k1 >> id_shift) != ((uint64_t)kg >> id_shift)) f = true;
        else if (pdense && pdense[i] == 2) f = dstart[i] == (int32_t)i;
        else if (pdense && pdense[i - 1] == 2) f = true;
        else f = state == 1;
        // the window's 32 flags as one word, and how many are set
        const unsigned word = __ballot_sync(FULL, f);
        if (lane == 0) {
            lfw[base >> 5] = word;
            lfc[base >> 5] = __popc(word);
        }
    }
}

// Leaf starts from the flag words (bit b of word w: position 32 w + b
// starts a leaf) and woff, the exclusive scan of their counts: one thread
// per word writes its starts in order; the last word's thread writes m and
// the closing entry lstart[m] = n.
__global__ void k_leaf_write(const uint32_t* __restrict__ lfw, const int32_t* __restrict__ woff, int64_t nw,
                             int64_t n, int32_t* __restrict__ lstart, uint32_t* __restrict__ ctrl, int algo)
{
    // skipped (aborted run, or the other algorithm's chain): m stays 0 and
    // every later stage finds no leaves
    if (!stage_on(ctrl, algo)) return;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = lfw[w];
        int32_t o = woff[w];
        while (word) {
            const int b = __ffs((int)word) - 1;
            word &= word - 1;
            lstart[o++] = (int32_t)(w * 32 + b);
        }
        if (w == nw - 1) {
            lstart[o] = (int32_t)n;
            ctrl[CTRL_M] = (uint32_t)o;
        }
    }
}

// leaf records (start, end | dense << 31) and the leaf keys
template <typename K>
__global__ void k_leaf_records(const int32_t* __restrict__ lstart, const uint8_t* __restrict__ pdense,
                               const K* __restrict__ keys, const uint32_t* __restrict__ ctrl, int id_shift,
                               int2* __restrict__ leafr, uint64_t* __restrict__ lkey, int32_t* __restrict__ linst,
                               int algo)
{
    if (!stage_on(ctrl, algo)) return;
    const int64_t m = ctrl[CTRL_M];
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = lstart[l], e = lstart[l + 1];
        const uint32_t dense = (pdense && pdense[s] == 2) ? 1u : 0u;
        leafr[l] = make_int2(s, (int32_t)((uint32_t)e | (dense << 31)));
        lkey[l] = (uint64_t)keys[s];
        if (linst) linst[l] = (int32_t)((uint64_t)keys[s] >> id_shift);
    }
}

// ---------------------------------------------------------------------------
// Leaf boxes: exact min/max of each leaf's points, stored at unified index
// (m-1) + l of the node-box array. A thread takes a leaf of at most TILE
// points (reading its contiguous points in turn: few instructions per point,
// and consecutive threads' ranges share cache lines); the leaves larger than
// that (dense cells) are taken afterwards by the whole warp, one at a time.
// Each warp also writes the union of its 32 leaves' boxes, the first level of
// the block summaries that the refit reads (sum1[w]: leaves 32 w .. 32 w + 31).
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_leaf_boxes(const typename Traits<D>::Point* __restrict__ sp, const int2* __restrict__ leafr,
                             const uint32_t* __restrict__ ctrl, typename Traits<D>::Box* __restrict__ nodebox,
                             typename Traits<D>::Box* __restrict__ sum1)
{
    using T = Traits<D>;
    const int lane = threadIdx.x & 31;
    const int64_t m = ctrl[CTRL_M];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < m; base += stride) {
        const int64_t l = base + lane;
        int s = 0, e = 0;
        if (l < m) {
            const int2 r = leafr[l];
            s = r.x;
            e = r.y & 0x7fffffff;
        }
        const bool small = l < m && e - s <= TILE;
        typename T::Box mine = T::empty_box();
        if (small) {
            typename T::Box b = T::empty_box();
            int j = s;
            if constexpr (D == 3) {
                // two 16-byte points per 256-bit load from an even index on
                if ((j & 1) && j < e) T::grow(b, sp[j++]);
                for (; j + 1 < e; j += 2) {
                    float4 p0, p1;
                    ldg256(&sp[j], p0, p1);
                    T::grow(b, p0);
                    T::grow(b, p1);
                }
            }
            for (; j < e; ++j) T::grow(b, sp[j]);
            nodebox[(m - 1) + l] = b;
            mine = b;
        }
        unsigned big = __ballot_sync(FULL, l < m && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int bs = __shfl_sync(FULL, s, src), be = __shfl_sync(FULL, e, src);
            typename T::Box b = T::empty_box();
            for (int j = bs + lane; j < be; j += 32) T::grow(b, sp[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) T::merge(b, T::shfl_xor(b, o));
            if (lane == 0) nodebox[(m - 1) + base + src] = b;
            if (lane == src) mine = b;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) T::merge(mine, T::shfl_xor(mine, o));
        if (lane == 0) sum1[base >> 5] = mine;
    }
}

// Higher block summaries: level k (k >= 2) entry j is the union of level-1
// entries [32^(k-1) j, 32^(k-1) (j + 1)), i.e. of 32^k consecutive leaves;
// the levels follow each other in `sum` (level 1 first; sizes and count as
// sum_level_size / sum_levels_entries). One warp per entry, reading level 1
// directly, so no level waits for another.
template <int D>
__global__ void k_box_levels(const uint32_t* __restrict__ ctrl, typename Traits<D>::Box* __restrict__ sum)
{
    using T = Traits<D>;
    const int lane = threadIdx.x & 31;
    const int64_t m = ctrl[CTRL_M];
    if (m <= 1) return;
    const int64_t n1 = sum_level_size(m, 1);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t off = n1;   // start of level 2
    int64_t span = 32;  // level-1 entries per entry of level k
    for (int k = 2; k <= SUM_LEVELS && sum_level_size(m, k - 1) > SUM_DIRECT; ++k, span <<= 5) {
        const int64_t nk = sum_level_size(m, k);
        for (int64_t j = warp; j < nk; j += nwarps) {
            typename T::Box b = T::empty_box();
            const int64_t e0 = j * span, e1 = min(e0 + span, n1);
            for (int64_t i = e0 + lane; i < e1; i += 32) T::merge(b, sum[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) T::merge(b, T::shfl_xor(b, o));
            if (lane == 0) sum[off + j] = b;
        }
        off += nk;
    }
}

// ---------------------------------------------------------------------------
// K7: Karras (2012) LBVH topology. For internal node i the direction, the far
// end of its range and the split come from the common-prefix length delta of
// the sorted leaf keys; equal keys are told apart by the leaf index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int kdelta(const uint64_t* __restrict__ k, int64_t m, int64_t i, int64_t j)
{
    if (j < 0 || j >= m) return -1;
    const uint64_t a = k[i], b = k[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_karras(const uint64_t* __restrict__ lkey, const uint32_t* __restrict__ ctrl, int64_t m_host,
                         int4* __restrict__ nmeta, int32_t* __restrict__ parent, int2* __restrict__ child_out,
                         int2* __restrict__ range_out, int32_t* __restrict__ first_out)
{
    const int64_t m = m_host >= 0 ? m_host : (int64_t)ctrl[CTRL_M];
    if (blockIdx.x == 0 && threadIdx.x == 0) parent[0] = -1;  // root (or the single leaf when m == 1)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m - 1; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (kdelta(lkey, m, i, i + 1) - kdelta(lkey, m, i, i - 1)) > 0 ? 1 : -1;
        const int dmin = kdelta(lkey, m, i, i - d);
        int64_t lmax = 2;
        while (kdelta(lkey, m, i, i + lmax * d) > dmin) lmax <<= 1;
        int64_t l = 0;
        for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
            if (kdelta(lkey, m, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = kdelta(lkey, m, i, j);
        int64_t s = 0, t = l;
        do {
            t = (t + 1) >> 1;
            if (kdelta(lkey, m, i, i + (s + t) * d) > dnode) s += t;
        } while (t > 1);
        const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
        const int64_t first = i < j ? i : j, last = i < j ? j : i;
        const int32_t left = (int32_t)(first == gamma ? (m - 1) + gamma : gamma);
        const int32_t right = (int32_t)(last == gamma + 1 ? (m - 1) + gamma + 1 : gamma + 1);
        nmeta[i] = make_int4(left, right, (int32_t)gamma, (int32_t)last);
        parent[left] = (int32_t)i;
        parent[right] = (int32_t)i;
        if (child_out) child_out[i] = make_int2(left, right);
        if (range_out) range_out[i] = make_int2((int32_t)first, (int32_t)last);
        if (first_out) first_out[i] = (int32_t)first;
    }
}

// ---------------------------------------------------------------------------
// K8: refit. The box of a node is the exact min/max of the boxes of the
// leaves it covers, a contiguous range: node i covers leaves [first_i,
// last_i], its left child [first_i, split_i] and its right child [split_i +
// 1, last_i]. So each node's child boxes are computed directly from the leaf
// boxes, with no dependency between nodes (no climbing, counters or fences):
// min and max are exact in any order, so the boxes are the bottom-up ones
// bit for bit. A node covering at most RF_SMALL leaves is done by its thread;
// longer ranges by the whole warp, from the partial blocks at both ends of
// each summary level and the full blocks of the next one (at most 64 loads a
// lane per level).
// ---------------------------------------------------------------------------
constexpr int RF_SMALL = 32;

template <int D>
__device__ __forceinline__ typename Traits<D>::Box ld_box(const typename Traits<D>::Box* b)
{
    typename Traits<D>::Box r;
    if constexpr (sizeof(typename Traits<D>::Box) == 32) ldg256(b, r.lo, r.hi);
    else r = *b;
    return r;
}

// union of leaf boxes a..b (inclusive), by the whole warp (all lanes, same a, b)
template <int D>
__device__ typename Traits<D>::Box range_box(const typename Traits<D>::Box* __restrict__ leafbox,
                                             const typename Traits<D>::Box* __restrict__ sum, int64_t m, int64_t a,
                                             int64_t b, int lane)
{
    using T = Traits<D>;
    typename T::Box acc = T::empty_box();
    const typename T::Box* arr = leafbox;
    int64_t off = 0, nk = sum_level_size(m, 1);
    for (int level = 0; a <= b && level <= SUM_LEVELS; ++level) {
        if (b - a < SUM_DIRECT || level == SUM_LEVELS) {
            for (int64_t j = a + lane; j <= b; j += 32) T::merge(acc, ld_box<D>(arr + j));
            break;
        }
        // the partial blocks at both ends at this level, the full blocks
        // between them at the next
        const int64_t ha = a + lane, tb = (b & ~(int64_t)31) + lane;
        if (ha <= (a | 31)) T::merge(acc, ld_box<D>(arr + ha));
        if (tb <= b) T::merge(acc, ld_box<D>(arr + tb));
        a = (a >> 5) + 1;
        b = (b >> 5) - 1;
        arr = sum + off;
        off += nk;
        nk = (nk + 31) >> 5;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) T::merge(acc, T::shfl_xor(acc, o));
    return acc;
}

template <int D>
__global__ void k_refit(uint32_t* __restrict__ ctrl, const int4* __restrict__ nmeta,
                        const int32_t* __restrict__ nfirst, typename Traits<D>::Box* __restrict__ nodebox,
                        const typename Traits<D>::Box* __restrict__ sum, typename Traits<D>::Node* __restrict__ nodes)
{
    using T = Traits<D>;
    using Box = typename T::Box;
    const int lane = threadIdx.x & 31;
    const int64_t m = ctrl[CTRL_M];
    if (m <= 1) return;
    const Box* leafbox = nodebox + (m - 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (the long ranges take all lanes)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < m - 1; base += stride) {
        const int64_t p = base + lane;
        int4 mt = make_int4(0, 0, 0, 0);
        int first = 0;
        bool ok = false;
        if (p < m - 1) {
            mt = nmeta[p];
            first = nfirst[p];
            // a range outside the leaves means a corrupt topology
            ok = first >= 0 && first <= mt.z && mt.z < mt.w && mt.w < m;
            if (!ok) atomicOr(&ctrl[CTRL_ERR], ERR_STACK);
        }
        const bool small = ok && mt.w - first < RF_SMALL;
        if (small) {
            Box L = T::empty_box(), R = T::empty_box();
            int j = first;
#pragma unroll 4
            for (; j <= mt.z; ++j) T::merge(L, ld_box<D>(leafbox + j));
#pragma unroll 4
            for (; j <= mt.w; ++j) T::merge(R, ld_box<D>(leafbox + j));
            Box U = L;
            T::merge(U, R);
            nodebox[p] = U;
            nodes[p] = T::make_node(L, R, mt.x, mt.y, mt.z, mt.w);
        }
        unsigned big = __ballot_sync(FULL, ok && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int f = __shfl_sync(FULL, first, src), g = __shfl_sync(FULL, mt.z, src),
                      w = __shfl_sync(FULL, mt.w, src);
            const Box L = range_box<D>(leafbox, sum, m, f, g, lane);
            const Box R = range_box<D>(leafbox, sum, m, (int64_t)g + 1, w, lane);
            if (lane == src) {
                Box U = L;
                T::merge(U, R);
                nodebox[p] = U;
                nodes[p] = T::make_node(L, R, mt.x, mt.y, mt.z, mt.w);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_density_estimate(const float* points, int64_t n, int dim, const GridParams* g, int min_pts,
                                   float auto_fraction, float auto_occupancy, const EstBuffers& eb, uint32_t* ctrl,
                                   cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(eb.table, 0xff, sizeof(unsigned long long) * EST_SLOTS, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(eb.counts, 0, sizeof(uint32_t) * EST_SLOTS, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(eb.result, 0, 4 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    const int smp = n < EST_SAMPLES ? (int)n : EST_SAMPLES;
    const int64_t stride = n > (int64_t(1) << 22) ? n >> 22 : 1;
    int64_t gb = (n / stride + 255) / 256;
    if (gb > 152 * 4) gb = 152 * 4;
#define EST_LAUNCH(D)                                                                      \
    do {                                                                                   \
        k_est_insert<D><<<1, 1024, 0, s>>>(points, n, smp, g, ctrl, eb.table, eb.slot);   \
        k_est_count<D><<<(unsigned)gb, 256, 0, s>>>(points, n, stride, g, ctrl, eb.table, eb.counts); \
    } while (0)
    GBD_DIM_SWITCH(dim, EST_LAUNCH)
#undef EST_LAUNCH
    k_est_result<<<1, 1024, 0, s>>>(eb.slot, smp, eb.counts, n, stride, min_pts, auto_fraction, auto_occupancy,
                                    eb.result, ctrl);
    note_launches(3);
    return cudaGetLastError();
}

static inline unsigned grid_for(int64_t work, int threads, int max_blocks)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

void launch_bounds(const float* pts, int64_t n, int dim, uint32_t* ctrl, cudaStream_t s)
{
#define BOUNDS_LAUNCH(D)                                                                            \
    k_bounds<D><<<grid_for(n * D, bounds_threads<D>(), 152 * 8), bounds_threads<D>(), 0, s>>>(pts, n, ctrl)
    GBD_DIM_SWITCH(dim, BOUNDS_LAUNCH)
#undef BOUNDS_LAUNCH
    note_launches(1);
}

void launch_run_begin(uint32_t* ctrl, int algo, cudaStream_t s)
{
    k_run_begin<<<1, 32, 0, s>>>(ctrl, algo);
    note_launches(1);
}

void launch_grid(uint32_t* ctrl, int dim, float eps, float factor, int max_axis_bits, GridParams* gp,
                 cudaStream_t s)
{
#define GRID_LAUNCH(D) k_grid<D><<<1, 32, 0, s>>>(ctrl, eps, factor, max_axis_bits, gp)
    GBD_DIM_SWITCH(dim, GRID_LAUNCH)
#undef GRID_LAUNCH
    note_launches(1);
}

void launch_morton32(const float* pts, int64_t n, int dim, const uint32_t* ctrl, int bits, uint32_t* keys,
                     uint32_t* vals, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    if (dim == 3) k_morton32<3><<<g, 256, 0, s>>>(pts, n, ctrl, bits, keys, vals);
    else k_morton32<2><<<g, 256, 0, s>>>(pts, n, ctrl, bits, keys, vals);
    note_launches(1);
}

void launch_morton64(const float* pts, int64_t n, int dim, const uint32_t* ctrl, int bits, uint64_t* keys,
                     uint32_t* vals, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
#define M64_LAUNCH(D) k_morton64<D><<<g, 256, 0, s>>>(pts, n, ctrl, bits, keys, vals)
    GBD_DIM_SWITCH(dim, M64_LAUNCH)
#undef M64_LAUNCH
    note_launches(1);
}

void launch_cellkey_packed(const float* pts, int64_t n, int dim, const GridParams* gp, const uint32_t* ctrl,
                           int idx_bits, int host_passes, uint64_t* words0, uint64_t* words1, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
#define CKP_LAUNCH(D) \
    k_cellkey_packed<D><<<g, 256, 0, s>>>(pts, n, gp, ctrl, idx_bits, host_passes, words0, words1)
    GBD_DIM_SWITCH(dim, CKP_LAUNCH)
#undef CKP_LAUNCH
    note_launches(1);
}

void launch_gather_packed(const float* pts, const uint64_t* words, int64_t n, int dim, int idx_bits, void* sp,
                          uint32_t* perm, uint64_t* keys, const uint32_t* ctrl, cudaStream_t s)
{
    const unsigned g = grid_for((n + 1) / 2, 256, 152 * 16);
    const bool a16 = (reinterpret_cast<uintptr_t>(pts) & 15) == 0;
#define GP_LAUNCH(D)                                                                                          \
    do {                                                                                                      \
        auto* spd = static_cast<typename Traits<D>::Point*>(sp);                                              \
        if (a16) k_gather_packed<D, true><<<g, 256, 0, s>>>(pts, words, n, idx_bits, spd, perm, keys, ctrl);  \
        else k_gather_packed<D, false><<<g, 256, 0, s>>>(pts, words, n, idx_bits, spd, perm, keys, ctrl);    \
    } while (0)
    GBD_DIM_SWITCH(dim, GP_LAUNCH)
#undef GP_LAUNCH
    note_launches(1);
}

void launch_morton_generic(const float* pts, int64_t n, int dim, const GridParams& gp, uint64_t* out, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    if (dim == 3) k_morton_generic<3><<<g, 256, 0, s>>>(pts, n, gp, out);
    else k_morton_generic<2><<<g, 256, 0, s>>>(pts, n, gp, out);
    note_launches(1);
}

void launch_gather(const float* pts, const uint32_t* perm, int64_t n, int dim, void* sp, const uint32_t* ctrl,
                   int algo, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
#define GATHER_LAUNCH(D) \
    k_gather<D><<<g, 256, 0, s>>>(pts, perm, n, static_cast<typename Traits<D>::Point*>(sp), ctrl, algo)
    GBD_DIM_SWITCH(dim, GATHER_LAUNCH)
#undef GATHER_LAUNCH
    note_launches(1);
}

// Leaf starts of n sorted keys into t.lstart and m into ctrl (flags as bit
// words in t.lf, their counts after them, the counts' scan in t.lidx).
template <typename K>
cudaError_t launch_leaf_starts(const K* keys, const int32_t* dstart, const uint8_t* pdense, int64_t n, int id_shift,
                               const DenseBoxTemps& t, uint32_t* ctrl, int algo, cudaStream_t s)
{
    const int64_t nw = (n + 31) / 32;
    uint32_t* words = reinterpret_cast<uint32_t*>(t.lf);
    int32_t* counts = t.lf + nw;
    k_leaf_flags<K><<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(keys, dstart, pdense, n, id_shift, words, counts,
                                                                ctrl, algo);
    cudaError_t e;
    if ((e = scan_i32(counts, t.lidx, nw, SCAN_ADD, false, t.scan_temp, s)) != cudaSuccess) return e;
    k_leaf_write<<<grid_for(nw, 256, 152 * 16), 256, 0, s>>>(words, t.lidx, nw, n, t.lstart, ctrl, algo);
    return cudaSuccess;
}

cudaError_t launch_densebox_leaves(const uint64_t* keys, const void* sp, int64_t n, int dim, int min_pts, float e2,
                                   const DenseBoxTemps& t, int2* leafr, uint64_t* lkey, uint32_t* ctrl,
                                   cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    cudaError_t e;
    if ((e = cudaMemsetAsync(t.pdense, 0, (size_t)n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctrl + CTRL_NCELLS, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
#define DC_LAUNCH(D)                                                                                         \
    k_dense_classify<D><<<g, 256, 0, s>>>(keys, static_cast<const typename Traits<D>::Point*>(sp), n, min_pts, e2, \
                                          t.pdense, t.dstart, ctrl)
    GBD_DIM_SWITCH(dim, DC_LAUNCH)
#undef DC_LAUNCH
    const int A = DBSCAN_ALGO_DENSEBOX;
    if ((e = launch_leaf_starts<uint64_t>(keys, t.dstart, t.pdense, n, 64, t, ctrl, A, s)) != cudaSuccess) return e;
    k_leaf_records<uint64_t><<<g, 256, 0, s>>>(t.lstart, t.pdense, keys, ctrl, 64, leafr, lkey, nullptr, A);
    note_launches(4);
    return cudaGetLastError();
}

// Leaves of a batch: keys carry the instance in their bits from id_shift up;
// tiles never cross instances. pdense/dstart come from the batch's dense-cell
// classification (null for FDBSCAN).
cudaError_t launch_batch_leaves(const uint64_t* keys, int64_t n, int id_shift, const DenseBoxTemps& t, int2* leafr,
                                uint64_t* lkey, int32_t* linst, uint32_t* ctrl, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    cudaError_t e;
    if ((e = launch_leaf_starts<uint64_t>(keys, t.dstart, t.pdense, n, id_shift, t, ctrl, -1, s)) != cudaSuccess)
        return e;
    k_leaf_records<uint64_t><<<g, 256, 0, s>>>(t.lstart, t.pdense, keys, ctrl, id_shift, leafr, lkey, linst, -1);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_tile_leaves(const uint32_t* keys32, int64_t n, const DenseBoxTemps& t, int2* leafr,
                               uint64_t* lkey, uint32_t* ctrl, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    cudaError_t e;
    const int A = DBSCAN_ALGO_FDBSCAN;
    if ((e = launch_leaf_starts<uint32_t>(keys32, nullptr, nullptr, n, 64, t, ctrl, A, s)) != cudaSuccess) return e;
    k_leaf_records<uint32_t><<<g, 256, 0, s>>>(t.lstart, nullptr, keys32, ctrl, 64, leafr, lkey, nullptr, A);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_tile_leaves64(const uint64_t* keys, int64_t n, const DenseBoxTemps& t, int2* leafr,
                                 uint64_t* lkey, uint32_t* ctrl, cudaStream_t s)
{
    const unsigned g = grid_for(n, 256, 152 * 16);
    cudaError_t e;
    const int A = DBSCAN_ALGO_FDBSCAN;
    if ((e = launch_leaf_starts<uint64_t>(keys, nullptr, nullptr, n, 64, t, ctrl, A, s)) != cudaSuccess) return e;
    k_leaf_records<uint64_t><<<g, 256, 0, s>>>(t.lstart, nullptr, keys, ctrl, 64, leafr, lkey, nullptr, A);
    note_launches(3);
    return cudaGetLastError();
}

void launch_lbvh(const void* sp, int dim, const int2* leafr, const uint64_t* lkey, int64_t m_cap, uint32_t* ctrl,
                 int4* nmeta, int32_t* parent, int32_t* nfirst, void* nodebox, void* nsum, void* nodes, cudaStream_t s,
                 int2* range_out)
{
    const unsigned g = grid_for(m_cap, 256, 152 * 16);
    const unsigned gl = grid_for(sum_levels_entries(m_cap) * 32, 256, 152 * 4);
#define LB_LAUNCH(D)                                                                                           \
    do {                                                                                                       \
        using Bx = typename Traits<D>::Box;                                                                    \
        k_leaf_boxes<D><<<g, 256, 0, s>>>(static_cast<const typename Traits<D>::Point*>(sp), leafr, ctrl,       \
                                           static_cast<Bx*>(nodebox), static_cast<Bx*>(nsum));                  \
        k_box_levels<D><<<gl, 256, 0, s>>>(ctrl, static_cast<Bx*>(nsum));                                       \
    } while (0)
    GBD_DIM_SWITCH(dim, LB_LAUNCH)
#undef LB_LAUNCH
    k_karras<<<g, 256, 0, s>>>(lkey, ctrl, -1, nmeta, parent, nullptr, range_out, nfirst);
#define RF_LAUNCH(D)                                                                                         \
    k_refit<D><<<g, 256, 0, s>>>(ctrl, nmeta, nfirst, static_cast<typename Traits<D>::Box*>(nodebox),          \
                                 static_cast<const typename Traits<D>::Box*>(nsum),                            \
                                 static_cast<typename Traits<D>::Node*>(nodes))
    GBD_DIM_SWITCH(dim, RF_LAUNCH)
#undef RF_LAUNCH
    note_launches(4);
}

void launch_karras_only(const uint64_t* lkey, int64_t m, int4* nmeta, int32_t* parent, int2* child_out,
                        int2* range_out, cudaStream_t s)
{
    k_karras<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(lkey, nullptr, m, nmeta, parent, child_out, range_out,
                                                        nullptr);
    note_launches(1);
}

}  // namespace gbd
