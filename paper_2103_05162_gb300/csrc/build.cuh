// Declarations shared by the pipeline stages (build.cu, traverse.cu, capi.cu).
#pragma once

#include "internal.cuh"

namespace gbd {

constexpr int MAX_DIM = 8;  // points of 2 to 8 dimensions

// calls F(D) with the compile-time dimension D equal to dim (2 .. MAX_DIM;
// arguments are checked before any launch)
#define GBD_DIM_SWITCH(dim, F)         \
    switch (dim) {                     \
    case 2: F(2); break;               \
    case 3: F(3); break;               \
    case 4: F(4); break;               \
    case 5: F(5); break;               \
    case 6: F(6); break;               \
    case 7: F(7); break;               \
    default: F(8); break;              \
    }

// bounds kernel block size: a multiple of D, so that a thread striding over
// the flat coordinates always sees the same axis
template <int D>
constexpr int bounds_threads()
{
    return D == 5 ? 320 : (D == 7 ? 448 : 384);
}

// Morton-code bits per axis of FDbscan's keys: 32-bit keys in 2D and 3D,
// 64-bit keys (at most 63 bits) above
inline int fdbscan_bits(int dim)
{
    return dim == 3 ? 10 : (dim == 2 ? 16 : 63 / dim);
}

// Slots of the per-workspace control block (uint32 words in device memory).
enum : int {
    CTRL_NONFINITE = 8,  // nonzero if a coordinate is NaN/Inf (batches)
    CTRL_ERR = 9,        // device error bits (ERR_*) of earlier runs, kept until a host sync point reads them
    CTRL_M = 10,         // number of BVH leaves
    CTRL_NCELLS = 11,    // number of dense cells (DenseBox)
    CTRL_WORK_PRE = 12,  // work counters of the persistent traversal kernels
    CTRL_WORK_MAIN = 13,
    CTRL_KIND_COUNT = 16,  // 3 words: leaves per kind (0 tile, 1 solid tile, 2 dense cell leaf)
    CTRL_KIND_FILL = 19,   // 3 words: fill counters of the per-kind leaf lists
    CTRL_KIND_WORK = 22,   // 3 words: work counters of the per-kind main kernels
    CTRL_WORK_END = 25,    // end of the per-phase counters (cleared before each phase)
    CTRL_ABORT = 26,       // error bits of the current run (ERR_*): set, every later stage does nothing
    CTRL_ALGO = 27,        // the algorithm the current run uses (DBSCAN_ALGO_FDBSCAN / _DENSEBOX)
    CTRL_KEYBITS = 28,     // DenseBox: cell-key bits of the current run's grid
    CTRL_EST_FRAC = 29,    // automatic choice: estimated dense-point share (float bits)
    CTRL_EST_OCC = 30,     // automatic choice: estimated mean cell occupancy (float bits)
    CTRL_LO = 32,          // MAX_DIM words: order-preserving min per axis
    CTRL_HI = 40,          // MAX_DIM words: order-preserving max per axis
    CTRL_WORDS = 48
};

constexpr unsigned ERR_STACK = 2u;  // traversal/refit limits exceeded (cannot happen for valid trees)

// Whether a stage of the current run goes ahead: not once the run is
// aborted (CTRL_ABORT: non-finite input, a sort that gave up), and, for a
// stage of one algorithm's chain (algo >= 0), only if the run chose that
// algorithm. All threads of a launch read the same words (written by earlier
// launches), so the decision is uniform.
__device__ __forceinline__ bool stage_on(const uint32_t* ctrl, int algo)
{
    if (!ctrl) return true;
    if (*(volatile const uint32_t*)(ctrl + CTRL_ABORT) != 0u) return false;
    return algo < 0 || *(volatile const uint32_t*)(ctrl + CTRL_ALGO) == (uint32_t)algo;
}

struct GridParams {
    float lo[MAX_DIM];
    float scale[MAX_DIM];     // per-axis scale (generic Morton codes)
    float inv_h;              // 1 / cell side (DenseBox cells)
    uint32_t cmax[MAX_DIM];   // largest cell index per axis
    int bits;           // bits per axis in the key
    int morton;         // 1: interleave, 0: pack axis by axis
};

// density estimate (automatic algorithm choice)
constexpr int EST_SAMPLES = 2048;
constexpr int EST_SLOTS = 4096;
struct EstBuffers {
    unsigned long long* table;  // EST_SLOTS cell keys
    int32_t* slot;              // EST_SAMPLES: the table slot of each sample's cell
    uint32_t* counts;           // EST_SLOTS: points per sampled cell
    uint32_t* result;           // 4 words: [0] samples whose cell holds >= minPts points, [2..3] the
                                // sum over the samples of their cell's point count (u64, 8-byte aligned)
};
// over the samples (min(n, EST_SAMPLES), strided; above 2^22 points the cells
// are counted on every (n >> 22)-th point, scaled): how many lie in DenseBox
// cells (grid g) of at least min_pts points, and the summed point counts of
// their cells (the size-biased mean occupancy once divided by the samples)
// The estimate then decides the algorithm on the device: DenseBox from a
// dense share of auto_fraction or a mean occupancy of auto_occupancy up,
// FDbscan otherwise (CTRL_ALGO, CTRL_EST_FRAC, CTRL_EST_OCC).
cudaError_t launch_density_estimate(const float* points, int64_t n, int dim, const GridParams* g, int min_pts,
                                   float auto_fraction, float auto_occupancy, const EstBuffers& eb, uint32_t* ctrl,
                                   cudaStream_t s);

struct DenseBoxTemps {
    uint8_t* pdense;    // n: 0 not dense, 1 dense cell within a tile, 2 dense cell as its own leaf
    int32_t* dstart;    // n: first point of the dense cell (valid where pdense != 0)
    int32_t* lf;        // n + 64: leaf-start flags as bit words (n / 32), then their counts
    int32_t* lidx;      // n: the counts' exclusive scan
    int32_t* lstart;    // n + 1
    int32_t* scan_temp; // scan_temp_words(n)
};

// ---------------------------------------------------------------------------
// key helpers: bit interleaving with axis 0 in the lowest bit
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread2(uint64_t x)  // 32 bits -> even bits
{
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
__device__ __forceinline__ uint64_t spread3(uint64_t x)  // 21 bits -> every third bit
{
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
// floor'd cell coordinate -> index in [0, cmax] (clamped as an integer, so
// that cmax is exact even where it is not representable in fp32)
__device__ __forceinline__ uint32_t cell_index(float t, uint32_t cmax)
{
    const uint32_t c = (uint32_t)fminf(fmaxf(t, 0.0f), 4294967040.0f);
    return c < cmax ? c : cmax;
}

template <int D>
__device__ __forceinline__ uint64_t interleave(const uint32_t* c)
{
    if (D == 3) return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    if (D == 2) return spread2(c[0]) | (spread2(c[1]) << 1);
    // above 3D: bit b of axis k goes to bit b * D + k (63 / D bits per axis)
    uint64_t key = 0;
#pragma unroll
    for (int b = 0; b < 63 / D; ++b)
#pragma unroll
        for (int k = 0; k < D; ++k) key |= (uint64_t)((c[k] >> b) & 1u) << (b * D + k);
    return key;
}

void launch_bounds(const float* pts, int64_t n, int dim, uint32_t* ctrl, cudaStream_t s);
// the run's first kernel: moves CTRL_ABORT's bits into CTRL_ERR (kept for
// the next host sync point), clears CTRL_ABORT and sets CTRL_ALGO
void launch_run_begin(uint32_t* ctrl, int algo, cudaStream_t s);
// DenseBox grid from the device-side bounds: cell side f * eps / sqrt(dim)
// (Sec. 4.2), coarsened until every axis fits max_axis_bits; writes *gp and
// CTRL_KEYBITS
void launch_grid(uint32_t* ctrl, int dim, float eps, float factor, int max_axis_bits, GridParams* gp,
                 cudaStream_t s);
// FDbscan keys (gated on CTRL_ALGO == FDBSCAN): 32-bit Morton codes in 2D/3D
void launch_morton32(const float* pts, int64_t n, int dim, const uint32_t* ctrl, int bits, uint32_t* keys,
                     uint32_t* vals, cudaStream_t s);
// FDbscan keys above 3D: 64-bit Morton codes, `bits` per axis
void launch_morton64(const float* pts, int64_t n, int dim, const uint32_t* ctrl, int bits, uint64_t* keys,
                     uint32_t* vals, cudaStream_t s);
void launch_morton_generic(const float* pts, int64_t n, int dim, const GridParams& gp, uint64_t* out,
                           cudaStream_t s);
// FDbscan gather (gated): sorted points from the sort's permutation
void launch_gather(const float* pts, const uint32_t* perm, int64_t n, int dim, void* sp, const uint32_t* ctrl,
                   int algo, cudaStream_t s);
// DenseBox keys packed above the point index for a keys-only sort (gated on
// DENSEBOX), written to words0 or words1 as sort_dev_input_alt(host_passes,
// the passes CTRL_KEYBITS needs) says; and the gather that splits the sorted
// words into permutation and keys
void launch_cellkey_packed(const float* pts, int64_t n, int dim, const GridParams* gp, const uint32_t* ctrl,
                           int idx_bits, int host_passes, uint64_t* words0, uint64_t* words1, cudaStream_t s);
void launch_gather_packed(const float* pts, const uint64_t* words, int64_t n, int dim, int idx_bits, void* sp,
                          uint32_t* perm, uint64_t* keys, const uint32_t* ctrl, cudaStream_t s);
cudaError_t launch_densebox_leaves(const uint64_t* keys, const void* sp, int64_t n, int dim, int min_pts, float e2,
                                   const DenseBoxTemps& t, int2* leafr, uint64_t* lkey, uint32_t* ctrl,
                                   cudaStream_t s);
// FDbscan leaves (gated on FDBSCAN): radix tiles of the Morton-sorted points
cudaError_t launch_tile_leaves(const uint32_t* keys32, int64_t n, const DenseBoxTemps& t, int2* leafr,
                               uint64_t* lkey, uint32_t* ctrl, cudaStream_t s);
cudaError_t launch_tile_leaves64(const uint64_t* keys, int64_t n, const DenseBoxTemps& t, int2* leafr,
                                 uint64_t* lkey, uint32_t* ctrl, cudaStream_t s);
// Block summaries of the leaf boxes (read by the refit): level k >= 1 holds
// ceil(m / 32^k) boxes, each the union of 32^k consecutive leaves; level
// k + 1 exists while level k holds more than SUM_DIRECT boxes (a range of at
// most SUM_DIRECT entries of one level is read directly).
constexpr int SUM_LEVELS = 7;    // 32^7 leaves: beyond any leaf count
constexpr int SUM_DIRECT = 64;
__host__ __device__ inline int64_t sum_level_size(int64_t m, int k)
{
    int64_t c = m;
    for (int i = 0; i < k; ++i) c = (c + 31) >> 5;
    return c;
}
__host__ __device__ inline int64_t sum_levels_entries(int64_t m)
{
    int64_t t = 0, c = sum_level_size(m, 1);
    for (int k = 1; k <= SUM_LEVELS; ++k) {
        t += c;
        if (c <= SUM_DIRECT) break;
        c = (c + 31) >> 5;
    }
    return t;
}
// leaf boxes, block summaries (nsum: sum_levels_entries(m_cap) boxes),
// Karras topology (nfirst: the first leaf of each internal node) and refit
void launch_lbvh(const void* sp, int dim, const int2* leafr, const uint64_t* lkey, int64_t m_cap, uint32_t* ctrl,
                 int4* nmeta, int32_t* parent, int32_t* nfirst, void* nodebox, void* nsum, void* nodes,
                 cudaStream_t s, int2* range_out = nullptr);
cudaError_t launch_batch_leaves(const uint64_t* keys, int64_t n, int id_shift, const DenseBoxTemps& t, int2* leafr,
                                uint64_t* lkey, int32_t* linst, uint32_t* ctrl, cudaStream_t s);
void launch_karras_only(const uint64_t* lkey, int64_t m, int4* nmeta, int32_t* parent, int2* child_out,
                        int2* range_out, cudaStream_t s);

// traverse.cu
constexpr int TRAVERSAL_SIBCAP = 8;   // sibling subtrees recorded per leaf
constexpr int TRAVERSAL_LEAFCAP = 48; // leaves within eps listed per leaf

struct ClusterArgs {
    const void* sp;        // sorted points
    const void* nodes;     // m-1 node records
    const void* nodebox;   // 2m-1 boxes (leaf boxes at m-1+l)
    const int2* leafr;     // m leaf records
    uint8_t* lsolid;       // m: 1 if all points of the leaf are core and in one set
    int32_t* klist;        // m: leaf indices grouped by kind
    const uint8_t* pdense; // n or null: dense-cell flags per sorted point (DenseBox)
    const int32_t* dstart; // n or null: first point of each point's dense cell
    const uint32_t* perm;  // sorted position -> input index
    int32_t* labels;       // n (union-find parents, sorted index space)
    uint8_t* core;         // n (sorted order)
    uint8_t* nbr;          // n: preprocessing's out-of-tile neighbour count of non-core points (lists on),
                           //    else 1 if another point is within eps
    int32_t* nlist = nullptr;  // n * lcap: out-of-tile neighbours found by preprocessing
    int lcap = 0;              // list entries per point (0: no lists)
    int32_t* canon;        // n (smallest input index per root)
    uint32_t* ctrl;
    int64_t n;
    int64_t m_cap;         // upper bound of m (grid sizing)
    int dim;
    float e2;
    int min_pts;
    int mode;
    int block;             // traversal block size
    // batches of independent instances (null for a single instance): the
    // instance of each leaf, per-instance eps^2 / minPts, and the root of
    // each instance's subtree; min_pts then holds the largest minPts
    const int32_t* linst = nullptr;
    const float* e2s = nullptr;
    const int32_t* mps = nullptr;
    const int32_t* iroot = nullptr;
    // tree links (parent of every node, children of internal nodes) and the
    // per-leaf traversal start written by launch_cluster_pre
    const int32_t* parent = nullptr;
    const int4* nmeta = nullptr;
    int32_t* tstart = nullptr;
    int2* tsib = nullptr;    // m_cap * TRAVERSAL_SIBCAP: (node, last leaf) of the sibling subtrees within eps
    int8_t* tnsib = nullptr; // m_cap: how many (-1: more than TRAVERSAL_SIBCAP, use tstart)
    int32_t* llist = nullptr;  // m_cap * TRAVERSAL_LEAFCAP: the leaves within eps of each leaf's box
    int16_t* lcount = nullptr; // m_cap: how many (-1: more than TRAVERSAL_LEAFCAP, walk the tree)
    // multi-minPts runs: neighbour counts capped at min_pts (null otherwise)
    int32_t* ncount = nullptr;
};
cudaError_t launch_cluster_init(const ClusterArgs& a, cudaStream_t s);
// per-leaf traversal starts (needed by both traversal phases)
cudaError_t launch_cluster_starts(const ClusterArgs& a, cudaStream_t s);
// preprocessing (minPts > 2, or counting for several minPts; nothing otherwise)
cudaError_t launch_cluster_pre(const ClusterArgs& a, cudaStream_t s);
// one minPts of a multi-minPts run: labels and core flags from a.ncount, then
// border claims from the lists; the caller then runs the main phase with
// min_pts = max(3, min_pts) (the core flags are exact, so the minPts <= 2
// forms, which find core points during the main phase, are not needed)
cudaError_t launch_cluster_from_counts(const ClusterArgs& a, int min_pts, cudaStream_t s);
// core flags from the caller (device, input order), after launch_cluster_init;
// the main phase then runs with min_pts = max(3, min_pts) and no lists
cudaError_t launch_cluster_core_from_input(const ClusterArgs& a, const uint8_t* core_in, cudaStream_t s);
cudaError_t launch_cluster_main(const ClusterArgs& a, cudaStream_t s);
cudaError_t launch_cluster_final(const ClusterArgs& a, int32_t* labels_out, uint8_t* core_out, cudaStream_t s);
// traversal counters (built with -DGBD_COUNTERS only)
bool counters_built();
cudaError_t counters_take(uint64_t* out);  // CNT_PHASES * CNT_KINDS values

}  // namespace gbd
