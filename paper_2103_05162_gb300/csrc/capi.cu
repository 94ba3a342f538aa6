// The C ABI of libgbdbscan (include/gbdbscan.h): argument checks, per-stream
// device workspaces and the enqueueing of the pipeline
//   bounds -> keys -> radix sort -> gather -> [DenseBox cells] -> leaves ->
//   LBVH topology -> refit -> union-find init -> [preprocessing] -> main ->
//   finalize -> relabel
// (Sec. 3.2 Algorithm 3 with the indexes of Sec. 4.1 / 4.2).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "build.cuh"
#include "capi_internal.h"

namespace gbd {

thread_local std::string t_err;

dbscan_status set_error(dbscan_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

void clear_error() { t_err.clear(); }

dbscan_status cuda_error(cudaError_t e, const char* what)
{
    return set_error(e == cudaErrorMemoryAllocation ? DBSCAN_ERR_OOM : DBSCAN_ERR_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

#define TRY_CUDA(x)                                         \
    do {                                                    \
        cudaError_t e_ = (x);                               \
        if (e_ != cudaSuccess) return cuda_error(e_, #x);   \
    } while (0)

// (above 3D the 3D thresholds: FDbscan's Morton grid is coarse there too)
Tuning g_tuning = {0,
                   0.0f,
                   1,
                   {0.0f, 0.0f, DEFAULT_AUTO_FRACTION_2D, DEFAULT_AUTO_FRACTION_3D, DEFAULT_AUTO_FRACTION_3D,
                    DEFAULT_AUTO_FRACTION_3D, DEFAULT_AUTO_FRACTION_3D, DEFAULT_AUTO_FRACTION_3D,
                    DEFAULT_AUTO_FRACTION_3D},
                   {0.0f, 0.0f, DEFAULT_AUTO_OCCUPANCY, DEFAULT_AUTO_OCCUPANCY, DEFAULT_AUTO_OCCUPANCY,
                    DEFAULT_AUTO_OCCUPANCY, DEFAULT_AUTO_OCCUPANCY, DEFAULT_AUTO_OCCUPANCY, DEFAULT_AUTO_OCCUPANCY}};

// ---------------------------------------------------------------------------
// the autotuner's table (traversal block size and DenseBox cell factor per
// kind of call)
// ---------------------------------------------------------------------------
thread_local RunTuning t_run = DEFAULT_RUN_TUNING;

bool TuneKey::operator<(const TuneKey& o) const
{
    const int a[7] = {kind, dim, log2n, min_pts, algo, mode, log2count};
    const int b[7] = {o.kind, o.dim, o.log2n, o.min_pts, o.algo, o.mode, o.log2count};
    for (int i = 0; i < 7; ++i)
        if (a[i] != b[i]) return a[i] < b[i];
    return false;
}

static int ceil_log2(int64_t v)
{
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < v) ++b;
    return b;
}

TuneKey tune_key(int kind, int dim, int64_t n, int min_pts, int algo, int mode, int64_t count)
{
    return TuneKey{kind, dim, ceil_log2(n), min_pts, algo, mode, kind == 1 ? ceil_log2(count) : 0};
}

namespace {
struct TuneEntry {
    RunTuning t;
    float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;
}  // namespace

bool autotune_on() { return g_tuning.block == 0 || g_tuning.cell_factor == 0.0f; }

bool tuned(const TuneKey& k)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_tune.count(k) != 0;
}

void store_tuning(const TuneKey& k, RunTuning t, float ms)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[k] = TuneEntry{t, ms};
}

RunTuning resolve_tuning(const TuneKey& k)
{
    RunTuning r = DEFAULT_RUN_TUNING;
    if (autotune_on()) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(k);
        if (it != g_tune.end()) r = it->second.t;
    }
    if (g_tuning.block != 0) r.block = g_tuning.block;
    if (g_tuning.cell_factor != 0.0f) r.cell_factor = g_tuning.cell_factor;
    return r;
}

int tuning_candidates(int algo, RunTuning* out, int cap)
{
    static const int blocks[3] = {64, 128, 256};
    static const float factors[3] = {1.0f, 0.75f, 0.5f};
    const int nf = algo == DBSCAN_ALGO_FDBSCAN ? 1 : 3;  // FDbscan has no grid
    int k = 0;
    for (int i = 0; i < nf; ++i) {
        const float f = g_tuning.cell_factor != 0.0f ? g_tuning.cell_factor : factors[i];
        for (int j = 0; j < 3; ++j) {
            const int b = g_tuning.block != 0 ? g_tuning.block : blocks[j];
            bool dup = false;
            for (int t = 0; t < k; ++t) dup = dup || (out[t].block == b && out[t].cell_factor == f);
            if (!dup && k < cap) out[k++] = RunTuning{b, f};
        }
    }
    return k;
}

// ---------------------------------------------------------------------------
// launch counting and opt-in per-stage timing (CUDA events on the stream)
// ---------------------------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<bool> g_profile{false};
static const char* kStageNames[DBSCAN_PROFILE_STAGES] = {"bounds", "keys", "sort", "gather", "leaves",
                                                         "lbvh", "init", "preprocess", "main", "finalize"};

struct ProfState {
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

// records the start/end of one stage on the stream when profiling is on
struct StageTimer {
    Workspace* w;
    cudaStream_t s;
    bool on;
    int stage = -1;
    cudaEvent_t a = nullptr;
    StageTimer(Workspace* w_, cudaStream_t s_) : w(w_), s(s_), on(g_profile.load()) {}
    void begin(int st)
    {
        if (!on) return;
        stage = st;
        a = w->prof->get();
        cudaEventRecord(a, s);
    }
    void end()
    {
        if (!on || stage < 0) return;
        cudaEvent_t b = w->prof->get();
        cudaEventRecord(b, s);
        w->prof->recs.push_back({stage, a, b});
        stage = -1;
    }
};

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
namespace {

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};

}  // namespace

// Device buffers of one pipeline run, carved from the workspace arena.
struct Plan {
    uint32_t* ctrl;
    void* keys;
    void* keys_alt;
    uint32_t* vals;
    uint32_t* vals_alt;
    uint32_t* hist;
    uint32_t* counters;
    uint32_t* status;
    void* sp;
    DenseBoxTemps db;
    int2* leafr;
    uint64_t* lkey;
    void* nodebox;
    void* nodes;
    int4* nmeta;
    int32_t* parent;
    int32_t* nfirst;  // first leaf of each internal node
    void* nsum;       // block summaries of the leaf boxes
    uint8_t* lsolid;
    int32_t* klist;
    int32_t* tstart;
    int2* tsib;
    int8_t* tnsib;
    int32_t* llist;
    int16_t* lcount;
    int32_t* labels;
    uint8_t* core;
    uint8_t* nbr;
    int32_t* canon;
    int32_t* nlist;  // n * lcap neighbour indices (preprocessing lists)
    int32_t* ncount; // n neighbour counts capped at the largest minPts (multi-minPts runs)
    EstBuffers est;  // density estimate (automatic algorithm choice)
    GridParams* grid;     // DenseBox grid, computed on the device from the bounds
    GridParams* grid_est; // the automatic choice's grid (cell side eps / sqrt(d), whatever the tuning)
};

int64_t leaf_cap(int64_t n, int algo)
{
    (void)algo;
    return n;  // tiles hold 1..TILE points, dense cells any number
}

// bytes of a sorted point, a box and a node record in `dim` dimensions
void record_sizes(int dim, size_t* pt, size_t* box, size_t* node)
{
#define SIZES(D)                                       \
    do {                                               \
        *pt = sizeof(typename Traits<D>::Point);       \
        *box = sizeof(typename Traits<D>::Box);        \
        *node = sizeof(typename Traits<D>::Node);      \
    } while (0)
    GBD_DIM_SWITCH(dim, SIZES)
#undef SIZES
}

size_t carve_plan(Plan& p, void* base, int64_t n, int dim, int algo, int lcap, bool counts = false)
{
    Carver c(base);
    const int64_t mc = leaf_cap(n, algo);
    size_t pt = 0, box = 0, node = 0;
    record_sizes(dim, &pt, &box, &node);
    p.ctrl = c.take<uint32_t>(CTRL_WORDS);
    p.keys = c.take<uint64_t>(n);
    p.keys_alt = c.take<uint64_t>(n);
    p.vals = c.take<uint32_t>(n);
    p.vals_alt = c.take<uint32_t>(n);
    p.hist = c.take<uint32_t>(SORT_MAX_PASSES * SORT_RADIX);
    p.counters = c.take<uint32_t>(8);
    p.status = c.take<uint32_t>(sort_status_words(n, 8, 64));
    p.sp = c.take<char>(pt * (size_t)n);
    if (algo != DBSCAN_ALGO_FDBSCAN) {  // DenseBox, or possibly (automatic choice)
        p.db.pdense = c.take<uint8_t>(n);
        p.db.dstart = c.take<int32_t>(n);
    } else {
        p.db = DenseBoxTemps{};
    }
    p.db.lf = c.take<int32_t>(n + 64);
    p.db.lidx = c.take<int32_t>(n);
    p.db.lstart = c.take<int32_t>(n + 1);
    p.db.scan_temp = c.take<int32_t>(scan_temp_words(n));
    p.leafr = c.take<int2>(mc);
    p.lkey = c.take<uint64_t>(mc);
    p.nodebox = c.take<char>(box * (size_t)(2 * mc));
    p.nodes = c.take<char>(node * (size_t)mc);
    p.nmeta = c.take<int4>(mc);
    p.parent = c.take<int32_t>(2 * mc);
    p.nfirst = c.take<int32_t>(mc);
    p.nsum = c.take<char>(box * (size_t)sum_levels_entries(mc));
    p.lsolid = c.take<uint8_t>(mc);
    p.klist = c.take<int32_t>(mc);
    p.tstart = c.take<int32_t>(mc);
    p.tsib = c.take<int2>(mc * TRAVERSAL_SIBCAP);
    p.tnsib = c.take<int8_t>(mc);
    p.llist = c.take<int32_t>(mc * TRAVERSAL_LEAFCAP);
    p.lcount = c.take<int16_t>(mc);
    p.labels = c.take<int32_t>(n);
    p.core = c.take<uint8_t>(n);
    p.nbr = c.take<uint8_t>(n);
    p.canon = c.take<int32_t>(n);
    p.nlist = c.take<int32_t>(n * lcap);
    p.ncount = counts ? c.take<int32_t>(n) : nullptr;
    p.est.table = c.take<unsigned long long>(EST_SLOTS);
    p.est.slot = c.take<int32_t>(EST_SAMPLES);
    p.est.counts = c.take<uint32_t>(EST_SLOTS);
    p.est.result = c.take<uint32_t>(4);
    p.grid = c.take<GridParams>(1);
    p.grid_est = c.take<GridParams>(1);
    return c.off + 256;
}

size_t workspace_bytes(int64_t n, int dim, int algo, int min_pts, int mode)
{
    Plan p;
    return carve_plan(p, nullptr, n, dim, algo, list_cap(min_pts, mode));
}

size_t workspace_bytes_multi(int64_t n, int dim, int algo, int max_min_pts, int mode)
{
    Plan p;
    return carve_plan(p, nullptr, n, dim, algo, list_cap(max_min_pts, mode), true);
}

// ---------------------------------------------------------------------------
// per (device, stream) workspaces
// ---------------------------------------------------------------------------
namespace {

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

}  // namespace

Workspace* get_workspace(cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_ws_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second;
    Workspace* w = new Workspace();
    w->device = dev;
    w->stream = s;
    if (cudaMallocHost(&w->ctrl_host, CTRL_WORDS * sizeof(uint32_t)) != cudaSuccess) {
        delete w;
        return nullptr;
    }
    memset(w->ctrl_host, 0, CTRL_WORDS * sizeof(uint32_t));
    w->prof = new ProfState();
    g_ws[key] = w;
    return w;
}

cudaError_t ensure_arena(Arena& a, size_t bytes, cudaStream_t s)
{
    if (a.cap >= bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (a.base) cudaFree(a.base);
    a.base = nullptr;
    a.cap = 0;
    size_t want = bytes + bytes / 8;  // headroom against regrowth
    e = cudaMalloc(&a.base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&a.base, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); return cudaErrorMemoryAllocation; }
        want = bytes;
    }
    a.cap = want;
    // the control block (first words of every arena layout) starts cleared
    return cudaMemsetAsync(a.base, 0, 256, s);
}

void release_stream_workspace(cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    Workspace* w = nullptr;
    {
        std::lock_guard<std::mutex> g(g_ws_mu);
        auto it = g_ws.find(std::make_pair(dev, s));
        if (it == g_ws.end()) return;
        w = it->second;
        g_ws.erase(it);
    }
    free_workspace(w);
}

void free_workspace(Workspace* w)
{
    cudaStreamSynchronize(w->stream);
    release_batch_graphs(w);
    if (w->gstream) {
        cudaStreamSynchronize(w->gstream);
        cudaStreamDestroy(w->gstream);
        cudaEventDestroy(w->fork);
        cudaEventDestroy(w->join);
    }
    if (w->main.base) cudaFree(w->main.base);
    if (w->aux.base) cudaFree(w->aux.base);
    if (w->io.base) cudaFree(w->io.base);
    if (w->ctrl_host) cudaFreeHost(w->ctrl_host);
    if (w->prof) {
        for (auto& r : w->prof->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : w->prof->pool) cudaEventDestroy(e);
        delete w->prof;
    }
    delete w;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
dbscan_status check_run_args(const void* points, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                             const void* labels_out)
{
    if (n < 0 || n >= (int64_t(1) << 30)) return set_error(DBSCAN_ERR_INVALID_ARG, "n = %lld out of range [0, 2^30)", (long long)n);
    if (dim < 2 || dim > MAX_DIM) return set_error(DBSCAN_ERR_INVALID_ARG, "dim must be in [2, 8] (got %d)", dim);
    if (!(eps > 0.0f) || !std::isfinite(eps)) return set_error(DBSCAN_ERR_INVALID_ARG, "eps must be positive and finite");
    if (min_pts < 1) return set_error(DBSCAN_ERR_INVALID_ARG, "min_pts must be >= 1 (got %d)", min_pts);
    if (mode != DBSCAN_MODE_DBSCAN && mode != DBSCAN_MODE_DBSCAN_STAR)
        return set_error(DBSCAN_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (algo != DBSCAN_ALGO_FDBSCAN && algo != DBSCAN_ALGO_DENSEBOX && algo != DBSCAN_ALGO_AUTO)
        return set_error(DBSCAN_ERR_INVALID_ARG, "unknown algo %d", algo);
    if (n > 0 && (!points || !labels_out)) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    return DBSCAN_OK;
}

// Bits per axis of the DenseBox cell keys: the Morton width of 64-bit keys
// (21 in 3D, 31 in 2D, 63 / dim above), and no more than what leaves room for
// the point index beside the key in one word, so that the keys-only sort of
// packed words always applies (the grid is coarsened on the device to fit;
// the per-cell guard keeps the result exact for any cell size).
int densebox_axis_bits(int dim, int idx_bits)
{
    const int morton = dim == 3 ? 21 : (dim == 2 ? 31 : 63 / dim);
    const int fit = (64 - idx_bits) / dim;
    return morton < fit ? morton : fit;
}

int index_bits(int64_t n)
{
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < n) ++b;
    return b;
}

// ---------------------------------------------------------------------------
// the pipeline
// ---------------------------------------------------------------------------
enum Stage { ST_BOUNDS, ST_KEYS, ST_SORT, ST_GATHER, ST_LEAVES, ST_LBVH, ST_INIT, ST_PRE, ST_MAIN, ST_FINAL };

// Stages a1-a7: bounds, keys, sort, gather, leaves (DenseBox cells dense for
// minPts = dense_mp), BVH. Fills the plan-dependent fields of `a`. Nothing
// here waits for the device: the DenseBox grid is computed from the bounds
// on the device (k_grid), the sort takes the passes the keys need there, and
// the automatic choice (DBSCAN_ALGO_AUTO) enqueues both algorithms' key,
// sort, gather and leaf stages, of which only the chosen chain runs
// (CTRL_ALGO). A non-finite coordinate or a sort that gives up sets
// CTRL_ABORT and every later stage does nothing; the next host sync point
// (dbscan_stream_status, dbscan_run_host, dbscan_run_sync) reports it.
dbscan_status build_index(Workspace* w, const Plan& p, StageTimer& T, const float* points, int64_t n, int dim,
                          float eps, int dense_mp, int algo, ClusterArgs& a, cudaStream_t s)
{
    w->last_algo = algo == DBSCAN_ALGO_AUTO ? -2 : algo;  // -2: chosen on the device
    TRY_CUDA(cudaMemsetAsync(p.ctrl + CTRL_LO, 0xff, MAX_DIM * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(p.ctrl + CTRL_HI, 0, MAX_DIM * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(p.ctrl + CTRL_M, 0, 2 * sizeof(uint32_t), s));
    launch_run_begin(p.ctrl, algo, s);
    T.begin(ST_BOUNDS);
    launch_bounds(points, n, dim, p.ctrl, s);
    T.end();
    TRY_CUDA(cudaGetLastError());
    const float e2 = eps * eps;
    const bool fd = algo != DBSCAN_ALGO_DENSEBOX, db = algo != DBSCAN_ALGO_FDBSCAN;
    const int idx_bits = index_bits(n);
    const int db_axis_bits = densebox_axis_bits(dim, idx_bits);
    const int db_key_bits = db_axis_bits * dim;
    if (algo == DBSCAN_ALGO_AUTO) {
        // the estimate's thresholds belong to the cells of Sec. 4.2 (f = 1)
        launch_grid(p.ctrl, dim, eps, 1.0f, db_axis_bits, p.grid_est, s);
        TRY_CUDA(launch_density_estimate(points, n, dim, p.grid_est, dense_mp, g_tuning.auto_fraction[dim],
                                         g_tuning.auto_occupancy[dim], p.est, p.ctrl, s));
    }
    // (after the estimate's grid: CTRL_KEYBITS is this grid's)
    if (db) launch_grid(p.ctrl, dim, eps, t_run.cell_factor, db_axis_bits, p.grid, s);

    SortBuffers sb;
    sb.keys_alt = p.keys_alt;
    sb.vals_alt = p.vals_alt;
    sb.hist = p.hist;
    sb.status = p.status;
    sb.counters = p.counters;
    sb.err = p.ctrl + CTRL_ABORT;  // a wait that runs out stops every later stage
    sb.ctl.abort = p.ctrl + CTRL_ABORT;
    sb.ctl.gate = p.ctrl + CTRL_ALGO;
    bool in_alt = false;
    const int64_t m_cap = leaf_cap(n, algo);
    uint32_t* perm = nullptr;

    if (fd) {  // FDbscan: Morton codes of the points (Sec. 4.1)
        SortBuffers sf = sb;
        sf.ctl.gate_val = DBSCAN_ALGO_FDBSCAN;
        const int bits = fdbscan_bits(dim);
        if (dim > 3) {  // 64-bit Morton codes
            uint64_t* k64 = static_cast<uint64_t*>(p.keys);
            T.begin(ST_KEYS);
            launch_morton64(points, n, dim, p.ctrl, bits, k64, p.vals, s);
            T.end();
            T.begin(ST_SORT);
            TRY_CUDA(sort_pairs_u64(k64, p.vals, n, bits * dim, sf, s, &in_alt));
            T.end();
            const uint64_t* keys_sorted = in_alt ? static_cast<uint64_t*>(p.keys_alt) : k64;
            perm = in_alt ? p.vals_alt : p.vals;
            T.begin(ST_GATHER);
            launch_gather(points, perm, n, dim, p.sp, p.ctrl, DBSCAN_ALGO_FDBSCAN, s);
            T.end();
            T.begin(ST_LEAVES);
            TRY_CUDA(launch_tile_leaves64(keys_sorted, n, p.db, p.leafr, p.lkey, p.ctrl, s));
            T.end();
        } else {
            uint32_t* k32 = static_cast<uint32_t*>(p.keys);
            T.begin(ST_KEYS);
            launch_morton32(points, n, dim, p.ctrl, bits, k32, p.vals, s);
            T.end();
            T.begin(ST_SORT);
            TRY_CUDA(sort_pairs_u32(k32, p.vals, n, bits * dim, sf, s, &in_alt));
            T.end();
            const uint32_t* keys_sorted = in_alt ? static_cast<uint32_t*>(p.keys_alt) : k32;
            perm = in_alt ? p.vals_alt : p.vals;
            T.begin(ST_GATHER);
            launch_gather(points, perm, n, dim, p.sp, p.ctrl, DBSCAN_ALGO_FDBSCAN, s);
            T.end();
            T.begin(ST_LEAVES);
            TRY_CUDA(launch_tile_leaves(keys_sorted, n, p.db, p.leafr, p.lkey, p.ctrl, s));
            T.end();
        }
    }
    if (db) {  // DenseBox: grid-cell keys packed above the point index (Sec. 4.2)
        SortBuffers sd = sb;
        sd.ctl.gate_val = DBSCAN_ALGO_DENSEBOX;
        sd.ctl.key_bits = p.ctrl + CTRL_KEYBITS;
        uint64_t* k64 = static_cast<uint64_t*>(p.keys);
        uint64_t* k64_alt = static_cast<uint64_t*>(p.keys_alt);
        T.begin(ST_KEYS);
        // (the sort runs no pass for n <= 1)
        launch_cellkey_packed(points, n, dim, p.grid, p.ctrl, idx_bits, n > 1 ? sort_passes(db_key_bits) : 0, k64,
                              k64_alt, s);
        T.end();
        T.begin(ST_SORT);
        TRY_CUDA(sort_keys_u64(k64, n, idx_bits, db_key_bits, sd, s, &in_alt));
        T.end();
        // the permutation goes where FDbscan's would (one buffer for the
        // stages after, whichever chain ran)
        uint32_t* dperm = fd ? perm : p.vals;
        uint64_t* unpacked = in_alt ? k64 : k64_alt;
        T.begin(ST_GATHER);
        launch_gather_packed(points, in_alt ? k64_alt : k64, n, dim, idx_bits, p.sp, dperm, unpacked, p.ctrl, s);
        T.end();
        perm = dperm;
        T.begin(ST_LEAVES);
        TRY_CUDA(launch_densebox_leaves(unpacked, p.sp, n, dim, dense_mp, e2, p.db, p.leafr, p.lkey, p.ctrl, s));
        T.end();
    }
    TRY_CUDA(cudaGetLastError());
    T.begin(ST_LBVH);
    launch_lbvh(p.sp, dim, p.leafr, p.lkey, m_cap, p.ctrl, p.nmeta, p.parent, p.nfirst, p.nodebox, p.nsum, p.nodes, s);
    T.end();
    TRY_CUDA(cudaGetLastError());

    a.sp = p.sp;
    a.nodes = p.nodes;
    a.nodebox = p.nodebox;
    a.leafr = p.leafr;
    a.lsolid = p.lsolid;
    a.klist = p.klist;
    a.tstart = p.tstart;
    a.tsib = p.tsib;
    a.tnsib = p.tnsib;
    a.llist = p.llist;
    a.lcount = p.lcount;
    a.parent = p.parent;
    a.nmeta = p.nmeta;
    // (automatic choice: the DenseBox flags are all zero when FDbscan ran)
    a.pdense = db ? p.db.pdense : nullptr;
    a.dstart = db ? p.db.dstart : nullptr;
    a.perm = perm;
    a.labels = p.labels;
    a.core = p.core;
    a.nbr = p.nbr;
    a.nlist = p.nlist;
    a.canon = p.canon;
    a.ctrl = p.ctrl;
    a.n = n;
    a.m_cap = m_cap;
    a.dim = dim;
    a.e2 = e2;
    a.block = t_run.block;
    return DBSCAN_OK;
}

dbscan_status run_pipeline(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                           int algo, int32_t* labels_out, uint8_t* core_out, cudaStream_t s)
{
    const int lcap = list_cap(min_pts, mode);
    TRY_CUDA(ensure_arena(w->main, workspace_bytes(n, dim, algo, min_pts, mode), s));
    Plan p;
    carve_plan(p, w->main.base, n, dim, algo, lcap);

    StageTimer T(w, s);
    ClusterArgs a;
    dbscan_status st = build_index(w, p, T, points, n, dim, eps, min_pts, algo, a, s);
    if (st != DBSCAN_OK) return st;
    a.min_pts = min_pts;
    a.mode = mode;
    a.lcap = lcap;
    T.begin(ST_INIT);
    TRY_CUDA(launch_cluster_init(a, s));
    TRY_CUDA(launch_cluster_starts(a, s));
    T.end();
    if (min_pts > 2) {
        T.begin(ST_PRE);
        TRY_CUDA(launch_cluster_pre(a, s));
        T.end();
    }
    T.begin(ST_MAIN);
    TRY_CUDA(launch_cluster_main(a, s));
    T.end();
    T.begin(ST_FINAL);
    TRY_CUDA(launch_cluster_final(a, labels_out, core_out, s));
    T.end();
    return DBSCAN_OK;
}

// Core flags only, in input order (the first pass of slab-wise clustering):
// the index, neighbour counts capped at min_pts, and the flags they decide.
dbscan_status run_core_flags(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int algo,
                             uint8_t* core_out, int32_t* labels_scratch, cudaStream_t s)
{
    const int cap_mp = min_pts < 2 ? 2 : min_pts;
    TRY_CUDA(ensure_arena(w->main, workspace_bytes_multi(n, dim, algo, cap_mp, DBSCAN_MODE_DBSCAN_STAR), s));
    Plan p;
    carve_plan(p, w->main.base, n, dim, algo, 0, true);
    StageTimer T(w, s);
    ClusterArgs a;
    dbscan_status st = build_index(w, p, T, points, n, dim, eps, cap_mp, algo, a, s);
    if (st != DBSCAN_OK) return st;
    a.min_pts = cap_mp;
    a.mode = DBSCAN_MODE_DBSCAN_STAR;  // no lists, no claims: only the counts are wanted
    a.lcap = 0;
    a.ncount = p.ncount;
    TRY_CUDA(cudaMemsetAsync(p.ncount, 0, sizeof(int32_t) * (size_t)n, s));
    TRY_CUDA(launch_cluster_init(a, s));
    TRY_CUDA(launch_cluster_starts(a, s));
    TRY_CUDA(launch_cluster_pre(a, s));
    TRY_CUDA(launch_cluster_from_counts(a, min_pts, s));
    TRY_CUDA(launch_cluster_final(a, labels_scratch, core_out, s));
    return DBSCAN_OK;
}

// Clustering with the core flags given (device, input order): the second pass
// of slab-wise clustering, where a slab's border points take their flags from
// the slab that owns them.
dbscan_status run_with_core(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                            int algo, const uint8_t* core_in, int32_t* labels_out, cudaStream_t s)
{
    TRY_CUDA(ensure_arena(w->main, workspace_bytes(n, dim, algo, 3, DBSCAN_MODE_DBSCAN_STAR), s));
    Plan p;
    carve_plan(p, w->main.base, n, dim, algo, 0);
    StageTimer T(w, s);
    ClusterArgs a;
    dbscan_status st = build_index(w, p, T, points, n, dim, eps, min_pts, algo, a, s);
    if (st != DBSCAN_OK) return st;
    a.min_pts = min_pts < 3 ? 3 : min_pts;  // the core flags are exact: the minPts >= 3 form
    a.mode = mode;
    a.lcap = 0;
    TRY_CUDA(launch_cluster_init(a, s));
    TRY_CUDA(launch_cluster_core_from_input(a, core_in, s));
    // no preprocessing ran: every non-core point may have a core neighbour
    TRY_CUDA(cudaMemsetAsync(p.nbr, 1, (size_t)n, s));
    TRY_CUDA(launch_cluster_starts(a, s));
    TRY_CUDA(launch_cluster_main(a, s));
    TRY_CUDA(launch_cluster_final(a, labels_out, nullptr, s));
    return DBSCAN_OK;
}

// Several minPts over one index (the multi-minPts sweep): the tree is built
// once (DenseBox cells dense for the largest minPts, which makes them dense
// for every smaller one), preprocessing counts neighbours once with its early
// exit at the largest minPts (a count capped there decides core for every
// minPts in the list, and the neighbour lists stay complete for each point
// that is non-core for some of them), then each minPts takes its own core
// flags, border claims, main phase and relabel.
dbscan_status run_multi(Workspace* w, const float* points, int64_t n, int dim, float eps, const int32_t* min_pts,
                        int count, int mode, int algo, int32_t* labels_out, uint8_t* core_out, cudaStream_t s)
{
    int max_mp = 1;
    for (int k = 0; k < count; ++k)
        if (min_pts[k] > max_mp) max_mp = min_pts[k];
    const int cap_mp = max_mp < 2 ? 2 : max_mp;  // counting needs at least "a neighbour or not"
    const int lcap = list_cap(cap_mp, mode);
    TRY_CUDA(ensure_arena(w->main, workspace_bytes_multi(n, dim, algo, cap_mp, mode), s));
    Plan p;
    carve_plan(p, w->main.base, n, dim, algo, lcap, true);

    StageTimer T(w, s);
    ClusterArgs a;
    dbscan_status st = build_index(w, p, T, points, n, dim, eps, cap_mp, algo, a, s);
    if (st != DBSCAN_OK) return st;
    a.min_pts = cap_mp;
    a.mode = mode;
    a.lcap = lcap;
    a.ncount = p.ncount;
    T.begin(ST_INIT);
    TRY_CUDA(cudaMemsetAsync(p.ncount, 0, sizeof(int32_t) * (size_t)n, s));
    TRY_CUDA(launch_cluster_init(a, s));
    TRY_CUDA(launch_cluster_starts(a, s));
    T.end();
    T.begin(ST_PRE);
    TRY_CUDA(launch_cluster_pre(a, s));
    T.end();
    for (int k = 0; k < count; ++k) {
        T.begin(ST_MAIN);
        TRY_CUDA(launch_cluster_from_counts(a, min_pts[k], s));
        ClusterArgs ak = a;
        ak.min_pts = min_pts[k] < 3 ? 3 : min_pts[k];
        TRY_CUDA(launch_cluster_main(ak, s));
        T.end();
        T.begin(ST_FINAL);
        TRY_CUDA(launch_cluster_final(a, labels_out + (size_t)k * n, core_out ? core_out + (size_t)k * n : nullptr,
                                      s));
        T.end();
    }
    return DBSCAN_OK;
}

}  // namespace gbd

using namespace gbd;

namespace gbd {

// the control words open every plan (single and batched), so the error word
// sits at the same place whatever ran last
dbscan_status workspace_status(Workspace* w, cudaStream_t s)
{
    TRY_CUDA(cudaStreamSynchronize(s));
    if (!w || !w->main.base) return DBSCAN_OK;
    Plan p;
    carve_plan(p, w->main.base, 0, 3, DBSCAN_ALGO_FDBSCAN, 0);
    // the error bits of earlier runs (CTRL_ERR) and of the last one (CTRL_ABORT)
    TRY_CUDA(cudaMemcpyAsync(w->ctrl_host, p.ctrl, CTRL_WORDS * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    const uint32_t err = w->ctrl_host[CTRL_ERR] | w->ctrl_host[CTRL_ABORT];
    if (err) {
        TRY_CUDA(cudaMemsetAsync(p.ctrl + CTRL_ERR, 0, sizeof(uint32_t), s));
        TRY_CUDA(cudaMemsetAsync(p.ctrl + CTRL_ABORT, 0, sizeof(uint32_t), s));
        TRY_CUDA(cudaStreamSynchronize(s));
        if (err & ERR_NONFINITE) return set_error(DBSCAN_ERR_NONFINITE, "input coordinates contain NaN or Inf");
        return set_error(DBSCAN_ERR_DEVICE_TIMEOUT, "device error bits 0x%x", err);
    }
    return DBSCAN_OK;
}

}  // namespace gbd

namespace gbd {

// The autotuner for one kind of dbscan_run call: the candidates are measured
// on the caller's own data (one warm-up run and two timed runs each, CUDA
// events on the stream), the fastest is stored for the key and left in
// t_run. Waits for the stream (the first call of a key is a sync point);
// device-side errors of the data are returned here.
dbscan_status autotune_single(Workspace* w, const TuneKey& key, const float* points, int64_t n, int dim, float eps,
                              int min_pts, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                              cudaStream_t s)
{
    RunTuning cand[16];
    const int nc = tuning_candidates(algo, cand, 16);
    cudaEvent_t a = nullptr, b = nullptr;
    TRY_CUDA(cudaEventCreate(&a));
    TRY_CUDA(cudaEventCreate(&b));
    float best = 3.0e38f;
    RunTuning bt = DEFAULT_RUN_TUNING;
    dbscan_status st = DBSCAN_OK;
    for (int i = 0; i < nc && st == DBSCAN_OK; ++i) {
        t_run = cand[i];
        st = run_pipeline(w, points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, s);
        if (st != DBSCAN_OK) break;
        cudaEventRecord(a, s);
        for (int r = 0; r < 2 && st == DBSCAN_OK; ++r)
            st = run_pipeline(w, points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, s);
        cudaEventRecord(b, s);
        if (st != DBSCAN_OK) break;
        st = workspace_status(w, s);
        if (st != DBSCAN_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            bt = cand[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != DBSCAN_OK) return st;
    store_tuning(key, bt, best / 2.0f);
    t_run = bt;
    return DBSCAN_OK;
}

// the tuning of one dbscan_run call: measured now if the autotuner is on and
// the key is new, else from the table (or the fixed knobs)
dbscan_status prepare_single(Workspace* w, const float* points, int64_t n, int dim, float eps, int min_pts, int mode,
                             int algo, int32_t* labels_out, uint8_t* core_out, cudaStream_t s)
{
    const TuneKey key = tune_key(0, dim, n, min_pts, algo, mode, 0);
    if (autotune_on() && !tuned(key))
        return autotune_single(w, key, points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, s);
    t_run = resolve_tuning(key);
    return DBSCAN_OK;
}

// dbscan_run_host and dbscan_run_host_async: copy in, cluster, copy out on
// the stream's staging area; `wait` makes it a sync point. Without the wait
// the host buffers must be page-locked, so that the copies are asynchronous.
bool host_pinned(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

dbscan_status run_host(const float* points_host, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                       int32_t* labels_host, uint8_t* core_host, dbscan_stream stream, bool wait)
{
    t_err.clear();
    dbscan_status st = check_run_args(points_host, n, dim, eps, min_pts, mode, algo, labels_host);
    if (st != DBSCAN_OK) return st;
    if (n == 0) return DBSCAN_OK;
    if (!wait && (!host_pinned(points_host) || !host_pinned(labels_host) || (core_host && !host_pinned(core_host))))
        return set_error(DBSCAN_ERR_INVALID_ARG, "dbscan_run_host_async needs page-locked (pinned) host buffers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    const size_t pbytes = sizeof(float) * (size_t)n * dim;
    const size_t lbytes = sizeof(int32_t) * (size_t)n;
    const size_t io = ((pbytes + 255) & ~size_t(255)) + ((lbytes + 255) & ~size_t(255)) + (size_t)n + 256;
    TRY_CUDA(ensure_arena(w->io, io, s));
    char* base = static_cast<char*>(w->io.base);
    float* dpts = reinterpret_cast<float*>(base);
    int32_t* dlab = reinterpret_cast<int32_t*>(base + ((pbytes + 255) & ~size_t(255)));
    uint8_t* dcore = reinterpret_cast<uint8_t*>(base + ((pbytes + 255) & ~size_t(255)) + ((lbytes + 255) & ~size_t(255)));
    TRY_CUDA(cudaMemcpyAsync(dpts, points_host, pbytes, cudaMemcpyHostToDevice, s));
    st = prepare_single(w, dpts, n, dim, eps, min_pts, mode, algo, dlab, core_host ? dcore : nullptr, s);
    if (st != DBSCAN_OK) return st;
    st = run_pipeline(w, dpts, n, dim, eps, min_pts, mode, algo, dlab, core_host ? dcore : nullptr, s);
    if (st != DBSCAN_OK) return st;
    TRY_CUDA(cudaMemcpyAsync(labels_host, dlab, lbytes, cudaMemcpyDeviceToHost, s));
    if (core_host) TRY_CUDA(cudaMemcpyAsync(core_host, dcore, (size_t)n, cudaMemcpyDeviceToHost, s));
    if (!wait) return DBSCAN_OK;  // device-side errors: at the next sync point on the stream
    return workspace_status(w, s);  // waits for the copies, then reports the run's device errors
}

}  // namespace gbd

extern "C" {

dbscan_status dbscan_run(const float* points, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                         int32_t* labels_out, uint8_t* core_out, dbscan_stream stream)
{
    t_err.clear();
    dbscan_status st = check_run_args(points, n, dim, eps, min_pts, mode, algo, labels_out);
    if (st != DBSCAN_OK) return st;
    if (n == 0) return DBSCAN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    st = prepare_single(w, points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, s);
    if (st != DBSCAN_OK) return st;
    return run_pipeline(w, points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, s);
}

dbscan_status dbscan_run_sync(const float* points, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                              int32_t* labels_out, uint8_t* core_out, dbscan_stream stream)
{
    dbscan_status st = dbscan_run(points, n, dim, eps, min_pts, mode, algo, labels_out, core_out, stream);
    if (st != DBSCAN_OK || n == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return workspace_status(get_workspace(s), s);
}

dbscan_status dbscan_run_multi(const float* points, int64_t n, int dim, float eps, const int32_t* min_pts,
                               int32_t count, int mode, int algo, int32_t* labels_out, uint8_t* core_out,
                               dbscan_stream stream)
{
    t_err.clear();
    if (count < 0 || count > 4096) return set_error(DBSCAN_ERR_INVALID_ARG, "count must be in [0, 4096]");
    if (count > 0 && !min_pts) return set_error(DBSCAN_ERR_INVALID_ARG, "null min_pts");
    for (int32_t k = 0; k < count; ++k) {
        dbscan_status st = check_run_args(points, n, dim, eps, min_pts[k], mode, algo, labels_out);
        if (st != DBSCAN_OK) return set_error(st, "min_pts[%d]: %s", k, t_err.c_str());
    }
    if (count == 0 || n == 0) return DBSCAN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    int max_mp = 1;
    for (int32_t k = 0; k < count; ++k) max_mp = min_pts[k] > max_mp ? min_pts[k] : max_mp;
    t_run = resolve_tuning(tune_key(0, dim, n, max_mp, algo, mode, 0));
    return run_multi(w, points, n, dim, eps, min_pts, count, mode, algo, labels_out, core_out, s);
}

dbscan_status dbscan_run_slabs(const float* points_host, int64_t n, int dim, float eps, int min_pts, int mode,
                               int algo, int32_t* labels_host, uint8_t* core_host, int64_t slab_points,
                               dbscan_stream stream)
{
    t_err.clear();
    if (n < 0 || n >= (int64_t(1) << 31))
        return set_error(DBSCAN_ERR_INVALID_ARG, "n = %lld out of range [0, 2^31)", (long long)n);
    dbscan_status st = check_run_args(points_host, 0, dim, eps, min_pts, mode, algo, labels_host);
    if (st != DBSCAN_OK) return st;
    if (n > 0 && (!points_host || !labels_host || !core_host))
        return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer (points, labels and core flags are all needed)");
    if (slab_points < 0) return set_error(DBSCAN_ERR_INVALID_ARG, "slab_points must be >= 0");
    if (n == 0) return DBSCAN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    t_run = resolve_tuning(tune_key(0, dim, slab_points > 0 && slab_points < n ? slab_points : n, min_pts, algo,
                                    mode, 0));
    return run_slabs(w, points_host, n, dim, eps, min_pts, mode, algo, labels_host, core_host,
                     slab_points > 0 ? slab_points : (int64_t(1) << 26), s);
}

dbscan_status dbscan_run_host(const float* points_host, int64_t n, int dim, float eps, int min_pts, int mode,
                              int algo, int32_t* labels_host, uint8_t* core_host, dbscan_stream stream)
{
    return run_host(points_host, n, dim, eps, min_pts, mode, algo, labels_host, core_host, stream, true);
}

dbscan_status dbscan_run_host_async(const float* points_host, int64_t n, int dim, float eps, int min_pts, int mode,
                                    int algo, int32_t* labels_host, uint8_t* core_host, dbscan_stream stream)
{
    return run_host(points_host, n, dim, eps, min_pts, mode, algo, labels_host, core_host, stream, false);
}

dbscan_status dbscan_run_batch(const float* points, const int64_t* offsets, const int32_t* dims, const float* eps,
                               const int32_t* min_pts, int32_t count, int mode, int algo, int32_t* labels_out,
                               uint8_t* core_out, dbscan_stream stream)
{
    t_err.clear();
    if (count < 0) return set_error(DBSCAN_ERR_INVALID_ARG, "count must be >= 0");
    if (count == 0) return DBSCAN_OK;
    if (!offsets || !dims || !eps || !min_pts) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    if (offsets[0] != 0) return set_error(DBSCAN_ERR_INVALID_ARG, "offsets[0] must be 0");
    if (algo == DBSCAN_ALGO_AUTO)
        return set_error(DBSCAN_ERR_INVALID_ARG, "batches take an explicit algorithm (FDBSCAN or DENSEBOX)");
    int64_t coords = 0;
    for (int32_t b = 0; b < count; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < 0) return set_error(DBSCAN_ERR_INVALID_ARG, "offsets must be non-decreasing (instance %d)", b);
        if (dims[b] != 2 && dims[b] != 3)
            return set_error(DBSCAN_ERR_INVALID_ARG, "instance %d: batches take 2D or 3D instances (got %d)", b,
                             dims[b]);
        dbscan_status st = check_run_args(points, nb, dims[b], eps[b], min_pts[b], mode, algo, labels_out);
        if (st != DBSCAN_OK) return set_error(st, "instance %d: %s", b, t_err.c_str());
        coords += nb * dims[b];
    }
    if (offsets[count] >= (int64_t(1) << 31)) return set_error(DBSCAN_ERR_INVALID_ARG, "too many points in total");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    (void)coords;
    std::vector<const float*> pp((size_t)count);
    std::vector<int32_t*> lp((size_t)count);
    std::vector<uint8_t*> cp((size_t)count);
    int64_t coff = 0;
    for (int32_t b = 0; b < count; ++b) {
        pp[b] = points + coff;
        lp[b] = labels_out + offsets[b];
        cp[b] = core_out ? core_out + offsets[b] : nullptr;
        coff += (offsets[b + 1] - offsets[b]) * dims[b];
    }
    int max_mp = 1;
    for (int32_t b = 0; b < count; ++b) max_mp = min_pts[b] > max_mp ? min_pts[b] : max_mp;
    const TuneKey key = tune_key(1, 0, offsets[count], max_mp, algo, mode, count);
    if (autotune_on() && !tuned(key) && offsets[count] > 0) {
        // the autotuner for this kind of batch: each candidate is launched
        // directly, captured and replayed; the replay is timed
        RunTuning cand[16];
        const int nc = tuning_candidates(algo, cand, 16);
        cudaEvent_t ea = nullptr, eb = nullptr;
        TRY_CUDA(cudaEventCreate(&ea));
        TRY_CUDA(cudaEventCreate(&eb));
        float best = 3.0e38f;
        RunTuning bt = DEFAULT_RUN_TUNING;
        dbscan_status st = DBSCAN_OK;
        for (int i = 0; i < nc && st == DBSCAN_OK; ++i) {
            t_run = cand[i];
            for (int r = 0; r < 2 && st == DBSCAN_OK; ++r)
                st = run_batch(w, count, offsets, pp.data(), dims, eps, min_pts, lp.data(),
                               core_out ? cp.data() : nullptr, mode, algo, s);
            if (st != DBSCAN_OK) break;
            cudaEventRecord(ea, s);
            st = run_batch(w, count, offsets, pp.data(), dims, eps, min_pts, lp.data(), core_out ? cp.data() : nullptr,
                           mode, algo, s);
            cudaEventRecord(eb, s);
            if (st == DBSCAN_OK) st = workspace_status(w, s);
            if (st != DBSCAN_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ea, eb);
            if (ms < best) {
                best = ms;
                bt = cand[i];
            }
        }
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        if (st != DBSCAN_OK) return st;
        store_tuning(key, bt, best);
    }
    t_run = resolve_tuning(key);
    return run_batch(w, count, offsets, pp.data(), dims, eps, min_pts, lp.data(), core_out ? cp.data() : nullptr,
                     mode, algo, s);
}

dbscan_status dbscan_stream_status(dbscan_stream stream)
{
    t_err.clear();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return gbd::workspace_status(get_workspace(s), s);
}

dbscan_status dbscan_release_workspaces(void)
{
    t_err.clear();
    std::lock_guard<std::mutex> g(g_ws_mu);
    for (auto& kv : g_ws) free_workspace(kv.second);
    g_ws.clear();
    return DBSCAN_OK;
}

const char* dbscan_last_error(void) { return t_err.c_str(); }

dbscan_status dbscan_profile_enable(int on)
{
    g_profile.store(on != 0);
    return DBSCAN_OK;
}

dbscan_status dbscan_profile_collect(dbscan_stream stream, double* ms_out, int64_t* launches_out)
{
    t_err.clear();
    if (!ms_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null ms_out");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TRY_CUDA(cudaStreamSynchronize(s));
    Workspace* w = get_workspace(s);
    for (int i = 0; i < DBSCAN_PROFILE_STAGES; ++i) {
        ms_out[i] = 0.0;
        if (launches_out) launches_out[i] = 0;
    }
    if (!w) return DBSCAN_OK;
    for (auto& r : w->prof->recs) {
        float ms = 0.f;
        TRY_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        ms_out[r.stage] += ms;
        if (launches_out) launches_out[r.stage] += 1;
        w->prof->pool.push_back(r.a);
        w->prof->pool.push_back(r.b);
    }
    w->prof->recs.clear();
    return DBSCAN_OK;
}

const char* dbscan_profile_stage_name(int stage)
{
    return (stage >= 0 && stage < DBSCAN_PROFILE_STAGES) ? kStageNames[stage] : "";
}

int64_t dbscan_kernel_launches(void) { return launches_so_far(); }

dbscan_status dbscan_last_stats(dbscan_stream stream, int64_t* stats_out)
{
    t_err.clear();
    if (!stats_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null stats_out");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TRY_CUDA(cudaStreamSynchronize(s));
    Workspace* w = get_workspace(s);
    stats_out[0] = stats_out[1] = 0;
    if (!w || !w->main.base) return DBSCAN_OK;
    uint32_t ctrl[CTRL_WORDS];
    TRY_CUDA(cudaMemcpy(ctrl, w->main.base, sizeof(ctrl), cudaMemcpyDeviceToHost));
    stats_out[0] = ctrl[CTRL_M];
    stats_out[1] = ctrl[CTRL_NCELLS];
    return DBSCAN_OK;
}

dbscan_status dbscan_last_choice(dbscan_stream stream, int* algo_out, float* estimates_out)
{
    t_err.clear();
    if (!algo_out || !estimates_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    *algo_out = w ? w->last_algo : -1;
    estimates_out[0] = -1.0f;
    estimates_out[1] = -1.0f;
    if (w && w->last_algo == -2 && w->main.base) {  // chosen on the device: wait and read it
        TRY_CUDA(cudaStreamSynchronize(s));
        TRY_CUDA(cudaMemcpyAsync(w->ctrl_host, w->main.base, CTRL_WORDS * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                 s));
        TRY_CUDA(cudaStreamSynchronize(s));
        const uint32_t a = w->ctrl_host[CTRL_ALGO];
        *algo_out = (a == DBSCAN_ALGO_FDBSCAN || a == DBSCAN_ALGO_DENSEBOX) ? (int)a : -1;
        memcpy(&estimates_out[0], &w->ctrl_host[CTRL_EST_FRAC], sizeof(float));
        memcpy(&estimates_out[1], &w->ctrl_host[CTRL_EST_OCC], sizeof(float));
    }
    return DBSCAN_OK;
}

dbscan_status dbscan_traversal_counters(uint64_t* out, int cap)
{
    t_err.clear();
    if (!out || cap < CNT_PHASES * CNT_KINDS) return set_error(DBSCAN_ERR_INVALID_ARG, "need 12 output words");
    if (!counters_built())
        return set_error(DBSCAN_ERR_NOT_FOUND, "this library was built without traversal counters (GBD_COUNTERS)");
    TRY_CUDA(counters_take(out));
    return DBSCAN_OK;
}

dbscan_status dbscan_test_sort_hooks(int64_t wait_limit, int stall_first_tile)
{
    t_err.clear();
    sort_set_test_hooks(wait_limit, stall_first_tile);
    return DBSCAN_OK;
}

dbscan_status dbscan_set_auto_threshold(int dim, float dense_fraction, float occupancy)
{
    t_err.clear();
    if (dim < 2 || dim > MAX_DIM) return set_error(DBSCAN_ERR_INVALID_ARG, "dim must be in [2, 8] (got %d)", dim);
    if (dense_fraction < 0.0f && occupancy < 0.0f) {  // restore the defaults
        g_tuning.auto_fraction[dim] = dim == 2 ? DEFAULT_AUTO_FRACTION_2D : DEFAULT_AUTO_FRACTION_3D;
        g_tuning.auto_occupancy[dim] = DEFAULT_AUTO_OCCUPANCY;
        return DBSCAN_OK;
    }
    if (!(dense_fraction >= 0.0f && dense_fraction <= 1.0f))
        return set_error(DBSCAN_ERR_INVALID_ARG, "dense_fraction must be in [0, 1]");
    if (!(occupancy >= 0.0f) || std::isinf(occupancy))
        return set_error(DBSCAN_ERR_INVALID_ARG, "occupancy must be finite and >= 0");
    g_tuning.auto_fraction[dim] = dense_fraction;
    g_tuning.auto_occupancy[dim] = occupancy;
    return DBSCAN_OK;
}

dbscan_status dbscan_set_border_lists(int on)
{
    t_err.clear();
    if (on != 0 && on != 1) return set_error(DBSCAN_ERR_INVALID_ARG, "on must be 0 or 1");
    g_tuning.border_lists = on;
    return DBSCAN_OK;
}

int dbscan_border_lists(void) { return g_tuning.border_lists; }

dbscan_status dbscan_set_tuning(int block_size, float cell_factor)
{
    t_err.clear();
    if (block_size != 0 && (block_size < 32 || block_size > 1024 || block_size % 32 != 0))
        return set_error(DBSCAN_ERR_INVALID_ARG, "block size must be a multiple of 32 in [32, 1024]");
    if (cell_factor != 0.0f && !(cell_factor > 0.0f && cell_factor <= 1.0f))
        return set_error(DBSCAN_ERR_INVALID_ARG, "cell factor must be in (0, 1]");
    g_tuning.block = block_size;
    g_tuning.cell_factor = cell_factor;
    return DBSCAN_OK;
}

dbscan_status dbscan_tuning_lookup(int batch, int dim, int64_t n, int min_pts, int mode, int algo, int64_t count,
                                   int* block_out, float* cell_factor_out, float* ms_out)
{
    t_err.clear();
    if (!block_out || !cell_factor_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null argument");
    const TuneKey key = tune_key(batch ? 1 : 0, batch ? 0 : dim, n, min_pts, algo, mode, count);
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return set_error(DBSCAN_ERR_NOT_FOUND, "no autotuned entry for this kind of call");
    *block_out = it->second.t.block;
    *cell_factor_out = it->second.t.cell_factor;
    if (ms_out) *ms_out = it->second.ms;
    return DBSCAN_OK;
}

dbscan_status dbscan_tuning_clear(void)
{
    t_err.clear();
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
    return DBSCAN_OK;
}

// ---------------------------------------------------------------------------
// component entry points
// ---------------------------------------------------------------------------
dbscan_status dbscan_sort_pairs_u64(uint64_t* keys, uint32_t* values, int64_t n, int key_bits, dbscan_stream stream)
{
    t_err.clear();
    if (n < 0 || n >= (int64_t(1) << 30)) return set_error(DBSCAN_ERR_INVALID_ARG, "n out of range");
    if (key_bits < 0 || key_bits > 64) return set_error(DBSCAN_ERR_INVALID_ARG, "key_bits must be in [0, 64]");
    if (n > 0 && (!keys || !values)) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    if (n <= 1 || key_bits == 0) return DBSCAN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    Carver c(nullptr);
    c.take<uint64_t>(n); c.take<uint32_t>(n); c.take<uint32_t>(SORT_MAX_PASSES * SORT_RADIX); c.take<uint32_t>(8);
    c.take<uint32_t>(sort_status_words(n, 8, key_bits)); c.take<uint32_t>(CTRL_WORDS);
    TRY_CUDA(ensure_arena(w->aux, c.off + 256, s));
    Carver d(w->aux.base);
    SortBuffers sb;
    sb.keys_alt = d.take<uint64_t>(n);
    sb.vals_alt = d.take<uint32_t>(n);
    sb.hist = d.take<uint32_t>(SORT_MAX_PASSES * SORT_RADIX);
    sb.counters = d.take<uint32_t>(8);
    sb.status = d.take<uint32_t>(sort_status_words(n, 8, key_bits));
    uint32_t* ctrl = d.take<uint32_t>(CTRL_WORDS);
    sb.err = ctrl + CTRL_ERR;
    TRY_CUDA(cudaMemsetAsync(ctrl, 0, CTRL_WORDS * sizeof(uint32_t), s));
    bool in_alt = false;
    TRY_CUDA(sort_pairs_u64(keys, values, n, key_bits, sb, s, &in_alt));
    if (in_alt) {
        TRY_CUDA(cudaMemcpyAsync(keys, sb.keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        TRY_CUDA(cudaMemcpyAsync(values, sb.vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    uint32_t err = 0;
    TRY_CUDA(cudaMemcpyAsync(&err, ctrl + CTRL_ERR, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (err) return set_error(DBSCAN_ERR_DEVICE_TIMEOUT, "radix sort look-back gave up (bits 0x%x)", err);
    return DBSCAN_OK;
}

dbscan_status dbscan_morton_codes(const float* points, int64_t n, int dim, const float* lo, const float* hi, int bits,
                                  uint64_t* codes_out, dbscan_stream stream)
{
    t_err.clear();
    if (n < 0 || (dim != 2 && dim != 3)) return set_error(DBSCAN_ERR_INVALID_ARG, "bad n or dim");
    if (bits < 1 || dim * bits > 64) return set_error(DBSCAN_ERR_INVALID_ARG, "need 1 <= bits and dim*bits <= 64");
    if (n > 0 && (!points || !codes_out || !lo || !hi)) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    if (n == 0) return DBSCAN_OK;
    GridParams g{};
    const float cells = std::ldexp(1.0f, bits);
    for (int k = 0; k < dim; ++k) {
        g.lo[k] = lo[k];
        const float ext = hi[k] - lo[k];
        g.scale[k] = ext > 0.0f ? cells / ext : 0.0f;
        g.cmax[k] = (uint32_t)(std::ldexp(1.0, bits) - 1.0);
    }
    g.bits = bits;
    launch_morton_generic(points, n, dim, g, codes_out, static_cast<cudaStream_t>(stream));
    TRY_CUDA(cudaGetLastError());
    return DBSCAN_OK;
}

dbscan_status dbscan_lbvh_topology(const uint64_t* leaf_keys, int64_t m, int32_t* children_out, int32_t* range_out,
                                   dbscan_stream stream)
{
    t_err.clear();
    if (m < 2 || m >= (int64_t(1) << 30)) return set_error(DBSCAN_ERR_INVALID_ARG, "need 2 <= m < 2^30");
    if (!leaf_keys || !children_out || !range_out) return set_error(DBSCAN_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace* w = get_workspace(s);
    if (!w) return set_error(DBSCAN_ERR_CUDA, "cannot create a workspace for this stream");
    Carver c(nullptr);
    c.take<int4>(m); c.take<int32_t>(2 * m);
    TRY_CUDA(ensure_arena(w->aux, c.off + 256, s));
    Carver d(w->aux.base);
    int4* nmeta = d.take<int4>(m);
    int32_t* parent = d.take<int32_t>(2 * m);
    launch_karras_only(leaf_keys, m, nmeta, parent, reinterpret_cast<int2*>(children_out),
                       reinterpret_cast<int2*>(range_out), s);
    TRY_CUDA(cudaGetLastError());
    return DBSCAN_OK;
}

}  // extern "C"
