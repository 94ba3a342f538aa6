// Batches of independent instances in one pipeline (dbscan_run_batch).
//
// All instances go through one pass of every stage instead of one pipeline
// each: keys carry the instance in their high bits, so one radix sort groups
// the points by instance and orders each instance along its own grid; tiles
// never cross instances; one Karras build over all leaves makes every
// instance one subtree (its leaves share the key prefix), whose root is where
// that instance's traversals start; the traversal kernels read eps^2 and
// minPts of each tile's instance. 2D instances are carried as 3D points with
// z = 0, which changes no distance: fl(s + fl(0 * 0)) = s.
//
// After one host wait for the per-instance bounding boxes (they size each
// instance's grid and the key width), the rest of the work is captured into
// a CUDA graph and launched; the executable graph is kept and replayed while
// the same buffers and shapes come back.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "build.cuh"
#include "capi_internal.h"

namespace gbd {

namespace {

// per-instance parameters on the device
struct InstDev {
    const float* pts;  // the instance's points (dim floats per row)
    int32_t* out;      // its labels
    uint8_t* cout;     // its core flags (or null)
    int64_t off;       // first row (in the concatenation of all instances)
    int32_t dim;
    float e2;
    int32_t min_pts;
    float lo[3];
    float scale[3];    // cell coordinate = floor((x - lo) * scale), clamped to cmax
    uint32_t cmax[3];
};

__device__ __forceinline__ int find_inst(const int64_t* __restrict__ offs, int count, int64_t row)
{
    int lo = 0, hi = count - 1;  // last b with offs[b] <= row
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float4 load_row(const InstDev& in, int64_t row)
{
    const float* p = in.pts + (row - in.off) * in.dim;
    return make_float4(p[0], p[1], in.dim == 3 ? p[2] : 0.0f, 0.0f);
}

// per-instance exact bounds (order-preserving uint min/max) and a NaN/Inf flag
__global__ void k_bbounds(const int64_t* __restrict__ offs,
                          const InstDev* __restrict__ inst, int count, int64_t n, uint32_t* __restrict__ bounds,
                          uint32_t* __restrict__ nonfinite)
{
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        const int b = valid ? find_inst(offs, count, i) : -1;
        float4 p = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        float4 q = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        bool bad = false;
        if (valid) {
            const float4 v = load_row(inst[b], i);
            bad = !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z);
            p = v;
            q = v;
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(nonfinite, 1u);
        const int b0 = __shfl_sync(FULL, b, 0);
        if (__all_sync(FULL, !valid || b == b0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                p.x = fminf(p.x, __shfl_xor_sync(FULL, p.x, o)); q.x = fmaxf(q.x, __shfl_xor_sync(FULL, q.x, o));
                p.y = fminf(p.y, __shfl_xor_sync(FULL, p.y, o)); q.y = fmaxf(q.y, __shfl_xor_sync(FULL, q.y, o));
                p.z = fminf(p.z, __shfl_xor_sync(FULL, p.z, o)); q.z = fmaxf(q.z, __shfl_xor_sync(FULL, q.z, o));
            }
            if (lane == 0 && b0 >= 0) {
                uint32_t* bb = bounds + 6 * b0;
                atomicMin(bb + 0, f2ord(p.x)); atomicMin(bb + 1, f2ord(p.y)); atomicMin(bb + 2, f2ord(p.z));
                atomicMax(bb + 3, f2ord(q.x)); atomicMax(bb + 4, f2ord(q.y)); atomicMax(bb + 5, f2ord(q.z));
            }
        } else if (valid) {
            uint32_t* bb = bounds + 6 * b;
            atomicMin(bb + 0, f2ord(p.x)); atomicMin(bb + 1, f2ord(p.y)); atomicMin(bb + 2, f2ord(p.z));
            atomicMax(bb + 3, f2ord(q.x)); atomicMax(bb + 4, f2ord(q.y)); atomicMax(bb + 5, f2ord(q.z));
        }
    }
}

// key = (instance << lb) | Morton code of the point's cell in its instance's grid
__global__ void k_bkeys(const int64_t* __restrict__ offs,
                        const InstDev* __restrict__ inst, int count, int64_t n, int lb, uint64_t* __restrict__ keys,
                        uint32_t* __restrict__ vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_inst(offs, count, i);
        const InstDev in = inst[b];
        const float4 v = load_row(in, i);
        uint32_t c[3];
        c[0] = cell_index(floorf(__fmul_rn(__fsub_rn(v.x, in.lo[0]), in.scale[0])), in.cmax[0]);
        c[1] = cell_index(floorf(__fmul_rn(__fsub_rn(v.y, in.lo[1]), in.scale[1])), in.cmax[1]);
        c[2] = cell_index(floorf(__fmul_rn(__fsub_rn(v.z, in.lo[2]), in.scale[2])), in.cmax[2]);
        keys[i] = ((uint64_t)b << lb) | interleave<3>(c);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_bgather(const int64_t* __restrict__ offs,
                          const InstDev* __restrict__ inst, int count, const uint32_t* __restrict__ perm, int64_t n,
                          float4* __restrict__ sp, const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;  // a sort that gave up: stale permutation words
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = perm[i];
        sp[i] = load_row(inst[find_inst(offs, count, row)], row);
    }
}

// dense cells of every instance (see k_dense_classify): runs of equal keys,
// with the instance's minPts and eps^2
__global__ void k_bdense_classify(const uint64_t* __restrict__ keys, const float4* __restrict__ sp, int64_t n,
                                  int lb, const InstDev* __restrict__ inst, uint8_t* __restrict__ pdense,
                                  int32_t* __restrict__ dstart, uint32_t* __restrict__ ctrl)
{
    using T = Traits<3>;
    if (!stage_on(ctrl, -1)) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; base < n; base += stride) {
        const int64_t i = base + lane;
        bool cand = false;
        if (i < n) {
            const uint64_t k = keys[i];
            const int mp = inst[k >> lb].min_pts;
            const int64_t j = i + mp - 1;
            cand = (i == 0 || keys[i - 1] != k) && j < n && keys[j] == k;
        }
        unsigned cm = __ballot_sync(FULL, cand);
        while (cm) {
            const int src = __ffs(cm) - 1;
            cm &= cm - 1;
            const int64_t c0 = __shfl_sync(FULL, i, src);
            const uint64_t k = keys[c0];
            const float e2 = inst[k >> lb].e2;
            typename T::Box bx = T::empty_box();
            int64_t e = c0;
            for (;;) {
                const int64_t t = e + lane;
                const bool in = t < n && keys[t] == k;
                if (in) T::grow(bx, sp[t]);
                const unsigned im = __ballot_sync(FULL, in);
                e += __popc(im);
                if (im != FULL) break;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) T::merge(bx, T::shfl_xor(bx, o));
            if (T::diag2(bx) > e2) continue;
            const uint8_t f = (e - c0 > TILE) ? 2 : 1;
            for (int64_t t = c0 + lane; t < e; t += 32) {
                pdense[t] = f;
                dstart[t] = (int32_t)c0;
            }
            if (lane == 0) atomicAdd(&ctrl[CTRL_NCELLS], 1u);
        }
    }
}

// the root of every instance's subtree: the node (or leaf) whose leaf range
// is exactly the instance's leaves
__global__ void k_inst_roots(const int2* __restrict__ range, const int32_t* __restrict__ linst,
                             const uint32_t* __restrict__ ctrl, int32_t* __restrict__ iroot)
{
    const int64_t m = ctrl[CTRL_M];
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < 2 * m - 1;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t f, l;
        if (x < m - 1) {
            f = range[x].x;
            l = range[x].y;
        } else {
            f = l = x - (m - 1);
        }
        const int b = linst[f];
        if (linst[l] == b && (f == 0 || linst[f - 1] != b) && (l == m - 1 || linst[l + 1] != b))
            iroot[b] = (int32_t)x;
    }
}

__global__ void k_binit(const uint64_t* __restrict__ keys, int lb, const InstDev* __restrict__ inst,
                        const uint8_t* __restrict__ pdense, const int32_t* __restrict__ dstart, int64_t n,
                        int32_t* __restrict__ labels, uint8_t* __restrict__ core, const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;  // a sort that gave up: stale keys would index past the instances
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (pdense && pdense[i]) {
            labels[i] = dstart[i];
            core[i] = 1;
        } else {
            labels[i] = (int32_t)i;
            core[i] = inst[keys[i] >> lb].min_pts == 1 ? 1 : 0;
        }
    }
}

// full compression and the smallest instance-relative index of a core point
// per root
__global__ void k_bfinalize(int32_t* labels, const uint8_t* __restrict__ core, const uint32_t* __restrict__ perm,
                            const uint64_t* __restrict__ keys, int lb, const InstDev* __restrict__ inst, int64_t n,
                            int32_t* __restrict__ canon, const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + (threadIdx.x & 31);
        const bool in = i < n;
        const int r = in ? uf_find(labels, (int)i) : 0;
        const int32_t v = in ? (int32_t)((int64_t)perm[i] - inst[keys[i] >> lb].off) : 0;
        warp_atomic_min(canon, r, v, in && core[i]);
    }
}

// outputs of every instance, in its own buffers (instance-relative labels)
__global__ void k_brelabel(const int32_t* labels, const uint8_t* __restrict__ core, const uint32_t* __restrict__ perm,
                           const uint64_t* __restrict__ keys, int lb, const InstDev* __restrict__ inst, int64_t n,
                           int mode, const int32_t* __restrict__ canon, const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;  // aborted batch: nothing is written
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool c = core[i] != 0;
        const int r = uf_root(labels, (int)i);
        const bool member = c || (mode == DBSCAN_MODE_DBSCAN && r != (int)i);
        const InstDev& in = inst[keys[i] >> lb];
        const int64_t o = (int64_t)perm[i] - in.off;
        in.out[o] = member ? canon[r] : -1;
        if (in.cout) in.cout[o] = c ? 1 : 0;
    }
}

unsigned grid_n(int64_t work, int threads = 256, int max_blocks = 152 * 16)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

struct BCarver {
    char* base;
    size_t off = 0;
    explicit BCarver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};

// device buffers of one batch
struct BatchPlan {
    uint32_t* ctrl;
    uint64_t* keys;
    uint64_t* keys_alt;
    uint32_t* vals;
    uint32_t* vals_alt;
    uint32_t* hist;
    uint32_t* counters;
    uint32_t* status;
    float4* sp;
    DenseBoxTemps db;
    int2* leafr;
    uint64_t* lkey;
    int32_t* linst;
    void* nodebox;
    void* nodes;
    int4* nmeta;
    int32_t* parent;
    int32_t* nfirst;  // first leaf of each internal node
    void* nsum;       // block summaries of the leaf boxes
    int2* range;
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
    uint32_t* bounds;   // count * 6 (+1: the non-finite flag)
    int64_t* offs;      // count + 1
    InstDev* inst;      // count
    float* e2s;         // count
    int32_t* mps;       // count
    int32_t* iroot;     // count
    int32_t* nlist;     // n * lcap
};

size_t carve_batch(BatchPlan& p, void* base, int64_t n, int count, int algo, int lcap)
{
    BCarver c(base);
    p.ctrl = c.take<uint32_t>(CTRL_WORDS);
    p.keys = c.take<uint64_t>(n);
    p.keys_alt = c.take<uint64_t>(n);
    p.vals = c.take<uint32_t>(n);
    p.vals_alt = c.take<uint32_t>(n);
    p.hist = c.take<uint32_t>(SORT_MAX_PASSES * SORT_RADIX);
    p.counters = c.take<uint32_t>(8);
    p.status = c.take<uint32_t>(sort_status_words(n, 8, 64));
    p.sp = c.take<float4>(n);
    p.db = DenseBoxTemps{};
    if (algo == DBSCAN_ALGO_DENSEBOX) {
        p.db.pdense = c.take<uint8_t>(n);
        p.db.dstart = c.take<int32_t>(n);
    }
    p.db.lf = c.take<int32_t>(n + 64);
    p.db.lidx = c.take<int32_t>(n);
    p.db.lstart = c.take<int32_t>(n + 1);
    p.db.scan_temp = c.take<int32_t>(scan_temp_words(n));
    p.leafr = c.take<int2>(n);
    p.lkey = c.take<uint64_t>(n);
    p.linst = c.take<int32_t>(n);
    p.nodebox = c.take<Traits<3>::Box>(2 * n);
    p.nodes = c.take<Traits<3>::Node>(n);
    p.nmeta = c.take<int4>(n);
    p.parent = c.take<int32_t>(2 * n);
    p.nfirst = c.take<int32_t>(n);
    p.nsum = c.take<Traits<3>::Box>((size_t)sum_levels_entries(n));
    p.range = c.take<int2>(n);
    p.lsolid = c.take<uint8_t>(n);
    p.klist = c.take<int32_t>(n);
    p.tstart = c.take<int32_t>(n);
    p.tsib = c.take<int2>(n * TRAVERSAL_SIBCAP);
    p.tnsib = c.take<int8_t>(n);
    p.llist = c.take<int32_t>(n * TRAVERSAL_LEAFCAP);
    p.lcount = c.take<int16_t>(n);
    p.labels = c.take<int32_t>(n);
    p.core = c.take<uint8_t>(n);
    p.nbr = c.take<uint8_t>(n);
    p.canon = c.take<int32_t>(n);
    p.bounds = c.take<uint32_t>(6 * (size_t)count + 1);
    p.offs = c.take<int64_t>((size_t)count + 1);
    p.inst = c.take<InstDev>((size_t)count);
    p.e2s = c.take<float>((size_t)count);
    p.mps = c.take<int32_t>((size_t)count);
    p.iroot = c.take<int32_t>((size_t)count);
    p.nlist = c.take<int32_t>(n * lcap);
    return c.off + 256;
}

// The graph of the stages after the bounds, kept per workspace.
// what a captured graph depends on (the instances' buffers are read from the
// device-side instance table, so they are not part of it)
struct BatchShape {
    void* ws = nullptr;
    int64_t n = 0;
    int count = 0, mode = -1, algo = -1, lb = 0, key_bits = 0, max_mp = 0, block = 0;
    bool operator==(const BatchShape& o) const
    {
        return ws == o.ws && n == o.n && count == o.count && mode == o.mode && algo == o.algo && lb == o.lb &&
               key_bits == o.key_bits && max_mp == o.max_mp && block == o.block;
    }
};

// Per workspace: the captured graph and the shape of the previous call. A
// shape is captured when it comes twice in a row and replayed while it
// repeats; a shape seen once (the usual case for the server's merged jobs)
// is launched directly, since capture and instantiation cost more than the
// launches they save.
struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    BatchShape captured, last;
    int kernels = 0;
};

std::mutex g_graph_mu;
std::vector<std::pair<Workspace*, BatchGraph>> g_graphs;

BatchGraph* graph_of(Workspace* w)
{
    for (auto& kv : g_graphs)
        if (kv.first == w) return &kv.second;
    g_graphs.emplace_back(w, BatchGraph{});
    return &g_graphs.back().second;
}

// Enqueues every stage after the bounds for the given plan.
cudaError_t enqueue_batch_stages(const BatchPlan& p, int64_t n, int count, int mode, int algo, int lb, int key_bits,
                                 int max_mp, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.ctrl + CTRL_M, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    k_bkeys<<<grid_n(n), 256, 0, s>>>(p.offs, p.inst, count, n, lb, p.keys, p.vals);
    note_launches(1);
    SortBuffers sb;
    sb.keys_alt = p.keys_alt;
    sb.vals_alt = p.vals_alt;
    sb.hist = p.hist;
    sb.status = p.status;
    sb.counters = p.counters;
    sb.err = p.ctrl + CTRL_ABORT;  // a wait that runs out stops every later stage
    sb.ctl.abort = p.ctrl + CTRL_ABORT;
    bool in_alt = false;
    if ((e = sort_pairs_u64(p.keys, p.vals, n, key_bits, sb, s, &in_alt)) != cudaSuccess) return e;
    const uint64_t* keys = in_alt ? p.keys_alt : p.keys;
    const uint32_t* perm = in_alt ? p.vals_alt : p.vals;
    k_bgather<<<grid_n(n), 256, 0, s>>>(p.offs, p.inst, count, perm, n, p.sp, p.ctrl);
    note_launches(1);
    if (algo == DBSCAN_ALGO_DENSEBOX) {
        if ((e = cudaMemsetAsync(p.db.pdense, 0, (size_t)n, s)) != cudaSuccess) return e;
        k_bdense_classify<<<grid_n(n), 256, 0, s>>>(keys, p.sp, n, lb, p.inst, p.db.pdense, p.db.dstart, p.ctrl);
        note_launches(1);
    }
    if ((e = launch_batch_leaves(keys, n, lb, p.db, p.leafr, p.lkey, p.linst, p.ctrl, s)) != cudaSuccess) return e;
    launch_lbvh(p.sp, 3, p.leafr, p.lkey, n, p.ctrl, p.nmeta, p.parent, p.nfirst, p.nodebox, p.nsum, p.nodes, s, p.range);
    k_inst_roots<<<grid_n(2 * n), 256, 0, s>>>(p.range, p.linst, p.ctrl, p.iroot);
    note_launches(1);
    // union-find init (per point instance parameters)
    if ((e = cudaMemsetAsync(p.ctrl + CTRL_WORK_PRE, 0, (CTRL_WORK_END - CTRL_WORK_PRE) * sizeof(uint32_t), s)) !=
        cudaSuccess)
        return e;
    k_binit<<<grid_n(n), 256, 0, s>>>(keys, lb, p.inst, p.db.pdense, p.db.dstart, n, p.labels, p.core, p.ctrl);
    note_launches(1);
    if ((e = cudaMemsetAsync(p.canon, 0x7f, sizeof(int32_t) * (size_t)n, s)) != cudaSuccess) return e;
    ClusterArgs a;
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
    a.pdense = p.db.pdense;
    a.dstart = p.db.dstart;
    a.perm = perm;
    a.labels = p.labels;
    a.core = p.core;
    a.nbr = p.nbr;
    a.nlist = p.nlist;
    a.lcap = list_cap(max_mp, mode);
    a.canon = p.canon;
    a.ctrl = p.ctrl;
    a.n = n;
    a.m_cap = n;
    a.dim = 3;
    a.e2 = 0.0f;
    a.min_pts = max_mp;
    a.mode = mode;
    a.block = t_run.block;
    a.linst = p.linst;
    a.e2s = p.e2s;
    a.mps = p.mps;
    a.iroot = p.iroot;
    if ((e = launch_cluster_starts(a, s)) != cudaSuccess) return e;
    if ((e = launch_cluster_pre(a, s)) != cudaSuccess) return e;
    if ((e = launch_cluster_main(a, s)) != cudaSuccess) return e;
    k_bfinalize<<<grid_n(n), 256, 0, s>>>(p.labels, p.core, perm, keys, lb, p.inst, n, p.canon, p.ctrl);
    k_brelabel<<<grid_n(n), 256, 0, s>>>(p.labels, p.core, perm, keys, lb, p.inst, n, mode, p.canon, p.ctrl);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace

// Host side of dbscan_run_batch (arguments already checked).
dbscan_status run_batch(Workspace* w, int32_t count, const int64_t* offsets, const float* const* points,
                        const int32_t* dims, const float* eps, const int32_t* min_pts, int32_t* const* labels,
                        uint8_t* const* cores, int mode, int algo, cudaStream_t s)
{
    if (algo != DBSCAN_ALGO_FDBSCAN && algo != DBSCAN_ALGO_DENSEBOX)
        return set_error(DBSCAN_ERR_INVALID_ARG, "batches take an explicit algorithm (FDBSCAN or DENSEBOX)");
    const int64_t n = offsets[count];
    if (n == 0) return DBSCAN_OK;
    int max_mp = 1;
    for (int b = 0; b < count; ++b)
        if (min_pts[b] > max_mp) max_mp = min_pts[b];
    // one list capacity for the batch (instances with minPts <= 2 keep none)
    const int lcap = list_cap(max_mp, mode);
    BatchPlan sizing;
    cudaError_t e = ensure_arena(w->main, carve_batch(sizing, nullptr, n, count, algo, lcap), s);
    if (e != cudaSuccess) return cuda_error(e, "batch workspace");
    BatchPlan p;
    carve_batch(p, w->main.base, n, count, algo, lcap);

    // per-instance static parameters, then the bounds
    std::vector<InstDev> inst((size_t)count);
    std::vector<float> e2s((size_t)count);
    std::vector<int32_t> mps((size_t)count);
    for (int b = 0; b < count; ++b) {
        InstDev& in = inst[b];
        memset(&in, 0, sizeof(in));
        in.pts = points[b];
        in.out = labels[b];
        in.cout = cores ? cores[b] : nullptr;
        in.off = offsets[b];
        in.dim = dims[b];
        in.e2 = eps[b] * eps[b];
        in.min_pts = min_pts[b];
        e2s[b] = in.e2;
        mps[b] = in.min_pts;
    }
    std::vector<uint32_t> hb(6 * (size_t)count + 1);
    for (int b = 0; b < count; ++b)
        for (int k = 0; k < 6; ++k) hb[6 * b + k] = k < 3 ? 0xffffffffu : 0u;
    hb[6 * (size_t)count] = 0;
#define BTRY(x)                                          \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_error(e_, #x); \
    } while (0)
    BTRY(cudaMemcpyAsync(p.offs, offsets, sizeof(int64_t) * ((size_t)count + 1), cudaMemcpyHostToDevice, s));
    BTRY(cudaMemcpyAsync(p.inst, inst.data(), sizeof(InstDev) * (size_t)count, cudaMemcpyHostToDevice, s));
    BTRY(cudaMemcpyAsync(p.bounds, hb.data(), sizeof(uint32_t) * hb.size(), cudaMemcpyHostToDevice, s));
    // fold the last run's abort bits into the error word and clear them
    launch_run_begin(p.ctrl, algo, s);
    k_bbounds<<<grid_n(n), 256, 0, s>>>(p.offs, p.inst, count, n, p.bounds, p.bounds + 6 * (size_t)count);
    note_launches(1);
    uint32_t err = 0;
    BTRY(cudaMemcpyAsync(hb.data(), p.bounds, sizeof(uint32_t) * hb.size(), cudaMemcpyDeviceToHost, s));
    BTRY(cudaMemcpyAsync(&err, p.ctrl + CTRL_ERR, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BTRY(cudaStreamSynchronize(s));
    if (err) {
        BTRY(cudaMemsetAsync(p.ctrl + CTRL_ERR, 0, sizeof(uint32_t), s));
        return set_error(DBSCAN_ERR_DEVICE_TIMEOUT, "earlier work on this stream reported device error bits 0x%x",
                         err);
    }
    if (hb[6 * (size_t)count]) return set_error(DBSCAN_ERR_NONFINITE, "input coordinates contain NaN or Inf");

    // per-instance grids. FDBSCAN: 2^10 cells per axis over the instance's
    // bounds (Morton ordering); DENSEBOX: cells of side f * eps / sqrt(dim)
    // (Sec. 4.2), all instances interleaving the same number of bits per axis
    int id_bits = 0;
    while ((int64_t(1) << id_bits) < count) ++id_bits;
    const int max_axis_bits = (64 - id_bits) / 3 < 21 ? (64 - id_bits) / 3 : 21;
    int bits = 1;
    std::vector<double> hcell((size_t)count, 0.0);
    for (int b = 0; b < count; ++b) {
        if (offsets[b + 1] == offsets[b]) continue;
        double ext = 0.0;
        for (int k = 0; k < 3; ++k) ext = std::fmax(ext, (double)ord2f(hb[6 * b + 3 + k]) - (double)ord2f(hb[6 * b + k]));
        if (algo == DBSCAN_ALGO_FDBSCAN) {
            bits = 10 < max_axis_bits ? 10 : max_axis_bits;
        } else {
            const double h = (double)t_run.cell_factor * (double)eps[b] / std::sqrt((double)dims[b]);
            hcell[b] = h;
            const double cells = std::floor(ext / h) + 1.0;
            while (bits < max_axis_bits && std::ldexp(1.0, bits) < cells + 1.0) ++bits;
        }
    }
    const double maxcells = std::ldexp(1.0, bits);
    for (int b = 0; b < count; ++b) {
        InstDev& in = inst[b];
        if (offsets[b + 1] == offsets[b]) continue;
        for (int k = 0; k < 3; ++k) {
            const float lo = ord2f(hb[6 * b + k]), hi = ord2f(hb[6 * b + 3 + k]);
            in.lo[k] = lo;
            const double ext = (double)hi - (double)lo;
            if (algo == DBSCAN_ALGO_FDBSCAN) {
                in.scale[k] = ext > 0.0 ? (float)(maxcells / ext) : 0.0f;
            } else {
                double h = hcell[b];
                double ext_max = 0.0;
                for (int t = 0; t < 3; ++t)
                    ext_max = std::fmax(ext_max, (double)ord2f(hb[6 * b + 3 + t]) - (double)ord2f(hb[6 * b + t]));
                if (ext_max / h >= maxcells - 2.0) h = ext_max / (maxcells - 2.0);  // coarsen: exact anyway
                in.scale[k] = (float)(1.0 / h);
            }
            in.cmax[k] = (uint32_t)(maxcells - 1.0);
        }
    }
    const int lb = 3 * bits;
    const int key_bits = lb + id_bits;
    BTRY(cudaMemcpyAsync(p.inst, inst.data(), sizeof(InstDev) * (size_t)count, cudaMemcpyHostToDevice, s));
    BTRY(cudaMemcpyAsync(p.e2s, e2s.data(), sizeof(float) * (size_t)count, cudaMemcpyHostToDevice, s));
    BTRY(cudaMemcpyAsync(p.mps, mps.data(), sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice, s));

    // the remaining stages run on the workspace's own stream (capture is not
    // possible on the legacy default stream), forked from and joined back to
    // the caller's stream: launched directly, or as a CUDA graph when the
    // same shape repeats (BatchGraph)
    if (!w->gstream) {
        BTRY(cudaStreamCreateWithFlags(&w->gstream, cudaStreamNonBlocking));
        BTRY(cudaEventCreateWithFlags(&w->fork, cudaEventDisableTiming));
        BTRY(cudaEventCreateWithFlags(&w->join, cudaEventDisableTiming));
    }
    cudaStream_t gs = w->gstream;
    BTRY(cudaEventRecord(w->fork, s));
    BTRY(cudaStreamWaitEvent(gs, w->fork, 0));
    std::unique_lock<std::mutex> lk(g_graph_mu);
    BatchGraph* g = graph_of(w);
    BatchShape shape;
    shape.ws = w->main.base;
    shape.n = n;
    shape.count = count;
    shape.mode = mode;
    shape.algo = algo;
    shape.lb = lb;
    shape.key_bits = key_bits;
    shape.max_mp = max_mp;
    shape.block = t_run.block;
    const bool replay = g->exec && g->captured == shape;
    const bool capture = !replay && g->last == shape;
    g->last = shape;
    if (!replay && !capture) {
        lk.unlock();
        cudaError_t ce = enqueue_batch_stages(p, n, count, mode, algo, lb, key_bits, max_mp, gs);
        if (ce != cudaSuccess) return cuda_error(ce, "batch stages");
        BTRY(cudaEventRecord(w->join, gs));
        BTRY(cudaStreamWaitEvent(s, w->join, 0));
        return DBSCAN_OK;
    }
    if (capture) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        g->captured = BatchShape{};
        cudaGraph_t graph = nullptr;
        const int64_t before = launches_so_far();
        BTRY(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = enqueue_batch_stages(p, n, count, mode, algo, lb, key_bits, max_mp, gs);
        cudaError_t ee = cudaStreamEndCapture(gs, &graph);
        if (ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_error(ce, "capturing the batch");
        }
        if (ee != cudaSuccess) return cuda_error(ee, "cudaStreamEndCapture");
        cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            g->exec = nullptr;
            return cuda_error(ie, "cudaGraphInstantiate");
        }
        g->kernels = (int)(launches_so_far() - before);
        g->captured = shape;
    } else {
        note_launches(g->kernels);
    }
    BTRY(cudaGraphLaunch(g->exec, gs));
    BTRY(cudaEventRecord(w->join, gs));
    BTRY(cudaStreamWaitEvent(s, w->join, 0));
#undef BTRY
    return DBSCAN_OK;
}

size_t batch_workspace_bytes(int64_t n, int count, int algo, int lcap)
{
    BatchPlan sizing;
    return carve_batch(sizing, nullptr, n, count, algo, lcap);
}

void release_batch_graphs(Workspace* w)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->first == w) {
            if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
            g_graphs.erase(it);
            return;
        }
    }
}

}  // namespace gbd
