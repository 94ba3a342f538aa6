// Point sets larger than device memory, on one GPU (out-of-core clustering):
// the points stay in host memory and are clustered slab by slab.
//
// Partition. The points are binned along their widest axis (65,536 bins of
// equal width); consecutive bins form slabs of at most slab_points points.
// A slab's halo is every point within eps of it along that axis (the bins
// that reach eps beyond its edges, plus one bin for rounding), so the whole
// eps-neighbourhood of every point the slab owns lies in the slab and its
// halo.
//
// Pass 1 (per slab, on the device): neighbour counts of slab + halo; the
// core flags of the owned points are exact.
// Pass 2 (per slab): slab + halo clustered with every point's core flag
// taken from its owner (so a halo point is core exactly when it is core in
// the whole set). Every eps-edge between two core points has an endpoint
// owned by some slab and the other in that slab's halo or the slab itself,
// so it is found there; no slab unites points that are not connected.
// Merge (host): the clusters a core point belongs to in the slabs that hold
// it (its owner's and those where it is in the halo) are united with a
// union-find over global point indices; a border point keeps the cluster its
// owner's slab gave it (all its neighbours are in that slab and halo). Each
// cluster is labelled by the smallest global index of its core points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

#include "capi_internal.h"

namespace gbd {

namespace {

constexpr int SLAB_BINS = 65536;

// f(lo, hi, t) over contiguous chunks of [0, n) on up to 16 host threads
template <class F>
void parallel_for(int64_t n, F f)
{
    int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n < (int64_t)nt * 65536) nt = (int)std::max<int64_t>(1, n / 65536);
    if (nt <= 1) {
        f((int64_t)0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt, t); });
    for (auto& x : th) x.join();
}

int host_threads(int64_t n)
{
    int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n < (int64_t)nt * 65536) nt = (int)std::max<int64_t>(1, n / 65536);
    return nt;
}

int32_t find_readonly(const std::vector<int32_t>& parent, int32_t x)
{
    while (parent[(size_t)x] != x) x = parent[(size_t)x];
    return x;
}

int32_t uf_find_host(std::vector<int32_t>& parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

void uf_union_host(std::vector<int32_t>& parent, int32_t a, int32_t b)
{
    a = uf_find_host(parent, a);
    b = uf_find_host(parent, b);
    if (a == b) return;
    if (a < b) parent[b] = a;
    else parent[a] = b;
}

struct Slab {
    int64_t own0, own1;    // owned rows: positions [own0, own1) of the bin-sorted order
    int64_t rows0, rows1;  // slab + halo rows
};

struct Pinned {
    void* p = nullptr;
    ~Pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace

dbscan_status run_slabs(Workspace* w, const float* P, int64_t n, int dim, float eps, int min_pts, int mode, int algo,
                        int32_t* labels, uint8_t* core, int64_t slab_points, cudaStream_t s)
{
    // axis of largest extent (and the non-finite check)
    const int nt = host_threads(n);
    std::vector<float> tlo((size_t)nt * dim, std::numeric_limits<float>::infinity());
    std::vector<float> thi((size_t)nt * dim, -std::numeric_limits<float>::infinity());
    std::vector<int> tbad((size_t)nt, 0);
    parallel_for(n, [&](int64_t a, int64_t b, int t) {
        float* l = &tlo[(size_t)t * dim];
        float* h = &thi[(size_t)t * dim];
        for (int64_t i = a; i < b; ++i)
            for (int k = 0; k < dim; ++k) {
                const float v = P[i * dim + k];
                if (!std::isfinite(v)) tbad[(size_t)t] = 1;
                l[k] = std::min(l[k], v);
                h[k] = std::max(h[k], v);
            }
    });
    std::vector<float> lo((size_t)dim, std::numeric_limits<float>::infinity());
    std::vector<float> hi((size_t)dim, -std::numeric_limits<float>::infinity());
    for (int t = 0; t < nt; ++t) {
        if (tbad[(size_t)t]) return set_error(DBSCAN_ERR_NONFINITE, "input coordinates contain NaN or Inf");
        for (int k = 0; k < dim; ++k) {
            lo[k] = std::min(lo[k], tlo[(size_t)t * dim + k]);
            hi[k] = std::max(hi[k], thi[(size_t)t * dim + k]);
        }
    }
    int ax = 0;
    for (int k = 1; k < dim; ++k)
        if ((double)hi[k] - lo[k] > (double)hi[ax] - lo[ax]) ax = k;
    const double ext = (double)hi[ax] - (double)lo[ax];
    const double wbin = ext > 0.0 ? ext / SLAB_BINS : 1.0;

    // counting sort of the point indices by bin (stable)
    // per-thread histograms over contiguous chunks; chunk t's points of bin b
    // go after those of chunks < t, so the order within a bin stays the
    // input order
    std::vector<uint16_t> bin((size_t)n);
    std::vector<int64_t> th((size_t)nt * SLAB_BINS, 0);
    parallel_for(n, [&](int64_t a, int64_t b, int t) {
        int64_t* h = &th[(size_t)t * SLAB_BINS];
        for (int64_t i = a; i < b; ++i) {
            const double v = std::floor(((double)P[i * dim + ax] - (double)lo[ax]) / wbin);
            const int c = v < 0.0 ? 0 : (v >= SLAB_BINS ? SLAB_BINS - 1 : (int)v);
            bin[(size_t)i] = (uint16_t)c;
            ++h[c];
        }
    });
    std::vector<int64_t> start((size_t)SLAB_BINS + 1, 0);
    for (int c = 0; c < SLAB_BINS; ++c) {
        int64_t sum = start[(size_t)c];
        for (int t = 0; t < nt; ++t) {
            const int64_t k = th[(size_t)t * SLAB_BINS + c];
            th[(size_t)t * SLAB_BINS + c] = sum;  // chunk t's first position in bin c
            sum += k;
        }
        start[(size_t)c + 1] = sum;
    }
    std::vector<int32_t> order((size_t)n);
    parallel_for(n, [&](int64_t a, int64_t b, int t) {
        int64_t* f = &th[(size_t)t * SLAB_BINS];
        for (int64_t i = a; i < b; ++i) order[(size_t)f[bin[(size_t)i]]++] = (int32_t)i;
    });
    std::vector<uint16_t>().swap(bin);
    std::vector<int64_t>().swap(th);

    // slabs of whole bins, at most slab_points owned points (at least one bin)
    const int64_t hbins = (int64_t)std::ceil((double)eps / wbin) + 1;
    std::vector<Slab> slabs;
    int64_t max_rows = 0;
    for (int b0 = 0; b0 < SLAB_BINS;) {
        int b1 = b0 + 1;
        while (b1 < SLAB_BINS && start[(size_t)b1 + 1] - start[(size_t)b0] <= slab_points) ++b1;
        const int h0 = (int)std::max<int64_t>(0, b0 - hbins);
        const int h1 = (int)std::min<int64_t>(SLAB_BINS, b1 + hbins);
        Slab sl{start[(size_t)b0], start[(size_t)b1], start[(size_t)h0], start[(size_t)h1]};
        if (sl.own1 > sl.own0) {
            slabs.push_back(sl);
            max_rows = std::max(max_rows, sl.rows1 - sl.rows0);
        }
        b0 = b1;
    }
    if (max_rows >= (int64_t(1) << 30))
        return set_error(DBSCAN_ERR_INVALID_ARG,
                         "a slab and its halo hold %lld points (at most 2^30): lower slab_points or eps",
                         (long long)max_rows);

    // staging: pinned host rows, device rows (the workspace's io arena)
    const size_t pbytes = ((sizeof(float) * (size_t)max_rows * dim) + 255) & ~size_t(255);
    const size_t lbytes = ((sizeof(int32_t) * (size_t)max_rows) + 255) & ~size_t(255);
    const size_t cbytes = ((size_t)max_rows + 255) & ~size_t(255);
    Pinned hp, hl, hc;
    cudaError_t e;
    if ((e = cudaMallocHost(&hp.p, pbytes)) != cudaSuccess) return cuda_error(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hl.p, lbytes)) != cudaSuccess) return cuda_error(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hc.p, cbytes)) != cudaSuccess) return cuda_error(e, "cudaMallocHost");
    float* hpts = static_cast<float*>(hp.p);
    int32_t* hlab = static_cast<int32_t*>(hl.p);
    uint8_t* hcore = static_cast<uint8_t*>(hc.p);
    if ((e = ensure_arena(w->io, pbytes + lbytes + 2 * cbytes, s)) != cudaSuccess) return cuda_error(e, "slab buffers");
    char* base = static_cast<char*>(w->io.base);
    float* dpts = reinterpret_cast<float*>(base);
    int32_t* dlab = reinterpret_cast<int32_t*>(base + pbytes);
    uint8_t* dcore_in = reinterpret_cast<uint8_t*>(base + pbytes + lbytes);
    uint8_t* dcore_out = reinterpret_cast<uint8_t*>(base + pbytes + lbytes + cbytes);

    auto gather = [&](const Slab& sl) {
        const int64_t m = sl.rows1 - sl.rows0;
        parallel_for(m, [&](int64_t a, int64_t b, int) {
            for (int64_t j = a; j < b; ++j)
                std::memcpy(hpts + j * dim, P + (int64_t)order[(size_t)(sl.rows0 + j)] * dim, sizeof(float) * dim);
        });
        return cudaMemcpyAsync(dpts, hpts, sizeof(float) * (size_t)m * dim, cudaMemcpyHostToDevice, s);
    };

    // pass 1: exact core flags of the owned points
    for (const Slab& sl : slabs) {
        const int64_t m = sl.rows1 - sl.rows0;
        if ((e = gather(sl)) != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync");
        dbscan_status st = run_core_flags(w, dpts, m, dim, eps, min_pts, algo, dcore_out, dlab, s);
        if (st != DBSCAN_OK) return st;
        if ((e = cudaMemcpyAsync(hcore, dcore_out, (size_t)m, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
        parallel_for(sl.own1 - sl.own0, [&](int64_t a, int64_t b, int) {
            for (int64_t r = sl.own0 + a; r < sl.own0 + b; ++r) core[order[(size_t)r]] = hcore[r - sl.rows0];
        });
    }

    // pass 2: clusters of slab + halo with the owners' core flags
    std::vector<std::pair<int32_t, int32_t>> halo;  // (core point, its cluster's label in a slab holding it as halo)
    for (const Slab& sl : slabs) {
        const int64_t m = sl.rows1 - sl.rows0;
        if ((e = gather(sl)) != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync");
        parallel_for(m, [&](int64_t a, int64_t b, int) {
            for (int64_t j = a; j < b; ++j) hcore[j] = core[order[(size_t)(sl.rows0 + j)]];
        });
        if ((e = cudaMemcpyAsync(dcore_in, hcore, (size_t)m, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
        dbscan_status st = run_with_core(w, dpts, m, dim, eps, min_pts, mode, algo, dcore_in, dlab, s);
        if (st != DBSCAN_OK) return st;
        if ((e = cudaMemcpyAsync(hlab, dlab, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
        const int ntm = host_threads(m);
        std::vector<std::vector<std::pair<int32_t, int32_t>>> thalo((size_t)ntm);
        parallel_for(m, [&](int64_t a, int64_t b, int t) {
            for (int64_t j = a; j < b; ++j) {
                const int64_t r = sl.rows0 + j;
                const int32_t gid = order[(size_t)r];
                // slab labels are the slab's row of a core point of the cluster
                const int32_t glab = hlab[j] >= 0 ? order[(size_t)(sl.rows0 + hlab[j])] : -1;
                if (r >= sl.own0 && r < sl.own1) labels[gid] = glab;
                else if (core[gid] && glab >= 0) thalo[(size_t)t].emplace_back(gid, glab);
            }
        });
        for (auto& v : thalo) halo.insert(halo.end(), v.begin(), v.end());
    }
    dbscan_status st = workspace_status(w, s);
    if (st != DBSCAN_OK) return st;

    // merge across slabs, then the smallest global index of a core point
    std::vector<int32_t> parent((size_t)n);
    parallel_for(n, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; ++i) parent[(size_t)i] = (int32_t)i;
    });
    for (const auto& h : halo) uf_union_host(parent, labels[h.first], h.second);
    // (no more writes to parent: the finds below only read it)
    std::vector<int32_t> root((size_t)n);
    parallel_for(n, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; ++i) root[(size_t)i] = labels[i] >= 0 ? find_readonly(parent, labels[i]) : -1;
    });
    std::vector<int32_t> cmin((size_t)n, std::numeric_limits<int32_t>::max());
    for (int64_t i = 0; i < n; ++i)
        if (core[i]) cmin[(size_t)root[(size_t)i]] = std::min(cmin[(size_t)root[(size_t)i]], (int32_t)i);
    parallel_for(n, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; ++i) labels[i] = root[(size_t)i] >= 0 ? cmin[(size_t)root[(size_t)i]] : -1;
    });
    return DBSCAN_OK;
}

}  // namespace gbd
