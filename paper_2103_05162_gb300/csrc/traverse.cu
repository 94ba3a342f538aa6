// The two traversal phases of the parallel disjoint-set DBSCAN (Sec. 3.2,
// Algorithm 3) over the BVH of Sec. 4.1/4.2, plus union-find initialisation,
// final compression (Sec. 4.3) and canonical relabelling.
//
// Work is organised per BVH leaf and per warp: a leaf is either a tile of up
// to 32 sorted points outside dense cells (one point per lane) or a whole
// dense cell (Sec. 4.2). A warp takes the next leaf from a global counter
// (persistent kernels), and its 32 lanes traverse the tree together with one
// shared stack: at each node every lane tests its own point against both
// children's boxes (stored in the node record) and the warp descends where
// any lane hits. At a leaf, pairs are tested either lane-per-query (looping
// over the leaf's points) or lane-per-leaf-point (looping over the queries
// that reached the leaf), whichever needs fewer steps.
//
// Two exact shortcuts cut the pair tests in dense regions:
//  * containment: when the farthest corner of a leaf's box is within eps of a
//    query, every point of the leaf is a neighbour (no per-point tests);
//  * solid leaves: a leaf whose points are all core and already one set
//    (every dense cell, and every tile that becomes so after its own pairs
//    are united) behaves like a dense cell of Sec. 4.2: one adjacent pair
//    decides, and nothing is tested when the two sides already share a root.
//
// Preprocessing (minPts > 2 only): each point outside dense cells counts its
// neighbours (itself included) and stops at minPts; points of dense cells are
// core by construction.
// Intra: each tile unites its own pairs and records whether it is solid.
// Main: each leaf visits only the leaves with index > its own (the pair mask
// of Sec. 4.1, Figure "pair traversal"), so every pair is seen once, and
// applies the rule of Algorithm 3 as it finds each pair, with no neighbour
// list: core-core pairs are united, a core point claims a non-core neighbour
// with one compare-and-swap (Sec. 3.2).
#include "build.cuh"

namespace gbd {

namespace {

constexpr int STACK = 128;  // > the largest possible tree depth (97 for 64-bit keys + index tie-break)

// Node access and the box tests of both children at once (packed pairs: the
// left child in the low half, the right child in the high half). The general
// template covers 4 to 8 dimensions; 2 and 3 are specialised.
template <int D> struct NB {
    using T = Traits<D>;
    struct PP { f32x2 c[D]; };
    __device__ static __forceinline__ PP pack(const typename T::Point& p)
    {
        PP r;
#pragma unroll
        for (int k = 0; k < D; ++k) r.c[k] = pk2(p.c[k], p.c[k]);
        return r;
    }
    __device__ static __forceinline__ typename T::Node load(const typename T::Node* n, int i)
    {
        typename T::Node r;
#pragma unroll
        for (int k = 0; k < D; ++k) r.ax[k] = __ldg(&n[i].ax[k]);
        r.m = __ldg(&n[i].m);
        return r;
    }
    __device__ static __forceinline__ typename T::Box box_l(const typename T::Node& n)
    {
        typename T::Box b = T::empty_box();
#pragma unroll
        for (int k = 0; k < D; ++k) { b.lo.c[k] = n.ax[k].x; b.hi.c[k] = n.ax[k].z; }
        return b;
    }
    __device__ static __forceinline__ typename T::Box box_r(const typename T::Node& n)
    {
        typename T::Box b = T::empty_box();
#pragma unroll
        for (int k = 0; k < D; ++k) { b.lo.c[k] = n.ax[k].y; b.hi.c[k] = n.ax[k].w; }
        return b;
    }
    __device__ static __forceinline__ void pd2(const typename T::Node& n, const PP& p, float& dl, float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap_rn2(pk2(n.ax[0].x, n.ax[0].y), pk2(n.ax[0].z, n.ax[0].w), p.c[0]));
#pragma unroll
        for (int k = 1; k < D; ++k)
            s = add2(s, sqr2(gap_rn2(pk2(n.ax[k].x, n.ax[k].y), pk2(n.ax[k].z, n.ax[k].w), p.c[k])));
        unpk2(s, dl, dr);
    }
    __device__ static __forceinline__ void bd2(const typename T::Node& n, const typename T::Box& q, float& dl,
                                               float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap2_rn2(pk2(q.lo.c[0], q.lo.c[0]), pk2(q.hi.c[0], q.hi.c[0]), pk2(n.ax[0].x, n.ax[0].y),
                                pk2(n.ax[0].z, n.ax[0].w)));
#pragma unroll
        for (int k = 1; k < D; ++k)
            s = add2(s, sqr2(gap2_rn2(pk2(q.lo.c[k], q.lo.c[k]), pk2(q.hi.c[k], q.hi.c[k]),
                                      pk2(n.ax[k].x, n.ax[k].y), pk2(n.ax[k].z, n.ax[k].w))));
        unpk2(s, dl, dr);
    }
    __device__ static __forceinline__ float pbox(const typename T::Point& p, const typename T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_dist2(p, b);
    }
    __device__ static __forceinline__ float bbox(const typename T::Box& q, const typename T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_box_dist2(q, b);
    }
    __device__ static __forceinline__ typename T::Point shfl(const typename T::Point& p, int src)
    {
        typename T::Point r = p;
#pragma unroll
        for (int k = 0; k < D; ++k) r.c[k] = __shfl_sync(FULL, p.c[k], src);
        return r;
    }
};
template <> struct NB<3> {
    using T = Traits<3>;
    struct PP { f32x2 x, y, z; };  // a point's coordinates, each twice
    __device__ static __forceinline__ PP pack(const T::Point& p) { return PP{pk2(p.x, p.x), pk2(p.y, p.y), pk2(p.z, p.z)}; }
    __device__ static __forceinline__ T::Node load(const T::Node* n, int i)
    {
        T::Node r;
        // 64-byte records at 64-byte boundaries: two 256-bit loads
        float4 mf;
        ldg256(&n[i].a, r.a, r.b);
        ldg256(&n[i].c, r.c, mf);
        r.m = make_int4(__float_as_int(mf.x), __float_as_int(mf.y), __float_as_int(mf.z), __float_as_int(mf.w));
        return r;
    }
    __device__ static __forceinline__ T::Box box_l(const T::Node& n)
    {
        return T::Box{make_float4(n.a.x, n.b.x, n.c.x, 0.f), make_float4(n.a.z, n.b.z, n.c.z, 0.f)};
    }
    __device__ static __forceinline__ T::Box box_r(const T::Node& n)
    {
        return T::Box{make_float4(n.a.y, n.b.y, n.c.y, 0.f), make_float4(n.a.w, n.b.w, n.c.w, 0.f)};
    }
    // squared point-to-box distances of both children (box_dist2's order)
    __device__ static __forceinline__ void pd2(const T::Node& n, const PP& p, float& dl, float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap_rn2(pk2(n.a.x, n.a.y), pk2(n.a.z, n.a.w), p.x));
        s = add2(s, sqr2(gap_rn2(pk2(n.b.x, n.b.y), pk2(n.b.z, n.b.w), p.y)));
        s = add2(s, sqr2(gap_rn2(pk2(n.c.x, n.c.y), pk2(n.c.z, n.c.w), p.z)));
        unpk2(s, dl, dr);
    }
    // squared box-to-box distances of both children from q (box_box_dist2's order)
    __device__ static __forceinline__ void bd2(const T::Node& n, const T::Box& q, float& dl, float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap2_rn2(pk2(q.lo.x, q.lo.x), pk2(q.hi.x, q.hi.x), pk2(n.a.x, n.a.y), pk2(n.a.z, n.a.w)));
        s = add2(s, sqr2(gap2_rn2(pk2(q.lo.y, q.lo.y), pk2(q.hi.y, q.hi.y), pk2(n.b.x, n.b.y), pk2(n.b.z, n.b.w))));
        s = add2(s, sqr2(gap2_rn2(pk2(q.lo.z, q.lo.z), pk2(q.hi.z, q.hi.z), pk2(n.c.x, n.c.y), pk2(n.c.z, n.c.w))));
        unpk2(s, dl, dr);
    }
    __device__ static __forceinline__ float pbox(const T::Point& p, const T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_dist2(p, b.lo.x, b.lo.y, b.lo.z, b.hi.x, b.hi.y, b.hi.z);
    }
    __device__ static __forceinline__ float bbox(const T::Box& q, const T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_box_dist2(q, b.lo.x, b.lo.y, b.lo.z, b.hi.x, b.hi.y, b.hi.z);
    }
    __device__ static __forceinline__ T::Point shfl(const T::Point& p, int src)
    {
        return make_float4(__shfl_sync(FULL, p.x, src), __shfl_sync(FULL, p.y, src), __shfl_sync(FULL, p.z, src), 0.f);
    }
};
template <> struct NB<2> {
    using T = Traits<2>;
    struct PP { f32x2 x, y; };
    __device__ static __forceinline__ PP pack(const T::Point& p) { return PP{pk2(p.x, p.x), pk2(p.y, p.y)}; }
    __device__ static __forceinline__ T::Node load(const T::Node* n, int i)
    {
        T::Node r;
        r.a = __ldg(&n[i].a); r.b = __ldg(&n[i].b); r.m = __ldg(&n[i].m);
        return r;
    }
    __device__ static __forceinline__ T::Box box_l(const T::Node& n)
    {
        return T::Box{make_float4(n.a.x, n.b.x, 0.f, 0.f), make_float4(n.a.z, n.b.z, 0.f, 0.f)};
    }
    __device__ static __forceinline__ T::Box box_r(const T::Node& n)
    {
        return T::Box{make_float4(n.a.y, n.b.y, 0.f, 0.f), make_float4(n.a.w, n.b.w, 0.f, 0.f)};
    }
    __device__ static __forceinline__ void pd2(const T::Node& n, const PP& p, float& dl, float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap_rn2(pk2(n.a.x, n.a.y), pk2(n.a.z, n.a.w), p.x));
        s = add2(s, sqr2(gap_rn2(pk2(n.b.x, n.b.y), pk2(n.b.z, n.b.w), p.y)));
        unpk2(s, dl, dr);
    }
    __device__ static __forceinline__ void bd2(const T::Node& n, const T::Box& q, float& dl, float& dr)
    {
        GBD_COUNT(CNT_BOX, 2);
        f32x2 s = sqr2(gap2_rn2(pk2(q.lo.x, q.lo.x), pk2(q.hi.x, q.hi.x), pk2(n.a.x, n.a.y), pk2(n.a.z, n.a.w)));
        s = add2(s, sqr2(gap2_rn2(pk2(q.lo.y, q.lo.y), pk2(q.hi.y, q.hi.y), pk2(n.b.x, n.b.y), pk2(n.b.z, n.b.w))));
        unpk2(s, dl, dr);
    }
    __device__ static __forceinline__ float pbox(const T::Point& p, const T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_dist2(p, b.lo.x, b.lo.y, b.hi.x, b.hi.y);
    }
    __device__ static __forceinline__ float bbox(const T::Box& q, const T::Box& b)
    {
        GBD_COUNT(CNT_BOX, 1);
        return T::box_box_dist2(q, b.lo.x, b.lo.y, b.hi.x, b.hi.y);
    }
    __device__ static __forceinline__ T::Point shfl(const T::Point& p, int src)
    {
        return make_float2(__shfl_sync(FULL, p.x, src), __shfl_sync(FULL, p.y, src));
    }
};

// Up to 32 staged points by coordinate (structure of arrays): two
// neighbouring points load as one packed pair per axis.
template <int D> struct __align__(16) SoA {
    float c[D][32];
    __device__ __forceinline__ void put(int l, const typename Traits<D>::Point& p)
    {
#pragma unroll
        for (int k = 0; k < D; ++k) c[k][l] = p.c[k];
    }
    __device__ __forceinline__ void d2pair(const typename NB<D>::PP& p, int u, float& d0, float& d1) const
    {
        GBD_COUNT(CNT_DIST, 2);
        f32x2 s = sqr2(sub2(p.c[0], *reinterpret_cast<const f32x2*>(&c[0][u])));
#pragma unroll
        for (int k = 1; k < D; ++k) s = add2(s, sqr2(sub2(p.c[k], *reinterpret_cast<const f32x2*>(&c[k][u]))));
        unpk2(s, d0, d1);
    }
    __device__ __forceinline__ float d2(const typename Traits<D>::Point& p, int u) const
    {
        GBD_COUNT(CNT_DIST, 1);
        float s = sqr_rn(__fsub_rn(p.c[0], c[0][u]));
#pragma unroll
        for (int k = 1; k < D; ++k) s = __fadd_rn(s, sqr_rn(__fsub_rn(p.c[k], c[k][u])));
        return s;
    }
};
template <> struct __align__(16) SoA<3> {
    float x[32], y[32], z[32];
    __device__ __forceinline__ void put(int l, const float4& p) { x[l] = p.x; y[l] = p.y; z[l] = p.z; }
    // dist2(p, point u) and dist2(p, point u + 1) for even u (p packed)
    __device__ __forceinline__ void d2pair(const NB<3>::PP& p, int u, float& d0, float& d1) const
    {
        GBD_COUNT(CNT_DIST, 2);
        const f32x2 bx = *reinterpret_cast<const f32x2*>(&x[u]);
        const f32x2 by = *reinterpret_cast<const f32x2*>(&y[u]);
        const f32x2 bz = *reinterpret_cast<const f32x2*>(&z[u]);
        f32x2 s = sqr2(sub2(p.x, bx));
        s = add2(s, sqr2(sub2(p.y, by)));
        s = add2(s, sqr2(sub2(p.z, bz)));
        unpk2(s, d0, d1);
    }
    __device__ __forceinline__ float d2(const float4& p, int u) const { return dist2(p, make_float4(x[u], y[u], z[u], 0.f)); }
};
template <> struct __align__(16) SoA<2> {
    float x[32], y[32];
    __device__ __forceinline__ void put(int l, const float2& p) { x[l] = p.x; y[l] = p.y; }
    __device__ __forceinline__ void d2pair(const NB<2>::PP& p, int u, float& d0, float& d1) const
    {
        GBD_COUNT(CNT_DIST, 2);
        const f32x2 bx = *reinterpret_cast<const f32x2*>(&x[u]);
        const f32x2 by = *reinterpret_cast<const f32x2*>(&y[u]);
        f32x2 s = sqr2(sub2(p.x, bx));
        s = add2(s, sqr2(sub2(p.y, by)));
        unpk2(s, d0, d1);
    }
    __device__ __forceinline__ float d2(const float2& p, int u) const { return dist2(p, make_float2(x[u], y[u])); }
};

template <int D>
struct WarpMem {
    SoA<D> soa;
    typename Traits<D>::Point buf[32];
    int stack[STACK];
    uint8_t cbuf[32];
};

// Warp-cooperative stack traversal from internal node `node` with sp
// entries already on the stack. Children whose last leaf is below
// v.mask_lo are never entered (the pair mask). v.leaf(L, mask, box) gets the
// lanes that reached leaf L and its box; it returns true to stop early.
template <int D, class V>
__device__ __forceinline__ void traverse_loop(const typename Traits<D>::Node* __restrict__ nodes, int64_t m, V& v,
                                              int* stack, uint32_t* ctrl, int node, int sp)
{
    const int lane = threadIdx.x & 31;
    const int leaf0 = (int)(m - 1);
    // a traversal enters each internal node at most once; more steps than
    // that can only come from a corrupt tree: flag it and stop
    int64_t steps = 0;
    for (;;) {
        if (++steps > m) {
            if (lane == 0) atomicOr(&ctrl[CTRL_ERR], ERR_STACK);
            return;
        }
        const auto nd = NB<D>::load(nodes, node);
        GBD_COUNT(CNT_NODE, lane == 0);
        bool hl, hr;
        v.hits(nd, hl, hr);
        const unsigned ml = nd.m.z >= v.mask_lo ? __ballot_sync(FULL, hl) : 0u;
        const unsigned mr = nd.m.w >= v.mask_lo ? __ballot_sync(FULL, hr) : 0u;
        int next = -1;
        // left child, then right child; one call site of v.leaf keeps the
        // kernel's code small
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const unsigned mk = c ? mr : ml;
            if (!mk) continue;
            const int child = c ? nd.m.y : nd.m.x;
            if (child >= leaf0) {
                GBD_COUNT(CNT_LEAF, lane == 0);
                if (v.leaf(child - leaf0, mk, c ? NB<D>::box_r(nd) : NB<D>::box_l(nd))) return;
            } else if (next < 0) {
                next = child;
            } else {
                if (sp >= STACK) {
                    if (lane == 0) atomicOr(&ctrl[CTRL_ERR], ERR_STACK);
                    return;
                }
                if (lane == 0) stack[sp] = child;
                ++sp;
            }
        }
        if (next < 0) {
            if (sp == 0) return;
            __syncwarp();
            next = stack[--sp];
        }
        node = next;
    }
}

// The traversal of one leaf's points from node `start` (an internal node,
// or the leaf itself when it is a whole tree).
// a node or leaf box: one 256-bit load where it is a 32-byte record (2D, 3D)
template <int D>
__device__ __forceinline__ typename Traits<D>::Box load_box(const typename Traits<D>::Box* __restrict__ nodebox,
                                                            int64_t i)
{
    typename Traits<D>::Box b;
    if constexpr (sizeof(typename Traits<D>::Box) == 32) ldg256(&nodebox[i], b.lo, b.hi);
    else b = nodebox[i];
    return b;
}

template <int D, class V>
__device__ __forceinline__ void traverse(const typename Traits<D>::Node* __restrict__ nodes,
                                         const typename Traits<D>::Box* __restrict__ nodebox, int64_t m, V& v,
                                         int* stack, uint32_t* ctrl, int start)
{
    const int leaf0 = (int)(m - 1);
    if (start >= leaf0) {
        typename Traits<D>::Box b;
        b.lo = nodebox[start].lo;
        b.hi = nodebox[start].hi;
        v.leaf(start - leaf0, v.root_mask(), b);
        return;
    }
    traverse_loop<D>(nodes, m, v, stack, ctrl, start, 0);
}

// The traversal of one leaf's points from the subtrees roots[0 .. n) (node,
// last leaf): the siblings along the leaf's path to its start node whose
// boxes come within eps of the leaf box. Every neighbour of the leaf's points
// outside the leaf lies in one of them (k_tile_start), so the path nodes
// themselves are not visited. Roots whose leaves all precede v.mask_lo are
// skipped; leaf roots are tested lane by lane against their box.
template <int D, class V>
__device__ __forceinline__ void traverse_roots(const typename Traits<D>::Node* __restrict__ nodes,
                                               const typename Traits<D>::Box* __restrict__ nodebox, int64_t m,
                                               V& v, int* stack, uint32_t* ctrl, const int2* __restrict__ roots,
                                               int n)
{
    const int lane = threadIdx.x & 31;
    const int leaf0 = (int)(m - 1);
    int sp = 0;
    for (int j = n - 1; j >= 0; --j) {  // pushed in reverse: the nearest sibling is taken first
        const int2 r = roots[j];
        if (r.y < v.mask_lo) continue;
        if (r.x >= leaf0) {
            typename Traits<D>::Box b;
            b.lo = nodebox[r.x].lo;
            b.hi = nodebox[r.x].hi;
            const unsigned mk = __ballot_sync(FULL, v.hit_box(b));
            GBD_COUNT(CNT_LEAF, lane == 0 && mk);
            if (mk && v.leaf(r.x - leaf0, mk, b)) return;
        } else {
            if (lane == 0) stack[sp] = r.x;
            ++sp;
        }
    }
    if (sp == 0) return;
    __syncwarp();
    const int node = stack[--sp];
    traverse_loop<D>(nodes, m, v, stack, ctrl, node, sp);
}

// per leaf: at most SIBCAP sibling subtrees are recorded (more: the start
// node is used instead), and at most LEAFCAP leaves within eps
constexpr int SIBCAP = TRAVERSAL_SIBCAP;
constexpr int LEAFCAP = TRAVERSAL_LEAFCAP;

// ---------------------------------------------------------------------------
// Preprocessing visitor: count neighbours up to minPts (Sec. 3.2, 4.1, 4.2).
// ---------------------------------------------------------------------------
// The bounding box of the points of the lanes with `on` (empty if none): a
// query box for all of them at once. For p inside it every per-axis gap to a
// box is at least the box-to-box gap (monotone rounding, same order of the
// sum), so a box farther than eps from it is farther from each point.
template <int D>
__device__ __forceinline__ typename Traits<D>::Box warp_box(const typename Traits<D>::Point& p, bool on)
{
    using T = Traits<D>;
    typename T::Box b = on ? T::point_box(p) : T::empty_box();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) T::merge(b, T::shfl_xor(b, o));
    return b;
}

// the lanes of a tile of k <= 32 points
__device__ __forceinline__ unsigned tile_lanes(int k) { return k >= 32 ? FULL : ((1u << k) - 1u); }

template <int D>
struct PreV {
    using T = Traits<D>;
    using P = typename T::Point;
    const P* __restrict__ sp;
    const int2* __restrict__ leafr;
    SoA<D>* soa;
    float e2;
    int min_pts;
    int mask_lo;
    int own;  // the query tile's own leaf, already counted
    int lane;
    P p;
    bool act;
    int cnt;
    // neighbour lists (null: none): lane l's query (point qs + l) records
    // its out-of-tile neighbours while its count is below minPts, so a query
    // that ends non-core has all of them (nl <= minPts - 1 = lcap)
    int32_t* nlist;
    int lcap;
    int qs;
    int nl;

    __device__ __forceinline__ void note(int idx)
    {
        if (nl < lcap) nlist[(int64_t)(qs + lane) * lcap + nl] = idx;
        ++nl;
    }

    typename NB<D>::PP pp;  // p, packed

    __device__ __forceinline__ void hits(const typename T::Node& n, bool& hl, bool& hr) const
    {
        float dl, dr;
        NB<D>::pd2(n, pp, dl, dr);
        hl = act && dl <= e2;
        hr = act && dr <= e2;
    }
    __device__ __forceinline__ bool hit_box(const typename T::Box& b) const { return act && NB<D>::pbox(p, b) <= e2; }
    __device__ __forceinline__ unsigned root_mask() const { return __ballot_sync(FULL, act); }
    // list entries are worth a first test against the box of the active queries
    static constexpr bool PREFILTER = true;
    static constexpr bool NEEDS_SOLID = false;
    // the box of the queries active when the walk starts (set before it;
    // queries only drop out, so it stays a bound for those still counting)
    typename T::Box qbox;
    __device__ __forceinline__ typename T::Box query_box() const { return qbox; }

    __device__ __forceinline__ bool leaf(int L, unsigned mask, const typename T::Box& box)
    {
        return leaf_rec(L, mask, box, __ldg(&leafr[L]), 0);
    }
    // the same with the leaf's record (start, end) already loaded
    __device__ bool leaf_rec(int L, unsigned mask, const typename T::Box& box, int2 r, int)
    {
        if (L == own) return false;
        const int s = r.x, e = r.y & 0x7fffffff;
        mask &= __ballot_sync(FULL, act);
        // the whole leaf within eps: count it at once
        const bool cont = ((mask >> lane) & 1u) && T::far_dist2(p, box) <= e2;
        if (cont) {
            cnt += e - s;
            if (cnt >= min_pts) act = false;
            else if (nlist)
                for (int u = s; u < e; ++u) note(u);
        }
        mask &= ~__ballot_sync(FULL, cont);
        for (int c = s; c < e && mask; c += 32) {
            const int k = min(32, e - c);
            if (__popc(mask) < k) {
                // lane per leaf point, looping over the queries in `mask`
                const bool in = lane < k;
                const P rp = in ? sp[c + lane] : sp[c];
                unsigned mm = mask;
                while (mm) {
                    const int q = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const P pq = NB<D>::shfl(p, q);
                    const unsigned h = __ballot_sync(FULL, in && dist2(pq, rp) <= e2);
                    if (!h) continue;  // the common case in sparse regions: nothing to record
                    if (nlist) {
                        // each hit leaf point writes itself into q's list
                        const int at = __shfl_sync(FULL, nl, q) + __popc(h & ((1u << lane) - 1u));
                        if (((h >> lane) & 1u) && at < lcap) nlist[(int64_t)(qs + q) * lcap + at] = c + lane;
                    }
                    if (lane == q) {
                        cnt += __popc(h);
                        nl += __popc(h);
                        if (cnt >= min_pts) act = false;
                    }
                }
            } else {
                // lane per query, looping over the staged leaf points two
                // at a time (packed); a count that reaches minPts stops
                if (lane < k) soa->put(lane, sp[c + lane]);
                __syncwarp();
                if ((mask >> lane) & 1u) {
                    int u = 0;
                    for (; u + 1 < k && act; u += 2) {
                        float d0, d1;
                        soa->d2pair(pp, u, d0, d1);
                        if (d0 <= e2) {
                            if (nlist) note(c + u);
                            if (++cnt >= min_pts) act = false;
                        }
                        if (d1 <= e2 && act) {
                            if (nlist) note(c + u + 1);
                            if (++cnt >= min_pts) act = false;
                        }
                    }
                    if (u < k && act && soa->d2(p, u) <= e2) {
                        if (nlist) note(c + u);
                        if (++cnt >= min_pts) act = false;
                    }
                }
                __syncwarp();
            }
            mask &= __ballot_sync(FULL, act);
        }
        return !__any_sync(FULL, act);
    }
};

// ---------------------------------------------------------------------------
// The pair rule of Algorithm 3 (Sec. 3.2), for a pair (a, b) within eps.
// ---------------------------------------------------------------------------
struct Rule {
    int* labels;
    uint8_t* core;
    int min_pts;
    // core-to-non-core claims: DBSCAN mode, and no preprocessing lists (with
    // lists every border point has already claimed a core neighbour)
    bool claims;

    __device__ __forceinline__ void unite(int a, int b) const
    {
        if (__ldcg(labels + a) == __ldcg(labels + b)) return;  // same parent: same set
        uf_union(labels, a, b);
    }
    // pair() with a per-lane memo of the last core partner's parent: a
    // partner with the same parent is in a set already united with a (sets
    // never split), so the union is skipped. Partners come in sorted order and
    // mostly share an intra-tile root, so most unions are skipped this way.
    __device__ __forceinline__ void pair_memo(int a, bool acore, int b, bool bcore, int& last) const
    {
        if (min_pts <= 2 || (acore && bcore)) {
            if (min_pts == 2) { core[a] = 1; core[b] = 1; }
            const int lb = __ldcg(labels + b);
            if (lb == last) return;
            unite(a, b);
            last = lb;
        } else if (claims) {
            if (acore) uf_claim(labels, b, a);
            else if (bcore) uf_claim(labels, a, b);
        }
    }
    // would point x (core flag xcore) change anything by joining the solid
    // leaf whose first point is s?
    __device__ __forceinline__ bool need_solid(int x, bool xcore, int s) const
    {
        if (min_pts <= 2 || xcore) {
            int a = x, b = s;
            uf_find2(labels, a, b);
            return a != b;
        }
        return claims && __ldcg(labels + x) == x;
    }
    __device__ __forceinline__ void join_solid(int x, bool xcore, int s) const
    {
        if (min_pts <= 2 || xcore) {
            if (min_pts == 2) core[x] = 1;
            uf_union(labels, x, s);
        } else {
            uf_claim(labels, x, s);
        }
    }
};

// Main visitor for a tile that is not solid (one point per lane).
template <int D>
struct MainPtV {
    using T = Traits<D>;
    using P = typename T::Point;
    const P* __restrict__ sp;
    const int2* __restrict__ leafr;
    const uint8_t* __restrict__ lsolid;
    const uint8_t* core;
    SoA<D>* soa;
    uint8_t* cbuf;
    Rule rule;
    float e2;
    int mask_lo;  // = own leaf index + 1: only leaves after this one
    int lane;
    int sQ;       // first point of own leaf
    P p;
    int q;
    bool valid;
    bool qcore;
    int last = -1;  // pair_memo state of this lane's query

    typename NB<D>::PP pp;  // p, packed

    __device__ __forceinline__ void hits(const typename T::Node& n, bool& hl, bool& hr) const
    {
        float dl, dr;
        NB<D>::pd2(n, pp, dl, dr);
        hl = valid && dl <= e2;
        hr = valid && dr <= e2;
    }
    __device__ __forceinline__ bool hit_box(const typename T::Box& b) const { return valid && NB<D>::pbox(p, b) <= e2; }
    static constexpr bool PREFILTER = true;
    static constexpr bool NEEDS_SOLID = true;
    typename T::Box qbox;  // the box of the valid queries (set before the walk)
    __device__ __forceinline__ typename T::Box query_box() const { return qbox; }
    __device__ __forceinline__ unsigned root_mask() const { return __ballot_sync(FULL, valid); }

    __device__ __forceinline__ bool leaf(int L, unsigned mask, const typename T::Box& box)
    {
        return leaf_rec(L, mask, box, __ldg(&leafr[L]), lsolid[L]);
    }
    // the same with the leaf's record and solid flag already loaded
    __device__ bool leaf_rec(int L, unsigned mask, const typename T::Box& box, int2 r, int solid)
    {
        if (L < mask_lo) return false;
        const int s = r.x, e = r.y & 0x7fffffff;
        const bool cont = ((mask >> lane) & 1u) && T::far_dist2(p, box) <= e2;
        if (!solid) {
            const int k = e - s;
            if (__popc(mask) < k) {
                const bool in = lane < k;
                const int ri = s + lane;
                const P rp = in ? sp[ri] : sp[s];
                const bool rc = in && core[ri];
                int rlast = -1;  // pair_memo state of this lane's leaf point
                unsigned mm = mask;
                while (mm) {
                    const int qq = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const P pq = NB<D>::shfl(p, qq);
                    const bool qc = __shfl_sync(FULL, qcore, qq);
                    const bool qcont = __shfl_sync(FULL, cont, qq);
                    if (in && (qcont || dist2(pq, rp) <= e2)) rule.pair_memo(ri, rc, sQ + qq, qc, rlast);
                    __syncwarp();
                }
            } else {
                if (lane < k) { soa->put(lane, sp[s + lane]); cbuf[lane] = core[s + lane]; }
                __syncwarp();
                if ((mask >> lane) & 1u) {
                    if (cont) {
                        for (int u = 0; u < k; ++u) rule.pair_memo(q, qcore, s + u, cbuf[u] != 0, last);
                    } else {
                        // two staged points at a time (packed)
                        int u = 0;
                        for (; u + 1 < k; u += 2) {
                            float d0, d1;
                            soa->d2pair(pp, u, d0, d1);
                            if (d0 <= e2) rule.pair_memo(q, qcore, s + u, cbuf[u] != 0, last);
                            if (d1 <= e2) rule.pair_memo(q, qcore, s + u + 1, cbuf[u + 1] != 0, last);
                        }
                        if (u < k && soa->d2(p, u) <= e2) rule.pair_memo(q, qcore, s + u, cbuf[u] != 0, last);
                    }
                }
                __syncwarp();
            }
            return false;
        }
        // solid leaf: one adjacent point decides (its points are all core and
        // already one set rooted at that of its first point s)
        const bool need = ((mask >> lane) & 1u) && rule.need_solid(q, qcore, s);
        if (need && cont) rule.join_solid(q, qcore, s);
        unsigned nm = __ballot_sync(FULL, need && !cont);
        if (nm) {
            // the leaf's points in chunks, each pruned to those within eps of
            // the box of the queries (exact, reading 3); each query still
            // looking is tested against the survivors until it finds one
            for (int c = s; c < e && nm; c += 32) {
                const int j = c + lane;
                const P rp = j < e ? sp[j] : sp[c];
                const bool keep = j < e && NB<D>::pbox(rp, qbox) <= e2;
                if (!__any_sync(FULL, keep)) continue;
                unsigned mm = nm;
                while (mm) {
                    const int qq = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const P pq = NB<D>::shfl(p, qq);
                    if (__any_sync(FULL, keep && dist2(pq, rp) <= e2)) {
                        if (lane == qq) rule.join_solid(q, qcore, s);
                        nm &= ~(1u << qq);
                    }
                }
                __syncwarp();
            }
        }
        return false;
    }
};

// Main visitor for a solid tile (one point per lane, all core, one set): the
// traversal keeps per-lane point tests; at a leaf one adjacent pair decides.
template <int D>
struct MainSolidV {
    using T = Traits<D>;
    using P = typename T::Point;
    const P* __restrict__ sp;
    const int2* __restrict__ leafr;
    const uint8_t* __restrict__ lsolid;
    const uint8_t* core;
    P* buf;
    Rule rule;
    float e2;
    int mask_lo;  // = own leaf index + 1
    int lane;
    int sQ;
    P p;
    bool valid;
    typename T::Box qb;

    typename NB<D>::PP pp;  // p, packed

    __device__ __forceinline__ void hits(const typename T::Node& n, bool& hl, bool& hr) const
    {
        float dl, dr;
        NB<D>::pd2(n, pp, dl, dr);
        hl = valid && dl <= e2;
        hr = valid && dr <= e2;
    }
    __device__ __forceinline__ bool hit_box(const typename T::Box& b) const { return valid && NB<D>::pbox(p, b) <= e2; }
    // the query box is the leaf box, which every listed leaf passes
    static constexpr bool PREFILTER = false;
    __device__ __forceinline__ typename T::Box query_box() const { return qb; }
    __device__ __forceinline__ unsigned root_mask() const { return __ballot_sync(FULL, valid); }

    __device__ bool leaf(int L, unsigned mask, const typename T::Box& box)
    {
        if (L < mask_lo) return false;
        const int2 r = __ldg(&leafr[L]);
        const int s = r.x, e = r.y & 0x7fffffff;
        if (lsolid[L]) {
            int same = 0;
            if (lane == 0) {
                int a = sQ, b = s;
                uf_find2(rule.labels, a, b);
                same = a == b;
            }
            if (__shfl_sync(FULL, same, 0)) return false;
            const bool act = (mask >> lane) & 1u;
            bool found = __any_sync(FULL, act && T::far_dist2(p, box) <= e2);
            // only the leaf's points within eps of this tile's box can be
            // partners (exact pruning, reading 3)
            const unsigned lt = (1u << lane) - 1u;
            for (int c = s; c < e && !found; c += 32) {
                const int k = min(32, e - c);
                const P rp = lane < k ? sp[c + lane] : sp[c];
                const bool keep = lane < k && NB<D>::pbox(rp, qb) <= e2;
                const unsigned km = __ballot_sync(FULL, keep);
                if (!km) continue;
                const int kk = __popc(km);
                if (__popc(mask) < kk) {
                    unsigned mm = mask;
                    while (mm && !found) {
                        const int qq = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const P pq = NB<D>::shfl(p, qq);
                        found = __any_sync(FULL, keep && dist2(pq, rp) <= e2);
                    }
                } else {
                    if (keep) buf[__popc(km & lt)] = rp;
                    __syncwarp();
                    bool h = false;
                    if (act)
                        for (int u = 0; u < kk; ++u)
                            if (dist2(p, buf[u]) <= e2) { h = true; break; }
                    __syncwarp();
                    found = __any_sync(FULL, h);
                }
            }
            if (found && lane == 0) uf_union(rule.labels, sQ, s);
            __syncwarp();
            return false;
        }
        // a tile that is not solid: one lane per tile point
        const int k = e - s;
        const bool in = lane < k;
        const int ri = s + lane;
        const P rp = in ? sp[ri] : sp[s];
        const bool rc = in && core[ri];
        const bool need = in && rule.need_solid(ri, rc, sQ);
        bool found = need && T::far_dist2(rp, qb) <= e2;
        unsigned mm = mask;
        while (mm && __any_sync(FULL, need && !found)) {
            const int qq = __ffs(mm) - 1;
            mm &= mm - 1;
            const P pq = NB<D>::shfl(p, qq);
            if (need && !found && dist2(rp, pq) <= e2) found = true;
        }
        if (need && found) rule.join_solid(ri, rc, sQ);
        __syncwarp();
        return false;
    }
};

// Main visitor for a dense cell larger than a tile as the query:
// its box is tested against the nodes; its points are all core and one set.
template <int D>
struct MainBoxV {
    using T = Traits<D>;
    using P = typename T::Point;
    const P* __restrict__ sp;
    const int2* __restrict__ leafr;
    const uint8_t* __restrict__ lsolid;
    const uint8_t* core;
    P* buf;
    Rule rule;
    float e2;
    int mask_lo;  // = own leaf index + 1
    int lane;
    int sQ, eQ;
    typename T::Box qb;
    // the cell's work can be split over `parts` warps: this one takes the
    // neighbour leaves with L % parts == part
    int part = 0, parts = 1;

    __device__ __forceinline__ void hits(const typename T::Node& n, bool& hl, bool& hr) const
    {
        float dl, dr;
        NB<D>::bd2(n, qb, dl, dr);
        hl = dl <= e2;
        hr = dr <= e2;
    }
    __device__ __forceinline__ bool hit_box(const typename T::Box& b) const { return NB<D>::bbox(qb, b) <= e2; }
    // the query box is the leaf box, which every listed leaf passes
    static constexpr bool PREFILTER = false;
    __device__ __forceinline__ typename T::Box query_box() const { return qb; }
    __device__ __forceinline__ unsigned root_mask() const { return FULL; }

    __device__ bool leaf(int L, unsigned, const typename T::Box& box)
    {
        if (L < mask_lo || L % parts != part) return false;
        const int2 r = __ldg(&leafr[L]);
        const int s = r.x, e = r.y & 0x7fffffff;
        const unsigned lt = (1u << lane) - 1u;
        if (lsolid[L]) {
            // solid against solid: any adjacent cross pair unites the two sets
            int same = 0;
            if (lane == 0) {
                int a = sQ, b = s;
                uf_find2(rule.labels, a, b);
                same = a == b;
            }
            if (__shfl_sync(FULL, same, 0)) return false;
            bool found = T::box_far2(qb, box) <= e2;
            // only the cell's points within eps of the other leaf's box can
            // have a partner there, and of the other leaf only the points
            // within eps of the cell's box (exact pruning, reading 3); the
            // survivors are compacted into the staging buffer
            for (int cq = sQ; cq < eQ && !found; cq += 32) {
                const int iq = cq + lane;
                const bool inq = iq < eQ;
                const P pq = inq ? sp[iq] : sp[sQ];
                const bool near = inq && NB<D>::pbox(pq, box) <= e2;
                if (!__any_sync(FULL, near)) continue;
                for (int c = s; c < e; c += 32) {
                    const int k = min(32, e - c);
                    const P rp = lane < k ? sp[c + lane] : sp[c];
                    const bool keep = lane < k && NB<D>::pbox(rp, qb) <= e2;
                    const unsigned km = __ballot_sync(FULL, keep);
                    if (!km) continue;
                    if (keep) buf[__popc(km & lt)] = rp;
                    __syncwarp();
                    const int kk = __popc(km);
                    bool h = false;
                    if (near)
                        for (int u = 0; u < kk; ++u)
                            if (dist2(pq, buf[u]) <= e2) { h = true; break; }
                    __syncwarp();
                    if (__any_sync(FULL, h)) { found = true; break; }
                }
            }
            if (found && lane == 0) uf_union(rule.labels, sQ, s);
            __syncwarp();
            return false;
        }
        // a tile that is not solid: one lane per tile point, against the
        // cell's points within eps of the tile's box
        const int k = e - s;
        const bool in = lane < k;
        const int ri = s + lane;
        const P rp = in ? sp[ri] : sp[s];
        const bool rc = in && core[ri];
        const bool need = in && rule.need_solid(ri, rc, sQ);
        bool found = need && T::far_dist2(rp, qb) <= e2;
        if (__any_sync(FULL, need && !found)) {
            for (int cq = sQ; cq < eQ; cq += 32) {
                if (!__any_sync(FULL, need && !found)) break;
                const int kq = min(32, eQ - cq);
                const P ap = lane < kq ? sp[cq + lane] : sp[sQ];
                const bool keep = lane < kq && NB<D>::pbox(ap, box) <= e2;
                const unsigned km = __ballot_sync(FULL, keep);
                if (!km) continue;
                if (keep) buf[__popc(km & lt)] = ap;
                __syncwarp();
                const int kk = __popc(km);
                if (need && !found)
                    for (int u = 0; u < kk; ++u)
                        if (dist2(rp, buf[u]) <= e2) { found = true; break; }
                __syncwarp();
            }
        }
        if (need && found) rule.join_solid(ri, rc, sQ);
        __syncwarp();
        return false;
    }
};

template <int D>
struct DevArgs {
    const typename Traits<D>::Point* sp;
    const typename Traits<D>::Node* nodes;
    const typename Traits<D>::Box* nodebox;
    const int2* leafr;
    uint8_t* lsolid;
    int32_t* klist;
    int32_t* labels;
    uint8_t* core;
    uint8_t* nbr;
    int32_t* nlist;
    int lcap;
    uint32_t* ctrl;
    float e2;
    int min_pts;
    int mode;
    // batches of independent instances: per-leaf instance and per-instance
    // eps^2, minPts and subtree root (all null for a single instance)
    const int32_t* linst;
    const float* e2s;
    const int32_t* mps;
    const int32_t* iroot;
    // per leaf: the node its traversals start at, and the sibling subtrees
    // along the way that come within eps (k_tile_start)
    int32_t* tstart;
    int2* tsib;
    int8_t* tnsib;
    // multi-minPts runs: neighbour counts capped at min_pts (null otherwise)
    int32_t* ncount;
    // per leaf: the leaves within eps of its box (k_leaf_lists; null: none)
    int32_t* llist;
    int16_t* lcount;
};

template <int D>
__device__ __forceinline__ float box_box(const typename Traits<D>::Box& a, const typename Traits<D>::Box& b)
{
    return Traits<D>::box_box_dist2(a, b);
}
template <>
__device__ __forceinline__ float box_box<3>(const Traits<3>::Box& a, const Traits<3>::Box& b)
{
    return Traits<3>::box_box_dist2(a, b.lo.x, b.lo.y, b.lo.z, b.hi.x, b.hi.y, b.hi.z);
}
template <>
__device__ __forceinline__ float box_box<2>(const Traits<2>::Box& a, const Traits<2>::Box& b)
{
    return Traits<2>::box_box_dist2(a, b.lo.x, b.lo.y, b.hi.x, b.hi.y);
}

// eps^2, minPts and the traversal start of the tile's instance
struct TileParams {
    float e2;
    int min_pts;
    int start;
};
template <int D>
__device__ __forceinline__ TileParams tile_params(const DevArgs<D>& a, int L)
{
    if (!a.linst) return TileParams{a.e2, a.min_pts, 0};
    const int b = a.linst[L];
    return TileParams{a.e2s[b], a.mps[b], a.iroot[b]};
}

// The lowest ancestor A of each leaf such that no point outside A's subtree
// is within eps of the leaf's box: walking up from the leaf, every sibling
// subtree whose box is within eps of the leaf box (box-to-box distance, the
// same exact pruning test as the traversal) moves the start up to the
// sibling's parent. Traversals for the leaf's points (each within the leaf
// box) then start at A instead of the root and skip the levels above it,
// where only one path could lead to a neighbour.
template <int D>
__global__ void k_tile_start(DevArgs<D> a, const int32_t* __restrict__ parent, const int4* __restrict__ nmeta)
{
    using T = Traits<D>;
    const int64_t m = a.ctrl[CTRL_M];
    const int leaf0 = (int)(m - 1);
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < m; L += (int64_t)gridDim.x * blockDim.x) {
        const TileParams tp = tile_params(a, (int)L);
        int cur = leaf0 + (int)L;
        int start = cur;
        int ns = 0;  // siblings recorded (-1: more than SIBCAP)
        int2* sib_out = a.tsib + L * SIBCAP;
        const typename T::Box tb = load_box<D>(a.nodebox, cur);
        // the depth of a tree over 64-bit keys with index tie-breaks is
        // below STACK; a longer walk means a corrupt tree: start at the root
        int steps = 0;
        while (cur != tp.start) {
            const int p = parent[cur];
            if (p < 0 || ++steps > STACK) {
                start = tp.start;
                ns = -1;
                break;
            }
            const int4 nm = nmeta[p];
            const int sib = nm.x == cur ? nm.y : nm.x;
            const typename T::Box sb = load_box<D>(a.nodebox, sib);
            if (box_box<D>(tb, sb) <= tp.e2) {
                start = p;
                if (ns >= 0 && ns < SIBCAP) {
                    // the sibling and the last leaf under it
                    sib_out[ns++] = make_int2(sib, sib >= leaf0 ? sib - leaf0 : nmeta[sib].w);
                } else {
                    ns = -1;
                }
            }
            cur = p;
        }
        a.tstart[L] = start;
        a.tnsib[L] = (int8_t)ns;
    }
}

// the traversal of leaf L's points: from its recorded sibling subtrees, or
// from its start node when it has more than SIBCAP of them
// The leaves whose boxes come within eps of each leaf's box (itself
// excluded), found once per leaf by one thread walking the subtrees recorded
// by k_tile_start with the leaf box as the query (box-to-box test, exact by
// the same monotone-rounding argument). Every neighbour of a point of the
// leaf lies in one of them, so the traversals of both phases can go through
// the list instead of the tree. More than LEAFCAP leaves: count -1, and the
// phases walk the tree for that leaf.
// (each thread's walk stack lives in shared memory as column threadIdx.x of
// [depth][LL_THREADS]: lanes at different depths still fall in distinct
// banks, where a local-memory stack costs a transaction per distinct depth;
// a walk deeper than LL_STACK gives up its list, and the phases walk the
// tree for that leaf)
constexpr int LL_THREADS = 256;
constexpr int LL_STACK = 48;

template <int D>
__global__ void __launch_bounds__(LL_THREADS) k_leaf_lists(DevArgs<D> a)
{
    using T = Traits<D>;
    const int64_t m = a.ctrl[CTRL_M];
    const int leaf0 = (int)(m - 1);
    __shared__ int s_stk[LL_STACK][LL_THREADS];
    int* const stk = &s_stk[0][threadIdx.x];  // stk[k * LL_THREADS]: entry k
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < m; L += (int64_t)gridDim.x * blockDim.x) {
        const TileParams tp = tile_params(a, (int)L);
        typename T::Box q;
        q = load_box<D>(a.nodebox, leaf0 + L);
        int32_t* out = a.llist + L * LEAFCAP;
        int cnt = 0, sp = 0;
        const int ns = a.tnsib[L];
        if (ns >= 0) {
            for (int j = 0; j < ns; ++j) {
                const int r = a.tsib[L * SIBCAP + j].x;
                if (r >= leaf0) {  // a leaf sibling: within eps of the box by construction
                    if (cnt < LEAFCAP) out[cnt] = r - leaf0;
                    ++cnt;
                } else if (sp < LL_STACK) {
                    stk[LL_THREADS * sp++] = r;
                } else {
                    cnt = LEAFCAP + 1;
                }
            }
        } else {
            cnt = LEAFCAP + 1;  // no recorded roots: the phases walk the tree
        }
        int64_t steps = 0;
        while (sp > 0 && cnt <= LEAFCAP) {
            if (++steps > m) {
                atomicOr(&a.ctrl[CTRL_ERR], ERR_STACK);
                cnt = LEAFCAP + 1;
                break;
            }
            const int node = stk[LL_THREADS * --sp];
            const auto nd = NB<D>::load(a.nodes, node);
            float dl, dr;
            NB<D>::bd2(nd, q, dl, dr);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if ((c ? dr : dl) > tp.e2) continue;
                const int child = c ? nd.m.y : nd.m.x;
                if (child >= leaf0) {
                    if (child - leaf0 != (int)L) {
                        if (cnt < LEAFCAP) out[cnt] = child - leaf0;
                        ++cnt;
                    }
                } else if (sp < LL_STACK) {
                    stk[LL_THREADS * sp++] = child;
                } else {
                    cnt = LEAFCAP + 1;
                }
            }
        }
        a.lcount[L] = cnt <= LEAFCAP ? (int16_t)cnt : (int16_t)-1;
    }
}

template <int D, class V>
__device__ __forceinline__ void walk(const DevArgs<D>& a, int64_t m, V& v, int* stack, int L)
{
    const int lc = a.lcount ? a.lcount[L] : -1;
    if (lc >= 0) {
        // the leaf list, no tree walk. Per-point queries: each lane tests
        // one listed leaf against the box of the warp's queries, then the
        // leaves that pass are taken in list order with the lane-wise test
        // of each query
        const int leaf0 = (int)(m - 1);
        const int lane = threadIdx.x & 31;
        const int32_t* lst = a.llist + (int64_t)L * LEAFCAP;
        if constexpr (!V::PREFILTER) {
            for (int j = 0; j < lc; ++j) {
                const int U = __ldg(&lst[j]);
                if (U < v.mask_lo) continue;
                typename Traits<D>::Box b;
                b.lo = a.nodebox[leaf0 + U].lo;
                b.hi = a.nodebox[leaf0 + U].hi;
                const unsigned mk = __ballot_sync(FULL, v.hit_box(b));
                GBD_COUNT(CNT_LEAF, lane == 0 && mk);
                if (mk && v.leaf(U, mk, b)) return;
            }
        } else {
            const typename Traits<D>::Box qb = v.query_box();
            for (int j0 = 0; j0 < lc; j0 += 32) {
                int U = -1, sol = 0;
                int2 r = make_int2(0, 0);
                bool cand = false;
                if (j0 + lane < lc) {
                    U = __ldg(&lst[j0 + lane]);
                    if (U >= v.mask_lo) {
                        typename Traits<D>::Box b;
                        b.lo = a.nodebox[leaf0 + U].lo;
                        b.hi = a.nodebox[leaf0 + U].hi;
                        cand = NB<D>::bbox(qb, b) <= v.e2;
                        // the records of all candidates in one lane-parallel load
                        if (cand) {
                            r = __ldg(&a.leafr[U]);
                            if constexpr (V::NEEDS_SOLID) sol = a.lsolid[U];
                        }
                    }
                }
                unsigned cm = __ballot_sync(FULL, cand);
                while (cm) {
                    const int src = __ffs(cm) - 1;
                    cm &= cm - 1;
                    const int Us = __shfl_sync(FULL, U, src);
                    const int2 rs = make_int2(__shfl_sync(FULL, r.x, src), __shfl_sync(FULL, r.y, src));
                    const int ss = V::NEEDS_SOLID ? __shfl_sync(FULL, sol, src) : 0;
                    typename Traits<D>::Box b;
                    b.lo = a.nodebox[leaf0 + Us].lo;
                    b.hi = a.nodebox[leaf0 + Us].hi;
                    const unsigned mk = __ballot_sync(FULL, v.hit_box(b));
                    GBD_COUNT(CNT_LEAF, lane == 0 && mk);
                    if (mk && v.leaf_rec(Us, mk, b, rs, ss)) return;
                }
            }
        }
        return;
    }
    const int ns = a.tnsib[L];
    if (ns >= 0) traverse_roots<D>(a.nodes, a.nodebox, m, v, stack, a.ctrl, a.tsib + (int64_t)L * SIBCAP, ns);
    else traverse<D>(a.nodes, a.nodebox, m, v, stack, a.ctrl, a.tstart[L]);
}

__device__ __forceinline__ int next_leaf(uint32_t* ctr)
{
    int L = 0;
    if ((threadIdx.x & 31) == 0) L = (int)atomicAdd(ctr, 1u);
    return __shfl_sync(FULL, L, 0);
}

// Register caps of the traversal kernels: 56 in 2D and 3D (nine 128-thread
// blocks per SM, measured fastest on the 16M halo workload); more above 3D,
// where a point and its packed copy take 3 D registers
template <int D>
constexpr int traversal_regs()
{
    return D <= 3 ? 56 : (D <= 5 ? 96 : 128);
}

template <int D>
__global__ void __maxnreg__(traversal_regs<D>()) k_pre(DevArgs<D> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpMem<D>* wm = reinterpret_cast<WarpMem<D>*>(smem) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t m = a.ctrl[CTRL_M];
    for (;;) {
        const int L = next_leaf(&a.ctrl[CTRL_WORK_PRE]);
        if (L >= m) break;
        const int2 r = a.leafr[L];
        if (r.y < 0) continue;  // dense cell: all core already
        const TileParams tp = tile_params(a, L);
        // Algorithm 3: no preprocessing for minPts <= 2 (counts for several
        // minPts are always taken)
        if (tp.min_pts <= 2 && !a.ncount) continue;
        const int s = r.x, e = r.y, k = e - s;
        const int q = s + lane;
        // points of dense cells inside the tile are core already
        const bool counts = q < e && !a.core[q];
        if (!__any_sync(FULL, counts)) continue;
        const typename Traits<D>::Point p = a.sp[q < e ? q : s];
        // the tile's own points first: in dense regions most queries reach
        // minPts here and need no traversal at all (two points at a time)
        wm->soa.put(lane, p);
        __syncwarp();
        const typename NB<D>::PP pp = NB<D>::pack(p);
        int cnt = 0;
        if (counts) {
            int u = 0;
            for (; u + 1 < k && cnt < tp.min_pts; u += 2) {
                float d0, d1;
                wm->soa.d2pair(pp, u, d0, d1);
                cnt += (d0 <= tp.e2) + (d1 <= tp.e2);
            }
            if (u < k && cnt < tp.min_pts && wm->soa.d2(p, u) <= tp.e2) ++cnt;
        }
        __syncwarp();
        PreV<D> v;
        v.sp = a.sp; v.leafr = a.leafr; v.soa = &wm->soa; v.e2 = tp.e2; v.min_pts = tp.min_pts;
        v.mask_lo = 0; v.own = L; v.lane = lane;
        v.act = counts && cnt < tp.min_pts;
        v.p = p;
        v.pp = pp;
        v.cnt = cnt;
        v.nlist = a.lcap > 0 ? a.nlist : nullptr;
        v.lcap = a.lcap;
        v.qs = s;
        v.nl = 0;
        const unsigned am = __ballot_sync(FULL, v.act);
        if (am) {
            // every point of the tile still counting: their box is the
            // leaf's own (exact min/max of the same points), no reduction
            v.qbox = am == tile_lanes(k) ? load_box<D>(a.nodebox, (m - 1) + L) : warp_box<D>(p, v.act);
            walk(a, m, v, wm->stack, L);
        }
        if (counts) {
            const bool c = v.cnt >= tp.min_pts;
            a.core[q] = c ? 1 : 0;
            // lists: how many out-of-tile neighbours the list of a non-core
            // point holds; else whether another point is within eps (the
            // count includes q)
            a.nbr[q] = a.lcap > 0 ? (c ? 0 : (uint8_t)v.nl) : (v.cnt >= 2 ? 1 : 0);
            if (a.ncount) a.ncount[q] = v.cnt;
        }
    }
}

// Border claims from preprocessing's lists (DBSCAN mode): a non-core point
// holds all its neighbours outside its tile; it joins the cluster of the
// first core one (Algorithm 3's claim of a border point, Sec. 3.2, made here
// from the border's side). Neighbours inside the tile are k_intra's.
__global__ void k_list_claims(const int32_t* __restrict__ nlist, int lcap, const uint8_t* __restrict__ nbr,
                              const uint8_t* __restrict__ core, int32_t* labels, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        if (core[q]) continue;
        const int k = nbr[q];
        const int32_t* row = nlist + q * lcap;
        for (int j = 0; j < k; ++j) {
            const int y = row[j];
            if (core[y]) {
                uf_claim(labels, (int)q, y);
                break;
            }
        }
    }
}

// Each tile resolves its own pairs (q, q') with q' > q. Every lane builds the
// bit mask of the tile points within eps of its point; the components of the
// core points follow from doubling reach sets (the union of the reach sets
// of the points already reached) over warp shuffles, at most five rounds for
// 32 points; each core point then joins its component's first point
// globally (at most one union per point), and a non-core point with a core
// neighbour in the tile claims it. Finally the tile records whether it is
// solid: all points core and in one set. Dense cells larger than a tile are
// solid by construction.
constexpr int INTRA_THREADS = 256;

template <int D>
__global__ void __launch_bounds__(INTRA_THREADS) k_intra(DevArgs<D> a)
{
    using P = typename Traits<D>::Point;
    __shared__ SoA<D> soa_s[INTRA_THREADS / 32];
    SoA<D>& soa = soa_s[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t m = a.ctrl[CTRL_M];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = wid; L < m; L += nw) {
        const int2 r = a.leafr[L];
        if (r.y < 0) {
            if (lane == 0) a.lsolid[L] = 1;
            continue;
        }
        const int s = r.x, k = r.y - r.x;
        const TileParams tp = tile_params(a, (int)L);
        const bool valid = lane < k;
        bool c = valid && a.core[s + lane];
        if (tp.min_pts > 2 && !__any_sync(FULL, c)) {
            // core flags known and none in the tile: no pair inside it
            // unites or claims anything, and it is not solid
            if (lane == 0) a.lsolid[L] = 0;
            continue;
        }
        const P p = a.sp[valid ? s + lane : s];
        // the tile's adjacency, two points at a time (packed)
        soa.put(lane, p);
        __syncwarp();
        unsigned adj = 0;
        if (valid) {
            const typename NB<D>::PP pp = NB<D>::pack(p);
            int j = 0;
            for (; j + 1 < k; j += 2) {
                float d0, d1;
                soa.d2pair(pp, j, d0, d1);
                adj |= (d0 <= tp.e2 ? 1u : 0u) << j;
                adj |= (d1 <= tp.e2 ? 2u : 0u) << j;
            }
            if (j < k && soa.d2(p, j) <= tp.e2) adj |= 1u << j;
            adj &= ~(1u << lane);
        }
        __syncwarp();
        if (tp.min_pts == 2) {
            // no preprocessing: a neighbour inside the tile makes a point core
            // (neighbours in other tiles are found by the main phase)
            c = valid && (c || adj != 0);
            if (c) a.core[s + lane] = 1;
        }
        const unsigned cm = __ballot_sync(FULL, c);
        if (tp.min_pts > 2 && a.mode == DBSCAN_MODE_DBSCAN && valid && !c && (adj & cm))
            uf_claim(a.labels, s + lane, s + __ffs(adj & cm) - 1);
        unsigned reach = c ? ((adj & cm) | (1u << lane)) : 0u;
        for (int it = 0; it < 5; ++it) {
            unsigned acc = reach;
            for (int j = 0; j < k; ++j) {
                const unsigned rj = __shfl_sync(FULL, reach, j);
                if ((reach >> j) & 1u) acc |= rj;
            }
            const bool changed = acc != reach;
            reach = acc;
            if (!__any_sync(FULL, changed)) break;
        }
        if (c) {
            const int lr = __ffs(reach) - 1;
            if (lr != lane) uf_union(a.labels, s + lane, s + lr);
        }
        __syncwarp();
        const int root = c ? uf_find(a.labels, s + lane) : -1;
        const int root0 = __shfl_sync(FULL, root, 0);
        const bool solid = __all_sync(FULL, !valid || (c && root == root0));
        if (lane == 0) a.lsolid[L] = solid ? 1 : 0;
        __syncwarp();
    }
}

// Leaf kinds for the main phase: 0 a tile that is not solid, 1 a solid tile,
// 2 a dense cell larger than a tile. Lists are grouped by kind; within a warp
// (32 consecutive leaves) the order is kept.
__device__ __forceinline__ int leaf_kind(const int2* leafr, const uint8_t* lsolid, int64_t L)
{
    return leafr[L].y < 0 ? 2 : (lsolid[L] ? 1 : 0);
}

__global__ void k_kinds_count(const int2* __restrict__ leafr, const uint8_t* __restrict__ lsolid, uint32_t* ctrl)
{
    const int lane = threadIdx.x & 31;
    const int64_t m = ctrl[CTRL_M];
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < m;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = base + lane;
        const int kind = L < m ? leaf_kind(leafr, lsolid, L) : -1;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const unsigned b = __ballot_sync(FULL, kind == t);
            if (lane == 0 && b) atomicAdd(&ctrl[CTRL_KIND_COUNT + t], (uint32_t)__popc(b));
        }
    }
}

__global__ void k_kinds_write(const int2* __restrict__ leafr, const uint8_t* __restrict__ lsolid, uint32_t* ctrl,
                              int32_t* __restrict__ klist)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t m = ctrl[CTRL_M];
    const uint32_t off[3] = {0u, ctrl[CTRL_KIND_COUNT], ctrl[CTRL_KIND_COUNT] + ctrl[CTRL_KIND_COUNT + 1]};
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < m;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = base + lane;
        const int kind = L < m ? leaf_kind(leafr, lsolid, L) : -1;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const unsigned b = __ballot_sync(FULL, kind == t);
            if (!b) continue;
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(&ctrl[CTRL_KIND_FILL + t], (uint32_t)__popc(b));
            at = __shfl_sync(FULL, at, 0);
            if (kind == t) klist[off[t] + at + __popc(b & lt)] = (int32_t)L;
        }
    }
}

// The main phase (KIND 0: tiles that are not solid, MainPtV; 1: solid
// tiles, MainSolidV; 2: dense cells larger than a tile, MainBoxV; 3: all of
// them in one launch), taken from the kinds' lists through a work counter.
// In one launch the dense cells come first -- few, each much work -- and the
// warps that finish them go on to the tiles instead of leaving the GPU idle
// until the slowest cell is done.
template <int D, int KIND>
__global__ void __maxnreg__(traversal_regs<D>()) k_main(DevArgs<D> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpMem<D>* wm = reinterpret_cast<WarpMem<D>*>(smem) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t m = a.ctrl[CTRL_M];
    const int64_t c0 = a.ctrl[CTRL_KIND_COUNT], c1 = a.ctrl[CTRL_KIND_COUNT + 1], c2 = a.ctrl[CTRL_KIND_COUNT + 2];
    // dense cells larger than a tile are few and each is much work: when
    // there are more warps than cells, up to 8 warps share a cell (split by
    // neighbour leaf), so that no warp is left with a whole large cell
    int parts = 1;
    if ((KIND == 2 || KIND == 3) && c2 > 0) {
        const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
        parts = (int)max((int64_t)1, min((int64_t)8, warps / c2));
    }
    const int64_t n2 = (KIND == 2 || KIND == 3) ? c2 * parts : 0;
    const int64_t total = KIND == 3 ? n2 + c1 + c0 : (KIND == 2 ? n2 : (KIND == 1 ? c1 : c0));
    for (;;) {
        const int idx = next_leaf(&a.ctrl[CTRL_KIND_WORK + (KIND == 3 ? 0 : KIND)]);
        if (idx >= total) break;
        // the list holds kind 0, then 1, then 2
        int kind, L, part = 0;
        if (KIND == 3) {
            if (idx < n2) {
                kind = 2;
                L = a.klist[c0 + c1 + idx / parts];
                part = idx % parts;
            } else if (idx < n2 + c1) {
                kind = 1;
                L = a.klist[c0 + (idx - n2)];
            } else {
                kind = 0;
                L = a.klist[idx - n2 - c1];
            }
        } else {
            kind = KIND;
            L = a.klist[(KIND == 0 ? 0 : (KIND == 1 ? c0 : c0 + c1)) + (KIND == 2 ? idx / parts : idx)];
            part = KIND == 2 ? idx % parts : 0;
        }
        const TileParams tp = tile_params(a, L);
        const bool listed = a.lcap > 0 && tp.min_pts > 2;
        const Rule rule{a.labels, a.core, tp.min_pts, a.mode == DBSCAN_MODE_DBSCAN && !listed};
        const int2 r = a.leafr[L];
        const int s = r.x, e = r.y & 0x7fffffff;
        if (kind == 0) {
            MainPtV<D> v;
            v.sp = a.sp; v.leafr = a.leafr; v.lsolid = a.lsolid; v.core = a.core; v.soa = &wm->soa;
            v.cbuf = wm->cbuf; v.rule = rule; v.e2 = tp.e2; v.mask_lo = L + 1; v.lane = lane; v.sQ = s;
            v.q = s + lane;
            const bool in = v.q < e;
            v.qcore = in && a.core[v.q];
            // after preprocessing a non-core point with no other point within
            // eps takes part in no pair, and in DBSCAN* no non-core point does
            // (with lists, non-core points took their pairs with core points
            // from their lists and need no traversal)
            v.valid = in && (tp.min_pts <= 2 || v.qcore || (rule.claims && a.nbr[v.q]));
            v.p = a.sp[in ? v.q : s];
            v.pp = NB<D>::pack(v.p);
            const unsigned vm = __ballot_sync(FULL, v.valid);
            if (vm) {
                v.qbox = vm == tile_lanes(e - s) ? load_box<D>(a.nodebox, (m - 1) + L) : warp_box<D>(v.p, v.valid);
                walk(a, m, v, wm->stack, L);
            }
        } else if (kind == 1) {
            MainSolidV<D> v;
            v.sp = a.sp; v.leafr = a.leafr; v.lsolid = a.lsolid; v.core = a.core; v.buf = wm->buf;
            v.rule = rule; v.e2 = tp.e2; v.mask_lo = L + 1; v.lane = lane; v.sQ = s;
            v.valid = s + lane < e;
            v.p = a.sp[v.valid ? s + lane : s];
            v.pp = NB<D>::pack(v.p);
            v.qb.lo = a.nodebox[(m - 1) + L].lo;
            v.qb.hi = a.nodebox[(m - 1) + L].hi;
            walk(a, m, v, wm->stack, L);
        } else {
            MainBoxV<D> v;
            v.sp = a.sp; v.leafr = a.leafr; v.lsolid = a.lsolid; v.core = a.core; v.buf = wm->buf;
            v.rule = rule; v.e2 = tp.e2; v.mask_lo = L + 1; v.lane = lane; v.sQ = s; v.eQ = e;
            v.part = part; v.parts = parts;
            v.qb.lo = a.nodebox[(m - 1) + L].lo;
            v.qb.hi = a.nodebox[(m - 1) + L].hi;
            walk(a, m, v, wm->stack, L);
        }
    }
}

// The same for one minPts of a multi-minPts run, with core flags from the
// neighbour counts (capped at the largest minPts, which decides every smaller
// one); points of dense cells are core for every minPts of the run.
__global__ void k_init_from_counts(const uint8_t* __restrict__ pdense, const int32_t* __restrict__ dstart,
                                   const int32_t* __restrict__ ncount, int64_t n, int min_pts,
                                   int32_t* __restrict__ labels, uint8_t* __restrict__ core)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (pdense && pdense[i]) {
            labels[i] = dstart[i];
            core[i] = 1;
        } else {
            labels[i] = (int32_t)i;
            core[i] = (min_pts <= 1 || ncount[i] >= min_pts) ? 1 : 0;
        }
    }
}

// Core flags given by the caller in input order (core_in[perm[i]]), for
// clustering a part of a larger point set whose flags were decided with the
// rest of it; points of dense cells are core in any case (every one of them
// has at least minPts neighbours inside its cell).
__global__ void k_core_from_input(const uint32_t* __restrict__ perm, const uint8_t* __restrict__ core_in,
                                  const uint8_t* __restrict__ pdense, int64_t n, uint8_t* __restrict__ core,
                                  const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;  // aborted run: perm may hold stale words
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        core[i] = ((pdense && pdense[i]) || core_in[perm[i]]) ? 1 : 0;
}

// labels[i] = i, or the first point of its dense cell (pre-united, Sec. 4.2);
// core = 1 in dense cells (and everywhere when minPts == 1)
__global__ void k_init(const uint8_t* __restrict__ pdense, const int32_t* __restrict__ dstart, int64_t n,
                       int min_pts, int32_t* __restrict__ labels, uint8_t* __restrict__ core)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (pdense && pdense[i]) {
            labels[i] = dstart[i];
            core[i] = 1;
        } else {
            labels[i] = (int32_t)i;
            core[i] = min_pts == 1 ? 1 : 0;
        }
    }
}

// full compression (Sec. 4.3) and the smallest input index per root
__global__ void k_finalize(int32_t* labels, const uint8_t* __restrict__ core, const uint32_t* __restrict__ perm,
                           int64_t n, int32_t* __restrict__ canon, const uint32_t* __restrict__ ctrl)
{
    if (!stage_on(ctrl, -1)) return;
    // warp-uniform trip count: warp_atomic_min needs all 32 lanes
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + (threadIdx.x & 31);
        const bool in = i < n;
        const int r = in ? uf_find(labels, (int)i) : 0;
        // (permutation and core flags are read once: evict-first)
        warp_atomic_min(canon, r, in ? (int32_t)__ldcs(perm + i) : 0, in && __ldcs(core + i));
    }
}

// output in input order: canonical label of the cluster, or -1
__global__ void k_relabel(const int32_t* labels, const uint8_t* __restrict__ core, const uint32_t* __restrict__ perm,
                          int64_t n, int mode, const int32_t* __restrict__ canon, int32_t* __restrict__ out,
                          uint8_t* __restrict__ core_out, const uint32_t* __restrict__ ctrl)
{
    // aborted run (non-finite input, a sort that gave up): perm may hold
    // stale words, so nothing is written; the error is reported at the next
    // host sync point
    if (!stage_on(ctrl, -1)) return;
    // the sequential reads (core flags, permutation, own label) stream
    // through L2 with evict-first priority, so that the lines of the
    // scattered output stay cached until they are complete
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool c = __ldcs(core + i) != 0;
        int r = (int)i;
        for (int p = __ldcs(labels + i); p != r; p = __ldcg(labels + r)) r = p;
        const bool member = c || (mode == DBSCAN_MODE_DBSCAN && r != (int)i);
        const uint32_t o = __ldcs(perm + i);
        out[o] = member ? canon[r] : -1;
        if (core_out) core_out[o] = c ? 1 : 0;
    }
}

#ifdef GBD_COUNTERS
__global__ void k_count_phase(int phase) { g_count_phase = phase; }
#endif

// the traversal counters' phase for the kernels that follow (counters build)
void count_phase(int phase, cudaStream_t s)
{
#ifdef GBD_COUNTERS
    k_count_phase<<<1, 1, 0, s>>>(phase);
#else
    (void)phase;
    (void)s;
#endif
}

// blocks of a persistent launch: as many as fit on all SMs at once
int persistent_blocks(const void* kernel, int block, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, smem);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

template <int D>
DevArgs<D> dev_args(const ClusterArgs& a)
{
    DevArgs<D> d;
    d.sp = static_cast<const typename Traits<D>::Point*>(a.sp);
    d.nodes = static_cast<const typename Traits<D>::Node*>(a.nodes);
    d.nodebox = static_cast<const typename Traits<D>::Box*>(a.nodebox);
    d.leafr = a.leafr;
    d.lsolid = a.lsolid;
    d.klist = a.klist;
    d.nbr = a.nbr;
    d.nlist = a.nlist;
    d.lcap = a.lcap;
    d.labels = a.labels;
    d.core = a.core;
    d.ctrl = a.ctrl;
    d.e2 = a.e2;
    d.min_pts = a.min_pts;
    d.mode = a.mode;
    d.linst = a.linst;
    d.e2s = a.e2s;
    d.mps = a.mps;
    d.iroot = a.iroot;
    d.tstart = a.tstart;
    d.tsib = a.tsib;
    d.tnsib = a.tnsib;
    d.llist = a.llist;
    d.lcount = a.lcount;
    d.ncount = a.ncount;
    return d;
}

template <int D>
void run_pre(const ClusterArgs& a, cudaStream_t s)
{
    static int blocks[33] = {};
    const size_t smem = sizeof(WarpMem<D>) * (size_t)(a.block / 32);
    int& g = blocks[a.block / 32];
    if (!g) g = persistent_blocks((const void*)k_pre<D>, a.block, smem);
    k_pre<D><<<g, a.block, smem, s>>>(dev_args<D>(a));
}

template <int D, int KIND>
void run_main_kind(const ClusterArgs& a, cudaStream_t s)
{
    static int blocks[33] = {};
    const size_t smem = sizeof(WarpMem<D>) * (size_t)(a.block / 32);
    int& g = blocks[a.block / 32];
    if (!g) g = persistent_blocks((const void*)k_main<D, KIND>, a.block, smem);
    k_main<D, KIND><<<g, a.block, smem, s>>>(dev_args<D>(a));
}

template <int D>
void run_main(const ClusterArgs& a, cudaStream_t s)
{
    int64_t gw = (a.m_cap * 32 + INTRA_THREADS - 1) / INTRA_THREADS;
    if (gw > 152 * 16) gw = 152 * 16;
    k_intra<D><<<(unsigned)gw, INTRA_THREADS, 0, s>>>(dev_args<D>(a));
    int64_t gk = (a.m_cap + 255) / 256;
    if (gk > 152 * 8) gk = 152 * 8;
    k_kinds_count<<<(unsigned)gk, 256, 0, s>>>(a.leafr, a.lsolid, a.ctrl);
    k_kinds_write<<<(unsigned)gk, 256, 0, s>>>(a.leafr, a.lsolid, a.ctrl, a.klist);
    run_main_kind<D, 3>(a, s);
}

}  // namespace

cudaError_t launch_cluster_init(const ClusterArgs& a, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.ctrl + CTRL_WORK_PRE, 0, (CTRL_WORK_END - CTRL_WORK_PRE) * sizeof(uint32_t), s)) !=
        cudaSuccess)
        return e;
    int64_t gn = (a.n + 255) / 256;
    if (gn > 152 * 16) gn = 152 * 16;
    k_init<<<(unsigned)gn, 256, 0, s>>>(a.pdense, a.dstart, a.n, a.min_pts, a.labels, a.core);
    note_launches(1);
    if ((e = cudaMemsetAsync(a.canon, 0x7f, sizeof(int32_t) * (size_t)a.n, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_cluster_from_counts(const ClusterArgs& a, int min_pts, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.ctrl + CTRL_WORK_PRE, 0, (CTRL_WORK_END - CTRL_WORK_PRE) * sizeof(uint32_t), s)) !=
        cudaSuccess)
        return e;
    int64_t gn = (a.n + 255) / 256;
    if (gn > 152 * 16) gn = 152 * 16;
    k_init_from_counts<<<(unsigned)gn, 256, 0, s>>>(a.pdense, a.dstart, a.ncount, a.n, min_pts, a.labels, a.core);
    note_launches(1);
    if ((e = cudaMemsetAsync(a.canon, 0x7f, sizeof(int32_t) * (size_t)a.n, s)) != cudaSuccess) return e;
    if (a.lcap > 0 && a.mode == DBSCAN_MODE_DBSCAN) {
        k_list_claims<<<(unsigned)gn, 256, 0, s>>>(a.nlist, a.lcap, a.nbr, a.core, a.labels, a.n);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_cluster_starts(const ClusterArgs& a, cudaStream_t s)
{
    count_phase(0, s);
    int64_t gm = (a.m_cap + 255) / 256;
    if (gm > 152 * 8) gm = 152 * 8;
#define TS_LAUNCH(D) k_tile_start<D><<<(unsigned)gm, 256, 0, s>>>(dev_args<D>(a), a.parent, a.nmeta)
    GBD_DIM_SWITCH(a.dim, TS_LAUNCH)
#undef TS_LAUNCH
    if (a.llist) {
#define LL_LAUNCH(D) k_leaf_lists<D><<<(unsigned)gm, LL_THREADS, 0, s>>>(dev_args<D>(a))
        GBD_DIM_SWITCH(a.dim, LL_LAUNCH)
#undef LL_LAUNCH
        note_launches(1);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cluster_pre(const ClusterArgs& a, cudaStream_t s)
{
    // Algorithm 3: no preprocessing for minPts <= 2 (counts for several minPts
    // are always taken)
    if (a.min_pts <= 2 && !a.ncount) return cudaSuccess;
    count_phase(1, s);
    cudaError_t e;
    // points that keep no list (instances of a batch with minPts <= 2) read 0
    if (a.lcap > 0 && (e = cudaMemsetAsync(a.nbr, 0, (size_t)a.n, s)) != cudaSuccess) return e;
#define PRE_RUN(D) run_pre<D>(a, s)
    GBD_DIM_SWITCH(a.dim, PRE_RUN)
#undef PRE_RUN
    note_launches(1);
    if (a.lcap > 0 && !a.ncount) {  // (several minPts: claims per minPts)
        int64_t gn = (a.n + 255) / 256;
        if (gn > 152 * 16) gn = 152 * 16;
        k_list_claims<<<(unsigned)gn, 256, 0, s>>>(a.nlist, a.lcap, a.nbr, a.core, a.labels, a.n);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_cluster_main(const ClusterArgs& a, cudaStream_t s)
{
    count_phase(2, s);
#define MAIN_RUN(D) run_main<D>(a, s)
    GBD_DIM_SWITCH(a.dim, MAIN_RUN)
#undef MAIN_RUN
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_cluster_core_from_input(const ClusterArgs& a, const uint8_t* core_in, cudaStream_t s)
{
    int64_t gn = (a.n + 255) / 256;
    if (gn > 152 * 16) gn = 152 * 16;
    k_core_from_input<<<(unsigned)gn, 256, 0, s>>>(a.perm, core_in, a.pdense, a.n, a.core, a.ctrl);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cluster_final(const ClusterArgs& a, int32_t* labels_out, uint8_t* core_out, cudaStream_t s)
{
    int64_t gn = (a.n + 255) / 256;
    if (gn > 152 * 16) gn = 152 * 16;
    k_finalize<<<(unsigned)gn, 256, 0, s>>>(a.labels, a.core, a.perm, a.n, a.canon, a.ctrl);
    k_relabel<<<(unsigned)gn, 256, 0, s>>>(a.labels, a.core, a.perm, a.n, a.mode, a.canon, labels_out, core_out,
                                           a.ctrl);
    note_launches(2);
    return cudaGetLastError();
}

bool counters_built()
{
#ifdef GBD_COUNTERS
    return true;
#else
    return false;
#endif
}

// the traversal counters since the last read ([phase][kind]), then zeroed
cudaError_t counters_take(uint64_t* out)
{
#ifdef GBD_COUNTERS
    unsigned long long h[CNT_PHASES * CNT_KINDS] = {};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(h, g_counts, sizeof(h));
    for (int i = 0; i < CNT_PHASES * CNT_KINDS; ++i) out[i] = h[i];
    const unsigned long long z[CNT_PHASES * CNT_KINDS] = {};
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_counts, z, sizeof(z));
    return e;
#else
    for (int i = 0; i < CNT_PHASES * CNT_KINDS; ++i) out[i] = 0;
    return cudaErrorNotSupported;
#endif
}

}  // namespace gbd
