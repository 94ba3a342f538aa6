// Internal declarations shared by the CUDA translation units of libgbdbscan.
// Nothing here is part of the public C ABI (see include/gbdbscan.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbdbscan.h"

namespace gbd {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TILE = 32;  // points per non-dense BVH leaf (one warp lane per point)
// radix sort geometry: the digit width of one pass, the digits, the most
// passes a key takes (64-bit keys) and the keys per look-back tile (256
// threads x 16)
constexpr int SORT_DIGIT_BITS = 9;
constexpr int SORT_RADIX = 1 << SORT_DIGIT_BITS;
constexpr int SORT_MAX_PASSES = (64 + SORT_DIGIT_BITS - 1) / SORT_DIGIT_BITS;
constexpr int SORT_TILE_KEYS = 256 * 16;

// bits of the device error words
constexpr unsigned ERR_SORT_TIMEOUT = 1u;  // a radix-sort look-back wait ran out
constexpr unsigned ERR_NONFINITE = 4u;     // the input holds a NaN or an infinity

// Upper bound on the iterations of any device-side wait. A wait that runs out
// sets an error bit and gives up its step, so no kernel can hang.
constexpr int SPIN_LIMIT = 1 << 22;

// ---------------------------------------------------------------------------
// Traversal counters (an opt-in build, -DGBD_COUNTERS; the product build
// compiles every GBD_COUNT to nothing): point-to-point distance tests,
// point- and box-to-box tests, node visits and leaf visits (both per warp),
// per phase (0 index lists, 1 preprocessing, 2 main phase), summed over the
// lanes that take part with one atomic per warp.
// ---------------------------------------------------------------------------
enum { CNT_DIST = 0, CNT_BOX = 1, CNT_NODE = 2, CNT_LEAF = 3, CNT_KINDS = 4, CNT_PHASES = 3 };
#ifdef GBD_COUNTERS
static __device__ unsigned long long g_counts[CNT_PHASES * CNT_KINDS];
static __device__ int g_count_phase;
__device__ __forceinline__ void gbd_count(int kind, unsigned v)
{
    const unsigned m = __activemask();
    const unsigned t = __reduce_add_sync(m, v);
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && t)
        atomicAdd(&g_counts[g_count_phase * CNT_KINDS + kind], (unsigned long long)t);
}
#define GBD_COUNT(kind, v) gbd_count((kind), (unsigned)(v))
#else
#define GBD_COUNT(kind, v) ((void)0)
#endif

// ---------------------------------------------------------------------------
// The distance test, fixed as the fp32 squared form with no fused multiply-add
// (explicit round-to-nearest intrinsics, which the compiler never contracts):
//   dk = fl(x_k - y_k); s = fl(d0*d0); s = fl(s + fl(dk*dk)); adjacent <=> s <= fl(eps*eps)
// dist(x, y) <= eps is the paper's test (Sec. 2.1); the rounding is this
// library's fixed reading of it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sqr_rn(float a) { return __fmul_rn(a, a); }

__device__ __forceinline__ float dist2(const float4& a, const float4& b)
{
    GBD_COUNT(CNT_DIST, 1);
    float s = sqr_rn(__fsub_rn(a.x, b.x));
    s = __fadd_rn(s, sqr_rn(__fsub_rn(a.y, b.y)));
    s = __fadd_rn(s, sqr_rn(__fsub_rn(a.z, b.z)));
    return s;
}

__device__ __forceinline__ float dist2(const float2& a, const float2& b)
{
    GBD_COUNT(CNT_DIST, 1);
    float s = sqr_rn(__fsub_rn(a.x, b.x));
    s = __fadd_rn(s, sqr_rn(__fsub_rn(a.y, b.y)));
    return s;
}

// A point of 4 to 8 dimensions: 8 floats (32 B: two 16-byte loads), the
// coordinates from D on unused.
template <int D>
struct __align__(16) PtN {
    float c[8];
};

// L2-coherent (L1-bypassing) copies of points, for the boxes the refit's
// threads hand to one another
__device__ __forceinline__ float4 ld_cg(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void st_cg(float4* p, const float4& v) { __stcg(p, v); }
__device__ __forceinline__ void st_cg(float2* p, const float2& v) { __stcg(p, v); }
template <int D>
__device__ __forceinline__ PtN<D> ld_cg(const PtN<D>* p)
{
    PtN<D> r;
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldcg(q), b = __ldcg(q + 1);
    r.c[0] = a.x; r.c[1] = a.y; r.c[2] = a.z; r.c[3] = a.w;
    r.c[4] = b.x; r.c[5] = b.y; r.c[6] = b.z; r.c[7] = b.w;
    return r;
}
template <int D>
__device__ __forceinline__ void st_cg(PtN<D>* p, const PtN<D>& v)
{
    float4* q = reinterpret_cast<float4*>(p);
    __stcg(q, make_float4(v.c[0], v.c[1], v.c[2], v.c[3]));
    __stcg(q + 1, make_float4(v.c[4], v.c[5], v.c[6], v.c[7]));
}

template <int D>
__device__ __forceinline__ float dist2(const PtN<D>& a, const PtN<D>& b)
{
    GBD_COUNT(CNT_DIST, 1);
    float s = sqr_rn(__fsub_rn(a.c[0], b.c[0]));
#pragma unroll
    for (int k = 1; k < D; ++k) s = __fadd_rn(s, sqr_rn(__fsub_rn(a.c[k], b.c[k])));
    return s;
}

// Gap between a coordinate p and the interval [lo, hi]: max(lo - p, p - hi, 0),
// each difference rounded. Rounding is monotone, so for every y in [lo, hi]
// |fl(p - y)| >= gap, and the squared box distance below is a lower bound of
// dist2(p, y) for every point y of the box: pruning with it is exact.
__device__ __forceinline__ float gap_rn(float lo, float hi, float p)
{
    return fmaxf(fmaxf(__fsub_rn(lo, p), __fsub_rn(p, hi)), 0.0f);
}

// Gap between intervals [alo, ahi] and [blo, bhi] (a lower bound of |a - b|
// after rounding, for a in A and b in B).
__device__ __forceinline__ float gap2_rn(float alo, float ahi, float blo, float bhi)
{
    return fmaxf(fmaxf(__fsub_rn(blo, ahi), __fsub_rn(alo, bhi)), 0.0f);
}

// ---------------------------------------------------------------------------
// Pairs of fp32 values in one 64-bit register, for the packed f32x2
// arithmetic of sm_100-family GPUs: each half is rounded to nearest even on
// its own, so sub2 / add2 / mul2 give exactly __fsub_rn / __fadd_rn /
// __fmul_rn per half, in half the instructions.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpk2(f32x2 v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sqr2(f32x2 a)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(r) : "l"(a));
    return r;
}
// gap_rn per half: max(lo - p, p - hi, 0)
__device__ __forceinline__ f32x2 gap_rn2(f32x2 lo, f32x2 hi, f32x2 p)
{
    float a0, a1, b0, b1;
    unpk2(sub2(lo, p), a0, a1);
    unpk2(sub2(p, hi), b0, b1);
    return pk2(fmaxf(fmaxf(a0, b0), 0.0f), fmaxf(fmaxf(a1, b1), 0.0f));
}
// gap2_rn per half, interval [alo, ahi] against the pair of intervals [blo, bhi]
__device__ __forceinline__ f32x2 gap2_rn2(f32x2 alo, f32x2 ahi, f32x2 blo, f32x2 bhi)
{
    float a0, a1, b0, b1;
    unpk2(sub2(blo, ahi), a0, a1);
    unpk2(sub2(alo, bhi), b0, b1);
    return pk2(fmaxf(fmaxf(a0, b0), 0.0f), fmaxf(fmaxf(a1, b1), 0.0f));
}

// ---------------------------------------------------------------------------
// Per-dimension storage traits.
//   Point: sorted coordinates (float2 in 2D, float4 with w unused in 3D,
//          PtN<D> from 4 to 8 dimensions).
//   Box:   an axis-aligned box (lo, hi points).
//   Node:  an internal BVH node holding both children's boxes, their indices,
//          the split (last leaf of the left child) and the last leaf it covers.
// The general template covers 4 to 8 dimensions; 2 and 3 are specialised.
// ---------------------------------------------------------------------------
template <int D> struct Traits {
    static_assert(D >= 4 && D <= 8, "dimensions 2 to 8");
    using Point = PtN<D>;
    struct Box { Point lo, hi; };
    // per axis (left lo, right lo, left hi, right hi), then (left child,
    // right child, split, last leaf): 16 D + 16 bytes
    struct Node { float4 ax[D]; int4 m; };

    __device__ static __forceinline__ Point load_point(const float* p, int64_t i)
    {
        Point r;
#pragma unroll
        for (int k = 0; k < 8; ++k) r.c[k] = k < D ? p[D * i + k] : 0.0f;
        return r;
    }
    __device__ static __forceinline__ float coord(const Point& p, int k) { return p.c[k]; }
    __device__ static __forceinline__ Box point_box(const Point& p) { return Box{p, p}; }
    __device__ static __forceinline__ Box empty_box()
    {
        Box b;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            b.lo.c[k] = k < D ? INFINITY : 0.0f;
            b.hi.c[k] = k < D ? -INFINITY : 0.0f;
        }
        return b;
    }
    __device__ static __forceinline__ void grow(Box& b, const Point& p)
    {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            b.lo.c[k] = fminf(b.lo.c[k], p.c[k]);
            b.hi.c[k] = fmaxf(b.hi.c[k], p.c[k]);
        }
    }
    __device__ static __forceinline__ void merge(Box& b, const Box& o)
    {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            b.lo.c[k] = fminf(b.lo.c[k], o.lo.c[k]);
            b.hi.c[k] = fmaxf(b.hi.c[k], o.hi.c[k]);
        }
    }
    __device__ static __forceinline__ Box shfl_xor(const Box& b, int m)
    {
        Box r = b;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            r.lo.c[k] = __shfl_xor_sync(FULL, b.lo.c[k], m);
            r.hi.c[k] = __shfl_xor_sync(FULL, b.hi.c[k], m);
        }
        return r;
    }
    __device__ static __forceinline__ float box_dist2(const Point& p, const Box& b)
    {
        float s = sqr_rn(gap_rn(b.lo.c[0], b.hi.c[0], p.c[0]));
#pragma unroll
        for (int k = 1; k < D; ++k) s = __fadd_rn(s, sqr_rn(gap_rn(b.lo.c[k], b.hi.c[k], p.c[k])));
        return s;
    }
    __device__ static __forceinline__ float box_box_dist2(const Box& a, const Box& b)
    {
        float s = sqr_rn(gap2_rn(a.lo.c[0], a.hi.c[0], b.lo.c[0], b.hi.c[0]));
#pragma unroll
        for (int k = 1; k < D; ++k) s = __fadd_rn(s, sqr_rn(gap2_rn(a.lo.c[k], a.hi.c[k], b.lo.c[k], b.hi.c[k])));
        return s;
    }
    __device__ static __forceinline__ float diag2(const Box& b) { return dist2(b.lo, b.hi); }
    __device__ static __forceinline__ float far_dist2(const Point& p, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(p.c[0], b.lo.c[0]), __fsub_rn(b.hi.c[0], p.c[0])));
#pragma unroll
        for (int k = 1; k < D; ++k)
            s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(p.c[k], b.lo.c[k]), __fsub_rn(b.hi.c[k], p.c[k]))));
        return s;
    }
    __device__ static __forceinline__ float box_far2(const Box& a, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(b.hi.c[0], a.lo.c[0]), __fsub_rn(a.hi.c[0], b.lo.c[0])));
#pragma unroll
        for (int k = 1; k < D; ++k)
            s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(b.hi.c[k], a.lo.c[k]), __fsub_rn(a.hi.c[k], b.lo.c[k]))));
        return s;
    }
    __device__ static __forceinline__ Node make_node(const Box& L, const Box& R, int left, int right, int split, int last)
    {
        Node n;
#pragma unroll
        for (int k = 0; k < D; ++k) n.ax[k] = make_float4(L.lo.c[k], R.lo.c[k], L.hi.c[k], R.hi.c[k]);
        n.m = make_int4(left, right, split, last);
        return n;
    }
};

template <> struct Traits<3> {
    using Point = float4;
    struct Box { float4 lo, hi; };
    // 64 B: per axis (left lo, right lo, left hi, right hi) in a, b, c (x, y,
    // z), so that one load gives the lo and hi pairs of both children on
    // that axis; m = (left child, right child, split, last leaf)
    struct Node { float4 a, b, c; int4 m; };

    __device__ static __forceinline__ Point load_point(const float* p, int64_t i)
    {
        return make_float4(p[3 * i], p[3 * i + 1], p[3 * i + 2], 0.0f);
    }
    __device__ static __forceinline__ float coord(const Point& p, int k) { return k == 0 ? p.x : (k == 1 ? p.y : p.z); }
    __device__ static __forceinline__ Box point_box(const Point& p) { return Box{p, p}; }
    __device__ static __forceinline__ Box empty_box()
    {
        return Box{make_float4(INFINITY, INFINITY, INFINITY, 0.f), make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f)};
    }
    __device__ static __forceinline__ void grow(Box& b, const Point& p)
    {
        b.lo.x = fminf(b.lo.x, p.x); b.lo.y = fminf(b.lo.y, p.y); b.lo.z = fminf(b.lo.z, p.z);
        b.hi.x = fmaxf(b.hi.x, p.x); b.hi.y = fmaxf(b.hi.y, p.y); b.hi.z = fmaxf(b.hi.z, p.z);
    }
    __device__ static __forceinline__ void merge(Box& b, const Box& o)
    {
        b.lo.x = fminf(b.lo.x, o.lo.x); b.lo.y = fminf(b.lo.y, o.lo.y); b.lo.z = fminf(b.lo.z, o.lo.z);
        b.hi.x = fmaxf(b.hi.x, o.hi.x); b.hi.y = fmaxf(b.hi.y, o.hi.y); b.hi.z = fmaxf(b.hi.z, o.hi.z);
    }
    __device__ static __forceinline__ Box shfl_xor(const Box& b, int m)
    {
        Box r;
        r.lo.x = __shfl_xor_sync(FULL, b.lo.x, m); r.lo.y = __shfl_xor_sync(FULL, b.lo.y, m);
        r.lo.z = __shfl_xor_sync(FULL, b.lo.z, m); r.hi.x = __shfl_xor_sync(FULL, b.hi.x, m);
        r.hi.y = __shfl_xor_sync(FULL, b.hi.y, m); r.hi.z = __shfl_xor_sync(FULL, b.hi.z, m);
        return r;
    }
    // squared distance from p to box (lower bound of dist2 to any point inside)
    __device__ static __forceinline__ float box_dist2(const Point& p, float lx, float ly, float lz, float hx, float hy, float hz)
    {
        float s = sqr_rn(gap_rn(lx, hx, p.x));
        s = __fadd_rn(s, sqr_rn(gap_rn(ly, hy, p.y)));
        s = __fadd_rn(s, sqr_rn(gap_rn(lz, hz, p.z)));
        return s;
    }
    __device__ static __forceinline__ float box_box_dist2(const Box& a, float lx, float ly, float lz, float hx, float hy, float hz)
    {
        float s = sqr_rn(gap2_rn(a.lo.x, a.hi.x, lx, hx));
        s = __fadd_rn(s, sqr_rn(gap2_rn(a.lo.y, a.hi.y, ly, hy)));
        s = __fadd_rn(s, sqr_rn(gap2_rn(a.lo.z, a.hi.z, lz, hz)));
        return s;
    }
    // diameter test of a box: the squared distance of its corners
    __device__ static __forceinline__ float diag2(const Box& b) { return dist2(b.lo, b.hi); }
    // squared distance from p to the farthest corner of b: an upper bound of
    // dist2(p, y) for every y in b (the same monotone-rounding argument), so
    // <= e2 means every point of b is within eps of p
    __device__ static __forceinline__ float far_dist2(const Point& p, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(p.x, b.lo.x), __fsub_rn(b.hi.x, p.x)));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(p.y, b.lo.y), __fsub_rn(b.hi.y, p.y))));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(p.z, b.lo.z), __fsub_rn(b.hi.z, p.z))));
        return s;
    }
    // the same between two boxes: every pair (a in A, b in B) is within it
    __device__ static __forceinline__ float box_far2(const Box& a, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(b.hi.x, a.lo.x), __fsub_rn(a.hi.x, b.lo.x)));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(b.hi.y, a.lo.y), __fsub_rn(a.hi.y, b.lo.y))));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(b.hi.z, a.lo.z), __fsub_rn(a.hi.z, b.lo.z))));
        return s;
    }
    __device__ static __forceinline__ Node make_node(const Box& L, const Box& R, int left, int right, int split, int last)
    {
        Node n;
        n.a = make_float4(L.lo.x, R.lo.x, L.hi.x, R.hi.x);
        n.b = make_float4(L.lo.y, R.lo.y, L.hi.y, R.hi.y);
        n.c = make_float4(L.lo.z, R.lo.z, L.hi.z, R.hi.z);
        n.m = make_int4(left, right, split, last);
        return n;
    }
};

// A 32-byte record (two float4) in one 256-bit read-only load (sm_100 and
// later); the address must be 32-byte aligned and the data read-only for the
// kernel's lifetime.
__device__ __forceinline__ void ldg256(const void* p, float4& x, float4& y)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w), "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
        : "l"(p));
}

// The same through L2 (ld.global.cg), for records that other threads of the
// running kernel write; volatile, so that it stays after the acquire that
// orders it.
__device__ __forceinline__ void ldcg256(const void* p, float4& x, float4& y)
{
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w), "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void stcg256(void* p, const float4& x, const float4& y)
{
    asm volatile("st.global.cg.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(x.x), "f"(x.y), "f"(x.z),
                 "f"(x.w), "f"(y.x), "f"(y.y), "f"(y.z), "f"(y.w)
                 : "memory");
}

template <> struct Traits<2> {
    using Point = float2;
    struct Box { float4 lo, hi; };  // z unused
    struct Node { float4 a, b; int4 m; };  // 48 B: per axis as in 3D (a: x, b: y), then m

    __device__ static __forceinline__ Point load_point(const float* p, int64_t i)
    {
        return make_float2(p[2 * i], p[2 * i + 1]);
    }
    __device__ static __forceinline__ float coord(const Point& p, int k) { return k == 0 ? p.x : p.y; }
    __device__ static __forceinline__ Box point_box(const Point& p)
    {
        return Box{make_float4(p.x, p.y, 0.f, 0.f), make_float4(p.x, p.y, 0.f, 0.f)};
    }
    __device__ static __forceinline__ Box empty_box()
    {
        return Box{make_float4(INFINITY, INFINITY, 0.f, 0.f), make_float4(-INFINITY, -INFINITY, 0.f, 0.f)};
    }
    __device__ static __forceinline__ void grow(Box& b, const Point& p)
    {
        b.lo.x = fminf(b.lo.x, p.x); b.lo.y = fminf(b.lo.y, p.y);
        b.hi.x = fmaxf(b.hi.x, p.x); b.hi.y = fmaxf(b.hi.y, p.y);
    }
    __device__ static __forceinline__ void merge(Box& b, const Box& o)
    {
        b.lo.x = fminf(b.lo.x, o.lo.x); b.lo.y = fminf(b.lo.y, o.lo.y);
        b.hi.x = fmaxf(b.hi.x, o.hi.x); b.hi.y = fmaxf(b.hi.y, o.hi.y);
    }
    __device__ static __forceinline__ Box shfl_xor(const Box& b, int m)
    {
        Box r = b;
        r.lo.x = __shfl_xor_sync(FULL, b.lo.x, m); r.lo.y = __shfl_xor_sync(FULL, b.lo.y, m);
        r.hi.x = __shfl_xor_sync(FULL, b.hi.x, m); r.hi.y = __shfl_xor_sync(FULL, b.hi.y, m);
        return r;
    }
    __device__ static __forceinline__ float box_dist2(const Point& p, float lx, float ly, float hx, float hy)
    {
        float s = sqr_rn(gap_rn(lx, hx, p.x));
        s = __fadd_rn(s, sqr_rn(gap_rn(ly, hy, p.y)));
        return s;
    }
    __device__ static __forceinline__ float box_box_dist2(const Box& a, float lx, float ly, float hx, float hy)
    {
        float s = sqr_rn(gap2_rn(a.lo.x, a.hi.x, lx, hx));
        s = __fadd_rn(s, sqr_rn(gap2_rn(a.lo.y, a.hi.y, ly, hy)));
        return s;
    }
    __device__ static __forceinline__ float diag2(const Box& b)
    {
        return dist2(make_float2(b.lo.x, b.lo.y), make_float2(b.hi.x, b.hi.y));
    }
    __device__ static __forceinline__ float far_dist2(const Point& p, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(p.x, b.lo.x), __fsub_rn(b.hi.x, p.x)));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(p.y, b.lo.y), __fsub_rn(b.hi.y, p.y))));
        return s;
    }
    __device__ static __forceinline__ float box_far2(const Box& a, const Box& b)
    {
        float s = sqr_rn(fmaxf(__fsub_rn(b.hi.x, a.lo.x), __fsub_rn(a.hi.x, b.lo.x)));
        s = __fadd_rn(s, sqr_rn(fmaxf(__fsub_rn(b.hi.y, a.lo.y), __fsub_rn(a.hi.y, b.lo.y))));
        return s;
    }
    __device__ static __forceinline__ Node make_node(const Box& L, const Box& R, int left, int right, int split, int last)
    {
        Node n;
        n.a = make_float4(L.lo.x, R.lo.x, L.hi.x, R.hi.x);
        n.b = make_float4(L.lo.y, R.lo.y, L.hi.y, R.hi.y);
        n.m = make_int4(left, right, split, last);
        return n;
    }
};

// ---------------------------------------------------------------------------
// Synchronisation-free union-find over a flat labels array (Sec. 4.3): the
// label of a point is its parent; a root is its own label. Unions hook the
// larger root under the smaller with one compare-and-swap, so every root is
// the smallest (sorted) index of its set. find() halves the path as it goes
// ("intermediate pointer jumping"): each visited element is pointed at its
// grandparent, which is always an ancestor, so concurrent finds stay correct.
// Reads bypass L1 (labels change under the feet of other SMs).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(int* L, int x)
{
    int p = __ldcg(L + x);
    while (p != x) {
        int gp = __ldcg(L + p);
        if (gp == p) return p;
        __stcg(L + x, gp);
        x = gp;
        p = __ldcg(L + x);
    }
    return x;
}

// find without writes (for read-only passes once the forest is final)
__device__ __forceinline__ int uf_root(const int* L, int x)
{
    int p = __ldcg(L + x);
    while (p != x) { x = p; p = __ldcg(L + x); }
    return x;
}

// The roots of a and b (into a and b), both chains walked in the same loop
// so that their loads overlap, with the same path halving as uf_find.
__device__ __forceinline__ void uf_find2(int* L, int& a, int& b)
{
    int pa = __ldcg(L + a), pb = __ldcg(L + b);
    while (pa != a || pb != b) {
        const int ga = pa != a ? __ldcg(L + pa) : a;
        const int gb = pb != b ? __ldcg(L + pb) : b;
        if (pa != a) {
            if (ga == pa) {
                a = pa;  // pa is the root
            } else {
                __stcg(L + a, ga);
                a = ga;
            }
        }
        if (pb != b) {
            if (gb == pb) {
                b = pb;
            } else {
                __stcg(L + b, gb);
                b = gb;
            }
        }
        pa = __ldcg(L + a);
        pb = __ldcg(L + b);
    }
}

__device__ __forceinline__ void uf_union(int* L, int a, int b)
{
    for (;;) {
        uf_find2(L, a, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicCAS(L + b, b, a);
        if (old == b) return;
    }
}

// A non-core point y joins the cluster of core point x if it has not joined
// one yet (labels[y] == y). The compare-and-swap replaces the critical
// section of Algorithm 3 (Sec. 3.2): y is never a union target, so a border
// point cannot bridge two clusters.
__device__ __forceinline__ void uf_claim(int* L, int y, int x)
{
    if (__ldcg(L + y) != y) return;
    int r = uf_find(L, x);
    atomicCAS(L + y, y, r);
}

// atomicMin(&a[key], v) for the lanes of the warp that are `active`, with the
// lanes that share a key combined first: one atomic per distinct key (the
// canonical-label minimum, where every core point of a large cluster would
// otherwise hit the same word). All 32 lanes must call it.
__device__ __forceinline__ void warp_atomic_min(int32_t* a, int key, int32_t v, bool active)
{
    const unsigned act = __ballot_sync(FULL, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(act, key);
    const int32_t m = __reduce_min_sync(peers, v);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(a + key, m);
}

// relaxed global loads/stores for look-back status words
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(uint64_t* p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// float <-> order-preserving uint (for atomic min/max of floats)
__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(uint32_t u)
{
    uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

// Count of kernels this library has launched (for the benchmark's claim of
// how many of its kernels ran); every launcher adds what it launches.
void note_launches(int k);
int64_t launches_so_far();

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).
// ---------------------------------------------------------------------------

// sort.cu
// passes of an LSD radix sort over `bits` key bits (SORT_DIGIT_BITS-bit digits)
__host__ __device__ __forceinline__ int sort_passes(int bits) { return (bits + SORT_DIGIT_BITS - 1) / SORT_DIGIT_BITS; }

// Device-side control of a sort inside the pipeline (all null: a plain sort).
//  * gate / gate_val: the sort runs only if *gate == gate_val (the algorithm
//    the run chose on the device);
//  * abort: the sort does not run if *abort is nonzero when a pass starts;
//  * key_bits: the key bits actually used, known on the device only, at most
//    the `bits` the host launched for: passes beyond them do nothing, and the
//    keys are written to the buffer (sort_dev_input_alt) from which the
//    passes that do run leave the result where all `bits` would have.
struct SortCtl {
    const uint32_t* gate = nullptr;
    uint32_t gate_val = 0;
    const uint32_t* abort = nullptr;
    const uint32_t* key_bits = nullptr;
};
// with host_passes launched and dev_passes needed: does the input go to the
// alternate buffer?
__host__ __device__ __forceinline__ bool sort_dev_input_alt(int host_passes, int dev_passes)
{
    return ((host_passes - dev_passes) & 1) != 0;
}

struct SortBuffers {
    void* keys_alt;        // n keys
    uint32_t* vals_alt;    // n values
    uint32_t* hist;        // SORT_MAX_PASSES * SORT_RADIX
    uint32_t* status;      // passes * tiles * SORT_RADIX (8-byte aligned)
    uint32_t* counters;    // SORT_MAX_PASSES
    uint32_t* err;         // device error word (ERR_SORT_TIMEOUT)
    SortCtl ctl;           // device-side control (pipeline sorts only)
};
// Test hooks of the look-back wait: the wait limit of every later sort
// (spins; negative restores SPIN_LIMIT) and, if stall_first_tile, tile 0 of
// every pass withholding its status words, so that every later tile's wait
// on it runs out (the sort then reports ERR_SORT_TIMEOUT and writes nothing
// from those tiles).
void sort_set_test_hooks(int64_t wait_limit, int stall_first_tile);
int64_t sort_tiles(int64_t n, int key_bytes);
size_t sort_status_words(int64_t n, int key_bytes, int bits);
// Sorts (keys, vals) by the low `bits` bits. On return *in_alt tells whether
// the sorted data ended in the alternate buffers.
cudaError_t sort_pairs_u32(uint32_t* keys, uint32_t* vals, int64_t n, int bits, const SortBuffers& sb,
                           cudaStream_t s, bool* in_alt);
cudaError_t sort_pairs_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, const SortBuffers& sb,
                           cudaStream_t s, bool* in_alt);
// Keys only, by bits [shift0, shift0 + bits): for words key << shift0 | index
// (distinct, so the order equals the stable order of the keys). The passes'
// values buffers are not touched.
cudaError_t sort_keys_u64(uint64_t* keys, int64_t n, int shift0, int bits, const SortBuffers& sb, cudaStream_t s,
                          bool* in_alt);

// scan.cu: out[i] = op(in[0..i]) (inclusive) or op(in[0..i-1]) (exclusive, out[0] = identity)
enum ScanOp { SCAN_ADD = 0, SCAN_MAX = 1 };
size_t scan_temp_words(int64_t n);
cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t n, ScanOp op, bool inclusive, int32_t* temp,
                     cudaStream_t s);

}  // namespace gbd
