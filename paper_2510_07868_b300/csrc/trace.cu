// BVH traversal for sm_103a: the closest hit of the extension stage of one bounce (Sec. 2,
// the wavefront formulation the method runs in) and the any-hit test of next-event
// estimation's shadow rays.  Persistent warps claim rays from the live queue; the
// traversal stack lives in shared memory.
#include <cfloat>
#include <cuda_fp16.h>

#include "bvh.h"
#include "wavefront.cuh"

namespace nrrs {

namespace {

constexpr int kExtendThreads = 256;
constexpr int kStack = 40;  // BVH build depth is capped below this
// A BVH2 whose deepest path holds at most this many inner nodes (the three-room scene's
// 1,000,026 triangles: 24) is traversed with a stack of this size: 16 KB less shared
// memory per block, which the SM gives to the L1 cache that holds the nodes.
constexpr int kShortStack = 24;
constexpr int kSteps = 8;   // node visits between ray fetch rounds

__device__ __forceinline__ uint32_t fbits(float f) { return __float_as_uint(f); }

// ------------------------------------------------------------------ traversal
struct Hit {
    float t;
    int slot;      // BVH-order triangle slot, -1 = miss
    uint32_t id;   // original triangle index (tie-break)
};

// One ray's traversal state.  The stack lives in shared memory, one column per thread
// (entry k at stk[k * stride]) so that lanes hit different banks.
struct Ray {
    V3 o, d, inv, oi;
    int node, sp;
    // per axis the byte selector that orders a binary16 (lo, hi) word as (near, far) for
    // this direction: identity when the component is positive, a half swap when negative
    uint32_t sel_x, sel_y, sel_z;
};

// A direction component that is exactly zero would make the slab products 0 * inf and
// inf - inf (NaN) and lose boxes; the reciprocal uses a tiny component of the same sign
// instead (the slab then spans everything or nothing along that axis, as it should).
__device__ __forceinline__ float safe_rcp(float x) {
    return 1.0f / (fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x);
}

// t_max bounds the query; a shadow ray (t_max finite) starts with id 0 so that a hit at
// exactly t_max does not count (the oracle's test is t < t_max).
__device__ __forceinline__ void ray_init(Ray& r, V3 o, V3 d, int root, Hit& h,
                                         float t_max = FLT_MAX) {
    r.o = o;
    r.d = d;
    r.inv = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    r.oi = v3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    r.sel_x = r.inv.x < 0.0f ? 0x1032u : 0x3210u;
    r.sel_y = r.inv.y < 0.0f ? 0x1032u : 0x3210u;
    r.sel_z = r.inv.z < 0.0f ? 0x1032u : 0x3210u;
    r.node = root;
    r.sp = 0;
    h = Hit{t_max, -1, t_max == FLT_MAX ? 0xFFFFFFFFu : 0u};
}

// Moller-Trumbore against triangle reference s; keeps the closest hit, equal distances
// going to the lower original triangle index.
__device__ __forceinline__ void intersect_tri(const SceneView& sc, const Ray& r, Hit& h, int s) {
    const float4 t0 = __ldg(&sc.tris[3 * s + 0]);
    const float4 t1 = __ldg(&sc.tris[3 * s + 1]);
    const float4 t2 = __ldg(&sc.tris[3 * s + 2]);
    const V3 v0 = xyz(t0), e1 = xyz(t1), e2 = xyz(t2);
    const V3 pv = cross3(r.d, e2);
    const float det = dot3(e1, pv);
    if (det == 0.0f) return;
    const float idet = 1.0f / det;
    const V3 tv = r.o - v0;
    const float u = dot3(tv, pv) * idet;
    if (u < 0.0f || u > 1.0f) return;
    const V3 qv = cross3(tv, e1);
    const float v = dot3(r.d, qv) * idet;
    if (v < 0.0f || u + v > 1.0f) return;
    const float t = dot3(e2, qv) * idet;
    const uint32_t id = fbits(t0.w);
    if (t > 0.0f && (t < h.t || (t == h.t && id < h.id))) {
        h.t = t;
        h.slot = s;
        h.id = id;
    }
}

// Slab test of one box against the ray, clipped to (0, h.t]; writes the entry distance.
__device__ __forceinline__ bool slab(const Ray& r, float hit_t, float lx, float hx, float ly,
                                     float hy, float lz, float hz, float* tn) {
    const float ax = fmaf(lx, r.inv.x, -r.oi.x), bx = fmaf(hx, r.inv.x, -r.oi.x);
    const float ay = fmaf(ly, r.inv.y, -r.oi.y), by = fmaf(hy, r.inv.y, -r.oi.y);
    const float az = fmaf(lz, r.inv.z, -r.oi.z), bz = fmaf(hz, r.inv.z, -r.oi.z);
    const float n = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.0f));
    const float f = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), hit_t));
    *tn = n;
    return n <= f;
}

// Visits one four-wide node: the four child boxes are tested together, leaf children
// are intersected at once, and the inner children entered are ordered near to far: the
// nearest is visited next and the others pushed farthest first.  The same closest hit
// as the BVH2 visit (same triangle test, same tie rule).  Returns true when the query
// ends.
__device__ __forceinline__ bool visit_node4(const SceneView& sc, Ray& r, Hit& h, int* stk,
                                            int stride) {
    const float4* N = sc.nodes4 + 8 * r.node;
    const float4 lx = __ldg(N + 0), hx = __ldg(N + 1), ly = __ldg(N + 2), hy = __ldg(N + 3);
    const float4 lz = __ldg(N + 4), hz = __ldg(N + 5);
    const int4 ch = __ldg(reinterpret_cast<const int4*>(N + 6));
    const int4 cn = __ldg(reinterpret_cast<const int4*>(N + 7));
    float tn[4];
    bool hit[4];
    hit[0] = slab(r, h.t, lx.x, hx.x, ly.x, hy.x, lz.x, hz.x, &tn[0]);
    hit[1] = slab(r, h.t, lx.y, hx.y, ly.y, hy.y, lz.y, hz.y, &tn[1]);
    hit[2] = slab(r, h.t, lx.z, hx.z, ly.z, hy.z, lz.z, hz.z, &tn[2]);
    hit[3] = slab(r, h.t, lx.w, hx.w, ly.w, hy.w, lz.w, hz.w, &tn[3]);
    const int code[4] = {ch.x, ch.y, ch.z, ch.w};
    const int count[4] = {cn.x, cn.y, cn.z, cn.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!hit[k] || code[k] >= 0) continue;
        const int first = ~code[k];
        for (int j = 0; j < count[k]; ++j) intersect_tri(sc, r, h, first + j);
    }
    // inner children still in reach after the leaf hits, sorted by entry distance
    float key[4];
    int nxt[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool in = hit[k] && code[k] >= 0 && tn[k] <= h.t;
        key[k] = in ? tn[k] : FLT_MAX;
        nxt[k] = in ? code[k] : -1;
    }
    auto cswap = [&](int i, int j) {
        if (key[j] < key[i]) {
            const float tk = key[i]; key[i] = key[j]; key[j] = tk;
            const int tc = nxt[i]; nxt[i] = nxt[j]; nxt[j] = tc;
        }
    };
    cswap(0, 1); cswap(2, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
#pragma unroll
    for (int k = 3; k >= 1; --k)
        if (nxt[k] >= 0 && r.sp < kStack) stk[(r.sp++) * stride] = nxt[k];
    if (nxt[0] >= 0) {
        r.node = nxt[0];
        return false;
    }
    if (r.sp == 0) return true;
    r.node = stk[(--r.sp) * stride];
    return false;
}

// ------------------------------------------------------------------ eight-wide tree
// Key order of a node's children for a ray of direction octant `oct` (bit k set when the
// direction's component k is negative): slot s (bit k set = the child's centre on the +
// side of axis k) gets key s ^ oct, so the children nearest the corner the ray comes
// from come first.  Permutes an 8-bit mask of slots into key order.
__device__ __forceinline__ uint32_t slot_to_key_mask(uint32_t m, uint32_t oct) {
    if (oct & 1u) m = ((m & 0x55u) << 1) | ((m & 0xAAu) >> 1);
    if (oct & 2u) m = ((m & 0x33u) << 2) | ((m & 0xCCu) >> 2);
    if (oct & 4u) m = ((m & 0x0Fu) << 4) | ((m & 0xF0u) >> 4);
    return m;
}

// Byte c of the pair as the float 2^23 + byte: one byte permute builds its bits
// (0x4B00_00bb), so no integer-to-float conversion is needed.
__device__ __forceinline__ float byte_f(uint2 w, int c) {
    return __uint_as_float(__byte_perm(c < 4 ? w.x : w.y, 0x4B000000u, 0x7650u + (uint32_t)(c & 3)));
}

// Visits one eight-wide node (bvh8.cu's layout): decodes the eight quantised child
// boxes (origin plus byte times a power of two per axis, the near and far planes picked
// by the ray's direction signs), intersects the triangles of the leaf children it
// enters, and returns the inner children entered that are still in reach as a mask in
// key order, with the node's first-child index and inner mask.  A plane's distance is
// fma(2^23 + byte, s, a - 2^23 s) with s = 2^e / d: the bias term rounds by at most half
// a step of s, inside the one-step widening the builder gives every box.
__device__ __forceinline__ uint32_t visit_node8(const SceneView& sc, const Ray& r, Hit& h,
                                                int node, uint32_t oct, uint32_t* base,
                                                uint32_t* imask, int* first) {
    const uint4* N = sc.nodes8 + 5 * (size_t)node;
    const uint4 w0 = __ldg(N + 0), w1 = __ldg(N + 1);
    const uint4 w2 = __ldg(N + 2), w3 = __ldg(N + 3), w4 = __ldg(N + 4);
    const float sx = __uint_as_float((w0.w & 0xFFu) << 23) * r.inv.x;
    const float sy = __uint_as_float(((w0.w >> 8) & 0xFFu) << 23) * r.inv.y;
    const float sz = __uint_as_float(((w0.w >> 16) & 0xFFu) << 23) * r.inv.z;
    const float ax = fmaf(__uint_as_float(w0.x), r.inv.x, -r.oi.x) - 8388608.0f * sx;
    const float ay = fmaf(__uint_as_float(w0.y), r.inv.y, -r.oi.y) - 8388608.0f * sy;
    const float az = fmaf(__uint_as_float(w0.z), r.inv.z, -r.oi.z) - 8388608.0f * sz;
    const uint2 lox = make_uint2(w2.x, w2.y), loy = make_uint2(w2.z, w2.w);
    const uint2 loz = make_uint2(w3.x, w3.y), hix = make_uint2(w3.z, w3.w);
    const uint2 hiy = make_uint2(w4.x, w4.y), hiz = make_uint2(w4.z, w4.w);
    const uint2 nx = (oct & 1u) ? hix : lox, fx = (oct & 1u) ? lox : hix;
    const uint2 ny = (oct & 2u) ? hiy : loy, fy = (oct & 2u) ? loy : hiy;
    const uint2 nz = (oct & 4u) ? hiz : loz, fz = (oct & 4u) ? loz : hiz;
    const uint32_t im = w0.w >> 24;
    float tn[8];
    uint32_t hits = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float n0 = fmaxf(fmaf(byte_f(nx, c), sx, ax), fmaf(byte_f(ny, c), sy, ay));
        const float f0 = fminf(fmaf(byte_f(fx, c), sx, ax), fmaf(byte_f(fy, c), sy, ay));
        tn[c] = fmaxf(n0, fmaxf(fmaf(byte_f(nz, c), sz, az), 0.0f));
        const float tf = fminf(f0, fminf(fmaf(byte_f(fz, c), sz, az), h.t));
        hits |= (tn[c] <= tf ? 1u : 0u) << c;
    }
    // leaf children entered: their triangles now (they can shorten h.t for the rest)
    uint32_t leaves = hits & ~im;
    while (leaves) {
        const int c = __ffs(leaves) - 1;
        leaves &= leaves - 1u;
        const uint32_t meta = ((c < 4 ? w1.z : w1.w) >> (8 * (c & 3))) & 0xFFu;
        const int first = (int)(w1.y + (meta & 31u));
        for (int j = 0; j < (int)(meta >> 5); ++j) intersect_tri(sc, r, h, first + j);
    }
    uint32_t inner = 0;
    float best = FLT_MAX;
    int nearest = -1;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if ((hits & im & (1u << c)) && tn[c] <= h.t) {
            inner |= 1u << c;
            if (tn[c] < best) {
                best = tn[c];
                nearest = c;
            }
        }
    *base = w1.x;
    *imask = im;
    *first = nearest;
    return slot_to_key_mask(inner, oct);
}

// One step of the eight-wide traversal: visit r.node, then descend into its nearest
// child entered (least entry distance; the others wait on the stack in key order), or
// take the next child of the last group on the stack.  A stack entry is (node << 8 | the mask of its children still to visit, in key
// order); the node's first-child index and inner mask are read again on the pop.  At
// most one entry per tree level, so the build's depth bound keeps it within kStack.
// Returns true when the query ends.
__device__ __forceinline__ bool step_node8(const SceneView& sc, Ray& r, Hit& h, int* stk,
                                           int stride, uint32_t oct) {
    uint32_t base, imask;
    int nearest;
    uint32_t keys = visit_node8(sc, r, h, r.node, oct, &base, &imask, &nearest);
    uint32_t group = (uint32_t)r.node;
    if (keys) {
        // descend into the nearest child entered first; the others wait in key order
        const uint32_t k = (uint32_t)nearest ^ oct;
        keys &= ~(1u << k);
        if (keys) stk[(r.sp++) * stride] = (int)(group << 8 | keys);
        r.node = (int)(base + (uint32_t)__popc(imask & ((1u << nearest) - 1u)));
        return false;
    }
    {
        if (r.sp == 0) return true;
        const uint32_t e = (uint32_t)stk[(--r.sp) * stride];
        group = e >> 8;
        keys = e & 0xFFu;
        const uint4* N = sc.nodes8 + 5 * (size_t)group;
        imask = __ldg(&N[0].w) >> 24;
        base = __ldg(&N[1].x);
    }
    const uint32_t k = (uint32_t)(__ffs(keys) - 1);
    keys &= keys - 1u;
    const uint32_t slot = k ^ oct;
    if (keys) stk[(r.sp++) * stride] = (int)(group << 8 | keys);
    r.node = (int)(base + (uint32_t)__popc(imask & ((1u << slot) - 1u)));
    return false;
}

// The (lo, hi) pair of binary16 values in one word of a half-precision node.
__device__ __forceinline__ float2 half_pair(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

// Three-operand minimum and maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Slab test of a binary16 box whose axis words hold (lo, hi): each word is first put in
// (near, far) order for the ray's direction, so no per-axis min/max is needed.  With
// lo <= hi and a fixed sign of 1/d the rounded plane distances keep their order, so the
// entry and exit distances equal slab()'s bit for bit.
__device__ __forceinline__ bool slab_half(const Ray& r, float hit_t, uint32_t wx, uint32_t wy,
                                          uint32_t wz, float* tn) {
    const float2 x = half_pair(__byte_perm(wx, 0u, r.sel_x));
    const float2 y = half_pair(__byte_perm(wy, 0u, r.sel_y));
    const float2 z = half_pair(__byte_perm(wz, 0u, r.sel_z));
    // (near, far) distances per axis, two correctly rounded FMAs per instruction
    const float2 tx = __ffma2_rn(x, make_float2(r.inv.x, r.inv.x), make_float2(-r.oi.x, -r.oi.x));
    const float2 ty = __ffma2_rn(y, make_float2(r.inv.y, r.inv.y), make_float2(-r.oi.y, -r.oi.y));
    const float2 tz = __ffma2_rn(z, make_float2(r.inv.z, r.inv.z), make_float2(-r.oi.z, -r.oi.z));
    const float n = max3f(tx.x, ty.x, fmaxf(tz.x, 0.0f));
    const float f = min3f(tx.y, ty.y, fminf(tz.y, hit_t));
    *tn = n;
    return n <= f;
}

// One inner-node step of the BVH2 traversal for every lane of the warp, free of divergent
// branches: a lane that does not go (`go` false) reads the root's node and keeps its
// state, so all lanes issue the same instructions.  Both child boxes are tested; leaf
// children entered are not intersected here but held as their raw child codes in the
// first free of three slots (leaf tests are postponed, see k_trace); inner children
// entered are descended near-first with the far one pushed; with neither, the next
// node comes off the stack (node -1: nothing left).  HALF: the 32-byte binary16 nodes
// (boxes rounded outward: one memory sector per visit, the same closest hits; a leaf's
// code packs its first reference and count), else the 64-byte FP32 nodes (a leaf's code
// is ~first, its count a field of its own, held in n0..n2 beside the slots).
template <bool HALF, int STACK>
__device__ __forceinline__ void step_bvh2(const SceneView& sc, Ray& r, const Hit& h, int* stk,
                                          int stride, bool go, int& code0, int& code1,
                                          int& code2, int& n0, int& n1, int& n2) {
    const int node = go ? r.node : 0;
    float t0n, t1n;
    bool b0, b1;
    int c0, c1, k0 = 0, k1 = 0;
    if (HALF) {
        const uint4 p = __ldg(&sc.nodes_h[2 * node + 0]);
        const uint4 q = __ldg(&sc.nodes_h[2 * node + 1]);
        b0 = slab_half(r, h.t, p.x, p.y, p.z, &t0n);
        b1 = slab_half(r, h.t, p.w, q.x, q.y, &t1n);
        c0 = (int)q.z;
        c1 = (int)q.w;
    } else {
        const float4 a = __ldg(&sc.nodes[4 * node + 0]);
        const float4 b = __ldg(&sc.nodes[4 * node + 1]);
        const float4 c = __ldg(&sc.nodes[4 * node + 2]);
        const int4 e = __ldg(reinterpret_cast<const int4*>(&sc.nodes[4 * node + 3]));
        b0 = slab(r, h.t, a.x, a.y, a.z, a.w, c.x, c.y, &t0n);
        b1 = slab(r, h.t, b.x, b.y, b.z, b.w, c.z, c.w, &t1n);
        c0 = e.x;
        c1 = e.y;
        k0 = e.z;
        k1 = e.w;
    }
    b0 = b0 && go;
    b1 = b1 && go;
    // leaves entered fill the free slots in order; a lane holding one leaf goes on
    // descending (it stops at two), so a node can add at most two more
    const int na = b0 && c0 < 0 ? c0 : 0, nb = b1 && c1 < 0 ? c1 : 0;
    const bool empty = code0 == 0;
    const int first = na != 0 ? na : nb, second = na != 0 ? nb : 0;
    if (!HALF) {
        const int kf = na != 0 ? k0 : k1, ks = na != 0 ? k1 : 0;
        n2 = go && !empty ? ks : n2;
        n1 = go ? (empty ? ks : kf) : n1;
        n0 = go && empty ? kf : n0;
    }
    code2 = go && !empty ? second : code2;
    code1 = go ? (empty ? second : first) : code1;
    code0 = go && empty ? first : code0;
    const bool i0 = b0 && c0 >= 0, i1 = b1 && c1 >= 0;
    const bool first1 = i1 && (!i0 || t1n < t0n);
    const int near_c = first1 ? c1 : c0;
    const int far_c = first1 ? c0 : c1;
    const bool push = i0 && i1 && r.sp < STACK;
    const bool none = go && !i0 && !i1;
    const bool pop = none && r.sp > 0;
    int* slot = stk + (pop ? r.sp - 1 : r.sp) * stride;
    if (push) *slot = far_c;
    const int popped = pop ? *slot : -1;
    r.sp += push ? 1 : pop ? -1 : 0;
    r.node = none ? popped : (go ? near_c : r.node);
}

// Intersects the triangles of a held leaf (raw child code, 0 = an empty slot; n its
// count in the FP32 nodes).
template <bool HALF>
__device__ __forceinline__ void test_leaf(const SceneView& sc, const Ray& r, Hit& h, int code,
                                          int n) {
    if (code >= 0) return;
    const uint32_t v = ~(uint32_t)code;
    const int first = HALF ? (int)(v & kLeafFirstMask) : (int)v;
    const int count = HALF ? (int)(v >> kLeafFirstBits) : n;
    for (int k = 0; k < count; ++k) intersect_tri(sc, r, h, first + k);
}

// One round of the BVH2 traversal for the warp: up to kSteps inner-node steps, then the
// tests of the leaves held.  The warp keeps stepping while some lane that still
// traverses holds no leaf yet; lanes that hold one step along speculatively (Aila and
// Laine's speculative while-while), which keeps lanes busy that would otherwise wait.
template <bool HALF, int STACK>
__device__ __forceinline__ void round_bvh2(const SceneView& sc, Ray& r, Hit& h, int* stk,
                                           int stride, bool active) {
    bool go = active && r.node >= 0;
    int code0 = 0, code1 = 0, code2 = 0, n0 = 0, n1 = 0, n2 = 0;
#pragma unroll
    for (int step = 0; step < kSteps; ++step) {
        step_bvh2<HALF, STACK>(sc, r, h, stk, stride, go, code0, code1, code2, n0, n1, n2);
        go = go && r.node >= 0 && (code1 | code2) == 0;
        if (!__any_sync(0xffffffffu, go && code0 == 0)) break;
    }
    test_leaf<HALF>(sc, r, h, code0, n0);
    test_leaf<HALF>(sc, r, h, code1, n1);
    test_leaf<HALF>(sc, r, h, code2, n2);
}

// Extension of depth `depth`, part 1: the closest hit of every live ray.  Persistent
// warps fetch rays dynamically: a lane whose query has ended stores its hit and takes
// the next unclaimed slot, so lanes stay busy despite divergent traversal lengths.  On
// the BVH2 the leaf tests are postponed (Aila and Laine's while-while traversal): lanes
// descend through inner nodes until every lane of the warp holds a leaf or has
// finished, then test their leaves together (round_bvh2).  Each slot's hit depends only on that slot's ray (the
// closest hit with the lower-index tie rule does not depend on the visiting order), so
// the result is deterministic.
// ANY: the shadow rays of next-event estimation, one per slot (t_max <= 0: none); the
// query ends at the first hit before t_max, and an unoccluded ray adds its
// contribution to the slot's deposit.
template <int WIDTH, bool ANY, int STACK = kStack>
__global__ void __launch_bounds__(kExtendThreads, 4)
k_trace(SceneView sc, QueueView cur, WorkView w, int depth, JobWork jobs) {
    __shared__ int s_stack[STACK * kExtendThreads];
    int* stk = s_stack + threadIdx.x;
    DevStats* st = w.st;
    const long long n = st->live[depth - 1];
    unsigned long long* ctr = ANY ? &st->sfetch[depth - 1] : &st->fetch[depth - 1];
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    long long idx = -1;
    bool exhausted = false;
    Ray ray;
    Hit h;
    for (;;) {
        const bool need = idx < 0 && !exhausted;
        const unsigned need_mask = __ballot_sync(0xffffffffu, need);
        if (need_mask) {
            const int leader = __ffs(need_mask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(need_mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                const long long my = (long long)base + __popc(need_mask & lt_mask);
                if (my < n) {
                    const float4 o4 = ANY ? w.sh_o[my] : cur.o[my];
                    if (!ANY || o4.w > 0.0f) {  // a slot without a shadow ray is skipped
                        idx = my;
                        // a batched render starts each ray at the root of its job's scene
                        int root = 0;
                        if (jobs.job) {
                            const uint32_t pix = __float_as_uint(ANY ? w.dep[idx].w : o4.w);
                            const JobDev* J = jobs.job + job_of_pixel(jobs.job, jobs.n, pix);
                            root = WIDTH == 4 ? __ldg(&J->root4) : WIDTH == 8 ? 0 : __ldg(&J->root);
                        }
                        if (ANY)
                            ray_init(ray, xyz(o4), xyz(w.sh_d[idx]), root, h, o4.w);
                        else
                            ray_init(ray, xyz(o4), xyz(cur.d[idx]), root, h);
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        // lanes that skipped a slot claim again on the next round
        if (__all_sync(0xffffffffu, idx < 0 && exhausted)) break;
        if (WIDTH == 8) {
            if (idx < 0) continue;
            const uint32_t oct = (ray.inv.x < 0.0f ? 1u : 0u) | (ray.inv.y < 0.0f ? 2u : 0u) |
                                 (ray.inv.z < 0.0f ? 4u : 0u);
            bool done = false;
            for (int step = 0; step < kSteps && !done; ++step)
                done = step_node8(sc, ray, h, stk, kExtendThreads, oct) || (ANY && h.slot >= 0);
            if (!done) continue;
        } else if (WIDTH == 4) {
            if (idx < 0) continue;
            bool done = false;
            for (int step = 0; step < kSteps && !done; ++step)
                done = visit_node4(sc, ray, h, stk, kExtendThreads) || (ANY && h.slot >= 0);
            if (!done) continue;
        } else {
            // every lane of the warp runs the round (its votes need all of them)
            if (sc.nodes_h)
                round_bvh2<true, STACK>(sc, ray, h, stk, kExtendThreads, idx >= 0);
            else
                round_bvh2<false, STACK>(sc, ray, h, stk, kExtendThreads, idx >= 0);
            if (idx < 0) continue;
            if (ANY && h.slot >= 0) ray.node = -1;  // occluded: the query is over
            if (ray.node >= 0) continue;
        }
        if (ANY) {
            if (h.slot < 0) {
                const float4 c = w.sh_c[idx];
                float4 e = w.dep[idx];
                e.x += c.x;
                e.y += c.y;
                e.z += c.z;
                w.dep[idx] = e;
            }
        } else {
            w.hit[idx] = make_float2(h.t, __int_as_float(h.slot));
        }
        idx = -1;
    }
}

}  // namespace

int extend_block_threads() { return kExtendThreads; }

int trace_stack_entries() { return kStack; }

int trace_short_stack_entries() { return kShortStack; }

int max_blocks_trace() {
    int nb = 1 << 30;
    int n[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], k_trace<2, false>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], k_trace<4, false>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[2], k_trace<2, true>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[3], k_trace<4, true>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[4], k_trace<8, false>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[5], k_trace<8, true>, kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[6], k_trace<2, false, kShortStack>,
                                                  kExtendThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[7], k_trace<2, true, kShortStack>,
                                                  kExtendThreads, 0);
    for (int k = 0; k < 8; ++k) nb = n[k] < nb ? n[k] : nb;
    return nb < 1 ? 1 : nb;
}

void launch_trace(const SceneView& sc, QueueView cur, const WorkView& w, int depth, int grid,
                  const JobWork& jobs, cudaStream_t s) {
    if (sc.nodes8)
        k_trace<8, false><<<grid, kExtendThreads, 0, s>>>(sc, cur, w, depth, jobs);
    else if (sc.nodes4)
        k_trace<4, false><<<grid, kExtendThreads, 0, s>>>(sc, cur, w, depth, jobs);
    else if (sc.short_stack)
        k_trace<2, false, kShortStack><<<grid, kExtendThreads, 0, s>>>(sc, cur, w, depth, jobs);
    else
        k_trace<2, false><<<grid, kExtendThreads, 0, s>>>(sc, cur, w, depth, jobs);
}

void launch_shadow(const SceneView& sc, const WorkView& w, int depth, int grid,
                   const JobWork& jobs, cudaStream_t s) {
    const QueueView none{};
    if (sc.nodes8)
        k_trace<8, true><<<grid, kExtendThreads, 0, s>>>(sc, none, w, depth, jobs);
    else if (sc.nodes4)
        k_trace<4, true><<<grid, kExtendThreads, 0, s>>>(sc, none, w, depth, jobs);
    else if (sc.short_stack)
        k_trace<2, true, kShortStack><<<grid, kExtendThreads, 0, s>>>(sc, none, w, depth, jobs);
    else
        k_trace<2, true><<<grid, kExtendThreads, 0, s>>>(sc, none, w, depth, jobs);
}

}  // namespace nrrs
