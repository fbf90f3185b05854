// GPU build of the compressed eight-wide BVH the extension stage can traverse instead of
// the host-built BVH2 (the paper's renderer traces with OptiX, Sec. 4 "System"; this is
// the hand-written stand-in for its acceleration structure).
//
// Build, all on the device:
//   1. per triangle its box (grown by a margin of 1e-5 of the scene size plus 4 ulp of
//      the largest coordinate, as the BVH2's boxes are, so FP32 slab tests never cut off
//      a hit) and the 30-bit Morton code of
//      the box centre; a stable LSD radix sort of the codes (8-bit digits);
//   2. PLOC (Meister & Bittner 2018): clusters in Morton order; every cluster finds the
//      neighbour within 16 positions whose merged box has the least surface area; mutual
//      nearest neighbours merge; the survivors are compacted in order; repeat until one
//      cluster is left.  Merges and survivors are numbered by prefix sums, so the tree is
//      the same on every run;
//   3. collapse to eight-wide nodes, one tree level per launch: a node takes its BVH2
//      node's two children and opens the child of largest area until it has eight or no
//      child can open (a child holding at most kLeafTris triangles stays whole, as a
//      leaf);
//      children are assigned slots by the octant of their centre relative to the node's
//      (a ray of direction octant r visits slot order s ^ r, near corners first), and
//      each node's inner children and leaf triangles are numbered by prefix sums;
//   4. quantisation (Ylitie, Karras & Laine 2017): per node an origin and a power-of-two
//      scale per axis, each child box as six bytes rounded outward and then widened by
//      one more step on each side (the origin sits two steps below the node's box and
//      252 steps span it), which leaves the traversal's byte decoding room for a rounding
//      error of up to half a step.
//
// Node (80 bytes, 5 x uint4):
//   w0 = (origin x, y, z (FP32 bits), exponent x | y << 8 | z << 16 | inner mask << 24)
//        exponents biased by 127: the scale of axis k is 2^(e_k - 127)
//   w1 = (first inner child, first triangle, meta bytes of slots 0-3, of slots 4-7)
//        meta: 0 = empty or inner slot; a leaf = count << 5 | triangle offset
//   w2 = (lo x bytes 0-3, lo x 4-7, lo y 0-3, lo y 4-7)
//   w3 = (lo z 0-3, lo z 4-7, hi x 0-3, hi x 4-7)
//   w4 = (hi y 0-3, hi y 4-7, hi z 0-3, hi z 4-7)
// Child box of slot c along axis k: [p_k + lo_k[c] 2^e_k, p_k + hi_k[c] 2^e_k].  An empty
// slot has lo = 255, hi = 0 (no ray enters it).  Inner children of a node are stored
// consecutively in slot order; so are the triangles of its leaves (each triangle once),
// in the 3 x float4 layout of the BVH2's references.
#include <cfloat>
#include <cstdio>
#include <vector>

#include "bvh8.h"

#include <algorithm>
#include <cstring>
#include <utility>

namespace nrrs {

namespace {

constexpr int kRadius = 16;        // PLOC search radius
// Most triangles a leaf slot holds.  Measured (traversal ms per frame, occluded room /
// 200k / 1M triangles): 3 per leaf 2.16 / 9.19 / 132, 2 per leaf 2.00 / 8.71 / 118, 1 per
// leaf 2.06 / 9.58 / 110.
constexpr int kLeafTris = 2;
constexpr int kThreads = 256;

struct Box3 {
    float3 lo, hi;
};

__device__ __forceinline__ float3 fmin3(float3 a, float3 b) {
    return make_float3(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z));
}
__device__ __forceinline__ float3 fmax3(float3 a, float3 b) {
    return make_float3(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z));
}
__device__ __forceinline__ float half_area(float3 lo, float3 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// 10 bits spread to every third bit (bit i to bit 3 i).
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_prim_codes(const float* __restrict__ tri, int n, float3 lo, float3 scale,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* v = tri + 9 * (size_t)i;
    float3 a = make_float3(v[0], v[1], v[2]);
    float3 b = a;
    for (int k = 1; k < 3; ++k) {
        const float3 p = make_float3(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
        a = fmin3(a, p);
        b = fmax3(b, p);
    }
    const float cx = 0.5f * (a.x + b.x), cy = 0.5f * (a.y + b.y), cz = 0.5f * (a.z + b.z);
    auto q = [](float c, float l, float s) {
        const float t = (c - l) * s;
        return (uint32_t)fminf(fmaxf(t, 0.0f), 1023.0f);
    };
    keys[i] = spread3(q(cx, lo.x, scale.x)) | (spread3(q(cy, lo.y, scale.y)) << 1) |
              (spread3(q(cz, lo.z, scale.z)) << 2);
    vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------- radix sort (stable)
// Per block of kThreads keys: digit counts; hist is digit-major: hist[d * nb + b].
__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift, int nb,
                          uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter with the block's keys in order: rank = digit offset of the block + keys of the
// same digit in earlier warps + earlier lanes of the same digit in this warp.
__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                             int shift, int nb, const uint32_t* __restrict__ off) {
    __shared__ uint32_t wcnt[kThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kThreads / 32) * 256; k += kThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const bool live = i < n;
    const uint32_t key = live ? kin[i] : 0u;
    const uint32_t d = live ? (key >> shift) & 255u : 256u;  // tail lanes: their own value
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int rank_w = __popc(same & ((1u << lane) - 1u));
    if (live && rank_w == 0) wcnt[w][d] = __popc(same);
    __syncthreads();
    if (threadIdx.x < 256) {  // exclusive prefix over warps, per digit
        uint32_t run = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            const uint32_t c = wcnt[k][threadIdx.x];
            wcnt[k][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    if (live) {
        const uint32_t dst = off[(size_t)d * nb + blockIdx.x] + wcnt[w][d] + rank_w;
        kout[dst] = key;
        vout[dst] = vin[i];
    }
}

// ---------------------------------------------------------------- exclusive scan (u32)
constexpr int kScanTile = 4 * 1024;

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* sh, uint32_t* total) {
    // sh: 33 entries (warp prefixes, then the total)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < nw) sh[lane] = si - s;
        if (lane == nw - 1) sh[32] = si;
    }
    __syncthreads();
    const uint32_t r = sh[w] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ in, int n,
                                                     uint32_t* __restrict__ sums) {
    __shared__ uint32_t sh[33];
    const long long base = (long long)blockIdx.x * kScanTile + 4 * threadIdx.x;
    uint32_t s = 0;
    for (int k = 0; k < 4; ++k)
        if (base + k < n) s += in[base + k];
    uint32_t total;
    block_scan_excl(s, sh, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the tile sums in place (at most 1024 x 4 tiles, 16M elements).
__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t* sums, int nt, uint32_t* total) {
    __shared__ uint32_t sh[33];
    uint32_t v[4], s = 0;
    for (int k = 0; k < 4; ++k) {
        const int j = 4 * threadIdx.x + k;
        v[k] = j < nt ? sums[j] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_scan_excl(s, sh, &tot);
    for (int k = 0; k < 4; ++k) {
        const int j = 4 * threadIdx.x + k;
        if (j < nt) sums[j] = run;
        run += v[k];
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t* __restrict__ in, int n,
                                                     const uint32_t* __restrict__ sums,
                                                     uint32_t* __restrict__ out) {
    __shared__ uint32_t sh[33];
    const long long base = (long long)blockIdx.x * kScanTile + 4 * threadIdx.x;
    uint32_t v[4], s = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_scan_excl(s, sh, &total) + sums[blockIdx.x];
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------- PLOC
// Leaf j of the sorted order: triangle vals[j]'s box grown by `pad`.
__global__ void k_leaf_boxes(const float* __restrict__ tri, const uint32_t* __restrict__ vals,
                             int n, float pad, float4* __restrict__ blo, float4* __restrict__ bhi,
                             uint32_t* __restrict__ cnt, uint32_t* __restrict__ clusters) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float* v = tri + 9 * (size_t)vals[j];
    float3 a = make_float3(v[0], v[1], v[2]);
    float3 b = a;
    for (int k = 1; k < 3; ++k) {
        const float3 p = make_float3(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
        a = fmin3(a, p);
        b = fmax3(b, p);
    }
    blo[j] = make_float4(a.x - pad, a.y - pad, a.z - pad, 0.0f);
    bhi[j] = make_float4(b.x + pad, b.y + pad, b.z + pad, 0.0f);
    cnt[j] = 1;
    clusters[j] = (uint32_t)j;
}

// Nearest neighbour of every cluster within kRadius positions (least merged area; ties
// to the lower position).
__global__ void __launch_bounds__(kThreads) k_ploc_nn(const uint32_t* __restrict__ C, int m,
                                                      const float4* __restrict__ blo,
                                                      const float4* __restrict__ bhi,
                                                      uint32_t* __restrict__ nn) {
    __shared__ float3 slo[kThreads + 2 * kRadius], shi[kThreads + 2 * kRadius];
    const int start = blockIdx.x * kThreads - kRadius;
    for (int k = threadIdx.x; k < kThreads + 2 * kRadius; k += kThreads) {
        const int j = start + k;
        if (j >= 0 && j < m) {
            const uint32_t c = C[j];
            const float4 a = blo[c], b = bhi[c];
            slo[k] = make_float3(a.x, a.y, a.z);
            shi[k] = make_float3(b.x, b.y, b.z);
        }
    }
    __syncthreads();
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= m) return;
    const int li = threadIdx.x + kRadius;
    float best = FLT_MAX;
    int bj = -1;
    for (int o = -kRadius; o <= kRadius; ++o) {
        const int j = i + o;
        if (o == 0 || j < 0 || j >= m) continue;
        const float a = half_area(fmin3(slo[li], slo[li + o]), fmax3(shi[li], shi[li + o]));
        if (a < best) {  // o ascending: equal areas keep the lower position
            best = a;
            bj = j;
        }
    }
    nn[i] = (uint32_t)bj;
}

// merge[i]: cluster i merges with its mutual neighbour and is the lower of the two;
// keep[i]: cluster i survives (as itself or as the merged node).
__global__ void k_ploc_flags(const uint32_t* __restrict__ nn, int m, uint32_t* __restrict__ merge,
                             uint32_t* __restrict__ keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j = (int)nn[i];
    const bool mutual = j >= 0 && (int)nn[j] == i;
    merge[i] = mutual && i < j ? 1u : 0u;
    keep[i] = mutual && i > j ? 0u : 1u;
}

__global__ void k_ploc_merge(const uint32_t* __restrict__ C, const uint32_t* __restrict__ nn,
                             int m, const uint32_t* __restrict__ mpos,
                             const uint32_t* __restrict__ kpos,
                             const uint32_t* __restrict__ merge, const uint32_t* __restrict__ keep,
                             int n_leaf, int next, float4* __restrict__ blo,
                             float4* __restrict__ bhi, uint32_t* __restrict__ cnt,
                             int2* __restrict__ kids, uint32_t* __restrict__ Cout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (merge[i]) {
        const uint32_t a = C[i], b = C[nn[i]];
        const uint32_t id = (uint32_t)(n_leaf + next) + mpos[i];
        const float4 la = blo[a], ha = bhi[a], lb = blo[b], hb = bhi[b];
        blo[id] = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), 0.0f);
        bhi[id] = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.0f);
        cnt[id] = cnt[a] + cnt[b];
        kids[id - n_leaf] = make_int2((int)a, (int)b);
        Cout[kpos[i]] = id;
    } else if (keep[i]) {
        Cout[kpos[i]] = C[i];
    }
}

// ---------------------------------------------------------------- collapse to 8 wide
struct Plan {
    int child[8];   // BVH2 node ids of the children (slot order), -1 = empty
    int ntri;       // triangles of the leaf children
    int ninner;     // inner children
};

__device__ __forceinline__ float node_area(const float4* blo, const float4* bhi, int id) {
    const float4 a = blo[id], b = bhi[id];
    return half_area(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z));
}

// Children of one eight-wide node: open the child of largest area until eight children
// or none can open (leaves, and subtrees of at most kLeafTris triangles, stay whole);
// then give the children slots by the octant of their box centre around the node's.
__global__ void k_collapse_plan(const int2* __restrict__ items, int n_items, int n_leaf,
                                const int2* __restrict__ kids, const uint32_t* __restrict__ cnt,
                                const float4* __restrict__ blo, const float4* __restrict__ bhi,
                                Plan* __restrict__ plans, uint32_t* __restrict__ ninner,
                                uint32_t* __restrict__ ntri) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items) return;
    const int root = items[k].x;
    int c[8], nc = 0;
    if (root < n_leaf) {
        c[nc++] = root;  // a one-triangle scene: the root holds a single leaf
    } else {
        const int2 kk = kids[root - n_leaf];
        c[nc++] = kk.x;
        c[nc++] = kk.y;
    }
    while (nc < 8) {
        int best = -1;
        float ba = -1.0f;
        for (int j = 0; j < nc; ++j) {
            if (c[j] < n_leaf || cnt[c[j]] <= (uint32_t)kLeafTris) continue;
            const float a = node_area(blo, bhi, c[j]);
            if (a > ba) {
                ba = a;
                best = j;
            }
        }
        if (best < 0) break;
        const int2 kk = kids[c[best] - n_leaf];
        c[best] = kk.x;
        c[nc++] = kk.y;
    }
    // slots: greedy assignment of (child, slot) pairs by the largest alignment of the
    // child's centre offset with the slot's octant direction
    const float4 pl = blo[root], ph = bhi[root];
    const float mx = 0.5f * (pl.x + ph.x), my = 0.5f * (pl.y + ph.y), mz = 0.5f * (pl.z + ph.z);
    float off[8][3];
    for (int j = 0; j < nc; ++j) {
        const float4 a = blo[c[j]], b = bhi[c[j]];
        off[j][0] = 0.5f * (a.x + b.x) - mx;
        off[j][1] = 0.5f * (a.y + b.y) - my;
        off[j][2] = 0.5f * (a.z + b.z) - mz;
    }
    Plan p;
    for (int s = 0; s < 8; ++s) p.child[s] = -1;
    unsigned used_c = 0, used_s = 0;
    for (int round = 0; round < nc; ++round) {
        float bs = -FLT_MAX;
        int bc = -1, bsl = -1;
        for (int j = 0; j < nc; ++j) {
            if (used_c >> j & 1u) continue;
            for (int s = 0; s < 8; ++s) {
                if (used_s >> s & 1u) continue;
                const float sc = (s & 1 ? off[j][0] : -off[j][0]) + (s & 2 ? off[j][1] : -off[j][1]) +
                                 (s & 4 ? off[j][2] : -off[j][2]);
                if (sc > bs) {
                    bs = sc;
                    bc = j;
                    bsl = s;
                }
            }
        }
        used_c |= 1u << bc;
        used_s |= 1u << bsl;
        p.child[bsl] = c[bc];
    }
    int ni = 0, nt = 0;
    for (int s = 0; s < 8; ++s) {
        const int id = p.child[s];
        if (id < 0) continue;
        if (id < n_leaf || cnt[id] <= (uint32_t)kLeafTris) nt += (int)cnt[id];
        else ++ni;
    }
    p.ninner = ni;
    p.ntri = nt;
    plans[k] = p;
    ninner[k] = (uint32_t)ni;
    ntri[k] = (uint32_t)nt;
}

constexpr float kSteps = 252.0f;  // quantisation steps spanning a node's box

// Smallest e with 252 * 2^e >= ext, as a biased exponent in [1, 254].
__device__ __forceinline__ int scale_exponent(float ext) {
    if (!(ext > 0.0f)) return 1;
    int e = (int)ceilf(log2f(ext * (1.0f / kSteps)));
    while (ldexpf(kSteps, e) < ext) ++e;
    while (e > -126 && ldexpf(kSteps, e - 1) >= ext) --e;
    e += 127;
    return e < 1 ? 1 : (e > 254 ? 254 : e);
}

__global__ void k_collapse_emit(const int2* __restrict__ items, int n_items, int n_leaf,
                                const int2* __restrict__ kids, const uint32_t* __restrict__ cnt,
                                const float4* __restrict__ blo, const float4* __restrict__ bhi,
                                const Plan* __restrict__ plans, const uint32_t* __restrict__ cbase,
                                const uint32_t* __restrict__ tbase, uint32_t node_base,
                                uint32_t tri_base, const uint32_t* __restrict__ vals,
                                const float* __restrict__ tri, const int32_t* __restrict__ mat,
                                uint4* __restrict__ nodes, float4* __restrict__ tris,
                                int2* __restrict__ next_items) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items) return;
    const int self = items[k].y;
    const Plan p = plans[k];
    const uint32_t first_child = node_base + cbase[k];
    const uint32_t first_tri = tri_base + tbase[k];
    // node box = union of the children's boxes; origin and scales
    float3 lo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX), hi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
    for (int s = 0; s < 8; ++s) {
        const int id = p.child[s];
        if (id < 0) continue;
        const float4 a = blo[id], b = bhi[id];
        lo = fmin3(lo, make_float3(a.x, a.y, a.z));
        hi = fmax3(hi, make_float3(b.x, b.y, b.z));
    }
    const int ex = scale_exponent(hi.x - lo.x), ey = scale_exponent(hi.y - lo.y),
              ez = scale_exponent(hi.z - lo.z);
    const float sx = ldexpf(1.0f, ex - 127), sy = ldexpf(1.0f, ey - 127), sz = ldexpf(1.0f, ez - 127);
    // the origin two steps below the box (rounded down: it only moves further below)
    const float3 org = make_float3(__fsub_rd(lo.x, 2.0f * sx), __fsub_rd(lo.y, 2.0f * sy),
                                   __fsub_rd(lo.z, 2.0f * sz));
    uint8_t q[6][8], meta[8];
    uint32_t imask = 0;
    int inner = 0, toff = 0;
    for (int s = 0; s < 8; ++s) {
        const int id = p.child[s];
        meta[s] = 0;
        if (id < 0) {
            q[0][s] = q[1][s] = q[2][s] = 255;
            q[3][s] = q[4][s] = q[5][s] = 0;
            continue;
        }
        const float4 a = blo[id], b = bhi[id];
        // outward: floor of the lower offsets minus one step, ceiling of the upper ones
        // plus one (offsets rounded down / up from the origin, so the step only widens);
        // the lower byte is >= 1 and the upper <= 255 by the choice of origin and scale
        auto qlo = [](float v, float o, float sc) {
            return (uint8_t)fminf(fmaxf(floorf(__fsub_rd(v, o) / sc) - 1.0f, 0.0f), 255.0f);
        };
        auto qhi = [](float v, float o, float sc) {
            return (uint8_t)fminf(fmaxf(ceilf(__fsub_ru(v, o) / sc) + 1.0f, 0.0f), 255.0f);
        };
        q[0][s] = qlo(a.x, org.x, sx);
        q[1][s] = qlo(a.y, org.y, sy);
        q[2][s] = qlo(a.z, org.z, sz);
        q[3][s] = qhi(b.x, org.x, sx);
        q[4][s] = qhi(b.y, org.y, sy);
        q[5][s] = qhi(b.z, org.z, sz);
        if (id >= n_leaf && cnt[id] > (uint32_t)kLeafTris) {
            imask |= 1u << s;
            next_items[cbase[k] + inner] = make_int2(id, (int)(first_child + inner));
            ++inner;
        } else {
            // the leaf's triangles: the BVH2 leaves of the subtree, left to right
            int stack[2 * kLeafTris], sp = 0, nt = 0;
            stack[sp++] = id;
            while (sp > 0) {
                const int v = stack[--sp];
                if (v < n_leaf) {
                    const uint32_t t = vals[v];
                    const float* w = tri + 9 * (size_t)t;
                    float4* o = tris + 3 * (size_t)(first_tri + toff + nt);
                    const float v0x = w[0], v0y = w[1], v0z = w[2];
                    o[0] = make_float4(v0x, v0y, v0z, __uint_as_float(t));
                    o[1] = make_float4(w[3] - v0x, w[4] - v0y, w[5] - v0z,
                                       __int_as_float(mat[t]));
                    o[2] = make_float4(w[6] - v0x, w[7] - v0y, w[8] - v0z, 0.0f);
                    ++nt;
                } else {
                    const int2 kk = kids[v - n_leaf];
                    stack[sp++] = kk.y;  // left child on top: popped first
                    stack[sp++] = kk.x;
                }
            }
            meta[s] = (uint8_t)((nt << 5) | toff);
            toff += nt;
        }
    }
    auto pack4 = [](const uint8_t* b) {
        return (uint32_t)b[0] | (uint32_t)b[1] << 8 | (uint32_t)b[2] << 16 | (uint32_t)b[3] << 24;
    };
    uint4* N = nodes + 5 * (size_t)self;
    N[0] = make_uint4(__float_as_uint(org.x), __float_as_uint(org.y), __float_as_uint(org.z),
                      (uint32_t)ex | (uint32_t)ey << 8 | (uint32_t)ez << 16 | imask << 24);
    N[1] = make_uint4(first_child, first_tri, pack4(meta), pack4(meta + 4));
    N[2] = make_uint4(pack4(q[0]), pack4(q[0] + 4), pack4(q[1]), pack4(q[1] + 4));
    N[3] = make_uint4(pack4(q[2]), pack4(q[2] + 4), pack4(q[3]), pack4(q[3] + 4));
    N[4] = make_uint4(pack4(q[4]), pack4(q[4] + 4), pack4(q[5]), pack4(q[5] + 4));
}

struct DevBuf {
    std::vector<void*> ptrs;
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * (n > 0 ? n : 1));
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return e;
    }
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
};

// Exclusive scan of in[n] into out[n]; total (device, nullable) receives the sum.
cudaError_t scan_u32(const uint32_t* in, int n, uint32_t* out, uint32_t* sums, uint32_t* total,
                     cudaStream_t s) {
    const int nt = (n + kScanTile - 1) / kScanTile;
    if (nt > 4 * 1024) return cudaErrorInvalidValue;
    if (n > 0) k_scan_tiles<<<nt, 1024, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, n > 0 ? nt : 0, total);
    if (n > 0) k_scan_apply<<<nt, 1024, 0, s>>>(in, n, sums, out);
    return cudaGetLastError();
}

// The clustered BVH2 of the build's first two steps (device arrays owned by `tmp`).
struct PlocTree {
    uint32_t* vals = nullptr;  // triangle of each leaf (sorted order)
    float4 *blo = nullptr, *bhi = nullptr;  // node boxes: leaves 0..n-1, merges n..2n-2
    uint32_t* cnt = nullptr;   // triangles under each node
    int2* kids = nullptr;      // children of merge node n + k at k
    uint32_t* sums = nullptr;  // scan scratch
    uint32_t* total = nullptr;
    uint32_t root = 0;
    int iters = 0;
};

cudaError_t ploc_build(const float* d_tri, int n, const float lo[3], const float hi[3],
                       cudaStream_t s, DevBuf& tmp, PlocTree* t) {
    cudaError_t e;
#define BK(x)                      \
    do {                           \
        e = (x);                   \
        if (e != cudaSuccess) return e; \
    } while (0)
    uint32_t *keys, *vals, *keys2, *vals2, *hist, *off, *sums, *total;
    const int nb = (n + kThreads - 1) / kThreads;
    BK(tmp.alloc(&keys, n));
    BK(tmp.alloc(&vals, n));
    BK(tmp.alloc(&keys2, n));
    BK(tmp.alloc(&vals2, n));
    BK(tmp.alloc(&hist, (size_t)256 * nb));
    BK(tmp.alloc(&off, (size_t)256 * nb));
    BK(tmp.alloc(&sums, 4 * 1024));
    BK(tmp.alloc(&total, 4));
    float ext = 0.0f, mag = 0.0f;
    float3 slo = make_float3(lo[0], lo[1], lo[2]), sc;
    float e3[3];
    for (int k = 0; k < 3; ++k) {
        e3[k] = hi[k] - lo[k];
        ext = fmaxf(ext, e3[k]);
        mag = fmaxf(mag, fmaxf(fabsf(lo[k]), fabsf(hi[k])));
    }
    sc = make_float3(e3[0] > 0 ? 1023.0f / e3[0] : 0.0f, e3[1] > 0 ? 1023.0f / e3[1] : 0.0f,
                     e3[2] > 0 ? 1023.0f / e3[2] : 0.0f);
    k_prim_codes<<<nb, kThreads, 0, s>>>(d_tri, n, slo, sc, keys, vals);
    for (int shift = 0; shift < 30; shift += 8) {
        k_rs_hist<<<nb, kThreads, 0, s>>>(keys, n, shift, nb, hist);
        BK(scan_u32(hist, 256 * nb, off, sums, nullptr, s));
        k_rs_scatter<<<nb, kThreads, 0, s>>>(keys, vals, keys2, vals2, n, shift, nb, off);
        std::swap(keys, keys2);
        std::swap(vals, vals2);
    }
    BK(cudaGetLastError());
    // PLOC: nodes 0 .. n-1 are the leaves (sorted order), n .. 2n-2 the merges
    float4 *blo, *bhi;
    uint32_t *cnt, *C, *C2, *nn, *merge, *keep, *mpos, *kpos;
    int2* kids;
    BK(tmp.alloc(&blo, 2 * (size_t)n));
    BK(tmp.alloc(&bhi, 2 * (size_t)n));
    BK(tmp.alloc(&cnt, 2 * (size_t)n));
    BK(tmp.alloc(&kids, n));
    BK(tmp.alloc(&C, n));
    BK(tmp.alloc(&C2, n));
    BK(tmp.alloc(&nn, n));
    BK(tmp.alloc(&merge, n));
    BK(tmp.alloc(&keep, n));
    BK(tmp.alloc(&mpos, n));
    BK(tmp.alloc(&kpos, n));
    // margin as the BVH2's: 1e-5 of the scene size and 4 ulp of the largest coordinate
    const float pad = 1e-5f * ext + 4.0f * 0x1p-23f * mag + 1e-30f;
    k_leaf_boxes<<<nb, kThreads, 0, s>>>(d_tri, vals, n, pad, blo, bhi, cnt, C);
    int m = n, next = 0, iters = 0;
    while (m > 1) {
        const int g = (m + kThreads - 1) / kThreads;
        k_ploc_nn<<<g, kThreads, 0, s>>>(C, m, blo, bhi, nn);
        k_ploc_flags<<<g, kThreads, 0, s>>>(nn, m, merge, keep);
        BK(scan_u32(merge, m, mpos, sums, total, s));
        BK(scan_u32(keep, m, kpos, sums, total + 1, s));
        k_ploc_merge<<<g, kThreads, 0, s>>>(C, nn, m, mpos, kpos, merge, keep, n, next, blo, bhi,
                                            cnt, kids, C2);
        uint32_t h[2];
        BK(cudaMemcpyAsync(h, total, 8, cudaMemcpyDeviceToHost, s));
        BK(cudaStreamSynchronize(s));
        if (h[0] == 0 || ++iters > 100000) return cudaErrorUnknown;  // no progress
        next += (int)h[0];
        m = (int)h[1];
        std::swap(C, C2);
    }
    BK(cudaMemcpyAsync(&t->root, C, 4, cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    t->vals = vals;
    t->blo = blo;
    t->bhi = bhi;
    t->cnt = cnt;
    t->kids = kids;
    t->sums = sums;
    t->total = total;
    t->iters = iters;
    return cudaSuccess;
#undef BK
}

}  // namespace

cudaError_t build_bvh8(const float* d_tri, const int32_t* d_mat, int n, const float lo[3],
                       const float hi[3], cudaStream_t s, Bvh8Device* out) {
    if (n < 1 || n >= (1 << 24)) return cudaErrorInvalidValue;
    DevBuf tmp;
    PlocTree t;
    cudaError_t e = ploc_build(d_tri, n, lo, hi, s, tmp, &t);
    if (e != cudaSuccess) return e;
    uint32_t* vals = t.vals;
    float4 *blo = t.blo, *bhi = t.bhi;
    uint32_t* cnt = t.cnt;
    int2* kids = t.kids;
    uint32_t *sums = t.sums, *total = t.total;
    const uint32_t root_id = t.root;
    const int iters = t.iters;
#define BK(x)                      \
    do {                           \
        e = (x);                   \
        if (e != cudaSuccess) return e; \
    } while (0)
    // collapse, one level per round
    const size_t max_nodes = (size_t)n;  // every eight-wide node has >= 2 children
    uint4* nodes;
    float4* tris;
    BK(cudaMalloc(&nodes, sizeof(uint4) * 5 * max_nodes));
    e = cudaMalloc(&tris, sizeof(float4) * 3 * (size_t)n);
    if (e != cudaSuccess) {
        cudaFree(nodes);
        return e;
    }
    auto fail_out = [&](cudaError_t err) {
        cudaFree(nodes);
        cudaFree(tris);
        return err;
    };
    int2 *items, *items2;
    Plan* plans;
    uint32_t *ninner, *ntri, *cb, *tb;
    if ((e = tmp.alloc(&items, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&items2, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&plans, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&ninner, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&ntri, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&cb, n)) != cudaSuccess) return fail_out(e);
    if ((e = tmp.alloc(&tb, n)) != cudaSuccess) return fail_out(e);
    const int2 root_item = make_int2((int)root_id, 0);
    if ((e = cudaMemcpyAsync(items, &root_item, sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail_out(e);
    int n_items = 1, depth = 0;
    uint32_t node_count = 1, tri_count = 0;
    while (n_items > 0) {
        const int g = (n_items + kThreads - 1) / kThreads;
        k_collapse_plan<<<g, kThreads, 0, s>>>(items, n_items, n, kids, cnt, blo, bhi, plans,
                                               ninner, ntri);
        if ((e = scan_u32(ninner, n_items, cb, sums, total, s)) != cudaSuccess) return fail_out(e);
        if ((e = scan_u32(ntri, n_items, tb, sums, total + 1, s)) != cudaSuccess) return fail_out(e);
        k_collapse_emit<<<g, kThreads, 0, s>>>(items, n_items, n, kids, cnt, blo, bhi, plans, cb, tb,
                                               node_count, tri_count, vals, d_tri, d_mat, nodes,
                                               tris, items2);
        uint32_t h[2];
        if ((e = cudaMemcpyAsync(h, total, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return fail_out(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_out(e);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail_out(e);
        node_count += h[0];
        tri_count += h[1];
        n_items = (int)h[0];
        std::swap(items, items2);
        ++depth;
        if (node_count > max_nodes) return fail_out(cudaErrorUnknown);
    }
    if (tri_count != (uint32_t)n) return fail_out(cudaErrorUnknown);
    out->nodes = nodes;
    out->tris = tris;
    out->n_nodes = node_count;
    out->depth = depth;
    out->ploc_iterations = iters;
    return cudaSuccess;
#undef BK
}

cudaError_t build_bvh2_ploc(const float* d_tri, const float* h_tri, const int32_t* h_mat, int n,
                            const float lo[3], const float hi[3], int max_depth, cudaStream_t s,
                            BvhHost* out, int* depth_out) {
    if (n < 2 || n >= (1 << 24)) return cudaErrorInvalidValue;
    DevBuf tmp;
    PlocTree t;
    cudaError_t e = ploc_build(d_tri, n, lo, hi, s, tmp, &t);
    if (e != cudaSuccess) return e;
    std::vector<int2> kids((size_t)n - 1);
    std::vector<float4> blo(2 * (size_t)n), bhi(2 * (size_t)n);
    std::vector<uint32_t> vals((size_t)n);
    if ((e = cudaMemcpy(kids.data(), t.kids, sizeof(int2) * (n - 1), cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(blo.data(), t.blo, sizeof(float4) * 2 * (size_t)n, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(bhi.data(), t.bhi, sizeof(float4) * 2 * (size_t)n, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(vals.data(), t.vals, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost)))
        return e;
    // depth-first preorder: inner nodes numbered as the BVH2 builder numbers them (self
    // before its subtrees, left first), leaves in the order they are met
    std::vector<int32_t> idx(2 * (size_t)n, -1);
    std::vector<int32_t> leaf_order;
    leaf_order.reserve(n);
    std::vector<std::pair<uint32_t, int>> stack;
    stack.emplace_back(t.root, 0);
    int32_t inner = 0, deepest = 0;
    while (!stack.empty()) {
        const auto [id, d] = stack.back();
        stack.pop_back();
        if (id < (uint32_t)n) {
            idx[id] = (int32_t)leaf_order.size();
            leaf_order.push_back((int32_t)id);
            continue;
        }
        idx[id] = inner++;
        deepest = std::max(deepest, d);
        const int2 k = kids[id - n];
        stack.emplace_back((uint32_t)k.y, d + 1);
        stack.emplace_back((uint32_t)k.x, d + 1);
    }
    if (depth_out) *depth_out = deepest;
    if (deepest > max_depth) return cudaErrorNotSupported;
    out->nodes.assign((size_t)inner, BvhNode{});
    for (uint32_t id = (uint32_t)n; id < 2u * (uint32_t)n - 1u; ++id) {
        if (idx[id] < 0) continue;
        const int2 k = kids[id - n];
        BvhNode& nd = out->nodes[(size_t)idx[id]];
        const uint32_t c[2] = {(uint32_t)k.x, (uint32_t)k.y};
        for (int j = 0; j < 2; ++j) {
            const float4 a = blo[c[j]], b = bhi[c[j]];
            float* xy = j == 0 ? nd.a : nd.b;
            xy[0] = a.x; xy[1] = b.x; xy[2] = a.y; xy[3] = b.y;
            nd.c[2 * j] = a.z;
            nd.c[2 * j + 1] = b.z;
            nd.d[j] = c[j] < (uint32_t)n ? ~idx[c[j]] : idx[c[j]];
            nd.d[2 + j] = c[j] < (uint32_t)n ? 1 : 0;
        }
    }
    out->n_ref = n;
    out->tris.assign((size_t)n * 12, 0.0f);
    for (int32_t sidx = 0; sidx < n; ++sidx) {
        const int32_t i = (int32_t)vals[leaf_order[sidx]];
        const float* v = h_tri + (size_t)i * 9;
        float* o = out->tris.data() + (size_t)sidx * 12;
        for (int k = 0; k < 3; ++k) {
            o[k] = v[k];
            o[4 + k] = v[3 + k] - v[k];  // correctly rounded FP32 differences
            o[8 + k] = v[6 + k] - v[k];
        }
        std::memcpy(&o[3], &i, 4);
        std::memcpy(&o[7], &h_mat[i], 4);
    }
    for (int k = 0; k < 3; ++k) {
        out->lo[k] = lo[k];
        out->hi[k] = hi[k];
    }
    return cudaSuccess;
}

}  // namespace nrrs
