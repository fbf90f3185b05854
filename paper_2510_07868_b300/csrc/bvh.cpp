// Host-side BVH2 build (binned SAH) and the device layouts it produces.
//
// Node (64 bytes, 4 x float4), both children's boxes stored in the parent so one fetch
// decides which children to visit:
//   a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   c = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   d = (child0, child1, count0, count1)   child >= 0: inner node index;
//                                          child <  0: leaf, first triangle ~child.
// A copy with half-precision boxes rounded outward (32 bytes per node, bvh.h) is what
// the traversal reads by default.
// Triangles (48 bytes, 3 x float4, in BVH leaf order):
//   (v0.xyz, original index), (e1 = v1 - v0, material id), (e2 = v2 - v0, 0)
//
// Large triangles enter the build as several references ("early split clipping",
// Ernst & Greiner 2007): a triangle whose box is long compared with the scene is cut
// into sub-boxes, each bounding the part of the triangle inside it, so walls do not
// make every node span the whole scene.  A reference carries the full triangle, so the
// intersection test and its result do not change; duplicates return the same hit.
#include "bvh.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

namespace nrrs {

namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const float* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    bool empty() const { return lo[0] > hi[0]; }
    double area() const {
        if (empty()) return 0.0;
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Prim {
    Box box;
    float c[3];
    int32_t id;
};

constexpr int kBins = 16;
constexpr int kSplitLevels = 10;       // at most 2^10 references per triangle
constexpr double kSplitFraction = 1.0 / 16.0;  // split boxes longer than this x scene size

// Bounds of the part of triangle v[3][3] inside box `clip` (Sutherland-Hodgman in FP64,
// rounded outward to float).  Returns an empty box if they do not overlap.
Box clipped_bounds(const double v[3][3], const double lo[3], const double hi[3]) {
    double poly[16][3], tmp[16][3];
    int n = 3;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) poly[i][k] = v[i][k];
    for (int ax = 0; ax < 3 && n > 0; ++ax) {
        for (int side = 0; side < 2 && n > 0; ++side) {
            const double plane = side ? hi[ax] : lo[ax];
            auto inside = [&](const double* p) { return side ? p[ax] <= plane : p[ax] >= plane; };
            int m = 0;
            for (int i = 0; i < n; ++i) {
                const double* a = poly[i];
                const double* b = poly[(i + 1) % n];
                const bool ia = inside(a), ib = inside(b);
                if (ia && m < 16) {
                    for (int k = 0; k < 3; ++k) tmp[m][k] = a[k];
                    ++m;
                }
                if (ia != ib && m < 16) {
                    const double t = (plane - a[ax]) / (b[ax] - a[ax]);
                    for (int k = 0; k < 3; ++k) tmp[m][k] = a[k] + t * (b[k] - a[k]);
                    tmp[m][ax] = plane;
                    ++m;
                }
            }
            n = m;
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < 3; ++k) poly[i][k] = tmp[i][k];
        }
    }
    Box out;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            out.lo[k] = std::min(out.lo[k], std::nextafter((float)poly[i][k], -FLT_MAX));
            out.hi[k] = std::max(out.hi[k], std::nextafter((float)poly[i][k], FLT_MAX));
        }
    return out;
}

void add_references(const double v[3][3], const Box& b, int32_t id, int level, double limit,
                    std::vector<Prim>& out) {
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (b.hi[k] - b.lo[k] > b.hi[ax] - b.lo[ax]) ax = k;
    if ((double)b.hi[ax] - b.lo[ax] <= limit || level >= kSplitLevels) {
        Prim p;
        p.box = b;
        for (int k = 0; k < 3; ++k) p.c[k] = 0.5f * (b.lo[k] + b.hi[k]);
        p.id = id;
        out.push_back(p);
        return;
    }
    const double mid = 0.5 * ((double)b.lo[ax] + b.hi[ax]);
    for (int half = 0; half < 2; ++half) {
        double lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            lo[k] = b.lo[k];
            hi[k] = b.hi[k];
        }
        if (half) lo[ax] = mid; else hi[ax] = mid;
        Box c = clipped_bounds(v, lo, hi);
        if (c.empty()) continue;
        // never grow past the parent box
        for (int k = 0; k < 3; ++k) {
            c.lo[k] = std::max(c.lo[k], b.lo[k]);
            c.hi[k] = std::min(c.hi[k], b.hi[k]);
        }
        add_references(v, c, id, level + 1, limit, out);
    }
}
constexpr int kLeafMax = 1;  // single-triangle leaves: no divergent multi-triangle loops
constexpr int kMaxBuildDepth = 38;  // traversal stack holds 40 entries

struct Builder {
    std::vector<Prim>& prims;
    std::vector<BvhNode>& nodes;
    float pad;  // boxes grow by this much so FP32 slab tests never cut off a hit

    // Returns the child encoding for prims[begin, end) and its bounds.
    int32_t build(int32_t begin, int32_t end, int depth, Box* out_box, int32_t* out_count) {
        Box b, cb;
        for (int32_t i = begin; i < end; ++i) {
            b.grow(prims[i].box);
            cb.grow(prims[i].c);
        }
        *out_box = b;
        const int32_t n = end - begin;
        if (n <= kLeafMax || depth >= kMaxBuildDepth) {
            *out_count = n;
            return ~begin;
        }
        // binned SAH over centroid bounds
        int best_axis = -1, best_split = -1;
        double best_cost = DBL_MAX;
        for (int ax = 0; ax < 3; ++ax) {
            const float ext = cb.hi[ax] - cb.lo[ax];
            if (!(ext > 0.0f)) continue;
            Box bb[kBins];
            int cnt[kBins] = {0};
            const float scale = kBins / ext;
            for (int32_t i = begin; i < end; ++i) {
                int k = std::min(kBins - 1, (int)((prims[i].c[ax] - cb.lo[ax]) * scale));
                cnt[k]++;
                bb[k].grow(prims[i].box);
            }
            double rA[kBins];
            int rN[kBins];
            Box acc;
            int na = 0;
            for (int k = kBins - 1; k > 0; --k) {
                acc.grow(bb[k]);
                na += cnt[k];
                rA[k] = acc.area();
                rN[k] = na;
            }
            Box lacc;
            int nl = 0;
            for (int k = 0; k < kBins - 1; ++k) {
                lacc.grow(bb[k]);
                nl += cnt[k];
                if (nl == 0 || rN[k + 1] == 0) continue;
                double cost = lacc.area() * nl + rA[k + 1] * rN[k + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = ax;
                    best_split = k;
                }
            }
        }
        int32_t mid;
        if (best_axis < 0) {
            mid = begin + n / 2;  // coincident centroids: split by count
        } else {
            const float ext = cb.hi[best_axis] - cb.lo[best_axis];
            const float scale = kBins / ext;
            auto it = std::partition(prims.begin() + begin, prims.begin() + end, [&](const Prim& p) {
                int k = std::min(kBins - 1, (int)((p.c[best_axis] - cb.lo[best_axis]) * scale));
                return k <= best_split;
            });
            mid = (int32_t)(it - prims.begin());
            if (mid == begin || mid == end) mid = begin + n / 2;
        }
        const int32_t self = (int32_t)nodes.size();
        nodes.emplace_back();
        Box lb, rb;
        int32_t lc = 0, rc = 0;
        int32_t l = build(begin, mid, depth + 1, &lb, &lc);
        int32_t r = build(mid, end, depth + 1, &rb, &rc);
        fill(nodes[self], inflate(lb), l, lc, inflate(rb), r, rc);
        *out_count = 0;
        return self;
    }

    Box inflate(Box b) const {
        if (b.empty()) return b;
        for (int k = 0; k < 3; ++k) {
            b.lo[k] -= pad;
            b.hi[k] += pad;
        }
        return b;
    }

    static void fill(BvhNode& nd, const Box& l, int32_t lc, int32_t ln, const Box& r, int32_t rcode,
                     int32_t rn) {
        nd.a[0] = l.lo[0]; nd.a[1] = l.hi[0]; nd.a[2] = l.lo[1]; nd.a[3] = l.hi[1];
        nd.b[0] = r.lo[0]; nd.b[1] = r.hi[0]; nd.b[2] = r.lo[1]; nd.b[3] = r.hi[1];
        nd.c[0] = l.lo[2]; nd.c[1] = l.hi[2]; nd.c[2] = r.lo[2]; nd.c[3] = r.hi[2];
        nd.d[0] = lc; nd.d[1] = rcode; nd.d[2] = ln; nd.d[3] = rn;
    }
};

}  // namespace

int bvh2_height(const std::vector<BvhNode>& nodes) {
    const size_t n = nodes.size();
    std::vector<int> h(n, 1);
    int best = 0;
    for (size_t k = n; k-- > 0;) {  // children before their parents
        for (int c = 0; c < 2; ++c) {
            const int32_t ch = nodes[k].d[c];
            if (ch < 0) continue;  // a leaf
            if ((size_t)ch <= k || (size_t)ch >= n) return -1;
            h[k] = std::max(h[k], 1 + h[ch]);
        }
        best = std::max(best, h[k]);
    }
    return best;
}

void build_bvh(const float* tri, int32_t n_tri, const int32_t* mat_id, BvhHost* out) {
    Box scene_box;
    for (int64_t i = 0; i < (int64_t)n_tri * 3; ++i) scene_box.grow(tri + i * 3);
    double scene_ext = 0.0;
    for (int k = 0; k < 3; ++k) scene_ext = std::max(scene_ext, (double)scene_box.hi[k] - scene_box.lo[k]);
    const double limit = kSplitFraction * scene_ext;
    std::vector<Prim> prims;
    prims.reserve((size_t)n_tri + 1024);
    for (int32_t i = 0; i < n_tri; ++i) {
        Box b;
        double v[3][3];
        for (int k = 0; k < 3; ++k) {
            b.grow(tri + (size_t)i * 9 + 3 * k);
            for (int a = 0; a < 3; ++a) v[k][a] = tri[(size_t)i * 9 + 3 * k + a];
        }
        add_references(v, b, i, 0, limit, prims);
    }
    const int32_t n_ref = (int32_t)prims.size();
    out->nodes.clear();
    Box all;
    for (const Prim& p : prims) all.grow(p.box);
    float ext = 0.0f, mag = 0.0f;
    for (int k = 0; k < 3; ++k) {
        ext = std::max(ext, all.hi[k] - all.lo[k]);
        mag = std::max(mag, std::max(std::fabs(all.lo[k]), std::fabs(all.hi[k])));
    }
    // the margin covers the slab test's rounding: 1e-5 of the scene's size, and at least
    // 4 ulp of the largest coordinate (the products o * (1/d) round relative to |o|)
    Builder bld{prims, out->nodes, 1e-5f * ext + 4.0f * 0x1p-23f * mag + 1e-30f};
    Box root_box;
    int32_t root_count = 0;
    int32_t root = bld.build(0, n_ref, 0, &root_box, &root_count);
    if (root < 0) {
        // whole scene is one leaf: make a root whose second child is empty
        out->nodes.emplace_back();
        Box empty;
        Builder::fill(out->nodes[0], bld.inflate(root_box), root, root_count, empty, ~0, 0);
    }
    out->n_ref = n_ref;
    out->tris.assign((size_t)n_ref * 12, 0.0f);
    for (int32_t s = 0; s < n_ref; ++s) {
        const int32_t i = prims[s].id;
        const float* v = tri + (size_t)i * 9;
        float* o = out->tris.data() + (size_t)s * 12;
        for (int k = 0; k < 3; ++k) {
            o[k] = v[k];
            o[4 + k] = v[3 + k] - v[k];  // correctly rounded FP32 difference
            o[8 + k] = v[6 + k] - v[k];
        }
        std::memcpy(&o[3], &i, 4);
        std::memcpy(&o[7], &mat_id[i], 4);
    }
    for (int k = 0; k < 3; ++k) {
        out->lo[k] = FLT_MAX;
        out->hi[k] = -FLT_MAX;
    }
    for (int64_t i = 0; i < (int64_t)n_tri * 3; ++i)
        for (int k = 0; k < 3; ++k) {
            out->lo[k] = std::min(out->lo[k], tri[i * 3 + k]);
            out->hi[k] = std::max(out->hi[k], tri[i * 3 + k]);
        }
}

namespace {

struct Entry {
    float lo[3], hi[3];
    int32_t code, count;
    double area() const {
        const double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1],
                     dz = (double)hi[2] - lo[2];
        return dx < 0.0 ? 0.0 : 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

Entry child_entry(const BvhNode& n, int side) {
    Entry e;
    const float* xy = side ? n.b : n.a;
    e.lo[0] = xy[0]; e.hi[0] = xy[1]; e.lo[1] = xy[2]; e.hi[1] = xy[3];
    e.lo[2] = n.c[2 * side]; e.hi[2] = n.c[2 * side + 1];
    e.code = n.d[side];
    e.count = n.d[2 + side];
    return e;
}

struct Collapser {
    const std::vector<BvhNode>& in;
    std::vector<Bvh4Node>& out;

    // Builds the four-wide node for BVH2 node n2: its two children, then repeatedly the
    // inner child of largest surface area replaced by its own two children, up to four.
    // Returns the node index and, in *stack, the most stack entries below it.
    int32_t build(int32_t n2, int* stack) {
        Entry e[4];
        int m = 2;
        e[0] = child_entry(in[n2], 0);
        e[1] = child_entry(in[n2], 1);
        while (m < 4) {
            int pick = -1;
            double best = -1.0;
            for (int k = 0; k < m; ++k)
                if (e[k].code >= 0 && e[k].area() > best) {
                    best = e[k].area();
                    pick = k;
                }
            if (pick < 0) break;
            const BvhNode& nd = in[e[pick].code];
            e[pick] = child_entry(nd, 0);
            e[m++] = child_entry(nd, 1);
        }
        const int32_t self = (int32_t)out.size();
        out.emplace_back();
        int inner = 0, below = 0;
        int32_t code[4], count[4];
        for (int k = 0; k < 4; ++k) {
            if (k < m && e[k].code >= 0) {
                int st = 0;
                code[k] = build(e[k].code, &st);
                count[k] = 0;
                below = std::max(below, st);
                ++inner;
            } else if (k < m) {
                code[k] = e[k].code;
                count[k] = e[k].count;
            } else {
                code[k] = ~0;
                count[k] = 0;
            }
        }
        Bvh4Node& o = out[self];
        for (int k = 0; k < 4; ++k) {
            const bool used = k < m;
            o.lox[k] = used ? e[k].lo[0] : 0.0f; o.hix[k] = used ? e[k].hi[0] : 0.0f;
            o.loy[k] = used ? e[k].lo[1] : 0.0f; o.hiy[k] = used ? e[k].hi[1] : 0.0f;
            o.loz[k] = used ? e[k].lo[2] : 0.0f; o.hiz[k] = used ? e[k].hi[2] : 0.0f;
            o.child[k] = code[k];
            o.count[k] = count[k];
        }
        // a visit pushes every inner child it enters but the nearest
        *stack = std::max(0, inner - 1) + below;
        return self;
    }
};

}  // namespace

// From the binary16 format: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits;
// normal values 2^e (1 + f / 1024) for e in [-14, 15], subnormals f 2^-24.  Every
// finite FP32 value is exact in FP64, so the magnitude's position between two
// neighbouring binary16 values is computed exactly and rounded by floor or ceil.
uint16_t half_directed(float x, bool up) {
    if (std::isnan(x)) return 0x7E00;
    const uint16_t sgn = std::signbit(x) ? 0x8000 : 0;
    const double a = std::fabs((double)x);
    if (a == 0.0) return sgn;
    const bool away = (sgn == 0) == up;  // the magnitude rounds away from zero
    if (a > 65504.0) return (uint16_t)(sgn | (away ? 0x7C00 : 0x7BFF));  // inf, or the largest
    int E;
    std::frexp(a, &E);                       // a = m 2^E, m in [0.5, 1)
    const int e = std::max(E - 1, -14);      // binary exponent, subnormals at -14
    const double steps = a / std::ldexp(1.0, e - 10);  // a in units of the spacing there
    const uint32_t k = (uint32_t)(away ? std::ceil(steps) : std::floor(steps));
    if (e == -14 && k < 1024u) return (uint16_t)(sgn | k);  // subnormal (k = 1024: 2^-14)
    // k in [1024, 2048]; 2048 carries into the next exponent
    const int ee = k == 2048u ? e + 1 : e;
    const uint32_t frac = k == 2048u ? 0u : k - 1024u;
    if (ee > 15) return (uint16_t)(sgn | 0x7C00);
    return (uint16_t)(sgn | ((uint32_t)(ee + 15) << 10) | frac);
}

bool pack_half_nodes(const BvhHost& b2, std::vector<BvhNodeH>* out) {
    out->assign(b2.nodes.size(), BvhNodeH{});
    for (size_t i = 0; i < b2.nodes.size(); ++i) {
        const BvhNode& n = b2.nodes[i];
        // (lo, hi) per axis: child 0 then child 1
        const float lohi[12] = {n.a[0], n.a[1], n.a[2], n.a[3], n.c[0], n.c[1],
                                n.b[0], n.b[1], n.b[2], n.b[3], n.c[2], n.c[3]};
        BvhNodeH& o = (*out)[i];
        for (int k = 0; k < 6; ++k)
            o.box[k] = (uint32_t)half_directed(lohi[2 * k], false) |
                       ((uint32_t)half_directed(lohi[2 * k + 1], true) << 16);
        for (int c = 0; c < 2; ++c) {
            const int32_t code = n.d[c];
            if (code >= 0) {
                o.child[c] = code;
                continue;
            }
            const uint32_t first = ~(uint32_t)code, count = (uint32_t)n.d[2 + c];
            if (first > kLeafFirstMask || count >= 32u) {
                out->clear();
                return false;
            }
            o.child[c] = (int32_t)~(first | (count << kLeafFirstBits));
        }
    }
    return true;
}

namespace {

double half_value(uint32_t bits16) {
    const uint32_t e = (bits16 >> 10) & 31u, f = bits16 & 1023u;
    const double mag = e == 31u ? HUGE_VAL : e == 0u ? std::ldexp((double)f, -24)
                                                      : std::ldexp(1024.0 + f, (int)e - 25);
    return (bits16 & 0x8000u) ? -mag : mag;
}

double box_area(const double* lo, const double* hi) {
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

}  // namespace

double half_node_growth(const BvhHost& b2, const std::vector<BvhNodeH>& h) {
    double sum = 0.0, qsum = 0.0;
    for (size_t i = 0; i < b2.nodes.size() && i < h.size(); ++i) {
        const BvhNode& nd = b2.nodes[i];
        const float lohi[12] = {nd.a[0], nd.a[1], nd.a[2], nd.a[3], nd.c[0], nd.c[1],
                                nd.b[0], nd.b[1], nd.b[2], nd.b[3], nd.c[2], nd.c[3]};
        for (int c = 0; c < 2; ++c) {
            if (nd.d[c] < 0 && nd.d[2 + c] == 0) continue;  // the empty child of a one-leaf root
            double lo[3], hi[3], qlo[3], qhi[3];
            for (int k = 0; k < 3; ++k) {
                lo[k] = lohi[6 * c + 2 * k];
                hi[k] = lohi[6 * c + 2 * k + 1];
                qlo[k] = half_value(h[i].box[3 * c + k] & 0xFFFFu);
                qhi[k] = half_value(h[i].box[3 * c + k] >> 16);
            }
            sum += box_area(lo, hi);
            qsum += box_area(qlo, qhi);
        }
    }
    return sum > 0.0 ? std::min(qsum / sum - 1.0, 1e6) : 0.0;
}

void collapse_bvh4(const BvhHost& b2, Bvh4Host* out) {
    out->nodes.clear();
    out->nodes.reserve(b2.nodes.size() / 2 + 1);
    Collapser c{b2.nodes, out->nodes};
    int stack = 0;
    c.build(0, &stack);
    out->max_stack = stack;
}

}  // namespace nrrs
