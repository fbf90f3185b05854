// Host BVH2 build; see bvh.cpp for the device layouts.
#pragma once
#include <cstdint>
#include <vector>

namespace nrrs {

struct BvhNode {
    float a[4], b[4], c[4];
    int32_t d[4];
};
static_assert(sizeof(BvhNode) == 64, "node is 4 x float4");

struct BvhHost {
    std::vector<BvhNode> nodes;  // nodes[0] is the root (always an inner node)
    std::vector<float> tris;     // 12 floats per triangle reference, BVH order
    int32_t n_ref = 0;           // triangle references (>= triangles: large ones are split)
    float lo[3], hi[3];          // scene bounds over all vertices
};

void build_bvh(const float* tri, int32_t n_tri, const int32_t* mat_id, BvhHost* out);

// Most inner nodes on any root-to-leaf path of the node array (one tree, or several
// trees appended one after another as in a batch), which bounds the traversal stack: a
// ray holds at most one pushed sibling per inner node on its current path.  Relies on
// every child being stored after its parent (depth-first preorder); -1 when it is not.
int bvh2_height(const std::vector<BvhNode>& nodes);

// Four-wide tree collapsed from the BVH2 (bvh.cpp): 128 bytes per node, the children's
// boxes as six float4 rows (lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of children 0..3), then the
// child codes (as BvhNode) and the leaf reference counts.  An unused slot is a leaf with
// no references.  The triangle references are the BVH2's, unchanged.
struct Bvh4Node {
    float lox[4], hix[4], loy[4], hiy[4], loz[4], hiz[4];
    int32_t child[4];
    int32_t count[4];
};
static_assert(sizeof(Bvh4Node) == 128, "node is 8 x float4");

struct Bvh4Host {
    std::vector<Bvh4Node> nodes;  // nodes[0] is the root
    int max_stack = 0;            // most stack entries a closest-hit traversal can hold
};

void collapse_bvh4(const BvhHost& b2, Bvh4Host* out);

// The BVH2 with half-precision boxes (32 bytes per node, two 16-byte rows): the six
// bounds of child 0 then of child 1, each (lo, hi) pair one word holding two IEEE
// binary16 values (lo in the low half), then the two child codes.  Each lower bound is
// rounded toward -inf and each upper bound toward +inf, so a box only grows: a ray that
// reaches a triangle through the FP32 box still reaches it, and the closest hit is
// unchanged (a few more boxes pass the slab test).  A leaf code is
// ~(first | count << 26).
struct BvhNodeH {
    uint32_t box[6];  // x0, y0, z0, x1, y1, z1: (lo | hi << 16)
    int32_t child[2];
};
static_assert(sizeof(BvhNodeH) == 32, "node is 2 x uint4");

constexpr uint32_t kLeafFirstBits = 26;
constexpr uint32_t kLeafFirstMask = (1u << kLeafFirstBits) - 1u;

// IEEE binary16 bits of x rounded toward +inf (up) or -inf.
uint16_t half_directed(float x, bool up);

// Packs the BVH2's nodes; false (out cleared) when a leaf does not fit the code (more
// than 31 references, or a first reference at or above 2^26).
bool pack_half_nodes(const BvhHost& b2, std::vector<BvhNodeH>* out);

// Relative growth of the summed child-box surface area from the FP32 tree to its
// packed copy (0 = no growth).  A ray's chance of entering a box scales with its area
// (the surface area heuristic's model), so this is the share of extra box visits to
// expect; it stays near 0 for scenes near the origin and grows for a scene far from it
// (binary16 spacing grows with magnitude).
double half_node_growth(const BvhHost& b2, const std::vector<BvhNodeH>& h);

// Growth above which scenes default to the FP32 nodes: one sector per visit instead of
// two measured 25-32 % faster traversal at about 1-2 % growth, so a tenth more visits
// still leaves the FP16 nodes ahead.
constexpr double kMaxHalfGrowth = 0.10;

}  // namespace nrrs
