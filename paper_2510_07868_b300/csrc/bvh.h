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

}  // namespace nrrs
