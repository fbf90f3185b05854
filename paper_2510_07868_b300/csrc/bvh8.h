// The compressed eight-wide BVH built on the device (bvh8.cu): layout and build.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bvh.h"

namespace nrrs {

// Device arrays of one built tree (owned by the caller after a successful build).
struct Bvh8Device {
    uint4* nodes = nullptr;   // 5 uint4 (80 bytes) per node, node 0 the root
    float4* tris = nullptr;   // 3 float4 per triangle, leaf order (the BVH2's layout)
    uint32_t n_nodes = 0;
    int depth = 0;            // node levels; a traversal holds at most depth - 1 groups
    int ploc_iterations = 0;  // rounds of the clustering
};

// Builds the tree of n triangles (d_tri [n][9] vertex coordinates, d_mat [n] material
// ids, both device) inside the scene box [lo, hi]; synchronizes `s`.  Temporary device
// memory is freed before it returns.
cudaError_t build_bvh8(const float* d_tri, const int32_t* d_mat, int n, const float lo[3],
                       const float hi[3], cudaStream_t s, Bvh8Device* out);

// The clustered BVH2 of the same build (Morton order, PLOC), laid out on the host in the
// host builder's format (depth-first preorder, one triangle per leaf, the triangles in
// leaf order) so the BVH2 traversal reads it unchanged.  cudaErrorNotSupported when the
// tree is deeper than max_depth (the traversal's stack bound); *depth_out gets the depth.
cudaError_t build_bvh2_ploc(const float* d_tri, const float* h_tri, const int32_t* h_mat, int n,
                            const float lo[3], const float hi[3], int max_depth, cudaStream_t s,
                            BvhHost* out, int* depth_out);

}  // namespace nrrs
