// Device primitives shared by the NRRS kernels: counter-based random numbers,
// small vector math, warp/block reductions.  sm_103a only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nrrs {

// ---------------------------------------------------------------- constants
constexpr int kMaxDepth = 32;
constexpr int kNF = 16;        // RRSNet input features
constexpr int kNH = 32;        // RRSNet hidden width (Sec. 4 "Network Architecture")
constexpr int kNParams = kNH * kNF + 2 * kNH * kNH + kNH;  // 2592
constexpr int kAidIn = 32;                                    // AID-NRRS inputs of RRSNet
constexpr int kAidParams = kNH * kAidIn + 2 * kNH * kNH + kNH;  // 3104
constexpr int kRrsParamsMax = kAidParams;
constexpr float kLeak = 0.01f; // Leaky ReLU slope
// Marks a vertex whose RRSNet factor came out non-finite during a render; the sum of q
// that follows replaces it with the throughput heuristic's factor.
constexpr float kQRepair = -2.0f;
constexpr float kRayOffset = 1e-4f;
constexpr uint32_t kLineageStep = 0x9E3779B9u;
constexpr uint32_t kNoHit = 0xFFFFFFFFu;

// Philox counter purposes (word 2 of the counter = depth << 8 | purpose).
constexpr uint32_t kPurposeJitter = 0u;
constexpr uint32_t kPurposeBsdf = 1u;
constexpr uint32_t kPurposeRrs = 3u;
constexpr uint32_t kPurposeNee = 5u;
// A shadow ray ends at (1 - margin) x the distance to its emitter point.
constexpr float kShadowMargin = 1e-4f;

enum Mode : int { kNone = 0, kPlainRR = 1, kHeurNorm = 2, kNet = 3, kNetMix = 4 };
enum Gate : int { kGateNet = 0, kGateHeur = 1, kGateFixed = 2, kGateAdrrs = 3 };

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., "Parallel Random Numbers: As Easy as 1, 2, 3" (SC 2011): ten rounds
// of the 4x32 Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and the key bumped
// by the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Draw for one (pixel, sample, depth, purpose, lineage) counter under key
// (seed_lo, seed_hi ^ frame).
__device__ __forceinline__ U4 draw(uint32_t key0, uint32_t key1, uint32_t pixel, uint32_t sample,
                                   uint32_t depth, uint32_t purpose, uint32_t lineage) {
    return philox4x32_10(U4{pixel, sample, (depth << 8) | purpose, lineage}, key0, key1);
}

// Top 24 bits scaled by 2^-24: exactly representable, in [0, 1).
__device__ __forceinline__ float u01(uint32_t w) {
    return __uint2float_rn(w >> 8) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------- vectors
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return V3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 normalize3(V3 a) { return a * (1.0f / sqrtf(dot3(a, a))); }
__device__ __forceinline__ V3 xyz(float4 a) { return V3{a.x, a.y, a.z}; }

__device__ __forceinline__ float lum(float r, float g, float b) {
    return 0.2126f * r + 0.7152f * g + 0.0722f * b;
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (warp butterflies, then warp 0 over warp totals).
// Every thread gets the result.  `sh` needs blockDim.x / 32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T t = lane < nw ? sh[lane] : T(0);
    if (wid == 0) {
        t = warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// Exclusive scan of one uint32 per thread over the block; returns the prefix and the
// block total.  `sh` needs blockDim.x / 32 + 1 elements.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        if (lane < nw) sh[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == nw - 1) sh[32] = wi;   // block total
    }
    __syncthreads();
    const uint32_t r = sh[wid] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

}  // namespace nrrs
