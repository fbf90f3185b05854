// StatNet's input encodings of Sec. 4 "Input Encoding" on the GPU: the trainable
// multiresolution hash grid of the position (Mueller et al. 2022; 8 levels of 2
// features, resolution 16 at the coarsest level and doubling per level, 2^18 entries per
// level) and one-blob encodings (Mueller et al. 2019) of the outgoing direction's
// spherical coordinates (4 bins each) and of the remapped roughness (8 bins).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nrrs {

constexpr int kGridLevels = 8;
constexpr int kGridF = 2;
constexpr uint32_t kGridT = 1u << 18;
constexpr int kGridBase = 16;
constexpr long long kGridParams = (long long)kGridLevels * kGridT * kGridF;  // 4,194,304
constexpr int kStatGridIn = 32;  // StatNet inputs with the encodings

// Entry of grid vertex (x, y, z) at level l: the dense index while (N_l + 1)^3 fits the
// table, else the spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861) mod T.
__device__ __forceinline__ uint32_t grid_index(int l, uint32_t x, uint32_t y, uint32_t z) {
    const uint32_t n1 = ((uint32_t)kGridBase << l) + 1u;
    if ((unsigned long long)n1 * n1 * n1 <= kGridT) return x + n1 * (y + n1 * z);
    return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & (kGridT - 1u);
}

// Cell of p at level l (the last cell for p = 1) and its fractional position.
__device__ __forceinline__ void grid_cell(int l, float px, float py, float pz, uint32_t* i0,
                                          float* f) {
    const float N = (float)(kGridBase << l);
    const float s[3] = {px * N, py * N, pz * N};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float fl = fminf(fmaxf(floorf(s[c]), 0.0f), N - 1.0f);
        i0[c] = (uint32_t)fl;
        f[c] = s[c] - fl;
    }
}

// 16 features (level-major) of p in [0, 1]^3: per level the trilinear interpolation of the
// cell's 8 corner entries.  table: [8][T] float2.
__device__ __forceinline__ void grid_encode(const float2* __restrict__ table, float px, float py,
                                            float pz, float* out) {
#pragma unroll
    for (int l = 0; l < kGridLevels; ++l) {
        uint32_t i0[3];
        float f[3];
        grid_cell(l, px, py, pz, i0, f);
        const float2* tl = table + (size_t)l * kGridT;
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
            const float w = (bx ? f[0] : 1.0f - f[0]) * (by ? f[1] : 1.0f - f[1]) *
                            (bz ? f[2] : 1.0f - f[2]);
            const float2 e = __ldg(&tl[grid_index(l, i0[0] + bx, i0[1] + by, i0[2] + bz)]);
            a0 = fmaf(w, e.x, a0);
            a1 = fmaf(w, e.y, a1);
        }
        out[2 * l] = a0;
        out[2 * l + 1] = a1;
    }
}

// Adds the table gradient of sum_j dout[j] encode(p)[j] (the adjoint of grid_encode).
__device__ __forceinline__ void grid_scatter(float* __restrict__ grad, float px, float py,
                                             float pz, const float* dout) {
#pragma unroll 1
    for (int l = 0; l < kGridLevels; ++l) {
        uint32_t i0[3];
        float f[3];
        grid_cell(l, px, py, pz, i0, f);
        float* gl = grad + (size_t)l * kGridT * kGridF;
        const float d0 = dout[2 * l], d1 = dout[2 * l + 1];
        if (d0 == 0.0f && d1 == 0.0f) continue;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
            const float w = (bx ? f[0] : 1.0f - f[0]) * (by ? f[1] : 1.0f - f[1]) *
                            (bz ? f[2] : 1.0f - f[2]);
            const uint32_t idx = grid_index(l, i0[0] + bx, i0[1] + by, i0[2] + bz);
            atomicAdd(&gl[2 * (size_t)idx], w * d0);
            atomicAdd(&gl[2 * (size_t)idx + 1], w * d1);
        }
    }
}

// One-blob: bin i of K holds exp(-((i + 1/2) / K - v)^2 K^2 / 2) (sigma = 1 / K).
template <int K>
__device__ __forceinline__ void one_blob(float v, float* out) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float d = ((float)i + 0.5f) - v * (float)K;
        out[i] = expf(-0.5f * d * d);
    }
}

// StatNet's 32 inputs: grid(p) (16), one-blob(theta / pi, 4) and one-blob((phi + pi) /
// (2 pi), 4) of w_o (theta from the z axis), one-blob(1 - exp(-alpha), 8).
__device__ __forceinline__ void statnet_grid_inputs(const float2* __restrict__ table, float px,
                                                    float py, float pz, float wx, float wy,
                                                    float wz, float alpha, float* x) {
    grid_encode(table, px, py, pz, x);
    const float theta = acosf(fminf(fmaxf(wz, -1.0f), 1.0f)) * 0.318309886183791f;
    const float phi = (atan2f(wy, wx) + 3.141592653589793f) * 0.159154943091895f;
    one_blob<4>(theta, x + 16);
    one_blob<4>(phi, x + 20);
    one_blob<8>(1.0f - expf(-alpha), x + 24);
}

__device__ __forceinline__ float boxcox_l(float x, float lambda) {
    if (lambda == 0.5f) return 2.0f * (sqrtf(x) - 1.0f);
    if (lambda == 0.0f) return logf(x);
    return (powf(x, lambda) - 1.0f) / lambda;
}

// AID-NRRS's 32 RRSNet inputs (Sec. 4 "Input Encoding"): RRSNet's own grid of the
// position (16), one-blob w_o as for StatNet (8), Box-Cox of the throughput (3) and of the
// pixel estimate's mean clamped at 0 (1), one-blob(1 - exp(-alpha), 4).
__device__ __forceinline__ void aid_inputs(const float2* __restrict__ table, float px, float py,
                                           float pz, float wx, float wy, float wz, float tx,
                                           float ty, float tz, float I, float alpha,
                                           float lambda, float* x) {
    grid_encode(table, px, py, pz, x);
    const float theta = acosf(fminf(fmaxf(wz, -1.0f), 1.0f)) * 0.318309886183791f;
    const float phi = (atan2f(wy, wx) + 3.141592653589793f) * 0.159154943091895f;
    one_blob<4>(theta, x + 16);
    one_blob<4>(phi, x + 20);
    x[24] = boxcox_l(tx, lambda);
    x[25] = boxcox_l(ty, lambda);
    x[26] = boxcox_l(tz, lambda);
    x[27] = boxcox_l(fmaxf(I, 0.0f), lambda);
    one_blob<4>(1.0f - expf(-alpha), x + 28);
}

}  // namespace nrrs
