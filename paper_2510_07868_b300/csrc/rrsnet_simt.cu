// RRSNet forward in FP32 on the CUDA cores (sm_103a).  Sec. 4 "Network Architecture":
// 16 -> 32 -> 32 -> 32 -> 1, no biases, Leaky ReLU after each hidden layer; output through
// Eq. rrsnet_activation.  The 2592 weights sit in shared memory and are read as 128-bit
// broadcasts (every lane of a warp reads the same weight).  A thread evaluates ROWS rows
// at once so that each weight read feeds ROWS multiply-adds: the kernel is bound by
// shared-memory issue at ROWS = 1 and by FMA issue and register pressure at ROWS = 2.
// Each row's sums run in the same order whatever ROWS is, so results are identical.
#include <cfloat>

#include "wavefront.cuh"

namespace nrrs {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float softplus_mod(float z) {
    return z < 0.0f ? log1pf(expf(z)) : fmaf(0.5f, z, 0.693147180559945f);
}

__device__ __forceinline__ float lrelu(float a) { return a > 0.0f ? a : kLeak * a; }

// y[r][j] = lrelu(sum_k W[j][k] x[r][k]) for ROWS rows; W row-major [32][KIN].
template <int ROWS, int KIN>
__device__ __forceinline__ void dense(const float* __restrict__ W, const float (&x)[ROWS][KIN],
                                      float (&y)[ROWS][kNH]) {
    const float4* W4 = reinterpret_cast<const float4*>(W);
#pragma unroll
    for (int j = 0; j < kNH; ++j) {
        float a[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) a[r] = 0.0f;
#pragma unroll
        for (int k4 = 0; k4 < KIN / 4; ++k4) {
            const float4 w = W4[j * (KIN / 4) + k4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                a[r] = fmaf(w.x, x[r][4 * k4 + 0], a[r]);
                a[r] = fmaf(w.y, x[r][4 * k4 + 1], a[r]);
                a[r] = fmaf(w.z, x[r][4 * k4 + 2], a[r]);
                a[r] = fmaf(w.w, x[r][4 * k4 + 3], a[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) y[r][j] = lrelu(a[r]);
    }
}

template <int ROWS>
__device__ __forceinline__ void forward(const float* __restrict__ w, const float (&x)[ROWS][kNF],
                                        float (&q)[ROWS]) {
    float h[ROWS][kNH], g[ROWS][kNH];
    dense<ROWS, kNF>(w, x, h);
    dense<ROWS, kNH>(w + kNH * kNF, h, g);
    dense<ROWS, kNH>(w + kNH * kNF + kNH * kNH, g, h);
    const float4* W4 = reinterpret_cast<const float4*>(w + kNH * kNF + 2 * kNH * kNH);
    float z[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) z[r] = 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < kNH / 4; ++k4) {
        const float4 ww = W4[k4];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            z[r] = fmaf(ww.x, h[r][4 * k4 + 0], z[r]);
            z[r] = fmaf(ww.y, h[r][4 * k4 + 1], z[r]);
            z[r] = fmaf(ww.z, h[r][4 * k4 + 2], z[r]);
            z[r] = fmaf(ww.w, h[r][4 * k4 + 3], z[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) q[r] = softplus_mod(z[r]);
}

__device__ __forceinline__ void load_row(const float4* __restrict__ feat, long long i,
                                         float (&x)[kNF]) {
    const float4* f = feat + 4 * i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = __ldg(f + k);
        x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
    }
}

// n rows (n_ptr: device count, else n_host).  With `sentinel`, only rows whose q is
// negative are evaluated (the render marks them so); `st` (nullable) receives the counts
// of evaluations and of non-finite results, which are stored as 0.  A thread takes rows
// i and i + ceil(n / ROWS) (ROWS = 2), so both halves are read coalesced.
template <int ROWS>
__global__ void __launch_bounds__(kThreads, ROWS == 1 ? 2 : 1)
k_rrsnet_simt(const float* __restrict__ params, const float4* __restrict__ feat,
              const long long* n_ptr, long long n_host, float* q, int sentinel, DevStats* st) {
    __shared__ __align__(16) float sW[kNParams];
    const long long n = n_ptr ? *n_ptr : n_host;
    const long long span = (n + ROWS - 1) / ROWS;
    if ((long long)blockIdx.x * blockDim.x >= span) return;  // no rows for this block
    for (int i = threadIdx.x; i < kNParams / 4; i += blockDim.x)
        reinterpret_cast<float4*>(sW)[i] = __ldg(reinterpret_cast<const float4*>(params) + i);
    __syncthreads();
    unsigned int evals = 0, nonfinite = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < span;
         i += (long long)gridDim.x * blockDim.x) {
        long long row[ROWS];
        bool act[ROWS];
        bool any = false;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            row[r] = i + r * span;
            act[r] = row[r] < n && (!sentinel || q[row[r]] < 0.0f);
            any |= act[r];
        }
        if (!any) continue;
        float x[ROWS][kNF];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (act[r]) {
                load_row(feat, row[r], x[r]);
            } else {
#pragma unroll
                for (int k = 0; k < kNF; ++k) x[r][k] = 0.0f;
            }
        }
        float out[ROWS];
        forward<ROWS>(sW, x, out);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (!act[r]) continue;
            float v = out[r];
            ++evals;
            if (!(v >= 0.0f && v <= FLT_MAX)) {
                v = sentinel ? kQRepair : 0.0f;
                ++nonfinite;
            }
            q[row[r]] = v;
        }
    }
    if (!st) return;
    evals = warp_sum(evals);
    nonfinite = warp_sum(nonfinite);
    if ((threadIdx.x & 31) == 0) {
        if (evals) atomicAdd(&st->net_evals, (unsigned long long)evals);
        if (nonfinite) {
            atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
            atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
        }
    }
}

}  // namespace

void launch_rrsnet_simt(int rows, int grid, const float* params, const float4* feat,
                        const long long* n_ptr, long long n_host, float* q, int sentinel,
                        DevStats* st, cudaStream_t s) {
    if (rows == 2)
        k_rrsnet_simt<2><<<grid, kThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel, st);
    else
        k_rrsnet_simt<1><<<grid, kThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel, st);
}

}  // namespace nrrs
