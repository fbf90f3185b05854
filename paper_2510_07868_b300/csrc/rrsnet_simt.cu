// RRSNet forward in FP32 on the CUDA cores (sm_103a).  Sec. 4 "Network Architecture":
// 16 -> 32 -> 32 -> 32 -> 1, no biases, Leaky ReLU after each hidden layer; output through
// Eq. rrsnet_activation.  The 2592 weights sit in shared memory and are read as 128-bit
// broadcasts (every lane of a warp reads the same weight).  A thread evaluates ROWS rows
// at once so that each weight read feeds ROWS multiply-adds: the kernel is bound by
// shared-memory issue at ROWS = 1 and by FMA issue and register pressure at ROWS = 2.
// Each row's sums run in the same order whatever ROWS is, so results are identical.
#include <cfloat>

#include "grid.cuh"
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

// StatNet's weights in shared memory: sized for the 32-input (encoded) network.
constexpr int kStatSmem = kNH * kStatGridIn + 2 * kNH * kNH + 6 * kNH;

// Roughness of the surface a row's ray hit (Lambertian: 1).
__device__ __forceinline__ float hit_roughness(const SceneView& sc, const float2* hit, long long i) {
    const int slot = __float_as_int(hit[i].y);
    const nrrs_material& m = sc.mats[__float_as_uint(__ldg(&sc.tris[3 * slot + 1].w))];
    return m.type == 0 ? 1.0f : m.roughness;
}

// StatNet's six outputs at row i (Sec. 3.2, 4): with a hash grid on the encodings of
// Sec. 4 "Input Encoding" (position, w_o, roughness), else on the vertex features with the
// throughput inputs zeroed.  sW: the weights in shared memory.
__device__ __forceinline__ void statnet_outputs(const float* sW, const float4* __restrict__ feat,
                                                long long i, const float2* grid, float alpha,
                                                float* out) {
    float h[1][kNH], g[1][kNH];
    int kin;
    if (grid) {
        float x[1][kStatGridIn];
        const float4 f0 = feat[4 * i], f1 = feat[4 * i + 1];
        statnet_grid_inputs(grid, f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, alpha, x[0]);
        dense<1, kStatGridIn>(sW, x, h);
        kin = kStatGridIn;
    } else {
        float x[1][kNF];
        load_row(feat, i, x[0]);
        x[0][13] = x[0][14] = x[0][15] = 0.0f;
        dense<1, kNF>(sW, x, h);
        kin = kNF;
    }
    const float* W2 = sW + kNH * kin;
    dense<1, kNH>(W2, h, g);
    dense<1, kNH>(W2 + kNH * kNH, g, h);
    const float* W4 = W2 + 2 * kNH * kNH;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        float z = 0.0f;
#pragma unroll
        for (int k = 0; k < kNH; ++k) z = fmaf(W4[o * kNH + k], h[0][k], z);
        out[o] = z;
    }
}

__device__ __forceinline__ void load_statnet(const float* __restrict__ stat, bool grid, float* sW) {
    const int n = (grid ? kNH * kStatGridIn : kNH * kNF) + 2 * kNH * kNH + 6 * kNH;
    for (int i = threadIdx.x; i < n / 4; i += blockDim.x)
        reinterpret_cast<float4*>(sW)[i] = __ldg(reinterpret_cast<const float4*>(stat) + i);
}

// ADRRS (NN) factors, Sec. 4 "Mix-Depth": StatNet (16 -> 32 -> 32 -> 32 -> 6, the
// throughput inputs zeroed as in its training) predicts E[<L>] per channel at each
// vertex the render marked (q < 0); r = lum(t) max(mean_rgb E[<L>], 0) / max(I_px, eps_I)
// is the path's expected contribution over the pixel estimate.  As in ADRRS's weight
// window, q = 1 for r in [1/3, 5/3] and q = r outside, clamped to [kAdrrsFloor, q_max]
// so a path predicted dark keeps a small survival probability.  Before any reference exists the factor is the throughput heuristic's.
// A non-finite prediction is marked for the heuristic stand-in (kQRepair).
constexpr float kAdrrsFloor = 0.05f;
// ADRRS's weight window (ratio 5 around the ideal throughput): lower bound 2 / (1 + 5),
// upper bound 5 times that, as fractions of the pixel estimate
constexpr float kAdrrsWindowLo = (float)(2.0 / 6.0);
constexpr float kAdrrsWindowHi = (float)(10.0 / 6.0);

__global__ void __launch_bounds__(kThreads, 2)
k_adrrs_simt(const float* __restrict__ stat, SceneView sc, const float4* __restrict__ feat,
             const float4* t, const float4* dep, const float2* hit, const long long* n_ptr,
             float* q, RenderParams rp, DevStats* st) {
    __shared__ __align__(16) float sW[kStatSmem];
    const long long n = *n_ptr;
    if ((long long)blockIdx.x * blockDim.x >= n) return;
    load_statnet(stat, rp.stat_grid != nullptr, sW);
    __syncthreads();
    const int has_ref = st->has_ref;
    unsigned int evals = 0, nonfinite = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(q[i] < 0.0f)) continue;
        const float4 t4 = t[i];
        const uint32_t pix = __float_as_uint(dep[i].w);
        const float l = lum(t4.x, t4.y, t4.z);
        float eps_I = st->eps_I;
        if (rp.jobs.job) eps_I = rp.jobs.eps_I[job_of_pixel(rp.jobs.job, rp.jobs.n, pix)];
        float v;
        if (!has_ref) {
            v = l;
        } else {
            float so[6];
            statnet_outputs(sW, feat, i, rp.stat_grid,
                            rp.stat_grid ? hit_roughness(sc, hit, i) : 0.0f, so);
            const float m = (so[0] + so[1] + so[2]) * (1.0f / 3.0f);
            const float* rr = rp.ref + 3 * (size_t)pix;
            const float den = fmaxf((rr[0] + rr[1] + rr[2]) / 3.0f, eps_I);
            // r: the path's expected contribution over the pixel estimate; inside the
            // weight window [1/3, 5/3] the path goes on unchanged
            v = den > 0.0f ? l * fmaxf(m, 0.0f) / den : rp.q_max;
            ++evals;
            if (!(v <= FLT_MAX)) {  // NaN or infinite prediction
                v = kQRepair;
                ++nonfinite;
            } else {
                if (v >= kAdrrsWindowLo && v <= kAdrrsWindowHi) v = 1.0f;
                v = fminf(fmaxf(v, kAdrrsFloor), rp.q_max);
            }
        }
        q[i] = v;
    }
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

// The NRRS inputs of RRSNet (Sec. 4 "Input Encoding") of each row the render marked for
// the network (q < 0): StatNet on the vertex features (throughput inputs zeroed, as
// trained) gives E[L_o] and E[L_o^2] per channel; the row becomes Box-Cox(max(E[L_o], 0)),
// Box-Cox(max(E[L_o^2], 0)), Box-Cox(t), Box-Cox(I_px mean, 0 before any estimate),
// 1 - exp(-roughness) (Lambertian: roughness 1), then five zeros.
__device__ __forceinline__ float boxcox_in(float x, float lambda) {
    if (lambda == 0.5f) return 2.0f * (sqrtf(x) - 1.0f);
    if (lambda == 0.0f) return logf(x);
    return (powf(x, lambda) - 1.0f) / lambda;
}

__global__ void __launch_bounds__(kThreads, 2)
k_nrrs_inputs(const float* __restrict__ stat, SceneView sc, const float4* __restrict__ feat,
              const float4* t, const float4* dep, const float2* hit, const long long* n_ptr,
              const float* q, float4* out, RenderParams rp) {
    __shared__ __align__(16) float sW[kStatSmem];
    const long long n = *n_ptr;
    if ((long long)blockIdx.x * blockDim.x >= n) return;
    load_statnet(stat, rp.stat_grid != nullptr, sW);
    __syncthreads();
    const float lam = rp.boxcox_lambda;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(q[i] < 0.0f)) continue;
        const float rough = hit_roughness(sc, hit, i);
        float so[6];
        statnet_outputs(sW, feat, i, rp.stat_grid, rough, so);
        float f[kNF];
#pragma unroll
        for (int o = 0; o < 6; ++o) f[o] = boxcox_in(fmaxf(so[o], 0.0f), lam);
        const float4 t4 = t[i];
        f[6] = boxcox_in(t4.x, lam);
        f[7] = boxcox_in(t4.y, lam);
        f[8] = boxcox_in(t4.z, lam);
        float I = 0.0f;
        if (rp.ref) {
            const float* rr = rp.ref + 3 * (size_t)__float_as_uint(dep[i].w);
            I = (rr[0] + rr[1] + rr[2]) / 3.0f;
        }
        f[9] = boxcox_in(fmaxf(I, 0.0f), lam);
        f[10] = 1.0f - expf(-rough);
#pragma unroll
        for (int k = 11; k < kNF; ++k) f[k] = 0.0f;
        float4* o4 = out + 4 * i;
        o4[0] = make_float4(f[0], f[1], f[2], f[3]);
        o4[1] = make_float4(f[4], f[5], f[6], f[7]);
        o4[2] = make_float4(f[8], f[9], f[10], f[11]);
        o4[3] = make_float4(f[12], f[13], f[14], f[15]);
    }
}

// AID-NRRS (Sec. 4 "Input Encoding"): RRSNet (32 -> 32 -> 32 -> 32 -> 1, FP32) on its own
// hash grid of the position, one-blob w_o and roughness, Box-Cox throughput and pixel
// estimate, for every row the render marked (q < 0); output through Eq. rrsnet_activation,
// a non-finite factor marked for the heuristic stand-in (kQRepair).
__global__ void __launch_bounds__(kThreads, 2)
k_aid_rrsnet(const float* __restrict__ params, const float2* __restrict__ rgrid, SceneView sc,
             const float4* __restrict__ feat, const float4* t, const float4* dep, const float2* hit,
             const long long* n_ptr, float* q, RenderParams rp, DevStats* st) {
    __shared__ __align__(16) float sW[kAidParams];
    const long long n = *n_ptr;
    if ((long long)blockIdx.x * blockDim.x >= n) return;
    for (int i = threadIdx.x; i < kAidParams / 4; i += blockDim.x)
        reinterpret_cast<float4*>(sW)[i] = __ldg(reinterpret_cast<const float4*>(params) + i);
    __syncthreads();
    unsigned int evals = 0, nonfinite = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(q[i] < 0.0f)) continue;
        const float4 f0 = feat[4 * i], f1 = feat[4 * i + 1], t4 = t[i];
        float I = 0.0f;
        if (rp.ref) {
            const float* rr = rp.ref + 3 * (size_t)__float_as_uint(dep[i].w);
            I = (rr[0] + rr[1] + rr[2]) / 3.0f;
        }
        float x[1][kAidIn];
        aid_inputs(rgrid, f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, t4.x, t4.y, t4.z, I,
                   hit_roughness(sc, hit, i), rp.boxcox_lambda, x[0]);
        float h[1][kNH], g[1][kNH];
        dense<1, kAidIn>(sW, x, h);
        dense<1, kNH>(sW + kNH * kAidIn, h, g);
        dense<1, kNH>(sW + kNH * kAidIn + kNH * kNH, g, h);
        const float* W4 = sW + kNH * kAidIn + 2 * kNH * kNH;
        float z = 0.0f;
#pragma unroll
        for (int k = 0; k < kNH; ++k) z = fmaf(W4[k], h[0][k], z);
        float v = softplus_mod(z);
        ++evals;
        if (!(v >= 0.0f && v <= FLT_MAX)) {
            v = kQRepair;
            ++nonfinite;
        }
        q[i] = v;
    }
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

void launch_aid_rrsnet(const float* params, const float2* rgrid, const SceneView& sc,
                       const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                       int grid, cudaStream_t s) {
    k_aid_rrsnet<<<grid, kThreads, 0, s>>>(params, rgrid, sc, w.feat, cur.t, w.dep, w.hit,
                                           &w.st->live[depth - 1], w.q, rp, w.st);
}

void launch_nrrs_inputs(const float* stat, const SceneView& sc, const WorkView& w, QueueView cur,
                        const RenderParams& rp, int depth, int grid, float4* out, cudaStream_t s) {
    k_nrrs_inputs<<<grid, kThreads, 0, s>>>(stat, sc, w.feat, cur.t, w.dep, w.hit,
                                            &w.st->live[depth - 1], w.q, out, rp);
}

void launch_adrrs(const float* stat, const SceneView& sc, const WorkView& w, QueueView cur,
                  const RenderParams& rp, int depth, int grid, cudaStream_t s) {
    k_adrrs_simt<<<grid, kThreads, 0, s>>>(stat, sc, w.feat, cur.t, w.dep, w.hit,
                                           &w.st->live[depth - 1], w.q, rp, w.st);
}

void launch_rrsnet_simt(int rows, int grid, const float* params, const float4* feat,
                        const long long* n_ptr, long long n_host, float* q, int sentinel,
                        DevStats* st, cudaStream_t s) {
    if (rows == 2)
        k_rrsnet_simt<2><<<grid, kThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel, st);
    else
        k_rrsnet_simt<1><<<grid, kThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel, st);
}

}  // namespace nrrs
