// RRSNet forward on the 5th-generation tensor cores (tcgen05, sm_103a), BF16 operands,
// FP32 accumulation in tensor memory.  Sec. 4 "Network Architecture": 16 -> 32 -> 32 ->
// 32 -> 1, no biases, Leaky ReLU after each hidden layer, Eq. rrsnet_activation on the
// output.  Layers 1-3 are M=128 x N=32 MMAs (K = 16, then K = 32 as two K = 16 steps);
// the 32 -> 1 output layer and the activation run in FP32 on the CUDA cores.
//
// Precision 17 rounds every operand once to BF16 (one MMA per K step).  Precision 16
// splits every operand v into two BF16 numbers, hi = bf16(v) and lo = bf16(v - hi), and
// takes each product as hi*hi + lo*hi + hi*lo (three MMAs into the same FP32
// accumulator); the dropped lo*lo term and the rounding of lo leave a relative error near
// 2^-16 per product instead of the 2^-8 of one BF16 pass.  Precision 8 (further down)
// uses E4M3 operands with power-of-two scales.  The layer building blocks are in tc.cuh,
// shared with the fused shade + RRSNet kernel of wavefront.cu.
//
// Shared-memory operands use the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 bytes apart (LBO), 8-row groups
// (K / 8) * 128 bytes apart (SBO).  One CTA of 128 threads owns one TMEM allocation of 32
// columns; thread t of the tile is row t and TMEM lane t.  One A buffer (K = 32 layout)
// serves all three layers: layer 1 reads its first 16 columns (the 8-row groups stay
// 512 bytes apart), and each layer's output overwrites it only after that layer's MMAs
// have completed.  Every thread loads its own feature row from global memory one tile
// ahead, so the CTA needs about 26 KB of shared memory (split) and eight fit on an SM.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cfloat>

#include "tc.cuh"
#include "wavefront.cuh"

namespace nrrs {

namespace {

// n_ptr: device row count (render) or null with n_host (stand-alone).  sentinel: only rows
// with q < 0 are evaluated and written (the render's NET slots), a non-finite factor is
// written as kQRepair for the heuristic to replace.
template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 8)  // 8 CTAs (8 tiles in flight) per SM
k_rrsnet_tc(const float* __restrict__ params, const float4* __restrict__ feat,
            const long long* n_ptr, long long n_host, float* q, int sentinel, DevStats* st,
            unsigned int* status) {
    __shared__ TcSmem<SPLIT> sm;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long n = n_ptr ? *n_ptr : n_host;
    if ((long long)blockIdx.x * kTcThreads >= n) return;  // no tile: allocate nothing
    tc_setup(&sm.tmem, &sm.bar, kTmemCols);
    tc_stage_weights<SPLIT>(sm, params, tid);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t bar = smem_u32(&sm.bar);
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    uint32_t phase = 0;
    unsigned int evals = 0, nonfinite = 0;
    bool failed = false;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    // this thread's feature row of the first tile (zeros past the end)
    float4 xr[4];
    auto load_row = [&](long long tile) {
        const long long row = tile * kTcThreads + tid;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            xr[k] = row < n ? __ldg(feat + 4 * row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    load_row(blockIdx.x);
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long row = tile * kTcThreads + tid;
        bool active = row < n;
        if (active && sentinel) active = q[row] < 0.0f;
        float x[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = active ? xr[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
        }
        // the next tile's row is fetched while this one runs through the network
        if (tile + gridDim.x < tiles) load_row(tile + gridDim.x);
        tc_store_input<SPLIT>(sm, tid, x);
        float h[32];
        if (!tc_hidden_layers<SPLIT>(sm, tmem, bar, taddr, phase, h)) {
            failed = true;
            break;
        }
        float qv = tc_output(sm.w4, h);
        if (active) {
            ++evals;
            if (!(qv >= 0.0f && qv <= FLT_MAX)) {
                qv = sentinel ? kQRepair : 0.0f;
                ++nonfinite;
            }
            q[row] = qv;
        }
        fence_before();
        __syncthreads();  // TMEM reads done before the next tile's MMA overwrites it
    }
    if (failed && tid == 0 && status) atomicOr(status, (unsigned int)NRRS_STATUS_TIMEOUT);
    if (st) {
        evals = warp_sum(evals);
        nonfinite = warp_sum(nonfinite);
        if ((tid & 31) == 0) {
            if (evals) atomicAdd(&st->net_evals, (unsigned long long)evals);
            if (nonfinite) {
                atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
                atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
            }
        }
    }
    tc_teardown(tmem, kTmemCols);
}

// ------------------------------------------------------------------ two tiles per CTA
// The same network and the same arithmetic as k_rrsnet_tc (identical factors, bit for
// bit), with two 128-row tiles in flight per CTA so that one tile's MMAs run while the
// CTA's threads convert the other's accumulator: each tile slot s has its own A operand,
// its own 32 TMEM columns (32 s .. 32 s + 31 of a 64-column allocation), its own MMA
// mbarrier, and a staging buffer into which one bulk copy (the non-tensor TMA path) brings
// the slot's next feature tile while the current one runs through the network.  CTA b
// owns tiles b, b + G, b + 2G, ... (G = gridDim.x); slot s takes every other one.  The
// threads visit the two slots in turn; a visit waits for the slot's MMAs, reads its
// accumulator, applies Leaky ReLU, and either writes the next layer's operand and issues
// that layer, or (after layer 3) writes the factor and starts the slot's next tile.
template <bool SPLIT>
struct __align__(128) Tc2Smem {
    static constexpr int NB = SPLIT ? 2 : 1;
    unsigned char w1[NB][32 * 16 * 2];
    unsigned char w2[NB][32 * 32 * 2];
    unsigned char w3[NB][32 * 32 * 2];
    unsigned char a[2][NB][128 * 32 * 2];  // A of each slot (hi, lo), K = 32 layout
    float4 stage[2][128 * 4];              // each slot's next feature tile (64 B rows)
    float w4[32];
    unsigned long long bar[2];   // MMA completion, per slot
    unsigned long long tbar[2];  // staged feature rows, per slot
    uint32_t tmem;
};

constexpr uint32_t kTmemCols2 = 64;

template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads)
k_rrsnet_tc2(const float* __restrict__ params, const float4* __restrict__ feat,
             const long long* n_ptr, long long n_host, float* q, int sentinel, DevStats* st,
             unsigned int* status) {
    extern __shared__ __align__(128) unsigned char tc2_dsm[];
    Tc2Smem<SPLIT>& sm = *reinterpret_cast<Tc2Smem<SPLIT>*>(tc2_dsm);
    constexpr int LO = SPLIT ? 1 : 0;  // index of the lo half (aliases hi without a split)
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long n = n_ptr ? *n_ptr : n_host;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    const long long G = gridDim.x;
    if ((long long)blockIdx.x >= tiles) return;  // no tile: allocate nothing
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(kTmemCols2));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // tile[s]: the slot's current tile (>= tiles: the slot has finished)
    long long tile[2] = {(long long)blockIdx.x, (long long)blockIdx.x + G};
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.tbar[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (tile[s] < tiles) stage_tile(sm.stage[s], feat, tile[s], n, smem_u32(&sm.tbar[s]));
    }
    auto store_w = [&](unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
        if (SPLIT)
            store_split1(hi, lo, off, v);
        else
            *reinterpret_cast<__nv_bfloat16*>(hi + off) = __float2bfloat16_rn(v);
    };
    for (int e = tid; e < 32 * 16; e += kTcThreads)
        store_w(sm.w1[0], sm.w1[LO], kmajor_off(e / 16, e % 16, 16), params[e]);
    for (int e = tid; e < 32 * 32; e += kTcThreads) {
        const uint32_t off = kmajor_off(e / 32, e % 32, 32);
        store_w(sm.w2[0], sm.w2[LO], off, params[512 + e]);
        store_w(sm.w3[0], sm.w3[LO], off, params[1536 + e]);
    }
    if (tid < 32) sm.w4[tid] = params[2560 + tid];
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    const uint64_t k16 = 256 >> 4;  // start address step of K = 16 (two core matrices)
    uint32_t ph[2] = {0u, 0u}, tph[2] = {0u, 0u};
    int layer[2] = {0, 0};           // the layer whose MMAs are in flight
    bool act[2] = {false, false};    // this thread's row of the slot's tile gets a factor
    bool pend[2] = {false, false};   // a staging copy into the slot's buffer is in flight
    pend[0] = true;
    pend[1] = tile[1] < tiles;
    unsigned int evals = 0, nonfinite = 0;
    bool failed = false;

    // MMAs of layer `l` (0-2) of slot s: hi*hi + lo*hi + hi*lo per K = 16 step (one
    // hi*hi without the split), into the slot's 32 accumulator columns.  Thread 0 only.
    auto issue = [&](int s, int l) {
        fence_after();
        const unsigned char* wb = l == 0 ? sm.w1[0] : l == 1 ? sm.w2[0] : sm.w3[0];
        const uint32_t wstep = l == 0 ? 32 * 16 * 2 : 32 * 32 * 2;  // hi -> lo
        const uint64_t b0 = smem_desc(smem_u32(wb), 128, l == 0 ? 256 : 512);
        const uint64_t b1 = smem_desc(smem_u32(wb) + wstep, 128, l == 0 ? 256 : 512);
        const uint64_t a0 = smem_desc(smem_u32(sm.a[s][0]), 128, 512);
        const uint64_t a1 = smem_desc(smem_u32(sm.a[s][LO]), 128, 512);
        const uint32_t d = tmem + 32u * (uint32_t)s;
        const int ksteps = l == 0 ? 1 : 2;
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t o = ks * k16;
            mma_bf16(d, a0 + o, b0 + o, ks > 0 ? 1u : 0u);
            if (SPLIT) {
                mma_bf16(d, a1 + o, b0 + o, 1u);
                mma_bf16(d, a0 + o, b1 + o, 1u);
            }
        }
        mma_commit(smem_u32(&sm.bar[s]));
    };

    // Starts slot s on tile[s]: waits for its staged rows, writes them as layer 1's
    // operand and (after the barrier) issues layer 1; thread 0 then stages the slot's
    // next tile into the buffer every thread has finished reading.  Returns false on a
    // timed-out wait (the whole CTA agrees).
    auto start = [&](int s, bool prior_ok) -> bool {
        const bool landed = mbar_wait(smem_u32(&sm.tbar[s]), tph[s]);
        const bool ok = landed && prior_ok;
        tph[s] ^= 1u;
        const long long row = tile[s] * kTcThreads + tid;
        bool a = row < n;
        if (a && sentinel) a = q[row] < 0.0f;
        act[s] = a;
        float x[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = a ? sm.stage[s][4 * tid + k] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
        }
        if (SPLIT) {
            store_split8(sm.a[s][0], sm.a[s][LO], tid, 0, 32, x);
            store_split8(sm.a[s][0], sm.a[s][LO], tid, 1, 32, x + 8);
        } else {
            store_bf16_8(sm.a[s][0], tid, 0, 32, x);
            store_bf16_8(sm.a[s][0], tid, 1, 32, x + 8);
        }
        fence_async_smem();
        fence_before();
        if (__syncthreads_or(!ok)) {
            if (landed) pend[s] = false;  // else the exit waits for the copy once more
            else tph[s] ^= 1u;
            return false;
        }
        const long long next = tile[s] + 2 * G;
        if (tid == 0) {
            issue(s, 0);
            if (next < tiles) stage_tile(sm.stage[s], feat, next, n, smem_u32(&sm.tbar[s]));
        }
        pend[s] = next < tiles;
        layer[s] = 0;
        return true;
    };

    // One visit of slot s (its MMAs of layer[s] are in flight).
    auto visit = [&](int s) -> bool {
        const bool ok = mbar_wait(smem_u32(&sm.bar[s]), ph[s]);
        ph[s] ^= 1u;
        fence_after();
        float h[32];
        tmem_ld32(lane_base + 32u * (uint32_t)s, h);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float2 sc = __fmul2_rn(make_float2(h[j], h[j + 1]), make_float2(kLeak, kLeak));
            h[j] = fmaxf(h[j], sc.x);
            h[j + 1] = fmaxf(h[j + 1], sc.y);
        }
        if (layer[s] < 2) {
            // the slot's MMAs are complete: its A buffer takes the next layer's operand
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (SPLIT)
                    store_split8(sm.a[s][0], sm.a[s][LO], tid, c, 32, h + 8 * c);
                else
                    store_bf16_8(sm.a[s][0], tid, c, 32, h + 8 * c);
            }
            fence_async_smem();
            fence_before();
            if (__syncthreads_or(!ok)) return false;
            ++layer[s];
            if (tid == 0) issue(s, layer[s]);
            return true;
        }
        float z = 0.0f;
#pragma unroll
        for (int k = 0; k < 32; k += 4) {  // the output row read as 128-bit broadcasts
            const float4 wv = *reinterpret_cast<const float4*>(&sm.w4[k]);
            z = fmaf(wv.x, h[k], z);
            z = fmaf(wv.y, h[k + 1], z);
            z = fmaf(wv.z, h[k + 2], z);
            z = fmaf(wv.w, h[k + 3], z);
        }
        float qv = softplus_mod_tc(z);
        if (act[s]) {
            ++evals;
            if (!(qv >= 0.0f && qv <= FLT_MAX)) {
                qv = sentinel ? kQRepair : 0.0f;
                ++nonfinite;
            }
            q[tile[s] * kTcThreads + tid] = qv;
        }
        tile[s] += 2 * G;
        // every lane's TMEM reads of this tile complete before the barrier in start(),
        // after which layer 1 of the next tile overwrites the slot's columns
        if (tile[s] < tiles) return start(s, ok);
        return !__syncthreads_or(!ok);
    };

    if (!start(0, true)) failed = true;
    if (!failed && tile[1] < tiles && !start(1, true)) failed = true;
    while (!failed && (tile[0] < tiles || tile[1] < tiles)) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (failed || tile[s] >= tiles) continue;
            if (!visit(s)) failed = true;
        }
    }
    if (failed) {
        // copies still in flight land before the CTA leaves (bounded waits)
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (pend[s]) mbar_wait(smem_u32(&sm.tbar[s]), tph[s]);
        if (tid == 0 && status) atomicOr(status, (unsigned int)NRRS_STATUS_TIMEOUT);
    }
    if (st) {
        evals = warp_sum(evals);
        nonfinite = warp_sum(nonfinite);
        if ((tid & 31) == 0) {
            if (evals) atomicAdd(&st->net_evals, (unsigned long long)evals);
            if (nonfinite) {
                atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
                atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols2));
    }
}

// ------------------------------------------------------------------ FP8 (E4M3)
// Same network with E4M3 operands (kind::f8f6f4, K = 32 per MMA, layer 1 zero-padded from
// 16 to 32) and FP32 accumulation.  Each operand tensor gets a power-of-two scale that
// puts its largest finite magnitude in (224, 448] (448 is the E4M3 maximum): one per
// weight matrix, one per 128-row activation tile (the A operand of each MMA).  Powers of
// two make the FP32 readback's unscaling exact, so the only error is the E4M3 rounding of
// the operands (relative 2^-4, absolute 2^-10 / scale in the subnormal range).  A row with
// a non-finite feature or hidden value is left out of its tile's scale and reports a
// non-finite factor; a non-finite hidden weight makes every factor non-finite.
struct __align__(128) Fp8Smem {
    unsigned char w[3][32 * 32];  // B of layers 1-3: N = 32 rows, K = 32 bytes
    unsigned char a[128 * 32];    // A: 128 rows, K = 32 bytes
    float w4[32];
    float4 stage[128 * 4];  // the tile's feature rows, staged by a bulk copy
    unsigned long long tbar;
    int staging;
    float red[4];
    float winv[3];  // 1 / weight scale of layers 1-3
    int wbad;       // a hidden-layer weight is not finite
    unsigned long long bar;
    uint32_t tmem;
};

// Byte offset of element (r, k) in a K-major, no-swizzle 8-bit operand with 32 columns.
__device__ __forceinline__ uint32_t kmajor8_off(int r, int k) {
    return (uint32_t)((r >> 3) * 256 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}

// kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3 (format 0), K-major, N = 32, M = 128.
constexpr uint32_t kIdescE4m3 = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, 0, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdescE4m3));
}

__device__ __forceinline__ float block_max128(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
}

// Largest power of two s with s * amax <= 448 (exponent clamped to +-60; 1 for amax 0).
__device__ __forceinline__ float e4m3_scale(float amax) {
    if (!(amax > 0.0f)) return 1.0f;
    int e;
    frexpf(448.0f / amax, &e);  // 448 / amax = m 2^e, m in [0.5, 1)
    return ldexpf(1.0f, max(-60, min(60, e - 1)));
}

// 32 values of row r (scaled by s) as E4M3 into the A tile.
__device__ __forceinline__ void store_e4m3_row(unsigned char* tile, int r, const float* v, float s) {
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const __nv_fp8x2_storage_t lo =
            __nv_cvt_float2_to_fp8x2(make_float2(v[4 * j] * s, v[4 * j + 1] * s), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(v[4 * j + 2] * s, v[4 * j + 3] * s), __NV_SATFINITE, __NV_E4M3);
        w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    *reinterpret_cast<uint4*>(tile + kmajor8_off(r, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(tile + kmajor8_off(r, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
}

__global__ void __launch_bounds__(kTcThreads)
k_rrsnet_fp8(const float* __restrict__ params, const float4* __restrict__ feat,
             const long long* n_ptr, long long n_host, float* q, int sentinel, DevStats* st,
             unsigned int* status) {
    __shared__ Fp8Smem sm;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long n = n_ptr ? *n_ptr : n_host;
    if ((long long)blockIdx.x * kTcThreads >= n) return;  // no tile: allocate nothing
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.tbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_tile(sm.stage, feat, blockIdx.x, n, smem_u32(&sm.tbar));  // first tile
        sm.staging = 1;
    }
    // per-matrix weight scales, then E4M3 B operands (W1 zero-padded to K = 32)
    const int off[3] = {0, 512, 1536}, kin[3] = {16, 32, 32};
    bool wbad = false;
    for (int l = 0; l < 3; ++l) {
        float m = 0.0f;
        for (int e = tid; e < 32 * kin[l]; e += kTcThreads) {
            const float a = fabsf(params[off[l] + e]);
            if (a <= FLT_MAX) m = fmaxf(m, a);
            else wbad = true;
        }
        m = block_max128(m, sm.red);
        const float sw = e4m3_scale(m);
        if (tid == 0) sm.winv[l] = 1.0f / sw;
        if (tid < 32) {
            float row[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) row[k] = k < kin[l] ? params[off[l] + tid * kin[l] + k] : 0.0f;
            store_e4m3_row(sm.w[l], tid, row, sw);
        }
    }
    if (tid < 32) sm.w4[tid] = params[2560 + tid];
    fence_async_smem();
    fence_before();
    wbad = __syncthreads_or(wbad);
    fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t bar = smem_u32(&sm.bar);
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    const uint64_t da = smem_desc(smem_u32(sm.a), 128, 256);
    uint64_t dw[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) dw[l] = smem_desc(smem_u32(sm.w[l]), 128, 256);
    uint32_t phase = 0, tphase = 0;
    const uint32_t tbar = smem_u32(&sm.tbar);
    unsigned int evals = 0, nonfinite = 0;
    bool failed = false;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    for (long long tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
        const long long row = tile * kTcThreads + tid;
        bool active = row < n;
        if (active && sentinel) active = q[row] < 0.0f;
        const bool staged = mbar_wait(tbar, tphase);  // this tile's rows are in sm.stage
        if (__syncthreads_or(!staged)) {
            failed = true;
            break;
        }
        tphase ^= 1u;
        if (tid == 0) sm.staging = 0;
        float h[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) h[k] = 0.0f;
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = sm.stage[4 * tid + k];
                h[4 * k] = v.x; h[4 * k + 1] = v.y; h[4 * k + 2] = v.z; h[4 * k + 3] = v.w;
            }
        }
        bool bad = wbad;
        for (int layer = 0; layer < 3 && !failed; ++layer) {
            float m = 0.0f;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float a = fabsf(h[k]);
                bad |= !(a <= FLT_MAX);
                m = fmaxf(m, a);
            }
            const float sa = e4m3_scale(block_max128(bad ? 0.0f : m, sm.red));
            store_e4m3_row(sm.a, tid, h, sa);
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                mma_e4m3(tmem, da, dw[layer]);
                mma_commit(bar);
                // every lane has read its staged row: stage the next tile
                if (layer == 0 && tile + gridDim.x < tiles) {
                    stage_tile(sm.stage, feat, tile + gridDim.x, n, tbar);
                    sm.staging = 1;
                }
            }
            // one thread waits for the MMAs; the barrier releases the others (no spinning)
            const bool ok = tid == 0 ? mbar_wait(bar, phase) : true;
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            fence_after();
            tmem_ld32(taddr, h);
            const float inv = (1.0f / sa) * sm.winv[layer];  // exact: powers of two
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float v = h[j] * inv;
                h[j] = v > 0.0f ? v : kLeak * v;
            }
            fence_before();
            __syncthreads();  // the MMA's reads of the A tile and this layer's TMEM reads are done
        }
        if (failed) break;
        float z = 0.0f;
#pragma unroll
        for (int k = 0; k < 32; k += 4) {  // the output row read as 128-bit broadcasts
            const float4 wv = *reinterpret_cast<const float4*>(&sm.w4[k]);
            z = fmaf(wv.x, h[k], z);
            z = fmaf(wv.y, h[k + 1], z);
            z = fmaf(wv.z, h[k + 2], z);
            z = fmaf(wv.w, h[k + 3], z);
        }
        float qv = softplus_mod_tc(z);
        if (active) {
            ++evals;
            if (bad || !(qv >= 0.0f && qv <= FLT_MAX)) {
                qv = sentinel ? kQRepair : 0.0f;
                ++nonfinite;
            }
            q[row] = qv;
        }
    }
    if (failed) {  // let a staging copy still in flight land before the CTA leaves
        __syncthreads();
        if (sm.staging) mbar_wait(tbar, tphase);
    }
    if (failed && tid == 0 && status) atomicOr(status, (unsigned int)NRRS_STATUS_TIMEOUT);
    if (st) {
        evals = warp_sum(evals);
        nonfinite = warp_sum(nonfinite);
        if ((tid & 31) == 0) {
            if (evals) atomicAdd(&st->net_evals, (unsigned long long)evals);
            if (nonfinite) {
                atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
                atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

}  // namespace

namespace {

// Dynamic shared memory of k_rrsnet_tc2, raised above the 48 KB default once per device.
template <bool SPLIT>
cudaError_t tc2_prepare() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_rrsnet_tc2<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Tc2Smem<SPLIT>));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

}  // namespace

int rrsnet_tc2_max_blocks(int precision) {
    static int cache[64][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int& c = cache[dev][precision == 17 ? 1 : 0];
    if (c > 0) return c;
    // resident CTAs from the SM's shared memory and registers (the CTA's dynamic shared
    // memory plus the per-block reservation; 128 threads at the kernel's register count,
    // allocated in units of 8 per thread)
    cudaFuncAttributes fa{};
    const size_t dyn = precision == 17 ? sizeof(Tc2Smem<false>) : sizeof(Tc2Smem<true>);
    const cudaError_t e = precision == 17 ? cudaFuncGetAttributes(&fa, k_rrsnet_tc2<false>)
                                          : cudaFuncGetAttributes(&fa, k_rrsnet_tc2<true>);
    int smem_sm = 0, reserved = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e != cudaSuccess || smem_sm <= 0 || regs_sm <= 0) return 1;
    const long long per_smem = (long long)dyn + (long long)fa.sharedSizeBytes + reserved;
    const long long per_regs = (long long)((fa.numRegs + 7) / 8 * 8) * kTcThreads;
    long long nb = std::min((long long)smem_sm / per_smem, (long long)regs_sm / per_regs);
    // each CTA holds 64 TMEM columns: at most 8 fit the SM's 512
    nb = std::min(nb, 8ll);
    c = nb < 1 ? 1 : (int)nb;
    return c;
}

void launch_rrsnet_tc(int precision, int variant, int grid, const float* params,
                      const float4* feat, const long long* n_ptr, long long n_host, float* q,
                      int sentinel, DevStats* st, unsigned int* status, cudaStream_t s) {
    if (variant == 1 && precision == 17) {
        if (tc2_prepare<false>() == cudaSuccess)
            k_rrsnet_tc2<false><<<grid, kTcThreads, sizeof(Tc2Smem<false>), s>>>(
                params, feat, n_ptr, n_host, q, sentinel, st, status);
    } else if (variant == 1 && precision == 16) {
        if (tc2_prepare<true>() == cudaSuccess)
            k_rrsnet_tc2<true><<<grid, kTcThreads, sizeof(Tc2Smem<true>), s>>>(
                params, feat, n_ptr, n_host, q, sentinel, st, status);
    } else if (precision == 8)
        k_rrsnet_fp8<<<grid, kTcThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel, st,
                                                 status);
    else if (precision == 17)
        k_rrsnet_tc<false><<<grid, kTcThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel,
                                                       st, status);
    else
        k_rrsnet_tc<true><<<grid, kTcThreads, 0, s>>>(params, feat, n_ptr, n_host, q, sentinel,
                                                      st, status);
}

}  // namespace nrrs
