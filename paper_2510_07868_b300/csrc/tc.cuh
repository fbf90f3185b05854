// Tensor-core building blocks shared by the RRSNet kernels (rrsnet_tc.cu) and the fused
// shade + RRSNet kernel (wavefront.cu): tcgen05 MMAs with BF16 operands in shared memory
// and FP32 accumulators in tensor memory (sm_103a), the mbarrier and proxy fences that
// order them, and the operand conversions.  RRSNet (Sec. 4 "Network Architecture"): 16 ->
// 32 -> 32 -> 32 -> 1, no biases, Leaky ReLU after each hidden layer, Eq.
// rrsnet_activation on the output; layers 1-3 are M = 128 x N = 32 MMAs (K = 16, then
// K = 32 as two K = 16 steps), the output layer runs in FP32 on the CUDA cores.
//
// Shared-memory operands use the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 bytes apart (LBO), 8-row groups
// (K / 8) * 128 bytes apart (SBO).  Thread t of a tile is row t and TMEM lane t.
#pragma once
#include <cuda_bf16.h>

#include <cfloat>

#include "wavefront.cuh"

namespace nrrs {

namespace {

constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 32;
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz: a wait this long is a fault

// SPLIT: every operand as the BF16 pair (hi, lo), three MMAs per product; otherwise one
// BF16 rounding per operand and one MMA (precision 17).
template <bool SPLIT>
struct __align__(128) TcSmem {
    static constexpr int NB = SPLIT ? 2 : 1;
    unsigned char w1[NB][32 * 16 * 2];   // B of layer 1 (hi, lo): N = 32 rows, K = 16
    unsigned char w2[NB][32 * 32 * 2];   // B of layer 2 (hi, lo)
    unsigned char w3[NB][32 * 32 * 2];   // B of layer 3 (hi, lo)
    unsigned char a[NB][128 * 32 * 2];   // A of every layer (hi, lo): 128 rows, K = 32 layout
    float w4[32];
    unsigned long long bar;
    uint32_t tmem;
};

// Byte offset of element (r, k) in a K-major, no-swizzle operand with K columns.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, leading and stride byte offsets (>> 4),
// descriptor version 1 at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                                ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdescBf16), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// Bounded wait on phase `phase` of the mbarrier; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// Bulk copy (the non-tensor TMA path) of `bytes` contiguous bytes of global memory into
// shared memory, completing on mbarrier `bar`; both addresses 16-byte aligned and
// `bytes` a multiple of 16.  Issued by one thread; the caller has ordered every earlier
// generic read of the destination before it (barrier + proxy fence).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Feature rows of tile `tile` (128 rows of 64 bytes, fewer in the last tile).
__device__ __forceinline__ void stage_tile(float4* stage, const float4* feat, long long tile,
                                           long long n, uint32_t bar) {
    const long long first = tile * 128;
    const long long rows = n - first < 128 ? n - first : 128;
    bulk_load(smem_u32(stage), feat + 4 * first, (uint32_t)(rows * 64), bar);
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Writes 8 consecutive values of row r (columns 8c .. 8c+7) into K-major tiles as the
// BF16 pair hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void store_split8(unsigned char* hi, unsigned char* lo, int r, int c,
                                             int K, const float* v) {
    __nv_bfloat162 ph[4], pl[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ph[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        // hi as FP32 (a BF16 is the top half of its FP32), then both residuals in one
        // packed subtraction (sm_100+), each rounded as a scalar one would be
        const uint32_t u = *reinterpret_cast<const uint32_t*>(&ph[j]);
        const float2 f = make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
        const float2 d = __fadd2_rn(make_float2(v[2 * j], v[2 * j + 1]), make_float2(-f.x, -f.y));
        pl[j] = __floats2bfloat162_rn(d.x, d.y);
    }
    const uint32_t off = kmajor_off(r, 8 * c, K);
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<uint4*>(ph);
    *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<uint4*>(pl);
}

// Writes 8 consecutive values of row r (columns 8c .. 8c+7) into a K-major tile as BF16.
__device__ __forceinline__ void store_bf16_8(unsigned char* hi, int r, int c, int K,
                                             const float* v) {
    __nv_bfloat162 ph[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) ph[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    *reinterpret_cast<uint4*>(hi + kmajor_off(r, 8 * c, K)) = *reinterpret_cast<uint4*>(ph);
}

__device__ __forceinline__ void store_split1(unsigned char* hi, unsigned char* lo, uint32_t off,
                                             float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ float softplus_mod_tc(float z) {
    return z < 0.0f ? log1pf(expf(z)) : fmaf(0.5f, z, 0.693147180559945f);
}

// Layer 1-3 weights of RRSNet (params packed as nrrs_set_rrsnet_params: W1 [32][16], W2
// [32][32], W3 [32][32], w4 [32]) as the B operands of a CTA's MMAs (K-major, BF16 or the
// split (hi, lo) pair) and the FP32 output row; every thread of the CTA takes part.
template <bool SPLIT, class Smem>
__device__ __forceinline__ void tc_stage_weights(Smem& sm, const float* __restrict__ params,
                                                 int tid) {
    constexpr int LO = SPLIT ? 1 : 0;
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
}

// Layer 1's operand: this thread's 16 features as row `tid` of the A buffer.
template <bool SPLIT, class Smem>
__device__ __forceinline__ void tc_store_input(Smem& sm, int tid, const float (&x)[16]) {
    if (SPLIT) {
        store_split8(sm.a[0], sm.a[1], tid, 0, 32, x);
        store_split8(sm.a[0], sm.a[1], tid, 1, 32, x + 8);
    } else {
        store_bf16_8(sm.a[0], tid, 0, 32, x);
        store_bf16_8(sm.a[0], tid, 1, 32, x + 8);
    }
}

// The three hidden layers of one 128-row tile whose layer-1 operand the CTA has written
// to sm.a: per layer the barrier, the MMAs issued by thread 0 (hi*hi + lo*hi + hi*lo per
// K = 16 step with the split, one hi*hi without), thread 0's wait for their completion,
// the accumulator read from this thread's TMEM lane and Leaky ReLU; the output of layers
// 1 and 2 becomes the next operand once every MMA read of the buffer is done.  On return
// h holds this thread's row of layer 3's activations.  False (for the whole CTA) after a
// timed-out wait.
template <bool SPLIT>
__device__ __forceinline__ bool tc_hidden_layers(TcSmem<SPLIT>& sm, uint32_t tmem, uint32_t bar,
                                                 uint32_t taddr, uint32_t& phase,
                                                 float (&h)[32]) {
    constexpr int LO = SPLIT ? 1 : 0;
    const int tid = threadIdx.x;
    const uint64_t k16 = 256 >> 4;  // start address step of K = 16 (two core matrices)
    for (int layer = 0; layer < 3; ++layer) {
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const unsigned char* wb = layer == 0 ? sm.w1[0] : layer == 1 ? sm.w2[0] : sm.w3[0];
            const uint32_t wstep = layer == 0 ? 32 * 16 * 2 : 32 * 32 * 2;  // hi -> lo
            const uint64_t b0 = smem_desc(smem_u32(wb), 128, layer == 0 ? 256 : 512);
            const uint64_t b1 = smem_desc(smem_u32(wb) + wstep, 128, layer == 0 ? 256 : 512);
            const uint64_t a0 = smem_desc(smem_u32(sm.a[0]), 128, 512);
            const uint64_t a1 = smem_desc(smem_u32(sm.a[LO]), 128, 512);
            const int ksteps = layer == 0 ? 1 : 2;
            for (int ks = 0; ks < ksteps; ++ks) {
                const uint64_t o = ks * k16;
                mma_bf16(tmem, a0 + o, b0 + o, ks > 0 ? 1u : 0u);
                if (SPLIT) {
                    mma_bf16(tmem, a1 + o, b0 + o, 1u);
                    mma_bf16(tmem, a0 + o, b1 + o, 1u);
                }
            }
            mma_commit(bar);
        }
        // one thread waits for the MMAs; the barrier releases the others (no spinning)
        const bool ok = tid == 0 ? mbar_wait(bar, phase) : true;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) return false;
        fence_after();
        tmem_ld32(taddr, h);
        // Leaky ReLU as max(x, slope x) (slope < 1), the scaling two lanes at a time
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float2 s = __fmul2_rn(make_float2(h[j], h[j + 1]), make_float2(kLeak, kLeak));
            h[j] = fmaxf(h[j], s.x);
            h[j + 1] = fmaxf(h[j + 1], s.y);
        }
        if (layer < 2) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (SPLIT)
                    store_split8(sm.a[0], sm.a[LO], tid, c, 32, h + 8 * c);
                else
                    store_bf16_8(sm.a[0], tid, c, 32, h + 8 * c);
            }
        }
    }
    return true;
}

// The 32 -> 1 output layer in FP32 and Eq. rrsnet_activation.
__device__ __forceinline__ float tc_output(const float* w4, const float (&h)[32]) {
    float z = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; k += 4) {  // the output row read as 128-bit broadcasts
        const float4 wv = *reinterpret_cast<const float4*>(&w4[k]);
        z = fmaf(wv.x, h[k], z);
        z = fmaf(wv.y, h[k + 1], z);
        z = fmaf(wv.z, h[k + 2], z);
        z = fmaf(wv.w, h[k + 3], z);
    }
    return softplus_mod_tc(z);
}

// Allocates the CTA's TMEM columns (warp 0) and initialises one MMA mbarrier (thread 0).
__device__ __forceinline__ void tc_setup(uint32_t* tmem_slot, unsigned long long* bar,
                                         uint32_t cols) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// Frees the CTA's TMEM columns once every thread's TMEM accesses are done.
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t cols) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(cols));
    }
}

}  // namespace

}  // namespace nrrs
