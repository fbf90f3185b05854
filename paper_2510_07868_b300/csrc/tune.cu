// RRSNet launch shapes per queue-size bucket and the autotuner that picks them.
//
// Queue sizes shrink unevenly from bounce to bounce and from scene to scene, and the best
// launch shape of the RRSNet kernel changes with the size: a small queue wants many
// short-lived blocks (or one row per thread), a large one wants the register-blocked
// two-rows-per-thread FP32 kernel or fewer tensor-core CTAs per SM.  The tuner times
// every candidate shape on synthetic feature rows at one size per power-of-two bucket and
// keeps the fastest; every candidate computes identical results, so the choice changes
// time only.
#include <algorithm>
#include <vector>

#include "wavefront.cuh"

namespace nrrs {

namespace {

// Deterministic synthetic features in [-1, 1) (timing input only).
__global__ void k_fill_features(float4* f, long long n, uint32_t seed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 4; ++k) {
        const U4 w = draw(seed, 0x7u, (uint32_t)i, (uint32_t)(i >> 32), 0u, 9u, (uint32_t)k);
        f[4 * i + k] = make_float4(2.0f * u01(w.x) - 1.0f, 2.0f * u01(w.y) - 1.0f,
                                   2.0f * u01(w.z) - 1.0f, 2.0f * u01(w.w) - 1.0f);
    }
}

}  // namespace

int tune_bucket(long long n) {
    if (n < 512) return 0;
    int lg = 0;
    while ((n >> (lg + 1)) != 0) ++lg;
    return std::min(kTuneBuckets - 1, lg - 8);
}

RrsnetChoice default_choice(int precision) {
    return precision == 32 ? RrsnetChoice{1, 2} : RrsnetChoice{0, 8};
}

std::vector<RrsnetChoice> tune_candidates(int precision) {
    if (precision == 32) return {{1, 2}, {1, 1}, {1, 4}, {2, 1}, {2, 2}};
    if (precision == 8) return {{0, 8}, {0, 1}, {0, 2}, {0, 4}, {0, 6}};
    // the one-tile kernel (default first), then the two-tile kernel
    std::vector<RrsnetChoice> c{default_choice(precision), {0, 2}, {0, 4}, {0, 6}};
    const int mx = rrsnet_tc2_max_blocks(precision);
    for (int b : {1, 2, 3, 4, 6, 8})
        if (b <= mx) c.push_back({1, b});
    return c;
}

void launch_rrsnet(int precision, RrsnetChoice c, int n_sm, const float* params,
                   const float4* feat, const long long* n_ptr, long long n_host, float* q,
                   int sentinel, DevStats* st, unsigned int* status, cudaStream_t s) {
    int bps = std::max(1, c.blocks_per_sm);
    // a persistent two-tile grid no larger than what stays resident
    if (precision != 32 && c.variant == 1) bps = std::min(bps, rrsnet_tc2_max_blocks(precision));
    long long grid = (long long)n_sm * bps;
    if (!n_ptr) {  // the row count is known here: no more blocks than there is work
        if (n_host <= 0) return;
        const long long need = precision == 32
                                   ? ((n_host + c.variant - 1) / c.variant + 255) / 256
                                   : (n_host + 127) / 128;
        grid = std::min(grid, need);
    }
    if (precision == 32)
        launch_rrsnet_simt(c.variant == 2 ? 2 : 1, (int)grid, params, feat, n_ptr, n_host, q,
                           sentinel, st, s);
    else
        launch_rrsnet_tc(precision, c.variant, (int)grid, params, feat, n_ptr, n_host, q, sentinel, st,
                         status, s);
}

// Times every candidate shape at 1.5 x 2^(b + 8) rows (capped at max_rows) for each
// bucket b and writes the fastest into table[b]; rows / ms_best / ms_default receive the
// timed size, the winner's and the default shape's mean launch time.
cudaError_t tune_rrsnet(int precision, int n_sm, const float* params, long long max_rows,
                        cudaStream_t s, RrsnetChoice* table, long long* rows, float* ms_best,
                        float* ms_default) {
    float4* feat = nullptr;
    float* q = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&feat, sizeof(float4) * 4 * (size_t)max_rows);
    if (err == cudaSuccess) err = cudaMalloc(&q, sizeof(float) * (size_t)max_rows);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) {
        k_fill_features<<<(unsigned)((max_rows + 255) / 256), 256, 0, s>>>(feat, max_rows, 12345u);
        err = cudaGetLastError();
    }
    const std::vector<RrsnetChoice> cand = tune_candidates(precision);
    for (int b = 0; b < kTuneBuckets && err == cudaSuccess; ++b) {
        const long long n = std::min(max_rows, 3ll << (b + 7));
        const int reps = (int)std::max(3ll, std::min(50ll, (1ll << 21) / n));
        float best = 0.0f;
        for (size_t k = 0; k < cand.size() && err == cudaSuccess; ++k) {
            for (int r = 0; r < 2; ++r)
                launch_rrsnet(precision, cand[k], n_sm, params, feat, nullptr, n, q, 0, nullptr,
                              nullptr, s);
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r)
                launch_rrsnet(precision, cand[k], n_sm, params, feat, nullptr, n, q, 0, nullptr,
                              nullptr, s);
            cudaEventRecord(e1, s);
            err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (k == 0) ms_default[b] = ms;
            if (k == 0 || ms < best) {
                best = ms;
                table[b] = cand[k];
            }
        }
        rows[b] = n;
        ms_best[b] = best;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaFree(feat);
    cudaFree(q);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return err;
}

}  // namespace nrrs
