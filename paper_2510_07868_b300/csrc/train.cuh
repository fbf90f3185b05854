// Device views and launchers of the training kernels (train.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wavefront.cuh"

namespace nrrs {

constexpr int kStatOut = 6;  // StatNet outputs: E[<L>] and E[<L>^2] per RGB channel
constexpr int kStatParams = kNH * kNF + 2 * kNH * kNH + kStatOut * kNH;  // 2752

// A recorded frame: slot (d, i) of depth d (0-based here) lives at d * C + i.
struct RecordView {
    float4* dep;      // deposit rgb, pixel bits
    float* q;         // q_orig
    float4* t;        // prefix throughput rgb, sample bits
    float4* feat;     // 4 float4 of RRSNet features per slot
    uint32_t* first;  // first child slot in the next depth
    uint32_t* X;      // children requested
    float4* S;        // suffix sum rgb, pixel bits (reverse pass)
    float4* feat_net; // NRRS inputs of RRSNet (4 float4 per slot) or NULL: RRSNet reads feat
    float* rough;     // roughness of each network vertex (StatNet's encoded inputs)
    long long C;
};

// The training batch: every slot of every depth, concatenated in depth order.
struct TrainBatch {
    long long offset[kMaxDepth + 1];  // offset[d] = first batch index of depth d
    long long total;    // recorded vertices of the frame
    long long batch;    // training slots: min(total, batch size)
    uint32_t phase;     // systematic-sampling offset phase / 2^32 in [0, 1)
    int D;
    uint32_t net_mask;  // depths whose slots carry RRSNet features
};

// Vertex of training slot i: systematic sampling of `batch` of the `total` recorded
// vertices with a random offset phi = phase / 2^32 (every vertex has inclusion
// probability batch / total; the identity when batch == total), in integers:
// floor((i + phi) total / batch) = floor((i total + floor(phi total)) / batch), since
// no multiple of batch lies strictly between two consecutive integers.
__host__ __device__ __forceinline__ long long batch_vertex(const TrainBatch& b, long long i) {
    if (b.batch >= b.total) return i;
    const unsigned long long total = (unsigned long long)b.total;
    const unsigned long long shift = (total * (unsigned long long)b.phase) >> 32;
    const unsigned __int128 num = (unsigned __int128)(unsigned long long)i * total + shift;
    const long long u = (long long)(num / (unsigned long long)b.batch);
    return u < b.total ? u : b.total - 1;
}

// kTrainGiven: plain inputs in RecordView::feat ([n][16]) and given output gradients in
// TrainArgs::gin ([n][n_out]); the kernel returns sum_s d(gin_s . out_s)/dW.
enum TrainMode : int {
    kTrainStatNet = 0,
    kTrainRrsWarmup = 1,
    kTrainRrsFull = 2,
    kTrainGiven = 3,
    kTrainGivenQ = 4  // as kTrainGiven, n_out 1, gradients given at q = softplus'(z)
};

struct TrainArgs {
    const float* params;  // weights of the network being trained
    float* m1;            // StatNet moments per slot (written by the StatNet pass)
    float* m2;
    const float* F;       // applied factor per depth
    const float* Fn;      // normalization factor without rate control per depth
    const float* E;       // pixel errors
    const float* Ebar;    // mean pixel error
    const float* ref;     // reference image [npix * 3] or null
    const int* k;         // training samples per pixel
    float eps, g1, g2, g3;
    float scale;          // factor on every sample's gradient (1/N for mean losses)
    const float* gin;     // kTrainGiven: output gradients [n][n_out]
    const float2* grid;   // the trained network's hash grid (StatNet on the encodings of
                          // Sec. 4, or RRSNet on the AID-NRRS inputs), else NULL
    float* dx;            // with grid: gradient at the 16 grid features per training slot
    float lambda;         // Box-Cox lambda of the AID-NRRS inputs
};

int train_tile();
void launch_reverse(const RecordView& r, int d, int D, const long long* live, int grid,
                    cudaStream_t s);
void launch_pixel_error(const RecordView& r, int spp, long long npix, const float* ref, float eps,
                        float* V, float* E, cudaStream_t s);
void launch_count_samples(const RecordView& r, const TrainBatch& b, int* k, int grid,
                          cudaStream_t s);

// E_acc = temporal EMA of E_cur; E_out = (2r+1)^2 filter of E_acc, guided by the pixel
// normals when nrm is not NULL (copy when r = 0)
void launch_error_smoothing(const float* E_cur, float* E_acc, float* E_out, int W, int H,
                            float alpha, int first, int radius, const float4* nrm, float power,
                            cudaStream_t s);
// The spatial filter alone (nrrs_error_filter).
void launch_error_filter(const float* in, const float4* nrm, int W, int H, int radius,
                         float power, float* out, cudaStream_t s);
// Per pixel: the normalised mean shading normal of its depth-1 vertices that went on
// (q > 0), w = 1; w = 0 when none did.
void launch_pixel_normals(const RecordView& r, int spp, long long npix, float4* nrm,
                          cudaStream_t s);
void launch_ref_fold(float* ref, const float* rgb, long long n3, int count, cudaStream_t s);
void launch_relmse(const float* img, const float* ref, long long n3, double eps, double* out,
                   cudaStream_t s);
// out[0] = sum E (L_min), out[1] = sum (E - Ebar)^2 (L_avg), *nsamples = sum k; part
// [3 G] and kpart [G] are scratch
void launch_pixel_terms(const float* E, long long n, const int* k, float* part,
                        long long* kpart, int G, float* Ebar, float* out, long long* nsamples,
                        cudaStream_t s);
cudaError_t launch_mlp_train(int which, const TrainArgs& a, const RecordView& r,
                             const TrainBatch& b, int grid, float* part, float* loss_part,
                             cudaStream_t s);
cudaError_t launch_mlp_grad_given(int n_out, bool at_q, const TrainArgs& a, const RecordView& r,
                                  const TrainBatch& b, int grid, float* part, float* loss_part,
                                  cudaStream_t s, int n_in = 16);
// StatNet's encoded inputs [n][32] of vertex features [n][16] and roughness [n].
void launch_statnet_inputs(const float4* feat, const float* rough, long long n,
                           const float2* table, float* out, cudaStream_t s);
// Adds to grad the hash-grid gradient of rows with features [n][16] and grid-feature
// gradients dx [n][16].
void launch_grid_backward(const float4* feat, const float* dx, long long n, float* grad,
                          cudaStream_t s);
void launch_reduce_grad(const float* part, int G, int P, float* grad, cudaStream_t s);
// Adds every training slot's grid-feature gradient (TrainArgs::dx) to the hash grid's
// entries (atomics; the order of the additions varies from run to run).
void launch_grid_scatter(const TrainArgs& a, const RecordView& r, const TrainBatch& b, int grid,
                         float* grad, cudaStream_t s);
void launch_reduce_loss(const float* part, int G, float* out, cudaStream_t s);
void launch_adam(float* P, const float* G, float* m, float* v, int n, int step, float lr,
                 float b1, float b2, float eps, int* bad, cudaStream_t s);
void launch_ema(float* E, const float* P, int n, float decay, cudaStream_t s);
void launch_rrsnet_dloss(const float* q_nrrs, const float* F, const float* Fn, const float* t,
                         const int* pixel, const float* m1, const float* m2, const float* E,
                         float Ebar, const float* Iref, const int* k, long long n,
                         float eps, float g1, float g2, float g3, float* dq, cudaStream_t s);

}  // namespace nrrs
