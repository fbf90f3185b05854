// Online training of RRSNet and StatNet on the GPU (Sec. 3.2 "Loss Design", Sec. 4
// "Training"): the reverse pass over a recorded frame, pixel errors, one persistent
// forward + backward kernel for both networks, the reduction of per-block gradients,
// Adam and the EMA of the weights.
#include <cfloat>

#include "grid.cuh"
#include "train.cuh"

namespace nrrs {

namespace {

constexpr int kTile = 128;  // samples per block tile of the training kernel

__device__ __forceinline__ uint32_t fb(float f) { return __float_as_uint(f); }

// Compensated (Kahan) sum in FP32: the running error of the additions is carried in c.
struct KahanSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s - c; }
};

// Count, mean and sum of squared deviations of a set of values (Welford), merged with
// Chan et al.'s pairwise rule, in FP32: the sum of squared deviations is accumulated
// directly, never as the difference sum x^2 - n mean^2.
struct Moments {
    float n = 0.0f, mean = 0.0f, m2 = 0.0f;
    __device__ __forceinline__ void add(float x) {
        n += 1.0f;
        const float d = x - mean;
        mean += d / n;
        m2 += d * (x - mean);
    }
    __device__ __forceinline__ void merge(const Moments& b) {
        const float nn = n + b.n;
        if (b.n == 0.0f) return;
        if (n == 0.0f) { *this = b; return; }
        const float d = b.mean - mean;
        const float f = b.n / nn;
        mean += d * f;
        m2 += b.m2 + d * d * n * f;
        n = nn;
    }
};

// Block-wide merge of per-thread moments in a fixed order (lane i takes lane i + o,
// then warp 0 merges the warp results); thread 0 returns the result.
__device__ Moments block_merge(Moments v, float* sh /* 3 * 32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Moments u;
        u.n = __shfl_down_sync(0xffffffffu, v.n, o);
        u.mean = __shfl_down_sync(0xffffffffu, v.mean, o);
        u.m2 = __shfl_down_sync(0xffffffffu, v.m2, o);
        if ((lane & (2 * o - 1)) == 0 && lane + o < 32) v.merge(u);
    }
    __syncthreads();
    if (lane == 0) {
        sh[3 * wid] = v.n;
        sh[3 * wid + 1] = v.mean;
        sh[3 * wid + 2] = v.m2;
    }
    __syncthreads();
    Moments r;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) {
            Moments u;
            u.n = sh[3 * w];
            u.mean = sh[3 * w + 1];
            u.m2 = sh[3 * w + 2];
            r.merge(u);
        }
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ reverse pass
// Suffix sums of depth d: S = own deposit + sum of the children's S (children of slot i
// are the slots [first_i, first_i + X_i) of depth d+1 that fit in the queue).  S / t is
// the vertex's estimate of outgoing radiance.
__global__ void k_reverse(RecordView r, int d, int D, const long long* live) {
    const long long n = live[d - 1];
    const long long nn = d < D ? live[d] : 0;
    const size_t base = (size_t)(d - 1) * r.C, nbase = (size_t)d * r.C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 dep = r.dep[base + i];
        float sx = dep.x, sy = dep.y, sz = dep.z;
        if (d < D) {
            const long long first = r.first[base + i];
            const long long last = first + r.X[base + i];
            for (long long j = first; j < last && j < nn; ++j) {
                const float4 c = r.S[nbase + j];
                sx += c.x; sy += c.y; sz += c.z;
            }
        }
        r.S[base + i] = make_float4(sx, sy, sz, dep.w);
    }
}

// Per pixel: V = unbiased variance over the spp primary samples of their suffix sums,
// divided by spp (the variance of the pixel estimate), mean over RGB; E = V / (I^2 + eps)
// with I the mean over RGB of the reference (Eq. loss-function_min).  Samples of pixel p
// are the depth-1 slots p*spp .. p*spp+spp-1.
__global__ void k_pixel_error(RecordView r, int spp, long long npix, const float* ref, float eps,
                              float* V, float* E) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    // two passes per channel in FP32: the mean, then the squared deviations from it
    float v = 0.0f;
    for (int c = 0; c < 3; ++c) {
        KahanSum m;
        for (int s = 0; s < spp; ++s) {
            const float4 S = r.S[p * spp + s];
            m.add(c == 0 ? S.x : c == 1 ? S.y : S.z);
        }
        const float mean = m.value() / (float)spp;
        KahanSum q;
        for (int s = 0; s < spp; ++s) {
            const float4 S = r.S[p * spp + s];
            const float dd = (c == 0 ? S.x : c == 1 ? S.y : S.z) - mean;
            q.add(dd * dd);
        }
        v += spp > 1 ? q.value() / (float)(spp - 1) / (float)spp : 0.0f;
    }
    v *= 1.0f / 3.0f;
    V[p] = v;
    const float I = ref ? (ref[3 * p] + ref[3 * p + 1] + ref[3 * p + 2]) * (1.0f / 3.0f) : 0.0f;
    E[p] = v / (I * I + eps);
}

// Temporal smoothing of the error map (Sec. 4 "Tackle Low Spp", Eq. error_temporal with
// alpha_mix): E_acc = (1 - alpha) E_acc + alpha E_cur (E_acc = E_cur on the first frame).
__global__ void k_error_temporal(const float* E_cur, float* E_acc, long long n, float alpha,
                                 int first) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    E_acc[p] = first ? E_cur[p] : (1.0f - alpha) * E_acc[p] + alpha * E_cur[p];
}

// Spatial smoothing of the error map (stands in for the denoiser the paper applies to
// the error map, Sec. 4 "Tackle Low Spp", which is guided by the normal buffer): the
// weighted mean over the (2r+1)^2 window clipped at the image border.  Without normals
// every weight is 1 (a box filter).  With normals, a pixel that has one weighs a
// neighbour with a normal by max(0, n_p . n_q)^power and one without by 0; a pixel
// without a normal weighs every neighbour by 1.  The centre always has weight 1.
// An integral power (ipow >= 0) is raised by repeated squaring, others by powf; the
// window's sums are compensated FP32 sums.
__device__ __forceinline__ float pow_by_squaring(float b, int n) {
    float r = 1.0f;
    for (; n > 0; n >>= 1) {
        if (n & 1) r *= b;
        b *= b;
    }
    return r;
}

__global__ void k_error_filter(const float* in, const float4* nrm, int W, int H, int r,
                               float power, int ipow, float* out) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)W * H) return;
    const int x = (int)(p % W), y = (int)(p / W);
    const float4 np = nrm ? nrm[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool guided = nrm && np.w > 0.0f;
    KahanSum s, c;
    for (int yy = max(0, y - r); yy <= min(H - 1, y + r); ++yy)
        for (int xx = max(0, x - r); xx <= min(W - 1, x + r); ++xx) {
            const long long q = (long long)yy * W + xx;
            float wq = 1.0f;
            if (guided && q != p) {
                const float4 nq = nrm[q];
                const float d = np.x * nq.x + np.y * nq.y + np.z * nq.z;
                wq = !(nq.w > 0.0f && d > 0.0f) ? 0.0f
                     : ipow >= 0                   ? pow_by_squaring(d, ipow)
                                                   : powf(d, power);
            }
            s.add(wq * in[q]);
            c.add(wq);
        }
    out[p] = s.value() / c.value();
}

__global__ void k_pixel_normals(RecordView r, int spp, long long npix, float4* nrm) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    int k = 0;
    for (int s = 0; s < spp; ++s) {
        const long long i = p * spp + s;
        if (!(r.q[i] > 0.0f)) continue;  // no vertex went on: no features were written
        const float4 f1 = r.feat[4 * i + 1], f2 = r.feat[4 * i + 2];
        nx += f1.z;
        ny += f1.w;
        nz += f2.x;
        ++k;
    }
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    nrm[p] = k > 0 && len > 0.0f ? make_float4(nx / len, ny / len, nz / len, 1.0f)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Folds the frame into the running mean of the frames so far.
__global__ void k_ref_fold(float* ref, const float* rgb, long long n3, int count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const float k = (float)count;
    ref[i] = (ref[i] * k + rgb[i]) / (k + 1.0f);
}

// k_i: trainable samples (recorded q_orig > 0 at a network depth) of every pixel.
__global__ void k_count_samples(RecordView r, TrainBatch b, int* k) {
    for (long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x; slot < b.batch;
         slot += (long long)gridDim.x * blockDim.x) {
        const long long u = batch_vertex(b, slot);
        int d = 0;
        while (d + 1 < b.D && b.offset[d + 1] <= u) ++d;
        if (!((b.net_mask >> d) & 1u)) continue;
        const long long i = u - b.offset[d];
        const size_t g = (size_t)d * r.C + i;
        if (r.q[g] > 0.0f) atomicAdd(&k[fb(r.dep[g].w)], 1);
    }
}

// Pixel-error terms, two fixed-order passes in FP32: per block (one contiguous chunk
// of pixels) the count, mean and sum of squared deviations of E (Welford per thread,
// Chan's merge across threads) and the exact integer sum of k; then one block merges
// the blocks in order into Ebar = mean E, L_min = sum_i E_i = n Ebar and
// L_avg = sum_i (E_i - Ebar)^2 (Eq. loss-function_min / _avg), and N = sum_i k_i, the
// training samples.
__global__ void k_pixel_partial(const float* E, long long n, const int* k, float* part,
                                long long* kpart) {
    __shared__ float sh[96];
    __shared__ long long shk[32];
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    Moments m;
    long long c = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        m.add(E[i]);
        c += k[i];
    }
    m = block_merge(m, sh);
    c = block_sum(c, shk);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = m.n;
        part[3 * blockIdx.x + 1] = m.mean;
        part[3 * blockIdx.x + 2] = m.m2;
        kpart[blockIdx.x] = c;
    }
}

__global__ void k_pixel_final(const float* part, const long long* kpart, int G, float* Ebar,
                              float* out, long long* nsamples) {
    __shared__ float sh[96];
    __shared__ long long shk[32];
    Moments m;
    long long c = 0;
    // each thread merges a contiguous run of blocks, so the order stays the blocks'
    const int per = (G + blockDim.x - 1) / blockDim.x;
    for (int g = threadIdx.x * per; g < (int)(threadIdx.x + 1) * per && g < G; ++g) {
        Moments u;
        u.n = part[3 * g + 0];
        u.mean = part[3 * g + 1];
        u.m2 = part[3 * g + 2];
        m.merge(u);
        c += kpart[g];
    }
    m = block_merge(m, sh);
    c = block_sum(c, shk);
    if (threadIdx.x == 0) {
        *Ebar = m.mean;
        out[0] = m.mean * m.n;
        out[1] = m.m2 > 0.0f ? m.m2 : 0.0f;
        *nsamples = c;
    }
}

// relMSE = mean over pixels and channels of (I - R)^2 / (R^2 + eps), fixed order:
// compensated FP32 sums per thread, then the block's sum.
__global__ void k_relmse(const float* img, const float* ref, long long n3, float eps,
                         double* out) {
    __shared__ float sh[32];
    KahanSum k;
    for (long long i = threadIdx.x; i < n3; i += blockDim.x) {
        const float d = img[i] - ref[i];
        k.add(d * d / (ref[i] * ref[i] + eps));
    }
    const float s = block_sum(k.value(), sh);
    if (threadIdx.x == 0) *out = n3 > 0 ? (double)(s / (float)n3) : 0.0;
}

// ------------------------------------------------------------------ MLP training
// Shared-memory layout of one tile (kTile samples): inputs X[kTile][KIN], hidden
// activations A1..A3[kTile][32] (post Leaky ReLU; their sign is the sign of the
// pre-activation), output gradients G[kTile][8], then the weights.  Each sample's row
// is padded by one float: with 32-float rows the warp's 32 samples would store into the
// same bank (32-way conflicts); with 33 every lane has its own.
template <int KIN>
struct TrainSmem {
    float X[kTile][KIN + 1];
    float A[3][kTile][kNH + 1];
    float G[kTile][9];
};

__device__ __forceinline__ float lrelu(float a) { return a > 0.0f ? a : kLeak * a; }

// Loss gradient of one sample at the network outputs; returns false for a sample that
// does not train.  `out` holds the raw outputs (RRSNet: pre-activation z).
template <int MODE>
__device__ __forceinline__ bool sample_grad(const TrainArgs& a, const RecordView& r, int d,
                                            long long i, const float* out, float* gout,
                                            KahanSum* loss) {
    const size_t g = (size_t)d * r.C + i;
    const float4 dep = r.dep[g];
    const float4 t = r.t[g];
    if (MODE == kTrainStatNet) {
        // targets: one-sample reflected radiance <L> = (S - deposit) / t per channel and <L>^2
        const float4 S = r.S[g];
        const float tt[3] = {t.x, t.y, t.z};
        const float ss[3] = {S.x - dep.x, S.y - dep.y, S.z - dep.z};
        for (int c = 0; c < 3; ++c) {
            const float L = tt[c] > 0.0f ? ss[c] / tt[c] : 0.0f;
            const float L2 = L * L;
            // relative L2 normalised by the (stop-gradient) prediction
            const float w1 = 1.0f / (out[c] * out[c] + a.eps);
            const float w2 = 1.0f / (out[3 + c] * out[3 + c] + a.eps);
            const float d1 = out[c] - L, d2 = out[3 + c] - L2;
            gout[c] = 2.0f * d1 * w1 * a.scale;
            gout[3 + c] = 2.0f * d2 * w2 * a.scale;
            loss->add(d1 * d1 * w1 + d2 * d2 * w2);
        }
        return true;
    }
    // RRSNet: q_nrrs = softplus'(z)
    const float z = out[0];
    const float q = z < 0.0f ? log1pf(expf(z)) : fmaf(0.5f, z, 0.693147180559945f);
    const float dqdz = z < 0.0f ? 1.0f / (1.0f + expf(-z)) : 0.5f;
    float dq;
    if (MODE == kTrainRrsWarmup) {
        // Sec. 4 "Training" step (1): regress to 1 with the relative L2 loss
        dq = 2.0f * (q - 1.0f) / (1.0f + a.eps);
        loss->add((q - 1.0f) * (q - 1.0f) / (1.0f + a.eps));
    } else {
        const float F = a.F[d], Fn = a.Fn[d];
        const float qu = F * r.q[g];  // factor the frame actually used
        const float tm = (t.x + t.y + t.z) * (1.0f / 3.0f);
        const float m1 = a.m1[g], m2 = a.m2[g];
        const float VH = fmaxf(m2 - m1 * m1, 0.0f);
        const float H = qu < 1.0f ? m2 : VH;  // Eq. gradient_transfer_rr_mc / splitting_mc
        const float dV = -tm * tm * H / (qu * qu);
        const uint32_t pix = fb(dep.w);
        const float I = a.ref ? (a.ref[3 * pix] + a.ref[3 * pix + 1] + a.ref[3 * pix + 2]) *
                                    (1.0f / 3.0f)
                              : 0.0f;
        const float dLdE = a.g1 * 2.0f * (a.E[pix] - *a.Ebar) + a.g2;
        const float dLdV = dLdE / (I * I + a.eps) / (float)max(a.k[pix], 1);
        const float qn = Fn * q;  // stop-gradient target of L_rrs
        dq = dLdV * dV * F + a.g3 * 2.0f * (q - qn);
        loss->add((q - qn) * (q - qn));
    }
    gout[0] = dq * dqdz * a.scale;
    return true;
}

// Weight-gradient ownership (register blocking): thread t owns row j = t / 4 of the
// gradients of W1, W2 and W3, columns [KIN/4 (t % 4), +KIN/4) of W1 and [8 (t % 4), +8) of
// W2 and W3, and entries t and t + kTile of W4.  Per sample it reads delta[j] once (shared
// by the row's 4 threads) and its inputs with 128-bit loads.
// KIN = 32: StatNet on the encodings of Sec. 4 (hash grid of the position, one-blob w_o
// and roughness), which also writes the gradient at its 16 grid features per slot.
template <int NOUT, int MODE, int KIN = kNF>
__global__ void __launch_bounds__(kTile, KIN == kNF ? 3 : 2)  // 32 inputs: 2 tiles fit in smem
k_mlp_train(TrainArgs a, RecordView r, TrainBatch b, float* part, float* loss_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem<KIN>& sm = *reinterpret_cast<TrainSmem<KIN>*>(smem_raw);
    float* W = reinterpret_cast<float*>(smem_raw + sizeof(TrainSmem<KIN>));
    constexpr int P = kNH * KIN + 2 * kNH * kNH + NOUT * kNH;
    constexpr int C1 = KIN / 4;  // W1 gradient columns per thread
    for (int p = threadIdx.x; p < P; p += blockDim.x) W[p] = a.params[p];
    const float* W1 = W;
    const float* W2 = W + kNH * KIN;
    const float* W3 = W2 + kNH * kNH;
    const float* W4 = W3 + kNH * kNH;
    const int tid = threadIdx.x;
    const int gj = tid >> 2, gq = tid & 3;
    float g1[C1], g2[8], g3[8], g4[2];
#pragma unroll
    for (int e = 0; e < C1; ++e) g1[e] = 0.0f;
#pragma unroll
    for (int e = 0; e < 8; ++e) g2[e] = g3[e] = 0.0f;
    g4[0] = g4[1] = 0.0f;
    KahanSum loss;
    const long long tiles = (b.batch + kTile - 1) / kTile;
    __syncthreads();
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long slot = tile * kTile + tid;
        // recorded vertex of this training slot (given rows: the slot itself)
        const long long u = MODE == kTrainGiven || MODE == kTrainGivenQ ? slot
                            : slot < b.batch ? batch_vertex(b, slot) : b.total;
        // ---- forward of this thread's sample
        float x[KIN];
        bool active = false;
        int d = 0;
        long long i = 0;
        if ((MODE == kTrainGiven || MODE == kTrainGivenQ) && u < b.total) {
            active = true;
            const float4* f = r.feat + (KIN / 4) * u;
#pragma unroll
            for (int k = 0; k < KIN / 4; ++k) {
                const float4 v = f[k];
                x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
            }
        } else if (u < b.total) {
            while (d + 1 < b.D && b.offset[d + 1] <= u) ++d;
            i = u - b.offset[d];
            const size_t g = (size_t)d * r.C + i;
            active = ((b.net_mask >> d) & 1u) && r.q[g] > 0.0f;
            if (active && KIN == kStatGridIn && MODE == kTrainStatNet) {
                // StatNet's encoded inputs: position and w_o from the vertex features
                const float4 f0 = r.feat[4 * g], f1 = r.feat[4 * g + 1];
                statnet_grid_inputs(a.grid, f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, r.rough[g], x);
            } else if (active && KIN == kAidIn) {
                // AID-NRRS inputs of RRSNet: its grid, w_o, throughput, pixel estimate
                const float4 f0 = r.feat[4 * g], f1 = r.feat[4 * g + 1], tt = r.t[g];
                const uint32_t pix = fb(r.dep[g].w);
                const float I = a.ref ? (a.ref[3 * pix] + a.ref[3 * pix + 1] + a.ref[3 * pix + 2]) *
                                            (1.0f / 3.0f)
                                      : 0.0f;
                aid_inputs(a.grid, f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, tt.x, tt.y, tt.z, I,
                           r.rough[g], a.lambda, x);
            } else if (active) {
                // StatNet learns from the vertex features; RRSNet reads its own inputs
                // (the NRRS encoding, when the scene uses it)
                const float4* f =
                    (MODE != kTrainStatNet && r.feat_net ? r.feat_net : r.feat) + 4 * g;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 v = f[k];
                    x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
                }
                if (MODE == kTrainStatNet) x[13] = x[14] = x[15] = 0.0f;  // no throughput
            }
        }
        if (!active) {
#pragma unroll
            for (int k = 0; k < KIN; ++k) x[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < KIN; ++k) sm.X[tid][k] = x[k];
        float h[kNH], hn[kNH];
#pragma unroll
        for (int j = 0; j < kNH; ++j) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < KIN; ++k) s = fmaf(W1[j * KIN + k], x[k], s);
            h[j] = lrelu(s);
            sm.A[0][tid][j] = h[j];
        }
#pragma unroll
        for (int j = 0; j < kNH; ++j) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < kNH; ++k) s = fmaf(W2[j * kNH + k], h[k], s);
            hn[j] = lrelu(s);
            sm.A[1][tid][j] = hn[j];
        }
#pragma unroll
        for (int j = 0; j < kNH; ++j) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < kNH; ++k) s = fmaf(W3[j * kNH + k], hn[k], s);
            h[j] = lrelu(s);
            sm.A[2][tid][j] = h[j];
        }
        float out[NOUT], gout[8];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < kNH; ++k) s = fmaf(W4[o * kNH + k], h[k], s);
            out[o] = s;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) gout[o] = 0.0f;
        if (MODE == kTrainGiven) {
            if (active)
#pragma unroll
                for (int o = 0; o < NOUT; ++o) gout[o] = a.gin[u * NOUT + o];
        } else if (MODE == kTrainGivenQ) {
            // chain dL/dq through Eq. rrsnet_activation: dq/dz = sigmoid(z) (z < 0), 1/2
            const float z = out[0];
            if (active) gout[0] = a.gin[u] * (z < 0.0f ? 1.0f / (1.0f + expf(-z)) : 0.5f);
        } else if (active) {
            if (MODE == kTrainStatNet && a.m1) {  // moments for the RRSNet gradient
                const size_t g = (size_t)d * r.C + i;
                a.m1[g] = (out[0] + out[1] + out[2]) * (1.0f / 3.0f);
                a.m2[g] = (out[3] + out[4] + out[5]) * (1.0f / 3.0f);
            }
            sample_grad<MODE>(a, r, d, i, out, gout, &loss);
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) sm.G[tid][o] = gout[o];
        // this sample's delta at layer 3: (W4^T g) * lrelu'(a3)
        float dl[kNH];
#pragma unroll
        for (int k = 0; k < kNH; ++k) {
            float s = 0.0f;
#pragma unroll
            for (int o = 0; o < NOUT; ++o) s = fmaf(W4[o * kNH + k], gout[o], s);
            dl[k] = s * (h[k] > 0.0f ? 1.0f : kLeak);
        }
        __syncthreads();
        // ---- W4 gradients: sum_s G[s][o] A3[s][k]
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int p = tid + e * kTile;
            if (p < NOUT * kNH) {
                const int o = p / kNH, k = p % kNH;
                float sacc = 0.0f;
                for (int q = 0; q < kTile; ++q) sacc = fmaf(sm.G[q][o], sm.A[2][q][k], sacc);
                g4[e] += sacc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kNH; ++k) sm.A[2][tid][k] = dl[k];  // A3 now holds delta3
        __syncthreads();
        // ---- W3 gradients: sum_s delta3[s][j] A2[s][k]
        for (int q = 0; q < kTile; ++q) {
            const float dj = sm.A[2][q][gj];
            const float* ar = &sm.A[1][q][8 * gq];  // padded rows: no 16-byte loads
#pragma unroll
            for (int e = 0; e < 8; ++e) g3[e] = fmaf(dj, ar[e], g3[e]);
        }
        // delta2 = (W3^T delta3) * lrelu'(a2)
#pragma unroll
        for (int k = 0; k < kNH; ++k) {
            float sacc = 0.0f;
#pragma unroll
            for (int j = 0; j < kNH; ++j) sacc = fmaf(W3[j * kNH + k], dl[j], sacc);
            h[k] = sacc * (hn[k] > 0.0f ? 1.0f : kLeak);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kNH; ++k) sm.A[1][tid][k] = h[k];  // A2 now holds delta2
        __syncthreads();
        // ---- W2 gradients: sum_s delta2[s][j] A1[s][k]
        for (int q = 0; q < kTile; ++q) {
            const float dj = sm.A[1][q][gj];
            const float* ar = &sm.A[0][q][8 * gq];  // padded rows: no 16-byte loads
#pragma unroll
            for (int e = 0; e < 8; ++e) g2[e] = fmaf(dj, ar[e], g2[e]);
        }
        // delta1 = (W2^T delta2) * lrelu'(a1); a1 is still in A1 for this thread
#pragma unroll
        for (int k = 0; k < kNH; ++k) {
            float sacc = 0.0f;
#pragma unroll
            for (int j = 0; j < kNH; ++j) sacc = fmaf(W2[j * kNH + k], h[j], sacc);
            dl[k] = sacc * (sm.A[0][tid][k] > 0.0f ? 1.0f : kLeak);
        }
        if (KIN == 32 && a.dx && slot < b.batch) {
            // gradient at the 16 grid features: W1^T delta1 (zero for a sample that does
            // not train); the grid's entries receive it in k_grid_scatter
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float sacc = 0.0f;
#pragma unroll
                for (int j = 0; j < kNH; ++j) sacc = fmaf(W1[j * KIN + c], dl[j], sacc);
                a.dx[slot * 16 + c] = sacc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kNH; ++k) sm.A[0][tid][k] = dl[k];  // A1 now holds delta1
        __syncthreads();
        // ---- W1 gradients: sum_s delta1[s][j] X[s][k]
        for (int q = 0; q < kTile; ++q) {
            const float dj = sm.A[0][q][gj];
            const float* xr = &sm.X[q][C1 * gq];
#pragma unroll
            for (int c = 0; c < C1; ++c) g1[c] = fmaf(dj, xr[c], g1[c]);
        }
        __syncthreads();
    }
    float* pb = part + (size_t)blockIdx.x * P;
#pragma unroll
    for (int e = 0; e < C1; ++e) pb[gj * KIN + C1 * gq + e] = g1[e];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        pb[kNH * KIN + gj * kNH + 8 * gq + e] = g2[e];
        pb[kNH * KIN + kNH * kNH + gj * kNH + 8 * gq + e] = g3[e];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int p = tid + e * kTile;
        if (p < NOUT * kNH) pb[kNH * KIN + 2 * kNH * kNH + p] = g4[e];
    }
    __shared__ float shl[32];
    const float lsum = block_sum(loss.value(), shl);
    if (tid == 0) loss_part[blockIdx.x] = lsum;
}

// Sum of the per-block gradients in block order (deterministic).
__global__ void k_reduce_grad(const float* part, int G, int P, float* grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float s = 0.0f;
    for (int b = 0; b < G; ++b) s += part[(size_t)b * P + p];
    grad[p] = s;
}

__global__ void k_reduce_loss(const float* part, int G, float* out) {
    __shared__ float sh[32];
    KahanSum k;
    for (int b = threadIdx.x; b < G; b += blockDim.x) k.add(part[b]);
    const float s = block_sum(k.value(), sh);
    if (threadIdx.x == 0) *out = s;
}

// Adam (Kingma & Ba): bias-corrected first and second moments; non-finite gradients
// set *bad and leave the weights untouched.
__global__ void k_adam(float* P, const float* G, float* m, float* v, int n, int step, float lr,
                       float b1, float b2, float eps, int* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    if (!(fabsf(g) <= FLT_MAX)) {
        if (bad) atomicOr(bad, 1);
        return;
    }
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_ema(float* E, const float* P, int n, float decay) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[i] = decay * E[i] + (1.0f - decay) * P[i];
}

// Stand-alone loss gradient on plain arrays (for parity tests): one thread per sample.
__global__ void k_rrsnet_dloss(const float* q_nrrs, const float* F, const float* Fn,
                               const float* t, const int* pixel, const float* m1, const float* m2,
                               const float* E, float Ebar, const float* Iref,
                               const int* k, long long n, float eps, float g1, float g2,
                               float g3, float* dq) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = pixel[s];
    const float qu = F[s] * q_nrrs[s];
    const float VH = fmaxf(m2[s] - m1[s] * m1[s], 0.0f);
    const float H = qu < 1.0f ? m2[s] : VH;
    const float dV = -t[s] * t[s] * H / (qu * qu);
    const float dLdE = g1 * 2.0f * (E[i] - Ebar) + g2;
    const float dLdV = dLdE / (Iref[i] * Iref[i] + eps) / (float)max(k[i], 1);
    dq[s] = dLdV * dV * F[s] + g3 * 2.0f * (q_nrrs[s] - Fn[s] * q_nrrs[s]);
}

template <int NOUT, int MODE, int KIN = kNF>
size_t train_smem() {
    return sizeof(TrainSmem<KIN>) + sizeof(float) * (kNH * KIN + 2 * kNH * kNH + NOUT * kNH);
}

template <int NOUT, int MODE, int KIN = kNF>
cudaError_t launch_train_t(const TrainArgs& a, const RecordView& r, const TrainBatch& b, int grid,
                           float* part, float* loss_part, cudaStream_t s) {
    const size_t smem = train_smem<NOUT, MODE, KIN>();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train<NOUT, MODE, KIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_train<NOUT, MODE, KIN><<<grid, kTile, smem, s>>>(a, r, b, part, loss_part);
    return cudaGetLastError();
}

// The hash grid's gradient: every training slot adds its grid-feature gradient (from the
// StatNet pass) to the 8 corner entries of its position's cell on every level.
__global__ void k_grid_scatter(TrainArgs a, RecordView r, TrainBatch b, float* grad) {
    for (long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x; slot < b.batch;
         slot += (long long)gridDim.x * blockDim.x) {
        float dx[16];
        bool any = false;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            dx[c] = a.dx[slot * 16 + c];
            any = any || dx[c] != 0.0f;
        }
        if (!any) continue;
        const long long u = batch_vertex(b, slot);
        int d = 0;
        while (d + 1 < b.D && b.offset[d + 1] <= u) ++d;
        const size_t g = (size_t)d * r.C + (u - b.offset[d]);
        const float4 f0 = r.feat[4 * g];
        grid_scatter(grad, f0.x, f0.y, f0.z, dx);
    }
}

}  // namespace

int train_tile() { return kTile; }

void launch_reverse(const RecordView& r, int d, int D, const long long* live, int grid,
                    cudaStream_t s) {
    k_reverse<<<grid, 256, 0, s>>>(r, d, D, live);
}

void launch_pixel_error(const RecordView& r, int spp, long long npix, const float* ref, float eps,
                        float* V, float* E, cudaStream_t s) {
    k_pixel_error<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(r, spp, npix, ref, eps, V, E);
}

void launch_count_samples(const RecordView& r, const TrainBatch& b, int* k, int grid,
                          cudaStream_t s) {
    k_count_samples<<<grid, 256, 0, s>>>(r, b, k);
}


void launch_relmse(const float* img, const float* ref, long long n3, double eps, double* out,
                   cudaStream_t s) {
    k_relmse<<<1, 1024, 0, s>>>(img, ref, n3, (float)eps, out);
}

// power as an exponent for repeated squaring, or -1 when it is not a small integer
static int integral_power(float power) {
    return power >= 0.0f && power <= 1024.0f && power == floorf(power) ? (int)power : -1;
}

void launch_error_smoothing(const float* E_cur, float* E_acc, float* E_out, int W, int H,
                            float alpha, int first, int radius, const float4* nrm, float power,
                            cudaStream_t s) {
    const long long n = (long long)W * H;
    const unsigned g = (unsigned)((n + 255) / 256);
    k_error_temporal<<<g, 256, 0, s>>>(E_cur, E_acc, n, alpha, first);
    if (radius > 0)
        k_error_filter<<<g, 256, 0, s>>>(E_acc, nrm, W, H, radius, power, integral_power(power),
                                         E_out);
    else
        cudaMemcpyAsync(E_out, E_acc, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
}

void launch_error_filter(const float* in, const float4* nrm, int W, int H, int radius,
                         float power, float* out, cudaStream_t s) {
    const long long n = (long long)W * H;
    k_error_filter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, nrm, W, H, radius, power,
                                                               integral_power(power), out);
}

void launch_pixel_normals(const RecordView& r, int spp, long long npix, float4* nrm,
                          cudaStream_t s) {
    k_pixel_normals<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(r, spp, npix, nrm);
}

void launch_ref_fold(float* ref, const float* rgb, long long n3, int count, cudaStream_t s) {
    k_ref_fold<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(ref, rgb, n3, count);
}

void launch_pixel_terms(const float* E, long long n, const int* k, float* part,
                        long long* kpart, int G, float* Ebar, float* out, long long* nsamples,
                        cudaStream_t s) {
    k_pixel_partial<<<G, 256, 0, s>>>(E, n, k, part, kpart);
    k_pixel_final<<<1, 256, 0, s>>>(part, kpart, G, Ebar, out, nsamples);
}

cudaError_t launch_mlp_train(int which, const TrainArgs& a, const RecordView& r,
                             const TrainBatch& b, int grid, float* part, float* loss_part,
                             cudaStream_t s) {
    switch (which) {
        case kTrainStatNet:
            if (a.grid)
                return launch_train_t<6, kTrainStatNet, kStatGridIn>(a, r, b, grid, part,
                                                                     loss_part, s);
            return launch_train_t<6, kTrainStatNet>(a, r, b, grid, part, loss_part, s);
        case kTrainRrsWarmup:
            if (a.grid)
                return launch_train_t<1, kTrainRrsWarmup, kAidIn>(a, r, b, grid, part, loss_part, s);
            return launch_train_t<1, kTrainRrsWarmup>(a, r, b, grid, part, loss_part, s);
        default:
            if (a.grid)
                return launch_train_t<1, kTrainRrsFull, kAidIn>(a, r, b, grid, part, loss_part, s);
            return launch_train_t<1, kTrainRrsFull>(a, r, b, grid, part, loss_part, s);
    }
}

cudaError_t launch_mlp_grad_given(int n_out, bool at_q, const TrainArgs& a, const RecordView& r,
                                  const TrainBatch& b, int grid, float* part, float* loss_part,
                                  cudaStream_t s, int n_in) {
    if (n_in == kStatGridIn)
        return launch_train_t<6, kTrainGiven, kStatGridIn>(a, r, b, grid, part, loss_part, s);
    if (at_q) return launch_train_t<1, kTrainGivenQ>(a, r, b, grid, part, loss_part, s);
    return n_out == 1 ? launch_train_t<1, kTrainGiven>(a, r, b, grid, part, loss_part, s)
                      : launch_train_t<6, kTrainGiven>(a, r, b, grid, part, loss_part, s);
}

void launch_grid_scatter(const TrainArgs& a, const RecordView& r, const TrainBatch& b, int grid,
                         float* grad, cudaStream_t s) {
    k_grid_scatter<<<grid, 256, 0, s>>>(a, r, b, grad);
}

namespace {
__global__ void k_statnet_inputs_rows(const float4* feat, const float* rough, long long n,
                                      const float2* table, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 f0 = feat[4 * i], f1 = feat[4 * i + 1];
    float x[kStatGridIn];
    statnet_grid_inputs(table, f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, rough[i], x);
#pragma unroll
    for (int k = 0; k < kStatGridIn; ++k) out[i * kStatGridIn + k] = x[k];
}

__global__ void k_grid_backward_rows(const float4* feat, const float* dx, long long n,
                                     float* grad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) d[c] = dx[i * 16 + c];
    const float4 f0 = feat[4 * i];
    grid_scatter(grad, f0.x, f0.y, f0.z, d);
}
}  // namespace

void launch_statnet_inputs(const float4* feat, const float* rough, long long n,
                           const float2* table, float* out, cudaStream_t s) {
    k_statnet_inputs_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(feat, rough, n, table, out);
}

void launch_grid_backward(const float4* feat, const float* dx, long long n, float* grad,
                          cudaStream_t s) {
    k_grid_backward_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(feat, dx, n, grad);
}

void launch_reduce_grad(const float* part, int G, int P, float* grad, cudaStream_t s) {
    k_reduce_grad<<<(P + 255) / 256, 256, 0, s>>>(part, G, P, grad);
}

void launch_reduce_loss(const float* part, int G, float* out, cudaStream_t s) {
    k_reduce_loss<<<1, 256, 0, s>>>(part, G, out);
}

void launch_adam(float* P, const float* G, float* m, float* v, int n, int step, float lr,
                 float b1, float b2, float eps, int* bad, cudaStream_t s) {
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(P, G, m, v, n, step, lr, b1, b2, eps, bad);
}

void launch_ema(float* E, const float* P, int n, float decay, cudaStream_t s) {
    k_ema<<<(n + 255) / 256, 256, 0, s>>>(E, P, n, decay);
}

void launch_rrsnet_dloss(const float* q_nrrs, const float* F, const float* Fn, const float* t,
                         const int* pixel, const float* m1, const float* m2, const float* E,
                         float Ebar, const float* Iref, const int* k, long long n,
                         float eps, float g1, float g2, float g3, float* dq, cudaStream_t s) {
    if (n <= 0) return;
    k_rrsnet_dloss<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q_nrrs, F, Fn, t, pixel, m1, m2, E,
                                                              Ebar, Iref, k, n, eps, g1, g2, g3, dq);
}

}  // namespace nrrs
