/*
 * NRRS oracle, training side: plain FP64 restatements of the pieces the GPU trains
 * RRSNet and StatNet with.  TEST INFRASTRUCTURE ONLY (see nrrs_oracle.c).
 *
 *   or_mlpn_forward / or_mlpn_backward
 *       A bias-free MLP 16 -> 32 -> 32 -> 32 -> n_out with Leaky ReLU (slope 0.01) after
 *       each hidden layer and no output activation (Sec. 4 "Network Architecture";
 *       StatNet has no output activation, Sec. 4 "Output & Activation").
 *   or_mlpk_forward / or_mlpk_backward
 *       The same network with n_in inputs (32 for StatNet on the encodings of Sec. 4
 *       "Input Encoding"); the backward pass also returns the gradient at the inputs,
 *       which the hash grid's entries receive.
 *   or_statnet_dloss
 *       Eq. loss-function_StatNet: relative L2 on the two predicted moments E[<L>] and
 *       E[<L>^2] (Sec. 4 "Output & Activation") against the one-sample targets <L> and
 *       <L>^2, per RGB channel, normalised by the stop-gradient PREDICTION:
 *       (a - b)^2 / (sg(a)^2 + eps).  (The printed equation puts sg() on b, the target,
 *       where it has no effect; the relative L2 it cites normalises by the prediction,
 *       whose gradient 2 (a - b) / (sg(a)^2 + eps) vanishes in expectation at a = E[b],
 *       so noisy one-sample targets do not pull the prediction towards zero.)
 *   or_pixel_error
 *       Eq. loss-function_min: E_i = V[<I_i>] / (I_i^2 + eps), V from the spp samples of
 *       the pixel, I_i the reference (Sec. 4 "Compromise": the accumulated earlier frames).
 *   or_rrsnet_dloss
 *       d L_RRSNet / d q_nrrs for L_RRSNet = g1 L_avg + g2 L_min + g3 L_rrs
 *       (Eq. loss-function_rrsnet, loss-function_avg, loss-function_min,
 *       loss-function_rrs), with dV/dq from Eq. gradient_transfer_rr_mc (q_used < 1) or
 *       Eq. gradient_transfer_splitting_mc (q_used >= 1), the pixel loss shared 1/k_i
 *       among the pixel's k_i training samples (Sec. 3.2), and q_used = F q_nrrs with F
 *       held constant.
 *   or_error_temporal, or_error_filter, or_pixel_normals
 *       Sec. 4 "Tackle Low Spp": the temporal EMA of the error map (alpha_mix), and the
 *       normal-guided spatial filter that stands in for the paper's denoiser, with the
 *       per-pixel first-hit normals that guide it.
 *   or_adam_step, or_ema
 *       Adam (Kingma & Ba) and the exponential moving average of the weights used for
 *       inference (Sec. 4 "Training").
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NF 16
#define NH 32
#define LEAK 0.01

#define NIN_MAX 32

static void layer_ptrs(const double* P, int n_in, const double* W[4]) {
    W[0] = P;
    W[1] = P + NH * n_in;
    W[2] = P + NH * n_in + NH * NH;
    W[3] = P + NH * n_in + 2 * NH * NH;
}

int64_t or_mlpn_param_count(int n_out) { return NH * NF + 2 * NH * NH + (int64_t)n_out * NH; }

int64_t or_mlpk_param_count(int n_in, int n_out) {
    return NH * (int64_t)n_in + 2 * NH * NH + (int64_t)n_out * NH;
}

void or_mlpk_forward(const double* P, int n_in, int n_out, const double* x, double* out,
                     double* pre, double* hid) {
    const double* W[4];
    layer_ptrs(P, n_in, W);
    double in[NIN_MAX > NH ? NIN_MAX : NH], h[NH];
    int nin = n_in;
    for (int k = 0; k < n_in; ++k) in[k] = x[k];
    for (int l = 0; l < 3; ++l) {
        for (int j = 0; j < NH; ++j) {
            double a = 0.0;
            for (int k = 0; k < nin; ++k) a += W[l][j * nin + k] * in[k];
            if (pre) pre[l * NH + j] = a;
            h[j] = a > 0.0 ? a : LEAK * a;
            if (hid) hid[l * NH + j] = h[j];
        }
        for (int j = 0; j < NH; ++j) in[j] = h[j];
        nin = NH;
    }
    for (int o = 0; o < n_out; ++o) {
        double a = 0.0;
        for (int k = 0; k < NH; ++k) a += W[3][o * NH + k] * in[k];
        out[o] = a;
    }
}

void or_mlpn_forward(const double* P, int n_out, const double* x, double* out, double* pre,
                     double* hid) {
    or_mlpk_forward(P, NF, n_out, x, out, pre, hid);
}

/* Accumulates into G the gradient of sum_o dout[o] * out[o] with respect to P; with
 * dx != NULL also writes its gradient with respect to the n_in inputs. */
void or_mlpk_backward(const double* P, int n_in, int n_out, const double* x, const double* dout,
                      double* G, double* dx) {
    double pre[3 * NH], hid[3 * NH], out[8];
    or_mlpk_forward(P, n_in, n_out, x, out, pre, hid);
    const double* W[4];
    layer_ptrs(P, n_in, W);
    double* GW[4] = {G, G + NH * n_in, G + NH * n_in + NH * NH, G + NH * n_in + 2 * NH * NH};
    double dh[NH], da[NH];
    for (int k = 0; k < NH; ++k) dh[k] = 0.0;
    for (int o = 0; o < n_out; ++o)
        for (int k = 0; k < NH; ++k) {
            GW[3][o * NH + k] += dout[o] * hid[2 * NH + k];
            dh[k] += dout[o] * W[3][o * NH + k];
        }
    for (int l = 2; l >= 0; --l) {
        const int nin = l == 0 ? n_in : NH;
        const double* input = l == 0 ? x : hid + (l - 1) * NH;
        for (int j = 0; j < NH; ++j) da[j] = dh[j] * (pre[l * NH + j] > 0.0 ? 1.0 : LEAK);
        for (int j = 0; j < NH; ++j)
            for (int k = 0; k < nin; ++k) GW[l][j * nin + k] += da[j] * input[k];
        if (l > 0)
            for (int k = 0; k < NH; ++k) {
                double s = 0.0;
                for (int j = 0; j < NH; ++j) s += W[l][j * nin + k] * da[j];
                dh[k] = s;
            }
        else if (dx)
            for (int k = 0; k < n_in; ++k) {
                double s = 0.0;
                for (int j = 0; j < NH; ++j) s += W[0][j * n_in + k] * da[j];
                dx[k] = s;
            }
    }
}

void or_mlpn_backward(const double* P, int n_out, const double* x, const double* dout,
                      double* G) {
    or_mlpk_backward(P, NF, n_out, x, dout, G, NULL);
}

/* Relative L2 of both moments; returns the loss of one sample and writes d/dpred with
 * the normalisation held constant (the stop-gradient). */
double or_statnet_dloss(const double* pred /*6: m1 rgb, m2 rgb*/, const double* L /*3*/,
                        double eps, double* dpred) {
    double loss = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double t1 = L[c], t2 = L[c] * L[c];
        const double d1 = pred[c] - t1, d2 = pred[3 + c] - t2;
        const double w1 = 1.0 / (pred[c] * pred[c] + eps);
        const double w2 = 1.0 / (pred[3 + c] * pred[3 + c] + eps);
        loss += d1 * d1 * w1 + d2 * d2 * w2;
        dpred[c] = 2.0 * d1 * w1;
        dpred[3 + c] = 2.0 * d2 * w2;
    }
    return loss;
}

/* Per pixel: V = unbiased variance of the spp sample values / spp (mean over RGB), and
 * E = V / (I_ref^2 + eps) with I_ref the mean over RGB of the reference pixel.
 * S1 holds the spp sample values of every pixel, [npix][spp][3]. */
void or_pixel_error(const double* S1, int64_t npix, int32_t spp, const double* ref, double eps,
                    double* V, double* E) {
    for (int64_t p = 0; p < npix; ++p) {
        double v = 0.0;
        for (int c = 0; c < 3; ++c) {
            double m = 0.0;
            for (int s = 0; s < spp; ++s) m += S1[(p * spp + s) * 3 + c];
            m /= spp;
            double q = 0.0;
            for (int s = 0; s < spp; ++s) {
                const double d = S1[(p * spp + s) * 3 + c] - m;
                q += d * d;
            }
            v += spp > 1 ? q / (spp - 1) / spp : 0.0;
        }
        V[p] = v / 3.0;
        const double I = (ref[3 * p] + ref[3 * p + 1] + ref[3 * p + 2]) / 3.0;
        E[p] = V[p] / (I * I + eps);
    }
}

/* d L_RRSNet / d q_nrrs for every training sample s.  Inputs per sample: the network
 * output q_nrrs, the applied factor F (q_used = F q_nrrs), the normalization factor
 * Fn of Eq. F_norm without rate control (q_norm = Fn q_nrrs, a constant), the mean
 * prefix throughput t, the pixel, and the StatNet moments m1 = E[<H>], m2 = E[<H>^2]
 * (means over RGB).  Per pixel: E_i, the reference I_i (mean over RGB) and the count k_i
 * of training samples.  terms[0..2] receive L_avg, L_min and L_rrs.
 * q_used (nullable) is the factor each sample's frame was split with; the gradient
 * transfer of Eq. gradient_transfer_rr_mc / splitting_mc is taken at it, since the
 * variance it differentiates is that of the frame as sampled (NULL: q_used = F q_nrrs,
 * the case when the frame was rendered with the trained weights). */
void or_rrsnet_dloss_at(int64_t n, const double* q_nrrs, const double* F, const double* Fn,
                        const double* q_used, const double* t, const int32_t* pixel,
                        const double* m1, const double* m2, int64_t npix, const double* E,
                        const double* Iref, const int64_t* k, double eps, double g1, double g2,
                        double g3, double* dq, double* terms) {
    double Ebar = 0.0;
    for (int64_t p = 0; p < npix; ++p) Ebar += E[p];
    Ebar /= (double)npix;
    double Lavg = 0.0, Lmin = 0.0, Lrrs = 0.0;
    for (int64_t p = 0; p < npix; ++p) {
        Lavg += (E[p] - Ebar) * (E[p] - Ebar);
        Lmin += E[p];
    }
    for (int64_t s = 0; s < n; ++s) {
        const int32_t i = pixel[s];
        const double qu = q_used ? q_used[s] : F[s] * q_nrrs[s];
        /* dV_i/dq_used: Eq. gradient_transfer_rr_mc for roulette (q_used < 1),
         * Eq. gradient_transfer_splitting_mc for splitting (q_used >= 1) */
        const double VH = fmax(m2[s] - m1[s] * m1[s], 0.0);
        const double H = qu < 1.0 ? m2[s] : VH;
        const double dV_dqu = -t[s] * t[s] * H / (qu * qu);
        /* d(g1 L_avg + g2 L_min)/dE_i = g1 2 (E_i - Ebar) + g2 (the Ebar terms cancel),
         * dE_i/dV_i = 1 / (I_i^2 + eps), shared 1/k_i */
        const double dL_dE = g1 * 2.0 * (E[i] - Ebar) + g2;
        const double dL_dV = dL_dE / (Iref[i] * Iref[i] + eps) / (double)k[i];
        const double qn = Fn[s] * q_nrrs[s];
        Lrrs += (q_nrrs[s] - qn) * (q_nrrs[s] - qn);
        dq[s] = dL_dV * dV_dqu * F[s] + g3 * 2.0 * (q_nrrs[s] - qn);
    }
    terms[0] = Lavg;
    terms[1] = Lmin;
    terms[2] = Lrrs;
}

void or_rrsnet_dloss(int64_t n, const double* q_nrrs, const double* F, const double* Fn,
                     const double* t, const int32_t* pixel, const double* m1, const double* m2,
                     int64_t npix, const double* E, const double* Iref, const int64_t* k,
                     double eps, double g1, double g2, double g3, double* dq, double* terms) {
    or_rrsnet_dloss_at(n, q_nrrs, F, Fn, NULL, t, pixel, m1, m2, npix, E, Iref, k, eps, g1, g2,
                       g3, dq, terms);
}

/* Temporal smoothing of the pixel error map, Sec. 4 "Tackle Low Spp" (Eq. error_temporal
 * applied to the error map, with alpha_mix): E_acc = (1 - alpha) E_acc + alpha E_cur,
 * and E_acc = E_cur on the first frame. */
void or_error_temporal(const double* E_cur, double* E_acc, int64_t n, double alpha, int first) {
    for (int64_t p = 0; p < n; ++p)
        E_acc[p] = first ? E_cur[p] : (1.0 - alpha) * E_acc[p] + alpha * E_cur[p];
}

/* The spatial filter of the error map, standing in for the normal-guided denoiser of
 * Sec. 4 "Tackle Low Spp": out[p] = sum_q w_pq in[q] / sum_q w_pq over the (2r+1)^2
 * window of p clipped at the image border.  nrm [W*H][4] (unit normal, w > 0 when the
 * pixel has one) or NULL.  w_pp = 1; without normals, or when p has none or power <= 0,
 * every w_pq = 1; otherwise w_pq = max(0, n_p . n_q)^power for a neighbour with a
 * normal and 0 for one without. */
void or_error_filter(const double* in, const double* nrm, int32_t W, int32_t H, int32_t r,
                     double power, double* out) {
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            const int64_t p = (int64_t)y * W + x;
            const int guided = nrm != NULL && power > 0.0 && nrm[4 * p + 3] > 0.0;
            double s = 0.0, c = 0.0;
            for (int32_t yy = y - r; yy <= y + r; ++yy)
                for (int32_t xx = x - r; xx <= x + r; ++xx) {
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    const int64_t q = (int64_t)yy * W + xx;
                    double w = 1.0;
                    if (guided && q != p) {
                        const double d = nrm[4 * p] * nrm[4 * q] + nrm[4 * p + 1] * nrm[4 * q + 1] +
                                         nrm[4 * p + 2] * nrm[4 * q + 2];
                        w = nrm[4 * q + 3] > 0.0 && d > 0.0 ? pow(d, power) : 0.0;
                    }
                    s += w * in[q];
                    c += w;
                }
            out[p] = s / c;
        }
}

/* Normals guiding the filter: per pixel the normalised mean shading normal of its
 * depth-1 vertices whose factor went on (q_orig > 0), w = 1; (0, 0, 0, 0) when none did.
 * feat1 [npix * spp][16] holds the vertex features of depth 1 (shading normal at
 * 6..8), q1 [npix * spp] their q_orig; the samples of pixel p are p * spp .. + spp - 1. */
void or_pixel_normals(const double* feat1, const double* q1, int64_t npix, int32_t spp,
                      double* nrm) {
    for (int64_t p = 0; p < npix; ++p) {
        double n[3] = {0.0, 0.0, 0.0};
        int k = 0;
        for (int32_t s = 0; s < spp; ++s) {
            const int64_t i = p * spp + s;
            if (!(q1[i] > 0.0)) continue;
            for (int c = 0; c < 3; ++c) n[c] += feat1[16 * i + 6 + c];
            ++k;
        }
        const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int c = 0; c < 3; ++c) nrm[4 * p + c] = k > 0 && len > 0.0 ? n[c] / len : 0.0;
        nrm[4 * p + 3] = k > 0 && len > 0.0 ? 1.0 : 0.0;
    }
}

/* Adam (Kingma & Ba 2015), step number `step` >= 1. */
void or_adam_step(double* P, const double* G, double* m, double* v, int64_t n, int64_t step,
                  double lr, double b1, double b2, double eps) {
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * G[i];
        v[i] = b2 * v[i] + (1.0 - b2) * G[i] * G[i];
        P[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

void or_ema(double* Eavg, const double* P, int64_t n, double decay) {
    for (int64_t i = 0; i < n; ++i) Eavg[i] = decay * Eavg[i] + (1.0 - decay) * P[i];
}

/* relMSE (Sec. 5): mean over pixels and channels of (I - R)^2 / (R^2 + eps). */
double or_relmse(const double* img, const double* ref, int64_t n3, double eps) {
    double s = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
        const double d = img[i] - ref[i];
        s += d * d / (ref[i] * ref[i] + eps);
    }
    return n3 > 0 ? s / (double)n3 : 0.0;
}
