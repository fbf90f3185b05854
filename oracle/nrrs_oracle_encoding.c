/*
 * NRRS oracle, input encodings of Sec. 4 "Input Encoding": plain FP64 restatements.
 * TEST INFRASTRUCTURE ONLY (see nrrs_oracle.c).
 *
 *   or_grid_encode / or_grid_backward
 *       The trainable multiresolution hash grid (Mueller et al. 2022, "Instant Neural
 *       Graphics Primitives") with the paper's sizes: 8 levels of 2 features, resolution
 *       16 at the coarsest level, doubling per level.  Level l has resolution
 *       N_l = 16 * 2^l and T = 2^18 entries of 2 features; a point p in [0, 1]^3 lies in
 *       the cell floor(p N_l) (the last cell for p = 1) and its feature is the trilinear
 *       interpolation of the cell's 8 corner entries.  A corner v in {0..N_l}^3 has entry
 *       v.x + (N_l+1) (v.y + (N_l+1) v.z) while (N_l+1)^3 <= T, else the spatial hash
 *       (v.x * 1 xor v.y * 2654435761 xor v.z * 805459861) mod T in 32-bit unsigned
 *       arithmetic.  Output: 16 features, level-major.  The table is [8][T][2].
 *   or_one_blob
 *       One-blob encoding (Mueller et al. 2019, "Neural Importance Sampling"): k bins on
 *       [0, 1], bin i holds the Gaussian kernel of width sigma = 1/k centred at the value,
 *       evaluated at the bin centre (i + 1/2) / k.
 *   or_statnet_grid_inputs
 *       StatNet's 32 inputs: the hash grid of the position (16), the one-blob encoding
 *       with 4 bins of each spherical coordinate of w_o (theta / pi from the z axis and
 *       (phi + pi) / (2 pi)), and of the roughness remapped by 1 - exp(-alpha) with 8
 *       bins.
 *   or_aid_inputs
 *       AID-NRRS's 32 RRSNet inputs (Sec. 4 "Input Encoding"): the position and w_o
 *       encoded as for StatNet (with RRSNet's own grid), Box-Cox (the render's lambda,
 *       0.5 in the paper) of the throughput per channel and of the pixel estimate's mean
 *       (clamped at 0), and the remapped roughness one-blob encoded with 4 bins.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define G_LEVELS 8
#define G_F 2
#define G_LOG2T 18
#define G_T (1u << G_LOG2T)
#define G_BASE 16

int64_t or_grid_param_count(void) { return (int64_t)G_LEVELS * G_T * G_F; }

uint32_t or_grid_index(int l, uint32_t x, uint32_t y, uint32_t z) {
    const uint64_t n1 = ((uint64_t)G_BASE << l) + 1;
    if (n1 * n1 * n1 <= G_T) return (uint32_t)(x + n1 * (y + n1 * z));
    return (x * 1u ^ y * 2654435761u ^ z * 805459861u) & (G_T - 1u);
}

/* Cell and trilinear weights of p at level l: corner k (bit c of k = offset along axis
 * c) has entry idx[k] and weight w[k]. */
static void grid_corners(int l, const double p[3], uint32_t idx[8], double w[8]) {
    const uint32_t N = (uint32_t)G_BASE << l;
    uint32_t i0[3];
    double f[3];
    for (int c = 0; c < 3; ++c) {
        double s = p[c] * (double)N;
        double fl = floor(s);
        if (fl < 0.0) fl = 0.0;
        if (fl > (double)(N - 1)) fl = (double)(N - 1);
        i0[c] = (uint32_t)fl;
        f[c] = s - fl;
    }
    for (int k = 0; k < 8; ++k) {
        double wk = 1.0;
        uint32_t v[3];
        for (int c = 0; c < 3; ++c) {
            const int b = (k >> c) & 1;
            v[c] = i0[c] + (uint32_t)b;
            wk *= b ? f[c] : 1.0 - f[c];
        }
        idx[k] = or_grid_index(l, v[0], v[1], v[2]);
        w[k] = wk;
    }
}

void or_grid_encode(const double* table, const double p[3], double out[16]) {
    for (int l = 0; l < G_LEVELS; ++l) {
        uint32_t idx[8];
        double w[8];
        grid_corners(l, p, idx, w);
        for (int f = 0; f < G_F; ++f) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += w[k] * table[((size_t)l * G_T + idx[k]) * G_F + f];
            out[G_F * l + f] = s;
        }
    }
}

/* Accumulates into grad (the table's shape) the gradient of sum_j dout[j] out[j]. */
void or_grid_backward(double* grad, const double p[3], const double dout[16]) {
    for (int l = 0; l < G_LEVELS; ++l) {
        uint32_t idx[8];
        double w[8];
        grid_corners(l, p, idx, w);
        for (int k = 0; k < 8; ++k)
            for (int f = 0; f < G_F; ++f)
                grad[((size_t)l * G_T + idx[k]) * G_F + f] += w[k] * dout[G_F * l + f];
    }
}

void or_one_blob(double v, int k, double* out) {
    for (int i = 0; i < k; ++i) {
        const double d = ((i + 0.5) / k - v) * k;  /* (centre - v) / sigma */
        out[i] = exp(-0.5 * d * d);
    }
}

void or_statnet_grid_inputs(const double* table, const double p[3], const double wo[3],
                            double alpha, double x[32]) {
    or_grid_encode(table, p, x);
    double z = wo[2] < -1.0 ? -1.0 : wo[2] > 1.0 ? 1.0 : wo[2];
    const double theta = acos(z) / M_PI;
    const double phi = (atan2(wo[1], wo[0]) + M_PI) / (2.0 * M_PI);
    or_one_blob(theta, 4, x + 16);
    or_one_blob(phi, 4, x + 20);
    or_one_blob(1.0 - exp(-alpha), 8, x + 24);
}

double or_boxcox(double t, double lambda);  /* nrrs_oracle.c */

void or_aid_inputs(const double* table, const double p[3], const double wo[3], const double t[3],
                   double I, double alpha, double lambda, double x[32]) {
    or_grid_encode(table, p, x);
    double z = wo[2] < -1.0 ? -1.0 : wo[2] > 1.0 ? 1.0 : wo[2];
    or_one_blob(acos(z) / M_PI, 4, x + 16);
    or_one_blob((atan2(wo[1], wo[0]) + M_PI) / (2.0 * M_PI), 4, x + 20);
    for (int c = 0; c < 3; ++c) x[24 + c] = or_boxcox(t[c], lambda);
    x[27] = or_boxcox(I > 0.0 ? I : 0.0, lambda);
    or_one_blob(1.0 - exp(-alpha), 4, x + 28);
}
