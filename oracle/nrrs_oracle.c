/*
 * NRRS oracle: a plain, slow, FP64 CPU restatement of one render of wavefront path
 * tracing with normalized Russian roulette and splitting (RRS), and of RRSNet.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path; the two meet only at the seeded
 * input arrays (scenes, weights, features) drawn by paper_2510_07868_b300/inputs.py.
 *
 * What each function follows (paper: "NRRS: Neural Russian Roulette and Splitting"):
 *   or_philox4x32_10   Salmon et al. 2011, Philox-4x32 with 10 rounds (published def.)
 *   or_camera_ray      pinhole camera (not in the paper; fixed convention)
 *   or_intersect       closest hit by brute force over all triangles (Moller-Trumbore)
 *   or_sample_lambert  cosine-weighted hemisphere via the concentric disk map
 *                      (Shirley & Chiu 1997) in the Duff et al. 2017 orthonormal basis
 *   or_sample_ggx      GGX microfacet (Walter et al. 2007) + Lambert mixture
 *   or_mlp_forward     RRSNet, Sec. 4 "Network Architecture" (3 hidden layers of 32,
 *                      Leaky ReLU) and the output activation of Eq. rrsnet_activation
 *   or_mlp_backward    the chain rule through the same network
 *   or_render          also ADRRS (NN) factors at NET_MIX depths with gate 3 (Sec. 4
 *                      "Mix-Depth"): lum(t) E[L_o] / I_px from StatNet's predicted mean
 *   or_render (rrsnet_inputs = 2)  AID-NRRS: RRSNet (32 inputs) on its own hash grid of
 *                      the position, one-blob w_o and roughness, Box-Cox t and I_px
 *   or_render (rrsnet_inputs = 1)  the NRRS network inputs of Sec. 4 "Input Encoding":
 *                      Box-Cox (lambda 0.5) of StatNet's E[L_o] and E[L_o^2] (per channel,
 *                      clamped at 0), of the throughput t and of the pixel estimate's
 *                      mean, and the roughness remapped by 1 - exp(-alpha)
 *   or_normalize       Eq. q_norm, Eq. F_norm, Eq. q_norm_rate, Eq. f_rate_prime and
 *                      the downscale-only compromise of Sec. 4 ("Compromise")
 *   or_split           Eq. rrs_factor: N_q = floor(q) + Bernoulli(q - floor(q))
 *   or_render          the level-synchronous loop of Sec. 3.1 / Fig. wavefront
 *   or_eval_bsdf       f cos and the sampling pdf of a given direction (both lobes),
 *                      for next-event estimation
 *   or_render (nee)    next-event estimation, on in the paper's experiments (Sec. 5):
 *                      one emitter point per vertex (triangle by area, uniform on it),
 *                      a shadow ray, and multiple importance sampling with the power
 *                      heuristic (Veach 1997) against emitters hit by BSDF sampling
 *   or_bernstein_exponent  Eq. bernstein_frate
 *
 * Parity notes:
 *   - The integer split decision is taken in FP32, the precision the kernel takes it
 *     in: q_used = fp32(F) * fp32(q_orig) rounded to FP32, r = q_used - floor(q_used)
 *     (exact), X = floor(q_used) + [U < r] with U = (w >> 8) * 2^-24.
 *   - Everything else is FP64.
 *   - The paper prints no GGX formula of its own; the lobe is pinned by identities of
 *     the microfacet model (normalised D, Smith's masking identity, the sampler's
 *     expected weight against quadrature, the closed form at normal incidence) and its
 *     Fresnel term by the exact dielectric Fresnel equations within Schlick's error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 3

#define OR_MODE_NONE 0
#define OR_MODE_PLAIN_RR 1
#define OR_MODE_HEUR_NORM 2
#define OR_MODE_NET 3
#define OR_MODE_NET_MIX 4

#define OR_GATE_NET 0
#define OR_GATE_HEUR 1
#define OR_GATE_FIXED 2
#define OR_GATE_ADRRS 3
#define OR_ADRRS_FLOOR 0.05  /* smallest ADRRS (NN) factor: RR stays unbiased */
/* ADRRS weight window of ratio 5 around the ideal throughput: bounds 2/(1+5), 5 x that */
#define OR_ADRRS_WINDOW_LO (2.0 / 6.0)
#define OR_ADRRS_WINDOW_HI (10.0 / 6.0)

#define OR_PURPOSE_JITTER 0u
#define OR_PURPOSE_BSDF 1u
#define OR_PURPOSE_RRS 3u
#define OR_PURPOSE_NEE 5u
#define OR_SHADOW_MARGIN 1e-4  /* a shadow ray stops at (1 - margin) x the emitter distance */

#define OR_MAX_DEPTH 64
#define OR_RAY_OFFSET 1e-4
#define OR_LINEAGE_STEP 0x9E3779B9u
#define OR_NO_HIT 0xFFFFFFFFu

/* ------------------------------------------------------------------ Philox */

static void or_mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32-10: ten rounds of the Philox S-box, key bumped by the Weyl constants
 * between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        or_mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        or_mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0, 1): the top 24 bits of a word times 2^-24 (exact in FP32 and FP64). */
static double or_u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

static void or_draw(uint32_t seed_lo, uint32_t seed_hi, uint32_t frame, uint32_t pixel,
                    uint32_t sample, uint32_t depth, uint32_t purpose, uint32_t lineage,
                    uint32_t out[4]) {
    uint32_t ctr[4] = {pixel, sample, (depth << 8) | purpose, lineage};
    uint32_t key[2] = {seed_lo, seed_hi ^ frame};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ vectors */

typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static v3 nrm(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }

/* ------------------------------------------------------------------ scene */

typedef struct {
    int32_t type;
    float albedo[3];
    float Le[3];
    float roughness;
    float F0;
    int32_t two_sided;
} or_material;

typedef struct {
    float pos[3];
    float look[3];
    float up[3];
    float vfov_deg;
} or_camera;

typedef struct {
    const float* tri;       /* [n_tri][9] */
    const int32_t* mat_id;  /* [n_tri] */
    const or_material* mats;
    int32_t n_tri;
    int32_t n_mat;
    const or_camera* cam;
} or_scene;

static v3 or_tri_vertex(const or_scene* s, int32_t t, int k) {
    const float* p = s->tri + (size_t)t * 9 + 3 * k;
    return mk(p[0], p[1], p[2]);
}

/* Closest hit over every triangle.  Ties on t go to the lower triangle index because
 * only a strictly smaller t replaces the current hit.  Returns the triangle or -1. */
int32_t or_intersect(const or_scene* s, const double o_[3], const double d_[3], double* t_out) {
    v3 o = mk(o_[0], o_[1], o_[2]), d = mk(d_[0], d_[1], d_[2]);
    double best = INFINITY;
    int32_t hit = -1;
    for (int32_t i = 0; i < s->n_tri; ++i) {
        v3 v0 = or_tri_vertex(s, i, 0);
        v3 e1 = sub(or_tri_vertex(s, i, 1), v0);
        v3 e2 = sub(or_tri_vertex(s, i, 2), v0);
        v3 pv = cross(d, e2);
        double det = dot(e1, pv);
        if (det == 0.0) continue;
        double inv = 1.0 / det;
        v3 tv = sub(o, v0);
        double u = dot(tv, pv) * inv;
        if (u < 0.0 || u > 1.0) continue;
        v3 qv = cross(tv, e1);
        double v = dot(d, qv) * inv;
        if (v < 0.0 || u + v > 1.0) continue;
        double t = dot(e2, qv) * inv;
        if (t <= 0.0) continue;
        if (t < best) {
            best = t;
            hit = i;
        }
    }
    *t_out = best;
    return hit;
}

/* Pinhole camera: right = up x look, up' = look x right; pixel row 0 at the top. */
void or_camera_ray(const or_camera* c, int32_t W, int32_t H, int32_t px, int32_t py,
                   double jx, double jy, double o[3], double d[3]) {
    v3 fw = nrm(mk(c->look[0], c->look[1], c->look[2]));
    v3 up = mk(c->up[0], c->up[1], c->up[2]);
    v3 right = nrm(cross(up, fw));
    v3 up2 = cross(fw, right);
    double th = tan(0.5 * (double)c->vfov_deg * M_PI / 180.0);
    double aspect = (double)W / (double)H;
    double sx = (2.0 * (px + jx) / W - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * (py + jy) / H) * th;
    v3 dir = nrm(add(fw, add(scl(right, sx), scl(up2, sy))));
    o[0] = c->pos[0]; o[1] = c->pos[1]; o[2] = c->pos[2];
    d[0] = dir.x; d[1] = dir.y; d[2] = dir.z;
}

/* ------------------------------------------------------------------ BSDFs */

/* Orthonormal basis around unit n (Duff et al. 2017). */
static void or_onb(v3 n, v3* b1, v3* b2) {
    double sign = copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double b = n.x * n.y * a;
    *b1 = mk(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
    *b2 = mk(b, sign + n.y * n.y * a, -n.y);
}

/* Concentric map of [0,1)^2 to the unit disk (Shirley & Chiu 1997). */
static void or_concentric(double u1, double u2, double* x, double* y) {
    double a = 2.0 * u1 - 1.0, b = 2.0 * u2 - 1.0;
    if (a == 0.0 && b == 0.0) { *x = 0.0; *y = 0.0; return; }
    double r, phi;
    if (fabs(a) > fabs(b)) { r = a; phi = (M_PI / 4.0) * (b / a); }
    else { r = b; phi = M_PI / 2.0 - (M_PI / 4.0) * (a / b); }
    *x = r * cos(phi);
    *y = r * sin(phi);
}

static v3 or_cosine_dir(v3 n, double u1, double u2) {
    double x, y;
    or_concentric(u1, u2, &x, &y);
    double z = sqrt(fmax(0.0, 1.0 - x * x - y * y));
    v3 b1, b2;
    or_onb(n, &b1, &b2);
    return add(add(scl(b1, x), scl(b2, y)), scl(n, z));
}

/* Lambertian: cosine-weighted direction; f cos / pdf = albedo exactly. */
void or_sample_lambert(const double n_[3], double u1, double u2, double wi[3]) {
    v3 w = or_cosine_dir(mk(n_[0], n_[1], n_[2]), u1, u2);
    wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
}

/* GGX normal distribution (Walter et al. 2007, Eq. 33) at cos(theta_h), roughness a:
 * D = a^2 / (pi ((a^2 - 1) cos^2 + 1)^2), normalised so that the projected microfacet
 * area integrates to one: integral of D(h) (n.h) over the hemisphere = 1. */
double or_ggx_D(double cos_h, double a) {
    double a2 = a * a, c2 = cos_h * cos_h;
    double den = (a2 - 1.0) * c2 + 1.0;
    return a2 / (M_PI * den * den);
}

/* Smith masking of GGX (Walter et al. 2007, Eq. 34) for a direction at cos(theta):
 * G1 = 2 / (1 + sqrt(1 + a^2 tan^2 theta)). */
double or_ggx_G1(double cos_w, double a) {
    double c2 = cos_w * cos_w;
    double tan2 = (1.0 - c2) / c2;
    return 2.0 / (1.0 + sqrt(1.0 + a * a * tan2));
}

/* GGX + Lambert "plastic" mixture.  Lobe chosen with probability 1/2 each:
 *   specular: h ~ D(h) cos(theta_h) (tan^2 theta_h = a^2 u1/(1-u1), phi = 2 pi u2),
 *             wi = reflect(wo, h);  diffuse: cosine-weighted.
 *   f   = D G1(wo) G1(wi) F_schlick(wi.h) / (4 cos_o cos_i) + (1 - F0) albedo / pi
 *   pdf = 0.5 D cos_h / (4 |wo.h|) + 0.5 cos_i / pi
 * Writes the weight f cos_i / pdf per channel; returns 0 and weight 0 if wi falls
 * below the shading hemisphere. */
int or_sample_ggx(const double n_[3], const double wo_[3], double albedo_[3], double rough,
                  double F0, double ulobe, double u1, double u2, double wi_[3], double w[3]) {
    v3 n = mk(n_[0], n_[1], n_[2]), wo = mk(wo_[0], wo_[1], wo_[2]);
    double a = rough;
    v3 wi;
    if (ulobe < 0.5) {
        double tan2 = a * a * u1 / (1.0 - u1);
        double cos_h = 1.0 / sqrt(1.0 + tan2);
        double sin_h = sqrt(fmax(0.0, 1.0 - cos_h * cos_h));
        double phi = 2.0 * M_PI * u2;
        v3 b1, b2;
        or_onb(n, &b1, &b2);
        v3 h = add(add(scl(b1, sin_h * cos(phi)), scl(b2, sin_h * sin(phi))), scl(n, cos_h));
        wi = sub(scl(h, 2.0 * dot(wo, h)), wo);
    } else {
        wi = or_cosine_dir(n, u1, u2);
    }
    wi_[0] = wi.x; wi_[1] = wi.y; wi_[2] = wi.z;
    double cos_i = dot(wi, n), cos_o = dot(wo, n);
    if (cos_i <= 0.0 || cos_o <= 0.0) { w[0] = w[1] = w[2] = 0.0; return 0; }
    v3 h = nrm(add(wo, wi));
    double cos_h = dot(h, n);
    double oh = dot(wo, h);
    double D = or_ggx_D(cos_h, a);
    double G = or_ggx_G1(cos_o, a) * or_ggx_G1(cos_i, a);
    double Fr = F0 + (1.0 - F0) * pow(1.0 - dot(wi, h), 5.0);
    double spec = D * G * Fr / (4.0 * cos_o * cos_i);
    double pdf = 0.5 * D * cos_h / (4.0 * fabs(oh)) + 0.5 * cos_i / M_PI;
    for (int c = 0; c < 3; ++c) {
        double f = spec + (1.0 - F0) * albedo_[c] / M_PI;
        w[c] = f * cos_i / pdf;
    }
    return 1;
}

/* f(wo, wi) cos_i per channel and the pdf with which the material's sampling picks wi
 * (solid angle): Lambertian f = albedo / pi, pdf = cos_i / pi; the GGX mixture as in
 * or_sample_ggx.  Returns 0 (all zero) when wi or wo is below the shading hemisphere. */
int or_eval_bsdf(const or_material* m, const double n_[3], const double wo_[3],
                 const double wi_[3], double fcos[3], double* pdf) {
    v3 n = mk(n_[0], n_[1], n_[2]), wo = mk(wo_[0], wo_[1], wo_[2]);
    v3 wi = mk(wi_[0], wi_[1], wi_[2]);
    double cos_i = dot(wi, n), cos_o = dot(wo, n);
    fcos[0] = fcos[1] = fcos[2] = 0.0;
    *pdf = 0.0;
    if (cos_i <= 0.0 || cos_o <= 0.0) return 0;
    if (m->type == 0) {
        for (int c = 0; c < 3; ++c) fcos[c] = m->albedo[c] / M_PI * cos_i;
        *pdf = cos_i / M_PI;
        return 1;
    }
    double a = m->roughness, F0 = m->F0;
    v3 h = nrm(add(wo, wi));
    double cos_h = dot(h, n);
    double oh = dot(wo, h);
    double D = or_ggx_D(cos_h, a);
    double G = or_ggx_G1(cos_o, a) * or_ggx_G1(cos_i, a);
    double Fr = F0 + (1.0 - F0) * pow(1.0 - dot(wi, h), 5.0);
    double spec = D * G * Fr / (4.0 * cos_o * cos_i);
    for (int c = 0; c < 3; ++c) fcos[c] = (spec + (1.0 - F0) * m->albedo[c] / M_PI) * cos_i;
    *pdf = 0.5 * D * cos_h / (4.0 * fabs(oh)) + 0.5 * cos_i / M_PI;
    return 1;
}

/* or_eval_bsdf for a GGX-mixture material given by its parameters (for the tests). */
int or_eval_ggx(const double n_[3], const double wo_[3], const double wi_[3],
                const double albedo[3], double rough, double F0, double fcos[3], double* pdf) {
    or_material m;
    memset(&m, 0, sizeof(m));
    m.type = 1;
    for (int c = 0; c < 3; ++c) m.albedo[c] = (float)albedo[c];
    m.roughness = (float)rough;
    m.F0 = (float)F0;
    return or_eval_bsdf(&m, n_, wo_, wi_, fcos, pdf);
}

/* Loops of or_sample_ggx and or_eval_ggx over m directions / sample triples (tests). */
void or_sample_ggx_batch(const double n_[3], const double wo_[3], double albedo[3], double rough,
                         double F0, const double* u, int64_t m, double* wi, double* w) {
    for (int64_t k = 0; k < m; ++k)
        or_sample_ggx(n_, wo_, albedo, rough, F0, u[3 * k], u[3 * k + 1], u[3 * k + 2],
                      wi + 3 * k, w + 3 * k);
}

void or_eval_ggx_batch(const double n_[3], const double wo_[3], const double* wi, int64_t m,
                       const double albedo[3], double rough, double F0, double* fcos,
                       double* pdf) {
    for (int64_t k = 0; k < m; ++k)
        or_eval_ggx(n_, wo_, wi + 3 * k, albedo, rough, F0, fcos + 3 * k, pdf + k);
}

/* ------------------------------------------------------------------ RRSNet */

#define OR_NF 16
#define OR_NH 32
#define OR_NPARAM (OR_NH * OR_NF + OR_NH * OR_NH * 2 + OR_NH)
#define OR_LEAK 0.01

/* Output activation of Eq. rrsnet_activation: ln(1 + e^x) for x < 0, x/2 + ln 2 else. */
double or_softplus_mod(double x) { return x < 0.0 ? log1p(exp(x)) : 0.5 * x + M_LN2; }
double or_softplus_mod_grad(double x) { return x < 0.0 ? exp(x) / (1.0 + exp(x)) : 0.5; }

/* Forward pass; W1 [32][16] | W2 [32][32] | W3 [32][32] | W4 [1][32] row-major, no
 * biases; Leaky ReLU (slope 0.01) after each hidden layer.  Optionally returns the
 * pre-activations a1..a3 ([3][32]) and hidden outputs h1..h3 ([3][32]) and z. */
double or_mlp_forward(const double* P, const double* x, double* pre, double* hid, double* z_out) {
    const double* W[4] = {P, P + OR_NH * OR_NF, P + OR_NH * OR_NF + OR_NH * OR_NH,
                          P + OR_NH * OR_NF + 2 * OR_NH * OR_NH};
    double in[OR_NH], out[OR_NH];
    int nin = OR_NF;
    for (int k = 0; k < OR_NF; ++k) in[k] = x[k];
    for (int l = 0; l < 3; ++l) {
        for (int j = 0; j < OR_NH; ++j) {
            double a = 0.0;
            for (int k = 0; k < nin; ++k) a += W[l][j * nin + k] * in[k];
            if (pre) pre[l * OR_NH + j] = a;
            out[j] = a > 0.0 ? a : OR_LEAK * a;
            if (hid) hid[l * OR_NH + j] = out[j];
        }
        for (int j = 0; j < OR_NH; ++j) in[j] = out[j];
        nin = OR_NH;
    }
    double z = 0.0;
    for (int k = 0; k < OR_NH; ++k) z += W[3][k] * in[k];
    if (z_out) *z_out = z;
    return or_softplus_mod(z);
}

/* Gradient of dq * q(x) with respect to every weight (accumulated into G). */
void or_mlp_backward(const double* P, const double* x, double dq, double* G) {
    double pre[3 * OR_NH], hid[3 * OR_NH], z;
    or_mlp_forward(P, x, pre, hid, &z);
    const double* W[4] = {P, P + OR_NH * OR_NF, P + OR_NH * OR_NF + OR_NH * OR_NH,
                          P + OR_NH * OR_NF + 2 * OR_NH * OR_NH};
    double* GW[4] = {G, G + OR_NH * OR_NF, G + OR_NH * OR_NF + OR_NH * OR_NH,
                     G + OR_NH * OR_NF + 2 * OR_NH * OR_NH};
    double dz = dq * or_softplus_mod_grad(z);
    double dh[OR_NH], da[OR_NH];
    for (int k = 0; k < OR_NH; ++k) {
        GW[3][k] += dz * hid[2 * OR_NH + k];
        dh[k] = dz * W[3][k];
    }
    for (int l = 2; l >= 0; --l) {
        int nin = l == 0 ? OR_NF : OR_NH;
        const double* input = l == 0 ? x : hid + (l - 1) * OR_NH;
        for (int j = 0; j < OR_NH; ++j) da[j] = dh[j] * (pre[l * OR_NH + j] > 0.0 ? 1.0 : OR_LEAK);
        for (int j = 0; j < OR_NH; ++j)
            for (int k = 0; k < nin; ++k) GW[l][j * nin + k] += da[j] * input[k];
        if (l > 0) {
            for (int k = 0; k < OR_NH; ++k) {
                double s = 0.0;
                for (int j = 0; j < OR_NH; ++j) s += W[l][j * nin + k] * da[j];
                dh[k] = s;
            }
        }
    }
}

/* Batched forward over n rows of float32 features (for tests). */
void or_mlp_forward_batch(const double* P, const float* X, int64_t n, double* q) {
    for (int64_t i = 0; i < n; ++i) {
        double x[OR_NF];
        for (int k = 0; k < OR_NF; ++k) x[k] = X[i * OR_NF + k];
        q[i] = or_mlp_forward(P, x, NULL, NULL, NULL);
    }
}

/* Box-Cox transform (lambda = 0.5 in Sec. 4 "Input Encoding"); lambda = 0 is log. */
double or_boxcox(double t, double lambda) {
    return lambda == 0.0 ? log(t) : (pow(t, lambda) - 1.0) / lambda;
}

/* ------------------------------------------------------------------ RRS */

/* Eq. F_norm with the rate-control factor of Eq. q_norm_rate, the adaptive alpha of
 * Eq. f_rate_prime, and downscale-only normalisation (Sec. 4, "Compromise"):
 *   F = min(1, f_rate * alpha * budget / sum_i q_i); F = 1 if the sum is 0. */
double or_normalize(const double* q, int64_t n, double budget, double f_rate, double alpha,
                    double* sum_out) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += q[i];
    if (sum_out) *sum_out = s;
    if (!(s > 0.0)) return 1.0;
    double F = f_rate * alpha * budget / s;
    return F < 1.0 ? F : 1.0;
}

/* Eq. rrs_factor, decided in FP32: returns X and writes the Bernoulli word pair. */
static uint32_t or_split_one(float F32, float q32, uint32_t seed_lo, uint32_t seed_hi,
                             uint32_t frame, uint32_t pixel, uint32_t sample, uint32_t depth,
                             uint32_t lineage, float* q_used, uint32_t* lineage_base) {
    volatile float qu = F32 * q32; /* one FP32 rounding, no contraction */
    float k = floorf(qu);
    float r = qu - k;
    uint32_t w[4];
    or_draw(seed_lo, seed_hi, frame, pixel, sample, depth, OR_PURPOSE_RRS, lineage, w);
    float U = (float)(w[0] >> 8) * (1.0f / 16777216.0f);
    *q_used = qu;
    *lineage_base = w[1];
    return (uint32_t)k + (U < r ? 1u : 0u);
}

/* Split counts and compaction of one queue (Eq. rrs_factor):
 *   X_i = floor(q_used_i) + [U_i < r_i], children of i at [prefix_i, prefix_i + X_i)
 *   in parent order; child j of i has lineage (w1_i + j * 0x9E3779B9) mod 2^32.
 * Children whose slot would be >= cap are dropped and counted.  Outputs:
 *   X[n], prefix[n] (exclusive scan of X), child_parent[min(S,cap)],
 *   child_lineage[min(S,cap)]; returns S (total requested children). */
int64_t or_split(const float* q_orig, int64_t n, float F32, const uint32_t* pixel,
                 const uint32_t* sample, const uint32_t* lineage, uint32_t depth,
                 uint32_t seed_lo, uint32_t seed_hi, uint32_t frame, int64_t cap, uint32_t* X,
                 int64_t* prefix, uint32_t* child_parent, uint32_t* child_lineage,
                 int64_t* dropped) {
    int64_t S = 0, drop = 0;
    for (int64_t i = 0; i < n; ++i) {
        float qu;
        uint32_t base;
        uint32_t x = or_split_one(F32, q_orig[i], seed_lo, seed_hi, frame, pixel[i], sample[i],
                                  depth, lineage[i], &qu, &base);
        X[i] = x;
        prefix[i] = S;
        /* slots S .. S + x - 1; those at or beyond cap are dropped (counted, not written) */
        int64_t kept = cap - S;
        if (kept < 0) kept = 0;
        if (kept > (int64_t)x) kept = (int64_t)x;
        for (int64_t j = 0; j < kept; ++j) {
            child_parent[S + j] = (uint32_t)i;
            child_lineage[S + j] = base + (uint32_t)j * OR_LINEAGE_STEP;
        }
        drop += (int64_t)x - kept;
        S += x;
    }
    *dropped = drop;
    return S;
}

/* Eq. bernstein_frate: P(S' >= N) <= exp(-N * c(f)),  c(f) = (1-f)^2 / (2f + 2(1-f)/3). */
double or_bernstein_exponent(double f_rate) {
    double g = 1.0 - f_rate;
    return g * g / (2.0 * f_rate + (2.0 / 3.0) * g);
}

/* StatNet forward (nrrs_oracle_train.c) and its encodings (nrrs_oracle_encoding.c) */
void or_mlpn_forward(const double* P, int n_out, const double* x, double* out, double* pre,
                     double* hid);
void or_mlpk_forward(const double* P, int n_in, int n_out, const double* x, double* out,
                     double* pre, double* hid);
void or_statnet_grid_inputs(const double* table, const double p[3], const double wo[3],
                            double alpha, double x[32]);
void or_aid_inputs(const double* table, const double p[3], const double wo[3], const double t[3],
                   double I, double alpha, double lambda, double x[32]);

/* ------------------------------------------------------------------ render */

typedef struct {
    int32_t width, height, spp, max_depth, mode;
    uint32_t seed_lo, seed_hi, frame;
    int64_t cap;            /* queue capacity C; 0 = 2 * W * H * spp */
    double f_rate;          /* Eq. q_norm_rate */
    double alpha0;          /* Eq. f_rate_prime, initial alpha */
    double q_max;           /* heuristic cap */
    double eps_rel;         /* heuristic: eps_I = eps_rel * mean(reference) */
    double boxcox_lambda;   /* throughput feature encoding */
    uint64_t gate;          /* NET_MIX: 2 bits per depth (0 NET, 1 HEUR, 2 FIXED) */
    const double* params;   /* RRSNet weights (NET / NET_MIX) */
    const double* pixel_ref;/* previous estimate [H*W*3] or NULL */
    const int32_t* pixels;  /* optional ascending pixel subset; normalised modes need
                               forced_F, since Sigma q spans the whole frame */
    int64_t n_pixels;
    double* rec;            /* optional per-vertex record [D][cap][OR_REC], see or_render */
    const float* forced_F;  /* optional [D]: the normalisation factor of every depth, taken
                               from a whole-frame render in place of Eq. F_norm over the
                               subset (test hook for sampled pixels of a full frame) */
    const double* stat_params; /* StatNet weights (ADRRS (NN) depths of NET_MIX) */
    int32_t nee;            /* next-event estimation with MIS (1) or BSDF sampling only (0) */
    int32_t rrsnet_inputs;  /* RRSNet inputs: 0 = the 16 vertex features, 1 = NRRS inputs
                               (needs stat_params), 2 = AID-NRRS inputs (needs rrs_grid;
                               params then has 32 inputs) */
    int32_t stat_encoding;  /* StatNet inputs: 0 = the 13 vertex features (throughput
                               inputs zeroed), 1 = hash grid + one-blob (needs stat_grid) */
    const double* stat_grid;/* StatNet's hash-grid table [8][2^18][2] */
    const double* rrs_grid; /* RRSNet's hash-grid table (AID-NRRS inputs) */
    int64_t budget;         /* N_px of Eq. F_norm: the expected paths per depth before rate
                               control; 0 = W * H * spp, the primary queue (Sec. 3.1) */
} or_render_args;

/* StatNet's six outputs at a vertex whose 16 features are x (position in the scene box,
 * -w_o, ...) and whose roughness is alpha. */
static void or_statnet_at(const or_render_args* a, const double x[16], double alpha,
                          double out[6]) {
    if (a->stat_encoding) {
        double x32[32];
        or_statnet_grid_inputs(a->stat_grid, x, x + 3, alpha, x32);
        or_mlpk_forward(a->stat_params, 32, 6, x32, out, NULL, NULL);
    } else {
        double xs[16];
        memcpy(xs, x, sizeof(xs));
        xs[13] = xs[14] = xs[15] = 0.0;
        or_mlpn_forward(a->stat_params, 6, xs, out, NULL, NULL);
    }
}

/* Per-vertex record: suffix sum S (rgb), own deposit (rgb), prefix throughput (rgb),
 * q_orig, q_used, X, first child slot, pixel, and the 16 vertex features RRSNet reads
 * (position in the scene box, w_o, shading normal, albedo, d / D, Box-Cox t; zero at
 * vertices that did not go on to a factor decision). */
#define OR_REC 30

typedef struct {
    int64_t live[OR_MAX_DEPTH + 1];
    double sum_q[OR_MAX_DEPTH + 1];
    float F[OR_MAX_DEPTH + 1];
    double alpha[OR_MAX_DEPTH + 1];
    int64_t dropped[OR_MAX_DEPTH + 1];
    int64_t requested[OR_MAX_DEPTH + 1];
    int64_t segments;
    int64_t nonfinite;
} or_render_stats;

typedef struct {
    double o[3], d[3], t[3];
    double pdf;             /* solid-angle pdf the direction was sampled with (0: camera) */
    uint32_t pixel, sample, lineage;
} or_path;

typedef struct {
    int32_t tri;            /* -1 = miss */
    double p[3], n[3];      /* hit point, shading normal facing -d */
    double q;               /* q_orig (0 = terminate) */
    int net_fallback;       /* the network's factor was non-finite: q is the heuristic's */
    double emit_w;          /* MIS weight of the emission found here (1 without NEE) */
    double nee[3];          /* next-event contribution, 0 when occluded or not taken */
    double feat[16];        /* the vertex features (record mode) */
} or_hitrec;

static double or_lum(const double t[3]) { return 0.2126 * t[0] + 0.7152 * t[1] + 0.0722 * t[2]; }

/* ------------------------------------------------------------------ next-event estimation */

/* Emitters: every triangle whose material emits (some Le channel > 0) and whose area is
 * positive, in triangle order.  One is chosen with probability area / A (A = their total
 * area): cdf[k] = fp32(sum of the first k + 1 areas / A), summed in FP64 in triangle
 * order, the last entry 1; a uniform u picks the first k with u < cdf[k] (u and cdf are
 * FP32 values, so the comparison is the FP32 one). */
typedef struct {
    int32_t n;
    int32_t* tri;
    float* cdf;
    double area;
} or_emitters;

static double or_tri_area(const or_scene* s, int32_t t) {
    v3 v0 = or_tri_vertex(s, t, 0);
    v3 c = cross(sub(or_tri_vertex(s, t, 1), v0), sub(or_tri_vertex(s, t, 2), v0));
    return 0.5 * sqrt(dot(c, c));
}

static int or_emits(const or_material* m) { return m->Le[0] > 0.0f || m->Le[1] > 0.0f || m->Le[2] > 0.0f; }

static int or_build_emitters(const or_scene* s, or_emitters* e) {
    memset(e, 0, sizeof(*e));
    e->tri = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->n_tri + 1));
    e->cdf = (float*)malloc(sizeof(float) * (size_t)(s->n_tri + 1));
    if (!e->tri || !e->cdf) return OR_ERR_OOM;
    for (int32_t i = 0; i < s->n_tri; ++i)
        if (or_emits(&s->mats[s->mat_id[i]]) && or_tri_area(s, i) > 0.0) {
            e->tri[e->n++] = i;
            e->area += or_tri_area(s, i);
        }
    double run = 0.0;
    for (int32_t k = 0; k < e->n; ++k) {
        run += or_tri_area(s, e->tri[k]);
        e->cdf[k] = k == e->n - 1 ? 1.0f : (float)(run / e->area);
    }
    return OR_OK;
}

/* Power heuristic with exponent 2 (Veach 1997): the weight of technique a against b. */
static double or_power_heuristic(double pa, double pb) {
    double a2 = pa * pa, b2 = pb * pb;
    return a2 / (a2 + b2);
}

/* Next-event estimation at a vertex (hit point hp, shading normal ns, outgoing wo,
 * throughput t) with the NEE draw w: an emitter triangle by area (w[0]), a uniform
 * point on it (sqrt(u1) (1 - u2) and sqrt(u1) u2 along its two edges, w[1], w[2]), and a
 * shadow ray from the offset origin that must reach (1 - margin) of the distance.  The
 * contribution t f cos_x Le w_light / p_light, with p_light = dist^2 / (|cos_l| A) the
 * solid-angle density of the emitter sample and w_light the power heuristic against
 * the BSDF's pdf of the same direction. */
static void or_nee(const or_scene* s, const or_emitters* E, const or_material* m, v3 hp, v3 ns,
                   v3 wo, const double t[3], const uint32_t w[4], double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (E->n == 0) return;
    const double u = or_u01(w[0]);
    int32_t k = 0;
    while (k < E->n - 1 && !(u < (double)E->cdf[k])) ++k;
    const int32_t lt = E->tri[k];
    const double su = sqrt(or_u01(w[1])), u2 = or_u01(w[2]);
    v3 v0 = or_tri_vertex(s, lt, 0);
    v3 e1 = sub(or_tri_vertex(s, lt, 1), v0), e2 = sub(or_tri_vertex(s, lt, 2), v0);
    v3 y = add(v0, add(scl(e1, su * (1.0 - u2)), scl(e2, su * u2)));
    v3 org = add(hp, scl(ns, OR_RAY_OFFSET));
    v3 v = sub(y, org);
    const double dist2 = dot(v, v);
    if (!(dist2 > 0.0)) return;
    const double dist = sqrt(dist2);
    v3 wl = scl(v, 1.0 / dist);
    const or_material* me = &s->mats[s->mat_id[lt]];
    const double cos_l = -dot(nrm(cross(e1, e2)), wl);
    if (!(cos_l > 0.0 || (me->two_sided && cos_l < 0.0))) return;
    double n_[3] = {ns.x, ns.y, ns.z}, wo_[3] = {wo.x, wo.y, wo.z}, wi_[3] = {wl.x, wl.y, wl.z};
    double fcos[3], pb;
    if (!or_eval_bsdf(m, n_, wo_, wi_, fcos, &pb)) return;
    const double pl = dist2 / (fabs(cos_l) * E->area);
    const double wmis = or_power_heuristic(pl, pb);
    double o_[3] = {org.x, org.y, org.z}, th;
    if (or_intersect(s, o_, wi_, &th) >= 0 && th < dist * (1.0 - OR_SHADOW_MARGIN)) return;
    for (int c = 0; c < 3; ++c) out[c] = t[c] * fcos[c] * me->Le[c] * wmis / pl;
}

static int or_is_normalized(int mode) {
    return mode == OR_MODE_HEUR_NORM || mode == OR_MODE_NET || mode == OR_MODE_NET_MIX;
}

/* One render, level-synchronous (the queue is normalised per depth, so every path of a
 * depth is processed before any of the next).  Deposits are summed per pixel in FP64
 * and divided by spp.  With trace != NULL, trace[(d-1)*cap*5 + 5*i + {0..4}] holds
 * (pixel, sample, lineage, triangle or 0xFFFFFFFF, X) of slot i at depth d, and
 * trace_count[d-1] the queue length.  With a->rec != NULL every vertex is recorded and,
 * after the last depth, a reverse pass fills its suffix sum: S = own deposit + the sum
 * of its children's S (children are the slots [first, first + X) of the next depth that
 * fit in the queue).  S / t is the vertex's estimate of outgoing radiance, the target
 * StatNet learns (Sec. 3.2 "Loss Design"). */
int or_render(const or_scene* s, const or_render_args* a, double* out_rgb,
              or_render_stats* st, uint32_t* trace, int64_t* trace_count) {
    const int32_t W = a->width, H = a->height, spp = a->spp, D = a->max_depth;
    if (W <= 0 || H <= 0 || spp <= 0 || D <= 0 || D > OR_MAX_DEPTH) return OR_ERR_ARG;
    const int64_t npix = (int64_t)W * H;
    const int64_t P = (a->pixels ? a->n_pixels : npix) * spp;
    const int64_t cap = a->cap > 0 ? a->cap : 2 * (int64_t)W * H * spp;
    const int64_t budget = a->budget > 0 ? a->budget : (int64_t)W * H * spp;
    if (a->pixels && or_is_normalized(a->mode) && !a->forced_F) return OR_ERR_ARG;
    if (a->mode == OR_MODE_NET_MIX && !a->stat_params)
        for (int32_t d = 1; d <= D; ++d)
            if (((a->gate >> (2 * (d - 1))) & 3u) == OR_GATE_ADRRS) return OR_ERR_ARG;
    if (a->rrsnet_inputs == 1 && !a->stat_params) return OR_ERR_ARG;
    if (a->rrsnet_inputs == 2 && !a->rrs_grid) return OR_ERR_ARG;
    if (a->stat_encoding && !a->stat_grid) return OR_ERR_ARG;
    if (P > cap) return OR_ERR_ARG;
    or_emitters E;
    memset(&E, 0, sizeof(E));
    if (a->nee && or_build_emitters(s, &E) != OR_OK) {
        free(E.tri); free(E.cdf);
        return OR_ERR_OOM;
    }
    /* queue storage: the capacity, or for a pixel subset 64 slots per primary path
     * (a subset's queue cannot be capped the way the whole frame's is; running out of
     * that room is reported as OR_ERR_OOM rather than dropping children) */
    int64_t room = cap;
    if (a->pixels && 64 * P < room) room = 64 * P;
    or_path* cur = (or_path*)calloc((size_t)room, sizeof(or_path));
    or_path* nxt = (or_path*)calloc((size_t)room, sizeof(or_path));
    or_hitrec* vx = (or_hitrec*)calloc((size_t)room, sizeof(or_hitrec));
    double* acc = (double*)calloc((size_t)npix * 3, sizeof(double));
    double* qbuf = (double*)calloc((size_t)room, sizeof(double));
    if (!cur || !nxt || !vx || !acc || !qbuf) {
        free(cur); free(nxt); free(vx); free(acc); free(qbuf); free(E.tri); free(E.cdf);
        return OR_ERR_OOM;
    }
    memset(st, 0, sizeof(*st));

    /* scene bounding box, for the position feature */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < (int64_t)s->n_tri * 3; ++i)
        for (int c = 0; c < 3; ++c) {
            double v = s->tri[i * 3 + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
    /* heuristic reference: eps_I = eps_rel * mean over pixels and channels */
    double ref_mean = 0.0;
    if (a->pixel_ref) {
        for (int64_t i = 0; i < npix * 3; ++i) ref_mean += a->pixel_ref[i];
        ref_mean /= (double)(npix * 3);
    }
    const double eps_I = a->eps_rel * ref_mean;

    /* primary queue, pixel-major and sample-minor */
    int64_t n = 0;
    for (int64_t pi = 0; pi < (a->pixels ? a->n_pixels : npix); ++pi) {
        int32_t pix = a->pixels ? a->pixels[pi] : (int32_t)pi;
        for (int32_t sidx = 0; sidx < spp; ++sidx) {
            uint32_t w[4];
            or_draw(a->seed_lo, a->seed_hi, a->frame, (uint32_t)pix, (uint32_t)sidx, 0,
                    OR_PURPOSE_JITTER, 0, w);
            or_path* p = &cur[n++];
            or_camera_ray(s->cam, W, H, pix % W, pix / W, or_u01(w[0]), or_u01(w[1]), p->o, p->d);
            p->t[0] = p->t[1] = p->t[2] = 1.0;
            p->pdf = 0.0;
            p->pixel = (uint32_t)pix;
            p->sample = (uint32_t)sidx;
            p->lineage = 0;
        }
    }

    double alpha = a->alpha0;
    for (int32_t depth = 1; depth <= D && n > 0; ++depth) {
        st->live[depth] = n;
        st->segments += n;
        /* extend + shade: closest hit, emission deposit, RRS factor q_orig */
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            or_path* p = &cur[i];
            or_hitrec* v = &vx[i];
            double t;
            v->tri = or_intersect(s, p->o, p->d, &t);
            v->q = 0.0;
            v->net_fallback = 0;
            v->emit_w = 1.0;
            v->nee[0] = v->nee[1] = v->nee[2] = 0.0;
            memset(v->feat, 0, sizeof(v->feat));
            if (v->tri < 0) continue;
            v3 o = mk(p->o[0], p->o[1], p->o[2]), d = mk(p->d[0], p->d[1], p->d[2]);
            v3 hp = add(o, scl(d, t));
            v3 v0 = or_tri_vertex(s, v->tri, 0);
            v3 ng = nrm(cross(sub(or_tri_vertex(s, v->tri, 1), v0), sub(or_tri_vertex(s, v->tri, 2), v0)));
            int front = dot(ng, d) < 0.0;
            v3 ns = front ? ng : scl(ng, -1.0);
            v->p[0] = hp.x; v->p[1] = hp.y; v->p[2] = hp.z;
            v->n[0] = ns.x; v->n[1] = ns.y; v->n[2] = ns.z;
            const or_material* m = &s->mats[s->mat_id[v->tri]];
            int black = m->albedo[0] == 0.0f && m->albedo[1] == 0.0f && m->albedo[2] == 0.0f;
            int dead = p->t[0] == 0.0 && p->t[1] == 0.0 && p->t[2] == 0.0;
            /* an emitter found by BSDF sampling: its MIS weight against the emitter
             * sample the previous vertex took (the camera's vertex has none) */
            if (a->nee && E.n > 0 && p->pdf > 0.0 && or_emits(m) && (front || m->two_sided)) {
                const double pl = t * t / (fabs(dot(ng, d)) * E.area);
                v->emit_w = or_power_heuristic(p->pdf, pl);
            }
            if (black || dead || depth == D) continue;
            {  /* the 16 vertex features of the record (RRSNet's inputs at NET depths) */
                for (int c = 0; c < 3; ++c) {
                    double ext = hi[c] - lo[c];
                    v->feat[c] = ext > 0.0 ? (v->p[c] - lo[c]) / ext : 0.5;
                }
                v->feat[3] = -d.x; v->feat[4] = -d.y; v->feat[5] = -d.z;
                v->feat[6] = ns.x; v->feat[7] = ns.y; v->feat[8] = ns.z;
                for (int c = 0; c < 3; ++c) v->feat[9 + c] = m->albedo[c];
                v->feat[12] = (double)depth / (double)D;
                for (int c = 0; c < 3; ++c) v->feat[13 + c] = or_boxcox(p->t[c], a->boxcox_lambda);
            }
            if (a->nee) {
                uint32_t w[4];
                or_draw(a->seed_lo, a->seed_hi, a->frame, p->pixel, p->sample, (uint32_t)depth,
                        OR_PURPOSE_NEE, p->lineage, w);
                or_nee(s, &E, m, hp, ns, scl(d, -1.0), p->t, w, v->nee);
            }
            int method;
            switch (a->mode) {
                case OR_MODE_NONE: method = -1; break;
                case OR_MODE_PLAIN_RR: method = -2; break;
                case OR_MODE_HEUR_NORM: method = OR_GATE_HEUR; break;
                case OR_MODE_NET: method = OR_GATE_NET; break;
                default: method = (int)((a->gate >> (2 * (depth - 1))) & 3u); break;
            }
            double q;
            /* the throughput heuristic: HEUR factors, and the stand-in for a network
             * factor that comes out non-finite */
            double heur = or_lum(p->t);
            if (a->pixel_ref) {
                const double* r = a->pixel_ref + 3 * (int64_t)p->pixel;
                double den = fmax((r[0] + r[1] + r[2]) / 3.0, eps_I);
                heur = den > 0.0 ? fmin(heur / den, a->q_max) : a->q_max;
            }
            if (method == -1 || method == OR_GATE_FIXED) {
                q = 1.0;
            } else if (method == -2) {
                q = fmin(1.0, or_lum(p->t));
            } else if (method == OR_GATE_HEUR) {
                q = heur;
            } else if (method == OR_GATE_ADRRS) {
                /* ADRRS (NN), Sec. 4 "Mix-Depth": the path's expected contribution
                 * lum(t) E[L_o] from StatNet (its throughput inputs zeroed, as trained),
                 * relative to the pixel estimate; the heuristic before any estimate */
                if (!a->pixel_ref) {
                    q = heur;
                } else {
                    double x[OR_NF], out[6];
                    for (int c = 0; c < 3; ++c) {
                        double ext = hi[c] - lo[c];
                        x[c] = ext > 0.0 ? (v->p[c] - lo[c]) / ext : 0.5;
                    }
                    x[3] = -d.x; x[4] = -d.y; x[5] = -d.z;
                    x[6] = ns.x; x[7] = ns.y; x[8] = ns.z;
                    for (int c = 0; c < 3; ++c) x[9 + c] = m->albedo[c];
                    x[12] = (double)depth / (double)D;
                    x[13] = x[14] = x[15] = 0.0;
                    or_statnet_at(a, x, m->type == 0 ? 1.0 : (double)m->roughness, out);
                    const double el = (out[0] + out[1] + out[2]) / 3.0;
                    const double* r = a->pixel_ref + 3 * (int64_t)p->pixel;
                    const double den = fmax((r[0] + r[1] + r[2]) / 3.0, eps_I);
                    /* r: the path's expected contribution over the pixel estimate; the
                     * weight window of ADRRS leaves the path alone inside [1/3, 5/3] */
                    q = den > 0.0 ? or_lum(p->t) * fmax(el, 0.0) / den : a->q_max;
                    if (!isfinite(q)) {
                        q = heur;
                        v->net_fallback = 1;
                    } else {
                        if (q >= OR_ADRRS_WINDOW_LO && q <= OR_ADRRS_WINDOW_HI) q = 1.0;
                        q = fmin(fmax(q, OR_ADRRS_FLOOR), a->q_max);
                    }
                }
            } else {
                double x[OR_NF];
                for (int c = 0; c < 3; ++c) {
                    double ext = hi[c] - lo[c];
                    x[c] = ext > 0.0 ? (v->p[c] - lo[c]) / ext : 0.5;
                }
                x[3] = -d.x; x[4] = -d.y; x[5] = -d.z;
                x[6] = ns.x; x[7] = ns.y; x[8] = ns.z;
                for (int c = 0; c < 3; ++c) x[9 + c] = m->albedo[c];
                x[12] = (double)depth / (double)D;
                for (int c = 0; c < 3; ++c) x[13 + c] = or_boxcox(p->t[c], a->boxcox_lambda);
                if (a->rrsnet_inputs == 2) {
                    /* AID-NRRS inputs (Sec. 4 "Input Encoding"): RRSNet's own grid of the
                     * position, one-blob w_o and roughness, Box-Cox t and I_px */
                    double I = 0.0, x32[32], z;
                    if (a->pixel_ref) {
                        const double* r = a->pixel_ref + 3 * (int64_t)p->pixel;
                        I = (r[0] + r[1] + r[2]) / 3.0;
                    }
                    or_aid_inputs(a->rrs_grid, x, x + 3, p->t, I,
                                  m->type == 0 ? 1.0 : (double)m->roughness, a->boxcox_lambda,
                                  x32);
                    or_mlpk_forward(a->params, 32, 1, x32, &z, NULL, NULL);
                    q = or_softplus_mod(z);
                } else if (a->rrsnet_inputs) {
                    /* NRRS inputs (Sec. 4 "Input Encoding"): StatNet's statistics at the
                     * vertex (its throughput inputs zeroed, as trained), the throughput,
                     * the pixel estimate's mean (0 before any) and the remapped roughness
                     * (a Lambertian surface counts as roughness 1); unused inputs 0 */
                    double st6[6];
                    const double rough = m->type == 0 ? 1.0 : (double)m->roughness;
                    or_statnet_at(a, x, rough, st6);
                    double I = 0.0;
                    if (a->pixel_ref) {
                        const double* r = a->pixel_ref + 3 * (int64_t)p->pixel;
                        I = (r[0] + r[1] + r[2]) / 3.0;
                    }
                    for (int c = 0; c < 6; ++c) x[c] = or_boxcox(fmax(st6[c], 0.0), a->boxcox_lambda);
                    for (int c = 0; c < 3; ++c) x[6 + c] = or_boxcox(p->t[c], a->boxcox_lambda);
                    x[9] = or_boxcox(fmax(I, 0.0), a->boxcox_lambda);
                    x[10] = 1.0 - exp(-rough);
                    for (int c = 11; c < OR_NF; ++c) x[c] = 0.0;
                }
                if (a->rrsnet_inputs != 2) q = or_mlp_forward(a->params, x, NULL, NULL, NULL);
                if (!(isfinite(q) && q >= 0.0)) {  /* a failing network: the heuristic */
                    q = heur;
                    v->net_fallback = 1;
                }
            }
            v->q = q;
        }
        /* deposits, in queue order: emission (MIS-weighted with NEE), then the
         * next-event contribution */
        for (int64_t i = 0; i < n; ++i) {
            const or_path* p = &cur[i];
            const or_hitrec* v = &vx[i];
            if (v->tri < 0) continue;
            const or_material* m = &s->mats[s->mat_id[v->tri]];
            v3 v0 = or_tri_vertex(s, v->tri, 0);
            v3 ng = cross(sub(or_tri_vertex(s, v->tri, 1), v0), sub(or_tri_vertex(s, v->tri, 2), v0));
            int front = dot(ng, mk(p->d[0], p->d[1], p->d[2])) < 0.0;
            for (int c = 0; c < 3; ++c) {
                double e = (front || m->two_sided) ? p->t[c] * m->Le[c] * v->emit_w : 0.0;
                acc[3 * (int64_t)p->pixel + c] += e + v->nee[c];
                if (a->rec) a->rec[((int64_t)(depth - 1) * cap + i) * OR_REC + 3 + c] = e + v->nee[c];
            }
        }
        /* non-finite network factors took the heuristic's; any other non-finite factor
         * terminates its path */
        for (int64_t i = 0; i < n; ++i) {
            if (vx[i].net_fallback) st->nonfinite++;
            if (!(isfinite(vx[i].q) && vx[i].q >= 0.0)) {
                vx[i].q = 0.0;
                st->nonfinite++;
            }
            /* the kernel holds q_orig in FP32; the sum and the decision see that value */
            qbuf[i] = (double)(float)vx[i].q;
        }
        float F32 = 1.0f;
        st->alpha[depth] = alpha;
        if (or_is_normalized(a->mode) && a->forced_F) {
            for (int64_t i = 0; i < n; ++i) st->sum_q[depth] += qbuf[i];
            F32 = a->forced_F[depth - 1];
        } else if (or_is_normalized(a->mode)) {
            double sum;
            double F = or_normalize(qbuf, n, (double)budget, a->f_rate, alpha, &sum);
            st->sum_q[depth] = sum;
            F32 = (float)F;
        } else {
            for (int64_t i = 0; i < n; ++i) st->sum_q[depth] += qbuf[i];
        }
        st->F[depth] = F32;
        /* split (Eq. rrs_factor) and BSDF sampling per child */
        int64_t S = 0, drop = 0;
        for (int64_t i = 0; i < n; ++i) {
            const or_path* p = &cur[i];
            const or_hitrec* v = &vx[i];
            float qu;
            uint32_t base;
            uint32_t X = or_split_one(F32, (float)qbuf[i], a->seed_lo, a->seed_hi, a->frame,
                                      p->pixel, p->sample, (uint32_t)depth, p->lineage, &qu, &base);
            if (a->rec) {
                double* r = a->rec + ((int64_t)(depth - 1) * cap + i) * OR_REC;
                for (int c = 0; c < 3; ++c) r[6 + c] = p->t[c];
                r[9] = qbuf[i];
                r[10] = (double)qu;
                r[11] = (double)X;
                r[12] = (double)S;
                r[13] = (double)p->pixel;
                for (int c = 0; c < 16; ++c) r[14 + c] = v->feat[c];
            }
            if (trace) {
                uint32_t* r = trace + ((int64_t)(depth - 1) * cap + i) * 5;
                r[0] = p->pixel; r[1] = p->sample; r[2] = p->lineage;
                r[3] = v->tri < 0 ? OR_NO_HIT : (uint32_t)v->tri;
                r[4] = X;
            }
            const or_material* m = v->tri >= 0 ? &s->mats[s->mat_id[v->tri]] : NULL;
            for (uint32_t j = 0; j < X; ++j) {
                int64_t slot = S + j;
                if (slot >= cap) { ++drop; continue; }
                if (slot >= room) {
                    free(cur); free(nxt); free(vx); free(acc); free(qbuf); free(E.tri); free(E.cdf);
                    return OR_ERR_OOM;
                }
                or_path* c = &nxt[slot];
                c->pixel = p->pixel;
                c->sample = p->sample;
                c->lineage = base + j * OR_LINEAGE_STEP;
                uint32_t w[4];
                or_draw(a->seed_lo, a->seed_hi, a->frame, c->pixel, c->sample, (uint32_t)depth,
                        OR_PURPOSE_BSDF, c->lineage, w);
                double wi[3], wt[3];
                double wo[3] = {-p->d[0], -p->d[1], -p->d[2]};
                if (m->type == 0) {
                    or_sample_lambert(v->n, or_u01(w[1]), or_u01(w[2]), wi);
                    for (int k = 0; k < 3; ++k) wt[k] = m->albedo[k];
                } else {
                    double alb[3] = {m->albedo[0], m->albedo[1], m->albedo[2]};
                    or_sample_ggx(v->n, wo, alb, m->roughness, m->F0, or_u01(w[0]), or_u01(w[1]),
                                  or_u01(w[2]), wi, wt);
                }
                c->pdf = 0.0;
                if (a->nee) {  /* the density the direction was drawn with, for MIS */
                    double fc[3];
                    or_eval_bsdf(m, v->n, wo, wi, fc, &c->pdf);
                }
                for (int k = 0; k < 3; ++k) {
                    c->o[k] = v->p[k] + OR_RAY_OFFSET * v->n[k];
                    c->d[k] = wi[k];
                    c->t[k] = p->t[k] * wt[k] / (double)qu;
                }
            }
            S += X;
        }
        if (trace_count) trace_count[depth - 1] = n;
        st->requested[depth] = S;
        st->dropped[depth] = drop;
        if (drop > 0) alpha *= 0.99; /* Eq. f_rate_prime with epsilon = 0.01 */
        or_path* tmp = cur; cur = nxt; nxt = tmp;
        n = S < cap ? S : cap;
    }
    for (int64_t i = 0; i < npix * 3; ++i) out_rgb[i] = acc[i] / (double)spp;
    if (a->rec) {
        /* reverse pass, deepest depth first */
        for (int32_t d = D; d >= 1; --d) {
            const int64_t nd = st->live[d];
            const int64_t nn = d < D ? st->live[d + 1] : 0;
            for (int64_t i = 0; i < nd; ++i) {
                double* r = a->rec + ((int64_t)(d - 1) * cap + i) * OR_REC;
                for (int c = 0; c < 3; ++c) r[c] = r[3 + c];
                const int64_t first = (int64_t)r[12], X = (int64_t)r[11];
                for (int64_t j = first; j < first + X && j < nn; ++j) {
                    const double* ch = a->rec + ((int64_t)d * cap + j) * OR_REC;
                    for (int c = 0; c < 3; ++c) r[c] += ch[c];
                }
            }
        }
    }
    free(cur); free(nxt); free(vx); free(acc); free(qbuf); free(E.tri); free(E.cdf);
    return OR_OK;
}
