// Wavefront bounce kernels for sm_103a: camera rays, shading (emission deposit, RRS
// factor), normalization, split counts + compaction, and the per-pixel accumulation
// (the closest-hit traversal is in trace.cu).  The method: "NRRS: Neural Russian Roulette and Splitting",
// Sec. 2 (Eq. rrs_factor), Sec. 3.1 (Eq. q_norm, F_norm, q_norm_rate, f_rate_prime),
// Sec. 4 (network, Eq. rrsnet_activation, "Compromise").
#include <cfloat>
#include <cstdio>

#include "tc.cuh"
#include "wavefront.cuh"

namespace nrrs {

namespace {

constexpr int kSplitThreads = 256;
constexpr int kReduceThreads = 1024;
constexpr uint32_t kMaxX = 1u << 23;  // q_used >= 2^23 has no fractional part in FP32

__device__ __forceinline__ uint32_t fbits(float f) { return __float_as_uint(f); }
__device__ __forceinline__ float bitsf(uint32_t u) { return __uint_as_float(u); }

__device__ __forceinline__ V3 tri_geom_normal(const SceneView& sc, int slot, int* mat) {
    const float4 t1 = __ldg(&sc.tris[3 * slot + 1]);
    const float4 t2 = __ldg(&sc.tris[3 * slot + 2]);
    *mat = (int)fbits(t1.w);
    return normalize3(cross3(xyz(t1), xyz(t2)));
}

__device__ __forceinline__ float boxcox(float t, float lambda) {
    if (lambda == 0.5f) return 2.0f * (sqrtf(t) - 1.0f);
    if (lambda == 0.0f) return logf(t);
    return (powf(t, lambda) - 1.0f) / lambda;
}

// The throughput heuristic (HEUR): q = min(lum(t) / max(I_px, eps_I), q_max) with I_px the
// mean over RGB of the reference pixel; q = lum(t) before any reference exists.
__device__ __forceinline__ float heur_factor(float4 t4, const RenderParams& rp, uint32_t pix,
                                            int has_ref, float eps_I) {
    const float l = lum(t4.x, t4.y, t4.z);
    if (!has_ref) return l;
    const float* rr = rp.ref + 3 * (size_t)pix;
    const float den = fmaxf((rr[0] + rr[1] + rr[2]) / 3.0f, eps_I);
    return den > 0.0f ? fminf(l / den, rp.q_max) : rp.q_max;
}

// A vertex whose RRSNet factor was non-finite (kQRepair) takes the heuristic's factor, so
// a failing network degrades to plain heuristic normalised RRS instead of ending paths.
__device__ __forceinline__ float repaired_q(const WorkView& w, QueueView cur,
                                           const RenderParams& rp, long long i, float eps_I) {
    float q = w.q[i];
    if (q != kQRepair) return q;
    q = heur_factor(cur.t[i], rp, fbits(w.dep[i].w), w.st->has_ref, eps_I);
    if (!(q >= 0.0f && q <= FLT_MAX)) q = 0.0f;
    w.q[i] = q;
    return q;
}

// ------------------------------------------------------------------ RRS split rule
// Eq. rrs_factor with the factor scaled by F (Eq. q_norm / q_norm_rate), decided in
// FP32: q_used = F * q (one rounding), X = floor(q_used) + [U < q_used - floor(q_used)].
__device__ __forceinline__ uint32_t split_decide(float F, float q, uint32_t key0, uint32_t key1,
                                                 uint32_t pixel, uint32_t sample, uint32_t depth,
                                                 uint32_t lineage, float* q_used,
                                                 uint32_t* lineage_base) {
    const float qu = __fmul_rn(F, q);
    *q_used = qu;
    if (!(qu > 0.0f)) {
        *lineage_base = 0u;
        return 0u;
    }
    const float k = floorf(qu);
    const float r = __fsub_rn(qu, k);
    const U4 w = draw(key0, key1, pixel, sample, depth, kPurposeRrs, lineage);
    *lineage_base = w.y;
    uint32_t X = (k >= (float)kMaxX ? kMaxX : (uint32_t)k) + (u01(w.x) < r ? 1u : 0u);
    return X > kMaxX ? kMaxX : X;
}

// ------------------------------------------------------------------ BSDF sampling
__device__ __forceinline__ void onb(V3 n, V3* b1, V3* b2) {  // Duff et al. 2017
    const float sign = copysignf(1.0f, n.z);
    const float a = -1.0f / (sign + n.z);
    const float b = n.x * n.y * a;
    *b1 = v3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    *b2 = v3(b, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ V3 cosine_dir(V3 n, float u1, float u2) {  // Shirley & Chiu 1997
    const float a = 2.0f * u1 - 1.0f, b = 2.0f * u2 - 1.0f;
    float x = 0.0f, y = 0.0f;
    if (a != 0.0f || b != 0.0f) {
        float r, phi;
        if (fabsf(a) > fabsf(b)) {
            r = a;
            phi = 0.785398163397448f * (b / a);
        } else {
            r = b;
            phi = 1.570796326794897f - 0.785398163397448f * (a / b);
        }
        float s, c;
        sincosf(phi, &s, &c);
        x = r * c;
        y = r * s;
    }
    const float z = sqrtf(fmaxf(0.0f, 1.0f - x * x - y * y));
    V3 b1, b2;
    onb(n, &b1, &b2);
    return b1 * x + b2 * y + n * z;
}

// GGX (Walter et al. 2007) + Lambert mixture, lobes picked with probability 1/2.
// Returns the weight f cos / pdf per channel (0 below the shading hemisphere) and, in
// pdf_out, the solid-angle pdf of the direction.
__device__ __forceinline__ V3 sample_ggx(V3 n, V3 wo, const nrrs_material& m, float ulobe,
                                         float u1, float u2, V3* wi_out, float* pdf_out) {
    const float a = m.roughness;
    V3 wi;
    if (ulobe < 0.5f) {
        const float tan2 = a * a * u1 / (1.0f - u1);
        const float cos_h = 1.0f / sqrtf(1.0f + tan2);
        const float sin_h = sqrtf(fmaxf(0.0f, 1.0f - cos_h * cos_h));
        float s, c;
        sincosf(6.283185307179586f * u2, &s, &c);
        V3 b1, b2;
        onb(n, &b1, &b2);
        const V3 h = b1 * (sin_h * c) + b2 * (sin_h * s) + n * cos_h;
        wi = h * (2.0f * dot3(wo, h)) - wo;
    } else {
        wi = cosine_dir(n, u1, u2);
    }
    *wi_out = wi;
    *pdf_out = 0.0f;
    const float cos_i = dot3(wi, n), cos_o = dot3(wo, n);
    if (cos_i <= 0.0f || cos_o <= 0.0f) return v3(0.0f, 0.0f, 0.0f);
    const V3 h = normalize3(wo + wi);
    const float cos_h = dot3(h, n), oh = dot3(wo, h);
    const float a2 = a * a;
    const float den = (a2 - 1.0f) * cos_h * cos_h + 1.0f;
    const float D = a2 / (3.141592653589793f * den * den);
    auto G1 = [&](float cw) {
        const float c2 = cw * cw;
        return 2.0f / (1.0f + sqrtf(1.0f + a2 * (1.0f - c2) / c2));
    };
    const float G = G1(cos_o) * G1(cos_i);
    const float om = 1.0f - dot3(wi, h);
    const float om2 = om * om;
    const float Fr = m.F0 + (1.0f - m.F0) * (om2 * om2 * om);
    const float spec = D * G * Fr / (4.0f * cos_o * cos_i);
    const float pdf = 0.5f * D * cos_h / (4.0f * fabsf(oh)) + 0.5f * cos_i / 3.141592653589793f;
    const float kd = (1.0f - m.F0) / 3.141592653589793f;
    const float s = cos_i / pdf;
    *pdf_out = pdf;
    return v3((spec + kd * m.albedo[0]) * s, (spec + kd * m.albedo[1]) * s,
              (spec + kd * m.albedo[2]) * s);
}

// f(wo, wi) cos_i per channel for a given direction, and the pdf with which the
// material's own sampling picks it (Lambertian: albedo / pi and cos_i / pi; the GGX
// mixture as sampled above).  Zero below the shading hemisphere.
__device__ __forceinline__ V3 bsdf_eval(V3 n, V3 wo, V3 wi, const nrrs_material& m, float* pdf) {
    const float cos_i = dot3(wi, n), cos_o = dot3(wo, n);
    *pdf = 0.0f;
    if (cos_i <= 0.0f || cos_o <= 0.0f) return v3(0.0f, 0.0f, 0.0f);
    constexpr float kInvPi = 0.318309886183791f;
    if (m.type == 0) {
        *pdf = cos_i * kInvPi;
        return v3(m.albedo[0] * kInvPi * cos_i, m.albedo[1] * kInvPi * cos_i,
                  m.albedo[2] * kInvPi * cos_i);
    }
    const float a = m.roughness, a2 = a * a;
    const V3 h = normalize3(wo + wi);
    const float cos_h = dot3(h, n), oh = dot3(wo, h);
    const float den = (a2 - 1.0f) * cos_h * cos_h + 1.0f;
    const float D = a2 / (3.141592653589793f * den * den);
    auto G1 = [&](float cw) {
        const float c2 = cw * cw;
        return 2.0f / (1.0f + sqrtf(1.0f + a2 * (1.0f - c2) / c2));
    };
    const float om = 1.0f - dot3(wi, h);
    const float om2 = om * om;
    const float Fr = m.F0 + (1.0f - m.F0) * (om2 * om2 * om);
    const float spec = D * G1(cos_o) * G1(cos_i) * Fr / (4.0f * cos_o * cos_i);
    const float kd = (1.0f - m.F0) * kInvPi;
    *pdf = 0.5f * D * cos_h / (4.0f * fabsf(oh)) + 0.5f * cos_i * kInvPi;
    return v3((spec + kd * m.albedo[0]) * cos_i, (spec + kd * m.albedo[1]) * cos_i,
              (spec + kd * m.albedo[2]) * cos_i);
}

// Power heuristic with exponent 2 (Veach 1997), the weight of the technique with
// density a against b, as 1 / (1 + (b / a)^2) so that large densities do not overflow.
__device__ __forceinline__ float power_heuristic(float a, float b) {
    const float r = b / a;
    return 1.0f / (1.0f + r * r);
}

// Next-event estimation at one vertex (hit point p, shading normal ns, outgoing wo,
// throughput t) from the NEE draw r: an emitter by area (r.x), a uniform point on it
// (sqrt(u1) (1 - u2), sqrt(u1) u2 along its edges; r.y, r.z) and the shadow ray from the
// offset origin to (1 - margin) of its distance.  The unoccluded contribution is
// t f cos_x Le w / p_light with p_light = dist^2 / (|cos_l| A) and w the power heuristic
// against the BSDF's pdf of the direction.  Writes the slot's shadow ray (t_max 0: none).
__device__ __forceinline__ void nee_vertex(const float4* __restrict__ emit,
                                           const float* __restrict__ cdf, int n_emit,
                                           float inv_area, const nrrs_material* mats, V3 p,
                                           V3 ns, V3 wo, const nrrs_material& m, float4 t4, U4 r,
                                           float4* sh_o, float4* sh_d, float4* sh_c) {
    *sh_o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (n_emit <= 0) return;
    const float u = u01(r.x);
    int lo = 0, hi = n_emit - 1;
    while (lo < hi) {  // first k with u < cdf[k]
        const int mid = (lo + hi) >> 1;
        if (u < __ldg(&cdf[mid])) hi = mid; else lo = mid + 1;
    }
    const float4 a0 = __ldg(&emit[3 * lo]), a1 = __ldg(&emit[3 * lo + 1]),
                 a2 = __ldg(&emit[3 * lo + 2]);
    const float su = sqrtf(u01(r.y)), u2 = u01(r.z);
    const V3 e1 = xyz(a1), e2 = xyz(a2);
    const V3 y = xyz(a0) + (e1 * (su * (1.0f - u2)) + e2 * (su * u2));
    const V3 org = p + ns * kRayOffset;
    const V3 v = y - org;
    const float dist2 = dot3(v, v);
    if (!(dist2 > 0.0f)) return;
    const float dist = sqrtf(dist2);
    const V3 wl = v * (1.0f / dist);
    const nrrs_material& me = mats[__float_as_uint(a0.w)];
    const float cos_l = -dot3(normalize3(cross3(e1, e2)), wl);
    if (!(cos_l > 0.0f || (me.two_sided && cos_l < 0.0f))) return;
    float pb;
    const V3 fc = bsdf_eval(ns, wo, wl, m, &pb);
    if (!(pb > 0.0f)) return;
    const float pl = dist2 * inv_area / fabsf(cos_l);
    const float s = power_heuristic(pl, pb) / pl;
    *sh_o = make_float4(org.x, org.y, org.z, dist * (1.0f - kShadowMargin));
    *sh_d = make_float4(wl.x, wl.y, wl.z, 0.0f);
    *sh_c = make_float4(t4.x * fc.x * me.Le[0] * s, t4.y * fc.y * me.Le[1] * s,
                        t4.z * fc.z * me.Le[2] * s, 0.0f);
}

// ------------------------------------------------------------------ kernels
// Sum of the reference image in FP32, in two fixed-order passes: one contiguous chunk per
// block, then the block sums (no FP64: the reference only sets the HEUR floor).
__global__ void k_ref_partial(const float* __restrict__ ref, long long n3, float* part) {
    __shared__ float sh[32];
    const long long chunk = (n3 + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n3 ? lo + chunk : n3;
    float s = 0.0f;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += ref[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_ref_prepare(const float* __restrict__ ref, long long n3, float eps_rel,
                              double alpha0, long long P, DevStats* st, const float* part,
                              int G) {
    __shared__ float sh[32];
    float s = 0.0f;
    if (ref)
        for (int b = threadIdx.x; b < G; b += blockDim.x) s += part[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        st->has_ref = ref != nullptr;
        st->eps_I = ref ? eps_rel * (s / (float)n3) : 0.0f;
        st->alpha_cur = alpha0;
        st->live[0] = P;
    }
}

__global__ void k_camera(CamView cam, RenderParams rp, QueueView out) {
    const long long P = (long long)rp.W * rp.H * rp.spp;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint32_t pixel = (uint32_t)(i / rp.spp), sample = (uint32_t)(i % rp.spp);
    const U4 w = draw(rp.fc->key0, rp.fc->key1, pixel, sample, 0u, kPurposeJitter, 0u);
    const int px = (int)(pixel % (uint32_t)rp.W), py = (int)(pixel / (uint32_t)rp.W);
    const float sx = (2.0f * ((float)px + u01(w.x)) / (float)rp.W - 1.0f) * cam.tan_half * cam.aspect;
    const float sy = (1.0f - 2.0f * ((float)py + u01(w.y)) / (float)rp.H) * cam.tan_half;
    const V3 fw = v3(cam.fw[0], cam.fw[1], cam.fw[2]);
    const V3 rt = v3(cam.right[0], cam.right[1], cam.right[2]);
    const V3 up = v3(cam.up[0], cam.up[1], cam.up[2]);
    const V3 d = normalize3(fw + (rt * sx + up * sy));
    out.o[i] = make_float4(cam.pos[0], cam.pos[1], cam.pos[2], bitsf(pixel));
    out.d[i] = make_float4(d.x, d.y, d.z, bitsf(0u));
    out.t[i] = make_float4(1.0f, 1.0f, 1.0f, bitsf(sample));
}

// Primary rays of a batched render: slot i belongs to the job whose primary range holds
// it; the job's camera and image size apply, and the random numbers are keyed by the
// job-local pixel (so each job sees the numbers a render of it alone would).
__global__ void k_camera_jobs(RenderParams rp, long long P, QueueView out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const JobDev* job = rp.jobs.job;
    int lo = 0, hi = rp.jobs.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&job[mid].prim_base) <= i) lo = mid; else hi = mid - 1;
    }
    const JobDev& J = job[lo];
    const long long li = i - J.prim_base;
    const uint32_t pixel = (uint32_t)(li / J.spp), sample = (uint32_t)(li % J.spp);
    const U4 w = draw(rp.fc->key0, rp.fc->key1, pixel, sample, 0u, kPurposeJitter, 0u);
    const CamView& cam = J.cam;
    const int px = (int)(pixel % (uint32_t)J.W), py = (int)(pixel / (uint32_t)J.W);
    const float sx = (2.0f * ((float)px + u01(w.x)) / (float)J.W - 1.0f) * cam.tan_half * cam.aspect;
    const float sy = (1.0f - 2.0f * ((float)py + u01(w.y)) / (float)J.H) * cam.tan_half;
    const V3 fw = v3(cam.fw[0], cam.fw[1], cam.fw[2]);
    const V3 rt = v3(cam.right[0], cam.right[1], cam.right[2]);
    const V3 up = v3(cam.up[0], cam.up[1], cam.up[2]);
    const V3 d = normalize3(fw + (rt * sx + up * sy));
    out.o[i] = make_float4(cam.pos[0], cam.pos[1], cam.pos[2],
                           bitsf((uint32_t)(J.pixel_base + pixel)));
    out.d[i] = make_float4(d.x, d.y, d.z, bitsf(0u));
    out.t[i] = make_float4(1.0f, 1.0f, 1.0f, bitsf(sample));
}

// Extension of depth `depth`, part 2, for slot i: the emission deposit, termination, and
// the RRS factor q_orig of the vertex; at NET depths the 16 features (f) and q = -1 for
// the network.  With NEE the emission found by BSDF sampling takes its MIS weight, and
// every vertex that goes on (the ones that get a factor) writes its shadow ray and
// contribution (so, sd, sk).  Returns q.
template <int KIND, bool NEE>
__device__ __forceinline__ float shade_slot(const SceneView& sc, const QueueView& cur,
                                            const WorkView& w, const RenderParams& rp,
                                            int depth, long long i, float eps_I, int has_ref,
                                            float4& dep, float4& so, float4& sd, float4& sk,
                                            float4 (&f)[4], unsigned int& nonfinite) {
    const float2 hh = w.hit[i];
    const int slot = __float_as_int(hh.y);
    const float4 o4 = cur.o[i];
    float q = 0.0f;
    dep = make_float4(0.0f, 0.0f, 0.0f, o4.w);
    so = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    sd = so;
    sk = so;
    if (slot >= 0) {
        const float4 d4 = cur.d[i];
        const float4 t4 = cur.t[i];
        int mi;
        const V3 ng = tri_geom_normal(sc, slot, &mi);
        const nrrs_material m = sc.mats[mi];
        const V3 d = xyz(d4);
        const bool front = dot3(ng, d) < 0.0f;
        // the job's depth limit, scene box, HEUR floor and emitters in a batched render
        int Dmax = rp.D;
        float lo3[3] = {sc.lo[0], sc.lo[1], sc.lo[2]};
        float ie3[3] = {sc.inv_ext[0], sc.inv_ext[1], sc.inv_ext[2]};
        float epsI = eps_I;
        uint32_t lpix = fbits(o4.w);
        const float4* emit = sc.emit;
        const float* ecdf = sc.emit_cdf;
        int n_emit = sc.n_emit;
        float inv_area = sc.inv_area;
        if (rp.jobs.job) {
            const int j = job_of_pixel(rp.jobs.job, rp.jobs.n, fbits(o4.w));
            const JobDev* J = rp.jobs.job + j;
            Dmax = J->D;
            for (int k = 0; k < 3; ++k) {
                lo3[k] = J->lo[k];
                ie3[k] = J->inv_ext[k];
            }
            epsI = rp.jobs.eps_I[j];
            lpix -= (uint32_t)J->pixel_base;
            if (NEE) {
                emit += 3 * (size_t)J->emit_base;
                ecdf += J->emit_base;
                n_emit = J->n_emit;
                inv_area = J->inv_area;
            }
        }
        if (front || m.two_sided) {
            float we = 1.0f;  // MIS weight against the previous vertex's emitter sample
            if (NEE && depth > 1 && n_emit > 0 &&
                (m.Le[0] > 0.0f || m.Le[1] > 0.0f || m.Le[2] > 0.0f)) {
                const float pb = cur.pdf[i];
                if (pb > 0.0f)
                    we = power_heuristic(pb, hh.x * hh.x * inv_area / fabsf(dot3(ng, d)));
            }
            dep.x = t4.x * m.Le[0] * we;
            dep.y = t4.y * m.Le[1] * we;
            dep.z = t4.z * m.Le[2] * we;
        }
        const bool black = m.albedo[0] == 0.0f && m.albedo[1] == 0.0f && m.albedo[2] == 0.0f;
        const bool dead = t4.x == 0.0f && t4.y == 0.0f && t4.z == 0.0f;
        if (!black && !dead && depth < Dmax) {
            if (NEE) {
                const U4 r = draw(rp.fc->key0, rp.fc->key1, lpix, fbits(t4.w),
                                  (uint32_t)depth, kPurposeNee, fbits(d4.w));
                const V3 ns = front ? ng : ng * -1.0f;
                nee_vertex(emit, ecdf, n_emit, inv_area, sc.mats, xyz(o4) + d * hh.x, ns,
                           d * -1.0f, m, t4, r, &so, &sd, &sk);
            }
            if (KIND == kFactorOne) {
                q = 1.0f;
            } else if (KIND == kFactorPlain) {
                q = fminf(1.0f, lum(t4.x, t4.y, t4.z));
            } else if (KIND == kFactorHeur) {
                q = heur_factor(t4, rp, fbits(o4.w), has_ref, epsI);
            } else {  // network depths (RRSNet or StatNet): features, q marked -1
                const V3 p = xyz(o4) + d * hh.x;
                const V3 ns = front ? ng : ng * -1.0f;
                f[0] = make_float4(
                    ie3[0] > 0.0f ? (p.x - lo3[0]) * ie3[0] : 0.5f,
                    ie3[1] > 0.0f ? (p.y - lo3[1]) * ie3[1] : 0.5f,
                    ie3[2] > 0.0f ? (p.z - lo3[2]) * ie3[2] : 0.5f, -d.x);
                f[1] = make_float4(-d.y, -d.z, ns.x, ns.y);
                f[2] = make_float4(ns.z, m.albedo[0], m.albedo[1], m.albedo[2]);
                f[3] = make_float4((float)depth / (float)Dmax, boxcox(t4.x, rp.boxcox_lambda),
                                   boxcox(t4.y, rp.boxcox_lambda),
                                   boxcox(t4.z, rp.boxcox_lambda));
                if (w.rough) w.rough[i] = m.type == 0 ? 1.0f : m.roughness;
                q = -1.0f;  // filled by the RRSNet kernel
            }
            if (KIND < kFactorNet && !(q >= 0.0f && q <= FLT_MAX)) {
                q = 0.0f;
                ++nonfinite;
            }
        }
    }
    return q;
}

// Extension of depth `depth`, part 2 (fixed grid-stride, coherent): shade_slot for every
// live slot; NET depths store the features for the RRSNet kernel.  Non-NET depths also
// write the block's FP64 partial sum of q (fixed assignment, so the sum is reproducible).
template <int KIND, bool NEE>
__global__ void __launch_bounds__(256)
k_shade(SceneView sc, QueueView cur, WorkView w, RenderParams rp, int depth) {
    __shared__ double sh[32];
    DevStats* st = w.st;
    const long long n = st->live[depth - 1];
    const int has_ref = st->has_ref;
    const float eps_I = st->eps_I;
    double qsum = 0.0;
    unsigned int nonfinite = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float4 dep, so, sd, sk, f[4];
        const float q = shade_slot<KIND, NEE>(sc, cur, w, rp, depth, i, eps_I, has_ref, dep, so,
                                              sd, sk, f, nonfinite);
        if (KIND >= kFactorNet && q == -1.0f) {  // RRSNet or StatNet (ADRRS) depths
            float4* fo = w.feat + 4 * i;
            fo[0] = f[0];
            fo[1] = f[1];
            fo[2] = f[2];
            fo[3] = f[3];
        }
        w.q[i] = q;
        w.dep[i] = dep;
        if (NEE) {
            w.sh_o[i] = so;
            if (so.w > 0.0f) {
                w.sh_d[i] = sd;
                w.sh_c[i] = sk;
            }
        }
        if (KIND < kFactorNet) qsum += (double)q;
    }
    if (KIND < kFactorNet) {
        qsum = block_sum(qsum, sh);
        if (threadIdx.x == 0) w.part[blockIdx.x] = qsum;
    }
    nonfinite = warp_sum(nonfinite);
    if ((threadIdx.x & 31) == 0 && nonfinite) {
        atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
        atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
    }
}

// NET depths in one pass (shade and RRSNet fused): each CTA of 128 threads shades 128
// consecutive slots (shade_slot), writes the features of the vertices that need a factor
// straight into shared memory as the BF16 operand of RRSNet's first layer (no round trip
// of the 64-byte feature rows through HBM), and runs the network on the tensor cores
// (tc_hidden_layers, tc_output), so the factor replaces the -1 mark before q is stored.
// The factors equal those k_rrsnet_tc computes from the same features, bit for bit; a
// non-finite one is stored as kQRepair for k_sum_q to replace by the heuristic's.
template <bool SPLIT, bool NEE>
__global__ void __launch_bounds__(kTcThreads, 6)
k_shade_rrsnet_tc(SceneView sc, QueueView cur, WorkView w, RenderParams rp, int depth) {
    __shared__ TcSmem<SPLIT> sm;
    DevStats* st = w.st;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long n = st->live[depth - 1];
    if ((long long)blockIdx.x * kTcThreads >= n) return;  // no tile: allocate nothing
    tc_setup(&sm.tmem, &sm.bar, kTmemCols);
    tc_stage_weights<SPLIT>(sm, rp.params, tid);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t bar = smem_u32(&sm.bar);
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    const int has_ref = st->has_ref;
    const float eps_I = st->eps_I;
    uint32_t phase = 0;
    unsigned int evals = 0, nonfinite = 0, shade_bad = 0;  // shade_bad stays 0 at NET depths
    bool failed = false;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long i = tile * kTcThreads + tid;
        float q = 0.0f;
        float x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = 0.0f;
        if (i < n) {
            float4 dep, so, sd, sk, f[4];
            q = shade_slot<kFactorNet, NEE>(sc, cur, w, rp, depth, i, eps_I, has_ref, dep, so,
                                            sd, sk, f, shade_bad);
            w.dep[i] = dep;
            if (NEE) {
                w.sh_o[i] = so;
                if (so.w > 0.0f) {
                    w.sh_d[i] = sd;
                    w.sh_c[i] = sk;
                }
            }
            if (q == -1.0f) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    x[4 * k] = f[k].x; x[4 * k + 1] = f[k].y;
                    x[4 * k + 2] = f[k].z; x[4 * k + 3] = f[k].w;
                }
            }
        }
        const bool net = i < n && q == -1.0f;
        tc_store_input<SPLIT>(sm, tid, x);
        float h[32];
        if (!tc_hidden_layers<SPLIT>(sm, tmem, bar, taddr, phase, h)) {
            failed = true;
            break;
        }
        if (net) {
            q = tc_output(sm.w4, h);
            ++evals;
            if (!(q >= 0.0f && q <= FLT_MAX)) {
                q = kQRepair;
                ++nonfinite;
            }
        }
        if (i < n) w.q[i] = q;
        fence_before();
        __syncthreads();  // TMEM reads done before the next tile's MMA overwrites it
    }
    if (failed && tid == 0) atomicOr(&st->status, (unsigned int)NRRS_STATUS_TIMEOUT);
    evals = warp_sum(evals);
    nonfinite = warp_sum(nonfinite);
    if ((tid & 31) == 0) {
        if (evals) atomicAdd(&st->net_evals, (unsigned long long)evals);
        if (nonfinite) {
            atomicAdd(&st->nonfinite, (unsigned long long)nonfinite);
            atomicOr(&st->status, (unsigned int)NRRS_STATUS_NONFINITE);
        }
    }
    tc_teardown(tmem, kTmemCols);
}

// FP64 partial sums of q over a fixed grid-stride assignment, so Sigma q is reproducible;
// non-finite network factors are replaced by the heuristic's on the way.
__global__ void __launch_bounds__(256) k_sum_q(WorkView w, QueueView cur, RenderParams rp,
                                               int depth) {
    __shared__ double sh[32];
    const long long n = w.st->live[depth - 1];
    const float eps_I = w.st->eps_I;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s += (double)repaired_q(w, cur, rp, i, eps_I);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) w.part[blockIdx.x] = s;
}

// Eq. F_norm / q_norm_rate / f_rate_prime, downscale only:
// F = min(1, f_rate * alpha * N_px / sum q), computed in FP64 and rounded to FP32.
__global__ void k_normalize_depth(WorkView w, RenderParams rp, int depth, int normalized) {
    __shared__ double sh[32];
    DevStats* st = w.st;
    double s = 0.0;
    for (int b = threadIdx.x; b < w.grid_red; b += blockDim.x) s += w.part[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        const double alpha = st->alpha_cur;
        double F = 1.0;
        if (normalized && s > 0.0) {
            F = (double)rp.f_rate * alpha * rp.budget / s;
            if (F > 1.0) F = 1.0;
        }
        st->sum_q[depth - 1] = s;
        st->alpha[depth - 1] = alpha;
        st->F[depth - 1] = (float)F;
        st->F_cur = (float)F;
    }
}

__device__ __forceinline__ void block_range(long long n, int* tiles_out, long long* begin,
                                            long long* end) {
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long chunk = ((per + kSplitThreads - 1) / kSplitThreads) * kSplitThreads;
    *begin = (long long)blockIdx.x * chunk;
    *end = *begin + chunk < n ? *begin + chunk : n;
    *tiles_out = *begin < *end ? (int)((*end - *begin + kSplitThreads - 1) / kSplitThreads) : 0;
}

// ------------------------------------------------------------------ batched renders
// Eq. F_norm per job: the queue holds the jobs one after another (it stays sorted by
// global pixel), so each block's contiguous slot range meets few jobs; the block writes
// an FP64 partial sum of q and a slot count for every job (zero where it meets none).
__global__ void __launch_bounds__(kSplitThreads) k_sum_q_jobs(WorkView w, QueueView cur,
                                                              RenderParams rp, int depth) {
    __shared__ double shd[32];
    __shared__ unsigned long long shc[32];
    const JobWork& J = rp.jobs;
    const long long n = w.st->live[depth - 1];
    long long begin, end;
    int tiles;
    block_range(n, &tiles, &begin, &end);
    double* part = J.part + (size_t)blockIdx.x * J.n;
    long long* cnt = J.cnt + (size_t)blockIdx.x * J.n;
    int j0 = 0, j1 = -1;
    if (begin < end) {
        j0 = job_of_pixel(J.job, J.n, fbits(w.dep[begin].w));
        j1 = job_of_pixel(J.job, J.n, fbits(w.dep[end - 1].w));
    }
    for (int j = threadIdx.x; j < J.n; j += blockDim.x)
        if (j < j0 || j > j1) {
            part[j] = 0.0;
            cnt[j] = 0;
        }
    for (long long i = begin + threadIdx.x; i < end; i += blockDim.x)
        if (w.q[i] == kQRepair)
            repaired_q(w, cur, rp, i,
                       J.eps_I[job_of_pixel(J.job, J.n, fbits(w.dep[i].w))]);
    __syncthreads();
    for (int j = j0; j <= j1; ++j) {
        const long long pb = J.job[j].pixel_base;
        const long long pe = j + 1 < J.n ? J.job[j + 1].pixel_base : 0x7FFFFFFFFFFFll;
        double s = 0.0;
        unsigned long long c = 0;
        for (long long i = begin + threadIdx.x; i < end; i += blockDim.x) {
            const long long pix = fbits(w.dep[i].w);
            if (pix >= pb && pix < pe) {
                s += (double)w.q[i];
                ++c;
            }
        }
        s = block_sum(s, shd);
        c = block_sum(c, shc);
        if (threadIdx.x == 0) {
            part[j] = s;
            cnt[j] = (long long)c;
        }
    }
}

// F_j = min(1, f_rate * alpha * N_j / sum_j q) with job j's budget N_j, summed over the
// blocks in a fixed order.
__global__ void k_normalize_jobs(WorkView w, RenderParams rp, int depth, int normalized,
                                 int G) {
    const JobWork& J = rp.jobs;
    DevStats* st = w.st;
    const double alpha = st->alpha_cur;
    for (int j = threadIdx.x; j < J.n; j += blockDim.x) {
        double s = 0.0;
        long long c = 0;
        for (int b = 0; b < G; ++b) {
            s += J.part[(size_t)b * J.n + j];
            c += J.cnt[(size_t)b * J.n + j];
        }
        double F = 1.0;
        if (normalized && s > 0.0) {
            F = (double)rp.f_rate * alpha * (double)J.budget_factor * (double)J.job[j].prims / s;
            if (F > 1.0) F = 1.0;
        }
        J.F_cur[j] = (float)F;
        J.F[(size_t)(depth - 1) * J.n + j] = (float)F;
        J.sum_q[(size_t)(depth - 1) * J.n + j] = s;
        J.live[(size_t)(depth - 1) * J.n + j] = c;
    }
    if (threadIdx.x == 0) {
        st->alpha[depth - 1] = alpha;
        st->F[depth - 1] = 0.0f;  // per job: see JobWork::F
        st->F_cur = 0.0f;
    }
}

// HEUR floor per job: eps_rel * mean of the reference over the job's pixels.
__global__ void k_ref_prepare_jobs(const float* __restrict__ ref, RenderParams rp, float eps_rel) {
    __shared__ float sh[32];
    const int j = blockIdx.x;
    const JobDev& J = rp.jobs.job[j];
    const long long n3 = 3ll * J.W * J.H;
    float s = 0.0f;
    if (ref)
        for (long long i = threadIdx.x; i < n3; i += blockDim.x) s += ref[3 * J.pixel_base + i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) rp.jobs.eps_I[j] = ref ? eps_rel * (s / (float)n3) : 0.0f;
}

// The decision trace of slot i at `depth` (tests): (pixel, sample, lineage, original
// triangle id or kNoHit, X) at its slot, or with a pixel mask a compact row
// (depth, pixel, sample, lineage, triangle, X) for marked pixels only.
__device__ __forceinline__ void trace_record(const SceneView& sc, const WorkView& w,
                                             const RenderParams& rp, int depth, long long i,
                                             float4 o4, float4 d4, float4 t4, uint32_t X) {
    const int slot = __float_as_int(w.hit[i].y);
    const uint32_t tri = slot < 0 ? kNoHit : fbits(__ldg(&sc.tris[3 * slot].w));
    const uint32_t pix = fbits(o4.w);
    if (rp.trace_mask) {
        if (!rp.trace_mask[pix]) return;
        const unsigned long long k = atomicAdd(rp.trace_count, 1ull);
        if (k >= (unsigned long long)rp.trace_rows) return;
        uint32_t* r = rp.trace + (size_t)k * 6;
        r[0] = (uint32_t)depth;
        r[1] = pix;
        r[2] = fbits(t4.w);
        r[3] = fbits(d4.w);
        r[4] = tri;
        r[5] = X;
        return;
    }
    uint32_t* r = rp.trace + ((size_t)(depth - 1) * rp.cap + i) * 5;
    r[0] = pix;
    r[1] = fbits(t4.w);
    r[2] = fbits(d4.w);
    r[3] = tri;
    r[4] = X;
}

__device__ __forceinline__ void kahan_add(float4* s_, float4* c_, float x, float y, float z) {
    float4 s = *s_, c = *c_;
    float in[3] = {x, y, z};
    float* sp[3] = {&s.x, &s.y, &s.z};
    float* cp[3] = {&c.x, &c.y, &c.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float yy = __fsub_rn(in[k], *cp[k]);
        const float t = __fadd_rn(*sp[k], yy);
        *cp[k] = __fsub_rn(__fsub_rn(t, *sp[k]), yy);
        *sp[k] = t;
    }
    *s_ = s;
    *c_ = c;
}

// Split counts of depth `depth` per block (Eq. rrs_factor), the optional trace, and the
// per-pixel accumulation of this depth's deposits: the queue is sorted by pixel, so the
// first slot of each pixel's run sums the run in order and adds it to the pixel's
// Kahan pair (deterministic, no atomics).
__global__ void __launch_bounds__(kSplitThreads)
k_split_count(SceneView sc, QueueView cur, WorkView w, RenderParams rp, int depth, int do_split) {
    __shared__ unsigned long long sh[32];
    DevStats* st = w.st;
    const uint32_t key0 = rp.fc->key0, key1 = rp.fc->key1;
    const long long n = st->live[depth - 1];
    const float F = st->F_cur;
    long long begin, end;
    int tiles;
    block_range(n, &tiles, &begin, &end);
    unsigned long long total = 0;
    for (int tile = 0; tile < tiles; ++tile) {
        const long long i = begin + (long long)tile * kSplitThreads + threadIdx.x;
        uint32_t X = 0;
        if (i < end) {
            const float4 dep = w.dep[i];
            const uint32_t pix = fbits(dep.w);
            const bool head = i == 0 || fbits(w.dep[i - 1].w) != pix;
            if (head) {
                float sx = dep.x, sy = dep.y, sz = dep.z;
                // the run's deposits in order, eight loads in flight at a time
                bool more = true;
                for (long long j0 = i + 1; more && j0 < n; j0 += 8) {
                    float4 e[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        e[k] = j0 + k < n ? w.dep[j0 + k] : make_float4(0.f, 0.f, 0.f, bitsf(~pix));
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (!more || fbits(e[k].w) != pix) {
                            more = false;
                        } else {
                            sx += e[k].x; sy += e[k].y; sz += e[k].z;
                        }
                    }
                }
                kahan_add(&w.acc_s[pix], &w.acc_c[pix], sx, sy, sz);
            }
            if (do_split || rp.trace) {
                const float4 o4 = cur.o[i];
                const float4 d4 = cur.d[i];
                const float4 t4 = cur.t[i];
                float qu;
                uint32_t base;
                float Fi = F;
                uint32_t lpix = fbits(o4.w);
                if (rp.jobs.job) {  // the job's factor; random numbers by job-local pixel
                    const int j = job_of_pixel(rp.jobs.job, rp.jobs.n, lpix);
                    Fi = rp.jobs.F_cur[j];
                    lpix -= (uint32_t)rp.jobs.job[j].pixel_base;
                }
                X = split_decide(Fi, w.q[i], key0, key1, lpix, fbits(t4.w),
                                 (uint32_t)depth, fbits(d4.w), &qu, &base);
                if (rp.trace) trace_record(sc, w, rp, depth, i, o4, d4, t4, X);
            }
        }
        total += (unsigned long long)X;
    }
    if (!do_split) return;
    total = block_sum(total, sh);
    if (threadIdx.x == 0) w.bcnt[blockIdx.x] = total;
}

// Exclusive scan of the per-block counts in 64-bit; sets the next queue length
// min(S, C), the drop count and the alpha back-off (Eq. f_rate_prime, epsilon 0.01).
__device__ void scan_counts(const unsigned long long* cnt, unsigned long long* off, int G,
                            unsigned long long* total_out) {
    __shared__ unsigned long long sh[kReduceThreads];
    const int per = (G + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    unsigned long long s = 0;
    for (int k = 0; k < per && b0 + k < G; ++k) s += cnt[b0 + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over thread sums (1024 entries, 10 steps)
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned long long v = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0ull;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = sh[threadIdx.x] - s;
    for (int k = 0; k < per && b0 + k < G; ++k) {
        off[b0 + k] = run;
        run += cnt[b0 + k];
    }
    if (threadIdx.x == blockDim.x - 1) *total_out = sh[threadIdx.x];
}

// Split of depth `depth` in one pass (count, compaction and scatter fused; Eq. rrs_factor
// and the bounded queue of Sec. 3.1).  Blocks claim 256-slot tiles in order; each tile
// decides every parent's X, finds its first child slot by a decoupled look-back over the
// earlier tiles' published counts (aggregate, or inclusive prefix once known) while the
// other warps add the tile's deposits per pixel run (run heads, as k_split_count), then
// writes its children.  Tiles
// are claimed in increasing order by running blocks, so every tile waited on belongs to
// a block that is running or done; each wait is bounded all the same (a timeout sets
// NRRS_STATUS_TIMEOUT and the tile drops its children rather than hang).  The last tile
// sets the next queue length, the drop count and the alpha back-off (Eq. f_rate_prime).
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagInclusive = 2ull << 62;
constexpr unsigned long long kFlagValue = (1ull << 62) - 1ull;
constexpr long long kLookbackCycles = 2000000000ll;  // ~1 s

__global__ void __launch_bounds__(kSplitThreads, 4)
k_split_fused(SceneView sc, QueueView cur, QueueView nxt, WorkView w, RenderParams rp,
              int depth) {
    __shared__ uint32_t sh[33];
    __shared__ long long s_tile;
    __shared__ unsigned long long s_excl;
    __shared__ int s_ok;
    DevStats* st = w.st;
    const uint32_t key0 = rp.fc->key0, key1 = rp.fc->key1;
    const long long n = st->live[depth - 1];
    const float F = st->F_cur;
    const long long tiles = (n + kSplitThreads - 1) / kSplitThreads;
    unsigned long long* ctr = &st->tiles[depth - 1];
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ctr, 1ull);
        __syncthreads();
        const long long t = s_tile;
        if (t >= tiles) break;
        const long long i = t * kSplitThreads + threadIdx.x;
        uint32_t X = 0, base = 0, lpix = 0;
        float qu = 0.0f;
        // a parent with children: its hit and hit triangle's edges, fetched ahead so that
        // their latency overlaps the scan and the look-back (the path state is read
        // again for the children instead of being held across them)
        float2 hh = make_float2(0.f, 0.f);
        float4 te1 = make_float4(0.f, 0.f, 0.f, 0.f), te2 = te1;
        if (i < n) {
            const float4 o4 = cur.o[i];
            const float4 d4 = cur.d[i];
            const float4 t4 = cur.t[i];
            hh = w.hit[i];
            float Fi = F;
            lpix = fbits(o4.w);
            if (rp.jobs.job) {  // the job's factor; random numbers by job-local pixel
                const int j = job_of_pixel(rp.jobs.job, rp.jobs.n, lpix);
                Fi = rp.jobs.F_cur[j];
                lpix -= (uint32_t)rp.jobs.job[j].pixel_base;
            }
            X = split_decide(Fi, w.q[i], key0, key1, lpix, fbits(t4.w), (uint32_t)depth,
                             fbits(d4.w), &qu, &base);
            if (rp.trace) trace_record(sc, w, rp, depth, i, o4, d4, t4, X);
            if (X > 0) {
                const int slot = __float_as_int(hh.y);
                te1 = __ldg(&sc.tris[3 * slot + 1]);
                te2 = __ldg(&sc.tris[3 * slot + 2]);
            }
        }
        uint32_t tile_total;
        const uint32_t pre = block_exclusive_scan(X, sh, &tile_total);
        if (threadIdx.x < 32) {  // warp 0: publish, then look back 32 tiles at a time
            const int lane = threadIdx.x;
            unsigned long long excl = 0;
            int ok = 1;
            if (lane == 0)
                atomicExch(&w.flags[t], (t == 0 ? kFlagInclusive : kFlagAggregate) | tile_total);
            const long long t0 = clock64();
            for (long long base = t - 1; base >= 0;) {
                const long long j = base - lane;  // lane 0 is the nearest predecessor
                const unsigned long long f =
                    j >= 0 ? *reinterpret_cast<volatile unsigned long long*>(&w.flags[j])
                           : (2ull << 62);  // before tile 0: an inclusive prefix of 0
                const unsigned incl = __ballot_sync(0xffffffffu, (f >> 62) == 2ull);
                const unsigned none = __ballot_sync(0xffffffffu, (f >> 62) == 0ull);
                const int stop = incl ? __ffs(incl) - 1 : 31;  // the window's last lane needed
                const unsigned need = stop == 31 ? 0xffffffffu : (2u << stop) - 1u;
                if (none & need) {  // a nearer tile has not published yet
                    if (clock64() - t0 > kLookbackCycles) {
                        ok = 0;
                        break;
                    }
                    continue;
                }
                excl += warp_sum(lane <= stop ? (f & kFlagValue) : 0ull);
                if (incl) break;
                base -= 32;
            }
            if (lane == 0) {
                if (t > 0) atomicExch(&w.flags[t], kFlagInclusive | (excl + tile_total));
                s_excl = excl;
                s_ok = ok;
                if (!ok) atomicOr(&st->status, (unsigned int)NRRS_STATUS_TIMEOUT);
                if (t == tiles - 1) {  // the whole depth's children are counted
                    const unsigned long long S = excl + tile_total;
                    const unsigned long long C = (unsigned long long)rp.cap;
                    const unsigned long long nn = S < C ? S : C;
                    st->requested[depth - 1] = (long long)S;
                    st->dropped[depth - 1] = (long long)(S - nn);
                    st->live[depth] = (long long)nn;
                    if (S > nn) {
                        st->alpha_cur *= 0.99;
                        st->status |= NRRS_STATUS_OVERFLOW_DROPPED;
                    }
                }
            }
        }
        // this depth's deposits, summed per pixel run by the run's first slot: after the
        // tile's count is published, so the serial run sums of the other warps overlap
        // warp 0's look-back instead of delaying the tiles that wait on this one
        if (i < n) {
            const float4 dep = w.dep[i];
            const uint32_t pix = fbits(dep.w);
            if (i == 0 || fbits(w.dep[i - 1].w) != pix) {
                float sx = dep.x, sy = dep.y, sz = dep.z;
                bool more = true;
                for (long long j0 = i + 1; more && j0 < n; j0 += 8) {
                    float4 e[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        e[k] = j0 + k < n ? w.dep[j0 + k] : make_float4(0.f, 0.f, 0.f, bitsf(~pix));
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (!more || fbits(e[k].w) != pix) {
                            more = false;
                        } else {
                            sx += e[k].x; sy += e[k].y; sz += e[k].z;
                        }
                    }
                }
                kahan_add(&w.acc_s[pix], &w.acc_c[pix], sx, sy, sz);
            }
        }
        __syncthreads();
        const unsigned long long first = s_excl + pre;
        if (rp.rec_first && i < n) {
            rp.rec_first[i] =
                (uint32_t)(first < (unsigned long long)rp.cap ? first : (unsigned long long)rp.cap);
            rp.rec_X[i] = X;
        }
        if (X > 0 && s_ok) {
            const float4 o4 = cur.o[i];
            const float4 d4 = cur.d[i];
            const float4 t4 = cur.t[i];
            const int mi = (int)fbits(te1.w);
            const V3 ng = normalize3(cross3(xyz(te1), xyz(te2)));
            const nrrs_material m = sc.mats[mi];
            const V3 d = xyz(d4);
            const V3 ns = dot3(ng, d) < 0.0f ? ng : ng * -1.0f;
            const V3 p = xyz(o4) + d * hh.x;
            const V3 org = p + ns * kRayOffset;
            const uint32_t smp = fbits(t4.w);
            const float iq = 1.0f / qu;
            for (uint32_t j = 0; j < X; ++j) {
                const unsigned long long dst = first + j;
                if (dst >= (unsigned long long)rp.cap) break;
                const uint32_t lin = base + j * kLineageStep;
                const U4 r = draw(key0, key1, lpix, smp, (uint32_t)depth, kPurposeBsdf, lin);
                V3 wi, wt;
                float pdf;
                if (m.type == 0) {
                    wi = cosine_dir(ns, u01(r.y), u01(r.z));
                    wt = v3(m.albedo[0], m.albedo[1], m.albedo[2]);
                    pdf = fmaxf(dot3(wi, ns), 0.0f) * 0.318309886183791f;
                } else {
                    wt = sample_ggx(ns, d * -1.0f, m, u01(r.x), u01(r.y), u01(r.z), &wi, &pdf);
                }
                if (rp.nee) nxt.pdf[dst] = pdf;  // for the MIS weight at the child's hit
                nxt.o[dst] = make_float4(org.x, org.y, org.z, o4.w);
                nxt.d[dst] = make_float4(wi.x, wi.y, wi.z, bitsf(lin));
                nxt.t[dst] = make_float4(t4.x * wt.x * iq, t4.y * wt.y * iq, t4.z * wt.z * iq, t4.w);
            }
        }
        __syncthreads();  // s_tile, s_excl and sh are reused by the next tile
    }
}

__global__ void k_finalize(WorkView w, RenderParams rp, float* __restrict__ rgb,
                           float* __restrict__ ref_mean, int update_ref, long long npix) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const float4 s = w.acc_s[p], c = w.acc_c[p];
    const int spp = rp.jobs.job ? rp.jobs.job[job_of_pixel(rp.jobs.job, rp.jobs.n, (uint32_t)p)].spp
                                : rp.spp;
    const float inv = 1.0f / (float)spp;
    const float r = (s.x - c.x) * inv, g = (s.y - c.y) * inv, b = (s.z - c.z) * inv;
    rgb[3 * p + 0] = r;
    rgb[3 * p + 1] = g;
    rgb[3 * p + 2] = b;
    if (update_ref && ref_mean) {
        // running mean of the frames so far (the reference I_px of Sec. 4 "Compromise")
        const float k = (float)rp.fc->ref_count;
        const float ik = 1.0f / (k + 1.0f);
        float* m = ref_mean + 3 * p;
        m[0] = (m[0] * k + r) * ik;
        m[1] = (m[1] * k + g) * ik;
        m[2] = (m[2] * k + b) * ik;
    }
}

// ------------------------------------------------------------------ plain-array entry points
__global__ void k_sum_part(const float* __restrict__ q, long long n, double* part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s += (double)q[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_norm_final(const double* part, int G, double budget, double f_rate, double alpha,
                             float* F_out, double* sum_out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) s += part[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        double F = 1.0;
        if (s > 0.0) {
            F = f_rate * alpha * budget / s;
            if (F > 1.0) F = 1.0;
        }
        *F_out = (float)F;
        *sum_out = s;
    }
}

__global__ void __launch_bounds__(kSplitThreads)
k_split_arr_count(SplitArrays a, unsigned long long* bcnt) {
    __shared__ unsigned long long sh[32];
    const float F = *a.F;
    long long begin, end;
    int tiles;
    block_range(a.n, &tiles, &begin, &end);
    unsigned long long total = 0;
    for (int tile = 0; tile < tiles; ++tile) {
        const long long i = begin + (long long)tile * kSplitThreads + threadIdx.x;
        if (i < end) {
            float qu;
            uint32_t base;
            const uint32_t X = split_decide(F, a.q[i], a.key0, a.key1, a.pixel[i], a.sample[i],
                                            a.depth, a.lineage[i], &qu, &base);
            a.X[i] = X;
            total += X;
        }
    }
    total = block_sum(total, sh);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = total;
}

__global__ void k_split_arr_scan(SplitArrays a, const unsigned long long* bcnt, unsigned long long* boff,
                                 int G) {
    __shared__ unsigned long long total;
    scan_counts(bcnt, boff, G, &total);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long C = (unsigned long long)a.cap;
        *a.total = (long long)total;
        *a.dropped = (long long)(total > C ? total - C : 0ull);
    }
}

__global__ void __launch_bounds__(kSplitThreads)
k_split_arr_scatter(SplitArrays a, const unsigned long long* boff) {
    __shared__ uint32_t sh[33];
    const float F = *a.F;
    long long begin, end;
    int tiles;
    block_range(a.n, &tiles, &begin, &end);
    unsigned long long carry = tiles ? boff[blockIdx.x] : 0ull;
    for (int tile = 0; tile < tiles; ++tile) {
        const long long i = begin + (long long)tile * kSplitThreads + threadIdx.x;
        uint32_t X = 0, base = 0;
        if (i < end) {
            float qu;
            X = split_decide(F, a.q[i], a.key0, a.key1, a.pixel[i], a.sample[i], a.depth,
                             a.lineage[i], &qu, &base);
        }
        uint32_t tile_total;
        const uint32_t pre = block_exclusive_scan(X, sh, &tile_total);
        if (i < end) a.prefix[i] = (long long)(carry + pre);
        for (uint32_t j = 0; j < X; ++j) {
            const unsigned long long dst = carry + pre + j;
            if (dst >= (unsigned long long)a.cap) break;
            a.child_parent[dst] = (uint32_t)i;
            a.child_lineage[dst] = base + j * kLineageStep;
        }
        carry += tile_total;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
int split_block_threads() { return kSplitThreads; }

void launch_ref_prepare(const float* ref, long long n3, float eps_rel, double alpha0, long long P,
                        DevStats* st, float* part, int G, cudaStream_t s) {
    if (ref) k_ref_partial<<<G, 256, 0, s>>>(ref, n3, part);
    k_ref_prepare<<<1, 256, 0, s>>>(ref, n3, eps_rel, alpha0, P, st, part, G);
}

void launch_camera(const CamView& cam, const RenderParams& rp, QueueView out, cudaStream_t s) {
    const long long P = (long long)rp.W * rp.H * rp.spp;
    const int threads = 256;
    k_camera<<<(unsigned)((P + threads - 1) / threads), threads, 0, s>>>(cam, rp, out);
}

void launch_shade(int kind, const SceneView& sc, QueueView cur, const WorkView& w,
                  const RenderParams& rp, int depth, cudaStream_t s) {
    const int G = w.grid_red;
#define NRRS_SHADE(K)                                                            \
    (rp.nee ? k_shade<K, true><<<G, 256, 0, s>>>(sc, cur, w, rp, depth)          \
            : k_shade<K, false><<<G, 256, 0, s>>>(sc, cur, w, rp, depth))
    switch (kind) {
        case kFactorOne: NRRS_SHADE(kFactorOne); break;
        case kFactorPlain: NRRS_SHADE(kFactorPlain); break;
        case kFactorHeur: NRRS_SHADE(kFactorHeur); break;
        case kFactorNet: NRRS_SHADE(kFactorNet); break;
        default: NRRS_SHADE(kFactorAdrrs); break;
    }
#undef NRRS_SHADE
}

void launch_shade_rrsnet(int precision, int n_sm, const SceneView& sc, QueueView cur,
                         const WorkView& w, const RenderParams& rp, int depth, cudaStream_t s) {
    const int G = n_sm * 6;  // persistent: six CTAs per SM stay resident
    if (precision == 17) {
        if (rp.nee)
            k_shade_rrsnet_tc<false, true><<<G, kTcThreads, 0, s>>>(sc, cur, w, rp, depth);
        else
            k_shade_rrsnet_tc<false, false><<<G, kTcThreads, 0, s>>>(sc, cur, w, rp, depth);
    } else {
        if (rp.nee)
            k_shade_rrsnet_tc<true, true><<<G, kTcThreads, 0, s>>>(sc, cur, w, rp, depth);
        else
            k_shade_rrsnet_tc<true, false><<<G, kTcThreads, 0, s>>>(sc, cur, w, rp, depth);
    }
}

void launch_sum_q(const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                  cudaStream_t s) {
    k_sum_q<<<w.grid_red, 256, 0, s>>>(w, cur, rp, depth);
}

void launch_normalize_depth(const WorkView& w, const RenderParams& rp, int depth, int normalized,
                            cudaStream_t s) {
    k_normalize_depth<<<1, kReduceThreads, 0, s>>>(w, rp, depth, normalized);
}

void launch_split_count(const SceneView& sc, QueueView cur, const WorkView& w,
                        const RenderParams& rp, int depth, int do_split, cudaStream_t s) {
    k_split_count<<<w.grid_split, kSplitThreads, 0, s>>>(sc, cur, w, rp, depth, do_split);
}

void launch_split_fused(const SceneView& sc, QueueView cur, QueueView nxt, const WorkView& w,
                        const RenderParams& rp, int depth, cudaStream_t s) {
    k_split_fused<<<w.grid_split, kSplitThreads, 0, s>>>(sc, cur, nxt, w, rp, depth);
}

void launch_finalize(const WorkView& w, const RenderParams& rp, float* rgb, float* ref_mean,
                     int update_ref, long long npix, cudaStream_t s) {
    k_finalize<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(w, rp, rgb, ref_mean, update_ref,
                                                               npix);
}

void launch_ref_prepare_jobs(const RenderParams& rp, float eps_rel, cudaStream_t s) {
    k_ref_prepare_jobs<<<rp.jobs.n, 1024, 0, s>>>(rp.ref, rp, eps_rel);
}

void launch_sum_q_jobs(const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                       cudaStream_t s) {
    k_sum_q_jobs<<<w.grid_red, kSplitThreads, 0, s>>>(w, cur, rp, depth);
}

void launch_normalize_jobs(const WorkView& w, const RenderParams& rp, int depth, int normalized,
                           cudaStream_t s) {
    k_normalize_jobs<<<1, 256, 0, s>>>(w, rp, depth, normalized, w.grid_red);
}

void launch_camera_jobs(const RenderParams& rp, long long P, QueueView out, cudaStream_t s) {
    k_camera_jobs<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(rp, P, out);
}

__global__ void k_frame_consts(FrameConsts* fc, uint32_t key0, uint32_t key1, int ref_count) {
    fc->key0 = key0;
    fc->key1 = key1;
    fc->ref_count = ref_count;
    fc->pad = 0;
}

void launch_frame_consts(FrameConsts* fc, uint32_t key0, uint32_t key1, int ref_count,
                         cudaStream_t s) {
    k_frame_consts<<<1, 1, 0, s>>>(fc, key0, key1, ref_count);
}


void launch_normalize_array(const float* q, long long n, double budget, double f_rate,
                            double alpha, double* part, int grid, float* F, double* sum,
                            cudaStream_t s) {
    k_sum_part<<<grid, 256, 0, s>>>(q, n, part);
    k_norm_final<<<1, kReduceThreads, 0, s>>>(part, grid, budget, f_rate, alpha, F, sum);
}

void launch_split_arrays(const SplitArrays& a, unsigned long long* bcnt, unsigned long long* boff,
                         int grid, cudaStream_t s) {
    k_split_arr_count<<<grid, kSplitThreads, 0, s>>>(a, bcnt);
    k_split_arr_scan<<<1, kReduceThreads, 0, s>>>(a, bcnt, boff, grid);
    k_split_arr_scatter<<<grid, kSplitThreads, 0, s>>>(a, boff);
}

}  // namespace nrrs
