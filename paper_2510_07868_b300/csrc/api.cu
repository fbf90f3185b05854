// C ABI of the NRRS bounce (include/nrrs.h): scene set-up, the per-depth launch
// sequence of one render, and the stand-alone stage entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bvh.h"
#include "wavefront.cuh"

using namespace nrrs;

namespace {

thread_local std::string g_last_error;

nrrs_status fail(nrrs_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

nrrs_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear sticky launch error state where possible
    return fail(e == cudaErrorMemoryAllocation ? NRRS_ERR_OOM : NRRS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

struct Workspace {
    long long cap = 0, npix = 0;
    int grid_red = 0, grid_split = 0;
    bool has_feat = false;
    float4* qo[2] = {nullptr, nullptr};
    float4* qd[2] = {nullptr, nullptr};
    float4* qt[2] = {nullptr, nullptr};
    float2* hit = nullptr;
    float* q = nullptr;
    float4* dep = nullptr;
    float4* feat = nullptr;
    double* part = nullptr;
    unsigned int* bcnt = nullptr;
    unsigned long long* boff = nullptr;
    float4* acc_s = nullptr;
    float4* acc_c = nullptr;
    DevStats* st = nullptr;

    void release() {
        for (int k = 0; k < 2; ++k) {
            cudaFree(qo[k]);
            cudaFree(qd[k]);
            cudaFree(qt[k]);
            qo[k] = qd[k] = qt[k] = nullptr;
        }
        cudaFree(hit); cudaFree(q); cudaFree(dep); cudaFree(feat); cudaFree(part); cudaFree(bcnt);
        cudaFree(boff); cudaFree(acc_s); cudaFree(acc_c); cudaFree(st);
        hit = nullptr; q = nullptr; dep = nullptr; feat = nullptr; part = nullptr; bcnt = nullptr;
        has_feat = false;
        boff = nullptr; acc_s = acc_c = nullptr; st = nullptr;
        cap = npix = 0;
    }
};

// Scratch for the plain-array stage entry points called without a scene.
struct Pool {
    double* part = nullptr;
    unsigned int* bcnt = nullptr;
    unsigned long long* boff = nullptr;
    int grid = 0;
};
std::mutex g_pool_mu;
std::map<int, Pool> g_pools;

int sm_count(int dev) {
    int n = 148;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

nrrs_status pool_for_device(int dev, Pool** out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    Pool& p = g_pools[dev];
    if (!p.part) {
        p.grid = sm_count(dev) * 8;
        CK(dalloc(&p.part, p.grid));
        CK(dalloc(&p.bcnt, p.grid));
        CK(dalloc(&p.boff, p.grid));
    }
    *out = &p;
    return NRRS_OK;
}

}  // namespace

namespace nrrs {
nrrs_status record_error(nrrs_status s, const char* msg) { return fail(s, msg); }
}  // namespace nrrs

struct nrrs_scene {
    int device = 0;
    int n_sm = 148;
    int64_t n_nodes = 0, n_tri = 0;
    float4* nodes = nullptr;
    float4* tris = nullptr;
    nrrs_material* mats = nullptr;
    float* params = nullptr;  // RRSNet weights, 2592 floats
    SceneView view{};
    CamView cam{};
    Workspace ws;
    int grid_trace = 0, grid_rrsnet = 0, grid_sum = 0;
    // running mean of earlier frames (HEUR reference), [npix * 3]
    float* ref_mean = nullptr;
    int ref_count = 0;
    int ref_w = 0, ref_h = 0;
    std::vector<cudaEvent_t> events;  // reused by profiled renders
};

namespace {

nrrs_status ensure_workspace(nrrs_scene* sc, long long cap, long long npix, bool need_feat) {
    Workspace& w = sc->ws;
    if (w.cap >= cap && w.npix >= npix && w.st) {
        if (need_feat && !w.has_feat) {
            CK(dalloc(&w.feat, (size_t)w.cap * 4));
            w.has_feat = true;
        }
        return NRRS_OK;
    }
    w.release();
    for (int k = 0; k < 2; ++k) {
        CK(dalloc(&w.qo[k], cap));
        CK(dalloc(&w.qd[k], cap));
        CK(dalloc(&w.qt[k], cap));
    }
    CK(dalloc(&w.hit, cap));
    CK(dalloc(&w.q, cap));
    CK(dalloc(&w.dep, cap));
    if (need_feat) {
        CK(dalloc(&w.feat, (size_t)cap * 4));
        w.has_feat = true;
    }
    w.grid_red = sc->grid_sum;
    w.grid_split = sc->n_sm * 8;
    CK(dalloc(&w.part, w.grid_red));
    CK(dalloc(&w.bcnt, w.grid_split));
    CK(dalloc(&w.boff, w.grid_split));
    CK(dalloc(&w.acc_s, npix));
    CK(dalloc(&w.acc_c, npix));
    CK(dalloc(&w.st, 1));
    w.cap = cap;
    w.npix = npix;
    return NRRS_OK;
}

void destroy(nrrs_scene* s) {
    if (!s) return;
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    s->ws.release();
    cudaFree(s->nodes);
    cudaFree(s->tris);
    cudaFree(s->mats);
    cudaFree(s->params);
    cudaFree(s->ref_mean);
    delete s;
}

struct V3d {
    double x, y, z;
};
V3d vcross(V3d a, V3d b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3d vnorm(V3d a) {
    double l = std::sqrt(a.x * a.x + a.y * a.y + a.z * a.z);
    return {a.x / l, a.y / l, a.z / l};
}

// Counts launches and, when profiling, brackets each launch with a pair of events on
// the launching stream.
struct StageTimer {
    nrrs_scene* sc;
    cudaStream_t s;
    bool on;
    int used = 0;
    unsigned launches = 0;
    std::vector<int> stage_of;
    cudaError_t begin(int stage) {
        ++launches;
        if (!on) return cudaSuccess;
        while ((int)sc->events.size() < used + 2) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            sc->events.push_back(e);
        }
        stage_of.push_back(stage);
        return cudaEventRecord(sc->events[used++], s);
    }
    cudaError_t end() {
        if (!on) return cudaSuccess;
        return cudaEventRecord(sc->events[used++], s);
    }
    void collect(nrrs_render_stats* st) {
        for (size_t k = 0; k < stage_of.size(); ++k) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, sc->events[2 * k], sc->events[2 * k + 1]) == cudaSuccess)
                st->stage_ms[stage_of[k]] += ms;
            st->stage_launches[stage_of[k]]++;
        }
    }
};

int factor_kind(int mode, uint64_t gate, int depth) {
    switch (mode) {
        case kNone: return kFactorOne;
        case kPlainRR: return kFactorPlain;
        case kHeurNorm: return kFactorHeur;
        case kNet: return kFactorNet;
        default: {
            const unsigned g = (unsigned)((gate >> (2 * (depth - 1))) & 3u);
            return g == kGateNet ? kFactorNet : g == kGateHeur ? kFactorHeur : kFactorOne;
        }
    }
}

}  // namespace

extern "C" {

const char* nrrs_status_string(nrrs_status s) {
    switch (s) {
        case NRRS_OK: return "ok";
        case NRRS_ERR_INVALID_ARG: return "invalid argument";
        case NRRS_ERR_CUDA: return "CUDA error";
        case NRRS_ERR_OOM: return "out of device memory";
        case NRRS_ERR_TIMEOUT: return "device wait timed out";
        case NRRS_ERR_NONFINITE: return "non-finite RRS factors";
        case NRRS_ERR_OVERFLOW_DROPPED: return "queue overflow, children dropped";
        case NRRS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* nrrs_last_error(void) { return g_last_error.c_str(); }

nrrs_status nrrs_create_scene(const float* tri, int32_t n_tri, const int32_t* tri_mat,
                              const nrrs_material* mats, int32_t n_mat, const nrrs_camera* cam,
                              int32_t device, nrrs_scene** out) {
    if (!out) return fail(NRRS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!tri || !tri_mat || !mats || !cam || n_tri < 1 || n_mat < 1)
        return fail(NRRS_ERR_INVALID_ARG, "NULL scene array or empty scene");
    for (int32_t i = 0; i < n_tri; ++i)
        if (tri_mat[i] < 0 || tri_mat[i] >= n_mat) return fail(NRRS_ERR_INVALID_ARG, "material id out of range");
    for (int32_t i = 0; i < n_mat; ++i)
        if (mats[i].type != 0 && mats[i].type != 1) return fail(NRRS_ERR_INVALID_ARG, "unknown material type");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(NRRS_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");

    BvhHost bvh;
    build_bvh(tri, n_tri, tri_mat, &bvh);

    nrrs_scene* s = new nrrs_scene();
    s->device = device;
    s->n_sm = sm_count(device);
    s->n_nodes = (int64_t)bvh.nodes.size();
    s->n_tri = n_tri;
    auto bail = [&](cudaError_t e, const char* what) {
        nrrs_status st = cuda_fail(e, what);
        destroy(s);
        return st;
    };
    cudaError_t e;
    if ((e = dalloc(&s->nodes, bvh.nodes.size() * 4)) != cudaSuccess) return bail(e, "alloc nodes");
    if ((e = dalloc(&s->tris, (size_t)bvh.n_ref * 3)) != cudaSuccess) return bail(e, "alloc tris");
    if ((e = dalloc(&s->mats, n_mat)) != cudaSuccess) return bail(e, "alloc mats");
    if ((e = dalloc(&s->params, kNParams)) != cudaSuccess) return bail(e, "alloc params");
    if ((e = cudaMemcpy(s->nodes, bvh.nodes.data(), bvh.nodes.size() * 64, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy nodes");
    if ((e = cudaMemcpy(s->tris, bvh.tris.data(), (size_t)bvh.n_ref * 48, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy tris");
    if ((e = cudaMemcpy(s->mats, mats, sizeof(nrrs_material) * n_mat, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy mats");
    if ((e = cudaMemset(s->params, 0, kNParams * sizeof(float))) != cudaSuccess) return bail(e, "zero params");

    s->view.nodes = s->nodes;
    s->view.tris = s->tris;
    s->view.mats = s->mats;
    for (int k = 0; k < 3; ++k) {
        s->view.lo[k] = bvh.lo[k];
        const float ext = bvh.hi[k] - bvh.lo[k];
        s->view.inv_ext[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
    }
    // camera basis in FP64, rounded once
    V3d fw = vnorm({cam->look[0], cam->look[1], cam->look[2]});
    V3d up = {cam->up[0], cam->up[1], cam->up[2]};
    V3d right = vnorm(vcross(up, fw));
    V3d up2 = vcross(fw, right);
    for (int k = 0; k < 3; ++k) s->cam.pos[k] = cam->pos[k];
    s->cam.fw[0] = (float)fw.x; s->cam.fw[1] = (float)fw.y; s->cam.fw[2] = (float)fw.z;
    s->cam.right[0] = (float)right.x; s->cam.right[1] = (float)right.y; s->cam.right[2] = (float)right.z;
    s->cam.up[0] = (float)up2.x; s->cam.up[1] = (float)up2.y; s->cam.up[2] = (float)up2.z;
    s->cam.tan_half = (float)std::tan(0.5 * (double)cam->vfov_deg * M_PI / 180.0);
    s->grid_trace = s->n_sm * max_blocks_trace();
    s->grid_rrsnet = s->n_sm * max_blocks_rrsnet();
    s->grid_sum = s->n_sm * 4;
    *out = s;
    return NRRS_OK;
}

nrrs_status nrrs_destroy_scene(nrrs_scene* scene) {
    if (!scene) return NRRS_OK;
    DeviceGuard g(scene->device);
    cudaDeviceSynchronize();
    destroy(scene);
    return NRRS_OK;
}

nrrs_status nrrs_scene_info(const nrrs_scene* scene, int64_t* n_nodes, int64_t* n_tri) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (n_nodes) *n_nodes = scene->n_nodes;
    if (n_tri) *n_tri = scene->n_tri;
    return NRRS_OK;
}

nrrs_status nrrs_set_rrsnet_params(nrrs_scene* scene, const float* params, int32_t n, void* stream) {
    if (!scene || !params || n != kNParams) return fail(NRRS_ERR_INVALID_ARG, "need 2592 host floats");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(scene->params, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

nrrs_status nrrs_get_rrsnet_params(nrrs_scene* scene, float* params, int32_t n, void* stream) {
    if (!scene || !params || n != kNParams) return fail(NRRS_ERR_INVALID_ARG, "need 2592 host floats");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(params, scene->params, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

nrrs_status nrrs_render(nrrs_scene* scene, int32_t width, int32_t height, int32_t spp,
                        int32_t max_depth, int32_t rrs_mode, const nrrs_render_opts* opts,
                        float* d_rgb, void* stream, nrrs_render_stats* stats) {
    if (!scene || !d_rgb) return fail(NRRS_ERR_INVALID_ARG, "scene or d_rgb is NULL");
    if (width < 1 || height < 1 || spp < 1 || max_depth < 1 || max_depth > NRRS_MAX_DEPTH)
        return fail(NRRS_ERR_INVALID_ARG, "bad image size, spp or depth");
    if (rrs_mode < NRRS_RRS_NONE || rrs_mode > NRRS_RRS_NET_MIX)
        return fail(NRRS_ERR_INVALID_ARG, "unknown rrs_mode");
    nrrs_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.seed_lo = 1; o.cap_factor = 2; o.f_rate = 0.85f; o.alpha0 = 1.0f; o.q_max = 16.0f;
    o.eps_rel = 0.01f; o.boxcox_lambda = 0.5f; o.precision = 32; o.update_ref = 1;
    if (opts) o = *opts;
    if (o.cap_factor < 1) return fail(NRRS_ERR_INVALID_ARG, "cap_factor < 1");
    if (!(o.f_rate > 0.0f && o.f_rate <= 1.0f) || !(o.alpha0 > 0.0f && o.alpha0 <= 1.0f))
        return fail(NRRS_ERR_INVALID_ARG, "f_rate and alpha0 must lie in (0, 1]");
    if (o.precision != 32) return fail(NRRS_ERR_UNSUPPORTED, "render supports precision 32");
    if (rrs_mode == NRRS_RRS_NET_MIX)
        for (int d = 1; d <= max_depth; ++d)
            if (((o.gate >> (2 * (d - 1))) & 3u) == 3u) return fail(NRRS_ERR_INVALID_ARG, "gate value 3");
    const long long npix = (long long)width * height;
    const long long P = npix * spp;
    const long long C = P * o.cap_factor;
    if (C >= (1ll << 31)) return fail(NRRS_ERR_INVALID_ARG, "capacity W*H*spp*cap_factor >= 2^31");

    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    bool uses_net = rrs_mode == NRRS_RRS_NET;
    if (rrs_mode == NRRS_RRS_NET_MIX)
        for (int d = 1; d <= max_depth; ++d)
            if (factor_kind(rrs_mode, o.gate, d) == kFactorNet) uses_net = true;
    nrrs_status rc = ensure_workspace(scene, C, npix, uses_net);
    if (rc != NRRS_OK) return rc;
    Workspace& ws = scene->ws;

    // reference image for HEUR factors
    bool uses_heur = rrs_mode == NRRS_RRS_HEUR_NORM;
    if (rrs_mode == NRRS_RRS_NET_MIX)
        for (int d = 1; d <= max_depth; ++d)
            if (factor_kind(rrs_mode, o.gate, d) == kFactorHeur) uses_heur = true;
    if (o.reset_ref || scene->ref_w != width || scene->ref_h != height) {
        scene->ref_count = 0;
        scene->ref_w = width;
        scene->ref_h = height;
        cudaFree(scene->ref_mean);
        scene->ref_mean = nullptr;
        CK(dalloc(&scene->ref_mean, (size_t)npix * 3));
        CK(cudaMemsetAsync(scene->ref_mean, 0, sizeof(float) * 3 * (size_t)npix, s));
    }
    const float* ref = o.d_pixel_ref ? o.d_pixel_ref : (scene->ref_count > 0 ? scene->ref_mean : nullptr);

    RenderParams rp{};
    rp.W = width; rp.H = height; rp.spp = spp; rp.D = max_depth;
    rp.cap = C;
    rp.key0 = o.seed_lo;
    rp.key1 = o.seed_hi ^ o.frame;
    rp.f_rate = o.f_rate;
    rp.q_max = o.q_max;
    rp.boxcox_lambda = o.boxcox_lambda;
    rp.ref = uses_heur ? ref : nullptr;
    rp.params = scene->params;
    rp.trace = o.d_trace;

    scene->cam.aspect = (float)width / (float)height;
    const int normalized = rrs_mode == NRRS_RRS_HEUR_NORM || rrs_mode == NRRS_RRS_NET ||
                           rrs_mode == NRRS_RRS_NET_MIX;

    CK(cudaMemsetAsync(ws.st, 0, sizeof(DevStats), s));
    CK(cudaMemsetAsync(ws.acc_s, 0, sizeof(float4) * npix, s));
    CK(cudaMemsetAsync(ws.acc_c, 0, sizeof(float4) * npix, s));
    StageTimer tm{scene, s, o.profile != 0};
#define TIMED(stage, call)           \
    do {                             \
        CK(tm.begin(stage));         \
        call;                        \
        CK(tm.end());                \
    } while (0)
    TIMED(NRRS_STAGE_INIT, launch_ref_prepare(rp.ref, npix * 3, o.eps_rel, (double)o.alpha0, P, ws.st, s));
    QueueView q[2];
    for (int k = 0; k < 2; ++k) q[k] = QueueView{ws.qo[k], ws.qd[k], ws.qt[k]};
    TIMED(NRRS_STAGE_INIT, launch_camera(scene->cam, rp, q[0], s));
    WorkView w{};
    w.hit = ws.hit; w.q = ws.q; w.dep = ws.dep; w.feat = ws.feat; w.part = ws.part;
    w.grid_red = ws.grid_red;
    w.bcnt = ws.bcnt; w.boff = ws.boff; w.grid_split = ws.grid_split;
    w.acc_s = ws.acc_s; w.acc_c = ws.acc_c; w.st = ws.st;
    int cur = 0;
    for (int d = 1; d <= max_depth; ++d) {
        const int kind = factor_kind(rrs_mode, o.gate, d);
        TIMED(NRRS_STAGE_EXTEND, launch_trace(scene->view, q[cur], w, d, scene->grid_trace, s));
        TIMED(NRRS_STAGE_SHADE, launch_shade(kind, scene->view, q[cur], w, rp, d, s));
        if (kind == kFactorNet) {
            WorkView wn = w;
            wn.grid_red = scene->grid_rrsnet;
            TIMED(NRRS_STAGE_RRSNET, launch_rrsnet_depth(wn, rp, d, s));
            TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q(w, d, s));
        }
        TIMED(NRRS_STAGE_NORMALIZE, launch_normalize_depth(w, rp, d, normalized, s));
        const int do_split = d < max_depth;
        TIMED(NRRS_STAGE_COUNT, launch_split_count(scene->view, q[cur], w, rp, d, do_split, s));
        if (do_split) {
            TIMED(NRRS_STAGE_SCAN, launch_split_scan(w, rp, d, s));
            TIMED(NRRS_STAGE_SCATTER, launch_split_scatter(scene->view, q[cur], q[cur ^ 1], w, rp, d, s));
            cur ^= 1;
        }
    }
    const int update = o.update_ref && !o.d_pixel_ref;
    TIMED(NRRS_STAGE_FINALIZE,
          launch_finalize(w, rp, d_rgb, scene->ref_mean, scene->ref_count, update, s));
#undef TIMED
    CK(cudaGetLastError());
    if (update) scene->ref_count++;
    if (stats) {
        DevStats h;
        CK(cudaMemcpyAsync(&h, ws.st, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::memset(stats, 0, sizeof(*stats));
        for (int d = 0; d < max_depth; ++d) {
            stats->live[d] = h.live[d];
            stats->sum_q[d] = h.sum_q[d];
            stats->F[d] = h.F[d];
            stats->alpha[d] = h.alpha[d];
            stats->requested[d] = h.requested[d];
            stats->dropped[d] = h.dropped[d];
            stats->segments += h.live[d];
        }
        stats->nonfinite = (int64_t)h.nonfinite;
        stats->net_evals = (int64_t)h.net_evals;
        stats->capacity = C;
        stats->status_bits = h.status;
        stats->kernel_launches = tm.launches;
        tm.collect(stats);
    }
    return NRRS_OK;
}

nrrs_status nrrs_query_factors(nrrs_scene* scene, const float* d_features, int64_t n,
                               int32_t precision, float* d_q, void* stream) {
    if (!scene || n < 0 || (n > 0 && (!d_features || !d_q)))
        return fail(NRRS_ERR_INVALID_ARG, "bad query arguments");
    if (precision != 32) return fail(NRRS_ERR_UNSUPPORTED, "precision must be 32");
    if (n == 0) return NRRS_OK;
    if ((reinterpret_cast<uintptr_t>(d_features) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_features must be 16-byte aligned");
    DeviceGuard g(scene->device);
    launch_query_factors(scene->params, d_features, n, d_q, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_normalize(nrrs_scene* scene, const float* d_q, int64_t n, double budget,
                           double f_rate, double alpha, float* d_F, double* d_sum, void* stream) {
    if (n < 0 || (n > 0 && !d_q) || !d_F || !d_sum || !(budget >= 0.0))
        return fail(NRRS_ERR_INVALID_ARG, "bad normalize arguments");
    int dev = 0;
    if (scene) dev = scene->device; else CK(cudaGetDevice(&dev));
    DeviceGuard g(dev);
    Pool* p = nullptr;
    nrrs_status rc = pool_for_device(dev, &p);
    if (rc != NRRS_OK) return rc;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    launch_normalize_array(d_q, n, budget, f_rate, alpha, p->part, p->grid, d_F, d_sum,
                           (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_split(nrrs_scene* scene, const float* d_q_orig, int64_t n, const float* d_F,
                       const uint32_t* d_pixel, const uint32_t* d_sample, const uint32_t* d_lineage,
                       uint32_t depth, uint32_t seed_lo, uint32_t seed_hi, uint32_t frame, int64_t cap,
                       uint32_t* d_X, int64_t* d_prefix, uint32_t* d_child_parent,
                       uint32_t* d_child_lineage, int64_t* d_total, int64_t* d_dropped, void* stream) {
    if (n < 0 || n >= (1ll << 31) || cap < 0 || cap >= (1ll << 31) || !d_F || !d_total || !d_dropped)
        return fail(NRRS_ERR_INVALID_ARG, "bad split sizes");
    if (n > 0 && (!d_q_orig || !d_pixel || !d_sample || !d_lineage || !d_X || !d_prefix))
        return fail(NRRS_ERR_INVALID_ARG, "NULL split array");
    if (cap > 0 && (!d_child_parent || !d_child_lineage))
        return fail(NRRS_ERR_INVALID_ARG, "NULL child arrays");
    int dev = 0;
    if (scene) dev = scene->device; else CK(cudaGetDevice(&dev));
    DeviceGuard g(dev);
    Pool* p = nullptr;
    nrrs_status rc = pool_for_device(dev, &p);
    if (rc != NRRS_OK) return rc;
    SplitArrays a{};
    a.q = d_q_orig; a.n = n; a.F = d_F; a.pixel = d_pixel; a.sample = d_sample; a.lineage = d_lineage;
    a.depth = depth; a.key0 = seed_lo; a.key1 = seed_hi ^ frame; a.cap = cap;
    a.X = d_X; a.prefix = reinterpret_cast<long long*>(d_prefix);
    a.child_parent = d_child_parent; a.child_lineage = d_child_lineage;
    a.total = reinterpret_cast<long long*>(d_total);
    a.dropped = reinterpret_cast<long long*>(d_dropped);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    launch_split_arrays(a, p->bcnt, p->boff, p->grid, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

}  // extern "C"
