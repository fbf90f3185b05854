// C ABI of the NRRS bounce (include/nrrs.h): scene set-up, the per-depth launch
// sequence of one render, and the stand-alone stage entry points.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bvh.h"
#include "bvh8.h"
#include "emitters.h"
#include "grid.cuh"
#include "train.cuh"
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
    unsigned long long* bcnt = nullptr;
    unsigned long long* boff = nullptr;
    float4* acc_s = nullptr;
    float4* acc_c = nullptr;
    DevStats* st = nullptr;
    FrameConsts* fc = nullptr;
    unsigned long long* flags = nullptr;  // look-back flags of the fused split
    long long n_flags = 0;
    float4* feat_net = nullptr;  // NRRS inputs of RRSNet (scenes with rrsnet_inputs = 1)
    // next-event estimation: sampling pdfs of both queues and the per-slot shadow rays
    bool has_nee = false;
    float* qpdf[2] = {nullptr, nullptr};
    float4* sh_o = nullptr;
    float4* sh_d = nullptr;
    float4* sh_c = nullptr;

    void release() {
        for (int k = 0; k < 2; ++k) {
            cudaFree(qo[k]);
            cudaFree(qd[k]);
            cudaFree(qt[k]);
            cudaFree(qpdf[k]);
            qo[k] = qd[k] = qt[k] = nullptr;
            qpdf[k] = nullptr;
        }
        cudaFree(sh_o); cudaFree(sh_d); cudaFree(sh_c);
        sh_o = sh_d = sh_c = nullptr;
        cudaFree(feat_net);
        feat_net = nullptr;
        has_nee = false;
        cudaFree(hit); cudaFree(q); cudaFree(dep); cudaFree(feat); cudaFree(part); cudaFree(bcnt);
        cudaFree(boff); cudaFree(acc_s); cudaFree(acc_c); cudaFree(st); cudaFree(fc);
        cudaFree(flags);
        fc = nullptr;
        flags = nullptr;
        n_flags = 0;
        hit = nullptr; q = nullptr; dep = nullptr; feat = nullptr; part = nullptr; bcnt = nullptr;
        has_feat = false;
        boff = nullptr; acc_s = acc_c = nullptr; st = nullptr;
        cap = npix = 0;
    }
};

// Scratch for the plain-array stage entry points called without a scene.
struct Pool {
    double* part = nullptr;
    unsigned long long* bcnt = nullptr;
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

// Training state of a scene: the recorded frame and both networks with their optimizer
// state (allocated on first use).
struct TrainState {
    RecordView rec{};
    long long rec_C = 0, npix = 0;
    int rec_D = 0;
    float *m1 = nullptr, *m2 = nullptr, *V = nullptr, *E = nullptr, *rgb = nullptr;
    float *E_cur = nullptr, *E_acc = nullptr;  // error map: this frame, temporal EMA
    float4* pnrm = nullptr;                      // pixel normals guiding the spatial filter
    int filter_launches = 0;                     // of the last step's spatial filter
    bool e_first = true;
    int* k = nullptr;
    bool nets = false;
    float *rrs_raw = nullptr, *rrs_m = nullptr, *rrs_v = nullptr, *rrs_good = nullptr;
    float *stat = nullptr, *stat_m = nullptr, *stat_v = nullptr, *stat_good = nullptr;
    float *grad_rrs = nullptr, *grad_stat = nullptr, *part = nullptr;
    float* loss_part = nullptr;
    double* scal = nullptr;       // relMSE of the Mix-Depth candidates (nrrs_relmse's layout)
    float* fscal = nullptr;       // [0] Ebar, [1] L_min, [2] L_avg, [3] StatNet loss, [4] RRSNet loss
    long long* kpart = nullptr;   // per-block sample counts of the pixel terms
    long long* nsamp = nullptr;   // training samples N
    float *Fd = nullptr, *Fnd = nullptr;
    int* bad = nullptr;
    int part_blocks = 0;
    long long step = 0, full_steps = 0;
    double loss_ema = 0.0, loss_min = 0.0;
    // StatNet's inputs: 0 = vertex features, 1 = the encodings of Sec. 4 with the hash grid
    int stat_enc = 0;
    float *grid = nullptr, *grid_m = nullptr, *grid_v = nullptr, *grid_good = nullptr;
    float *grid_grad = nullptr, *dx = nullptr;
    long long dx_cap = 0;
    // AID-NRRS: RRSNet's hash grid, trained (raw) and its EMA for rendering
    float *rgrid = nullptr, *rgrid_raw = nullptr, *rgrid_m = nullptr, *rgrid_v = nullptr;
    float *rgrid_good = nullptr, *rgrid_grad = nullptr;
    int stat_n() const {
        return (stat_enc ? kNH * kStatGridIn : kNH * kNF) + 2 * kNH * kNH + kStatOut * kNH;
    }

    void release_record() {
        cudaFree(rec.dep); cudaFree(rec.q); cudaFree(rec.t); cudaFree(rec.feat);
        cudaFree(rec.feat_net);
        cudaFree(rec.rough);
        cudaFree(rec.first); cudaFree(rec.X); cudaFree(rec.S);
        cudaFree(m1); cudaFree(m2); cudaFree(V); cudaFree(E); cudaFree(k); cudaFree(rgb);
        cudaFree(E_cur); cudaFree(E_acc); cudaFree(pnrm);
        rec = RecordView{};
        m1 = m2 = V = E = rgb = E_cur = E_acc = nullptr;
        pnrm = nullptr;
        e_first = true;
        k = nullptr;
        rec_C = npix = 0;
        rec_D = 0;
    }
    void release_all() {
        release_record();
        float* fs[] = {rrs_raw, rrs_m, rrs_v, rrs_good, stat, stat_m, stat_v, stat_good,
                       grad_rrs, grad_stat, part, Fd, Fnd,
                       grid, grid_m, grid_v, grid_good, grid_grad, dx,
                       rgrid, rgrid_raw, rgrid_m, rgrid_v, rgrid_good, rgrid_grad};
        for (float* f : fs) cudaFree(f);
        grid = grid_m = grid_v = grid_good = grid_grad = dx = nullptr;
        rgrid = rgrid_raw = rgrid_m = rgrid_v = rgrid_good = rgrid_grad = nullptr;
        dx_cap = 0;
        cudaFree(loss_part);
        cudaFree(scal);
        cudaFree(fscal);
        cudaFree(kpart);
        cudaFree(nsamp);
        cudaFree(bad);
        nets = false;
    }
};

struct nrrs_scene {
    int device = 0;
    int n_sm = 148;
    // NET depths at precisions 16 and 17 shade and run RRSNet in one kernel (features in
    // shared memory); off: k_shade, then k_rrsnet_tc on the features in HBM
    bool fuse_net = true;
    // the BVH2's height (most inner nodes on a root-to-leaf path, -1 unknown) and the
    // traversal stack asked for (0: the short stack when the tree fits it)
    int bvh2_h = -1;
    int stack_req = 0;
    int64_t n_nodes = 0, n_tri = 0;
    float4* nodes = nullptr;
    float4* nodes4 = nullptr;  // four-wide tree (NULL when its stack bound exceeds the kernel's)
    uint4* nodes_h = nullptr;  // BVH2 with FP16 boxes (NULL when a leaf does not fit its code)
    int bvh_width = 2;
    float4* tris = nullptr;
    // the input triangles ([n_tri][9] vertices, material ids) for the device-built
    // eight-wide tree, and that tree once built (nrrs_set_traversal(8))
    float* tri_raw = nullptr;
    int32_t* mat_raw = nullptr;
    float scene_lo[3] = {0, 0, 0}, scene_hi[3] = {0, 0, 0};
    Bvh8Device bvh8;
    float bvh8_build_ms = 0.0f;
    nrrs_material* mats = nullptr;
    float4* emit = nullptr;      // next-event estimation: emitter triangles and area CDF
    float* emit_cdf = nullptr;
    float* params = nullptr;  // RRSNet weights, 2592 floats
    SceneView view{};
    CamView cam{};
    Workspace ws;
    int grid_trace = 0, grid_sum = 0;
    // RRSNet launch shapes per queue-size bucket (FP32, split BF16, E4M3, BF16), set by
    // the tuner
    RrsnetChoice tune[4][kTuneBuckets];
    bool tuned[4] = {false, false, false, false};
    // live counts of the last render that returned stats: the queue sizes expected at
    // each depth of the next frame (scaled by its primary count)
    long long last_live[NRRS_MAX_DEPTH] = {};
    long long last_P = 0;
    // the last training step fell back: the next render uses the heuristic at NET depths
    bool heur_next = false;
    // RRSNet inputs: 0 = the 16 vertex features, 1 = the NRRS inputs built from StatNet
    int rrsnet_inputs = 0;
    // running mean of earlier frames (HEUR reference), [npix * 3]
    float* ref_mean = nullptr;
    int ref_count = 0;
    int ref_w = 0, ref_h = 0;
    std::vector<cudaEvent_t> events;  // reused by profiled renders
    TrainState train;
    // graph-captured renders: capture stream and executable graphs per launch shape
    cudaStream_t capture_stream = nullptr;
    // batched render (nrrs_create_batch): the job table and its per-job work arrays
    int n_jobs = 0;
    std::vector<JobDev> jobs_host;
    JobDev* jobs_dev = nullptr;
    long long batch_P = 0, batch_npix = 0;
    int batch_D = 0;
    JobWork jw{};
    int jw_grid = 0;
    std::vector<float> job_F;        // last batched render with stats, [D][n_jobs]
    std::vector<double> job_sum_q;
    std::vector<long long> job_live;
    struct GraphEntry {
        uint64_t shape;             // launch shape: kernels and their order
        uint64_t args;              // every launch argument except the per-frame constants
        cudaGraphExec_t exec;
        unsigned launches;          // kernels in the graph
        std::vector<int> stage_of;  // stage of every bracketed launch (profiled graphs)
    };
    std::vector<GraphEntry> graphs;
    int32_t bvh_builder = 0;  // 0 host binned SAH, 1 device PLOC (nrrs_set_bvh_builder)
};

namespace {

// RRSNet's weight count: 16 inputs, or 32 with the AID-NRRS inputs.
int rrs_n(const nrrs_scene* sc) { return sc->rrsnet_inputs == 2 ? kAidParams : kNParams; }
// RRSNet's weights (and, with the AID-NRRS inputs, its hash grid) afresh for the current
// input mode (below).
nrrs_status init_rrsnet_shape(nrrs_scene* sc);

nrrs_status alloc_nee(Workspace& w) {
    if (w.has_nee) return NRRS_OK;
    for (int k = 0; k < 2; ++k) CK(dalloc(&w.qpdf[k], (size_t)w.cap));
    CK(dalloc(&w.sh_o, (size_t)w.cap));
    CK(dalloc(&w.sh_d, (size_t)w.cap));
    CK(dalloc(&w.sh_c, (size_t)w.cap));
    w.has_nee = true;
    return NRRS_OK;
}

nrrs_status ensure_workspace(nrrs_scene* sc, long long cap, long long npix, bool need_feat,
                             bool need_nee = false) {
    Workspace& w = sc->ws;
    if (w.cap >= cap && w.npix >= npix && w.st) {
        if (need_feat && !w.has_feat) {
            CK(dalloc(&w.feat, (size_t)w.cap * 4));
            w.has_feat = true;
        }
        if (need_nee) return alloc_nee(w);
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
    CK(dalloc(&w.fc, 1));
    w.n_flags = cap / split_block_threads() + 2;  // one look-back flag per split tile
    CK(dalloc(&w.flags, (size_t)w.n_flags));
    w.cap = cap;
    w.npix = npix;
    if (need_nee) return alloc_nee(w);
    return NRRS_OK;
}

void destroy(nrrs_scene* s) {
    if (!s) return;
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
    cudaFree(s->jobs_dev);
    cudaFree(s->jw.F_cur); cudaFree(s->jw.eps_I); cudaFree(s->jw.part); cudaFree(s->jw.cnt);
    cudaFree(s->jw.F); cudaFree(s->jw.sum_q); cudaFree(s->jw.live);
    if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
    s->train.release_all();
    s->ws.release();
    cudaFree(s->nodes);
    cudaFree(s->nodes4);
    cudaFree(s->nodes_h);
    cudaFree(s->tris);
    cudaFree(s->tri_raw);
    cudaFree(s->mat_raw);
    cudaFree(s->bvh8.nodes);
    cudaFree(s->bvh8.tris);
    cudaFree(s->mats);
    cudaFree(s->emit);
    cudaFree(s->emit_cdf);
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
    unsigned mask;           // stages to time (bit k = stage k)
    bool capturing = false;  // events become graph nodes (recorded when the graph runs)
    bool open = false;       // the current launch is bracketed
    int used = 0;
    unsigned launches = 0;
    std::vector<int> stage_of;
    cudaError_t begin(int stage) {
        ++launches;
        open = ((mask >> stage) & 1u) != 0;
        if (!open) return cudaSuccess;
        while ((int)sc->events.size() < used + 2) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            sc->events.push_back(e);
        }
        stage_of.push_back(stage);
        return record(sc->events[used++]);
    }
    cudaError_t end() {
        if (!open) return cudaSuccess;
        open = false;
        return record(sc->events[used++]);
    }
    cudaError_t record(cudaEvent_t e) {
        return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                         : cudaEventRecord(e, s);
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

int precision_index(int precision) {
    return precision == 32 ? 0 : precision == 16 ? 1 : precision == 8 ? 2 : 3;
}

// Launch shape of the RRSNet kernel for a queue of about n rows.
RrsnetChoice rrsnet_choice(const nrrs_scene* sc, int precision, long long n) {
    const int p = precision_index(precision);
    return sc->tuned[p] ? sc->tune[p][tune_bucket(n)] : default_choice(precision);
}

int factor_kind(int mode, uint64_t gate, int depth) {
    switch (mode) {
        case kNone: return kFactorOne;
        case kPlainRR: return kFactorPlain;
        case kHeurNorm: return kFactorHeur;
        case kNet: return kFactorNet;
        default: {
            const unsigned g = (unsigned)((gate >> (2 * (depth - 1))) & 3u);
            return g == kGateNet    ? kFactorNet
                   : g == kGateHeur ? kFactorHeur
                   : g == kGateAdrrs ? kFactorAdrrs
                                    : kFactorOne;
        }
    }
}

}  // namespace

namespace {

// Camera basis in FP64, rounded once (nrrs_camera).
CamView cam_view(const nrrs_camera& cam) {
    CamView c{};
    V3d fw = vnorm({cam.look[0], cam.look[1], cam.look[2]});
    V3d up = {cam.up[0], cam.up[1], cam.up[2]};
    V3d right = vnorm(vcross(up, fw));
    V3d up2 = vcross(fw, right);
    for (int k = 0; k < 3; ++k) c.pos[k] = cam.pos[k];
    c.fw[0] = (float)fw.x; c.fw[1] = (float)fw.y; c.fw[2] = (float)fw.z;
    c.right[0] = (float)right.x; c.right[1] = (float)right.y; c.right[2] = (float)right.z;
    c.up[0] = (float)up2.x; c.up[1] = (float)up2.y; c.up[2] = (float)up2.z;
    c.tan_half = (float)std::tan(0.5 * (double)cam.vfov_deg * M_PI / 180.0);
    c.aspect = 1.0f;
    return c;
}

// Uploads a built BVH (and its triangle references), the materials and the camera
// (NULL for a batch, whose cameras live in the job table) into a new scene.
// The BVH2 traversal takes the short stack when the tree is known to fit it, unless the
// long one was asked for.
int short_stack_on(const nrrs_scene* s) {
    const bool fits = s->bvh2_h >= 0 && s->bvh2_h <= trace_short_stack_entries();
    return fits && s->stack_req != trace_stack_entries() ? 1 : 0;
}

nrrs_status upload_scene(const BvhHost& bvh, const Bvh4Host* bvh4, int64_t n_tri,
                         const nrrs_material* mats, int32_t n_mat, const nrrs_camera* cam,
                         const EmitterHost& em, int device, nrrs_scene** out) {
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
    if ((e = dalloc(&s->params, kRrsParamsMax)) != cudaSuccess) return bail(e, "alloc params");
    if ((e = cudaMemcpy(s->nodes, bvh.nodes.data(), bvh.nodes.size() * 64, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy nodes");
    if ((e = cudaMemcpy(s->tris, bvh.tris.data(), (size_t)bvh.n_ref * 48, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy tris");
    if ((e = cudaMemcpy(s->mats, mats, sizeof(nrrs_material) * n_mat, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy mats");
    if ((e = cudaMemset(s->params, 0, kRrsParamsMax * sizeof(float))) != cudaSuccess) return bail(e, "zero params");
    if (!em.cdf.empty()) {
        if ((e = dalloc(&s->emit, em.tri.size())) != cudaSuccess) return bail(e, "alloc emitters");
        if ((e = dalloc(&s->emit_cdf, em.cdf.size())) != cudaSuccess) return bail(e, "alloc emitter cdf");
        if ((e = cudaMemcpy(s->emit, em.tri.data(), sizeof(float4) * em.tri.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy emitters");
        if ((e = cudaMemcpy(s->emit_cdf, em.cdf.data(), sizeof(float) * em.cdf.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy emitter cdf");
    }
    s->view.emit = s->emit;
    s->view.emit_cdf = s->emit_cdf;
    s->view.n_emit = (int)em.cdf.size();
    s->view.inv_area = em.area > 0.0 ? (float)(1.0 / em.area) : 0.0f;

    if (bvh4 && !bvh4->nodes.empty()) {
        if ((e = dalloc(&s->nodes4, bvh4->nodes.size() * 8)) != cudaSuccess) return bail(e, "alloc nodes4");
        if ((e = cudaMemcpy(s->nodes4, bvh4->nodes.data(), bvh4->nodes.size() * 128,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy nodes4");
    }
    std::vector<BvhNodeH> half;
    bool half_default = false;
    if (pack_half_nodes(bvh, &half)) {
        half_default = half_node_growth(bvh, half) <= kMaxHalfGrowth;
        if ((e = dalloc(&s->nodes_h, half.size() * 2)) != cudaSuccess) return bail(e, "alloc half nodes");
        if ((e = cudaMemcpy(s->nodes_h, half.data(), half.size() * sizeof(BvhNodeH),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy half nodes");
    }
    s->view.nodes = s->nodes;
    s->view.nodes4 = nullptr;  // the BVH2 unless nrrs_set_traversal(4): measured no faster
    // FP16 boxes unless rounding grows them too much, or nrrs_set_bvh_precision(32)
    s->view.nodes_h = half_default ? s->nodes_h : nullptr;
    s->bvh2_h = bvh2_height(bvh.nodes);
    s->view.short_stack = short_stack_on(s);
    s->view.tris = s->tris;
    s->view.mats = s->mats;
    for (int k = 0; k < 3; ++k) {
        s->view.lo[k] = bvh.lo[k];
        const float ext = bvh.hi[k] - bvh.lo[k];
        s->view.inv_ext[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
    }
    if (cam) s->cam = cam_view(*cam);
    s->grid_trace = s->n_sm * max_blocks_trace();
    s->grid_sum = s->n_sm * 4;
    *out = s;
    return NRRS_OK;
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
    Bvh4Host bvh4;
    collapse_bvh4(bvh, &bvh4);
    const bool wide = bvh4.max_stack <= trace_stack_entries();
    const EmitterHost em = build_emitters(tri, n_tri, tri_mat, mats);
    nrrs_status rc = upload_scene(bvh, wide ? &bvh4 : nullptr, n_tri, mats, n_mat, cam, em, device, out);
    if (rc != NRRS_OK) return rc;
    nrrs_scene* s = *out;
    for (int k = 0; k < 3; ++k) {
        s->scene_lo[k] = bvh.lo[k];
        s->scene_hi[k] = bvh.hi[k];
    }
    cudaError_t e = dalloc(&s->tri_raw, (size_t)n_tri * 9);
    if (e == cudaSuccess) e = dalloc(&s->mat_raw, (size_t)n_tri);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->tri_raw, tri, sizeof(float) * 9 * (size_t)n_tri, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->mat_raw, tri_mat, sizeof(int32_t) * (size_t)n_tri, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        destroy(s);
        *out = nullptr;
        return cuda_fail(e, "upload triangles");
    }
    return NRRS_OK;
}

nrrs_status nrrs_destroy_scene(nrrs_scene* scene) {
    if (!scene) return NRRS_OK;
    DeviceGuard g(scene->device);
    cudaDeviceSynchronize();
    destroy(scene);
    return NRRS_OK;
}

nrrs_status nrrs_set_traversal(nrrs_scene* scene, int32_t width) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (width != 2 && width != 4 && width != 8)
        return fail(NRRS_ERR_INVALID_ARG, "width must be 2, 4 or 8");
    if (width == 4 && !scene->nodes4)
        return fail(NRRS_ERR_UNSUPPORTED, "no four-wide tree (its stack bound is too deep)");
    if (width == 8) {
        if (scene->n_jobs > 0 || !scene->tri_raw)
            return fail(NRRS_ERR_UNSUPPORTED, "the eight-wide tree is built for single scenes");
        if (!scene->bvh8.nodes) {
            DeviceGuard g(scene->device);
            if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
            const auto t0 = std::chrono::steady_clock::now();
            Bvh8Device b;
            cudaError_t e = build_bvh8(scene->tri_raw, scene->mat_raw, (int)scene->n_tri,
                                       scene->scene_lo, scene->scene_hi, nullptr, &b);
            if (e != cudaSuccess) return cuda_fail(e, "eight-wide BVH build");
            scene->bvh8_build_ms = std::chrono::duration<float, std::milli>(
                                       std::chrono::steady_clock::now() - t0).count();
            if (b.depth > trace_stack_entries()) {
                cudaFree(b.nodes);
                cudaFree(b.tris);
                return fail(NRRS_ERR_UNSUPPORTED, "eight-wide tree deeper than the traversal stack");
            }
            scene->bvh8 = b;
        }
        scene->view.nodes8 = scene->bvh8.nodes;
        scene->view.tris = scene->bvh8.tris;
        scene->view.nodes4 = nullptr;
    } else {
        scene->view.nodes8 = nullptr;
        scene->view.tris = scene->tris;
        scene->view.nodes4 = width == 4 ? scene->nodes4 : nullptr;
    }
    scene->bvh_width = width;
    return NRRS_OK;
}

nrrs_status nrrs_set_bvh_builder(nrrs_scene* scene, int32_t builder, float* build_ms) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (builder != 0 && builder != 1)
        return fail(NRRS_ERR_INVALID_ARG, "builder must be 0 (host binned SAH) or 1 (device PLOC)");
    if (scene->n_jobs > 0 || !scene->tri_raw || scene->n_tri < 2)
        return fail(NRRS_ERR_UNSUPPORTED, "the BVH2 is rebuilt for single scenes of two or more triangles");
    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    CK(cudaDeviceSynchronize());
    const size_t nt = (size_t)scene->n_tri;
    std::vector<float> tri(nt * 9);
    std::vector<int32_t> mat(nt);
    CK(cudaMemcpy(tri.data(), scene->tri_raw, sizeof(float) * tri.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mat.data(), scene->mat_raw, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost));
    const auto t0 = std::chrono::steady_clock::now();
    BvhHost bvh;
    if (builder == 0) {
        build_bvh(tri.data(), (int32_t)nt, mat.data(), &bvh);
    } else {
        int depth = 0;
        const cudaError_t e = build_bvh2_ploc(scene->tri_raw, tri.data(), mat.data(), (int)nt,
                                              scene->scene_lo, scene->scene_hi,
                                              trace_stack_entries() - 2, nullptr, &bvh, &depth);
        if (e == cudaErrorNotSupported)
            return fail(NRRS_ERR_UNSUPPORTED, "device-built BVH2 deeper than the traversal stack");
        if (e != cudaSuccess) return cuda_fail(e, "device BVH2 build");
    }
    if (build_ms)
        *build_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    Bvh4Host bvh4;
    collapse_bvh4(bvh, &bvh4);
    std::vector<BvhNodeH> half;
    const bool has_half = pack_half_nodes(bvh, &half);
    float4 *nodes = nullptr, *tris = nullptr, *nodes4 = nullptr;
    uint4* nodes_h = nullptr;
    auto bail = [&](cudaError_t e, const char* what) {
        cudaFree(nodes);
        cudaFree(tris);
        cudaFree(nodes4);
        cudaFree(nodes_h);
        return cuda_fail(e, what);
    };
    cudaError_t e;
    if ((e = dalloc(&nodes, bvh.nodes.size() * 4)) != cudaSuccess) return bail(e, "alloc nodes");
    if ((e = dalloc(&tris, (size_t)bvh.n_ref * 3)) != cudaSuccess) return bail(e, "alloc tris");
    if ((e = cudaMemcpy(nodes, bvh.nodes.data(), bvh.nodes.size() * 64, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy nodes");
    if ((e = cudaMemcpy(tris, bvh.tris.data(), (size_t)bvh.n_ref * 48, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "copy tris");
    if (bvh4.max_stack <= trace_stack_entries() && !bvh4.nodes.empty()) {
        if ((e = dalloc(&nodes4, bvh4.nodes.size() * 8)) != cudaSuccess) return bail(e, "alloc nodes4");
        if ((e = cudaMemcpy(nodes4, bvh4.nodes.data(), bvh4.nodes.size() * 128,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy nodes4");
    }
    if (has_half) {
        if ((e = dalloc(&nodes_h, half.size() * 2)) != cudaSuccess) return bail(e, "alloc half nodes");
        if ((e = cudaMemcpy(nodes_h, half.data(), half.size() * sizeof(BvhNodeH),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "copy half nodes");
    }
    const bool half_on = nodes_h && half_node_growth(bvh, half) <= kMaxHalfGrowth;
    // captured graphs hold the old tree's addresses: drop them before freeing it
    for (auto& ge : scene->graphs) cudaGraphExecDestroy(ge.exec);
    scene->graphs.clear();
    cudaFree(scene->nodes);
    cudaFree(scene->tris);
    cudaFree(scene->nodes4);
    cudaFree(scene->nodes_h);
    scene->nodes = nodes;
    scene->tris = tris;
    scene->nodes4 = nodes4;
    scene->nodes_h = nodes_h;
    scene->n_nodes = (int64_t)bvh.nodes.size();
    scene->view.nodes = nodes;
    scene->view.nodes_h = half_on ? nodes_h : nullptr;
    scene->bvh2_h = bvh2_height(bvh.nodes);
    if (scene->stack_req == trace_short_stack_entries() &&
        !(scene->bvh2_h >= 0 && scene->bvh2_h <= trace_short_stack_entries()))
        scene->stack_req = 0;  // the new tree is too tall for the stack asked for
    scene->view.short_stack = short_stack_on(scene);
    if (scene->bvh_width == 4 && !nodes4) scene->bvh_width = 2;
    if (scene->bvh_width != 8) {
        scene->view.tris = tris;
        scene->view.nodes4 = scene->bvh_width == 4 ? nodes4 : nullptr;
    }
    scene->bvh_builder = builder;
    return NRRS_OK;
}

nrrs_status nrrs_bvh8_info(const nrrs_scene* scene, nrrs_bvh8_stats* out) {
    if (!scene || !out) return fail(NRRS_ERR_INVALID_ARG, "NULL scene or out");
    std::memset(out, 0, sizeof(*out));
    out->nodes = scene->bvh8.n_nodes;
    out->triangles = scene->bvh8.nodes ? scene->n_tri : 0;
    out->depth = scene->bvh8.depth;
    out->iterations = scene->bvh8.ploc_iterations;
    out->build_ms = scene->bvh8_build_ms;
    return NRRS_OK;
}

nrrs_status nrrs_bvh8_export(const nrrs_scene* scene, uint32_t* nodes, int64_t max_nodes,
                             float* tris, int64_t max_tris) {
    if (!scene || !nodes || !tris) return fail(NRRS_ERR_INVALID_ARG, "NULL argument");
    if (!scene->bvh8.nodes) return fail(NRRS_ERR_UNSUPPORTED, "no eight-wide tree built");
    if (max_nodes < (int64_t)scene->bvh8.n_nodes || max_tris < scene->n_tri)
        return fail(NRRS_ERR_INVALID_ARG, "export buffers too small");
    DeviceGuard g(scene->device);
    CK(cudaMemcpy(nodes, scene->bvh8.nodes, sizeof(uint4) * 5 * (size_t)scene->bvh8.n_nodes,
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tris, scene->bvh8.tris, sizeof(float4) * 3 * (size_t)scene->n_tri,
                  cudaMemcpyDeviceToHost));
    return NRRS_OK;
}

nrrs_status nrrs_set_bvh_precision(nrrs_scene* scene, int32_t bits) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (bits != 16 && bits != 32) return fail(NRRS_ERR_INVALID_ARG, "bits must be 16 or 32");
    if (bits == 16 && !scene->nodes_h)
        return fail(NRRS_ERR_UNSUPPORTED, "no FP16 nodes (a leaf does not fit the packed code)");
    scene->view.nodes_h = bits == 16 ? scene->nodes_h : nullptr;
    return NRRS_OK;
}

nrrs_status nrrs_set_shade_fusion(nrrs_scene* scene, int32_t on) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (on != 0 && on != 1) return fail(NRRS_ERR_INVALID_ARG, "on must be 0 or 1");
    scene->fuse_net = on != 0;
    return NRRS_OK;
}

nrrs_status nrrs_set_traversal_stack(nrrs_scene* scene, int32_t entries) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (entries != 0 && entries != trace_short_stack_entries() &&
        entries != trace_stack_entries())
        return fail(NRRS_ERR_INVALID_ARG, "entries must be 0, 24 or 40");
    if (entries == trace_short_stack_entries() &&
        !(scene->bvh2_h >= 0 && scene->bvh2_h <= entries))
        return fail(NRRS_ERR_UNSUPPORTED, "the BVH2 is taller than the short stack");
    scene->stack_req = entries;
    scene->view.short_stack = short_stack_on(scene);
    return NRRS_OK;
}

nrrs_status nrrs_traversal_stack_info(const nrrs_scene* scene, int32_t* height,
                                      int32_t* entries) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (height) *height = scene->bvh2_h;
    if (entries)
        *entries = scene->view.short_stack ? trace_short_stack_entries() : trace_stack_entries();
    return NRRS_OK;
}

nrrs_status nrrs_set_rrsnet_inputs(nrrs_scene* scene, int32_t mode) {
    if (!scene || mode < 0 || mode > 2) return fail(NRRS_ERR_INVALID_ARG, "bad RRSNet input mode");
    if (mode == scene->rrsnet_inputs) return NRRS_OK;
    DeviceGuard g(scene->device);
    // recorded inputs of an earlier mode must not feed training
    cudaFree(scene->train.rec.feat_net);
    scene->train.rec.feat_net = nullptr;
    cudaFree(scene->train.rec.rough);
    scene->train.rec.rough = nullptr;
    const bool reshape = (mode == 2) != (scene->rrsnet_inputs == 2);
    scene->rrsnet_inputs = mode;
    if (reshape) return init_rrsnet_shape(scene);  // 16 <-> 32 inputs: weights afresh
    return NRRS_OK;
}

nrrs_status nrrs_scene_info(const nrrs_scene* scene, int64_t* n_nodes, int64_t* n_tri) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (n_nodes) *n_nodes = scene->n_nodes;
    if (n_tri) *n_tri = scene->n_tri;
    return NRRS_OK;
}

nrrs_status nrrs_set_rrsnet_params(nrrs_scene* scene, const float* params, int32_t n, void* stream) {
    if (!scene || !params || n != rrs_n(scene))
        return fail(NRRS_ERR_INVALID_ARG, "need 2592 host floats (3104 with AID-NRRS inputs)");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(scene->params, params, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

nrrs_status nrrs_get_rrsnet_params(nrrs_scene* scene, float* params, int32_t n, void* stream) {
    if (!scene || !params || n != rrs_n(scene))
        return fail(NRRS_ERR_INVALID_ARG, "need 2592 host floats (3104 with AID-NRRS inputs)");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(params, scene->params, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

}  // extern "C"

namespace {

// Fills defaults into a render-options struct.
nrrs_render_opts render_defaults() {
    nrrs_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.seed_lo = 1; o.cap_factor = 2; o.f_rate = 0.85f; o.alpha0 = 1.0f; o.q_max = 16.0f;
    o.eps_rel = 0.01f; o.boxcox_lambda = 0.5f; o.precision = 32; o.update_ref = 1;
    return o;
}

nrrs_status validate_render(nrrs_scene* scene, int32_t width, int32_t height, int32_t spp,
                            int32_t max_depth, int32_t rrs_mode, const nrrs_render_opts& o) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (width < 1 || height < 1 || spp < 1 || max_depth < 1 || max_depth > NRRS_MAX_DEPTH)
        return fail(NRRS_ERR_INVALID_ARG, "bad image size, spp or depth");
    if (rrs_mode < NRRS_RRS_NONE || rrs_mode > NRRS_RRS_NET_MIX)
        return fail(NRRS_ERR_INVALID_ARG, "unknown rrs_mode");
    if (o.cap_factor < 1) return fail(NRRS_ERR_INVALID_ARG, "cap_factor < 1");
    if (o.budget_factor < 0 || o.budget_factor > o.cap_factor)
        return fail(NRRS_ERR_INVALID_ARG, "budget_factor must lie in [0, cap_factor]");
    if (!(o.f_rate > 0.0f && o.f_rate <= 1.0f) || !(o.alpha0 > 0.0f && o.alpha0 <= 1.0f))
        return fail(NRRS_ERR_INVALID_ARG, "f_rate and alpha0 must lie in (0, 1]");
    if (o.precision != 32 && o.precision != 16 && o.precision != 8 && o.precision != 17)
        return fail(NRRS_ERR_UNSUPPORTED, "render supports precision 32, 16, 17 and 8");
    if (o.nee != 0 && o.nee != 1) return fail(NRRS_ERR_INVALID_ARG, "nee must be 0 or 1");
    if (scene->rrsnet_inputs == 2 && o.precision != 32)
        return fail(NRRS_ERR_UNSUPPORTED, "AID-NRRS inputs run in FP32 (precision 32)");
    const long long C = (long long)width * height * spp * o.cap_factor;
    if (C >= (1ll << 31)) return fail(NRRS_ERR_INVALID_ARG, "capacity W*H*spp*cap_factor >= 2^31");
    if (o.d_trace && o.d_trace_mask && (!o.d_trace_count || o.trace_rows < 1))
        return fail(NRRS_ERR_INVALID_ARG, "a masked trace needs d_trace_count and trace_rows >= 1");
    return NRRS_OK;
}

// Record buffers of a frame (every depth's slots) for the reverse pass and training.
nrrs_status ensure_record(nrrs_scene* sc, long long C, int D, long long npix) {
    TrainState& t = sc->train;
    if (t.rec_C >= C && t.rec_D >= D && t.npix >= npix) {
        if (sc->rrsnet_inputs && !t.rec.feat_net)
            CK(dalloc(&t.rec.feat_net, (size_t)t.rec_C * t.rec_D * 4));
        if ((t.stat_enc || sc->rrsnet_inputs == 2) && !t.rec.rough)
            CK(dalloc(&t.rec.rough, (size_t)t.rec_C * t.rec_D));
        return NRRS_OK;
    }
    t.release_record();
    const size_t n = (size_t)C * D;
    CK(dalloc(&t.rec.dep, n));
    CK(dalloc(&t.rec.q, n));
    CK(dalloc(&t.rec.t, n));
    CK(dalloc(&t.rec.feat, n * 4));
    CK(dalloc(&t.rec.first, n));
    CK(dalloc(&t.rec.X, n));
    CK(dalloc(&t.rec.S, n));
    CK(dalloc(&t.m1, n));
    CK(dalloc(&t.m2, n));
    CK(dalloc(&t.V, npix));
    CK(dalloc(&t.E, npix));
    CK(dalloc(&t.E_cur, npix));
    CK(dalloc(&t.E_acc, npix));
    CK(dalloc(&t.pnrm, npix));
    CK(dalloc(&t.k, npix));
    CK(dalloc(&t.rgb, npix * 3));
    if (sc->rrsnet_inputs) CK(dalloc(&t.rec.feat_net, n * 4));
    if (t.stat_enc || sc->rrsnet_inputs == 2) CK(dalloc(&t.rec.rough, n));
    t.rec.C = C;
    t.rec_C = C;
    t.rec_D = D;
    t.npix = npix;
    return NRRS_OK;
}

// Ends a stream capture left open by an early return.
struct CaptureGuard {
    cudaStream_t cs = nullptr;
    bool active = false;
    ~CaptureGuard() {
        if (!active) return;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
    }
};

uint64_t mix_key(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h;
}

// Ends the capture on `cs` and brings the scene's executable graph for this launch shape
// up to date: an in-place update when the topology matches, else a new instantiation.
// Returns the entry, which the caller launches.
nrrs_status finish_capture(nrrs_scene* sc, CaptureGuard& cg, uint64_t shape, uint64_t args,
                           nrrs_scene::GraphEntry** out) {
    cudaGraph_t g = nullptr;
    cg.active = false;
    CK(cudaStreamEndCapture(cg.cs, &g));
    auto& gs = sc->graphs;
    size_t slot = gs.size();
    for (size_t k = 0; k < gs.size(); ++k)
        if (gs[k].shape == shape) slot = k;
    if (slot < gs.size()) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gs[slot].exec, g, &info) != cudaSuccess) {
            cudaGetLastError();  // clear the failed update
            cudaGraphExecDestroy(gs[slot].exec);
            gs.erase(gs.begin() + slot);
            slot = gs.size();
        }
    }
    if (slot == gs.size()) {
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        if (gs.size() >= 8) {  // keep the 8 most recent launch shapes
            cudaGraphExecDestroy(gs.front().exec);
            gs.erase(gs.begin());
        }
        gs.push_back({shape, 0, exec, 0, {}});
        slot = gs.size() - 1;
    }
    cudaGraphDestroy(g);
    gs[slot].args = args;
    *out = &gs[slot];
    return NRRS_OK;
}

nrrs_status ensure_train_nets(nrrs_scene* sc, cudaStream_t s);  // training state (below)

// One frame (see nrrs_render); with `rec` every depth's slots are recorded.
nrrs_status render_impl(nrrs_scene* scene, int32_t width, int32_t height, int32_t spp,
                        int32_t max_depth, int32_t rrs_mode, const nrrs_render_opts& o,
                        float* d_rgb, cudaStream_t s, nrrs_render_stats* stats,
                        const RecordView* rec, const float* params) {
    // a batched render takes its sizes from the job table (width = all pixels, height 1)
    const bool batch = scene->n_jobs > 0;
    const long long npix = batch ? scene->batch_npix : (long long)width * height;
    const long long P = batch ? scene->batch_P : npix * spp;
    const long long C = P * o.cap_factor;
    // after a failed training step the network sits out one frame: its depths take the
    // throughput heuristic (plain heuristic normalised RRS)
    const bool heur_frame = scene->heur_next && !rec &&
                            (rrs_mode == NRRS_RRS_NET || rrs_mode == NRRS_RRS_NET_MIX);
    auto kind_of = [&](int d) {
        const int k = factor_kind(rrs_mode, o.gate, d);
        return heur_frame && k == kFactorNet ? (int)kFactorHeur : k;
    };
    bool uses_net = false, uses_adrrs = false;  // features are written for both
    for (int d = 1; d <= max_depth; ++d) {
        if (kind_of(d) == kFactorNet) uses_net = true;
        if (kind_of(d) == kFactorAdrrs) uses_adrrs = true;
    }
    // RRSNet fed the NRRS inputs needs StatNet at its depths
    const bool nrrs_inputs = scene->rrsnet_inputs == 1 && uses_net;
    const bool aid_inputs = scene->rrsnet_inputs == 2 && uses_net;
    if (aid_inputs) {  // RRSNet's hash grid lives with the training state
        nrrs_status trc = ensure_train_nets(scene, s);
        if (trc != NRRS_OK) return trc;
    }
    if (uses_adrrs || nrrs_inputs) {  // StatNet's weights (trained by nrrs_train_step)
        nrrs_status trc = ensure_train_nets(scene, s);
        if (trc != NRRS_OK) return trc;
        uses_net = true;
    }
    const bool nee = o.nee != 0;
    nrrs_status rc = ensure_workspace(scene, C, npix, uses_net, nee);
    if (rc != NRRS_OK) return rc;
    Workspace& ws = scene->ws;
    if (nrrs_inputs && !ws.feat_net) CK(dalloc(&ws.feat_net, (size_t)ws.cap * 4));
    if (batch && scene->jw_grid < ws.grid_red) {  // per-block, per-job partials
        const int n = scene->n_jobs;
        cudaFree(scene->jw.part);
        cudaFree(scene->jw.cnt);
        scene->jw.part = nullptr;
        scene->jw.cnt = nullptr;
        CK(dalloc(&scene->jw.part, (size_t)ws.grid_red * n));
        CK(dalloc(&scene->jw.cnt, (size_t)ws.grid_red * n));
        scene->jw_grid = ws.grid_red;
    }

    // reference image for HEUR factors
    // HEUR factors, and the repair of non-finite network factors, read the reference
    bool uses_heur = uses_net;
    for (int d = 1; d <= max_depth; ++d)
        if (kind_of(d) == kFactorHeur) uses_heur = true;
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
    rp.budget = (double)P * (double)(o.budget_factor > 0 ? o.budget_factor : 1);
    rp.fc = ws.fc;
    rp.f_rate = o.f_rate;
    rp.q_max = o.q_max;
    rp.boxcox_lambda = o.boxcox_lambda;
    rp.ref = uses_heur ? ref : nullptr;
    rp.params = params ? params : scene->params;
    rp.trace = o.d_trace;
    rp.trace_mask = o.d_trace ? o.d_trace_mask : nullptr;
    rp.trace_count = reinterpret_cast<unsigned long long*>(o.d_trace_count);
    rp.trace_rows = o.trace_rows;
    rp.nee = nee ? 1 : 0;
    rp.stat_grid = scene->train.nets && scene->train.stat_enc
                       ? reinterpret_cast<const float2*>(scene->train.grid)
                       : nullptr;
    if (batch) {
        rp.jobs = scene->jw;
        rp.jobs.cap_factor = o.cap_factor;
        rp.jobs.budget_factor = o.budget_factor > 0 ? o.budget_factor : 1;
    } else {
        scene->cam.aspect = (float)width / (float)height;
    }
    const int normalized = rrs_mode == NRRS_RRS_HEUR_NORM || rrs_mode == NRRS_RRS_NET ||
                           rrs_mode == NRRS_RRS_NET_MIX;
    const int update = o.update_ref && !o.d_pixel_ref;
    // the fused shade + RRSNet kernel serves the tensor-core precisions on the 16 vertex
    // features (not the NRRS or AID inputs, which need StatNet or the grid first)
    const bool fuse = scene->fuse_net && (o.precision == 16 || o.precision == 17) &&
                      !nrrs_inputs && !aid_inputs;

    // RRSNet launch shape per depth, from the queue sizes of the last frame
    RrsnetChoice net_shape[NRRS_MAX_DEPTH];
    for (int d = 1; d <= max_depth; ++d) {
        long long n = P;
        if (d > 1 && scene->last_P > 0)
            n = (long long)((double)scene->last_live[d - 1] * (double)P / (double)scene->last_P);
        net_shape[d - 1] = rrsnet_choice(scene, o.precision, n);
    }

    // the per-frame constants go to device memory ahead of the frame's launches
    launch_frame_consts(ws.fc, o.seed_lo, o.seed_hi ^ o.frame, scene->ref_count, s);
    unsigned extra_launches = 1 + (rp.ref ? 1u : 0u);  // + the reference's partial sums

    // profile 1 = every stage; otherwise bit (k + 1) selects stage k
    const unsigned pmask = o.profile == 1 ? 0xFFFFFFFFu : ((unsigned)o.profile >> 1);
    StageTimer tm{scene, s, pmask};

    // The frame's launch sequence.  In graph mode it is recorded once per set of launch
    // arguments on the scene's capture stream and replayed on the caller's stream.
    auto enqueue = [&](cudaStream_t s) -> nrrs_status {
        CK(cudaMemsetAsync(ws.st, 0, sizeof(DevStats), s));
        CK(cudaMemsetAsync(ws.acc_s, 0, sizeof(float4) * npix, s));
        CK(cudaMemsetAsync(ws.acc_c, 0, sizeof(float4) * npix, s));
#define TIMED(stage, call)           \
    do {                             \
        CK(tm.begin(stage));         \
        call;                        \
        CK(tm.end());                \
    } while (0)
        TIMED(NRRS_STAGE_INIT,
              launch_ref_prepare(rp.ref, npix * 3, o.eps_rel, (double)o.alpha0, P, ws.st,
                                 reinterpret_cast<float*>(ws.part), ws.grid_red, s));
        if (batch) TIMED(NRRS_STAGE_INIT, launch_ref_prepare_jobs(rp, o.eps_rel, s));
        QueueView q[2];
        for (int k = 0; k < 2; ++k)
            q[k] = QueueView{ws.qo[k], ws.qd[k], ws.qt[k], nee ? ws.qpdf[k] : nullptr};
        if (batch)
            TIMED(NRRS_STAGE_INIT, launch_camera_jobs(rp, P, q[0], s));
        else
            TIMED(NRRS_STAGE_INIT, launch_camera(scene->cam, rp, q[0], s));
        WorkView w{};
        w.hit = ws.hit; w.q = ws.q; w.dep = ws.dep; w.feat = ws.feat; w.part = ws.part;
        w.grid_red = ws.grid_red;
        w.bcnt = ws.bcnt; w.boff = ws.boff; w.grid_split = ws.grid_split;
        w.flags = ws.flags;
        w.acc_s = ws.acc_s; w.acc_c = ws.acc_c; w.st = ws.st;
        if (nee) {
            w.sh_o = ws.sh_o; w.sh_d = ws.sh_d; w.sh_c = ws.sh_c;
        }
        RenderParams r = rp;
        int cur = 0;
        float4* feat_net = ws.feat_net;
        for (int d = 1; d <= max_depth; ++d) {
            const int kind = kind_of(d);
            if (rec) {  // this depth's factors, deposits and features go straight to the record
                const size_t off = (size_t)(d - 1) * rec->C;
                w.q = rec->q + off;
                w.dep = rec->dep + off;
                w.feat = rec->feat + off * 4;
                if (nrrs_inputs) feat_net = rec->feat_net + off * 4;
                w.rough = rec->rough ? rec->rough + off : nullptr;
                r.rec_first = rec->first + off;
                r.rec_X = rec->X + off;
                CK(cudaMemcpyAsync(rec->t + off, q[cur].t, sizeof(float4) * C,
                                   cudaMemcpyDeviceToDevice, s));
            }
            TIMED(NRRS_STAGE_EXTEND,
                  launch_trace(scene->view, q[cur], w, d, scene->grid_trace, r.jobs, s));
            // NET depths on the tensor cores: shading and RRSNet in one kernel (the
            // features stay in shared memory) unless they must be recorded
            const bool fused = fuse && kind == kFactorNet && !rec;
            if (fused)
                TIMED(NRRS_STAGE_RRSNET,
                      launch_shade_rrsnet(o.precision, scene->n_sm, scene->view, q[cur], w, r, d,
                                          s));
            else
                TIMED(NRRS_STAGE_SHADE, launch_shade(kind, scene->view, q[cur], w, r, d, s));
            if (nee)  // shadow rays: unoccluded contributions join the deposits
                TIMED(NRRS_STAGE_SHADOW,
                      launch_shadow(scene->view, w, d, scene->grid_trace, r.jobs, s));
            if (kind == kFactorNet && aid_inputs) {  // AID-NRRS: RRSNet on its grid, FP32
                TIMED(NRRS_STAGE_RRSNET,
                      launch_aid_rrsnet(r.params, reinterpret_cast<const float2*>(scene->train.rgrid),
                                        scene->view, w, q[cur], r, d, scene->n_sm * 4, s));
                if (!batch) TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q(w, q[cur], r, d, s));
            } else if (kind == kFactorNet && fused) {
                if (!batch) TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q(w, q[cur], r, d, s));
            } else if (kind == kFactorNet) {
                if (nrrs_inputs)  // StatNet, then the NRRS inputs of RRSNet
                    TIMED(NRRS_STAGE_RRSNET,
                          launch_nrrs_inputs(scene->train.stat, scene->view, w, q[cur], r, d,
                                             scene->n_sm * 4, feat_net, s));
                TIMED(NRRS_STAGE_RRSNET,
                      launch_rrsnet(o.precision, net_shape[d - 1], scene->n_sm, r.params,
                                    nrrs_inputs ? feat_net : w.feat, &w.st->live[d - 1], 0, w.q,
                                    1, w.st, &w.st->status, s));
                if (!batch) TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q(w, q[cur], r, d, s));
            } else if (kind == kFactorAdrrs) {
                TIMED(NRRS_STAGE_RRSNET,
                      launch_adrrs(scene->train.stat, scene->view, w, q[cur], r, d,
                                   scene->n_sm * 4, s));
                if (!batch) TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q(w, q[cur], r, d, s));
            }
            if (batch) {  // Eq. F_norm per job
                TIMED(NRRS_STAGE_NORMALIZE, launch_sum_q_jobs(w, q[cur], r, d, s));
                TIMED(NRRS_STAGE_NORMALIZE, launch_normalize_jobs(w, r, d, normalized, s));
            } else {
                TIMED(NRRS_STAGE_NORMALIZE, launch_normalize_depth(w, r, d, normalized, s));
            }
            if (d < max_depth) {  // count, compaction and scatter in one pass
                CK(cudaMemsetAsync(ws.flags, 0, sizeof(unsigned long long) * ws.n_flags, s));
                TIMED(NRRS_STAGE_SCATTER,
                      launch_split_fused(scene->view, q[cur], q[cur ^ 1], w, r, d, s));
                cur ^= 1;
            } else {  // the last depth only deposits
                TIMED(NRRS_STAGE_COUNT, launch_split_count(scene->view, q[cur], w, r, d, 0, s));
                if (rec) CK(cudaMemsetAsync(r.rec_X, 0, sizeof(uint32_t) * C, s));
            }
        }
        TIMED(NRRS_STAGE_FINALIZE,
              launch_finalize(w, r, d_rgb, scene->ref_mean, update, npix, s));
        if (rec)
            for (int d = max_depth; d >= 1; --d)
                TIMED(NRRS_STAGE_REVERSE,
                      launch_reverse(*rec, d, max_depth, ws.st->live, ws.grid_red, s));
#undef TIMED
        CK(cudaGetLastError());
        return NRRS_OK;
    };

    if (!o.graph) {
        nrrs_status erc = enqueue(s);
        if (erc != NRRS_OK) return erc;
    } else {
        // shape: what fixes the kernels and their order; args: every launch argument
        // (pointers, sizes, options) apart from the per-frame constants
        uint64_t shape = 0;
        const uint64_t sv[] = {(uint64_t)width, (uint64_t)height, (uint64_t)spp,
                               (uint64_t)max_depth, (uint64_t)rrs_mode, (uint64_t)o.precision,
                               o.gate, (uint64_t)(rec != nullptr), (uint64_t)o.profile,
                               (uint64_t)heur_frame, (uint64_t)nee, (uint64_t)nrrs_inputs,
                               (uint64_t)fuse};
        for (uint64_t v : sv) shape = mix_key(shape, v);
        uint64_t args = shape;
        auto fbits = [](float f) { uint32_t u; std::memcpy(&u, &f, 4); return (uint64_t)u; };
        const uint64_t av[] = {(uint64_t)o.cap_factor, (uint64_t)o.budget_factor,
                               fbits(o.f_rate), fbits(o.alpha0),
                               fbits(o.q_max), fbits(o.eps_rel), fbits(o.boxcox_lambda),
                               (uint64_t)update, (uint64_t)(uintptr_t)rp.ref,
                               (uint64_t)(uintptr_t)rp.params, (uint64_t)(uintptr_t)o.d_trace,
                               (uint64_t)(uintptr_t)d_rgb, (uint64_t)(uintptr_t)scene->ref_mean,
                               (uint64_t)(uintptr_t)ws.st, (uint64_t)(uintptr_t)ws.qo[0],
                               (uint64_t)(uintptr_t)ws.feat, (uint64_t)ws.cap,
                               (uint64_t)(uintptr_t)(rec ? rec->q : nullptr),
                               (uint64_t)(rec ? rec->C : 0),
                               (uint64_t)fbits(scene->cam.aspect),
                               (uint64_t)(uintptr_t)scene->jw.part,
                               (uint64_t)(uintptr_t)scene->view.nodes4,
                               (uint64_t)(uintptr_t)scene->view.nodes_h,
                               (uint64_t)scene->view.short_stack,
                               (uint64_t)(uintptr_t)scene->train.stat,
                               (uint64_t)o.cap_factor, (uint64_t)(uintptr_t)ws.sh_o,
                               (uint64_t)(uintptr_t)ws.qpdf[0], (uint64_t)(uintptr_t)ws.feat_net,
                               (uint64_t)(uintptr_t)(rec ? rec->feat_net : nullptr),
                               (uint64_t)(uintptr_t)rp.stat_grid,
                               (uint64_t)(uintptr_t)(rec ? rec->rough : nullptr),
                               (uint64_t)scene->rrsnet_inputs,
                               (uint64_t)(uintptr_t)scene->train.rgrid,
                               (uint64_t)(uintptr_t)rp.trace_mask,
                               (uint64_t)(uintptr_t)rp.trace_count, (uint64_t)rp.trace_rows,
                               (uint64_t)(uintptr_t)scene->view.nodes8,
                               (uint64_t)(uintptr_t)scene->view.tris};
        for (uint64_t v : av) args = mix_key(args, v);
        for (int d = 1; d <= max_depth; ++d)
            args = mix_key(args, (uint64_t)(net_shape[d - 1].variant * 64 +
                                            net_shape[d - 1].blocks_per_sm));
        nrrs_scene::GraphEntry* ge = nullptr;
        for (auto& e : scene->graphs)
            if (e.shape == shape && e.args == args) ge = &e;
        if (!ge) {
            if (!scene->capture_stream)
                CK(cudaStreamCreateWithFlags(&scene->capture_stream, cudaStreamNonBlocking));
            CaptureGuard cg;
            cg.cs = scene->capture_stream;
            CK(cudaStreamBeginCapture(cg.cs, cudaStreamCaptureModeRelaxed));
            cg.active = true;
            tm.s = cg.cs;
            tm.capturing = true;
            nrrs_status erc = enqueue(cg.cs);
            if (erc != NRRS_OK) return erc;
            erc = finish_capture(scene, cg, shape, args, &ge);
            if (erc != NRRS_OK) return erc;
            ge->launches = tm.launches;
            ge->stage_of = tm.stage_of;
        } else {
            tm.launches = ge->launches;
            tm.stage_of = ge->stage_of;
        }
        CK(cudaGraphLaunch(ge->exec, s));
    }
    tm.launches += extra_launches;
    if (heur_frame) scene->heur_next = false;
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
        stats->status_bits = h.status | (heur_frame ? NRRS_STATUS_HEUR_FALLBACK : 0u);
        stats->kernel_launches = tm.launches;
        tm.collect(stats);
        for (int d = 0; d < NRRS_MAX_DEPTH; ++d) scene->last_live[d] = d < max_depth ? h.live[d] : 0;
        scene->last_P = P;
        if (batch) {
            const size_t m = (size_t)max_depth * scene->n_jobs;
            scene->job_F.resize(m);
            scene->job_sum_q.resize(m);
            scene->job_live.resize(m);
            CK(cudaMemcpy(scene->job_F.data(), scene->jw.F, sizeof(float) * m,
                          cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(scene->job_sum_q.data(), scene->jw.sum_q, sizeof(double) * m,
                          cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(scene->job_live.data(), scene->jw.live, sizeof(long long) * m,
                          cudaMemcpyDeviceToHost));
        }
    }
    return NRRS_OK;
}

}  // namespace

extern "C" {

nrrs_status nrrs_render(nrrs_scene* scene, int32_t width, int32_t height, int32_t spp,
                        int32_t max_depth, int32_t rrs_mode, const nrrs_render_opts* opts,
                        float* d_rgb, void* stream, nrrs_render_stats* stats) {
    if (!scene || !d_rgb) return fail(NRRS_ERR_INVALID_ARG, "scene or d_rgb is NULL");
    if (scene->n_jobs > 0) return fail(NRRS_ERR_INVALID_ARG, "a batch renders with nrrs_render_batch");
    nrrs_render_opts o = opts ? *opts : render_defaults();
    nrrs_status rc = validate_render(scene, width, height, spp, max_depth, rrs_mode, o);
    if (rc != NRRS_OK) return rc;
    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const long long npix = (long long)width * height;
    const long long C = npix * spp * o.cap_factor;
    const RecordView* rec = nullptr;
    if (o.d_suffix) {
        rc = ensure_record(scene, C, max_depth, npix);
        if (rc != NRRS_OK) return rc;
        scene->train.rec.C = C;
        rec = &scene->train.rec;
    }
    rc = render_impl(scene, width, height, spp, max_depth, rrs_mode, o, d_rgb, s, stats, rec,
                     nullptr);
    if (rc != NRRS_OK) return rc;
    if (o.d_suffix)
        for (int d = 0; d < max_depth; ++d)
            CK(cudaMemcpyAsync(o.d_suffix + (size_t)d * C * 4, rec->S + (size_t)d * C,
                               sizeof(float4) * C, cudaMemcpyDeviceToDevice, s));
    return NRRS_OK;
}

}  // extern "C"

extern "C" {

nrrs_status nrrs_create_batch(const nrrs_job* jobs, int32_t n_jobs, int32_t device,
                              nrrs_scene** out) {
    if (!out) return fail(NRRS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > NRRS_MAX_JOBS)
        return fail(NRRS_ERR_INVALID_ARG, "need 1 .. NRRS_MAX_JOBS jobs");
    long long npix = 0, P = 0;
    int Dmax = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const nrrs_job& J = jobs[j];
        if (!J.tri || !J.tri_mat || !J.mats || !J.cam || J.n_tri < 1 || J.n_mat < 1)
            return fail(NRRS_ERR_INVALID_ARG, "NULL job array or empty job scene");
        if (J.width < 1 || J.height < 1 || J.spp < 1 || J.max_depth < 1 ||
            J.max_depth > NRRS_MAX_DEPTH)
            return fail(NRRS_ERR_INVALID_ARG, "bad job image size, spp or depth");
        for (int32_t i = 0; i < J.n_tri; ++i)
            if (J.tri_mat[i] < 0 || J.tri_mat[i] >= J.n_mat)
                return fail(NRRS_ERR_INVALID_ARG, "material id out of range");
        for (int32_t i = 0; i < J.n_mat; ++i)
            if (J.mats[i].type != 0 && J.mats[i].type != 1)
                return fail(NRRS_ERR_INVALID_ARG, "unknown material type");
        npix += (long long)J.width * J.height;
        P += (long long)J.width * J.height * J.spp;
        Dmax = std::max(Dmax, (int)J.max_depth);
    }
    if (npix >= (1ll << 31) || 2 * P >= (1ll << 31))
        return fail(NRRS_ERR_INVALID_ARG, "batch too large (pixels or paths >= 2^31)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(NRRS_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");

    // one BVH per job, merged: child indices, triangle references and material ids are
    // rebased so that every job's tree is a separate root in the same arrays
    BvhHost all;
    Bvh4Host all4;
    bool wide = true;
    std::vector<nrrs_material> mats;
    std::vector<JobDev> jd(n_jobs);
    EmitterHost em_all;  // each job's emitters, one range per job (materials rebased)
    int64_t n_tri = 0;
    long long pbase = 0, prim = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const nrrs_job& J = jobs[j];
        BvhHost b;
        build_bvh(J.tri, J.n_tri, J.tri_mat, &b);
        Bvh4Host b4;
        collapse_bvh4(b, &b4);
        wide = wide && b4.max_stack <= trace_stack_entries();
        const int32_t node4_off = (int32_t)all4.nodes.size();
        const int32_t node_off = (int32_t)all.nodes.size();
        const int32_t ref_off = all.n_ref;
        const int32_t mat_off = (int32_t)mats.size();
        for (BvhNode nd : b.nodes) {
            for (int k = 0; k < 2; ++k)
                nd.d[k] = nd.d[k] >= 0 ? nd.d[k] + node_off : ~(~nd.d[k] + ref_off);
            all.nodes.push_back(nd);
        }
        for (Bvh4Node nd : b4.nodes) {
            for (int k = 0; k < 4; ++k)
                nd.child[k] = nd.child[k] >= 0 ? nd.child[k] + node4_off
                                               : ~(~nd.child[k] + ref_off);
            all4.nodes.push_back(nd);
        }
        for (int32_t r = 0; r < b.n_ref; ++r) {
            float t[12];
            std::memcpy(t, &b.tris[(size_t)r * 12], sizeof(t));
            int32_t m;
            std::memcpy(&m, &t[7], 4);
            m += mat_off;
            std::memcpy(&t[7], &m, 4);
            all.tris.insert(all.tris.end(), t, t + 12);
        }
        all.n_ref += b.n_ref;
        mats.insert(mats.end(), J.mats, J.mats + J.n_mat);
        n_tri += J.n_tri;
        JobDev& d = jd[j];
        const EmitterHost em = build_emitters(J.tri, J.n_tri, J.tri_mat, J.mats);
        d.emit_base = (int)em_all.cdf.size();
        d.n_emit = (int)em.cdf.size();
        d.inv_area = em.area > 0.0 ? (float)(1.0 / em.area) : 0.0f;
        for (size_t k = 0; k < em.tri.size(); ++k) {
            float4 v = em.tri[k];
            if (k % 3 == 0) {
                uint32_t m;
                std::memcpy(&m, &v.w, 4);
                m += (uint32_t)mat_off;
                std::memcpy(&v.w, &m, 4);
            }
            em_all.tri.push_back(v);
        }
        em_all.cdf.insert(em_all.cdf.end(), em.cdf.begin(), em.cdf.end());
        em_all.area += em.area;
        d.pixel_base = pbase;
        d.prim_base = prim;
        d.prims = (long long)J.width * J.height * J.spp;
        d.W = J.width; d.H = J.height; d.spp = J.spp; d.D = J.max_depth;
        d.root = node_off;
        d.root4 = node4_off;
        for (int k = 0; k < 3; ++k) {
            d.lo[k] = b.lo[k];
            const float ext = b.hi[k] - b.lo[k];
            d.inv_ext[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
            all.lo[k] = j == 0 ? b.lo[k] : std::min(all.lo[k], b.lo[k]);
            all.hi[k] = j == 0 ? b.hi[k] : std::max(all.hi[k], b.hi[k]);
        }
        d.cam = cam_view(*J.cam);
        d.cam.aspect = (float)J.width / (float)J.height;
        pbase += (long long)J.width * J.height;
        prim += d.prims;
    }
    nrrs_scene* s = nullptr;
    nrrs_status rc = upload_scene(all, wide ? &all4 : nullptr, n_tri, mats.data(),
                                  (int32_t)mats.size(), nullptr, em_all, device, &s);
    if (rc != NRRS_OK) return rc;
    s->n_jobs = n_jobs;
    s->jobs_host = jd;
    s->batch_P = P;
    s->batch_npix = npix;
    s->batch_D = Dmax;
    JobWork& w = s->jw;
    w.n = n_jobs;
    cudaError_t e = dalloc(&s->jobs_dev, (size_t)n_jobs);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->jobs_dev, jd.data(), sizeof(JobDev) * n_jobs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dalloc(&w.F_cur, (size_t)n_jobs);
    if (e == cudaSuccess) e = dalloc(&w.eps_I, (size_t)n_jobs);
    if (e == cudaSuccess) e = dalloc(&w.F, (size_t)kMaxDepth * n_jobs);
    if (e == cudaSuccess) e = dalloc(&w.sum_q, (size_t)kMaxDepth * n_jobs);
    if (e == cudaSuccess) e = dalloc(&w.live, (size_t)kMaxDepth * n_jobs);
    w.job = s->jobs_dev;
    if (e != cudaSuccess) {
        nrrs_status st = cuda_fail(e, "batch tables");
        destroy(s);
        return st;
    }
    *out = s;
    return NRRS_OK;
}

nrrs_status nrrs_render_batch(nrrs_scene* scene, int32_t rrs_mode, const nrrs_render_opts* opts,
                              float* d_rgb, void* stream, nrrs_render_stats* stats,
                              int64_t* job_live, float* job_F, double* job_sum_q) {
    if (!scene || !d_rgb) return fail(NRRS_ERR_INVALID_ARG, "scene or d_rgb is NULL");
    if (scene->n_jobs == 0) return fail(NRRS_ERR_INVALID_ARG, "not a batch (nrrs_create_batch)");
    nrrs_render_opts o = opts ? *opts : render_defaults();
    if (o.d_trace || o.d_suffix)
        return fail(NRRS_ERR_UNSUPPORTED, "trace and suffix records are single-scene only");
    nrrs_status rc = validate_render(scene, 1, 1, 1, scene->batch_D, rrs_mode, o);
    if (rc != NRRS_OK) return rc;
    if (scene->batch_P * o.cap_factor >= (1ll << 31))
        return fail(NRRS_ERR_INVALID_ARG, "capacity >= 2^31");
    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    nrrs_render_stats local;
    const bool want_jobs = job_live || job_F || job_sum_q;
    rc = render_impl(scene, (int32_t)scene->batch_npix, 1, 1, scene->batch_D, rrs_mode, o, d_rgb,
                     (cudaStream_t)stream, stats ? stats : (want_jobs ? &local : nullptr),
                     nullptr, nullptr);
    if (rc != NRRS_OK) return rc;
    const int n = scene->n_jobs, D = scene->batch_D;
    for (int j = 0; j < n; ++j)
        for (int d = 0; d < NRRS_MAX_DEPTH; ++d) {
            const bool in = d < D;
            const size_t k = (size_t)d * n + j;
            if (job_live) job_live[(size_t)j * NRRS_MAX_DEPTH + d] = in ? scene->job_live[k] : 0;
            if (job_F) job_F[(size_t)j * NRRS_MAX_DEPTH + d] = in ? scene->job_F[k] : 0.0f;
            if (job_sum_q) job_sum_q[(size_t)j * NRRS_MAX_DEPTH + d] = in ? scene->job_sum_q[k] : 0.0;
        }
    return NRRS_OK;
}

nrrs_status nrrs_batch_info(const nrrs_scene* scene, int32_t* n_jobs, int64_t* pixel_base,
                            int64_t* n_pixels_total) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (n_jobs) *n_jobs = scene->n_jobs;
    if (pixel_base)
        for (int j = 0; j < scene->n_jobs; ++j) pixel_base[j] = scene->jobs_host[j].pixel_base;
    if (n_pixels_total) *n_pixels_total = scene->batch_npix;
    return NRRS_OK;
}

}  // extern "C"

extern "C" {

nrrs_status nrrs_query_factors(nrrs_scene* scene, const float* d_features, int64_t n,
                               int32_t precision, float* d_q, void* stream) {
    if (!scene || n < 0 || (n > 0 && (!d_features || !d_q)))
        return fail(NRRS_ERR_INVALID_ARG, "bad query arguments");
    if (precision != 32 && precision != 16 && precision != 8 && precision != 17)
        return fail(NRRS_ERR_UNSUPPORTED, "precision must be 32, 16, 17 or 8");
    if (scene->rrsnet_inputs == 2)
        return fail(NRRS_ERR_UNSUPPORTED, "the AID-NRRS network encodes its inputs inside the render");
    if (n == 0) return NRRS_OK;
    if ((reinterpret_cast<uintptr_t>(d_features) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_features must be 16-byte aligned");
    DeviceGuard g(scene->device);
    launch_rrsnet(precision, rrsnet_choice(scene, precision, n), scene->n_sm, scene->params,
                  reinterpret_cast<const float4*>(d_features), nullptr, n, d_q, 0, nullptr,
                  nullptr, (cudaStream_t)stream);
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

namespace {

// Xavier-uniform start for StatNet from a fixed linear congruential stream (the library
// has no other source of randomness for it; callers may overwrite it with nrrs_set_params).
void default_statnet(std::vector<float>& w, int n_in) {
    const int shapes[4][2] = {{kNH, n_in}, {kNH, kNH}, {kNH, kNH}, {kStatOut, kNH}};
    uint64_t x = 0x5eed5eed12345ull;
    size_t p = 0;
    for (auto& sh : shapes) {
        const double a = std::sqrt(6.0 / (sh[0] + sh[1]));
        for (int i = 0; i < sh[0] * sh[1]; ++i) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            const double u = (double)(x >> 11) * (1.0 / 9007199254740992.0);
            w[p++] = (float)((2.0 * u - 1.0) * a);
        }
    }
}

// StatNet's weights afresh for its current inputs (and the hash grid's entries uniform in
// +-1e-4, as Instant-NGP starts them, from the same fixed stream), moments zeroed.
nrrs_status init_statnet(nrrs_scene* sc, cudaStream_t s) {
    TrainState& t = sc->train;
    const int n = t.stat_n();
    std::vector<float> w(n);
    default_statnet(w, t.stat_enc ? kStatGridIn : kNF);
    CK(cudaMemcpy(t.stat, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.stat_good, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    CK(cudaMemsetAsync(t.stat_m, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(t.stat_v, 0, sizeof(float) * n, s));
    if (t.stat_enc) {
        if (!t.grid) {
            CK(dalloc(&t.grid, (size_t)kGridParams));
            CK(dalloc(&t.grid_m, (size_t)kGridParams));
            CK(dalloc(&t.grid_v, (size_t)kGridParams));
            CK(dalloc(&t.grid_good, (size_t)kGridParams));
            CK(dalloc(&t.grid_grad, (size_t)kGridParams));
        }
        std::vector<float> g((size_t)kGridParams);
        uint64_t x = 0x6a09e667f3bcc908ull;
        for (auto& v : g) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            v = (float)(((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * 1e-4);
        }
        CK(cudaMemcpy(t.grid, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(t.grid_good, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice));
        CK(cudaMemsetAsync(t.grid_m, 0, sizeof(float) * g.size(), s));
        CK(cudaMemsetAsync(t.grid_v, 0, sizeof(float) * g.size(), s));
    }
    return NRRS_OK;
}

constexpr int kStatParamsMax = kNH * kStatGridIn + 2 * kNH * kNH + kStatOut * kNH;

nrrs_status ensure_train_nets(nrrs_scene* sc, cudaStream_t s) {
    TrainState& t = sc->train;
    if (t.nets) return NRRS_OK;
    CK(dalloc(&t.rrs_raw, kRrsParamsMax));
    CK(dalloc(&t.rrs_m, kRrsParamsMax));
    CK(dalloc(&t.rrs_v, kRrsParamsMax));
    CK(dalloc(&t.rrs_good, kRrsParamsMax));
    CK(dalloc(&t.stat, kStatParamsMax));
    CK(dalloc(&t.stat_m, kStatParamsMax));
    CK(dalloc(&t.stat_v, kStatParamsMax));
    CK(dalloc(&t.stat_good, kStatParamsMax));
    CK(dalloc(&t.grad_rrs, kRrsParamsMax));
    CK(dalloc(&t.grad_stat, kStatParamsMax));
    t.part_blocks = sc->n_sm * 3;
    CK(dalloc(&t.part, (size_t)t.part_blocks * kStatParamsMax));
    CK(dalloc(&t.loss_part, t.part_blocks));
    CK(dalloc(&t.scal, 8));
    CK(dalloc(&t.fscal, 8));
    CK(dalloc(&t.kpart, t.part_blocks));
    CK(dalloc(&t.nsamp, 1));
    CK(dalloc(&t.Fd, kMaxDepth));
    CK(dalloc(&t.Fnd, kMaxDepth));
    CK(dalloc(&t.bad, 1));
    const int nr = rrs_n(sc);
    CK(cudaMemcpyAsync(t.rrs_raw, sc->params, sizeof(float) * nr, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t.rrs_good, sc->params, sizeof(float) * nr, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(t.rrs_m, 0, sizeof(float) * nr, s));
    CK(cudaMemsetAsync(t.rrs_v, 0, sizeof(float) * nr, s));
    nrrs_status rc = init_statnet(sc, s);
    if (rc != NRRS_OK) return rc;
    t.nets = true;
    return NRRS_OK;
}

nrrs_status init_rrsnet_shape(nrrs_scene* sc) {
    nrrs_status rc = ensure_train_nets(sc, nullptr);
    if (rc != NRRS_OK) return rc;
    TrainState& t = sc->train;
    const int nr = rrs_n(sc);
    std::vector<float> w(nr, 0.0f);
    if (sc->rrsnet_inputs == 2) {
        // Xavier-uniform start of the 32-input network (fixed stream), grid entries +-1e-4
        const int shapes[4][2] = {{kNH, kAidIn}, {kNH, kNH}, {kNH, kNH}, {1, kNH}};
        uint64_t x = 0x3c6ef372fe94f82bull;
        size_t p = 0;
        for (auto& sh : shapes) {
            const double a = std::sqrt(6.0 / (sh[0] + sh[1]));
            for (int i = 0; i < sh[0] * sh[1]; ++i) {
                x = x * 6364136223846793005ull + 1442695040888963407ull;
                w[p++] = (float)(((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * a);
            }
        }
        if (!t.rgrid) {
            float** gs[] = {&t.rgrid, &t.rgrid_raw, &t.rgrid_m, &t.rgrid_v, &t.rgrid_good,
                            &t.rgrid_grad};
            for (float** gp : gs) CK(dalloc(gp, (size_t)kGridParams));
        }
        std::vector<float> g((size_t)kGridParams);
        for (auto& v : g) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            v = (float)(((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * 1e-4);
        }
        for (float* gd : {t.rgrid, t.rgrid_raw, t.rgrid_good})
            CK(cudaMemcpy(gd, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice));
        CK(cudaMemset(t.rgrid_m, 0, sizeof(float) * g.size()));
        CK(cudaMemset(t.rgrid_v, 0, sizeof(float) * g.size()));
    }
    for (float* d : {sc->params, t.rrs_raw, t.rrs_good})
        CK(cudaMemcpy(d, w.data(), sizeof(float) * nr, cudaMemcpyHostToDevice));
    CK(cudaMemset(t.rrs_m, 0, sizeof(float) * nr));
    CK(cudaMemset(t.rrs_v, 0, sizeof(float) * nr));
    CK(cudaDeviceSynchronize());
    return NRRS_OK;
}

nrrs_train_opts train_defaults() {
    nrrs_train_opts o;
    std::memset(&o, 0, sizeof(o));
    o.width = 256; o.height = 256; o.spp = 2; o.max_depth = 16;
    o.seed_lo = 1; o.warmup_steps = 20;
    o.lr_rrsnet = 3e-4f; o.lr_statnet = 5e-3f;
    o.gamma1 = 0.01f; o.gamma2 = 0.05f; o.gamma3 = 0.01f;
    o.eps = 0.01f; o.ema_decay = 0.99f; o.f_rate = 0.85f;
    o.alpha_mix = 0.5f; o.error_filter_radius = 2; o.error_filter_power = 8.0f;
    return o;
}

}  // namespace

extern "C" {

nrrs_status nrrs_set_params(nrrs_scene* scene, int32_t which, const float* params, int32_t n,
                            void* stream) {
    if (!scene || !params) return fail(NRRS_ERR_INVALID_ARG, "NULL scene or params");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    nrrs_status rc = ensure_train_nets(scene, s);
    if (rc != NRRS_OK) return rc;
    TrainState& t = scene->train;
    const long long want = which == NRRS_NET_STATNET ? t.stat_n()
                           : which == NRRS_NET_STATNET_GRID || which >= NRRS_NET_RRSNET_GRID
                               ? kGridParams
                               : rrs_n(scene);
    if (which < 0 || which > 5 || n != want) return fail(NRRS_ERR_INVALID_ARG, "bad network or size");
    if (which == NRRS_NET_STATNET_GRID && !t.stat_enc)
        return fail(NRRS_ERR_UNSUPPORTED, "StatNet has no hash grid (nrrs_set_statnet_encoding)");
    if (which >= NRRS_NET_RRSNET_GRID && scene->rrsnet_inputs != 2)
        return fail(NRRS_ERR_UNSUPPORTED, "RRSNet has no hash grid (nrrs_set_rrsnet_inputs(2))");
    float* dst = which == NRRS_NET_RRSNET ? scene->params : which == NRRS_NET_RRSNET_TRAIN ? t.rrs_raw
                 : which == NRRS_NET_STATNET ? t.stat : which == NRRS_NET_STATNET_GRID ? t.grid
                 : which == NRRS_NET_RRSNET_GRID ? t.rgrid : t.rgrid_raw;
    CK(cudaMemcpyAsync(dst, params, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    if (which == NRRS_NET_RRSNET_GRID_TRAIN) {
        CK(cudaMemcpyAsync(t.rgrid_good, params, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(t.rgrid_m, 0, sizeof(float) * n, s));
        CK(cudaMemsetAsync(t.rgrid_v, 0, sizeof(float) * n, s));
    }
    if (which == NRRS_NET_STATNET || which == NRRS_NET_STATNET_GRID) {
        float* good = which == NRRS_NET_STATNET ? t.stat_good : t.grid_good;
        float* m = which == NRRS_NET_STATNET ? t.stat_m : t.grid_m;
        float* v = which == NRRS_NET_STATNET ? t.stat_v : t.grid_v;
        CK(cudaMemcpyAsync(good, params, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(m, 0, sizeof(float) * n, s));
        CK(cudaMemsetAsync(v, 0, sizeof(float) * n, s));
    }
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

nrrs_status nrrs_set_statnet_encoding(nrrs_scene* scene, int32_t mode) {
    if (!scene || (mode != 0 && mode != 1)) return fail(NRRS_ERR_INVALID_ARG, "bad StatNet encoding");
    DeviceGuard g(scene->device);
    nrrs_status rc = ensure_train_nets(scene, nullptr);
    if (rc != NRRS_OK) return rc;
    TrainState& t = scene->train;
    if (t.stat_enc == mode) return NRRS_OK;
    t.stat_enc = mode;
    cudaFree(t.rec.rough);  // recorded roughness belongs to the encoded inputs
    t.rec.rough = nullptr;
    rc = init_statnet(scene, nullptr);
    if (rc != NRRS_OK) return rc;
    CK(cudaDeviceSynchronize());
    return NRRS_OK;
}

nrrs_status nrrs_get_params(nrrs_scene* scene, int32_t which, float* params, int32_t n, void* stream) {
    if (!scene || !params) return fail(NRRS_ERR_INVALID_ARG, "NULL scene or params");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    nrrs_status rc = ensure_train_nets(scene, s);
    if (rc != NRRS_OK) return rc;
    TrainState& t = scene->train;
    const long long want = which == NRRS_NET_STATNET ? t.stat_n()
                           : which == NRRS_NET_STATNET_GRID || which >= NRRS_NET_RRSNET_GRID
                               ? kGridParams
                               : rrs_n(scene);
    if (which < 0 || which > 5 || n != want) return fail(NRRS_ERR_INVALID_ARG, "bad network or size");
    if (which == NRRS_NET_STATNET_GRID && !t.stat_enc)
        return fail(NRRS_ERR_UNSUPPORTED, "StatNet has no hash grid (nrrs_set_statnet_encoding)");
    if (which >= NRRS_NET_RRSNET_GRID && scene->rrsnet_inputs != 2)
        return fail(NRRS_ERR_UNSUPPORTED, "RRSNet has no hash grid (nrrs_set_rrsnet_inputs(2))");
    const float* src = which == NRRS_NET_RRSNET ? scene->params : which == NRRS_NET_RRSNET_TRAIN ? t.rrs_raw
                       : which == NRRS_NET_STATNET ? t.stat : which == NRRS_NET_STATNET_GRID ? t.grid
                       : which == NRRS_NET_RRSNET_GRID ? t.rgrid : t.rgrid_raw;
    CK(cudaMemcpyAsync(params, src, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NRRS_OK;
}

namespace {
nrrs_status mlp_grad_impl(nrrs_scene* scene, int32_t n_out, bool at_q, const float* d_params,
                          const float* d_x, const float* d_gout, int64_t n, float* d_grad,
                          void* stream, int n_in = kNF) {
    if ((reinterpret_cast<uintptr_t>(d_x) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_x must be 16-byte aligned");
    DeviceGuard g(scene->device);
    cudaStream_t s = (cudaStream_t)stream;
    nrrs_status rc = ensure_train_nets(scene, s);
    if (rc != NRRS_OK) return rc;
    TrainState& t = scene->train;
    const int P = kNH * n_in + 2 * kNH * kNH + n_out * kNH;
    TrainArgs a{};
    a.params = d_params;
    a.gin = d_gout;
    a.scale = 1.0f;
    RecordView r{};
    r.feat = reinterpret_cast<float4*>(const_cast<float*>(d_x));
    r.C = n;
    TrainBatch b{};
    b.D = 1;
    b.total = n;
    b.batch = n;
    b.net_mask = 1u;
    CK(launch_mlp_grad_given(n_out, at_q, a, r, b, t.part_blocks, t.part, t.loss_part, s, n_in));
    launch_reduce_grad(t.part, t.part_blocks, P, d_grad, s);
    CK(cudaGetLastError());
    return NRRS_OK;
}
}  // namespace

nrrs_status nrrs_mlp_grad(nrrs_scene* scene, int32_t n_out, const float* d_params, const float* d_x,
                          const float* d_gout, int64_t n, float* d_grad, void* stream) {
    if (!scene || (n_out != 1 && n_out != kStatOut) || n < 0 || !d_params || !d_grad ||
        (n > 0 && (!d_x || !d_gout)))
        return fail(NRRS_ERR_INVALID_ARG, "bad mlp_grad arguments");
    return mlp_grad_impl(scene, n_out, false, d_params, d_x, d_gout, n, d_grad, stream);
}

nrrs_status nrrs_statnet_grad(nrrs_scene* scene, const float* d_params, const float* d_x,
                              const float* d_gout, int64_t n, float* d_grad, void* stream) {
    if (!scene || n < 0 || !d_params || !d_grad || (n > 0 && (!d_x || !d_gout)))
        return fail(NRRS_ERR_INVALID_ARG, "bad statnet_grad arguments");
    return mlp_grad_impl(scene, kStatOut, false, d_params, d_x, d_gout, n, d_grad, stream,
                         kStatGridIn);
}

nrrs_status nrrs_statnet_inputs(nrrs_scene* scene, const float* d_feat, const float* d_rough,
                                int64_t n, float* d_x, void* stream) {
    if (!scene || n < 0 || (n > 0 && (!d_feat || !d_rough || !d_x)))
        return fail(NRRS_ERR_INVALID_ARG, "bad statnet_inputs arguments");
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_feat must be 16-byte aligned");
    if (!scene->train.nets || !scene->train.stat_enc)
        return fail(NRRS_ERR_UNSUPPORTED, "StatNet has no hash grid (nrrs_set_statnet_encoding)");
    if (n == 0) return NRRS_OK;
    DeviceGuard g(scene->device);
    launch_statnet_inputs(reinterpret_cast<const float4*>(d_feat), d_rough, n,
                          reinterpret_cast<const float2*>(scene->train.grid), d_x,
                          (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_grid_backward(nrrs_scene* scene, const float* d_feat, const float* d_dx,
                               int64_t n, float* d_grad, void* stream) {
    if (!scene || n < 0 || !d_grad || (n > 0 && (!d_feat || !d_dx)))
        return fail(NRRS_ERR_INVALID_ARG, "bad grid_backward arguments");
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_feat must be 16-byte aligned");
    if (n == 0) return NRRS_OK;
    DeviceGuard g(scene->device);
    launch_grid_backward(reinterpret_cast<const float4*>(d_feat), d_dx, n, d_grad,
                         (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_rrsnet_backward(nrrs_scene* scene, const float* d_params, const float* d_x,
                                 const float* d_gq, int64_t n, float* d_grad, void* stream) {
    if (!scene || n < 0 || !d_params || !d_grad || (n > 0 && (!d_x || !d_gq)))
        return fail(NRRS_ERR_INVALID_ARG, "bad rrsnet_backward arguments");
    return mlp_grad_impl(scene, 1, true, d_params, d_x, d_gq, n, d_grad, stream);
}

nrrs_status nrrs_tune_rrsnet(nrrs_scene* scene, int32_t precision, void* stream,
                             nrrs_tune_report* report) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (precision != 32 && precision != 16 && precision != 8 && precision != 17)
        return fail(NRRS_ERR_INVALID_ARG, "precision must be 32, 16, 17 or 8");
    static_assert(NRRS_TUNE_BUCKETS == kTuneBuckets, "bucket count");
    DeviceGuard g(scene->device);
    RrsnetChoice table[kTuneBuckets];
    long long rows[kTuneBuckets];
    float best[kTuneBuckets], dflt[kTuneBuckets];
    cudaError_t e = tune_rrsnet(precision, scene->n_sm, scene->params, 12582912ll,
                                (cudaStream_t)stream, table, rows, best, dflt);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(NRRS_ERR_OOM, "tuner buffers");
    }
    CK(e);
    const int p = precision_index(precision);
    for (int b = 0; b < kTuneBuckets; ++b) scene->tune[p][b] = table[b];
    scene->tuned[p] = true;
    if (report) {
        std::memset(report, 0, sizeof(*report));
        report->precision = precision;
        report->n_buckets = kTuneBuckets;
        for (int b = 0; b < kTuneBuckets; ++b) {
            report->rows[b] = rows[b];
            report->variant[b] = table[b].variant;
            report->blocks_per_sm[b] = table[b].blocks_per_sm;
            report->ms_best[b] = best[b];
            report->ms_default[b] = dflt[b];
        }
    }
    return NRRS_OK;
}

nrrs_status nrrs_set_rrsnet_shape(nrrs_scene* scene, int32_t precision, int32_t bucket,
                                  int32_t variant, int32_t blocks_per_sm) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (precision != 32 && precision != 16 && precision != 8 && precision != 17)
        return fail(NRRS_ERR_INVALID_ARG, "precision must be 32, 16, 17 or 8");
    if (bucket < -1 || bucket >= kTuneBuckets) return fail(NRRS_ERR_INVALID_ARG, "bad bucket");
    const bool ok_variant = precision == 32   ? (variant == 1 || variant == 2)
                            : precision == 8 ? variant == 0
                                             : (variant == 0 || variant == 1);
    if (!ok_variant || blocks_per_sm < 1 || blocks_per_sm > 32)
        return fail(NRRS_ERR_INVALID_ARG, "bad launch shape");
    const int p = precision_index(precision);
    if (!scene->tuned[p])
        for (int b = 0; b < kTuneBuckets; ++b) scene->tune[p][b] = default_choice(precision);
    for (int b = 0; b < kTuneBuckets; ++b)
        if (bucket < 0 || b == bucket) scene->tune[p][b] = RrsnetChoice{variant, blocks_per_sm};
    scene->tuned[p] = true;
    return NRRS_OK;
}

nrrs_status nrrs_rrsnet_forward(const float* d_params, const float* d_x, int64_t n, float* d_q,
                                void* stream) {
    if (n < 0 || !d_params || (n > 0 && (!d_x || !d_q)))
        return fail(NRRS_ERR_INVALID_ARG, "bad rrsnet_forward arguments");
    if ((reinterpret_cast<uintptr_t>(d_x) & 15u) != 0)
        return fail(NRRS_ERR_INVALID_ARG, "d_x must be 16-byte aligned");
    if (n == 0) return NRRS_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    launch_rrsnet(32, default_choice(32), sm_count(dev), d_params,
                  reinterpret_cast<const float4*>(d_x), nullptr, n, d_q, 0, nullptr, nullptr,
                  (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_rrsnet_dloss(const float* d_q_nrrs, const float* d_F, const float* d_Fn,
                              const float* d_t, const int32_t* d_pixel, const float* d_m1,
                              const float* d_m2, const float* d_E, double Ebar, const float* d_Iref,
                              const int32_t* d_k, int64_t n, float eps, float g1, float g2, float g3,
                              float* d_dq, void* stream) {
    if (n < 0 || (n > 0 && (!d_q_nrrs || !d_F || !d_Fn || !d_t || !d_pixel || !d_m1 || !d_m2 ||
                            !d_E || !d_Iref || !d_k || !d_dq)))
        return fail(NRRS_ERR_INVALID_ARG, "bad rrsnet_dloss arguments");
    launch_rrsnet_dloss(d_q_nrrs, d_F, d_Fn, d_t, d_pixel, d_m1, d_m2, d_E, (float)Ebar, d_Iref, d_k, n,
                        eps, g1, g2, g3, d_dq, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_ema(float* d_avg, const float* d_params, int32_t n, float decay, void* stream) {
    if (n < 0 || (n > 0 && (!d_avg || !d_params)) || !(decay >= 0.0f && decay <= 1.0f))
        return fail(NRRS_ERR_INVALID_ARG, "bad ema arguments");
    if (n > 0) launch_ema(d_avg, d_params, n, decay, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int32_t n,
                           int32_t step, float lr, float b1, float b2, float eps, void* stream) {
    if (n < 0 || step < 1 || (n > 0 && (!d_params || !d_grad || !d_m || !d_v)))
        return fail(NRRS_ERR_INVALID_ARG, "bad adam arguments");
    if (n > 0) launch_adam(d_params, d_grad, d_m, d_v, n, step, lr, b1, b2, eps, nullptr, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_train_step(nrrs_scene* scene, const nrrs_train_opts* opts, void* stream,
                            nrrs_train_stats* out) {
    if (!scene) return fail(NRRS_ERR_INVALID_ARG, "scene is NULL");
    if (scene->n_jobs > 0) return fail(NRRS_ERR_UNSUPPORTED, "training runs on a single scene");
    nrrs_train_opts o = opts ? *opts : train_defaults();
    nrrs_render_opts ro = render_defaults();
    ro.seed_lo = o.seed_lo;
    ro.seed_hi = o.seed_hi;
    ro.f_rate = o.f_rate;
    ro.d_pixel_ref = o.d_pixel_ref;
    ro.graph = o.graph;
    ro.nee = o.nee;
    nrrs_status rc = validate_render(scene, o.width, o.height, o.spp, o.max_depth, NRRS_RRS_NET, ro);
    if (rc != NRRS_OK) return rc;
    if (o.warmup_steps < 0 || !(o.eps > 0.0f) || !(o.ema_decay >= 0.0f && o.ema_decay < 1.0f) ||
        o.batch_size < 0)
        return fail(NRRS_ERR_INVALID_ARG, "bad training options");
    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    TrainState& t = scene->train;
    rc = ensure_train_nets(scene, s);
    if (rc != NRRS_OK) return rc;
    const int D = o.max_depth;
    const long long npix = (long long)o.width * o.height;
    const long long C = npix * o.spp * 2;
    if (t.npix != npix || scene->ref_w != o.width || scene->ref_h != o.height) t.e_first = true;
    rc = ensure_record(scene, C, D, npix);
    if (rc != NRRS_OK) return rc;
    t.rec.C = C;
    ro.frame = o.frame + (uint32_t)t.step;
    ro.update_ref = 0;  // the reference is the mean of the earlier frames; folded in below

    // 1. a recorded frame with the inference weights, NET factors at every depth
    nrrs_render_stats rs;
    rc = render_impl(scene, o.width, o.height, o.spp, D, NRRS_RRS_NET, ro, t.rgb, s, &rs, &t.rec,
                     nullptr);
    if (rc != NRRS_OK) return rc;
    TrainBatch b{};
    b.D = D;
    b.net_mask = D >= 32 ? 0xFFFFFFFFu : ((1u << D) - 1u);
    float Fh[kMaxDepth], Fnh[kMaxDepth];
    long long off = 0;
    for (int d = 0; d < D; ++d) {
        b.offset[d] = off;
        off += rs.live[d];
        Fh[d] = rs.F[d];
        // Eq. F_norm with the frame's budget N_px (the primary queue), downscale only, no
        // rate control
        const double fn = rs.sum_q[d] > 0.0 ? (double)(npix * o.spp) / rs.sum_q[d] : 1.0;
        Fnh[d] = (float)(fn < 1.0 ? fn : 1.0);
    }
    b.offset[D] = off;
    b.total = off;
    // Sec. 4 "Training": batches of 2^19 vertices, drawn by systematic sampling with an
    // offset that changes every step (a hash of the seeds and the step)
    const long long bs = o.batch_size > 0 ? o.batch_size : (1ll << 19);
    b.batch = std::min(off, bs);
    {
        uint64_t z = ((uint64_t)o.seed_lo << 32 | o.seed_hi) ^ (0x9E3779B97F4A7C15ull * (t.step + 1));
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;  // splitmix64 finaliser
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        b.phase = (uint32_t)(z >> 32);
    }
    CK(cudaMemcpy(t.Fd, Fh, sizeof(float) * D, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.Fnd, Fnh, sizeof(float) * D, cudaMemcpyHostToDevice));

    // 2. pixel errors against the reference (the mean of the earlier frames), smoothed in
    //    time (alpha_mix) and space (a filter guided by the first-hit normals, standing in
    //    for the denoiser; off from step error_filter_until on, as the paper turns its
    //    denoiser off for the last part of training)
    const bool have_ref = o.d_pixel_ref != nullptr || scene->ref_count > 0;
    const float* ref = o.d_pixel_ref ? o.d_pixel_ref : (scene->ref_count > 0 ? scene->ref_mean : t.rgb);
    launch_pixel_error(t.rec, o.spp, npix, ref, o.eps, t.V, t.E_cur, s);
    const int radius =
        o.error_filter_until > 0 && t.step >= o.error_filter_until ? 0 : o.error_filter_radius;
    const bool guided = radius > 0 && o.error_filter_power > 0.0f;
    if (guided) launch_pixel_normals(t.rec, o.spp, npix, t.pnrm, s);
    t.filter_launches = (radius > 0 ? 1 : 0) + (guided ? 1 : 0);
    launch_error_smoothing(t.E_cur, t.E_acc, t.E, o.width, o.height, o.alpha_mix, t.e_first ? 1 : 0,
                           radius, guided ? t.pnrm : nullptr, o.error_filter_power, s);
    t.e_first = false;
    if (!o.d_pixel_ref) {
        launch_ref_fold(scene->ref_mean, t.rgb, npix * 3, scene->ref_count, s);
        scene->ref_count++;
    }
    (void)have_ref;
    CK(cudaMemsetAsync(t.k, 0, sizeof(int) * npix, s));
    launch_count_samples(t.rec, b, t.k, scene->n_sm * 4, s);
    // Ebar, then L_min, L_avg, N (the partials borrow the gradient scratch)
    launch_pixel_terms(t.E, npix, t.k, t.part, t.kpart, t.part_blocks, t.fscal + 0, t.fscal + 1,
                       t.nsamp, s);
    float fterms[2];
    long long n_samples = 0;
    CK(cudaMemcpyAsync(fterms, t.fscal + 1, sizeof(float) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&n_samples, t.nsamp, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double host_terms[2] = {fterms[0], fterms[1]};  // L_min, L_avg
    const double N = (double)n_samples;

    // 3. StatNet (moments for the gradient transfer), then RRSNet
    TrainArgs a{};
    a.m1 = t.m1;
    a.m2 = t.m2;
    a.F = t.Fd;
    a.Fn = t.Fnd;
    a.E = t.E;
    a.Ebar = t.fscal + 0;
    a.ref = ref;
    a.k = t.k;
    a.eps = o.eps;
    a.g1 = o.gamma1;
    a.g2 = o.gamma2;
    a.g3 = o.gamma3;
    a.params = t.stat;
    a.scale = N > 0 ? (float)(1.0 / N) : 0.0f;
    const int stat_n = t.stat_n();
    const int rrs_np = rrs_n(scene);
    const bool aid = scene->rrsnet_inputs == 2;
    if (t.stat_enc || aid) {  // a hash grid trains: gradients at its features per slot
        if (t.dx_cap < b.batch) {
            cudaFree(t.dx);
            t.dx = nullptr;
            t.dx_cap = 0;
            CK(dalloc(&t.dx, (size_t)b.batch * 16));
            t.dx_cap = b.batch;
        }
    }
    if (t.stat_enc) {  // StatNet on the encodings: its hash grid
        a.grid = reinterpret_cast<const float2*>(t.grid);
        a.dx = t.dx;
    }
    a.lambda = 0.5f;  // the training frame's Box-Cox lambda (render default)
    CK(launch_mlp_train(kTrainStatNet, a, t.rec, b, t.part_blocks, t.part, t.loss_part, s));
    launch_reduce_grad(t.part, t.part_blocks, stat_n, t.grad_stat, s);
    launch_reduce_loss(t.loss_part, t.part_blocks, t.fscal + 3, s);
    if (t.stat_enc) {
        CK(cudaMemsetAsync(t.grid_grad, 0, sizeof(float) * (size_t)kGridParams, s));
        launch_grid_scatter(a, t.rec, b, scene->n_sm * 8, t.grid_grad, s);
    }
    a.grid = nullptr;
    a.dx = nullptr;
    const bool warm = t.step < o.warmup_steps;
    a.params = t.rrs_raw;
    a.scale = warm ? (N > 0 ? (float)(1.0 / N) : 0.0f) : 1.0f;
    if (aid) {  // AID-NRRS: RRSNet on its own hash grid
        a.grid = reinterpret_cast<const float2*>(t.rgrid_raw);
        a.dx = t.dx;
    }
    CK(launch_mlp_train(warm ? kTrainRrsWarmup : kTrainRrsFull, a, t.rec, b, t.part_blocks, t.part,
                        t.loss_part, s));
    launch_reduce_grad(t.part, t.part_blocks, rrs_np, t.grad_rrs, s);
    launch_reduce_loss(t.loss_part, t.part_blocks, t.fscal + 4, s);
    if (o.debug) {  // what the step is about to apply, for checks against a reference
        nrrs_train_debug& dbg = *o.debug;
        if (dbg.grad_statnet)
            CK(cudaMemcpyAsync(dbg.grad_statnet, t.grad_stat, sizeof(float) * stat_n,
                               cudaMemcpyDeviceToHost, s));
        if (dbg.grad_rrsnet)
            CK(cudaMemcpyAsync(dbg.grad_rrsnet, t.grad_rrs, sizeof(float) * rrs_np,
                               cudaMemcpyDeviceToHost, s));
        if (dbg.pixel_var)
            CK(cudaMemcpyAsync(dbg.pixel_var, t.V, sizeof(float) * npix, cudaMemcpyDeviceToHost, s));
        if (dbg.pixel_error)
            CK(cudaMemcpyAsync(dbg.pixel_error, t.E, sizeof(float) * npix, cudaMemcpyDeviceToHost, s));
        if (dbg.samples)
            CK(cudaMemcpyAsync(dbg.samples, t.k, sizeof(int) * npix, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&dbg.ebar, t.fscal + 0, sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        dbg.vertices = b.total;
        dbg.batch = b.batch;
    }
    if (aid) {
        CK(cudaMemsetAsync(t.rgrid_grad, 0, sizeof(float) * (size_t)kGridParams, s));
        launch_grid_scatter(a, t.rec, b, scene->n_sm * 8, t.rgrid_grad, s);
    }

    // 4. Adam for both networks (Sec. 4 "Training": lr 0.005 StatNet, 0.0003 RRSNet)
    CK(cudaMemsetAsync(t.bad, 0, sizeof(int), s));
    const int step = (int)t.step + 1;
    launch_adam(t.stat, t.grad_stat, t.stat_m, t.stat_v, stat_n, step, o.lr_statnet, 0.9f,
                0.999f, 1e-8f, t.bad, s);
    if (t.stat_enc)  // the grid's entries take tiny gradients: Instant-NGP's epsilon 1e-15
        launch_adam(t.grid, t.grid_grad, t.grid_m, t.grid_v, (int)kGridParams, step,
                    o.lr_statnet, 0.9f, 0.999f, 1e-15f, t.bad, s);
    launch_adam(t.rrs_raw, t.grad_rrs, t.rrs_m, t.rrs_v, rrs_np, step, o.lr_rrsnet, 0.9f, 0.999f,
                1e-8f, t.bad, s);
    if (aid)
        launch_adam(t.rgrid_raw, t.rgrid_grad, t.rgrid_m, t.rgrid_v, (int)kGridParams, step,
                    o.lr_rrsnet, 0.9f, 0.999f, 1e-15f, t.bad, s);
    int bad = 0;
    float flosses[2];
    CK(cudaMemcpyAsync(&bad, t.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(flosses, t.fscal + 3, sizeof(float) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double losses[2] = {flosses[0], flosses[1]};
    const double loss_stat = N > 0 ? losses[0] / N : 0.0;
    const double loss_rrs_warm = N > 0 ? losses[1] / N : 0.0;
    const double L_rrs = losses[1];
    const double L_total = warm ? loss_rrs_warm
                                : o.gamma1 * host_terms[1] + o.gamma2 * host_terms[0] + o.gamma3 * L_rrs;
    int fallback = 0;
    if (bad || !std::isfinite(L_total) || !std::isfinite(loss_stat)) fallback = 1;
    // fallback monitor: after the warm-up, a slow loss EMA far above its running minimum
    // (divergence; single-frame Monte Carlo noise of the pixel errors is heavy-tailed)
    if (!fallback && !warm) {
        t.loss_ema = t.full_steps == 0 ? L_total : 0.98 * t.loss_ema + 0.02 * L_total;
        t.loss_min = t.full_steps == 0 ? t.loss_ema : std::min(t.loss_min, t.loss_ema);
        t.full_steps++;
        if (t.full_steps > 50 && t.loss_ema > 10.0 * t.loss_min) fallback = 2;
    }
    if (fallback) {  // restore the last good weights and forget the moments
        scene->heur_next = true;
        CK(cudaMemcpyAsync(t.rrs_raw, t.rrs_good, sizeof(float) * rrs_np, cudaMemcpyDeviceToDevice, s));
        if (aid) {
            CK(cudaMemcpyAsync(t.rgrid_raw, t.rgrid_good, sizeof(float) * (size_t)kGridParams,
                               cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(t.rgrid_m, 0, sizeof(float) * (size_t)kGridParams, s));
            CK(cudaMemsetAsync(t.rgrid_v, 0, sizeof(float) * (size_t)kGridParams, s));
        }
        CK(cudaMemcpyAsync(t.stat, t.stat_good, sizeof(float) * stat_n, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(t.rrs_m, 0, sizeof(float) * rrs_np, s));
        CK(cudaMemsetAsync(t.rrs_v, 0, sizeof(float) * rrs_np, s));
        CK(cudaMemsetAsync(t.stat_m, 0, sizeof(float) * stat_n, s));
        CK(cudaMemsetAsync(t.stat_v, 0, sizeof(float) * stat_n, s));
        if (t.stat_enc) {
            CK(cudaMemcpyAsync(t.grid, t.grid_good, sizeof(float) * (size_t)kGridParams,
                               cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(t.grid_m, 0, sizeof(float) * (size_t)kGridParams, s));
            CK(cudaMemsetAsync(t.grid_v, 0, sizeof(float) * (size_t)kGridParams, s));
        }
        if (fallback == 2) {
            t.loss_ema = t.loss_min;
        }
    } else {
        CK(cudaMemcpyAsync(t.rrs_good, t.rrs_raw, sizeof(float) * rrs_np, cudaMemcpyDeviceToDevice, s));
        if (aid)
            CK(cudaMemcpyAsync(t.rgrid_good, t.rgrid_raw, sizeof(float) * (size_t)kGridParams,
                               cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(t.stat_good, t.stat, sizeof(float) * stat_n, cudaMemcpyDeviceToDevice, s));
        if (t.stat_enc)
            CK(cudaMemcpyAsync(t.grid_good, t.grid, sizeof(float) * (size_t)kGridParams,
                               cudaMemcpyDeviceToDevice, s));
        // inference weights: EMA of the trained weights (Sec. 4 "Training", as in NRC), with
        // the usual warm start decay_t = min(decay, (1 + t) / (10 + t))
        const float warm_decay = (float)(1.0 + (double)t.step) / (float)(10.0 + (double)t.step);
        launch_ema(scene->params, t.rrs_raw, rrs_np, std::min(o.ema_decay, warm_decay), s);
        if (aid)  // the rendering grid is the EMA of the trained one, as the weights are
            launch_ema(t.rgrid, t.rgrid_raw, (int)kGridParams, std::min(o.ema_decay, warm_decay),
                       s);
        t.step++;
    }
    CK(cudaGetLastError());
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->step = t.step;
        out->samples = (int64_t)N;
        out->segments = rs.segments;
        out->loss_statnet = loss_stat;
        out->loss_rrsnet = warm ? loss_rrs_warm : L_total;
        out->loss_avg = host_terms[1];
        out->loss_min = host_terms[0];
        out->loss_rrs = warm ? 0.0 : L_rrs;
        out->phase = warm ? 1 : 2;
        out->fallback = fallback;
        // frame kernels; pixel error, temporal EMA, pixel normals + spatial filter,
        // reference fold, sample counts, mean, loss terms; 2 x (train, reduce grad,
        // reduce loss); 2 Adam; EMA
        out->kernel_launches = (int64_t)rs.kernel_launches + 2 + t.filter_launches +
                               (t.stat_enc ? 2 : 0) + (aid ? 3 : 0) +
                               (o.d_pixel_ref ? 0 : 1) + 3 + 6 + 2 + (fallback ? 0 : 1);
    }
    return NRRS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ Mix-Depth (Sec. 3.3)
extern "C" {

int64_t nrrs_mixdepth_candidates(int32_t max_depth, int32_t t_d) {
    if (max_depth < 1 || max_depth > NRRS_MAX_DEPTH || t_d < 1) return -1;
    int64_t total = 0;
    for (int start = 0; start < max_depth; start += t_d) {
        const int len = std::min(t_d, max_depth - start);
        int64_t c = 1;
        for (int k = 0; k < len; ++k) c *= 3;
        total += c;
    }
    return total;
}

nrrs_status nrrs_relmse(const float* d_img, const float* d_ref, int64_t n_pixels, double eps,
                        double* d_out, void* stream) {
    if (n_pixels < 0 || !d_out || (n_pixels > 0 && (!d_img || !d_ref)))
        return fail(NRRS_ERR_INVALID_ARG, "bad relmse arguments");
    launch_relmse(d_img, d_ref, n_pixels * 3, eps, d_out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_error_filter(const float* d_in, const float* d_normals, int32_t width,
                              int32_t height, int32_t radius, float power, float* d_out,
                              void* stream) {
    if (!d_in || !d_out || width < 1 || height < 1 || radius < 0)
        return fail(NRRS_ERR_INVALID_ARG, "bad error filter arguments");
    const float4* nrm = power > 0.0f ? reinterpret_cast<const float4*>(d_normals) : nullptr;
    if (radius == 0) {
        CK(cudaMemcpyAsync(d_out, d_in, sizeof(float) * (size_t)width * height,
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
        return NRRS_OK;
    }
    launch_error_filter(d_in, nrm, width, height, radius, power, d_out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NRRS_OK;
}

nrrs_status nrrs_mixdepth_search(nrrs_scene* scene, const nrrs_mixdepth_opts* opts, void* stream,
                                 nrrs_mixdepth_result* out) {
    if (!scene || !opts || !out) return fail(NRRS_ERR_INVALID_ARG, "NULL argument");
    if (scene->n_jobs > 0) return fail(NRRS_ERR_UNSUPPORTED, "Mix-Depth search runs on a single scene");
    const nrrs_mixdepth_opts o = *opts;
    const int D = o.max_depth;
    const int64_t total = nrrs_mixdepth_candidates(D, o.t_d);
    if (total < 0) return fail(NRRS_ERR_INVALID_ARG, "bad max_depth or t_d");
    if (o.max_candidates > 0 && total > o.max_candidates)
        return fail(NRRS_ERR_INVALID_ARG, "more candidates than max_candidates");
    nrrs_render_opts ro = render_defaults();
    ro.seed_lo = o.seed_lo;
    ro.seed_hi = o.seed_hi;
    ro.frame = o.frame;  // every candidate sees the same random numbers
    ro.update_ref = 0;
    ro.nee = o.nee;
    ro.precision = o.precision == 0 ? 32 : o.precision;
    nrrs_status rc = validate_render(scene, o.width, o.height, o.spp, D, NRRS_RRS_NET_MIX, ro);
    if (rc != NRRS_OK) return rc;
    DeviceGuard g(scene->device);
    if (!g.ok) return fail(NRRS_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const long long npix = (long long)o.width * o.height;
    const float* ref = o.d_pixel_ref ? o.d_pixel_ref
                                     : (scene->ref_count > 0 && scene->ref_w == o.width &&
                                        scene->ref_h == o.height ? scene->ref_mean : nullptr);
    if (!ref) return fail(NRRS_ERR_INVALID_ARG, "no reference image for the relMSE estimate");
    ro.d_pixel_ref = ref;
    rc = ensure_train_nets(scene, s);
    if (rc != NRRS_OK) return rc;
    TrainState& t = scene->train;
    if (t.npix < npix) {
        rc = ensure_record(scene, npix * o.spp * 2, 1, npix);
        if (rc != NRRS_OK) return rc;
    }
    // method digit order per depth: FIXED, HEUR or ADRRS (NN), NET (cheapest first; ties
    // keep the first)
    const uint64_t digit_gate[3] = {NRRS_GATE_FIXED,
                                    o.adrrs ? (uint64_t)NRRS_GATE_ADRRS : (uint64_t)NRRS_GATE_HEUR,
                                    NRRS_GATE_NET};
    uint64_t gate = 0;
    for (int d = 0; d < D; ++d) gate |= (uint64_t)NRRS_GATE_FIXED << (2 * d);
    double best_score = 0.0, best_rel = 0.0;
    int64_t best_segs = 0, evaluated = 0;
    for (int start = 0; start < D; start += o.t_d) {
        const int len = std::min(o.t_d, D - start);
        int64_t ncand = 1;
        for (int k = 0; k < len; ++k) ncand *= 3;
        uint64_t seg_best = gate;
        double seg_score = INFINITY;
        for (int64_t c = 0; c < ncand; ++c) {
            uint64_t gc = gate;
            int64_t x = c;
            for (int k = 0; k < len; ++k) {
                const int depth = start + k;
                gc &= ~(3ull << (2 * depth));
                gc |= digit_gate[x % 3] << (2 * depth);
                x /= 3;
            }
            ro.gate = gc;
            nrrs_render_stats rs;
            rc = render_impl(scene, o.width, o.height, o.spp, D, NRRS_RRS_NET_MIX, ro, t.rgb, s, &rs,
                             nullptr, nullptr);
            if (rc != NRRS_OK) return rc;
            launch_relmse(t.rgb, ref, npix * 3, 0.01, t.scal + 7, s);
            double rel = 0.0;
            CK(cudaMemcpyAsync(&rel, t.scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            ++evaluated;
            const double score = rel * (double)rs.segments;  // inverse efficiency
            if (score < seg_score) {
                seg_score = score;
                seg_best = gc;
                best_rel = rel;
                best_segs = rs.segments;
            }
        }
        gate = seg_best;
        best_score = seg_score;
    }
    std::memset(out, 0, sizeof(*out));
    out->gate = gate;
    out->score = best_score;
    out->relmse = best_rel;
    out->segments = best_segs;
    out->evaluated = evaluated;
    return NRRS_OK;
}

}  // extern "C"
