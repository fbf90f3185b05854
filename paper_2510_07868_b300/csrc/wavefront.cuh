// Device views and launchers of the wavefront bounce kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nrrs.h"
#include "common.cuh"

namespace nrrs {

struct SceneView {
    const float4* nodes;  // 4 float4 per node (bvh.cpp)
    const float4* nodes4; // four-wide tree, 8 float4 per node; NULL = traverse the BVH2
    const uint4* nodes_h; // the BVH2 with FP16 boxes, 2 uint4 per node; NULL = FP32 nodes
    const uint4* nodes8;  // compressed eight-wide tree (bvh8.cu), 5 uint4 per node; when set
                          // it is traversed and `tris` is that tree's triangle order
    const float4* tris;   // 3 float4 per triangle, BVH order
    const nrrs_material* mats;
    float lo[3];          // scene box, for the position feature
    float inv_ext[3];     // 1 / extent, 0 for a flat axis (feature = 0.5 there)
    // next-event estimation: emitting triangles (3 float4 each: v0 + material bits,
    // e1, e2) and their area CDF; a batch keeps one range per job (JobDev)
    const float4* emit;
    const float* emit_cdf;
    int n_emit;
    float inv_area;       // 1 / total emitter area
    int short_stack;      // 1: the BVH2's deepest path fits the short traversal stack
};

struct CamView {
    float pos[3], fw[3], right[3], up[3];
    float tan_half, aspect;
};

// Path state, structure of arrays (one slot per path, 48 bytes):
//   o = (origin, pixel bits), d = (direction, lineage bits), t = (throughput, sample bits)
struct QueueView {
    float4* o;
    float4* d;
    float4* t;
    float* pdf;  // next-event estimation: solid-angle pdf the direction was sampled with
};

// Device-resident per-render statistics; the host copies it once per render.
struct DevStats {
    long long live[kMaxDepth + 1];  // live[d-1] = queue length at depth d
    double sum_q[kMaxDepth];
    double alpha[kMaxDepth];
    long long requested[kMaxDepth];
    long long dropped[kMaxDepth];
    float F[kMaxDepth];
    unsigned long long fetch[kMaxDepth];  // dynamic ray-fetch counters of k_extend
    unsigned long long tiles[kMaxDepth];  // tile claims of the fused split
    unsigned long long sfetch[kMaxDepth]; // dynamic shadow-ray fetch counters
    unsigned long long nonfinite;
    unsigned long long net_evals;
    double alpha_cur;               // adaptive alpha (Eq. f_rate_prime), carried over depths
    float F_cur;                    // factor applied at the current depth
    float eps_I;                    // HEUR floor eps_rel * mean(reference)
    unsigned int status;            // NRRS_STATUS_* bits
    int has_ref;
};

// Per-bounce scratch shared by the kernels of one render.
struct WorkView {
    float2* hit;       // [C] (distance, BVH triangle slot bits; -1 = miss)
    float* q;          // [C] q_orig
    float4* dep;       // [C] (deposited radiance rgb, pixel bits)
    float4* feat;      // [C][4] RRSNet features (NET depths)
    double* part;      // [grid_red] partial sums of q
    int grid_red;      // blocks of the kernel that produced `part` at this depth
    unsigned long long* flags;  // [C / 256 + 1] look-back flags of the fused split
    unsigned long long* bcnt;  // [grid_split] children per block (64-bit: a block's
                               // parents may request up to 2^23 children each)
    unsigned long long* boff;  // [grid_split] exclusive prefix of bcnt
    int grid_split;
    float4* acc_s;     // [npix] Kahan sum (rgb)
    float4* acc_c;     // [npix] Kahan compensation (rgb)
    DevStats* st;
    // next-event estimation, per slot: shadow ray (origin, t_max <= 0: none),
    // (direction, -), and the unoccluded contribution (rgb, -)
    float4* sh_o;
    float4* sh_d;
    float4* sh_c;
    float* rough;      // [C] roughness of each network vertex (training of the grid StatNet)
};

// Per-frame values read by the kernels from device memory, so that one recorded launch
// sequence (a CUDA graph) serves every frame of the same shape.
struct FrameConsts {
    uint32_t key0, key1;  // Philox key
    int ref_count;        // frames folded into the running reference mean so far
    int pad;
};

// One job of a batched render: its own scene (BVH root, materials already rebased into
// the merged arrays), camera, image and depth, sharing the queue and the RRSNet.  Jobs
// are laid out one after another: global pixel = pixel_base + local pixel, primary slot
// = prim_base + local primary index (pixel-major, sample-minor).
struct JobDev {
    long long pixel_base, prim_base;
    long long prims;     // W * H * spp; the job's budget is C_j = cap_factor * prims
    int W, H, spp, D;
    int root;            // BVH2 root node of the job's scene
    int root4;           // four-wide root node (when the batch has a four-wide tree)
    float lo[3], inv_ext[3];  // the job's scene box (position feature)
    int emit_base, n_emit;    // the job's emitters in the merged emitter table
    float inv_area;           // 1 / the job's total emitter area
    CamView cam;
};

// Per-job device arrays of a batched render.
struct JobWork {
    const JobDev* job;   // [n]
    int n;
    int cap_factor;
    int budget_factor;   // job j's normalisation budget = budget_factor * prims
    float* F_cur;        // [n] normalisation factor of the current depth
    float* eps_I;        // [n] HEUR floor of each job
    double* part;        // [grid_red][n] per-block partial sums of q
    long long* cnt;      // [grid_red][n] per-block slot counts
    float* F;            // [kMaxDepth][n]
    double* sum_q;       // [kMaxDepth][n]
    long long* live;     // [kMaxDepth][n]
};

// Job of a global pixel (binary search over the jobs' pixel bases).
__device__ __forceinline__ int job_of_pixel(const JobDev* job, int n, uint32_t pix) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&job[mid].pixel_base) <= (long long)pix) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct RenderParams {
    int W, H, spp, D;
    long long cap;        // C
    double budget;        // N_px of Eq. F_norm (single scene; a batch: JobWork::budget_factor)
    const FrameConsts* fc;
    JobWork jobs;         // batched render (jobs.job != nullptr), else unused
    float f_rate;
    float q_max;
    float boxcox_lambda;
    const float* ref;     // reference image [npix*3] (running mean or caller's) or null
    const float* params;  // RRSNet weights (device, 2592 floats)
    uint32_t* trace;      // optional per-depth trace
    const uint8_t* trace_mask;         // with trace: compact rows for the marked pixels only
    unsigned long long* trace_count;   // rows recorded (compact form)
    long long trace_rows;              // capacity of the compact form
    uint32_t* rec_first;  // record mode: first child slot of every parent of this depth
    uint32_t* rec_X;      // record mode: children requested by every parent of this depth
    int nee;              // next-event estimation with MIS at every vertex
    const float2* stat_grid;  // StatNet's hash grid (StatNet reads the encodings of Sec. 4)
                              // or NULL (StatNet reads the vertex features)
};

enum FactorKind : int {
    kFactorOne = 0,
    kFactorPlain = 1,
    kFactorHeur = 2,
    kFactorNet = 3,   // RRSNet
    kFactorAdrrs = 4  // ADRRS (NN): StatNet's radiance over the pixel estimate
};

int extend_block_threads();
int split_block_threads();
int max_blocks_trace();  // resident blocks per SM
int trace_stack_entries();  // traversal stack size per ray
int trace_short_stack_entries();  // the short stack, for BVH2s no taller than it

void launch_ref_prepare(const float* ref, long long n3, float eps_rel, double alpha0,
                        long long P, DevStats* st, float* part, int G, cudaStream_t s);
void launch_camera(const CamView& cam, const RenderParams& rp, QueueView out, cudaStream_t s);
void launch_trace(const SceneView& sc, QueueView cur, const WorkView& w, int depth, int grid,
                  const JobWork& jobs, cudaStream_t s);
// Shadow rays of next-event estimation (any hit): adds the contribution of every
// unoccluded ray to the slot's deposit.
void launch_shadow(const SceneView& sc, const WorkView& w, int depth, int grid,
                   const JobWork& jobs, cudaStream_t s);
// NET depths with shading and the tensor-core RRSNet (precision 16: split BF16, 17:
// BF16) fused in one kernel; the features stay in shared memory.  Same q, deposits and
// shadow rays as launch_shade(kFactorNet) followed by launch_rrsnet with sentinel.
void launch_shade_rrsnet(int precision, int n_sm, const SceneView& sc, QueueView cur,
                         const WorkView& w, const RenderParams& rp, int depth, cudaStream_t s);
void launch_shade(int kind, const SceneView& sc, QueueView cur, const WorkView& w,
                  const RenderParams& rp, int depth, cudaStream_t s);

void launch_sum_q(const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                  cudaStream_t s);
void launch_normalize_depth(const WorkView& w, const RenderParams& rp, int depth, int normalized,
                            cudaStream_t s);
void launch_split_count(const SceneView& sc, QueueView cur, const WorkView& w,
                        const RenderParams& rp, int depth, int do_split, cudaStream_t s);
void launch_split_fused(const SceneView& sc, QueueView cur, QueueView nxt, const WorkView& w,
                        const RenderParams& rp, int depth, cudaStream_t s);
void launch_finalize(const WorkView& w, const RenderParams& rp, float* rgb, float* ref_mean,
                     int update_ref, long long npix, cudaStream_t s);
// Batched renders: per-job HEUR floors, per-job sums of q and normalisation factors.
void launch_ref_prepare_jobs(const RenderParams& rp, float eps_rel, cudaStream_t s);
void launch_sum_q_jobs(const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                       cudaStream_t s);
void launch_normalize_jobs(const WorkView& w, const RenderParams& rp, int depth, int normalized,
                           cudaStream_t s);
void launch_camera_jobs(const RenderParams& rp, long long P, QueueView out, cudaStream_t s);
void launch_frame_consts(FrameConsts* fc, uint32_t key0, uint32_t key1, int ref_count,
                         cudaStream_t s);

// RRSNet forward over n feature rows (n_ptr: device count, else n_host); with `sentinel`
// only rows whose q is negative are evaluated; st / status are nullable.
// rrsnet_simt.cu: FP32 on the CUDA cores, `rows` (1 or 2) rows per thread.
void launch_rrsnet_simt(int rows, int grid, const float* params, const float4* feat,
                        const long long* n_ptr, long long n_host, float* q, int sentinel,
                        DevStats* st, cudaStream_t s);
// NRRS inputs (Sec. 4 "Input Encoding") of the rows the shade kernel marked for the
// network, from StatNet and the vertex state, written to `out` ([C][4] float4).
void launch_nrrs_inputs(const float* stat, const SceneView& sc, const WorkView& w, QueueView cur,
                        const RenderParams& rp, int depth, int grid, float4* out, cudaStream_t s);
// AID-NRRS factors (RRSNet on its hash grid and encoded inputs, FP32) of the marked rows.
void launch_aid_rrsnet(const float* params, const float2* rgrid, const SceneView& sc,
                       const WorkView& w, QueueView cur, const RenderParams& rp, int depth,
                       int grid, cudaStream_t s);
// ADRRS (NN) factors of the vertices the shade kernel marked (rrsnet_simt.cu).
void launch_adrrs(const float* stat, const SceneView& sc, const WorkView& w, QueueView cur,
                  const RenderParams& rp, int depth, int grid, cudaStream_t s);
// rrsnet_tc.cu: tensor cores; precision 16 = split BF16 operands, 17 = BF16 operands, 8 =
// E4M3 operands with per-tensor scales; FP32 accumulation.  Variant 0: one tile in flight
// per CTA; variant 1 (precisions 16 and 17): two tiles per CTA, the same factors.
void launch_rrsnet_tc(int precision, int variant, int grid, const float* params,
                      const float4* feat, const long long* n_ptr, long long n_host, float* q,
                      int sentinel, DevStats* st, unsigned int* status, cudaStream_t s);
// Resident CTAs per SM of the two-tile kernel at precision 16 or 17 (at least 1).
int rrsnet_tc2_max_blocks(int precision);

// Launch shape of the RRSNet kernel for one queue size: the autotuner's unit (tune.cu).
struct RrsnetChoice {
    int variant;        // FP32: rows per thread (1 or 2); tensor cores: tiles per CTA - 1
    int blocks_per_sm;  // grid = SMs x blocks_per_sm (extra blocks exit at once)
};
constexpr int kTuneBuckets = 17;  // bucket b: floor(log2 n) = b + 8, clamped to [0, 16]
int tune_bucket(long long n);
RrsnetChoice default_choice(int precision);
void launch_rrsnet(int precision, RrsnetChoice c, int n_sm, const float* params,
                   const float4* feat, const long long* n_ptr, long long n_host, float* q,
                   int sentinel, DevStats* st, unsigned int* status, cudaStream_t s);
cudaError_t tune_rrsnet(int precision, int n_sm, const float* params, long long max_rows,
                        cudaStream_t s, RrsnetChoice* table, long long* rows, float* ms_best,
                        float* ms_default);

// Stand-alone entry points on plain arrays.
void launch_normalize_array(const float* q, long long n, double budget, double f_rate,
                            double alpha, double* part, int grid, float* F, double* sum,
                            cudaStream_t s);
struct SplitArrays {
    const float* q;
    long long n;
    const float* F;
    const uint32_t* pixel;
    const uint32_t* sample;
    const uint32_t* lineage;
    uint32_t depth, key0, key1;
    long long cap;
    uint32_t* X;
    long long* prefix;
    uint32_t* child_parent;
    uint32_t* child_lineage;
    long long* total;
    long long* dropped;
};
void launch_split_arrays(const SplitArrays& a, unsigned long long* bcnt, unsigned long long* boff,
                         int grid, cudaStream_t s);

}  // namespace nrrs
