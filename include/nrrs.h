/*
 * nrrs.h -- C ABI of the B300 (sm_103a) implementation of one bounce of wavefront
 * path tracing with normalized Russian roulette and splitting (RRS) and RRSNet,
 * after "NRRS: Neural Russian Roulette and Splitting" (arXiv 2510.07868).
 *
 * Conventions for every entry point:
 *   - Every call returns an nrrs_status; nothing throws across the ABI.
 *     nrrs_last_error() returns a short text for the calling thread's last failure.
 *   - Pointers named d_* are DEVICE pointers owned by the caller (for example torch
 *     tensors); they must be contiguous, of the stated element type, and stay valid
 *     until the enqueued work finishes.  Pointers without the prefix are HOST pointers
 *     owned by the caller and are only read (or written) during the call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device work is
 *     enqueued on it; a call returns before the work completes unless stated.
 *   - Device-side failures (queue overflow drops, non-finite factors, timeouts) are
 *     reported through status bits in the stats structs; kernels never trap.
 *   - A scene and the buffers it owns belong to the device passed to
 *     nrrs_create_scene; calls on a scene make that device current.
 */
#ifndef NRRS_H
#define NRRS_H

#include <stdint.h>

#if defined(__GNUC__)
#define NRRS_API __attribute__((visibility("default")))
#else
#define NRRS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nrrs_status {
    NRRS_OK = 0,
    NRRS_ERR_INVALID_ARG = 1,      /* a pointer, size or enum is out of range */
    NRRS_ERR_CUDA = 2,             /* a CUDA runtime call failed (see nrrs_last_error) */
    NRRS_ERR_OOM = 3,              /* device allocation failed */
    NRRS_ERR_TIMEOUT = 4,          /* a bounded device wait gave up */
    NRRS_ERR_NONFINITE = 5,        /* RRSNet produced NaN/Inf factors (paths terminated) */
    NRRS_ERR_OVERFLOW_DROPPED = 6, /* children beyond the queue capacity were dropped */
    NRRS_ERR_UNSUPPORTED = 7       /* valid request this build does not implement */
} nrrs_status;

/* Device status bits reported in nrrs_render_stats.status_bits. */
#define NRRS_STATUS_OVERFLOW_DROPPED 0x1u
#define NRRS_STATUS_NONFINITE 0x2u
#define NRRS_STATUS_TIMEOUT 0x4u
#define NRRS_STATUS_HEUR_FALLBACK 0x8u /* NET depths used the heuristic this frame (the
                                          last training step fell back)               */

/* How the RRS factor q of a path vertex is chosen (Sec. 2 "Unified RRS Framework",
 * Sec. 3.1 normalization, Sec. 3.3 Mix-Depth). */
typedef enum nrrs_rrs_mode {
    NRRS_RRS_NONE = 0,      /* q = 1 and no normalization: the plain path tracer */
    NRRS_RRS_PLAIN_RR = 1,  /* q = min(1, lum(t)): throughput roulette, no normalization */
    NRRS_RRS_HEUR_NORM = 2, /* q = min(lum(t) / max(I_px, eps_I), q_max), normalized */
    NRRS_RRS_NET = 3,       /* q = RRSNet(features), normalized */
    NRRS_RRS_NET_MIX = 4    /* per-depth choice among NET / HEUR / FIXED, normalized */
} nrrs_rrs_mode;

/* Mix-Depth methods, 2 bits per depth in nrrs_render_opts.gate (depth d uses bits
 * 2(d-1)..2(d-1)+1).  FIXED is fixed RR = 1 (q = 1). */
#define NRRS_GATE_NET 0u
#define NRRS_GATE_HEUR 1u
#define NRRS_GATE_FIXED 2u
#define NRRS_GATE_ADRRS 3u /* ADRRS (NN), Sec. 4 "Mix-Depth": r = lum(t) max(E[L_o], 0) /
                              max(I_px, eps_I) with E[L_o] the mean over RGB of StatNet's
                              predicted radiance (throughput inputs zeroed, as it is
                              trained); q = 1 inside the weight window [1/3, 5/3], else r,
                              clamped to [0.05, q_max]; the throughput heuristic before
                              any reference exists */

#define NRRS_MAX_DEPTH 32
#define NRRS_N_FEATURES 16
#define NRRS_HIDDEN 32
#define NRRS_RRSNET_PARAMS 2592 /* 32x16 + 32x32 + 32x32 + 1x32, no biases */
#define NRRS_STATNET_PARAMS 2752 /* 32x16 + 32x32 + 32x32 + 6x32, no biases */
#define NRRS_STATNET_GRID_PARAMS 3264 /* StatNet on the encodings: 32x32 + 32x32 + 32x32 + 6x32 */
#define NRRS_GRID_PARAMS 4194304 /* hash grid: 8 levels x 2^18 entries x 2 features */

/* Networks for nrrs_set_params / nrrs_get_params. */
#define NRRS_NET_RRSNET 0       /* RRSNet weights renders use (the EMA of the trained ones) */
#define NRRS_NET_RRSNET_TRAIN 1 /* RRSNet weights Adam updates                             */
#define NRRS_NET_STATNET 2      /* StatNet: 16 -> 32 -> 32 -> 32 -> 6, no output activation
                                   (32 inputs with the encodings of nrrs_set_statnet_encoding:
                                   NRRS_STATNET_GRID_PARAMS weights)                       */
#define NRRS_NET_STATNET_GRID 3 /* StatNet's hash grid, [8][2^18][2] (NRRS_GRID_PARAMS)   */
#define NRRS_NET_RRSNET_GRID 4  /* AID-NRRS: RRSNet's hash grid renders use (EMA)          */
#define NRRS_NET_RRSNET_GRID_TRAIN 5 /* AID-NRRS: RRSNet's hash grid Adam updates         */
#define NRRS_AID_RRSNET_PARAMS 3104 /* RRSNet on the AID-NRRS inputs: 32x32 + 32x32x2 + 32 */

/* Material record, 40 bytes.  type 0 = Lambertian (albedo), 1 = GGX + Lambert
 * "plastic" mixture (roughness is the GGX alpha, F0 the Schlick reflectance at normal
 * incidence).  Emission Le leaves the front face (the side of e1 x e2 with
 * e1 = v1 - v0, e2 = v2 - v0) or both faces when two_sided != 0.  Scattering is
 * always two-sided.  A material whose albedo is 0 in every channel ends the path. */
typedef struct nrrs_material {
    int32_t type;
    float albedo[3];
    float Le[3];
    float roughness;
    float F0;
    int32_t two_sided;
} nrrs_material;

/* Pinhole camera, 40 bytes.  right = normalize(up x look), up' = look x right; pixel
 * (x, y) with y = 0 at the top maps to look + sx right + sy up' with
 * sx = (2 (x + jx) / W - 1) tan(vfov/2) W/H and sy = (1 - 2 (y + jy) / H) tan(vfov/2). */
typedef struct nrrs_camera {
    float pos[3];
    float look[3];
    float up[3];
    float vfov_deg;
} nrrs_camera;

typedef struct nrrs_scene nrrs_scene; /* opaque; owns every device buffer it allocates */

/* Options of one render (NULL = all defaults, shown in brackets). */
typedef struct nrrs_render_opts {
    uint32_t seed_lo, seed_hi;  /* Philox key = (seed_lo, seed_hi ^ frame)         [1, 0] */
    uint32_t frame;             /* frame index                                      [0]    */
    int32_t cap_factor;         /* queue capacity C = cap_factor * W * H * spp (children
                                   beyond it are dropped and counted)               [2]    */
    float f_rate;               /* rate-control factor, Eq. q_norm_rate             [0.85] */
    float alpha0;               /* initial adaptive alpha, Eq. f_rate_prime         [1]    */
    float q_max;                /* HEUR cap                                         [16]   */
    float eps_rel;              /* HEUR: eps_I = eps_rel * mean(I_ref)              [0.01] */
    float boxcox_lambda;        /* throughput feature encoding                      [0.5]  */
    int32_t precision;          /* RRSNet arithmetic: 32 (FP32 SIMT), 16 (split BF16
                                   operands), 17 (BF16 operands rounded once) or 8
                                   (E4M3 operands), tensor cores with FP32
                                   accumulation; at 16 and 17 the NET depths shade
                                   and evaluate RRSNet in one kernel unless
                                   nrrs_set_shade_fusion(scene, 0)              [32]   */
    uint64_t gate;              /* NET_MIX method per depth (NRRS_GATE_*)           [0]    */
    const float* d_pixel_ref;   /* device [H*W*3] reference I_px for HEUR, or NULL to use
                                   the scene's running mean of earlier frames       [NULL] */
    int32_t update_ref;         /* fold this frame into the scene's running mean    [1]    */
    int32_t reset_ref;          /* forget the running mean before this frame        [0]    */
    uint32_t* d_trace;          /* device [max_depth][C][5] u32 or NULL: per depth and
                                   queue slot (pixel, sample, lineage, triangle or
                                   0xFFFFFFFF, X); for tests                        [NULL] */
    int32_t profile;            /* record CUDA events around kernel launches on
                                   `stream`; per-stage times land in stats.  1 = every
                                   launch; otherwise bit (k + 1) times the launches of
                                   stage k only (4 = NRRS_STAGE_EXTEND)             [0]    */
    int32_t graph;              /* capture the frame's launches (the whole bounce loop)
                                   into a CUDA graph on a scene-owned stream and launch
                                   that graph on `stream`; the executable graph is kept
                                   per launch shape and updated in place with each
                                   call's arguments                                 [0]    */
    float* d_suffix;            /* device [max_depth][C][4] float or NULL: record the frame
                                   and write every vertex's suffix sum S (rgb, pixel bits):
                                   its own deposit plus its children's S, so S / t is the
                                   vertex's outgoing-radiance estimate               [NULL] */
    int32_t nee;                /* next-event estimation (the paper's experiments run with
                                   it on, Sec. 5): 1 = at every vertex that goes on, one
                                   point on an emitting triangle (chosen by area, uniform
                                   on it) and a shadow ray, combined with the emitters
                                   that BSDF sampling hits by the power heuristic
                                   (Veach 1997); a vertex's deposit is then its
                                   MIS-weighted emission plus its unoccluded next-event
                                   contribution.  0 = BSDF sampling only            [0]    */
    const uint8_t* d_trace_mask; /* device [H*W] or NULL: with d_trace, record only the
                                   queue slots of pixels whose byte is non-zero, as a
                                   compact list: d_trace is then device [trace_rows][6]
                                   u32 of (depth, pixel, sample, lineage, triangle or
                                   0xFFFFFFFF, X) in no fixed order, for sampled pixels
                                   of frames too large for a whole trace; for tests [NULL] */
    uint64_t* d_trace_count;    /* with d_trace_mask: device u64 the render adds the rows
                                   it recorded to (zero it first); rows beyond trace_rows
                                   are counted, not written                         [NULL] */
    int64_t trace_rows;         /* rows d_trace holds with d_trace_mask             [0]    */
    int32_t budget_factor;      /* N_px of Eq. F_norm, the paths each depth may expect
                                   before rate control: budget_factor * W * H * spp.  0 or
                                   1 = the primary queue's size (Sec. 3.1: "the
                                   preallocated size of the primary workqueue"); the
                                   queue's capacity C (cap_factor) is enforced on integers
                                   on top and must hold it (budget_factor <= cap_factor) [0] */
} nrrs_render_opts;

/* Stages of one render, indexing nrrs_render_stats.stage_ms / stage_launches. */
#define NRRS_STAGE_INIT 0      /* reference mean + camera rays                      */
#define NRRS_STAGE_EXTEND 1    /* BVH traversal: closest hit per live ray           */
#define NRRS_STAGE_NORMALIZE 2 /* FP64 sum of q, F                                  */
#define NRRS_STAGE_COUNT 3     /* split counts per block + per-pixel accumulation   */
#define NRRS_STAGE_SCAN 4      /* block offsets, next queue length, alpha           */
#define NRRS_STAGE_SCATTER 5   /* children + BSDF sampling into the next queue      */
#define NRRS_STAGE_FINALIZE 6  /* frame estimate + running reference                */
#define NRRS_STAGE_RRSNET 7    /* RRSNet (FP32) on the NET depths' features         */
#define NRRS_STAGE_SHADE 8     /* emission deposit, RRS factor or features, sum q   */
#define NRRS_STAGE_REVERSE 9   /* record mode: suffix sums, deepest depth first     */
#define NRRS_STAGE_SHADOW 10   /* next-event estimation: any-hit shadow rays        */
#define NRRS_N_STAGES 11

/* Per-render statistics; filled only when a non-NULL pointer is passed (the call then
 * synchronizes `stream`).  Index d-1 holds depth d (1-based, camera hit = depth 1). */
typedef struct nrrs_render_stats {
    int64_t live[NRRS_MAX_DEPTH];      /* queue length traced at depth d                */
    double sum_q[NRRS_MAX_DEPTH];      /* FP64 sum of q_orig over the queue             */
    float F[NRRS_MAX_DEPTH];           /* applied factor min(1, f alpha C / sum_q)      */
    double alpha[NRRS_MAX_DEPTH];      /* adaptive alpha used at depth d                */
    int64_t requested[NRRS_MAX_DEPTH]; /* children requested (sum of X)                 */
    int64_t dropped[NRRS_MAX_DEPTH];   /* children beyond the capacity                  */
    int64_t segments;                  /* sum of live: rays traced                      */
    int64_t nonfinite;                 /* vertices whose factor was NaN/Inf/negative    */
    int64_t net_evals;                 /* RRSNet evaluations                            */
    int64_t capacity;                  /* C                                             */
    uint32_t status_bits;              /* NRRS_STATUS_* seen during the render          */
    uint32_t kernel_launches;          /* kernels this render launched                  */
    float stage_ms[12];                /* opts->profile: summed event time per stage    */
    int32_t stage_launches[12];        /* opts->profile: launches per stage             */
} nrrs_render_stats;

NRRS_API const char* nrrs_status_string(nrrs_status s);
NRRS_API const char* nrrs_last_error(void);

/* Build a scene on `device`: copies the triangles ([n_tri][9] float, v0 v1 v2),
 * per-triangle material ids ([n_tri] int32 in [0, n_mat)), materials and camera to the
 * device and builds a binned-SAH BVH2 on the host.  RRSNet weights start at zero
 * (q = ln 2 everywhere) until nrrs_set_rrsnet_params.  *out receives the scene.
 * Errors: INVALID_ARG on NULL pointers, n_tri < 1, n_mat < 1 or a bad material id;
 * OOM / CUDA on device failures (nothing is leaked). */
NRRS_API nrrs_status nrrs_create_scene(const float* tri, int32_t n_tri, const int32_t* tri_mat,
                              const nrrs_material* mats, int32_t n_mat, const nrrs_camera* cam,
                              int32_t device, nrrs_scene** out);

/* ---------------------------------------------------------------- batched renders
 * Many independent render jobs, each with its own scene, camera, image size, spp and
 * depth, traced together: every kernel of a bounce processes all jobs' paths at once and
 * all jobs share one RRSNet (the batch's weights, nrrs_set_rrsnet_params).  Eq. F_norm is
 * applied per job (the sum of q and the budget C_j = cap_factor * W_j * H_j * spp_j of
 * each job); the queue capacity sum_j C_j is enforced on the shared queue.  A job's
 * paths draw the random numbers a render of that job alone would draw (Philox counters
 * use the job-local pixel), so a job's image equals its own nrrs_render output up to
 * last-bit differences of the per-job FP64 sum of q.  No counterpart in the paper, which
 * renders one scene at a time. */
#define NRRS_MAX_JOBS 256
typedef struct nrrs_job {
    const float* tri;            /* host [n_tri][9], as nrrs_create_scene               */
    int32_t n_tri;
    const int32_t* tri_mat;      /* host [n_tri]                                        */
    const nrrs_material* mats;   /* host [n_mat]                                        */
    int32_t n_mat;
    const nrrs_camera* cam;      /* host                                                */
    int32_t width, height, spp, max_depth;
} nrrs_job;

/* Builds a batch scene: one BVH per job, merged into shared arrays with one root per
 * job.  Jobs are laid out in order: job j's pixels start at pixel_base_j = sum of the
 * earlier jobs' W * H (see nrrs_batch_info).  The result is an nrrs_scene: weights,
 * tuning and destruction use the scene entry points; nrrs_render, nrrs_train_step and
 * nrrs_mixdepth_search refuse it.  Errors: INVALID_ARG (NULL or empty job, bad sizes,
 * more than NRRS_MAX_JOBS jobs, 2^31 or more pixels or paths); OOM; CUDA. */
NRRS_API nrrs_status nrrs_create_batch(const nrrs_job* jobs, int32_t n_jobs, int32_t device,
                                       nrrs_scene** out);

/* One frame of every job (Sec. 3.1 per job, as nrrs_render).  d_rgb: device float
 * [sum_j H_j W_j][3], job j's image at pixel_base_j.  stats (nullable): totals over the
 * batch (F is 0: factors are per job).  job_live, job_F, job_sum_q (nullable, host,
 * [n_jobs][NRRS_MAX_DEPTH]): per job and depth the queue length, the factor F_j and the
 * sum of q.  Options as nrrs_render except d_trace and d_suffix (UNSUPPORTED).
 * Errors: INVALID_ARG (not a batch, bad options); UNSUPPORTED; OOM; CUDA. */
NRRS_API nrrs_status nrrs_render_batch(nrrs_scene* batch, int32_t rrs_mode,
                                       const nrrs_render_opts* opts, float* d_rgb, void* stream,
                                       nrrs_render_stats* stats, int64_t* job_live, float* job_F,
                                       double* job_sum_q);

/* Number of jobs (0 for a single scene), each job's first pixel ([n_jobs], nullable) and
 * the total pixel count (nullable). */
NRRS_API nrrs_status nrrs_batch_info(const nrrs_scene* scene, int32_t* n_jobs,
                                     int64_t* pixel_base, int64_t* n_pixels_total);

/* Chooses the traversal tree of later renders (the paper traces with OptiX, Sec. 4
 * "System"; these are its stand-ins): 2 = the host-built BVH2 (default), 4 = a four-wide
 * tree collapsed from it (available when its worst-case traversal stack fits the
 * kernel's 40 entries), 8 = a compressed eight-wide tree built on the device on first
 * use (Morton order, PLOC clustering, collapse to eight children with leaves of up to
 * 2 triangles, child boxes quantised to one byte per plane against a per-node origin
 * and power-of-two scales, 80 bytes per node; Ylitie, Karras & Laine 2017), traversed
 * nearest child first with the remaining children as node groups on the stack in the
 * ray's octant order.  Every tree gives the same closest hits; on the measured scenes
 * the BVH2 with FP16 boxes traverses fastest.  The first call with 8 builds (device memory about 200 bytes per
 * triangle while it runs, 80 bytes per node and 48 per triangle after) and synchronizes
 * the device.  Errors: INVALID_ARG (NULL scene, width not 2, 4 or 8); UNSUPPORTED (4
 * without a four-wide tree; 8 on a batch, or a tree deeper than the 40-entry stack);
 * CUDA, OOM. */
NRRS_API nrrs_status nrrs_set_traversal(nrrs_scene* scene, int32_t width);

/* The device-built eight-wide tree (nrrs_set_traversal(8)); all zero before it is built. */
typedef struct nrrs_bvh8_stats {
    int64_t nodes;       /* eight-wide nodes                                        */
    int64_t triangles;   /* triangles in its leaves (each once)                     */
    int32_t depth;       /* node levels                                             */
    int32_t iterations;  /* clustering rounds of the build                          */
    float build_ms;      /* wall time of the build, including its synchronization  */
} nrrs_bvh8_stats;
NRRS_API nrrs_status nrrs_bvh8_info(const nrrs_scene* scene, nrrs_bvh8_stats* out);

/* Host copies of the eight-wide tree, for tests: nodes [nodes][20] u32 (five 16-byte rows
 * per node: origin xyz as FP32 bits and exponents | inner mask << 24; first inner
 * child, first triangle, leaf meta bytes; then the lower x, y, z and upper x, y, z bytes
 * of the eight child boxes), tris [triangles][12] float (v0, original id bits; e1,
 * material id bits; e2, 0).  Errors: INVALID_ARG (NULL, buffers too small); UNSUPPORTED
 * (not built); CUDA. */
NRRS_API nrrs_status nrrs_bvh8_export(const nrrs_scene* scene, uint32_t* nodes,
                                      int64_t max_nodes, float* tris, int64_t max_tris);

/* Chooses the box precision of the BVH2 that later renders traverse: 16 = a copy of
 * the tree with every child box rounded outward to IEEE binary16 (32-byte nodes, one
 * memory sector per visit), 32 = the FP32 boxes (64-byte nodes).  The rounded boxes
 * contain the FP32 ones, so both give the same closest hits (a few more boxes pass the
 * slab test).  The default is 16 unless the rounding grows the child boxes' summed
 * surface area (the expected box visits) by more than 10 % (a scene far from the origin,
 * where binary16 is coarse), then 32.  The four-wide tree of nrrs_set_traversal(4) keeps FP32 boxes.  Errors: INVALID_ARG (NULL scene, bits not 16 or 32); UNSUPPORTED (16 when
 * the scene has no FP16 copy: a leaf with more than 31 references, or 2^26 or more
 * references). */
NRRS_API nrrs_status nrrs_set_bvh_precision(nrrs_scene* scene, int32_t bits);

/* The BVH2 traversal's stack (no counterpart in the paper; its renderer traces with
 * OptiX).  A ray holds at most one pushed sibling per inner node on its current path, so
 * a tree whose root-to-leaf paths hold at most 24 inner nodes (the height) is traversed
 * with a 24-entry stack, otherwise with the 40-entry one the build's depth cap fits;
 * the short stack leaves 16 KB more of each SM's on-chip memory to the L1 cache that
 * holds the nodes.  entries = 0 (the default) chooses by the height, 40 always takes the
 * long stack, 24 the short one.  Both find the same closest hits.  The choice follows
 * later tree rebuilds (nrrs_set_bvh_builder); the eight- and four-wide trees keep their
 * own stacks.  Errors: INVALID_ARG (NULL scene, entries not 0, 24 or 40); UNSUPPORTED
 * (24 for a taller tree, or one whose height is unknown). */
NRRS_API nrrs_status nrrs_set_traversal_stack(nrrs_scene* scene, int32_t entries);

/* The BVH2's height (-1 when its node order does not allow computing it) and the stack
 * entries per ray the BVH2 traversal uses now.  Either pointer may be NULL.
 * Errors: INVALID_ARG (NULL scene). */
NRRS_API nrrs_status nrrs_traversal_stack_info(const nrrs_scene* scene, int32_t* height,
                                               int32_t* entries);

/* Chooses how later renders evaluate RRSNet at their NET depths on the tensor cores
 * (precisions 16 and 17, the 16 vertex features of Sec. 4 "Network Architecture"):
 * on = 1 (the default) shades the depth's vertices and runs the network in one kernel,
 * the features going from registers into shared memory as the first layer's operand;
 * on = 0 writes them to device memory (64 bytes per vertex) for a separate RRSNet kernel.
 * Both give the same factors, deposits and images, bit for bit.  Training frames (which
 * record the features) and the NRRS / AID inputs always take the separate kernels.
 * Errors: INVALID_ARG (NULL scene, on not 0 or 1). */
NRRS_API nrrs_status nrrs_set_shade_fusion(nrrs_scene* scene, int32_t on);

/* Rebuilds the scene's BVH2 (and its FP16 copy and four-wide collapse) with another
 * builder: 0 = the host binned-SAH builder of nrrs_create_scene (the default), 1 = the
 * device build of the eight-wide tree stopped before its collapse (Morton order, then
 * PLOC clustering; one triangle per leaf, depth-first node order).  Both trees hold every
 * triangle with the same vertices and the traversal returns the closest hit with the
 * lower-id tie rule, so renders do not depend on the builder; only the traversal cost
 * does.  The FP16 choice is redone for the new tree (rule of nrrs_set_bvh_precision).
 * build_ms (may be NULL) gets the build's wall time.  Synchronizes the device and drops
 * the scene's captured graphs.  Errors: INVALID_ARG (NULL scene, builder not 0 or 1);
 * UNSUPPORTED (a batch scene, fewer than two triangles, a device tree deeper than the
 * traversal stack); CUDA / OOM (the old tree is kept). */
NRRS_API nrrs_status nrrs_set_bvh_builder(nrrs_scene* scene, int32_t builder, float* build_ms);

/* Chooses what RRSNet reads at the network depths of later renders and training steps
 * (the weights are the caller's to match; a change between modes 0/1 and 2 changes the
 * network's shape and starts RRSNet afresh):
 *   0 (default) the 16 vertex features: position in the scene box, -w_o, the shading
 *     normal, albedo, d / D and Box-Cox(t) per channel;
 *   1 the NRRS inputs of Sec. 4 "Input Encoding": StatNet runs first at every network
 *     vertex (its throughput inputs zeroed, as trained) and RRSNet reads
 *     Box-Cox(max(E[L_o], 0)) and Box-Cox(max(E[L_o^2], 0)) per channel, Box-Cox(t) per
 *     channel, Box-Cox(mean of the pixel estimate; 0 before any), 1 - exp(-roughness)
 *     (Lambertian surfaces count as roughness 1) and five zeros, Box-Cox with the render's
 *     boxcox_lambda.  StatNet's weights are the scene's (nrrs_set_params / training);
 *   2 the AID-NRRS inputs of Sec. 4 "Input Encoding": RRSNet (32 -> 32 -> 32 -> 32 -> 1,
 *     NRRS_AID_RRSNET_PARAMS weights, FP32 only) reads its own trainable hash grid of the
 *     position (as nrrs_set_statnet_encoding describes; NRRS_NET_RRSNET_GRID for renders,
 *     the EMA of NRRS_NET_RRSNET_GRID_TRAIN), one-blob (4 bins) of w_o's spherical
 *     coordinates, Box-Cox(t) per channel, Box-Cox(max(mean I_px, 0)) and one-blob (4
 *     bins) of 1 - exp(-roughness); nrrs_query_factors refuses this mode.
 * Errors: INVALID_ARG (NULL scene, mode not 0, 1 or 2); OOM; CUDA. */
NRRS_API nrrs_status nrrs_set_rrsnet_inputs(nrrs_scene* scene, int32_t mode);

/* Chooses StatNet's inputs (everywhere StatNet runs: training, ADRRS (NN), NRRS inputs):
 *   0 (default) the 13 vertex features of RRSNet with the throughput inputs zeroed
 *     (16 -> 32 -> 32 -> 32 -> 6, NRRS_STATNET_PARAMS weights);
 *   1 the encodings of Sec. 4 "Input Encoding": a trainable multiresolution hash grid of
 *     the position in the scene box (8 levels x 2 features, resolution 16 doubling per
 *     level, 2^18 entries per level; dense indexing while (N+1)^3 fits, else the spatial
 *     hash x*1 ^ y*2654435761 ^ z*805459861 mod 2^18; trilinear interpolation), one-blob
 *     encodings (4 bins) of w_o's spherical coordinates (theta / pi from the z axis,
 *     (phi + pi) / (2 pi)) and one-blob (8 bins) of 1 - exp(-roughness), 32 inputs
 *     (NRRS_STATNET_GRID_PARAMS weights + NRRS_GRID_PARAMS grid entries, trained by the
 *     same Adam steps; the grid with epsilon 1e-15).
 * A change starts StatNet afresh (default weights, grid entries uniform in +-1e-4).
 * Errors: INVALID_ARG (NULL scene, mode not 0 or 1); OOM; CUDA. */
NRRS_API nrrs_status nrrs_set_statnet_encoding(nrrs_scene* scene, int32_t mode);

/* Free every device buffer of the scene (synchronizes the device). NULL is a no-op. */
NRRS_API nrrs_status nrrs_destroy_scene(nrrs_scene* scene);

/* Host copies of the BVH for inspection: node count and triangle count after build. */
NRRS_API nrrs_status nrrs_scene_info(const nrrs_scene* scene, int64_t* n_nodes, int64_t* n_tri);

/* Replace / read the RRSNet weights (host, NRRS_RRSNET_PARAMS floats, packed
 * W1[32][16] | W2[32][32] | W3[32][32] | W4[1][32], row-major).  Sec. 4 "Network
 * Architecture": three hidden layers of 32 with Leaky ReLU (slope 0.01), output
 * activation of Eq. rrsnet_activation.  set is stream-ordered on `stream`. */
NRRS_API nrrs_status nrrs_set_rrsnet_params(nrrs_scene* scene, const float* params, int32_t n,
                                   void* stream);
NRRS_API nrrs_status nrrs_get_rrsnet_params(nrrs_scene* scene, float* params, int32_t n, void* stream);

/* One frame: W x H pixels, spp samples, camera hit = depth 1 ... max_depth, with the RRS
 * factors of `rrs_mode` (Sec. 3.1: every depth is normalized for HEUR/NET/NET_MIX,
 * downscale only, Sec. 4 "Compromise").  Writes the frame estimate, the mean over spp
 * of the deposited radiance, to d_rgb (device [H][W][3] float).
 * Limits: 1 <= max_depth <= NRRS_MAX_DEPTH, W*H*spp*cap_factor < 2^31.
 * A network factor that comes out non-finite takes the throughput heuristic's factor
 * (the method degrades to plain heuristic normalised RRS for that vertex), and after a
 * training step that fell back the next frame uses the heuristic at every network depth
 * (NRRS_STATUS_HEUR_FALLBACK).
 * Errors: INVALID_ARG (bad sizes, mode, NULL d_rgb); OOM; CUDA.  Overflow drops and
 * non-finite factors are not errors: they are counted in stats (status_bits). */
NRRS_API nrrs_status nrrs_render(nrrs_scene* scene, int32_t width, int32_t height, int32_t spp,
                        int32_t max_depth, int32_t rrs_mode, const nrrs_render_opts* opts,
                        float* d_rgb, void* stream, nrrs_render_stats* stats);

/* RRSNet inference on n feature rows (device [n][16] float, 16-byte aligned) -> device
 * d_q [n] float.
 * precision 32 = FP32 SIMT; 16 = tensor cores (tcgen05.mma kind::f16) with every MMA
 * operand split into two BF16 numbers (hi + lo, three MMAs per product) and FP32
 * accumulation; 17 = the same tensor cores with every operand rounded once to BF16
 * (one MMA per product); 8 = tensor cores (kind::f8f6f4) with E4M3 operands, one scale
 * per weight matrix and per 128-row activation tile, a power of two putting its largest
 * magnitude in (224, 448], FP32 accumulation.  The 32 -> 1 output layer and the
 * activation run in FP32 in all of them.
 * Feature layout (16 raw features in place of the paper's
 * encoded inputs of Sec. 4 "Input Encoding"): position normalised to the scene box (3),
 * outgoing direction (3), shading normal (3), albedo (3), depth / max_depth (1),
 * Box-Cox(t) with lambda = boxcox_lambda per throughput channel (3).
 * Errors: INVALID_ARG (n < 0, NULL with n > 0); UNSUPPORTED (unknown precision). */
NRRS_API nrrs_status nrrs_query_factors(nrrs_scene* scene, const float* d_features, int64_t n,
                               int32_t precision, float* d_q, void* stream);

/* Normalization of one queue (Eq. q_norm, Eq. F_norm, Eq. q_norm_rate, downscale only):
 * sum = FP64 sum of d_q[0..n), F = min(1, f_rate * alpha * budget / sum) (1 if
 * sum == 0) rounded to FP32.  Writes d_F[0] (float) and d_sum[0] (double).
 * `scene` only selects the device (NULL = the current device).  Scratch: per-block
 * partial sums in a per-device pool the library allocates once; calls that overlap on
 * the GPU (different streams) share it and race, so keep them on one stream. */
NRRS_API nrrs_status nrrs_normalize(nrrs_scene* scene, const float* d_q, int64_t n, double budget,
                           double f_rate, double alpha, float* d_F, double* d_sum,
                           void* stream);

/* Split counts and compaction of one queue (Eq. rrs_factor), the integer core of the
 * bounce.  For parent i: q_used = fp32(F * q_orig_i), k = floor(q_used),
 * r = q_used - k, U = (Philox4x32-10(key, ctr).x >> 8) * 2^-24 with
 * key = (seed_lo, seed_hi ^ frame), ctr = (pixel_i, sample_i, depth << 8 | 3, lineage_i),
 * X_i = k + [U < r].  Children of i take slots [prefix_i, prefix_i + X_i) in parent
 * order; child j gets lineage (ctr-output.y + j * 0x9E3779B9) mod 2^32.  Slots >= cap
 * are not written (dropped).  Outputs (device): d_X[n] u32, d_prefix[n] i64 exclusive
 * prefix of X, d_child_parent[cap] u32, d_child_lineage[cap] u32, d_total[0] i64 = sum X,
 * d_dropped[0] i64.  d_F is a device float.  Requires n < 2^31, cap < 2^31; X is
 * clamped at 2^23 (q_used >= 2^23 has no fractional part in FP32).
 * `scene` only selects the device (NULL = the current device).  Scratch: per-block
 * child counts and offsets in the same per-device pool as nrrs_normalize (same race
 * rule: overlapping calls on different streams race). */
NRRS_API nrrs_status nrrs_split(nrrs_scene* scene, const float* d_q_orig, int64_t n, const float* d_F,
                       const uint32_t* d_pixel, const uint32_t* d_sample,
                       const uint32_t* d_lineage, uint32_t depth, uint32_t seed_lo,
                       uint32_t seed_hi, uint32_t frame, int64_t cap, uint32_t* d_X,
                       int64_t* d_prefix, uint32_t* d_child_parent, uint32_t* d_child_lineage,
                       int64_t* d_total, int64_t* d_dropped, void* stream);

/* nrrs_split without any device allocation.  The paper has no counterpart: this
 * exists for callers that cannot allocate device memory on the call path, such as an
 * engine that gave all device memory to its own arena at start-up, or a frame loop
 * that cannot afford the device-wide synchronization cudaMalloc / cudaFree may cause.
 * Same arguments, layouts, outputs and results as nrrs_split (without `scene`); it
 * runs on the current device.  Its per-block scratch (256 KiB: a 64-bit child count
 * and offset per block) is a fixed array compiled into the library, present on every
 * GPU that loads it until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called.
 * Limit: n <= 67,108,864 parents (4096 per block, 16384 blocks); larger n returns
 * NRRS_ERR_INVALID_ARG with a message in nrrs_last_error().
 * The first call on a device looks up the array's device address (once per device).
 * Under CUDA's lazy module loading (the default) that lookup is also what loads this
 * part of the library onto the device: the driver then places its code and the array
 * in device memory once, which allocates and may synchronize.  A caller that cannot
 * take that stall makes one call at start-up (n = 0 and cap = 0 suffice; d_F,
 * d_total and d_dropped must still be device pointers), on each device it will use,
 * before any stream capture; later calls allocate nothing.  Every call shares the one array,
 * so calls that overlap on the GPU (for example on two streams) race and corrupt each
 * other's results; keep them ordered on one stream. */
NRRS_API nrrs_status nrrs_split_noalloc(const float* d_q_orig, int64_t n, const float* d_F,
                                        const uint32_t* d_pixel, const uint32_t* d_sample,
                                        const uint32_t* d_lineage, uint32_t depth,
                                        uint32_t seed_lo, uint32_t seed_hi, uint32_t frame,
                                        int64_t cap, uint32_t* d_X, int64_t* d_prefix,
                                        uint32_t* d_child_parent, uint32_t* d_child_lineage,
                                        int64_t* d_total, int64_t* d_dropped, void* stream);

/* ------------------------------------------------------------------ training */

/* What one training step computed, for checking the step against a reference
 * implementation: host buffers, each nullable, that nrrs_train_step fills after both
 * networks' gradients are summed and before its Adam updates (filling them synchronizes
 * the stream).  Sizes: W*H for the per-pixel arrays; the weight counts of
 * nrrs_get_params for the gradients. */
typedef struct nrrs_train_debug {
    float* grad_statnet;   /* summed StatNet weight gradient the step applies (1/N mean) */
    float* grad_rrsnet;    /* summed RRSNet weight gradient (warm-up: 1/N mean; full loss:
                              the sum of Eq. loss-function_rrsnet's gradient)            */
    float* pixel_var;      /* V_i of the recorded frame (variance of the pixel estimate)  */
    float* pixel_error;    /* E_i after the temporal EMA and the spatial filter: the map
                              the loss uses                                              */
    int32_t* samples;      /* k_i, training samples per pixel                            */
    float ebar;            /* out: mean of pixel_error                                   */
    int64_t vertices;      /* out: vertices recorded in the frame                        */
    int64_t batch;         /* out: training slots drawn from them                        */
} nrrs_train_debug;

/* One online training step (Sec. 3.2 "Loss Design", Sec. 4 "Training").  Options (NULL =
 * defaults in brackets). */
typedef struct nrrs_train_opts {
    int32_t width, height, spp, max_depth; /* training frame          [256, 256, 2, 16] */
    uint32_t seed_lo, seed_hi, frame;      /* Philox key; frame = frame + step  [1, 0, 0] */
    int32_t warmup_steps;                  /* steps of step (1): RRSNet -> 1        [20] */
    float lr_rrsnet, lr_statnet;           /* Adam learning rates        [3e-4, 5e-3]   */
    float gamma1, gamma2, gamma3;          /* Eq. loss-function_rrsnet [.01, .05, .01] */
    float eps;                             /* Eq. loss-function_min / StatNet     [0.01] */
    float ema_decay;                       /* EMA of the RRSNet weights for rendering; step t
                                              uses min(ema_decay, (1+t)/(10+t))     [0.99] */
    float f_rate;                          /* rate control of the training frame  [0.85] */
    const float* d_pixel_ref;              /* device [H*W*3] reference I, or NULL for the
                                              scene's running mean of its frames   [NULL] */
    float alpha_mix;                       /* temporal EMA of the error map, Eq.
                                              error_temporal                        [0.5] */
    int32_t error_filter_radius;           /* (2r+1)^2 spatial filter on the error map in
                                              place of the paper's denoiser (Sec. 4
                                              "Tackle Low Spp"); 0 = off              [2] */
    int32_t graph;                         /* record the training frame through a CUDA
                                              graph (nrrs_render_opts.graph)          [0] */
    int32_t batch_size;                    /* training vertices per step, drawn from the
                                              recorded frame by systematic sampling
                                              with a per-step offset; 0 = 2^19
                                              (Sec. 4 "Training")                     [0] */
    int32_t nee;                           /* next-event estimation in the training frame
                                              (nrrs_render_opts.nee)                  [0] */
    float error_filter_power;              /* guidance by the first-hit normals, as the
                                              paper's denoiser takes the normal buffer:
                                              neighbours weigh max(0, n_p . n_q)^power
                                              (nrrs_error_filter); <= 0 = plain box   [8] */
    int32_t error_filter_until;            /* the spatial filter is off from this step on
                                              (the paper disables its denoiser for the last
                                              part of training, where it biases the
                                              error); 0 = never off                   [0] */
    nrrs_train_debug* debug;               /* host, nullable: filled as described at
                                              nrrs_train_debug                     [NULL] */
} nrrs_train_opts;

typedef struct nrrs_train_stats {
    int64_t step;         /* successful steps so far                                     */
    int64_t samples;      /* training samples: vertices where RRSNet was evaluated        */
    int64_t segments;     /* rays traced by the training frame                            */
    double loss_statnet;  /* mean relative L2 of StatNet (Eq. loss-function_StatNet)      */
    double loss_rrsnet;   /* phase 1: mean relative L2 to 1; phase 2: L_RRSNet            */
    double loss_avg;      /* L_avg = sum_i (E_i - mean E)^2                               */
    double loss_min;      /* L_min = sum_i E_i                                            */
    double loss_rrs;      /* L_rrs = sum_s (q_nrrs - q_norm)^2 (phase 2)                  */
    int32_t phase;        /* 1 = warm-up (step (1) of Sec. 4), 2 = full loss              */
    int32_t fallback;     /* 0 ok; 1 non-finite gradients or loss; 2 divergence (after 50
                             full-loss steps, a 0.98-EMA of the loss above 10x its running
                             minimum): the last good weights were restored and the step
                             was not counted                                              */
    int64_t kernel_launches; /* kernels the step launched (frame and training)            */
} nrrs_train_stats;

/* Renders one recorded frame with NET factors at every depth (the inference weights),
 * runs the reverse pass (suffix sums S; reflected radiance (S - deposit) / t per vertex),
 * computes pixel errors E_i = V_i / (I_i^2 + eps) from the spp samples of each pixel, then
 * trains StatNet on <L> and <L>^2 (relative L2) and RRSNet (phase 1: relative L2 to 1;
 * phase 2: g1 L_avg + g2 L_min + g3 L_rrs with dV/dq from Eq. gradient_transfer_rr_mc /
 * splitting_mc using the StatNet moments, shared 1/k_i per pixel), one Adam step each,
 * and updates the rendering weights to the EMA of the trained ones.  Synchronizes
 * `stream`.  Errors: INVALID_ARG (sizes as nrrs_render, bad options); OOM; CUDA. */
NRRS_API nrrs_status nrrs_train_step(nrrs_scene* scene, const nrrs_train_opts* opts, void* stream,
                                     nrrs_train_stats* stats);

/* Host copies in/out of a network's weights (n = NRRS_RRSNET_PARAMS or
 * NRRS_STATNET_PARAMS).  Setting StatNet also clears its Adam moments. */
NRRS_API nrrs_status nrrs_set_params(nrrs_scene* scene, int32_t which, const float* params,
                                     int32_t n, void* stream);
NRRS_API nrrs_status nrrs_get_params(nrrs_scene* scene, int32_t which, float* params, int32_t n,
                                     void* stream);

/* Backward pass of the bias-free MLP 16 -> 32 -> 32 -> 32 -> n_out (n_out 1 = RRSNet
 * before its output activation, 6 = StatNet): d_grad = sum over the n rows of
 * d(gout_s . out_s) / dW, with inputs d_x [n][16] (16-byte aligned), output gradients
 * d_gout [n][n_out], weights d_params (packed as nrrs_set_rrsnet_params).  Sums per
 * block of 128 rows, then over blocks in a fixed order (reproducible).  Scratch: the
 * scene's training buffers. */
NRRS_API nrrs_status nrrs_mlp_grad(nrrs_scene* scene, int32_t n_out, const float* d_params,
                                   const float* d_x, const float* d_gout, int64_t n, float* d_grad,
                                   void* stream);

/* nrrs_mlp_grad for StatNet on the encodings (32 -> 32 -> 32 -> 32 -> 6): d_x [n][32]
 * (16-byte aligned), d_gout [n][6], d_params NRRS_STATNET_GRID_PARAMS weights, d_grad the
 * same size.  Errors: INVALID_ARG; CUDA. */
NRRS_API nrrs_status nrrs_statnet_grad(nrrs_scene* scene, const float* d_params, const float* d_x,
                                       const float* d_gout, int64_t n, float* d_grad,
                                       void* stream);

/* StatNet's 32 encoded inputs (nrrs_set_statnet_encoding(1)) of n vertices: d_feat
 * [n][16] vertex features as the renders write them (position in the scene box in 0..2,
 * -w_o in 3..5; 16-byte aligned), d_rough [n] roughness (Lambertian 1), out d_x [n][32],
 * with the scene's hash grid.  Errors: INVALID_ARG; UNSUPPORTED (no grid); CUDA. */
NRRS_API nrrs_status nrrs_statnet_inputs(nrrs_scene* scene, const float* d_feat,
                                         const float* d_rough, int64_t n, float* d_x,
                                         void* stream);

/* Adds to d_grad (device, NRRS_GRID_PARAMS floats, the grid's layout) the gradient of
 * sum_i d_dx[i] . grid(p_i) for the positions p_i of d_feat [n][16] (16-byte aligned)
 * and grid-feature gradients d_dx [n][16]: the adjoint of the encoding, by atomic adds
 * (the order of the additions is not fixed).  Errors: INVALID_ARG; CUDA. */
NRRS_API nrrs_status nrrs_grid_backward(nrrs_scene* scene, const float* d_feat, const float* d_dx,
                                        int64_t n, float* d_grad, void* stream);

/* Autotuner of the RRSNet launch shape (no counterpart in the paper; it serves Sec. 4's
 * network in a queue whose size changes per bounce).  For every queue-size bucket b
 * (floor(log2 n) = b + 8, clamped to 0 .. NRRS_TUNE_BUCKETS - 1) it times each candidate
 * shape of the `precision` kernel (32: rows per thread 1 or 2 x blocks per SM; 16, 17:
 * one or two 128-row tiles in flight per CTA x CTAs per SM; 8: tensor-core CTAs per SM)
 * on 1.5 x 2^(b + 8) synthetic rows (at most 12,582,912) with
 * the scene's weights, and keeps the fastest for the scene.  Later renders pick the shape
 * of each depth from the bucket of that depth's queue size in the last frame rendered
 * with stats (W*H*spp before any), nrrs_query_factors from its n.  Every shape gives
 * identical results.  Allocates about 0.85 GB while it runs; synchronizes `stream`.
 * `report` (nullable, host) receives the table and the timings.
 * Errors: INVALID_ARG (NULL scene, unknown precision); OOM; CUDA. */
#define NRRS_TUNE_BUCKETS 17
typedef struct nrrs_tune_report {
    int32_t precision;
    int32_t n_buckets;                        /* NRRS_TUNE_BUCKETS                   */
    int64_t rows[NRRS_TUNE_BUCKETS];          /* rows timed per bucket               */
    int32_t variant[NRRS_TUNE_BUCKETS];       /* FP32: rows per thread; 16, 17: tiles
                                                 in flight per CTA - 1; 8: 0           */
    int32_t blocks_per_sm[NRRS_TUNE_BUCKETS]; /* grid = SMs x blocks_per_sm          */
    float ms_best[NRRS_TUNE_BUCKETS];         /* mean launch time, chosen shape      */
    float ms_default[NRRS_TUNE_BUCKETS];      /* mean launch time, untuned shape     */
} nrrs_tune_report;
NRRS_API nrrs_status nrrs_tune_rrsnet(nrrs_scene* scene, int32_t precision, void* stream,
                                      nrrs_tune_report* report);

/* Sets the RRSNet launch shape of one queue-size bucket (or of all, bucket = -1) by hand,
 * as nrrs_tune_rrsnet would: variant 1 or 2 rows per thread at precision 32, 0 (one tile
 * in flight per CTA) or 1 (two) at precisions 16 and 17, 0 at precision 8;
 * 1 <= blocks_per_sm <= 32 (the two-tile kernel runs at most as many CTAs per SM as stay
 * resident).  Results do not depend on it.
 * Errors: INVALID_ARG (NULL scene, unknown precision, bucket or shape out of range). */
NRRS_API nrrs_status nrrs_set_rrsnet_shape(nrrs_scene* scene, int32_t precision, int32_t bucket,
                                           int32_t variant, int32_t blocks_per_sm);

/* RRSNet forward with caller-supplied weights (Sec. 4 "Network Architecture", Eq.
 * rrsnet_activation): d_q[s] = softplus'(MLP(d_x[s])) in FP32 on the CUDA cores, d_params
 * device [2592] packed as nrrs_set_rrsnet_params, d_x device [n][16] (16-byte aligned).
 * Needs no scene.  Errors: INVALID_ARG (n < 0, NULL pointers, misaligned d_x). */
NRRS_API nrrs_status nrrs_rrsnet_forward(const float* d_params, const float* d_x, int64_t n,
                                         float* d_q, void* stream);

/* RRSNet backward through its output activation: d_grad [2592] = sum over the n rows of
 * gq_s d q_s / d W, q_s = softplus'(MLP(x_s)) as nrrs_rrsnet_forward, gq device [n].
 * Summation order as nrrs_mlp_grad (reproducible); scratch: the scene's training
 * buffers.  Errors: INVALID_ARG (n < 0, NULL pointers, misaligned d_x); OOM; CUDA. */
NRRS_API nrrs_status nrrs_rrsnet_backward(nrrs_scene* scene, const float* d_params,
                                          const float* d_x, const float* d_gq, int64_t n,
                                          float* d_grad, void* stream);

/* d L_RRSNet / d q_nrrs for n training samples (Sec. 3.2): with q_used = F q_nrrs,
 * dV/dq_used = -t^2 H / q_used^2, H = m2 if q_used < 1 (Eq. gradient_transfer_rr_mc) else
 * max(m2 - m1^2, 0) (Eq. gradient_transfer_splitting_mc);
 * dq = (g1 2 (E_i - Ebar) + g2) / (I_i^2 + eps) / k_i * dV/dq_used * F + g3 2 (q - Fn q).
 * Per-sample arrays [n]; per-pixel arrays d_E, d_Iref, d_k indexed by d_pixel. */
NRRS_API nrrs_status nrrs_rrsnet_dloss(const float* d_q_nrrs, const float* d_F, const float* d_Fn,
                                       const float* d_t, const int32_t* d_pixel, const float* d_m1,
                                       const float* d_m2, const float* d_E, double Ebar,
                                       const float* d_Iref, const int32_t* d_k, int64_t n,
                                       float eps, float g1, float g2, float g3, float* d_dq,
                                       void* stream);

/* One Adam step (Kingma & Ba, bias-corrected) on n weights, step >= 1.  Non-finite
 * gradients leave their weight and moments untouched. */
NRRS_API nrrs_status nrrs_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v,
                                    int32_t n, int32_t step, float lr, float b1, float b2,
                                    float eps, void* stream);

/* The exponential moving average of the weights that rendering uses (Sec. 4
 * "Training", as in NRC): d_avg[i] = decay d_avg[i] + (1 - decay) d_params[i] in FP32,
 * device arrays [n].  nrrs_train_step applies it with decay min(ema_decay,
 * (1 + t) / (10 + t)) at step t.  Errors: INVALID_ARG (n < 0, NULL with n > 0, decay
 * outside [0, 1]); CUDA. */
NRRS_API nrrs_status nrrs_ema(float* d_avg, const float* d_params, int32_t n, float decay,
                              void* stream);

/* ------------------------------------------------------------------ Mix-Depth */

/* Candidates Mix-Depth evaluates (Sec. 3.3): the depths are cut into segments of t_d
 * bounces and each segment is searched exhaustively over {NET, HEUR, FIXED}^len, so
 * sum over segments of 3^len (brute force 3^D when max_depth <= t_d).  -1 on bad input. */
NRRS_API int64_t nrrs_mixdepth_candidates(int32_t max_depth, int32_t t_d);

typedef struct nrrs_mixdepth_opts {
    int32_t width, height, spp, max_depth; /* the estimation renders (spp 1 in the paper) */
    int32_t t_d;                           /* segment length of the heuristic search (6)  */
    int32_t max_candidates;                /* refuse larger searches (0 = no limit)        */
    uint32_t seed_lo, seed_hi, frame;      /* one key for every candidate render           */
    const float* d_pixel_ref;              /* device [H*W*3] reference, or NULL for the
                                              scene's running mean of its frames            */
    int32_t adrrs;                         /* candidates per depth: 0 = FIXED, HEUR, NET;
                                              1 = FIXED, ADRRS (NN), NET (the paper's set) */
    int32_t nee;                           /* next-event estimation in the candidate renders
                                              (nrrs_render_opts.nee)                        */
    int32_t precision;                     /* RRSNet arithmetic of the candidate renders
                                              (nrrs_render_opts.precision); 0 = 32          */
} nrrs_mixdepth_opts;

typedef struct nrrs_mixdepth_result {
    uint64_t gate;     /* chosen method per depth (NRRS_GATE_*, 2 bits per depth)          */
    double score;      /* relMSE x segments of the chosen candidate (lower is better)      */
    double relmse;     /* relMSE of its estimation render against the reference            */
    int64_t segments;  /* rays it traced                                                   */
    int64_t evaluated; /* candidates rendered                                              */
} nrrs_mixdepth_result;

/* Mix-Depth search (Sec. 3.3, Brute-Force and Heuristic Search): segment by segment from
 * the shallowest, every combination of {FIXED, HEUR, NET} for the segment's depths is
 * rendered with the earlier depths at their chosen methods and the later ones at fixed
 * RR, and scored by relMSE(render, reference) x segments traced (the inverse of the
 * efficiency 1 / (error x cost) with the deterministic ray count as the cost); the lowest
 * score wins, ties keep the cheaper method.  Synchronizes `stream` per candidate.
 * Errors: INVALID_ARG (sizes, no reference, too many candidates); OOM; CUDA. */
NRRS_API nrrs_status nrrs_mixdepth_search(nrrs_scene* scene, const nrrs_mixdepth_opts* opts,
                                          void* stream, nrrs_mixdepth_result* out);

/* The spatial filter of the training error map (Sec. 4 "Tackle Low Spp"; it stands in
 * for the paper's normal-guided denoiser).  out[p] = sum_q w_pq in[q] / sum_q w_pq over
 * the (2r+1)^2 window of pixel p clipped at the image border.  d_normals NULL or
 * power <= 0: w = 1 (box filter).  Otherwise d_normals is device float [W*H][4] (unit
 * normal xyz, w > 0 when the pixel has one): a pixel with a normal weighs a neighbour
 * with one by max(0, n_p . n_q)^power and one without by 0; a pixel without a normal
 * weighs all by 1; the centre always weighs 1.  d_in, d_out: device float [W*H] (not
 * overlapping).  Errors: INVALID_ARG (NULL arrays, W or H < 1, radius < 0); CUDA. */
NRRS_API nrrs_status nrrs_error_filter(const float* d_in, const float* d_normals, int32_t width,
                                       int32_t height, int32_t radius, float power, float* d_out,
                                       void* stream);

/* relMSE = mean over pixels and RGB of (I - R)^2 / (R^2 + eps) (Sec. 5), in FP64; device
 * images [n_pixels][3], result written to the device double d_out. */
NRRS_API nrrs_status nrrs_relmse(const float* d_img, const float* d_ref, int64_t n_pixels,
                                 double eps, double* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NRRS_H */
