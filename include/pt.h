/*
 * pt.h -- C ABI of the GB300 path-tracing megakernel and its PRB adjoint.
 *
 * The library renders images with a unidirectional path tracer and
 * differentiates a loss on them with respect to scene parameters, the problem
 * stated in the introduction of the Dr.Jit paper (Sec. 1) and decomposed into
 * megakernels in Fig. 7 (Sec. 4):
 *   - pt_render_forward  : megakernel #1, the primal path tracer;
 *   - pt_render_backward : megakernels #2 + #3 fused, Path Replay
 *                          Backpropagation (Sec. 4.1) with detached BSDF
 *                          sampling and attached BSDF values (Sec. 4.9);
 *   - pt_cache_*         : a learned radiance cache that terminates paths
 *                          (not in the paper; the paper mentions caches only
 *                          as future work, Sec. 3.2);
 *   - pt_render_batch    : many cameras/scenes in one persistent launch.
 *
 * Conventions
 *   - Every function returns PT_OK (0) or a negative PT_ERR_* code; nothing
 *     aborts.  pt_status_string() names a code.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Rendering calls are asynchronous on it; device-side faults the kernels
 *     detect (e.g. BVH stack overflow, queue timeouts) are recorded in a
 *     per-scene status word read by pt_last_device_status().
 *   - Scene geometry and materials are COPIED into library-owned device memory
 *     by pt_scene_create.  Differentiable parameters (pt_params) and gradient
 *     buffers (pt_grads) are BORROWED device pointers: they must stay valid
 *     until the stream has passed the call.  Gradients are ACCUMULATED (+=),
 *     never cleared by the library.
 *   - Images are float32 RGB, row-major [n_cams][rows][cols][3], row 0 = top.
 *     With a crop rectangle, rows/cols are the crop's.
 *   - The kernels need no scratch memory beyond their inputs and outputs.
 */
#ifndef PT_H_
#define PT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define PT_OK 0
#define PT_ERR_ARG (-1)      /* invalid argument or descriptor */
#define PT_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define PT_ERR_OOM (-3)      /* device allocation failed */
#define PT_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define PT_ERR_BVH (-5)      /* BVH missing, or traversal stack overflow */
#define PT_ERR_STATE (-6)    /* call order violated (e.g. render before bvh_build) */

/* ------------------------------------------------------------------ limits */
#define PT_MAX_TEX 8      /* texture slots per scene */
#define PT_MAX_CAMS 64    /* cameras per pt_render_forward/backward call */

/* ------------------------------------------------------------------ materials
 * BSDF codes (the polymorphic call of Sec. 3.1/3.3: one code path per type,
 * dispatched per lane):
 *   NONE       black; a path that reaches it stops (pure emitters).
 *   DIFFUSE    Lambertian, f = albedo/pi; albedo constant or textured.
 *   CONDUCTOR  rough GGX microfacet conductor, Schlick Fresnel (F0 per shape),
 *              uncorrelated Smith shadowing, Walter-2007 half-vector sampling.
 *   DIELECTRIC smooth interface of relative IOR eta, exact Fresnel.
 *   BLEND      w * diffuse + (1-w) * GGX conductor (the lobe is chosen with
 *              probabilities w, 1-w).
 */
enum { PT_BSDF_NONE = 0, PT_BSDF_DIFFUSE = 1, PT_BSDF_CONDUCTOR = 2, PT_BSDF_DIELECTRIC = 3, PT_BSDF_BLEND = 4 };

/* One shape record (the closure data of App. B: scalars inline, textures by
 * slot).  A triangle's shape is tri_shape[t]. */
typedef struct {
  int32_t bsdf;          /* PT_BSDF_* */
  int32_t tex;           /* texture slot of the albedo (DIFFUSE/BLEND), -1 = constant */
  int32_t albedo_index;  /* row of pt_params.albedo used when tex < 0, -1 = black */
  int32_t rough_index;   /* entry of pt_params.roughness, -1 = use `alpha` */
  float alpha;           /* fixed GGX roughness when rough_index < 0 */
  float eta;             /* DIELECTRIC: interior/exterior IOR */
  float diffuse_weight;  /* BLEND: w */
  float f0[3];           /* CONDUCTOR/BLEND: Schlick reflectance at normal incidence */
  float emission[3];     /* radiance emitted on the front side (normal = (v1-v0)x(v2-v0)) */
} pt_shape;

/* Scene input (host memory, copied). */
typedef struct {
  int32_t n_tris;
  const float* vertices;     /* [n_tris][3][3] */
  const float* uvs;          /* [n_tris][3][2] or NULL (all zero) */
  const int32_t* tri_shape;  /* [n_tris] */
  int32_t n_shapes;
  const pt_shape* shapes;    /* [n_shapes] */
  int32_t env_w, env_h;      /* environment map size, 0 = none */
  const float* env;          /* [env_h][env_w][4] RGBA, equirectangular, row 0 looks along +y,
                                column angle from +x toward +z */
} pt_scene_desc;

typedef struct pt_scene pt_scene;
typedef struct pt_cache pt_cache;

/* Copy geometry, shape table and environment map to the device, and build the
 * emitter tables (area-proportional triangle CDF; environment map marginal and
 * conditional CDFs over luminance x sin(theta)).  Synchronous.  *out receives
 * a handle owned by the caller (pt_scene_destroy).
 * Errors: PT_ERR_ARG (NULL pointers, n_tris <= 0, shape index out of range,
 * bad BSDF code, tex slot >= PT_MAX_TEX, non-finite vertices / uvs / shape
 * scalars, negative or non-finite emission or environment radiance, emitting
 * shapes of zero total area), PT_ERR_OOM, PT_ERR_CUDA.  All checks run before any
 * device call. */
int pt_scene_create(const pt_scene_desc* desc, pt_scene** out);
void pt_scene_destroy(pt_scene* scene);

/* ------------------------------------------------------------------ BVH */
enum { PT_BVH_BINARY = 0, PT_BVH_WIDE = 1 };
typedef struct {
  int32_t layout;        /* PT_BVH_BINARY (2-wide, float boxes) or PT_BVH_WIDE
                            (8-wide, 8-bit quantised child boxes) */
  int32_t max_leaf_tris; /* 1..8 for BINARY, 1..3 for WIDE (0 = default 4 / 3) */
  int32_t n_bins;        /* SAH bins, 4..64 (0 = 32) */
} pt_bvh_opts;

/* Build the acceleration structure on the host (binned SAH over triangle
 * centroids, Sec. 3.1 delegates this to Embree/OptiX; here it is our own) and
 * upload it.  Re-callable; replaces the previous BVH.  Synchronous.
 * opts may be NULL (defaults).  Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA. */
int pt_bvh_build(pt_scene* scene, const pt_bvh_opts* opts);

typedef struct {
  int64_t n_tris, n_nodes, node_bytes, tri_bytes, env_bytes;
  int32_t layout, depth;
  double sah_cost;
} pt_scene_info;
int pt_scene_get_info(const pt_scene* scene, pt_scene_info* info);

/* ------------------------------------------------------------------ rendering */
typedef struct {
  float origin[3], target[3], up[3];
  float vfov_deg;  /* vertical field of view of the pinhole */
} pt_camera;

enum { PT_DISPATCH_SWITCH = 0, PT_DISPATCH_MATCH = 1 };

/* Counters filled by instrumented launches (pt_render_desc.counters). */
enum {
  PT_CNT_PATHS = 0,      /* camera samples traced */
  PT_CNT_RAYS = 1,       /* closest-hit rays (camera + continuation) */
  PT_CNT_SHADOW = 2,     /* shadow (any-hit) rays */
  PT_CNT_NODES = 3,      /* BVH nodes visited (all rays) */
  PT_CNT_TRIS = 4,       /* ray/triangle tests */
  PT_CNT_TEX = 5,        /* texture lookups */
  PT_CNT_ATOMICS = 6,    /* gradient atomics issued after aggregation */
  PT_CNT_GRAD_TERMS = 7, /* gradient terms before aggregation */
  PT_CNT_V_DIFFUSE = 8,  /* shaded vertices per BSDF type: diffuse, */
  PT_CNT_V_CONDUCTOR = 9,   /* GGX conductor, */
  PT_CNT_V_DIELECTRIC = 10, /* smooth dielectric, */
  PT_CNT_V_BLEND = 11,      /* diffuse + GGX blend */
  PT_CNT_ENV = 12,       /* environment-map lookups (escaped rays and env light samples) */
  PT_CNT_TEX_TERMS = 13, /* texel gradient terms (float4) among PT_CNT_GRAD_TERMS */
  PT_CNT_WARP_NODE_STEPS = 14, /* traversal node-loop iterations, counted once per warp: the
                                  traversal's SIMT efficiency is PT_CNT_NODES / (32 x this) */
  PT_CNT_WARP_LOOP_STEPS = 15, /* megakernel iterations, once per warp: lanes that traced a ray
                                  are (PT_CNT_RAYS + PT_CNT_SHADOW) / (32 x this) */
  PT_N_COUNTERS = 16
};

typedef struct {
  int32_t n_cams;             /* 1..PT_MAX_CAMS; cameras share size and spp */
  const pt_camera* cams;      /* host [n_cams]; camera i uses RNG stream prefix i */
  int32_t width, height;      /* full image size (pixel -> RNG stream mapping) */
  int32_t spp;                /* samples per pixel, >= 1, <= 4096 */
  int32_t max_depth;          /* path segments; 1 = directly visible emission only */
  int32_t rr_depth;           /* Russian roulette at vertices reached by segment >= rr_depth; -1 = off */
  int32_t nee;                /* next-event estimation + MIS (1) or BSDF sampling only (0) */
  uint64_t seed;              /* PCG32 initstate; initseq = (cam<<40)|(pixel<<12)|sample */
  int32_t dispatch;           /* PT_DISPATCH_SWITCH or PT_DISPATCH_MATCH (warp ballot grouping) */
  int32_t crop_x0, crop_y0, crop_w, crop_h;  /* crop_w == 0: whole image */
  int32_t lanes_per_pixel;    /* 1,2,4,..,32 threads sharing a pixel's samples; 0 = auto */
  int32_t block_size;         /* threads per CTA (multiple of 32, <= 1024); 0 = auto */
  int32_t tex_aggregate;      /* backward only: 1 = warp-aggregate texel gradient atomics
                                 (__match_any_sync + shuffle tree), 0 = one float4 atomic per term */
  /* instrumentation (device pointers; all NULL for the production path) */
  float* dbg_sample_L;        /* [n_cams][rows][cols][spp][3] per-sample radiance */
  uint32_t* dbg_sample_hash;  /* [n_cams][rows][cols][spp] FNV-1a of the path's discrete decisions */
  unsigned long long* counters; /* [PT_N_COUNTERS], accumulated */
  /* radiance cache (NULL = plain path tracing).  Paths end at the first non-delta
   * vertex reached by segment >= cache_bounce: emission there is added as usual,
   * then beta * max(cache(x, w_o, n, alpha), 0) replaces the rest of the path
   * (the cache predicts reflected radiance).  Needs cache max_queries >=
   * n_cams * rows * cols * spp.  The backward pass uses the cache radiance as a
   * detached incident radiance at that vertex. */
  struct pt_cache* cache;
  int32_t cache_bounce;         /* >= 1 */
  /* pt_render_backward only, PT_PRB_*: SPLIT runs the paper's separate phases -- a
   * forward kernel stores every sample's radiance (12 B per sample in scene-owned
   * scratch grown with cudaMalloc, which synchronises the device), then a
   * replay-only adjoint kernel; FUSED traces each sample for its radiance and
   * replays it in one kernel (no scratch).  AUTO (0) = SPLIT.  SPLIT applies to the
   * plain adjoint (no cache, env gradients, texel aggregation or counters); the
   * others run fused. */
  int32_t prb_mode;
  /* PT_SCHED_*: how threads take work.  PERSISTENT: a grid that fills the GPU once,
   * each lane taking the next (pixel, lane) unit from a scene-owned counter when its
   * unit has no samples left (the forward then adds lane sums into the image with
   * float atomics when lanes_per_pixel > 1, so the image's last bits may vary from
   * run to run); STATIC: one unit per thread.  PERSISTENT applies to the forward,
   * split-PRB radiance pass and replay, and forward mode with switch dispatch and no
   * cache or instrumentation (STATIC otherwise).  AUTO (0) = STATIC (measured as fast
   * or faster on every kernel).  Calls on one scene must not overlap on the GPU (the
   * counter is per scene). */
  int32_t schedule;
} pt_render_desc;
enum { PT_PRB_AUTO = 0, PT_PRB_FUSED = 1, PT_PRB_SPLIT = 2 };
enum { PT_SCHED_AUTO = 0, PT_SCHED_PERSISTENT = 1, PT_SCHED_STATIC = 2 };

/* Differentiable parameters: borrowed device pointers. */
typedef struct {
  const float* albedo;        /* [n_albedo][3] constant albedos */
  int32_t n_albedo;
  const float* tex[PT_MAX_TEX]; /* each [tex_h][tex_w][4] RGBA (A unused); nearest lookup
                                   x = min(int(u*w), w-1), y = min(int(v*h), h-1) (App. B) */
  int32_t tex_w[PT_MAX_TEX], tex_h[PT_MAX_TEX];
  int32_t n_tex;
  const float* roughness;     /* [n_rough] GGX alpha per entry */
  int32_t n_rough;
  const float* env;           /* [env_h][env_w][4] environment radiance used for shading, the
                                 scene's map dimensions; NULL = the map given to pt_scene_create.
                                 Importance sampling always uses the scene's map (detached
                                 sampling, Sec. 4.9), so the render is linear in this input. */
} pt_params;

/* Gradient outputs: borrowed device pointers, accumulated (+=); NULL = not wanted. */
typedef struct {
  float* albedo;              /* [n_albedo][3] */
  float* tex[PT_MAX_TEX];     /* each [tex_h][tex_w][4] */
  float* roughness;           /* [n_rough] */
  float* env;                 /* [env_h][env_w][4] environment radiance (emitter gradients,
                                 Sec. 4.10: PRB differentiating the environment map) */
} pt_grads;

/* Primal render (Fig. 7, megakernel #1): image = mean over spp of the path
 * tracer's per-sample radiance.  image: device, [n_cams][rows][cols][3], overwritten.
 * Errors: PT_ERR_ARG, PT_ERR_STATE (no BVH), PT_ERR_CUDA (launch failure). */
int pt_render_forward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                      float* image, void* stream);

/* Adjoint render by Path Replay Backpropagation (Sec. 4.1, Fig. 7 #2+#3):
 * each sample is traced once to obtain its radiance L, then replayed from the
 * same PCG32 state while the remaining radiance L_rem = L - (contributions so
 * far) is maintained; at every vertex the BSDF values' derivatives
 * (d f/d theta)/f (Sec. 4.9) times the radiance they carry, weighted by
 * grad_image/spp, are scatter-added into `grads` (warp-aggregated atomics).
 * grad_image: device, same layout as the forward image, = dLoss/dImage.
 * For decorrelated gradients pass a seed different from the forward's.
 * Errors: as pt_render_forward. */
int pt_render_backward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                       const float* grad_image, const pt_grads* grads, void* stream);

/* ------------------------------------------------------------------ batching
 * Many cameras over several scenes, of uneven size and spp, in one persistent
 * pass per phase: the (job, tile) work items are sorted longest first and handed,
 * one per warp, to the warps of grid = ctas_per_sm x SMs resident CTAs by a global
 * atomic counter.  The forward kernel renders every tile; the adjoint kernel,
 * launched right after it on the same stream, replays every tile of the jobs with
 * a target using the job's backward seed and dLoss/dI = 2 (I - T) / (3 W H),
 * accumulating into the job's gradient buffers.
 * Not in the paper (its megakernels render one image at a time). */
typedef struct {
  pt_scene* scene;             /* all jobs of a batch must use the same BVH layout */
  pt_camera camera;
  int32_t width, height, spp, max_depth, rr_depth, nee;
  uint64_t seed, backward_seed;
  pt_params params;            /* borrowed device pointers */
  pt_grads grads;              /* accumulated (+=); NULL members are skipped */
  float* image;                /* device [height][width][3], written */
  const float* target;         /* device [height][width][3]; NULL = forward only */
} pt_job;

typedef struct {
  int32_t tile;                /* tile side in pixels (one warp's work item), 1..256 */
  int32_t lanes_per_pixel;     /* threads per pixel (power of two <= 32; capped at spp) */
  int32_t ctas_per_sm;         /* resident CTAs per SM, 1..8 */
  int32_t block_size;          /* threads per CTA, multiple of 32, <= 256 */
} pt_batch_opts;

typedef struct pt_batch pt_batch;

/* Validate the jobs, build and upload the job table and the sorted work list
 * (synchronous; device memory owned by the batch).  opts may be NULL
 * (tile 4, 4 lanes, 4 CTAs/SM, 128 threads).  Errors: PT_ERR_ARG (bad job or
 * option, mixed BVH layouts), PT_ERR_STATE (scene without BVH), PT_ERR_OOM. */
int pt_batch_create(const pt_job* jobs, int n_jobs, const pt_batch_opts* opts, pt_batch** out);
/* Reset the work counters and launch the two persistent kernels on `stream`: one
 * memset and two launches, no allocation or host synchronisation, so the call can
 * be captured into one CUDA graph and replayed with a single graph launch. */
int pt_batch_run(pt_batch* batch, void* stream);
int pt_batch_info(const pt_batch* batch, int* n_items);
void pt_batch_destroy(pt_batch* batch);
/* create + run + synchronise + destroy. */
int pt_render_batch(const pt_job* jobs, int n_jobs, const pt_batch_opts* opts, void* stream);

/* Batched render that allocates no device memory (no counterpart in the paper).
 * For callers that may not call cudaMalloc: code running inside a host application
 * or framework that owns the whole device-memory budget, or that forbids device
 * allocation once it has started.  It does the work of pt_batch_create +
 * pt_batch_run, but its scratch -- the job table, the forward and adjoint work lists
 * and the two work counters -- lives in one file-scope device array of about
 * PT_NOALLOC_MAX_JOBS * 3.6 KB + 2 * PT_NOALLOC_MAX_ITEMS * 12 B (~1.8 MB), which
 * every GPU that loads the library holds until the process exits.  The caller
 * still passes inputs and outputs (jobs, with their images, targets, parameters and
 * gradient buffers).
 *   - Limits: n_jobs <= PT_NOALLOC_MAX_JOBS and at most PT_NOALLOC_MAX_ITEMS tiles
 *     in total (ceil(w/tile) * ceil(h/tile) summed over jobs); larger requests
 *     return PT_ERR_ARG before anything is launched (use a larger tile, or
 *     pt_batch_create).
 *   - The first call on a device (with that device current) looks up the array's
 *     device address with cudaGetSymbolAddress; make that first call before any
 *     stream capture.
 *   - A `stream` that is capturing is refused with PT_ERR_STATE: the call copies its
 *     tables from host memory that it frees on return.  pt_batch_create +
 *     pt_batch_run is the form to capture.
 *   - Every call reuses the same array, which keeps the last call's contents; the
 *     work counters are cleared on `stream` before each launch.  Calls whose work
 *     overlaps on the GPU (other streams, or other host threads) race on the array:
 *     serialise them.
 *   - Asynchronous on `stream`; the host-side tables are copied with
 *     cudaMemcpyAsync from pageable memory, which returns once they are consumed. */
#define PT_NOALLOC_MAX_JOBS 64
#define PT_NOALLOC_MAX_ITEMS 65536
int pt_render_batch_noalloc(const pt_job* jobs, int n_jobs, const pt_batch_opts* opts, void* stream);

/* Forward-mode derivative of the render (the paper's forward-mode AD, Sec. 1 and
 * Sec. 4: image-space derivatives "for debugging and visualization"): in one pass,
 * image (as pt_render_forward) and image_dot = d image / d eps at eps = 0 of the
 * render with parameters params + eps * tangent, with sampling detached exactly as
 * in pt_render_backward (so sum(grad_image * image_dot) equals <gradient, tangent>
 * of the backward pass with the same seed).  tangent: device pointers with the
 * layouts of params (NULL members mean zero); texture sizes must match.
 * No radiance cache, crop allowed.  Errors: as pt_render_forward. */
int pt_render_jvp(pt_scene* scene, const pt_render_desc* desc, const pt_params* params, const pt_params* tangent,
                  float* image, float* image_dot, void* stream);

/* Wavefront variant (Sec. 3.4 "wavefront-style evaluation", Sec. 3.5: the megakernel
 * against wavefront execution).  The same estimator as pt_render_forward /
 * pt_render_backward (same random numbers and decisions), computed by one kernel per
 * stage with the path state in device memory: a wave of whole pixels runs max_depth
 * rounds of closest-hit traversal, shading, shadow traversal and finish, each over a
 * queue of paths.  calls: PT_WF_TRACED = one shading kernel with the material switch
 * inside; PT_WF_GROUPED = paths sorted into one queue per material by the closest-hit
 * kernel, one shading kernel per material.  wave_paths: samples per wave (0 = 4 Mi;
 * rounded down to whole pixels; at most 2^28).  Scratch (about 360 B per path of a
 * wave) is owned by the scene, grown on demand (cudaMalloc, which synchronises the
 * device) and freed with it; calls on one scene must be ordered on one stream.
 * desc: dbg_sample_L / dbg_sample_hash honoured by the forward; counters, cache and
 * (backward) per-sample outputs are PT_ERR_ARG; lanes_per_pixel, block_size and
 * dispatch are ignored.  Errors: as pt_render_forward / _backward, PT_ERR_OOM. */
enum { PT_WF_TRACED = 0, PT_WF_GROUPED = 1 };
typedef struct pt_wavefront_opts {
  int32_t calls;       /* PT_WF_TRACED or PT_WF_GROUPED */
  int32_t wave_paths;  /* 0 = default */
} pt_wavefront_opts;
int pt_wavefront_forward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                         const pt_wavefront_opts* opts, float* image, void* stream);
int pt_wavefront_backward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                          const pt_wavefront_opts* opts, const float* grad_image, const pt_grads* grads,
                          void* stream);

/* Tensor-core engine of the cache MLP: PT_CACHE_TCGEN05 (default) runs inference,
 * the training forward/backward chain and the weight gradients on the
 * 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory, 128
 * records per MMA tile); PT_CACHE_MMA_SYNC uses warp-level mma.sync (16 records
 * per warp tile, activations in registers), kept for comparison.  Both round
 * inputs and activations to BF16 and accumulate in FP32. */
enum { PT_CACHE_TCGEN05 = 0, PT_CACHE_MMA_SYNC = 1 };
int pt_cache_set_engine(pt_cache* cache, int engine);
/* Reads (after synchronising `stream`) and clears the cache's device status word:
 * PT_OK, or PT_ERR_TIMEOUT if a bounded wait on the tensor core gave up (the
 * outputs of that call are then incomplete). */
int pt_cache_status(pt_cache* cache, void* stream, int* status);
/* Checkpoint / resume of cache training (no counterpart in the paper): the FP32
 * master weights, Adam's first and second moments (each PT_CACHE_N_PARAMS floats,
 * host memory) and the Adam step count.  set_state restores all of them (the BF16
 * weights are re-derived), so training continues exactly as if uninterrupted.
 * Both synchronise the device. */
int pt_cache_get_state(pt_cache* cache, float* weights, float* m, float* v, int32_t* step);
int pt_cache_set_state(pt_cache* cache, const float* weights, const float* m, const float* v, int32_t step);

/* Failure injection for the bounded waits of the tcgen05 kernels (no counterpart in
 * the paper): each MMA step polls its completion barrier at most `limit` times
 * (default PT_CACHE_WAIT_LIMIT_DEFAULT) before the kernel gives up, records
 * PT_ERR_TIMEOUT in the cache's status word (pt_cache_status) and returns after
 * letting the MMA in flight finish (that last wait always uses the default).
 * limit = 0 makes the timeout path run deterministically. */
#define PT_CACHE_WAIT_LIMIT_DEFAULT (1u << 22)
int pt_cache_set_wait_limit(pt_cache* cache, uint32_t limit);

/* Reverse mode with checkpoints (Sec. 4.10: differentiating a standard path tracer
 * whose loop keeps one checkpoint per scattering event, against PRB).
 * pt_ckpt_forward renders like pt_render_forward and stores, before every
 * closest-hit ray, the loop state of the path (PCG32 state, ray, throughput, MIS
 * state, depth: 64 B) plus each sample's vertex count.  pt_ckpt_backward, called
 * with the same scene, desc and params, recomputes each sample's vertices from
 * their checkpoints last to first and accumulates the gradients of
 * sum(grad_image * image) like pt_render_backward with the forward's seed (the
 * same estimator; no radiance pass, the radiance of the later vertices is summed
 * on the way back).  Gradients as pt_render_backward, including env.
 * The buffer holds max_samples (n_cams * rows * cols * spp of a call) x max_depth
 * checkpoints; pt_ckpt_create allocates it (cudaMalloc, synchronous) and clears
 * the counts.  Calls with more samples or depth than the buffer holds, counters,
 * per-sample outputs or a cache are PT_ERR_ARG.  A backward call after a forward
 * with a different desc reads whatever checkpoints are stored (vertex counts are
 * clamped to the buffer, so it stays in bounds) and returns a wrong gradient. */
typedef struct pt_ckpt pt_ckpt;
int pt_ckpt_create(int64_t max_samples, int32_t max_depth, pt_ckpt** out);
void pt_ckpt_destroy(pt_ckpt* ckpt);
int pt_ckpt_bytes(const pt_ckpt* ckpt, int64_t* bytes);
int pt_ckpt_forward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params, pt_ckpt* ckpt,
                    float* image, void* stream);
int pt_ckpt_backward(pt_scene* scene, const pt_render_desc* desc, const pt_params* params, pt_ckpt* ckpt,
                     const float* grad_image, const pt_grads* grads, void* stream);

/* ------------------------------------------------------------------ reparameterized PRB
 * Gradients with respect to shape TRANSLATIONS through visibility (Sec. 4.7,
 * reparameterizations; Sec. 4.8, the derivative terms of moving vertices; warp
 * field after Bangaru et al. 2020).  The parameters are one translation per
 * shape (all of its vertices move together; a surface point keeps its
 * barycentric coordinates).  Every traced ray -- the camera ray and, at diffuse,
 * GGX-conductor and blend vertices, the light-sample ray and the BSDF-sampled ray
 * -- is reparameterized: n_aux auxiliary rays in a von Mises-Fisher lobe
 * (concentration kappa) around it estimate a warp field V that follows the
 * geometry they hit (the closer surface dominating near silhouettes, escaping rays
 * weighted `miss`), and the ray contributes m.V + R div V, R = grad_image .
 * (radiance the ray carries), m = R times the ray's cosine (or, for camera rays,
 * the pinhole's image-plane density) term plus, at glossy vertices, the BSDF's
 * gradients in its two directions.  Rays leaving dielectric vertices are not
 * reparameterized (their directional terms stay detached; the paper notes that
 * specular interfaces are an open problem).  The warp estimator is consistent,
 * not unbiased: its ratio of sample sums is jackknife-corrected.  Because the
 * camera warp also moves the pixels' own footprints (box filter), each edge of a
 * pixel of the crop adds (grad_image right/below - left/above, 0 outside the crop)
 * . integral over the edge of L times the warp's image-plane velocity across it,
 * estimated by edge_spp paths through uniform points of every edge (PCG32 stream
 * camera << 40 | edge << 12 | sample | 2^61; edge = y (width + 1) + x for the
 * vertical edge left of pixel (x, y), (width + 1) height + y width + x for the
 * horizontal one above it; auxiliary stream | 2^62); on the image border this is
 * the flux of radiance entering or leaving the image.  Optionally (border > 0)
 * the camera warp is instead windowed to zero within `border` pixels of the image
 * border, which biases whatever moves there.  The camera is static; its
 * translation is minus the sum of all shapes' translations (the environment lies
 * at infinity).
 *
 * A radiance pass (as split PRB: the forward megakernel storing each sample's
 * radiance, 12 B per sample, in scene-owned scratch grown with cudaMalloc, which
 * synchronises the device) precedes a replay (PRB) with the warps in which the
 * lanes of a warp trace the auxiliary rays of one or two rays together;
 * auxiliary random numbers come from a second PCG32 stream of the sample
 * (initseq | 2^62): 2 n_aux for the camera ray, then 4 n_aux at every vertex that
 * draws its 8 path uniforms (light-sample ray first, then BSDF ray), used or not.
 *
 * grad_translation: device float [n_shapes][3], accumulated (+=).  rays: device
 * counter of the rays traced (radiance pass -- counted as the replay's path and
 * shadow rays, which it repeats --, replay, auxiliary and the warps' own center
 * rays, the pixel-edge paths and their warps), accumulated; NULL = not wanted.
 * desc.counters: node and triangle visits of the replay and pixel-edge kernels
 * (not of the radiance pass).  desc: as for pt_render_backward (the seed is used
 * for both passes); block_size must be 0 or 128; no cache or per-sample outputs.  opts: NULL = defaults
 * (pt_reparam_defaults).  Errors: PT_ERR_ARG (options out of range: 2 <= n_aux <=
 * 32, 0 < kappa <= 1e6, kernel_scale >= 1, 0 <= power <= 16, miss >= 0, eps > 0,
 * border >= 0, jackknife 0/1, 0 <= edge_spp <= 4096; with edge_spp > 0 the image's
 * edge count (width + 1) height + width (height + 1) below 2^28), PT_ERR_STATE,
 * PT_ERR_CUDA. */
typedef struct {
  int32_t n_aux;        /* auxiliary rays per reparameterized ray (16) */
  float kappa;          /* vMF concentration of the auxiliary lobe (1000) */
  float kernel_scale;   /* the weighting kernel is this many times more concentrated (8) */
  float power;          /* depth-weight exponent: g = (t0 / t)^power (2) */
  float miss;           /* weight of an auxiliary ray that escapes (0.01) */
  float eps;            /* floor of the normaliser, per auxiliary ray (1e-4) */
  float border;         /* camera-warp window width at the image border, pixels; 0 = none (0) */
  int32_t jackknife;    /* leave-one-out correction of the ratio's 1/N bias (1) */
  int32_t edge_spp;     /* paths per pixel edge for the pixel-edge term, 0 = off (1) */
} pt_reparam_opts;
void pt_reparam_defaults(pt_reparam_opts* opts);
int pt_render_backward_reparam(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                               const pt_reparam_opts* opts, const float* grad_image, float* grad_translation,
                               unsigned long long* rays, void* stream);
/* The same estimator with every triangle corner's position as a parameter (the
 * paper's vertex-position optimisation, Sec. 4.10): a surface point moves with its
 * barycentric weights, so the warp's plane points carry the barycentric
 * coordinates of the (extended) hit triangle, and the cosine and (glossy BSDFs)
 * the BSDF value of a moving vertex add the derivative of its triangle's turning
 * normal.  grad_vertices: device float
 * [n_tris][3][3] in the order of pt_scene_desc.vertices (corner k of triangle t at
 * [t][k]), accumulated; shared positions are the caller's to sum.  The per-corner
 * gradients of a shape sum to its translation gradient.  Same arguments, counters
 * and errors as pt_render_backward_reparam. */
int pt_render_backward_reparam_vertices(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                                        const pt_reparam_opts* opts, const float* grad_image, float* grad_vertices,
                                        unsigned long long* rays, void* stream);

/* Forward mode of the same estimator (the paper's forward derivative of a
 * translated mesh, Sec. 4.7, Fig. "bunny": without reparameterization the
 * silhouettes' and reflections' derivatives are missing): image_dot = d image /
 * d eps of the render with every shape s moved by eps * dir_translation[s], in one
 * pass without a radiance pass.  Each reparameterized ray's warp returns its
 * tangential value V and div V for the direction; the path carries the per-channel
 * derivative of its log throughput, and the pixel-edge term's edge paths add
 * their flux to the two pixels of their edge.  With the same seed, sum(grad_image *
 * image_dot) equals <dir_translation, gradient of pt_render_backward_reparam> up
 * to float rounding (the same estimator in the other mode).  dir_translation:
 * device float [n_shapes][3]; image (NULL: not wanted) and image_dot: device float
 * [n_cams][crop_h][crop_w][3], overwritten (zeroed on the stream, then
 * accumulated).  rays: as pt_render_backward_reparam (path, shadow, auxiliary,
 * center and edge rays).  desc: as pt_render_backward_reparam, no counters.
 * Errors: as pt_render_backward_reparam. */
int pt_render_jvp_reparam(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                          const pt_reparam_opts* opts, const float* dir_translation, float* image, float* image_dot,
                          unsigned long long* rays, void* stream);
/* The same along a direction of every triangle corner's position: dir_vertices,
 * device float [n_tris][3][3] in the order of pt_scene_desc.vertices (corner k of
 * triangle t at [t][k]); a surface point moves with its barycentric weights, and
 * a moving vertex's cosine and glossy BSDF value follow its triangle's turning
 * normal.  Pairs with pt_render_backward_reparam_vertices as the translation form
 * with pt_render_backward_reparam.  Other arguments and errors as above. */
int pt_render_jvp_reparam_vertices(pt_scene* scene, const pt_render_desc* desc, const pt_params* params,
                                   const pt_reparam_opts* opts, const float* dir_vertices, float* image,
                                   float* image_dot, unsigned long long* rays, void* stream);

/* Ray queries against the scene's BVH, through the same traversal the path tracer runs
 * (the scene-intersection call of the paper's rendering API, Sec. 3.1, which Mitsuba 3
 * hands to Embree or OptiX; here the library's own 2- or 8-wide BVH).  Asynchronous on
 * stream.  rays: device [n][6] floats (origin xyz, direction xyz; t is measured in units
 * of the direction, which need not be unit length); tmax: device [n] or NULL (no limit);
 * any_hit = 0: the closest hit with 0 < t < tmax (ties in t go to the smaller triangle
 * index); any_hit = 1: some hit with 0 < t < tmax (shadow-ray semantics).  Outputs
 * (device): t [n] (INFINITY on a miss), prim [n] (the input index of the hit triangle as
 * given to pt_scene_create, -1 on a miss), uv [n][2] or NULL (barycentric coordinates of
 * the hit on that triangle: p = (1 - u - v) v0 + u v1 + v v2).  A ray with a non-finite
 * component or a zero direction misses.  Errors: PT_ERR_ARG (n <
 * 0, null pointers with n > 0), PT_ERR_STATE (no BVH built), PT_ERR_CUDA (launch); a
 * traversal stack overflow is reported later by pt_last_device_status as PT_ERR_BVH. */
int pt_trace_rays(pt_scene* scene, const float* rays, const float* tmax, int n, int any_hit, float* t, int* prim,
                  float* uv, void* stream);

/* Reads (and clears) the scene's device status word after synchronising
 * `stream`: *out = PT_OK or the first PT_ERR_* a kernel recorded. */
int pt_last_device_status(pt_scene* scene, void* stream, int* out);

const char* pt_status_string(int status);

/* ------------------------------------------------------------------ radiance cache
 * A small MLP that predicts the radiance reflected at a surface point toward a
 * direction (Mueller et al. 2021, "Real-time Neural Radiance Caching"); the paper
 * itself names caches only as an open direction (Sec. 3.2).  Input: raw records
 * of 10 floats (position[3], unit direction toward the previous vertex[3], shading
 * normal[3], GGX roughness or 1 for diffuse), encoded in-kernel into 64 features:
 * position normalised to [box_lo, box_hi] with sin/cos(2^k pi x), k < 6; direction
 * and normal mapped to [0,1] with k < 2; roughness; three constant ones.  Network:
 * five 64x64 ReLU layers and a 64x3 linear head, no biases; BF16 weights and
 * activations, FP32 accumulation (tensor cores).  Loss: relative L2,
 * sum_c (y_c - t_c)^2 / (y_c^2 + 0.01) (denominator not differentiated), mean over
 * the batch.  Optimiser: Adam.  Weight layout (FP32, PT_CACHE_N_PARAMS): layer l
 * (0..4) at l*4096 as [out 64][in 64], then the head [3][64]. */
#define PT_CACHE_N_PARAMS 20672

typedef struct {
  float box_lo[3], box_hi[3];   /* position-encoding box (scene bounds) */
  int32_t batch;                /* training batch, multiple of 64 (e.g. 65536) */
  int32_t max_queries;          /* capacity of cache-terminated samples per render call */
  int32_t max_records;          /* capacity of training records per pt_cache_train call */
  int32_t max_paths;            /* capacity of training paths per pt_cache_train call */
  float lr, beta1, beta2, eps;  /* Adam */
  const float* init_weights;    /* host [PT_CACHE_N_PARAMS] or NULL (uniform +-sqrt(6/64) from `seed`) */
  uint64_t seed;
  float ema;                    /* in [0, 1): 0 = queries use the trained weights; else every Adam step
                                   also updates A = ema * A + (1 - ema) * W (A starts at the initial
                                   weights) and queries, cache-terminated renders and their adjoint use
                                   A (Polyak averaging: the weights' step-to-step noise averaged out) */
} pt_cache_desc;

/* Allocate weights, Adam state and all buffers on the current device (synchronous).
 * Errors: PT_ERR_ARG (batch not a positive multiple of 64, empty box, negative
 * capacities), PT_ERR_OOM, PT_ERR_CUDA. */
int pt_cache_create(const pt_cache_desc* desc, pt_cache** out);
void pt_cache_destroy(pt_cache* cache);
/* Synchronous copies of the FP32 master weights; set also resets Adam. */
int pt_cache_get_weights(pt_cache* cache, float* host_out);
int pt_cache_set_weights(pt_cache* cache, const float* host_in);
/* rgb[i] = MLP(encode(raw[i])), device pointers raw [n][10], rgb [n][3]; async on stream. */
int pt_cache_query(pt_cache* cache, const float* raw, float* rgb, int n, void* stream);
/* The input encoding both inference engines feed to the first layer, as BF16 bits:
 * features [n][64] (device, 16-byte aligned) from raw [n][10] (device); async on
 * stream.  The frequency encoding of the radiance cache above (Mueller et al. 2021;
 * the paper names caches only as an open direction, Sec. 3.2): position normalised
 * to the box, sin and cos of 2^k pi x for k = 0..5 per axis (features 0..35, sin at
 * even indices); inputs outside [-2^15, 2^15] after normalisation are clamped to it;
 * direction and normal mapped to [0, 1] with k = 0, 1 (36..47, 48..59); roughness
 * (60); the constant 1 (61..63).  Octave k = 0 of each coordinate is an FP32 sin /
 * cos within 2 ulp, octave k > 0 follows by k double-angle steps and lies within
 * 2^k * 4 * 2^-24 (absolute) of the exact pair; each value is then rounded to BF16.
 * Errors: PT_ERR_ARG (null pointers with n > 0, n < 0,
 * unaligned output), PT_ERR_CUDA (launch). */
int pt_cache_encode(pt_cache* cache, const float* raw, uint16_t* features, int n, void* stream);
/* Synchronous copies of the averaged weights A (see pt_cache_desc.ema); set_weights
 * also sets A to the given weights. */
int pt_cache_get_average(pt_cache* cache, float* host_out);
int pt_cache_set_average(pt_cache* cache, const float* host_in);
/* `steps` Adam steps on batches taken in order from device records raw [n][10],
 * target [n][3] (wrapping); async on stream. */
int pt_cache_train_records(pt_cache* cache, const float* raw, const float* target, int n, int steps, void* stream);
/* Relative-L2 loss of the last optimisation step (synchronises the stream). */
int pt_cache_last_loss(pt_cache* cache, void* stream, float* out);
/* Online training step: trace the samples of `desc` as full-length training paths
 * (desc->cache is ignored), record at every non-delta vertex below max_depth the
 * raw features and the reflected radiance the rest of the path carried,
 * (L_path - L_up_to_vertex) / throughput, then run `steps` optimisation steps on
 * those records.  Needs max_paths >= samples of desc; records beyond max_records
 * are dropped.  Synchronises the stream once (to read the record count).
 * *n_records (optional) receives the number of records used. */
int pt_cache_train(pt_cache* cache, pt_scene* scene, const pt_render_desc* desc, const pt_params* params, int steps,
                   void* stream, int* n_records);
/* Synchronous host copy of the records of the last pt_cache_train call (for
 * inspection): raw [n][10], target [n][3], meta [n][2] = (sample index
 * pixel * spp + sample, depth of the vertex); any pointer may be NULL.
 * *n_out = min(cap, records kept). */
int pt_cache_read_records(pt_cache* cache, int cap, float* raw, float* target, int* meta, int* n_out);

/* ---------------------------------------------------------------- measurement probes
 * The roofs that bound the traversal's node and triangle fetches (through L2; the
 * paper's Sec. 3.5 finds the megakernel memory-latency bound) and the adjoint's
 * gradient scatter (atomic scatter-adds, Sec. 4.1), which the driver's peak table
 * does not hold.  Both calls are asynchronous on `stream`; time them with events.
 *
 * pt_probe_read: reads the device buffer buf [bytes] (16-byte aligned, bytes a
 * multiple of 16) `passes` times with 16-byte loads cached in L2 only (keep it
 * smaller than L2 to measure L2, larger to measure HBM) and adds the sum of all
 * floats read to *sink (device float, accumulated).  Errors: PT_ERR_ARG.
 *
 * pt_probe_atomic: n_updates fire-and-forget atomic adds of 1.0 to the n_addr
 * addresses of dst (device; width 1: floats, width 4: float4 elements, dst 16-byte
 * aligned), update i going to element (i * 2654435761) mod n_addr -- spread over a
 * large buffer, or colliding on a few elements.  Every element receives
 * n_updates / n_addr (+1) adds.  Errors: PT_ERR_ARG. */
int pt_probe_read(const void* buf, long long bytes, int passes, float* sink, void* stream);
int pt_probe_atomic(float* dst, long long n_addr, long long n_updates, int width, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PT_H_ */
