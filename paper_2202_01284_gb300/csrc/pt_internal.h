// Internal device-side data layout shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pt.h"

namespace ptgb {

// Shape record on the device: four 16-byte words (one __ldg each).
struct alignas(16) DevShape {
  int bsdf, tex, albedo_index, rough_index;  // word 0
  float alpha, eta, wd, emitter;              // word 1 (emitter: 1.0 if it emits)
  float f0x, f0y, f0z, pad0;                  // word 2
  float lex, ley, lez, pad1;                  // word 3
};

// Camera precomputed on the host (double -> float).
struct DevCamera {
  float ox, oy, oz;
  float fx, fy, fz;   // forward
  float rx, ry, rz;   // right * tan(vfov/2) * aspect
  float ux, uy, uz;   // up * tan(vfov/2)
};

struct DevScene {
  // geometry in BVH leaf order: three float4 per triangle (v0 | orig id bits, e1, e2)
  const float4* tri_v;
  // attributes in leaf order: (u0, v0, u1, v1), (u2, v2, shape bits, 0)
  const float4* tri_a;
  const float4* nodes;   // binary: 4 float4 per node; wide: 5 uint4 per node
  int layout;            // PT_BVH_BINARY / PT_BVH_WIDE
  int n_tris;
  const DevShape* shapes;
  int n_shapes;
  // area lights: 4 float4 per light triangle: v0 (w = orig tri id bits), v1, v2, Le
  const float4* lights;
  const float* light_cdf;  // [n_lights + 1], normalised
  const int* light_guide;  // [light_g + 1]: first index picked for u = g / light_g
  int light_g;
  int n_lights;
  float light_area;
  // environment map
  const float4* env;       // [h][w]
  const float* env_marg;   // [h + 1]
  const float* env_cond;   // [h][w + 1]
  const float* env_p;      // [h][w] pixel probabilities
  const int* env_marg_guide;  // [env_gm + 1]
  const int* env_cond_guide;  // [h][env_gc + 1]
  int env_gm, env_gc;
  int env_w, env_h;
  int* status;             // device status word (first error wins)
};

struct DevParams {
  const float* albedo;
  const float4* tex[PT_MAX_TEX];
  int tex_w[PT_MAX_TEX], tex_h[PT_MAX_TEX];
  const float* rough;
  const float4* env;  // environment radiance for shading (NULL: the scene's map)
  int n_albedo, n_rough;
};

struct DevGrads {
  float* albedo;
  float4* tex[PT_MAX_TEX];
  float* rough;
  float4* env;
  int n_albedo, n_rough;
};

// Everything one render launch needs (passed by value as the kernel parameter;
// batched launches keep arrays of them in device memory and copy records with
// 16-byte loads, hence the alignment).
struct alignas(16) LaunchArgs {
  DevScene scene;
  DevParams params;
  DevParams tangent;          // forward mode: direction in parameter space (NULL members = 0)
  DevGrads grads;
  int n_cams, width, height, spp, max_depth, rr_depth, nee, dispatch;
  int crop_x0, crop_y0, crop_w, crop_h;
  int lanes_per_pixel, log2_lanes;
  int tex_aggregate;
  unsigned long long seed, seed_adj;  // forward / adjoint PCG32 initstate
  long long n_units;          // n_cams * crop_w * crop_h * lanes_per_pixel
  float* image;               // forward output
  float* image_dot;           // forward mode: derivative of the image along `tangent`
  const float* grad_image;    // adjoint input
  const float* target;        // batched jobs: L2-loss target image (NULL = forward only)
  float loss_scale;           // batched jobs: dLoss/dI = 2 * (I - T) * loss_scale
  float* dbg_L;
  uint32_t* dbg_hash;
  unsigned long long* counters;
  // persistent launches: work counter (units handed out so far), zeroed before the launch
  unsigned long long* queue;
  long long queue_pad_;
  // radiance cache: 0 off, 1 terminate + write queries, 2 terminate + read cache
  // radiance (adjoint), 3 full-length training paths writing records
  int cache_mode, cache_bounce;
  float* q_raw;        // [slots][10]
  float* q_beta;       // [slots][3]
  const float* q_rgb;  // [slots][3]
  float* r_raw;        // [max_records][10]
  float* r_aux;        // [max_records][8]: beta(3), L_before(3), path id bits, pad
  float* path_L;       // [slots][3]
  unsigned* r_count;   // records written (may exceed max_records: extra ones dropped)
  long long max_records;
  // reverse-mode checkpoints (one per path vertex): 4 words of 16 B per vertex,
  // word-major [vertex][word][slot]; ck_count[slot] = vertices of the sample
  uint4* ck_state;
  int* ck_count;
  long long ck_slots;
  float* sample_L;             // split PRB: [slots][3] radiance of each sample (adjoint seed)
  DevCamera cams[PT_MAX_CAMS];
};
static_assert(sizeof(LaunchArgs) % 16 == 0, "job records are copied with 16-byte loads");

// Implemented in pt_nrc.cu (radiance-cache kernels used by the render launchers).
int cache_infer(pt_cache* c, const float* raw, float* rgb, long long n, cudaStream_t st);
int cache_optimise(pt_cache* c, const float* raw, const float* target, long long n, int steps, cudaStream_t st);
struct CacheBuffers {
  float *q_raw, *q_beta, *q_rgb, *r_raw, *r_aux, *r_target, *path_L;
  unsigned* r_count;
  long long max_queries, max_records, max_paths;
};
CacheBuffers cache_buffers(pt_cache* c);

// Host helpers of the render entry points (pt_render.cu): validate a render
// description and parameters into launch arguments; block and grid of a launch.
int fill_launch(pt_scene* s, const pt_render_desc* r, const pt_params* p, LaunchArgs& A);
int launch_dims(const pt_render_desc* r, const LaunchArgs& A, int& block, long long& grid);
// Split-PRB radiance pass (the forward megakernel with seed_adj storing each sample's
// radiance, 12 B per sample, into scene-owned scratch grown with cudaMalloc);
// A.sample_L points at the scratch afterwards.
int radiance_pass(pt_scene* s, const pt_render_desc* r, LaunchArgs& A, cudaStream_t cs);

}  // namespace ptgb

// Library-side scene object behind the opaque pt_scene handle.
struct pt_scene {
  ptgb::DevScene dev;       // device pointers handed to kernels
  // host copies needed for (re)building the BVH
  int n_tris = 0;
  float* h_vertices = nullptr;  // [n][3][3]
  float* h_uvs = nullptr;       // [n][3][2]
  int* h_tri_shape = nullptr;   // [n]
  int n_shapes = 0;
  int has_bvh = 0;
  int max_tex_slot = -1;        // highest texture slot any shape uses
  int max_albedo_row = -1;
  int max_rough = -1;
  // device allocations owned by the scene
  void* d_tri_v = nullptr;
  void* d_tri_a = nullptr;
  void* d_nodes = nullptr;
  void* d_shapes = nullptr;
  void* d_lights = nullptr;
  void* d_light_cdf = nullptr;
  void* d_env = nullptr;
  void* d_env_marg = nullptr;
  void* d_env_cond = nullptr;
  void* d_env_p = nullptr;
  void* d_light_guide = nullptr;
  void* d_env_marg_guide = nullptr;
  void* d_env_cond_guide = nullptr;
  void* d_status = nullptr;     // 256 B: status word, then the work counter
  unsigned long long* queue = nullptr;  // work counter of persistent launches (inside d_status)
  void* d_wf = nullptr;         // wavefront scratch (grown on demand)
  size_t wf_bytes = 0;
  void* d_sample_L = nullptr;   // split PRB: per-sample radiance (grown on demand)
  size_t sample_L_bytes = 0;
  pt_scene_info info{};
};
