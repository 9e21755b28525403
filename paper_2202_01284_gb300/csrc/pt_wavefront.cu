// Wavefront variant of the forward render and of the PRB adjoint (Sec. 3.4,
// wavefront-style evaluation; Sec. 3.5 compares it with the megakernel).
//
// The per-path code is the megakernel's (path_start / path_shade / path_finish):
// only the loop is unrolled into one kernel per stage, with the path state kept
// in device memory between the stages.  A wave of paths (whole pixels, all their
// samples) runs max_depth rounds of
//     closest-hit traversal -> shading -> shadow traversal -> finish,
// each stage over a queue of path slots that the previous stage filled.  Two
// modes for the polymorphic material call, the two options the paper gives for
// calls inside wavefront loops:
//   TRACED  - one shading kernel, the material switch inside it;
//   GROUPED - the closest-hit kernel sorts the paths into one queue per material
//             and one shading kernel per material runs over its queue.
// Same random numbers, same decisions, same estimator as the megakernel.
#include <algorithm>
#include <cstring>

#include "pt_path.cuh"

namespace ptgb {
namespace {

constexpr int kStateWords = (int)((sizeof(PathState) + 15) / 16);
constexpr int kMaterials = 5;  // queue 0: misses and PT_BSDF_NONE; 1..4: the BSDF types
enum { C_RAY = 0, C_SHADOW = 1, C_TYPE = 2, kCounts = 8 };
constexpr int kBlock = 256;
// adjoint stages: environment gradients and texel aggregation available
template <bool ADJ>
constexpr int kWfFeat = ADJ ? (FEAT_EGRAD | FEAT_TEXAGG) : 0;
constexpr int kTraceMinBlocks = 4;  // 64 registers: latency-bound traversal wants occupancy
constexpr int kShadeMinBlocks = 3;  // 85 registers, as the adjoint megakernel

// Scratch of one wave (device memory owned by the scene, grown on demand).
struct WfArgs {
  uint4* state;            // [kStateWords][cap]: 16-byte words of PathState, word-major
  Hit* hit;                // [cap] closest hit of the current round
  unsigned char* occ;      // [cap] shadow ray blocked
  float* L;                // [cap][3] radiance of each finished sample
  int* q[2];               // path-ray queues, alternating by round
  int* sq;                 // shadow-ray queue
  int* tq[kMaterials];     // per-material queues (GROUPED)
  int* counts;             // [rounds + 1][kCounts]
  int cap;                 // slots (samples) in a wave
  long long pix0;          // first pixel (dense crop index) of the wave
  int n_pix;               // pixels in the wave
  int grad_pass;           // adjoint: 0 = radiance pass, 1 = replay with gradients
};

__device__ __forceinline__ void load_state(const WfArgs& W, int i, PathState& P) {
  uint4 buf[kStateWords];
#pragma unroll
  for (int k = 0; k < kStateWords; ++k) buf[k] = W.state[(size_t)k * W.cap + i];
  memcpy(&P, buf, sizeof(PathState));
}

__device__ __forceinline__ void store_state(const WfArgs& W, int i, const PathState& P) {
  uint4 buf[kStateWords];
  memcpy(buf, &P, sizeof(PathState));
#pragma unroll
  for (int k = 0; k < kStateWords; ++k) W.state[(size_t)k * W.cap + i] = buf[k];
}

// Loads only the 16-byte words that hold bytes [OFF, OFF + SIZE) of the state.
template <size_t OFF, size_t SIZE>
__device__ __forceinline__ void load_field(const WfArgs& W, int i, void* dst) {
  constexpr int w0 = (int)(OFF / 16), w1 = (int)((OFF + SIZE + 15) / 16);
  uint4 buf[w1 - w0];
#pragma unroll
  for (int k = w0; k < w1; ++k) buf[k - w0] = W.state[(size_t)k * W.cap + i];
  memcpy(dst, reinterpret_cast<const char*>(buf) + (OFF - 16 * w0), SIZE);
}

// Appends slot i to a queue.  Lanes are grouped by their queue (the counter's
// address: the converged lanes of one call site may target different queues),
// one atomic per group.
__device__ __forceinline__ void push(int* q, int* count, int i) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, (unsigned long long)count);
  const int lane = lane_id();
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(peers));
  base = __shfl_sync(active, base, leader);
  q[base + rank] = i;
}

__device__ __forceinline__ int* counts_of(const WfArgs& W, int round) { return W.counts + round * kCounts; }

__device__ __forceinline__ float3 pixel_dl(const LaunchArgs& A, const PathState& P) {
  const long long pix = P.slot / A.spp;
  const float inv = 1.0f / (float)A.spp;
  return f3(A.grad_image[3 * pix] * inv, A.grad_image[3 * pix + 1] * inv, A.grad_image[3 * pix + 2] * inv);
}

// A finished sample: its radiance (and, on request, the per-sample outputs).
__device__ __forceinline__ void finish_sample(const LaunchArgs& A, const WfArgs& W, int i, const PathState& P) {
  W.L[3 * i] = P.L.x;
  W.L[3 * i + 1] = P.L.y;
  W.L[3 * i + 2] = P.L.z;
  if (A.dbg_L) {
    A.dbg_L[3 * P.slot] = P.L.x;
    A.dbg_L[3 * P.slot + 1] = P.L.y;
    A.dbg_L[3 * P.slot + 2] = P.L.z;
  }
  if (A.dbg_hash) A.dbg_hash[P.slot] = P.fh.h;
}

template <bool ADJ>
__global__ void __launch_bounds__(kBlock) wf_start(const __grid_constant__ LaunchArgs A, const __grid_constant__ WfArgs W) {
  const int n = W.n_pix * A.spp;
  const long long per_cam = (long long)A.crop_w * A.crop_h;
  Counters<false> cnt;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long pix = W.pix0 + i / A.spp;
    const int s = i % A.spp;
    const int cam = (int)(pix / per_cam);
    const long long rem = pix - (long long)cam * per_cam;
    const int iy = (int)(rem / A.crop_w);
    const int px = A.crop_x0 + (int)(rem - (long long)iy * A.crop_w), py = A.crop_y0 + iy;
    PathState P;
    path_start<false>(A, P, ADJ ? A.seed_adj : A.seed, cam, px, py, s, pix, cnt);
    P.Lrem = (ADJ && W.grad_pass) ? f3(W.L[3 * i], W.L[3 * i + 1], W.L[3 * i + 2]) : f3(0.f, 0.f, 0.f);
    store_state(W, i, P);
    W.q[0][i] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) counts_of(W, 0)[C_RAY] = n;
}

// Closest-hit (SHADOW = false) or shadow (SHADOW = true) traversal of a queue.
// GROUPED: the closest-hit pass also files each path under its material.
template <int LAYOUT, bool SHADOW, bool GROUPED>
__global__ void __launch_bounds__(kBlock, kTraceMinBlocks) wf_trace(const __grid_constant__ LaunchArgs A, const __grid_constant__ WfArgs W,
                                                   int round) {
  int* c = counts_of(W, round);
  const int n = SHADOW ? c[C_SHADOW] : c[C_RAY];
  const int* q = SHADOW ? W.sq : W.q[round & 1];
  Counters<false> cnt;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = q[j];
    float3 o, d;
    float tmax = INFINITY;
    if constexpr (SHADOW) {
      load_field<offsetof(PathState, so), sizeof(float3)>(W, i, &o);
      load_field<offsetof(PathState, sd), sizeof(float3)>(W, i, &d);
      load_field<offsetof(PathState, stmax), sizeof(float)>(W, i, &tmax);
    } else {
      load_field<offsetof(PathState, ro), sizeof(float3)>(W, i, &o);
      load_field<offsetof(PathState, rd), sizeof(float3)>(W, i, &d);
    }
    const Hit h = LAYOUT == PT_BVH_WIDE ? trace_wide<false>(A.scene, o, d, tmax, SHADOW, cnt)
                                        : trace_binary<false>(A.scene, o, d, tmax, SHADOW, cnt);
    if constexpr (SHADOW) {
      W.occ[i] = h.pos >= 0 ? 1 : 0;
    } else {
      W.hit[i] = h;
      if constexpr (GROUPED) {
        int type = 0;
        if (h.pos >= 0) {
          const int shape = __float_as_int(__ldg(&A.scene.tri_a[2 * h.pos + 1]).z);
          type = __ldg(reinterpret_cast<const int*>(&A.scene.shapes[shape]));
          if (type < 0 || type >= kMaterials) type = 0;
        }
        push(W.tq[type], &c[C_TYPE + type], i);
      }
    }
  }
}

// Shading after the closest hit; paths without a shadow ray are finished here.
// QUEUE < 0: the round's ray queue (TRACED); else that material's queue.
template <bool ADJ, int DISPATCH, int QUEUE>
__global__ void __launch_bounds__(kBlock, kShadeMinBlocks) wf_shade(const __grid_constant__ LaunchArgs A, const __grid_constant__ WfArgs W,
                                                   int round) {
  int* c = counts_of(W, round);
  int* cn = counts_of(W, round + 1);
  const int n = QUEUE < 0 ? c[C_RAY] : c[C_TYPE + (QUEUE < 0 ? 0 : QUEUE)];
  const int* q = QUEUE < 0 ? W.q[round & 1] : W.tq[QUEUE < 0 ? 0 : QUEUE];
  const bool grad_pass = ADJ && W.grad_pass;
  Counters<false> cnt;
  GradSink sink;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = q[j];
    PathState P;
    load_state(W, i, P);
    const Hit h = W.hit[i];
    const float3 dl = grad_pass ? pixel_dl(A, P) : f3(0.f, 0.f, 0.f);
    bool alive = path_shade<ADJ, false, false, DISPATCH, kWfFeat<ADJ>>(A, P, h, grad_pass, dl, sink, cnt);
    if (alive && P.has_shadow) {
      store_state(W, i, P);
      push(W.sq, &c[C_SHADOW], i);
      continue;
    }
    if (alive) alive = path_finish<ADJ, false, false, kWfFeat<ADJ>>(A, P, false, grad_pass, dl, sink, cnt);
    if (alive) {
      store_state(W, i, P);
      push(W.q[(round + 1) & 1], &cn[C_RAY], i);
    } else {
      finish_sample(A, W, i, P);
    }
  }
}

// After the shadow ray: add the light sample, continue or end the path.
template <bool ADJ>
__global__ void __launch_bounds__(kBlock, kShadeMinBlocks) wf_finish(const __grid_constant__ LaunchArgs A, const __grid_constant__ WfArgs W,
                                                    int round) {
  int* c = counts_of(W, round);
  int* cn = counts_of(W, round + 1);
  const int n = c[C_SHADOW];
  const bool grad_pass = ADJ && W.grad_pass;
  Counters<false> cnt;
  GradSink sink;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = W.sq[j];
    PathState P;
    load_state(W, i, P);
    const float3 dl = grad_pass ? pixel_dl(A, P) : f3(0.f, 0.f, 0.f);
    const bool alive = path_finish<ADJ, false, false, kWfFeat<ADJ>>(A, P, W.occ[i] != 0, grad_pass, dl, sink, cnt);
    if (alive) {
      store_state(W, i, P);
      push(W.q[(round + 1) & 1], &cn[C_RAY], i);
    } else {
      finish_sample(A, W, i, P);
    }
  }
}

// Film: box filter over each pixel's consecutive samples (fixed order, no atomics).
__global__ void __launch_bounds__(kBlock) wf_film(const __grid_constant__ LaunchArgs A, const __grid_constant__ WfArgs W) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < W.n_pix; k += gridDim.x * blockDim.x) {
    float3 sum = f3(0.f, 0.f, 0.f);
    for (int s = 0; s < A.spp; ++s) {
      const float* l = &W.L[3 * ((size_t)k * A.spp + s)];
      sum = sum + f3(l[0], l[1], l[2]);
    }
    const float inv = 1.0f / (float)A.spp;
    const long long pix = W.pix0 + k;
    A.image[3 * pix] = sum.x * inv;
    A.image[3 * pix + 1] = sum.y * inv;
    A.image[3 * pix + 2] = sum.z * inv;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves the wave scratch out of the scene's buffer (grown if too small).
int wave_scratch(pt_scene* s, int cap, int rounds, WfArgs& W) {
  const size_t n = (size_t)cap;
  size_t off = 0;
  const size_t o_state = off; off += align256(n * kStateWords * 16);
  const size_t o_hit = off; off += align256(n * sizeof(Hit));
  const size_t o_occ = off; off += align256(n);
  const size_t o_L = off; off += align256(n * 12);
  const size_t o_q = off; off += align256(n * 4) * (3 + kMaterials);
  const size_t o_c = off; off += align256((size_t)(rounds + 1) * kCounts * 4);
  if (s->wf_bytes < off) {
    if (s->d_wf) cudaFree(s->d_wf);
    s->d_wf = nullptr;
    s->wf_bytes = 0;
    if (cudaMalloc(&s->d_wf, off) != cudaSuccess) {
      cudaGetLastError();
      return PT_ERR_OOM;
    }
    s->wf_bytes = off;
  }
  char* b = static_cast<char*>(s->d_wf);
  W.state = reinterpret_cast<uint4*>(b + o_state);
  W.hit = reinterpret_cast<Hit*>(b + o_hit);
  W.occ = reinterpret_cast<unsigned char*>(b + o_occ);
  W.L = reinterpret_cast<float*>(b + o_L);
  int* qs = reinterpret_cast<int*>(b + o_q);
  const size_t qstride = align256(n * 4) / 4;
  W.q[0] = qs;
  W.q[1] = qs + qstride;
  W.sq = qs + 2 * qstride;
  for (int t = 0; t < kMaterials; ++t) W.tq[t] = qs + (3 + t) * qstride;
  W.counts = reinterpret_cast<int*>(b + o_c);
  W.cap = cap;
  return PT_OK;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
  }
  return n;
}

// One pass of the wavefront loop over one wave.
template <bool ADJ, int LAYOUT>
void run_rounds(const LaunchArgs& A, const WfArgs& W, int mode, int grid, cudaStream_t cs) {
  const dim3 gd(grid), bd(kBlock);
  wf_start<ADJ><<<gd, bd, 0, cs>>>(A, W);
  for (int r = 0; r < A.max_depth; ++r) {
    if (mode == PT_WF_GROUPED) {
      wf_trace<LAYOUT, false, true><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_SWITCH, 0><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_FIXED + PT_BSDF_DIFFUSE, PT_BSDF_DIFFUSE><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_FIXED + PT_BSDF_CONDUCTOR, PT_BSDF_CONDUCTOR><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_FIXED + PT_BSDF_DIELECTRIC, PT_BSDF_DIELECTRIC><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_FIXED + PT_BSDF_BLEND, PT_BSDF_BLEND><<<gd, bd, 0, cs>>>(A, W, r);
    } else {
      wf_trace<LAYOUT, false, false><<<gd, bd, 0, cs>>>(A, W, r);
      wf_shade<ADJ, PT_DISPATCH_SWITCH, -1><<<gd, bd, 0, cs>>>(A, W, r);
    }
    wf_trace<LAYOUT, true, false><<<gd, bd, 0, cs>>>(A, W, r);
    wf_finish<ADJ><<<gd, bd, 0, cs>>>(A, W, r);
  }
}

template <bool ADJ>
int run_wavefront(pt_scene* s, const LaunchArgs& A, const pt_wavefront_opts* o, cudaStream_t cs) {
  const int mode = o ? o->calls : PT_WF_TRACED;
  if (mode != PT_WF_TRACED && mode != PT_WF_GROUPED) return PT_ERR_ARG;
  long long want = (o && o->wave_paths > 0) ? o->wave_paths : (4ll << 20);
  if (want > (1ll << 28)) return PT_ERR_ARG;
  const long long n_pix = (long long)A.n_cams * A.crop_w * A.crop_h;
  long long pix_per_wave = std::max(1ll, want / A.spp);
  pix_per_wave = std::min(pix_per_wave, n_pix);
  const int cap = (int)(pix_per_wave * A.spp);
  WfArgs W;
  std::memset(&W, 0, sizeof W);
  int st = wave_scratch(s, cap, A.max_depth, W);
  if (st != PT_OK) return st;
  const int grid = (int)std::min<long long>((cap + kBlock - 1) / kBlock, 8ll * sm_count());
  const size_t counts_bytes = (size_t)(A.max_depth + 1) * kCounts * 4;
  for (long long p0 = 0; p0 < n_pix; p0 += pix_per_wave) {
    W.pix0 = p0;
    W.n_pix = (int)std::min(pix_per_wave, n_pix - p0);
    for (int pass = 0; pass < (ADJ ? 2 : 1); ++pass) {
      W.grad_pass = pass;
      if (cudaMemsetAsync(W.counts, 0, counts_bytes, cs) != cudaSuccess) return PT_ERR_CUDA;
      if (A.scene.layout == PT_BVH_WIDE) run_rounds<ADJ, PT_BVH_WIDE>(A, W, mode, grid, cs);
      else run_rounds<ADJ, PT_BVH_BINARY>(A, W, mode, grid, cs);
    }
    if (!ADJ) wf_film<<<std::max(1, std::min(grid, (W.n_pix + kBlock - 1) / kBlock)), kBlock, 0, cs>>>(A, W);
  }
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

}  // namespace
}  // namespace ptgb

using namespace ptgb;

extern "C" int pt_wavefront_forward(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                    const pt_wavefront_opts* o, float* image, void* stream) {
  LaunchArgs A;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (!image || r->cache || r->counters) return PT_ERR_ARG;
  A.image = image;
  return run_wavefront<false>(s, A, o, (cudaStream_t)stream);
}

extern "C" int pt_wavefront_backward(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                     const pt_wavefront_opts* o, const float* grad_image, const pt_grads* g,
                                     void* stream) {
  LaunchArgs A;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (!grad_image || !g || r->cache || r->counters || r->dbg_sample_L || r->dbg_sample_hash) return PT_ERR_ARG;
  A.grad_image = grad_image;
  A.grads.albedo = g->albedo;
  A.grads.rough = g->roughness;
  for (int t = 0; t < PT_MAX_TEX; ++t) A.grads.tex[t] = reinterpret_cast<float4*>(g->tex[t]);
  if (g->env && s->dev.env_w <= 0) return PT_ERR_ARG;
  A.grads.env = reinterpret_cast<float4*>(g->env);
  A.grads.n_albedo = p->n_albedo;
  A.grads.n_rough = p->n_rough;
  return run_wavefront<true>(s, A, o, (cudaStream_t)stream);
}
