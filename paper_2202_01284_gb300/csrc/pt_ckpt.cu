// Reverse-mode differentiation of the path tracer with checkpoints (Sec. 4.10, the
// comparison of PRB with differentiating a standard path tracer whose loop keeps
// one checkpoint per scattering event; Sec. 4.3 on loops).
//
// Forward: the megakernel stores the loop state at the start of every path vertex
// (pt_ckpt_forward).  Reverse: each sample's vertices are recomputed from their
// checkpoints in reverse order; the radiance S arriving from the later vertices is
// known when vertex k is processed, so the gradient terms are
//   dL * (C_nee * (df_nee/dθ)/f_nee + S * (df_bsdf/dθ)/f_bsdf)
// -- the same estimator as PRB (whose L_rem equals S) without PRB's extra pass
// that recomputes the path radiance, at the price of 64 B of checkpoint per vertex.
#include <algorithm>
#include <cstring>

#include "pt_mega.cuh"

struct pt_ckpt {
  uint4* d_state = nullptr;  // [max_depth][4][max_samples]
  int* d_count = nullptr;    // [max_samples]
  long long max_samples = 0;
  int max_depth = 0;
  long long bytes = 0;
};

namespace ptgb {
namespace {

template <int LAYOUT>
// the plain forward's cap (48 registers: 39.9 ms against 40.6 at 64)
__global__ void PT_FWD_BOUNDS ckpt_forward_kernel(const __grid_constant__ LaunchArgs A) {
  megakernel<false, false, false, LAYOUT, PT_DISPATCH_SWITCH, FEAT_CKPT>(
      A, (long long)blockIdx.x * blockDim.x + threadIdx.x, crop_tile(A));
}

// Finish vertex k of the reverse sweep and fold its radiance into S.
template <int FEAT>
__device__ __forceinline__ void reverse_finish(const LaunchArgs& A, PathState& P, bool alive, bool occluded,
                                               float3& S, float3 dl, GradSink& sink, Counters<false>& cnt) {
  if (alive) {
    const bool lit = P.has_shadow && !occluded;
    // radiance that flows through this vertex's sampled direction: everything the
    // later vertices contributed (path_finish removes the light sample again)
    P.Lrem = (lit ? P.c_nee : f3(0.f, 0.f, 0.f)) + S;
    path_finish<true, false, false, FEAT>(A, P, occluded, true, dl, sink, cnt);
  }
  S = S + P.L;  // this vertex's own emission and light sample
}

// One thread per (pixel, sample subset) as the megakernel; each sample's vertices
// are processed last to first, one traversal per lane per loop iteration.
template <int LAYOUT, bool EGRAD>
__global__ void __launch_bounds__(256, PT_ADJ_MIN_BLOCKS) ckpt_reverse_kernel(const __grid_constant__ LaunchArgs A) {
  constexpr int FEAT = FEAT_TEXAGG | (EGRAD ? FEAT_EGRAD : 0);
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PixelOf px{};
  const bool valid = unit_pixel(A, unit, crop_tile(A), px);
  Counters<false> cnt;
  GradSink sink;
  const int lane_in_pix = (int)(unit & (A.lanes_per_pixel - 1));
  float3 dl = f3(0.f, 0.f, 0.f);
  if (valid) {
    const float inv = 1.0f / (float)A.spp;
    dl = f3(A.grad_image[3 * px.pix] * inv, A.grad_image[3 * px.pix + 1] * inv, A.grad_image[3 * px.pix + 2] * inv);
  }
  int next_s = lane_in_pix;
  int k = -1;  // vertex being processed (-1: none)
  long long slot = 0;
  bool want_shadow = false;
  float3 S = f3(0.f, 0.f, 0.f);
  PathState P;
  for (;;) {
    while (k < 0 && valid && next_s < A.spp) {
      slot = px.pix * A.spp + next_s;
      next_s += A.lanes_per_pixel;
      k = min(A.ck_count[slot], A.max_depth) - 1;  // clamped: never past the stored vertices
      S = f3(0.f, 0.f, 0.f);
      want_shadow = false;
    }
    const bool active = k >= 0;
    if (!__any_sync(0xffffffffu, active)) break;
    if (!active) continue;
    if (!want_shadow) {
      load_checkpoint(A, slot, k, P);
      const Hit hit = LAYOUT == PT_BVH_WIDE ? trace_wide<false>(A.scene, P.ro, P.rd, INFINITY, false, cnt)
                                            : trace_binary<false>(A.scene, P.ro, P.rd, INFINITY, false, cnt);
      const bool alive = path_shade<true, false, false, PT_DISPATCH_SWITCH, FEAT>(A, P, hit, true, dl, sink, cnt);
      if (alive && P.has_shadow) {
        want_shadow = true;
      } else {
        reverse_finish<FEAT>(A, P, alive, false, S, dl, sink, cnt);
        --k;
      }
    } else {
      const Hit hit = LAYOUT == PT_BVH_WIDE ? trace_wide<false>(A.scene, P.so, P.sd, P.stmax, true, cnt)
                                            : trace_binary<false>(A.scene, P.so, P.sd, P.stmax, true, cnt);
      want_shadow = false;
      reverse_finish<FEAT>(A, P, true, hit.pos >= 0, S, dl, sink, cnt);
      --k;
    }
  }
}

// Launch arguments shared by the two entry points: the checkpoint buffers must
// hold this launch's samples and depth.
int ckpt_args(pt_scene* s, const pt_render_desc* r, const pt_params* p, pt_ckpt* ck, LaunchArgs& A) {
  if (!ck) return PT_ERR_ARG;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (r->cache || r->counters || r->dbg_sample_L || r->dbg_sample_hash) return PT_ERR_ARG;
  const long long slots = (long long)A.n_cams * A.crop_w * A.crop_h * A.spp;
  if (slots > ck->max_samples || A.max_depth > ck->max_depth) return PT_ERR_ARG;
  A.ck_state = ck->d_state;
  A.ck_count = ck->d_count;
  A.ck_slots = ck->max_samples;
  return PT_OK;
}

}  // namespace
}  // namespace ptgb

using namespace ptgb;

extern "C" int pt_ckpt_create(int64_t max_samples, int32_t max_depth, pt_ckpt** out) {
  if (!out || max_samples < 1 || max_depth < 1 || max_depth > 1024) return PT_ERR_ARG;
  *out = nullptr;
  pt_ckpt* ck = new (std::nothrow) pt_ckpt();
  if (!ck) return PT_ERR_OOM;
  ck->max_samples = max_samples;
  ck->max_depth = max_depth;
  const size_t state = (size_t)max_samples * (size_t)max_depth * 4 * sizeof(uint4);
  const size_t count = (size_t)max_samples * sizeof(int);
  if (cudaMalloc(&ck->d_state, state) != cudaSuccess || cudaMalloc(&ck->d_count, count) != cudaSuccess) {
    cudaGetLastError();
    if (ck->d_state) cudaFree(ck->d_state);
    delete ck;
    return PT_ERR_OOM;
  }
  if (cudaMemset(ck->d_count, 0, count) != cudaSuccess) {
    cudaFree(ck->d_state);
    cudaFree(ck->d_count);
    delete ck;
    return PT_ERR_CUDA;
  }
  ck->bytes = (long long)(state + count);
  *out = ck;
  return PT_OK;
}

extern "C" void pt_ckpt_destroy(pt_ckpt* ck) {
  if (!ck) return;
  cudaFree(ck->d_state);
  cudaFree(ck->d_count);
  delete ck;
}

extern "C" int pt_ckpt_bytes(const pt_ckpt* ck, int64_t* bytes) {
  if (!ck || !bytes) return PT_ERR_ARG;
  *bytes = ck->bytes;
  return PT_OK;
}

extern "C" int pt_ckpt_forward(pt_scene* s, const pt_render_desc* r, const pt_params* p, pt_ckpt* ck, float* image,
                               void* stream) {
  LaunchArgs A;
  int st = ckpt_args(s, r, p, ck, A);
  if (st != PT_OK) return st;
  if (!image) return PT_ERR_ARG;
  A.image = image;
  int block;
  long long grid;
  if ((st = launch_dims(r, A, block, grid)) != PT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  if (s->dev.layout == PT_BVH_WIDE) ckpt_forward_kernel<PT_BVH_WIDE><<<(unsigned)grid, block, 0, cs>>>(A);
  else ckpt_forward_kernel<PT_BVH_BINARY><<<(unsigned)grid, block, 0, cs>>>(A);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_ckpt_backward(pt_scene* s, const pt_render_desc* r, const pt_params* p, pt_ckpt* ck,
                                const float* grad_image, const pt_grads* g, void* stream) {
  LaunchArgs A;
  int st = ckpt_args(s, r, p, ck, A);
  if (st != PT_OK) return st;
  if (!grad_image || !g) return PT_ERR_ARG;
  A.grad_image = grad_image;
  A.grads.albedo = g->albedo;
  A.grads.rough = g->roughness;
  for (int t = 0; t < PT_MAX_TEX; ++t) A.grads.tex[t] = reinterpret_cast<float4*>(g->tex[t]);
  if (g->env && s->dev.env_w <= 0) return PT_ERR_ARG;
  A.grads.env = reinterpret_cast<float4*>(g->env);
  A.grads.n_albedo = p->n_albedo;
  A.grads.n_rough = p->n_rough;
  int block;
  long long grid;
  if ((st = launch_dims(r, A, block, grid)) != PT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const dim3 gd((unsigned)grid), bd(block);
  if (s->dev.layout == PT_BVH_WIDE) {
    if (A.grads.env) ckpt_reverse_kernel<PT_BVH_WIDE, true><<<gd, bd, 0, cs>>>(A);
    else ckpt_reverse_kernel<PT_BVH_WIDE, false><<<gd, bd, 0, cs>>>(A);
  } else {
    if (A.grads.env) ckpt_reverse_kernel<PT_BVH_BINARY, true><<<gd, bd, 0, cs>>>(A);
    else ckpt_reverse_kernel<PT_BVH_BINARY, false><<<gd, bd, 0, cs>>>(A);
  }
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
