// The path-tracing megakernel (forward, forward mode, fused PRB adjoint, and the
// forward pass that writes reverse-mode checkpoints), its launch bounds and the
// mapping from thread units to pixels.  Shared by the render, batch and
// checkpoint translation units.
#pragma once

#include "pt_path.cuh"

namespace ptgb {

template <bool INSTR>
__device__ __forceinline__ void flush_counters(const LaunchArgs& A, Counters<INSTR>& cnt) {
  if constexpr (INSTR) {
    if (A.counters) {
#pragma unroll
      for (int i = 0; i < kCounters; ++i) {
        unsigned long long v = cnt.c[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane_id() == 0 && v) atomicAdd(&A.counters[i], v);
      }
    }
  }
}

struct PixelOf {
  int cam, px, py;
  long long pix;  // dense index of the pixel in the output image
};
// A rectangle of pixels (of n_cams cameras) processed by one launch or one work item.
struct Tile {
  int x0, y0, w, h, n_cams;
};
// Pixel of `unit` (pixel-major, lanes_per_pixel consecutive units per pixel) inside
// the tile; false if the unit lies outside the tile or outside the image crop.
__device__ __forceinline__ bool unit_pixel(const LaunchArgs& A, long long unit, const Tile& t, PixelOf& r) {
  const long long pix = unit >> A.log2_lanes;
  const long long per_cam = (long long)t.w * t.h;
  if (unit < 0 || pix >= per_cam * t.n_cams) return false;
  r.cam = (int)(pix / per_cam);
  const long long rem = pix - (long long)r.cam * per_cam;
  const int iy = (int)(rem / t.w);
  const int ix = (int)(rem - (long long)iy * t.w);
  r.px = t.x0 + ix;
  r.py = t.y0 + iy;
  if (r.px >= A.crop_x0 + A.crop_w || r.py >= A.crop_y0 + A.crop_h) return false;
  r.pix = ((long long)r.cam * A.crop_h + (r.py - A.crop_y0)) * A.crop_w + (r.px - A.crop_x0);
  return true;
}

// The megakernel: forward (ADJ = false) or fused PRB adjoint (ADJ = true).
// Each thread owns the samples s = lane_in_pixel + k * lanes_per_pixel of one
// pixel; in the adjoint every sample is traced twice (pass 0: radiance L,
// pass 1: replay with L_rem and gradient scatter) by the same code.
// The loop state at the start of path vertex k (before its closest-hit ray),
// enough to recompute the vertex: PCG32 state, ray, throughput, MIS state, depth.
// Checkpoint k of sample `slot` is words [k][0..3][slot] (word-major: the lanes of
// a warp store neighbouring slots).
__device__ __forceinline__ void store_checkpoint(const LaunchArgs& A, const PathState& P) {
  const size_t k = (size_t)(P.depth - 1);
  const size_t n = (size_t)A.ck_slots;
  uint4* dst = A.ck_state + k * 4 * n + P.slot;
  dst[0] = make_uint4((uint32_t)P.rng.state, (uint32_t)(P.rng.state >> 32), (uint32_t)P.rng.inc,
                      (uint32_t)(P.rng.inc >> 32));
  dst[n] = make_uint4(__float_as_uint(P.ro.x), __float_as_uint(P.ro.y), __float_as_uint(P.ro.z),
                      __float_as_uint(P.rd.x));
  dst[2 * n] = make_uint4(__float_as_uint(P.rd.y), __float_as_uint(P.rd.z), __float_as_uint(P.beta.x),
                          __float_as_uint(P.beta.y));
  dst[3 * n] = make_uint4(__float_as_uint(P.beta.z), __float_as_uint(P.prev_pdf),
                          (uint32_t)P.depth | (P.prev_delta ? 0x80000000u : 0u), 0u);
}

__device__ __forceinline__ void load_checkpoint(const LaunchArgs& A, long long slot, int k, PathState& P) {
  const size_t n = (size_t)A.ck_slots;
  const uint4* src = A.ck_state + (size_t)k * 4 * n + slot;
  const uint4 w0 = src[0], w1 = src[n], w2 = src[2 * n], w3 = src[3 * n];
  P.rng.state = (unsigned long long)w0.x | ((unsigned long long)w0.y << 32);
  P.rng.inc = (unsigned long long)w0.z | ((unsigned long long)w0.w << 32);
  P.ro = f3(__uint_as_float(w1.x), __uint_as_float(w1.y), __uint_as_float(w1.z));
  P.rd = f3(__uint_as_float(w1.w), __uint_as_float(w2.x), __uint_as_float(w2.y));
  P.beta = f3(__uint_as_float(w2.z), __uint_as_float(w2.w), __uint_as_float(w3.x));
  P.prev_pdf = __uint_as_float(w3.y);
  P.depth = (int)(w3.z & 0x7fffffffu);
  P.prev_delta = (w3.z >> 31) != 0u;
  P.slot = slot;
  P.cache_done = false;
  P.fh.h = 0u;
  P.L = f3(0.f, 0.f, 0.f);
  P.Lrem = f3(0.f, 0.f, 0.f);
}

// dLoss/dI of a pixel divided by spp (the adjoint's per-sample weight).
__device__ __forceinline__ float3 pixel_dl(const LaunchArgs& A, long long pix) {
  const float inv = 1.0f / (float)A.spp;
  if (A.target) {  // batched jobs: L2 loss against the job's target
    const float k = 2.0f * A.loss_scale * inv;
    return f3((A.image[3 * pix] - A.target[3 * pix]) * k, (A.image[3 * pix + 1] - A.target[3 * pix + 1]) * k,
              (A.image[3 * pix + 2] - A.target[3 * pix + 2]) * k);
  }
  return f3(A.grad_image[3 * pix] * inv, A.grad_image[3 * pix + 1] * inv, A.grad_image[3 * pix + 2] * inv);
}

// Film of a persistent launch: a unit's sample sum goes straight to its pixel with
// one lane per pixel, else it is added to the (zeroed) image with float atomics.
template <bool JVP>
__device__ __forceinline__ void film_unit(const LaunchArgs& A, long long pix, float3 sum, float3 sum_dot) {
  const float inv = 1.0f / (float)A.spp;
  float* im = A.image + 3 * pix;
  if (A.lanes_per_pixel == 1) {
    im[0] = sum.x * inv;
    im[1] = sum.y * inv;
    im[2] = sum.z * inv;
  } else {
    atomicAdd(im, sum.x * inv);
    atomicAdd(im + 1, sum.y * inv);
    atomicAdd(im + 2, sum.z * inv);
  }
  if constexpr (JVP) {
    float* d = A.image_dot + 3 * pix;
    if (A.lanes_per_pixel == 1) {
      d[0] = sum_dot.x * inv;
      d[1] = sum_dot.y * inv;
      d[2] = sum_dot.z * inv;
    } else {
      atomicAdd(d, sum_dot.x * inv);
      atomicAdd(d + 1, sum_dot.y * inv);
      atomicAdd(d + 2, sum_dot.z * inv);
    }
  }
}

// FEAT_CKPT (forward only): store a checkpoint before every closest-hit ray and
// the vertex count of every sample (reverse mode with checkpoints, Sec. 4.10).
// PERSIST: the thread is one lane of a persistent grid: `unit` is ignored, and a
// lane whose unit has no samples left takes the next unit from the launch's work
// counter A.queue (one atomic per warp for all lanes that need one, so a warp's
// new units are consecutive: neighbouring samples of the same pixels), until the
// counter passes A.n_units.  Lanes never wait for the slowest unit of their warp
// or block, only for the last units of the launch.
template <bool ADJ, bool JVP, bool INSTR, int LAYOUT, int DISPATCH, int FEAT = 0, bool PERSIST = false>
__device__ __forceinline__ void megakernel(const LaunchArgs& A, long long unit, const Tile& tile) {
  constexpr bool CKPT = (FEAT & FEAT_CKPT) != 0;
  PixelOf px{};
  bool valid = PERSIST ? false : unit_pixel(A, unit, tile, px);
  Counters<INSTR> cnt;
  if constexpr (INSTR) {
    for (int i = 0; i < kCounters; ++i) cnt.c[i] = 0;
  }
  GradSink sink;
  int lane_in_pix = (int)(unit & (A.lanes_per_pixel - 1));
  float3 dl = f3(0.f, 0.f, 0.f);
  if constexpr (ADJ && !PERSIST) {
    if (valid) dl = pixel_dl(A, px.pix);
  }
  float3 pix_sum = f3(0.f, 0.f, 0.f);
  float3 pix_sum_dot = f3(0.f, 0.f, 0.f);
  float3 L_pass0 = f3(0.f, 0.f, 0.f);
  int next_s = lane_in_pix;
  // FEAT_REPLAY: every sample is replayed once from the radiance the forward stored
  constexpr bool REPLAY = ADJ && (FEAT & FEAT_REPLAY) != 0;
  constexpr bool FILM = !ADJ && (FEAT & FEAT_SAMPLE_L) == 0;
  int pass = REPLAY ? 1 : 0;
  bool has_path = false;
  bool want_shadow = false;  // the lane's next traversal is its pending shadow ray
  bool retired = !PERSIST;   // persistent lanes: the work counter has run out
  PathState P;
  for (;;) {
    if constexpr (PERSIST) {
      const bool need = !has_path && !retired && !(valid && next_s < A.spp);
      if (FILM && need && valid && A.image) film_unit<JVP>(A, px.pix, pix_sum, pix_sum_dot);
      const unsigned m = __ballot_sync(0xffffffffu, need);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane_id() == leader) base = atomicAdd(A.queue, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) {
          unit = (long long)(base + (unsigned long long)__popc(m & ((1u << lane_id()) - 1u)));
          valid = false;
          if (unit >= A.n_units) {
            retired = true;
          } else {
            valid = unit_pixel(A, unit, tile, px);
            lane_in_pix = (int)(unit & (A.lanes_per_pixel - 1));
            next_s = lane_in_pix;
            pix_sum = pix_sum_dot = L_pass0 = f3(0.f, 0.f, 0.f);
            pass = REPLAY ? 1 : 0;
            if constexpr (ADJ) {
              if (valid) dl = pixel_dl(A, px.pix);
            }
          }
        }
      }
    }
    if (!has_path && valid && next_s < A.spp) {
      // one call site for both passes: the replay starts from identical code
      // the split-PRB radiance pass traces the adjoint's samples
      path_start<INSTR>(A, P, (ADJ || (FEAT & FEAT_SAMPLE_L)) ? A.seed_adj : A.seed, px.cam, px.px, px.py, next_s,
                        px.pix, cnt);
      if constexpr (REPLAY) {
        const float* l = A.sample_L + 3 * P.slot;
        P.Lrem = f3(l[0], l[1], l[2]);
      } else if constexpr (ADJ) {
        P.Lrem = L_pass0;
      }
      has_path = true;
      want_shadow = false;
    }
    if (!__any_sync(0xffffffffu, has_path || !retired)) break;
    if constexpr (INSTR) {
      if (lane_id() == 0) cnt.add(15, 1);
    }
    if (has_path) {
      // one traversal per lane per iteration: its path ray or its shadow ray
      cnt.add(want_shadow ? 2 : 1, 1);
      const float3 o = want_shadow ? P.so : P.ro, d = want_shadow ? P.sd : P.rd;
      const float tmax = want_shadow ? P.stmax : INFINITY;
      if constexpr (CKPT) {
        if (!want_shadow) store_checkpoint(A, P);
      }
      const Hit hit = LAYOUT == PT_BVH_WIDE ? trace_wide<INSTR>(A.scene, o, d, tmax, want_shadow, cnt)
                                            : trace_binary<INSTR>(A.scene, o, d, tmax, want_shadow, cnt);
      const bool grad_pass = ADJ && pass == 1;
      bool alive = true, finish = true, occ = false;
      if (!want_shadow) {
        alive = path_shade<ADJ, JVP, INSTR, DISPATCH, FEAT>(A, P, hit, grad_pass, dl, sink, cnt);
        finish = alive && !P.has_shadow;
        want_shadow = alive && P.has_shadow;
      } else {
        occ = hit.pos >= 0;
        want_shadow = false;
      }
      if (finish) {
        if constexpr (ADJ) alive = path_finish_body<ADJ, JVP, INSTR, FEAT>(A, P, occ, grad_pass, dl, sink, cnt);
        else alive = path_finish<ADJ, JVP, INSTR, FEAT>(A, P, occ, grad_pass, dl, sink, cnt);
      }
      if (!alive) {
        has_path = false;
        if constexpr (CKPT) A.ck_count[P.slot] = P.depth;
        if constexpr (!ADJ && (FEAT & FEAT_CACHE) != 0) {
          if (A.cache_mode == 1 && !P.cache_done) {  // no cache query for this sample
            float* r = A.q_raw + P.slot * 10;
#pragma unroll
            for (int k = 0; k < 10; ++k) r[k] = 0.0f;
            float* b = A.q_beta + P.slot * 3;
            b[0] = b[1] = b[2] = 0.0f;
          } else if (A.cache_mode == 3) {
            float* pl = A.path_L + P.slot * 3;
            pl[0] = P.L.x;
            pl[1] = P.L.y;
            pl[2] = P.L.z;
          }
        }
        if constexpr (!ADJ && (FEAT & FEAT_SAMPLE_L) != 0) {
          float* l = A.sample_L + 3 * P.slot;
          l[0] = P.L.x;
          l[1] = P.L.y;
          l[2] = P.L.z;
        }
        if (ADJ && !REPLAY && pass == 0) {
          L_pass0 = P.L;  // replay the same sample next: L_rem starts from its radiance
          pass = 1;
        } else {
          pix_sum = pix_sum + P.L;
          if (JVP) pix_sum_dot = pix_sum_dot + P.L_dot;
          if constexpr (INSTR && !ADJ) {
            const long long si = px.pix * A.spp + next_s;
            if (A.dbg_L) {
              A.dbg_L[3 * si] = P.L.x;
              A.dbg_L[3 * si + 1] = P.L.y;
              A.dbg_L[3 * si + 2] = P.L.z;
            }
            if (A.dbg_hash) A.dbg_hash[si] = P.fh.h;
          }
          next_s += A.lanes_per_pixel;
          pass = REPLAY ? 1 : 0;
          L_pass0 = f3(0.f, 0.f, 0.f);
        }
      }
    }
  }
  if constexpr (!ADJ && !PERSIST) {
    for (int off = 1; off < A.lanes_per_pixel; off <<= 1) {
      pix_sum.x += __shfl_xor_sync(0xffffffffu, pix_sum.x, off);
      pix_sum.y += __shfl_xor_sync(0xffffffffu, pix_sum.y, off);
      pix_sum.z += __shfl_xor_sync(0xffffffffu, pix_sum.z, off);
    }
    if constexpr (JVP) {
      for (int off = 1; off < A.lanes_per_pixel; off <<= 1) {
        pix_sum_dot.x += __shfl_xor_sync(0xffffffffu, pix_sum_dot.x, off);
        pix_sum_dot.y += __shfl_xor_sync(0xffffffffu, pix_sum_dot.y, off);
        pix_sum_dot.z += __shfl_xor_sync(0xffffffffu, pix_sum_dot.z, off);
      }
    }
    if (valid && lane_in_pix == 0 && A.image && (FEAT & FEAT_SAMPLE_L) == 0) {
      const float inv = 1.0f / (float)A.spp;
      A.image[3 * px.pix] = pix_sum.x * inv;
      A.image[3 * px.pix + 1] = pix_sum.y * inv;
      A.image[3 * px.pix + 2] = pix_sum.z * inv;
      if (JVP) {
        A.image_dot[3 * px.pix] = pix_sum_dot.x * inv;
        A.image_dot[3 * px.pix + 1] = pix_sum_dot.y * inv;
        A.image_dot[3 * px.pix + 2] = pix_sum_dot.z * inv;
      }
    }
  }
  flush_counters<INSTR>(A, cnt);
}

// Minimum resident CTAs of 256 threads per SM requested from ptxas (register cap).
// Measured on the 196k-triangle sphere workload (forward + adjoint step): with the
// per-vertex shading out of line, more resident warps beat fewer spills -- the
// forward runs best at 5 CTAs (48 registers: 45.6 ms; 46.4 at 64, 62 at 128) once
// the production instances carry no fingerprint or adjoint-only state, the fused
// adjoint at 3 (80 registers; the batched kernels measured 381 ms there, 387 at 64).
// With the shorter node visit (one FMA per box plane, a hit mask per node) the forward
// still prefers 5 CTAs (37.3 ms; 38.1 at 64 registers, 39.9 at 40), while the split-PRB
// replay and the forward-mode kernel moved to 4 (their own caps in pt_render.cu).
// With two box planes per packed FMA the forward and the radiance pass run best at 56
// registers (36.0 ms each; 36.5 at 48, 37.1 at 64), a cap that no CTA count of 256
// threads gives, so those kernels take it directly (PT_FWD_REGS, any block size up to
// 256 threads); so does the checkpointed forward (38.6 ms against 39.3 at 48).
#ifndef PT_LB_THREADS
#define PT_LB_THREADS 256  // block size the replay register cap is computed for
#endif
#ifndef PT_FWD_REGS
#define PT_FWD_REGS 56
#endif
#define PT_FWD_BOUNDS __maxnreg__(PT_FWD_REGS)
// The batched forward keeps 64 registers (measured there).
#ifndef PT_OTHER_FWD_MIN_BLOCKS
#define PT_OTHER_FWD_MIN_BLOCKS 4
#endif
#ifndef PT_ADJ_MIN_BLOCKS
#define PT_ADJ_MIN_BLOCKS 3
#endif

__device__ __forceinline__ Tile crop_tile(const LaunchArgs& A) {
  return Tile{A.crop_x0, A.crop_y0, A.crop_w, A.crop_h, A.n_cams};
}

}  // namespace ptgb
