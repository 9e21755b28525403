// Per-path device code shared by the megakernels and the wavefront kernels:
// the path state, camera-ray start, the shading step after a closest hit and
// the finishing step after the (optional) shadow ray, plus the gradient sink.
#pragma once

#include "pt_device.cuh"

namespace ptgb {

// Optional features compiled into an instantiation of the per-vertex code (each
// costs the production kernels instruction-cache space when compiled in):
// environment-radiance gradients, radiance-cache modes, warp-aggregated texel
// atomics, reverse-mode checkpoints; split PRB: the forward writes each sample's
// radiance, the adjoint replays only (no radiance pass of its own).
enum : int {
  FEAT_EGRAD = 1, FEAT_CACHE = 2, FEAT_TEXAGG = 4, FEAT_CKPT = 8, FEAT_SAMPLE_L = 16, FEAT_REPLAY = 32,
  FEAT_NOHASH = 64,  // no decision fingerprint (instances that never output it)
  FEAT_LEAN = 128,   // production megakernel instances: no remaining radiance outside the
                     // adjoint, the continuation ray written straight into the path's ray
  FEAT_ALL = 7
};

// Linkage of the per-vertex steps below (experiments build them inline).
#ifdef PT_SHADE_INLINE
#define PT_SHADE_FN __forceinline__
#else
#define PT_SHADE_FN __noinline__
#endif
#ifdef PT_FINISH_INLINE
#define PT_FINISH_FN __forceinline__
#else
#define PT_FINISH_FN PT_SHADE_FN
#endif

// Per-vertex gradient sink of the adjoint: warp-aggregated atomics.
// Constant-albedo rows and roughness entries are few and heavily shared, so the
// lanes of a warp that hit the same entry are reduced with a shuffle tree and one
// lane issues the atomic; texels are many and rarely shared, so aggregation is
// optional for them.  (No per-CTA shared-memory staging: its end-of-CTA barrier
// kept finished warps resident and cost more than the atomics it saved.)
struct GradSink {
  template <bool INSTR, bool TEXAGG>
  __device__ __forceinline__ void add(const LaunchArgs& A, const Material& m, float3 g_alb, float g_alpha,
                                      Counters<INSTR>& cnt) {
    const DevGrads& G = A.grads;
    if (m.alb_kind == 2) {
      float4* dst = G.tex[m.tex];
      if (dst) {
        cnt.add(7, 1);
        cnt.add(13, 1);
        if (TEXAGG && A.tex_aggregate) {
          float v[3] = {g_alb.x, g_alb.y, g_alb.z};
          unsigned long long key = ((unsigned long long)m.tex << 32) | (unsigned)m.alb_ref;
          unsigned active = __activemask();
          unsigned peers = __match_any_sync(active, key);
          int lane = lane_id();
          int n = __popc(peers);
          int rank = __popc(peers & ((1u << lane) - 1u));
          int maxn = __reduce_max_sync(active, (unsigned)n);
          for (int s = 1; s < maxn; s <<= 1) {
            int src_rank = rank + s;
            int src = src_rank < n ? nth_set_bit(peers, src_rank) : lane;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              float x = __shfl_sync(active, v[k], src);
              if ((rank & (2 * s - 1)) == 0 && src_rank < n) v[k] += x;
            }
          }
          if (rank == 0) {
            atomicAdd(&dst[m.alb_ref], make_float4(v[0], v[1], v[2], 0.0f));
            cnt.add(6, 1);
          }
        } else {
          atomicAdd(&dst[m.alb_ref], make_float4(g_alb.x, g_alb.y, g_alb.z, 0.0f));
          cnt.add(6, 1);
        }
      }
    } else if (m.alb_kind == 1 && G.albedo) {
      cnt.add(7, 1);
      float v[3] = {g_alb.x, g_alb.y, g_alb.z};
      if (warp_aggregate<3>((unsigned)m.alb_ref, v)) {
        atomicAdd(&G.albedo[3 * m.alb_ref + 0], v[0]);
        atomicAdd(&G.albedo[3 * m.alb_ref + 1], v[1]);
        atomicAdd(&G.albedo[3 * m.alb_ref + 2], v[2]);
        cnt.add(6, 1);
      }
    }
    if (m.rough >= 0 && G.rough && (m.type == PT_BSDF_CONDUCTOR || m.type == PT_BSDF_BLEND)) {
      cnt.add(7, 1);
      float v[1] = {g_alpha};
      if (warp_aggregate<1>((unsigned)m.rough, v)) {
        atomicAdd(&G.rough[m.rough], v[0]);
        cnt.add(6, 1);
      }
    }
  }
  // Environment radiance of pixel `idx` (emitter gradient): warp-aggregated, as
  // coherent rays escape through the same pixel of a coarse map.
  template <bool INSTR>
  __device__ __forceinline__ void add_env(const LaunchArgs& A, int idx, float3 g, Counters<INSTR>& cnt) {
    cnt.add(7, 1);
    float v[3] = {g.x, g.y, g.z};
    if (warp_aggregate<3>((unsigned)idx, v)) {
      atomicAdd(&A.grads.env[idx], make_float4(v[0], v[1], v[2], 0.0f));
      cnt.add(6, 1);
    }
  }
};

// Both log-derivative factors of one BSDF value, (df_alb / f, df_alpha / f) per
// channel, from one reciprocal of f (0 where f is 0).
__device__ __forceinline__ void log_derivs(float3 df_alb, float3 df_alpha, float3 f, float3& r_alb, float3& r_a) {
  const float3 inv = f3(f.x > 0.0f ? 1.0f / f.x : 0.0f, f.y > 0.0f ? 1.0f / f.y : 0.0f,
                        f.z > 0.0f ? 1.0f / f.z : 0.0f);
  r_alb = df_alb * inv;
  r_a = df_alpha * inv;
}

__device__ __forceinline__ float3 offset_origin(float3 p, float3 ng, float3 d) {
  float eps = 1e-4f * fmaxf(1.0f, fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))));
  return p + ng * (dot3(ng, d) >= 0.0f ? eps : -eps);
}

// State of one lane's current path.  The megakernel loop below advances every
// lane by one path vertex per iteration (closest hit -> shading + light sample +
// BSDF sample -> shadow ray -> finish), and a lane whose path ended starts its
// next sample in the same iteration ("path regeneration"), so the warp keeps
// traversing together instead of waiting for its longest path.
struct PathState {
  Pcg32 rng;
  float3 ro, rd;      // current ray
  float3 beta, L, Lrem;
  float prev_pdf;
  int depth;
  bool prev_delta;
  Fnv fh;
  // ---- pending vertex (between the shading step and the shadow ray)
  float3 so, sd;      // shadow ray
  float stmax;
  float3 c_nee;       // NEE contribution if unoccluded
  float3 r_nee_alb, r_bsdf_alb;  // (df/dalbedo)/f per channel (NEE / sampled direction)
  float3 r_nee_a, r_bsdf_a;      // (df/dalpha)/f per channel
  int nee_env;        // env pixel of the light sample (-1: area light or none)
  float3 nee_env_d;   // d (NEE contribution) / d (env radiance of that pixel)
  float3 w_next;      // throughput factor of the sampled direction
  float3 no, nd;      // continuation ray
  float pdf_next;
  float u6;
  int lobe;
  int alb_kind, alb_ref, tex, rough, mtype;
  bool has_shadow, ok_next, delta_next, has_params;
  long long slot;     // sample index (pixel * spp + sample): radiance-cache query / path id
  bool cache_done;    // a cache query was written for this sample
  // forward-mode tangents (image derivative along a parameter direction)
  float3 beta_dot, L_dot, c_nee_dot, w_next_dot;
};

// The camera ray through image point (fx, fy) (pixel units, y down) and the path's
// initial state; the RNG has drawn the point's two uniforms already.
template <bool INSTR>
__device__ __forceinline__ void path_start_at(const LaunchArgs& A, PathState& P, int ci, float fx, float fy,
                                              Counters<INSTR>& cnt) {
  const DevCamera& cam = A.cams[ci];
  float sx = 2.0f * fx / A.width - 1.0f;
  float sy = 1.0f - 2.0f * fy / A.height;
  P.ro = f3(cam.ox, cam.oy, cam.oz);
  P.rd = normalize3(f3(cam.fx + cam.rx * sx + cam.ux * sy, cam.fy + cam.ry * sx + cam.uy * sy,
                       cam.fz + cam.rz * sx + cam.uz * sy));
  P.beta = f3(1.f, 1.f, 1.f);
  P.L = f3(0.f, 0.f, 0.f);
  P.beta_dot = f3(0.f, 0.f, 0.f);
  P.L_dot = f3(0.f, 0.f, 0.f);
  P.prev_delta = true;
  P.prev_pdf = 0.0f;
  P.depth = 1;
  cnt.add(0, 1);
}

// Sample si of pixel (px, py) of camera ci: its PCG32 stream (camera << 40 |
// pixel << 12 | sample) and a uniform point of the pixel.
template <bool INSTR>
__device__ __forceinline__ void path_start(const LaunchArgs& A, PathState& P, unsigned long long seed, int ci, int px,
                                           int py, int si, long long pix, Counters<INSTR>& cnt) {
  P.slot = pix * A.spp + si;
  P.cache_done = false;
  unsigned long long pixel = (unsigned long long)py * (unsigned long long)A.width + (unsigned long long)px;
  P.rng.seed(seed, ((unsigned long long)ci << 40) | (pixel << 12) | (unsigned long long)si);
  P.fh.h = 2166136261u;
  float j0 = P.rng.uniform(), j1 = P.rng.uniform();
  path_start_at<INSTR>(A, P, ci, px + j0, py + j1, cnt);
}

// Shading step after the closest hit.  Returns false if the path ended here.
// Not inlined (nor is path_finish): with their own register allocation the
// traversal loop of the megakernel keeps more registers (measured: adjoint -15 %,
// forward -4 % on the 196k-triangle sphere workload).
template <bool ADJ, bool JVP, bool INSTR, int DISPATCH, int FEAT = 0>
__device__ PT_SHADE_FN bool path_shade(const LaunchArgs& A, PathState& P, const Hit& hit, bool grad_pass, float3 dl,
                                        GradSink& sink,
                                           Counters<INSTR>& cnt) {
  const DevScene& S = A.scene;
  constexpr bool EGRAD = (FEAT & FEAT_EGRAD) != 0;
  constexpr bool HASH = (FEAT & FEAT_NOHASH) == 0;
  constexpr bool KEEP_L = !(ADJ && (FEAT & FEAT_REPLAY));  // the replay works from the stored radiance
  // the remaining radiance: the adjoint's, and the reparameterized kernels' (they call
  // this step without ADJ); not the production forward instances'
  constexpr bool KEEP_LREM = ADJ || (FEAT & FEAT_LEAN) == 0;
  // production instances write the continuation ray straight into the path's ray
  // (nothing reads the old one between this step and path_finish there)
  constexpr bool DIRECT_NEXT = (FEAT & FEAT_LEAN) != 0;
  const bool has_area = S.n_lights > 0;
  const bool has_env = S.env_w > 0;
  const float p_env = has_env ? (has_area ? 0.5f : 1.0f) : 0.0f;
  const float p_area = has_area ? 1.0f - p_env : 0.0f;
  P.has_shadow = false;
  if (hit.pos < 0) {
    if constexpr (HASH) P.fh.add(0xffffffffu);
    if (has_env) {
      cnt.add(12, 1);
      int ex, ey;
      env_pixel(S, P.rd, ex, ey);
      const int ei = ey * S.env_w + ex;
      float3 Le = xyz(__ldg(&(A.params.env ? A.params.env : S.env)[ei]));
      float w = 1.0f;
      if (!P.prev_delta && A.nee) {
        float st = sqrtf(fmaxf(0.0f, 1.0f - P.rd.y * P.rd.y));
        w = power_heuristic(P.prev_pdf, p_env * env_pdf_at(S, ex, ey, st));
      }
      float3 c = P.beta * Le * w;
      if constexpr (KEEP_L) P.L = P.L + c;
      if constexpr (KEEP_LREM) P.Lrem = P.Lrem - c;
      if (JVP) {
        P.L_dot = P.L_dot + P.beta_dot * Le * w;
        if (A.tangent.env) P.L_dot = P.L_dot + P.beta * xyz(__ldg(&A.tangent.env[ei])) * w;
      }
      if (ADJ && EGRAD && grad_pass && A.grads.env) sink.add_env<INSTR>(A, ei, dl * P.beta * w, cnt);
    }
    return false;
  }
  const float4 tv0 = __ldg(&S.tri_v[3 * hit.pos]);
  const float4 tv1 = __ldg(&S.tri_v[3 * hit.pos + 1]);
  const float4 tv2 = __ldg(&S.tri_v[3 * hit.pos + 2]);
  if constexpr (HASH) P.fh.add(__float_as_uint(tv0.w));
  const float4 ta0 = __ldg(&S.tri_a[2 * hit.pos]);
  const float4 ta1 = __ldg(&S.tri_a[2 * hit.pos + 1]);
  const int shape = __float_as_int(ta1.z);
  const int4* shp = reinterpret_cast<const int4*>(&S.shapes[shape]);
  const int4 sw0 = __ldg(shp);
  const float4 sw1 = __ldg(reinterpret_cast<const float4*>(shp + 1));
  const float3 ng = normalize3(cross3(xyz(tv1), xyz(tv2)));
  const float3 wi_w = -P.rd;
  const float cos_front = dot3(ng, wi_w);
  if (sw1.w > 0.0f && cos_front > 0.0f) {
    const float4 sw3 = __ldg(reinterpret_cast<const float4*>(shp + 3));
    float w = 1.0f;
    if (!P.prev_delta && A.nee) {
      float pdf_l = p_area * hit.t * hit.t / (cos_front * S.light_area);
      w = power_heuristic(P.prev_pdf, pdf_l);
    }
    float3 c = P.beta * xyz(sw3) * w;
    if constexpr (KEEP_L) P.L = P.L + c;
    if constexpr (KEEP_LREM) P.Lrem = P.Lrem - c;
    if (JVP) P.L_dot = P.L_dot + P.beta_dot * xyz(sw3) * w;
  }
  if (P.depth >= A.max_depth) return false;
  float u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) u[k] = P.rng.uniform();
  const int type = sw0.x;
  if (type == PT_BSDF_NONE) return false;
  cnt.add(7 + type, 1);  // PT_CNT_V_DIFFUSE .. PT_CNT_V_BLEND

  const float3 p = P.ro + P.rd * hit.t;
  const float b0 = 1.0f - hit.u - hit.v;
  const float tu = b0 * ta0.x + hit.u * ta0.z + hit.v * ta1.x;
  const float tvv = b0 * ta0.y + hit.u * ta0.w + hit.v * ta1.y;
  // ---- material: closure record + differentiable parameters
  Material m;
  m.type = type;
  m.tex = sw0.y;
  m.alpha = sw1.x;
  m.eta = sw1.y;
  m.wd = sw1.z;
  m.rough = sw0.w;
  m.alb_kind = 0;
  m.alb_ref = 0;
  m.albedo = f3(0.f, 0.f, 0.f);
  if (m.rough >= 0) m.alpha = __ldg(&A.params.rough[m.rough]);
  m.f0 = xyz(__ldg(reinterpret_cast<const float4*>(shp + 2)));
  uint32_t texel_word = 0xffffffffu;
  if (type == PT_BSDF_DIFFUSE || type == PT_BSDF_BLEND) {
    if (m.tex >= 0) {
      // nearest lookup (App. B): pos = min(uint(uv * res), res - 1), texel [pos.y, pos.x]
      const int w = A.params.tex_w[m.tex], h = A.params.tex_h[m.tex];
      const int x = min((int)(fmaxf(tu, 0.0f) * (float)w), w - 1);
      const int y = min((int)(fmaxf(tvv, 0.0f) * (float)h), h - 1);
      const int idx = y * w + x;
      m.albedo = xyz(__ldg(&A.params.tex[m.tex][idx]));
      m.alb_kind = 2;
      m.alb_ref = idx;
      texel_word = (uint32_t)idx;
      cnt.add(5, 1);
    } else if (sw0.z >= 0) {
      const float* a = &A.params.albedo[3 * sw0.z];
      m.albedo = f3(__ldg(a), __ldg(a + 1), __ldg(a + 2));
      m.alb_kind = 1;
      m.alb_ref = sw0.z;
    }
  }
  if constexpr (HASH) P.fh.add(texel_word);
  // tangent of the differentiable inputs along the JVP direction
  float3 alb_dot = f3(0.f, 0.f, 0.f);
  float alpha_dot = 0.0f;
  if constexpr (JVP) {
    if (m.alb_kind == 2 && A.tangent.tex[m.tex]) alb_dot = xyz(__ldg(&A.tangent.tex[m.tex][m.alb_ref]));
    else if (m.alb_kind == 1 && A.tangent.albedo) {
      const float* a = &A.tangent.albedo[3 * m.alb_ref];
      alb_dot = f3(__ldg(a), __ldg(a + 1), __ldg(a + 2));
    }
    if (m.rough >= 0 && A.tangent.rough) alpha_dot = __ldg(&A.tangent.rough[m.rough]);
  }

  const bool entering = cos_front > 0.0f;
  const float3 n_s = entering ? ng : -ng;
  // ---- radiance cache: terminate into the cache, or record training data
  if ((FEAT & FEAT_CACHE) && A.cache_mode != 0 && type != PT_BSDF_DIELECTRIC) {
    const float rough = (type == PT_BSDF_CONDUCTOR || type == PT_BSDF_BLEND) ? m.alpha : 1.0f;
    if (A.cache_mode == 3) {
      const unsigned active = __activemask();
      const int lane = lane_id(), leader = __ffs(active) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(A.r_count, (unsigned)__popc(active));
      base = __shfl_sync(active, base, leader);
      const long long idx = (long long)base + __popc(active & ((1u << lane) - 1u));
      if (idx < A.max_records) {
        float* r = A.r_raw + idx * 10;
        r[0] = p.x; r[1] = p.y; r[2] = p.z;
        r[3] = wi_w.x; r[4] = wi_w.y; r[5] = wi_w.z;
        r[6] = n_s.x; r[7] = n_s.y; r[8] = n_s.z;
        r[9] = rough;
        float* a = A.r_aux + idx * 8;
        a[0] = P.beta.x; a[1] = P.beta.y; a[2] = P.beta.z;
        a[3] = P.L.x; a[4] = P.L.y; a[5] = P.L.z;
        a[6] = __int_as_float((int)P.slot);
        a[7] = __int_as_float(P.depth);
      }
    } else if (P.depth >= A.cache_bounce) {
      if (A.cache_mode == 1) {
        float* r = A.q_raw + P.slot * 10;
        r[0] = p.x; r[1] = p.y; r[2] = p.z;
        r[3] = wi_w.x; r[4] = wi_w.y; r[5] = wi_w.z;
        r[6] = n_s.x; r[7] = n_s.y; r[8] = n_s.z;
        r[9] = rough;
        float* b = A.q_beta + P.slot * 3;
        b[0] = P.beta.x; b[1] = P.beta.y; b[2] = P.beta.z;
        P.cache_done = true;
      } else {
        const float* q = A.q_rgb + P.slot * 3;
        const float3 c = P.beta * f3(fmaxf(q[0], 0.f), fmaxf(q[1], 0.f), fmaxf(q[2], 0.f));
        if constexpr (KEEP_L) P.L = P.L + c;
        if constexpr (KEEP_LREM) P.Lrem = P.Lrem - c;
      }
      return false;
    }
  }
  const Frame fr = make_frame(n_s);
  const float3 wi = fr.to_local(wi_w);
  if (EGRAD) P.nee_env = -1;
  if (JVP) P.c_nee_dot = f3(0.f, 0.f, 0.f);
  if (ADJ) P.r_nee_alb = P.r_nee_a = P.r_bsdf_alb = P.r_bsdf_a = f3(0.f, 0.f, 0.f);

  // ---- next-event estimation: light sample + BSDF value toward it
  if (type != PT_BSDF_DIELECTRIC && A.nee && (has_area || has_env)) {
    const bool pick_env = has_env && (!has_area || u[7] < 0.5f);
    float3 dir, Le;
    float pdf_l = 0.0f, dist = INFINITY;
    bool valid = false;
    int env_i = -1;
    if (pick_env) {
      const int y = cdf_pick_guided(S.env_marg, S.env_marg_guide, S.env_gm, u[1]);
      const float* cond = S.env_cond + (size_t)y * (S.env_w + 1);
      const int x = cdf_pick_guided(cond, S.env_cond_guide + (size_t)y * (S.env_gc + 1), S.env_gc, u[2]);
      const float m0 = __ldg(&S.env_marg[y]), m1 = __ldg(&S.env_marg[y + 1]);
      const float c0 = __ldg(&cond[x]), c1 = __ldg(&cond[x + 1]);
      const float fv = (u[1] - m0) / (m1 - m0);
      const float fu = (u[2] - c0) / (c1 - c0);
      // theta = pi (y + fv) / H, phi = 2 pi (x + fu) / W, through sin/cos of pi * a
      float st, ct, sp, cp;
      sincospif((y + fv) / S.env_h, &st, &ct);
      sincospif(2.0f * (x + fu) / S.env_w, &sp, &cp);
      dir = f3(st * cp, ct, st * sp);
      env_i = y * S.env_w + x;
      Le = xyz(__ldg(&(A.params.env ? A.params.env : S.env)[env_i]));
      pdf_l = p_env * env_pdf_at(S, x, y, st);
      valid = pdf_l > 0.0f;
      if constexpr (HASH) P.fh.add(0x80000000u | (uint32_t)(y * S.env_w + x));
      cnt.add(12, 1);
    } else {
      const int k = cdf_pick_guided(S.light_cdf, S.light_guide, S.light_g, u[0]);
      const float4 l0 = __ldg(&S.lights[4 * k]);
      const float4 l1 = __ldg(&S.lights[4 * k + 1]);
      const float4 l2 = __ldg(&S.lights[4 * k + 2]);
      const float4 l3 = __ldg(&S.lights[4 * k + 3]);
      const float su = sqrtf(u[1]);
      const float lb0 = 1.0f - su, lb1 = u[2] * su;
      const float3 q = xyz(l0) * lb0 + xyz(l1) * lb1 + xyz(l2) * (1.0f - lb0 - lb1);
      const float3 dv = q - p;
      dist = sqrtf(dot3(dv, dv));
      dir = dv * (1.0f / dist);
      const float3 nl = normalize3(cross3(xyz(l1) - xyz(l0), xyz(l2) - xyz(l0)));
      const float cos_l = -dot3(nl, dir);
      Le = xyz(l3);
      if (cos_l > 0.0f && dist > 0.0f) {
        pdf_l = p_area * dist * dist / (cos_l * S.light_area);
        valid = true;
      }
      if constexpr (HASH) P.fh.add(__float_as_uint(l0.w));
    }
    const float3 wl = fr.to_local(dir);
    BsdfEval ev;
    dispatch_bsdf<DISPATCH>(type, [&]<int T>() {
      if constexpr (T != PT_BSDF_DIELECTRIC) ev = bsdf_eval<T, ADJ || JVP>(m, wi, wl);
    });
    if (valid && wl.z > 0.0f && max3f(ev.f) > 0.0f) {
      P.has_shadow = true;
      P.so = offset_origin(p, ng, dir);
      P.sd = dir;
      P.stmax = pick_env ? INFINITY : dist * (1.0f - 1e-3f);
      const float w = power_heuristic(pdf_l, ev.pdf);
      const float s_env = wl.z * w / pdf_l;  // d scale / d Le
      const float3 scale = Le * s_env;
      P.c_nee = P.beta * ev.f * scale;
      if (JVP) {
        const float3 f_dot = ev.df_alb * alb_dot + ev.df_alpha * alpha_dot;
        P.c_nee_dot = (P.beta_dot * ev.f + P.beta * f_dot) * scale;
        if (env_i >= 0 && A.tangent.env)
          P.c_nee_dot = P.c_nee_dot + P.beta * ev.f * xyz(__ldg(&A.tangent.env[env_i])) * s_env;
      }
      if (ADJ && EGRAD && grad_pass && env_i >= 0 && A.grads.env) {
        P.nee_env = env_i;
        P.nee_env_d = P.beta * ev.f * s_env;
      }
      if (ADJ && grad_pass) {
        log_derivs(ev.df_alb, ev.df_alpha, ev.f, P.r_nee_alb, P.r_nee_a);
      }
    }
  }
  // ---- BSDF sampling (detached) with its attached value
  BsdfSample bs;
  dispatch_bsdf<DISPATCH>(type, [&]<int T>() { bs = bsdf_sample<T, ADJ || JVP>(m, wi, entering, u[3], u[4], u[5]); });
  if constexpr (JVP) {
    P.w_next_dot = f3(0.f, 0.f, 0.f);
    if (bs.ok && !bs.delta)
      P.w_next_dot = (bs.ev.df_alb * alb_dot + bs.ev.df_alpha * alpha_dot) * (bs.wo.z / bs.pdf);
  }
  if constexpr (HASH) P.lobe = bs.lobe;
  P.ok_next = bs.ok;
  P.delta_next = bs.delta;
  P.w_next = bs.weight;
  P.pdf_next = bs.pdf;
  P.u6 = u[6];
  if (ADJ && grad_pass && bs.ok && !bs.delta) {
    log_derivs(bs.ev.df_alb, bs.ev.df_alpha, bs.ev.f, P.r_bsdf_alb, P.r_bsdf_a);
  }
  if (bs.ok) {
    const float3 wo = fr.to_world(bs.wo);
    if constexpr (DIRECT_NEXT) {
      P.ro = offset_origin(p, ng, wo);
      P.rd = wo;
    } else {
      P.no = offset_origin(p, ng, wo);
      P.nd = wo;
    }
  }
  if (ADJ) {
    P.alb_kind = m.alb_kind;
    P.alb_ref = m.alb_ref;
    P.tex = m.tex;
    P.rough = m.rough;
    P.has_params = m.alb_kind != 0 || m.rough >= 0;
  }
  if constexpr (ADJ || HASH || (FEAT & FEAT_LEAN) == 0) P.mtype = type;
  return true;
}

// Finish the vertex once the shadow ray is resolved.  Returns false if the path ended.
template <bool ADJ, bool JVP, bool INSTR, int FEAT = 0>
__device__ __forceinline__ bool path_finish_body(const LaunchArgs& A, PathState& P, bool occluded, bool grad_pass,
                                                 float3 dl, GradSink& sink, Counters<INSTR>& cnt) {
  constexpr bool HASH = (FEAT & FEAT_NOHASH) == 0;
  constexpr bool KEEP_L = !(ADJ && (FEAT & FEAT_REPLAY));
  constexpr bool KEEP_LREM = ADJ || (FEAT & FEAT_LEAN) == 0;
  if constexpr (HASH) {
    if (A.nee && P.mtype != PT_BSDF_DIELECTRIC && (A.scene.n_lights > 0 || A.scene.env_w > 0))
      P.fh.add(P.has_shadow ? (occluded ? 1u : 0u) : 2u);
  }
  const bool lit = P.has_shadow && !occluded;
  if (lit) {
    if constexpr (KEEP_L) P.L = P.L + P.c_nee;
    if constexpr (KEEP_LREM) P.Lrem = P.Lrem - P.c_nee;
    if (JVP) P.L_dot = P.L_dot + P.c_nee_dot;
    if (ADJ && (FEAT & FEAT_EGRAD) && grad_pass && P.nee_env >= 0)
      sink.add_env<INSTR>(A, P.nee_env, dl * P.nee_env_d, cnt);
  }
  if constexpr (HASH) P.fh.add((uint32_t)P.lobe);
  if constexpr (HASH) {
    if (P.delta_next) P.fh.add(0xfffffffeu);
  }
  if (ADJ && grad_pass && P.has_params) {
    const float3 cn = lit ? P.c_nee : f3(0.f, 0.f, 0.f);
    const float3 lr = P.ok_next ? f3(fmaxf(P.Lrem.x, 0.f), fmaxf(P.Lrem.y, 0.f), fmaxf(P.Lrem.z, 0.f))
                                : f3(0.f, 0.f, 0.f);
    const float3 g_alb = dl * (cn * P.r_nee_alb + lr * P.r_bsdf_alb);
    const float3 ga = dl * (cn * P.r_nee_a + lr * P.r_bsdf_a);
    Material m;
    m.type = P.mtype;
    m.alb_kind = P.alb_kind;
    m.alb_ref = P.alb_ref;
    m.tex = P.tex;
    m.rough = P.rough;
    sink.add<INSTR, (FEAT & FEAT_TEXAGG) != 0>(A, m, g_alb, ga.x + ga.y + ga.z, cnt);
  }
  if (!P.ok_next) return false;
  if (JVP) P.beta_dot = P.beta_dot * P.w_next + P.beta * P.w_next_dot;
  P.beta = P.beta * P.w_next;
  P.prev_delta = P.delta_next;
  P.prev_pdf = P.pdf_next;
  if constexpr ((FEAT & FEAT_LEAN) == 0) {
    P.ro = P.no;
    P.rd = P.nd;
  }
  if (A.rr_depth >= 0 && P.depth >= A.rr_depth) {
    const float q = fminf(max3f(P.beta), 0.95f);
    const bool cont = P.u6 < q;
    if constexpr (HASH) P.fh.add(cont ? 1u : 0u);
    if (!cont) return false;
    P.beta = P.beta * (1.0f / q);
    if (JVP) P.beta_dot = P.beta_dot * (1.0f / q);
  }
  ++P.depth;
  return true;
}

// Out of line, except where the megakernel calls the body directly (the adjoint
// instances: measured replay 61.7 vs 62.8 ms inline; the forward is faster out of line).
template <bool ADJ, bool JVP, bool INSTR, int FEAT = 0>
__device__ PT_FINISH_FN bool path_finish(const LaunchArgs& A, PathState& P, bool occluded, bool grad_pass,
                                         float3 dl, GradSink& sink, Counters<INSTR>& cnt) {
  return path_finish_body<ADJ, JVP, INSTR, FEAT>(A, P, occluded, grad_pass, dl, sink, cnt);
}

}  // namespace ptgb
