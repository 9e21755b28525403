// Device code of the path-tracing megakernel and its PRB adjoint (sm_103a).
//
// One thread traces whole paths (megakernel, Fig. 7 #1): camera ray, closest-hit
// traversal, surface interaction, per-material BSDF work reached through a
// per-lane polymorphic dispatch, next-event estimation with MIS, BSDF
// sampling, Russian roulette.  The adjoint (Fig. 7 #2 + #3 fused) runs the
// same loop body twice per sample: pass 0 recovers the sample's radiance L,
// pass 1 replays the identical path from the same PCG32 state, subtracting
// each contribution from L (arithmetic invertibility, Sec. 4.1) and
// scatter-adding (dL * radiance * (df/dtheta)/f) into parameter gradients
// (Sec. 4.9: detached sampling, attached BSDF values).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_internal.h"

namespace ptgb {

#define PT_PI 3.14159265358979323846f
#define PT_INV_PI 0.31830988618379067154f
#define PT_STACK 64
// 1/x through the correctly rounded reciprocal: the same value as the IEEE
// division 1.0f / x, without the division's general code path.
// Correctly rounded reciprocal (the same bits as 1.0f / x under IEEE division, whatever
// a source's division flags)
#define PT_RCP(x) __frcp_rn(x)

// ---------------------------------------------------------------- float3 helpers
__device__ __forceinline__ float3 f3(float a, float b, float c) { return make_float3(a, b, c); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrtf(dot3(a, a)); }
__device__ __forceinline__ float max3f(float3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------- PCG32 (O'Neill 2014)
struct Pcg32 {
  unsigned long long state, inc;
  __device__ __forceinline__ void seed(unsigned long long initstate, unsigned long long initseq) {
    state = 0ull;
    inc = (initseq << 1) | 1ull;
    next();
    state += initstate;
    next();
  }
  __device__ __forceinline__ uint32_t next() {
    unsigned long long old = state;
    state = old * 6364136223846793005ull + inc;
    uint32_t xs = (uint32_t)(((old >> 18) ^ old) >> 27);
    uint32_t rot = (uint32_t)(old >> 59);
    return __funnelshift_r(xs, xs, rot);  // rotate right by rot
  }
  // top 24 bits scaled by 2^-24: exactly representable
  __device__ __forceinline__ float uniform() { return (float)(next() >> 8) * (1.0f / 16777216.0f); }
};

// ---------------------------------------------------------------- FNV-1a decision fingerprint
struct Fnv {
  uint32_t h;
  __device__ __forceinline__ void add(uint32_t w) { h = (h ^ w) * 16777619u; }
};

// ---------------------------------------------------------------- instrumentation
constexpr int kCounters = 16;  // PT_CNT_PATHS .. PT_CNT_WARP_LOOP_STEPS
template <bool INSTR>
struct Counters {
  __device__ __forceinline__ void add(int, unsigned) {}
};
template <>
struct Counters<true> {
  unsigned c[kCounters];
  __device__ __forceinline__ void add(int i, unsigned v) { c[i] += v; }
};

__device__ __forceinline__ void set_status(const DevScene& s, int code) {
  if (s.status) atomicCAS(s.status, 0, code);
}

// ---------------------------------------------------------------- traversal (binary BVH)
struct Ray {
  float3 o, d;
};
struct Hit {
  int pos;      // leaf-order triangle position, -1 = miss
  float t, u, v;
};

// The ray's inverse direction for the box tests (only they use it): the hardware
// reciprocal, within 1 ulp; the boxes' padding (3e-6 relative plus the absolute pad and
// the 8-wide layout's 2^-8-step margin) is far wider than that.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float3 safe_inv(float3 d) {
  const float eps = 1e-20f;
  return f3(rcp_approx(fabsf(d.x) > eps ? d.x : copysignf(eps, d.x)),
            rcp_approx(fabsf(d.y) > eps ? d.y : copysignf(eps, d.y)),
            rcp_approx(fabsf(d.z) > eps ? d.z : copysignf(eps, d.z)));
}

// Moller-Trumbore in FP32 (edges inclusive, det == 0 misses).  Updates the
// closest hit; ties in t go to the smaller original triangle id.
__device__ __forceinline__ bool tri_test(const float4* __restrict__ tv, int pos, const Ray& r, float& best_t,
                                         int& best_pos, uint32_t& best_orig, float& bu, float& bv) {
  float4 a = __ldg(&tv[3 * pos]);
  float4 b = __ldg(&tv[3 * pos + 1]);
  float4 c = __ldg(&tv[3 * pos + 2]);
  float3 v0 = xyz(a), e1 = xyz(b), e2 = xyz(c);
  float3 p = cross3(r.d, e2);
  float det = dot3(e1, p);
  if (det == 0.0f) return false;
  float inv = PT_RCP(det);
  float3 s = r.o - v0;
  float u = dot3(s, p) * inv;
  if (u < 0.0f || u > 1.0f) return false;
  float3 q = cross3(s, e1);
  float v = dot3(r.d, q) * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  float t = dot3(e2, q) * inv;
  if (!(t > 0.0f)) return false;
  uint32_t orig = __float_as_uint(a.w);
  if (t < best_t || (best_pos >= 0 && t == best_t && orig < best_orig)) {
    best_t = t;
    best_pos = pos;
    best_orig = orig;
    bu = u;
    bv = v;
    return true;
  }
  return false;
}

// Closest hit (any_hit = false) or any hit before tmax (any_hit = true) on the
// 2-wide BVH.  "While-while" structure (Aila & Laine 2009): an inner loop walks
// inner nodes until the lane holds a leaf, a second loop intersects leaves, so
// lanes of a warp stay in the same phase longer than with one if/else loop.
template <bool INSTR>
__device__ __forceinline__ Hit trace_binary(const DevScene& S, float3 ro, float3 rd, float tmax, bool any_hit,
                                         Counters<INSTR>& cnt) {
  Hit h;
  h.pos = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  Ray r;
  r.o = ro;
  r.d = rd;
  uint32_t best_orig = 0xffffffffu;
  const float3 inv = safe_inv(rd);
  const float3 oi = ro * inv;
  int stack[PT_STACK];
  int sp = 0;
  int cur = 0;
  const float4* __restrict__ N = S.nodes;
  unsigned n_nodes = 0, n_tris = 0, warp_steps = 0;
  const int kDone = 0x7fffffff;
  while (cur != kDone) {
    // ---- inner nodes
    while (cur >= 0 && cur != kDone) {
      ++n_nodes;
      if constexpr (INSTR) {
        if (lane_id() == __ffs(__activemask()) - 1) ++warp_steps;
      }
      const float4 w0 = __ldg(&N[4 * cur]);
      const float4 w1 = __ldg(&N[4 * cur + 1]);
      const float4 w2 = __ldg(&N[4 * cur + 2]);
      const float4 w3 = __ldg(&N[4 * cur + 3]);
      const float a0 = w0.x * inv.x - oi.x, a1 = w0.y * inv.x - oi.x;
      const float b0 = w0.z * inv.y - oi.y, b1 = w0.w * inv.y - oi.y;
      const float c0 = w2.x * inv.z - oi.z, c1 = w2.y * inv.z - oi.z;
      const float tn0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fmaxf(fminf(c0, c1), 0.0f));
      const float tf0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fminf(fmaxf(c0, c1), h.t));
      const float d0 = w1.x * inv.x - oi.x, d1 = w1.y * inv.x - oi.x;
      const float e0 = w1.z * inv.y - oi.y, e1 = w1.w * inv.y - oi.y;
      const float g0 = w2.z * inv.z - oi.z, g1 = w2.w * inv.z - oi.z;
      const float tn1 = fmaxf(fmaxf(fminf(d0, d1), fminf(e0, e1)), fmaxf(fminf(g0, g1), 0.0f));
      const float tf1 = fminf(fminf(fmaxf(d0, d1), fmaxf(e0, e1)), fminf(fmaxf(g0, g1), h.t));
      const bool hit0 = tn0 <= tf0, hit1 = tn1 <= tf1;
      const int ch0 = __float_as_int(w3.x), ch1 = __float_as_int(w3.y);
      if (hit0 && hit1) {
        int nearc = ch0, farc = ch1;
        if (tn1 < tn0) {
          nearc = ch1;
          farc = ch0;
        }
        if (sp >= PT_STACK) {
          set_status(S, PT_ERR_BVH);
          cur = kDone;
          break;
        }
        stack[sp++] = farc;
        cur = nearc;
      } else if (hit0) {
        cur = ch0;
      } else if (hit1) {
        cur = ch1;
      } else {
        cur = sp > 0 ? stack[--sp] : kDone;
      }
    }
    // ---- leaves
    while (cur < 0) {
      const int leaf = ~cur;
      const int first = leaf >> 3, count = (leaf & 7) + 1;
      n_tris += count;
      bool found = false;
      for (int i = 0; i < count; ++i) found |= tri_test(S.tri_v, first + i, r, h.t, h.pos, best_orig, h.u, h.v);
      if (found && any_hit) {
        cur = kDone;
        break;
      }
      cur = sp > 0 ? stack[--sp] : kDone;
    }
  }
  cnt.add(3, n_nodes);
  cnt.add(4, n_tris);
  cnt.add(14, warp_steps);
  return h;
}

// Three-input FP32 minimum / maximum (one instruction on sm_100 and later; exact, so
// the same values as two chained fminf / fmaxf).
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// Both lanes of a packed pair in one 64-bit register.
__device__ __forceinline__ uint64_t pack_f32x2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
// (qn A + B, qf A + B) with AA = (A, A), BB = (B, B): one packed FP32 FMA (sm_100 and
// later), rounded per lane exactly as two fmaf.
__device__ __forceinline__ void plane_pair(float qn, float qf, uint64_t AA, uint64_t BB, float& tn, float& tf) {
  asm("{\n .reg .b64 q, d;\n mov.b64 q, {%2, %3};\n fma.rn.f32x2 d, q, %4, %5;\n mov.b64 {%0, %1}, d;\n}"
      : "=f"(tn), "=f"(tf)
      : "f"(qn), "f"(qf), "l"(AA), "l"(BB));
}

// Closest hit / any hit on the 8-wide compressed BVH (80-byte nodes: origin,
// per-axis power-of-two steps, inner-child mask, child and triangle bases, and
// 8-bit child box planes; see bvh_build.h).  Each visited node tests its eight
// child boxes with one FMA per plane, the near and far planes of an axis as one packed
// FMA (near/far planes picked once per node from
// the ray direction), intersects the triangles of hit leaf children at once, and
// pushes the remaining hit inner children as one (base, mask) group.  Children
// are visited in the order of the slot octants relative to the ray direction.
template <bool INSTR>
__device__ __forceinline__ Hit trace_wide(const DevScene& S, float3 ro, float3 rd, float tmax, bool any_hit,
                                          Counters<INSTR>& cnt) {
  Hit h;
  h.pos = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  Ray r;
  r.o = ro;
  r.d = rd;
  uint32_t best_orig = 0xffffffffu;
  const float3 inv = safe_inv(rd);
  const uint32_t flip = (rd.x >= 0.0f ? 1u : 0u) | (rd.y >= 0.0f ? 2u : 0u) | (rd.z >= 0.0f ? 4u : 0u);
  const uint4* __restrict__ N = reinterpret_cast<const uint4*>(S.nodes);
  uint2 stack[32];
  int sp = 0;
  int node = 0;
  unsigned n_nodes = 0, n_tris = 0;
  unsigned warp_steps = 0;
  for (;;) {
    ++n_nodes;
    if constexpr (INSTR) {
      if (lane_id() == __ffs(__activemask()) - 1) ++warp_steps;
    }
    const uint4 w0 = __ldg(&N[5 * node]);
    const uint4 w1 = __ldg(&N[5 * node + 1]);
    const uint4 w2 = __ldg(&N[5 * node + 2]);
    const uint4 w3 = __ldg(&N[5 * node + 3]);
    const uint4 w4 = __ldg(&N[5 * node + 4]);
    const uint32_t ex = w0.w & 0xffu, ey = (w0.w >> 8) & 0xffu, ez = (w0.w >> 16) & 0xffu;
    const uint32_t imask = w0.w >> 24;
    // plane q of an axis with step s sits at t = q a + b, a = s / d, b = (origin - o) / d.
    // A plane byte enters as the float 1 + q 2^-15 (one byte permute builds it), so that
    // q a + b = (1 + q 2^-15) A + B with A = 2^15 a (the node stores the exponent of
    // 2^15 s) and B = b - A in one FMA: one FMA per plane.  B's rounding moves a plane by
    // at most 2^-9 of a step; the builder keeps 2^-8 of a step between every child box
    // and its planes.
    const float Ax = __uint_as_float(ex << 23) * inv.x;
    const float Ay = __uint_as_float(ey << 23) * inv.y;
    const float Az = __uint_as_float(ez << 23) * inv.z;
    const float Bx = fmaf(__uint_as_float(w0.x) - ro.x, inv.x, -Ax);
    const float By = fmaf(__uint_as_float(w0.y) - ro.y, inv.y, -Ay);
    const float Bz = fmaf(__uint_as_float(w0.z) - ro.z, inv.z, -Az);
    const uint64_t AAx = pack_f32x2(Ax, Ax), AAy = pack_f32x2(Ay, Ay), AAz = pack_f32x2(Az, Az);
    const uint64_t BBx = pack_f32x2(Bx, Bx), BBy = pack_f32x2(By, By), BBz = pack_f32x2(Bz, Bz);
    // near / far plane bytes per axis (lo planes are near for a positive direction)
    const uint32_t nx0 = rd.x >= 0.0f ? w2.x : w3.z, nx1 = rd.x >= 0.0f ? w2.y : w3.w;
    const uint32_t fx0 = rd.x >= 0.0f ? w3.z : w2.x, fx1 = rd.x >= 0.0f ? w3.w : w2.y;
    const uint32_t ny0 = rd.y >= 0.0f ? w2.z : w4.x, ny1 = rd.y >= 0.0f ? w2.w : w4.y;
    const uint32_t fy0 = rd.y >= 0.0f ? w4.x : w2.z, fy1 = rd.y >= 0.0f ? w4.y : w2.w;
    const uint32_t nz0 = rd.z >= 0.0f ? w3.x : w4.z, nz1 = rd.z >= 0.0f ? w3.y : w4.w;
    const uint32_t fz0 = rd.z >= 0.0f ? w4.z : w3.x, fz1 = rd.z >= 0.0f ? w4.w : w3.y;
    // hit slots in slot order; empty slots hold inverted boxes that the slab test rejects
    // (and one that passes anyway, a degenerate box below FP32 resolution, is a leaf of
    // zero triangles), so no per-slot bookkeeping beyond one compare and one OR
    uint32_t hitm = 0;
#pragma unroll
    for (int sl = 0; sl < 8; ++sl) {
      // byte q of a plane word -> the float 1 + q 2^-15 (bits 0x3F80qq00): one byte
      // permute, no shift/mask and no int->float convert
      const uint32_t sel = 0x7604u | ((uint32_t)(sl & 3) << 4);
      const float qnx = __uint_as_float(__byte_perm(sl < 4 ? nx0 : nx1, 0x3F800000u, sel));
      const float qfx = __uint_as_float(__byte_perm(sl < 4 ? fx0 : fx1, 0x3F800000u, sel));
      const float qny = __uint_as_float(__byte_perm(sl < 4 ? ny0 : ny1, 0x3F800000u, sel));
      const float qfy = __uint_as_float(__byte_perm(sl < 4 ? fy0 : fy1, 0x3F800000u, sel));
      const float qnz = __uint_as_float(__byte_perm(sl < 4 ? nz0 : nz1, 0x3F800000u, sel));
      const float qfz = __uint_as_float(__byte_perm(sl < 4 ? fz0 : fz1, 0x3F800000u, sel));
      // near and far plane of an axis in one packed FMA; entry and exit in two
      // three-input min / max each
      float tnx, tfx, tny, tfy, tnz, tfz;
      plane_pair(qnx, qfx, AAx, BBx, tnx, tfx);
      plane_pair(qny, qfy, AAy, BBy, tny, tfy);
      plane_pair(qnz, qfz, AAz, BBz, tnz, tfz);
      const float tn = max3f(fmaxf(tnx, 0.0f), tny, tnz);
      const float tf = min3f(fminf(tfx, h.t), tfy, tfz);
      if (tn <= tf) hitm |= 1u << sl;
    }
    uint32_t leaf_hits = hitm & ~imask;
    uint32_t inner_hits = hitm & imask;
    // inner hits in octant order: slot sl -> bit sl ^ flip (three masked swaps)
    inner_hits = (flip & 1u) ? ((inner_hits & 0x55u) << 1) | ((inner_hits >> 1) & 0x55u) : inner_hits;
    inner_hits = (flip & 2u) ? ((inner_hits & 0x33u) << 2) | ((inner_hits >> 2) & 0x33u) : inner_hits;
    inner_hits = (flip & 4u) ? ((inner_hits & 0x0Fu) << 4) | ((inner_hits >> 4) & 0x0Fu) : inner_hits;
    // triangles of the hit leaf children
    bool stop = false;
    while (leaf_hits) {
      const int sl = __ffs(leaf_hits) - 1;
      leaf_hits &= leaf_hits - 1;
      const uint32_t meta = ((sl < 4 ? w1.z : w1.w) >> (8 * (sl & 3))) & 0xffu;
      const int count = (int)(meta >> 5), first = (int)w1.y + (int)(meta & 31u);
      n_tris += count;
      bool found = false;
      for (int i = 0; i < count; ++i) found |= tri_test(S.tri_v, first + i, r, h.t, h.pos, best_orig, h.u, h.v);
      if (found && any_hit) {
        stop = true;
        break;
      }
    }
    if (stop) break;
    // next node: nearest-octant hit child, the rest stays on the stack as one group
    uint32_t base = w1.x, gmask = imask, hits = inner_hits;
    if (hits == 0u) {
      if (sp == 0) break;
      const uint2 e = stack[sp - 1];
      --sp;
      base = e.x;
      gmask = e.y & 0xffu;
      hits = e.y >> 8;
    }
    const int k = __ffs(hits) - 1;
    hits &= hits - 1;
    const int sl = k ^ (int)flip;
    node = (int)base + __popc(gmask & ((1u << sl) - 1u));
    if (hits) {
      if (sp >= 32) {
        set_status(S, PT_ERR_BVH);
        break;
      }
      stack[sp++] = make_uint2(base, gmask | (hits << 8));
    }
  }
  cnt.add(3, n_nodes);
  cnt.add(4, n_tris);
  cnt.add(14, warp_steps);
  return h;
}

// ---------------------------------------------------------------- shading frame
// Orthonormal basis around n (Duff et al. 2017), branch on n.z >= 0 so +0/-0 agree.
struct Frame {
  float3 s, t, n;
  __device__ __forceinline__ float3 to_local(float3 w) const { return f3(dot3(w, s), dot3(w, t), dot3(w, n)); }
  __device__ __forceinline__ float3 to_world(float3 v) const { return s * v.x + t * v.y + n * v.z; }
};
__device__ __forceinline__ Frame make_frame(float3 n) {
  float sign = n.z >= 0.0f ? 1.0f : -1.0f;
  float a = -PT_RCP(sign + n.z);
  float b = n.x * n.y * a;
  Frame f;
  f.n = n;
  f.s = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  f.t = f3(b, sign + n.y * n.y * a, -n.y);
  return f;
}

// ---------------------------------------------------------------- materials
struct Material {
  int type;
  float3 albedo;
  float alpha, eta, wd;
  float3 f0;
  int alb_kind;     // 0 none, 1 constant row, 2 texel
  int alb_ref;      // row, or linear texel index
  int tex;          // texture slot (alb_kind == 2)
  int rough;        // roughness entry or -1
};

// BSDF value, pdf and (for the adjoint) partial derivatives of f per channel.
struct BsdfEval {
  float3 f;
  float pdf;
  float3 df_alb;    // d f_c / d albedo_c
  float3 df_alpha;  // d f_c / d alpha
};

__device__ __forceinline__ float ggx_D(float a, float c) {
  float a2 = a * a;
  float den = c * c * (a2 - 1.0f) + 1.0f;
  return a2 / (PT_PI * den * den);
}
__device__ __forceinline__ float ggx_G1(float a, float c, float* dlog) {
  float T = (1.0f - c * c) / (c * c);
  float s = sqrtf(1.0f + a * a * T);
  if (dlog) *dlog = -(a * T / s) / (1.0f + s);
  return 2.0f * PT_RCP(1.0f + s);  // 2 / (1 + s) exactly: scaling by 2 is exact
}
__device__ __forceinline__ float schlick(float f0, float cd) {
  float m = 1.0f - cd;
  float m2 = m * m;
  return f0 + (1.0f - f0) * (m2 * m2 * m);
}

// GGX conductor value (+ d f / d alpha when GRAD); wi, wo above the surface.
template <bool GRAD>
__device__ __forceinline__ float3 ggx_eval(float a, float3 f0, float3 wi, float3 wo, float* pdf, float3* dfa) {
  float3 h = normalize3(wi + wo);
  float D = ggx_D(a, h.z);
  float dl_i, dl_o;
  float G = ggx_G1(a, wi.z, GRAD ? &dl_i : nullptr) * ggx_G1(a, wo.z, GRAD ? &dl_o : nullptr);
  float cd = dot3(wi, h);
  float k = D * G / (4.0f * wi.z * wo.z);
  float3 f = f3(schlick(f0.x, cd) * k, schlick(f0.y, cd) * k, schlick(f0.z, cd) * k);
  *pdf = D * h.z / (4.0f * fabsf(dot3(wo, h)));
  if (GRAD) {
    float c2 = h.z * h.z;
    float dlog = 2.0f / a - 4.0f * a * c2 / (c2 * (a * a - 1.0f) + 1.0f) + dl_i + dl_o;
    *dfa = f * dlog;
  }
  return f;
}

// Evaluate a non-delta BSDF of compile-time type T (local space, n = +z).
template <int T, bool GRAD>
__device__ __forceinline__ BsdfEval bsdf_eval(const Material& m, float3 wi, float3 wo) {
  BsdfEval e;
  e.f = f3(0.f, 0.f, 0.f);
  e.pdf = 0.0f;
  e.df_alb = f3(0.f, 0.f, 0.f);
  e.df_alpha = f3(0.f, 0.f, 0.f);
  if (!(wi.z > 0.0f) || !(wo.z > 0.0f)) return e;
  if (T == PT_BSDF_DIFFUSE) {
    e.f = m.albedo * PT_INV_PI;
    e.pdf = wo.z * PT_INV_PI;
    if (GRAD) e.df_alb = f3(PT_INV_PI, PT_INV_PI, PT_INV_PI);
  } else if (T == PT_BSDF_CONDUCTOR) {
    e.f = ggx_eval<GRAD>(m.alpha, m.f0, wi, wo, &e.pdf, &e.df_alpha);
  } else if (T == PT_BSDF_BLEND) {
    float pg;
    float3 dga;
    float3 g = ggx_eval<GRAD>(m.alpha, m.f0, wi, wo, &pg, &dga);
    float w = m.wd;
    e.f = m.albedo * (w * PT_INV_PI) + g * (1.0f - w);
    e.pdf = w * wo.z * PT_INV_PI + (1.0f - w) * pg;
    if (GRAD) {
      float k = w * PT_INV_PI;
      e.df_alb = f3(k, k, k);
      e.df_alpha = dga * (1.0f - w);
    }
  }
  return e;
}

// Cosine-weighted hemisphere, mapping of the paper's ambient-occlusion example
// (Sec. 3.1): phi = 2 pi u4, sin^2(theta) = u5.
__device__ __forceinline__ float3 cosine_sample(float u4, float u5) {
  float s, c;
  sincospif(2.0f * u4, &s, &c);  // the angle 2 pi u4 without rounding 2 pi u4 first
  float r = sqrtf(u5);
  return f3(c * r, s * r, sqrtf(1.0f - u5));
}
// Walter et al. 2007: phi = 2 pi u4, tan^2(theta_h) = a^2 u5 / (1 - u5).
__device__ __forceinline__ bool ggx_sample(float a, float3 wi, float u4, float u5, float3& wo) {
  float s, c;
  sincospif(2.0f * u4, &s, &c);  // the angle 2 pi u4 without rounding 2 pi u4 first
  float tan2 = a * a * u5 / (1.0f - u5);
  float ct = rsqrtf(1.0f + tan2);
  float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
  float3 h = f3(st * c, st * s, ct);
  wo = h * (2.0f * dot3(wi, h)) - wi;
  return wo.z > 0.0f;
}

// Exact unpolarised Fresnel of a dielectric interface; eta = n_t / n_i.
__device__ __forceinline__ float fresnel_dielectric(float cos_i, float eta, float& cos_t) {
  float sin2_t = (1.0f - cos_i * cos_i) / (eta * eta);
  if (sin2_t >= 1.0f) {
    cos_t = 0.0f;
    return 1.0f;
  }
  cos_t = sqrtf(1.0f - sin2_t);
  float rs = (cos_i - eta * cos_t) / (cos_i + eta * cos_t);
  float rp = (eta * cos_i - cos_t) / (eta * cos_i + cos_t);
  return 0.5f * (rs * rs + rp * rp);
}

struct BsdfSample {
  float3 wo;       // local
  float3 weight;   // f cos / pdf (delta: the branch weight)
  float pdf;       // solid-angle pdf (0 for delta)
  BsdfEval ev;     // value at wo (non-delta; for the adjoint)
  int lobe;        // 0 diffuse, 1 ggx, 2 reflect, 3 refract
  bool ok, delta;
};

template <int T, bool GRAD>
__device__ __forceinline__ BsdfSample bsdf_sample(const Material& m, float3 wi, bool entering, float u3, float u4,
                                                  float u5) {
  BsdfSample s;
  s.ok = true;
  s.delta = false;
  s.pdf = 0.0f;
  s.lobe = 0;
  s.weight = f3(0.f, 0.f, 0.f);
  if (T == PT_BSDF_DIELECTRIC) {
    float eta = entering ? m.eta : PT_RCP(m.eta);
    float cos_t;
    float F = fresnel_dielectric(wi.z, eta, cos_t);
    s.delta = true;
    if (u3 < F) {
      s.wo = f3(-wi.x, -wi.y, wi.z);
      s.weight = f3(1.f, 1.f, 1.f);
      s.lobe = 2;
    } else {
      float ie = PT_RCP(eta);
      s.wo = f3(-wi.x * ie, -wi.y * ie, -cos_t);
      float k = ie * ie;
      s.weight = f3(k, k, k);
      s.lobe = 3;
    }
    s.ev.f = f3(0.f, 0.f, 0.f);
    return s;
  }
  if (T == PT_BSDF_DIFFUSE) {
    s.wo = cosine_sample(u4, u5);
  } else if (T == PT_BSDF_CONDUCTOR) {
    s.ok = ggx_sample(m.alpha, wi, u4, u5, s.wo);
    s.lobe = 1;
  } else {  // blend
    if (u3 < m.wd) {
      s.wo = cosine_sample(u4, u5);
    } else {
      s.ok = ggx_sample(m.alpha, wi, u4, u5, s.wo);
      s.lobe = 1;
    }
  }
  if (!s.ok) return s;
  s.ev = bsdf_eval<T, GRAD>(m, wi, s.wo);
  s.pdf = s.ev.pdf;
  if (!(s.pdf > 0.0f) || !(max3f(s.ev.f) > 0.0f)) {
    s.ok = false;
    return s;
  }
  s.weight = s.ev.f * (s.wo.z / s.pdf);
  return s;
}

// Polymorphic call over the BSDF type (compile-time dispatch mode).  MATCH: the
// warp votes once per type and runs each type's code with only its lanes active
// (ballot grouping); SWITCH: plain per-lane branch.
// Internal mode for kernels that only ever see one material (the grouped
// wavefront shading kernels): PT_DISPATCH_FIXED + type compiles that type alone.
constexpr int PT_DISPATCH_FIXED = 16;

template <int MODE, class F>
__device__ __forceinline__ void dispatch_bsdf(int type, F&& f) {
  if constexpr (MODE >= PT_DISPATCH_FIXED) {
    if (type == MODE - PT_DISPATCH_FIXED) f.template operator()<MODE - PT_DISPATCH_FIXED>();
  } else if constexpr (MODE == PT_DISPATCH_MATCH) {
    unsigned active = __activemask();
    if (__any_sync(active, type == PT_BSDF_DIFFUSE)) { if (type == PT_BSDF_DIFFUSE) f.template operator()<PT_BSDF_DIFFUSE>(); }
    if (__any_sync(active, type == PT_BSDF_CONDUCTOR)) { if (type == PT_BSDF_CONDUCTOR) f.template operator()<PT_BSDF_CONDUCTOR>(); }
    if (__any_sync(active, type == PT_BSDF_DIELECTRIC)) { if (type == PT_BSDF_DIELECTRIC) f.template operator()<PT_BSDF_DIELECTRIC>(); }
    if (__any_sync(active, type == PT_BSDF_BLEND)) { if (type == PT_BSDF_BLEND) f.template operator()<PT_BSDF_BLEND>(); }
  } else {
    switch (type) {
      case PT_BSDF_DIFFUSE: f.template operator()<PT_BSDF_DIFFUSE>(); break;
      case PT_BSDF_CONDUCTOR: f.template operator()<PT_BSDF_CONDUCTOR>(); break;
      case PT_BSDF_DIELECTRIC: f.template operator()<PT_BSDF_DIELECTRIC>(); break;
      case PT_BSDF_BLEND: f.template operator()<PT_BSDF_BLEND>(); break;
      default: break;
    }
  }
}

// ---------------------------------------------------------------- emitters
__device__ __forceinline__ int cdf_pick(const float* __restrict__ cdf, int n, float u) {
  // first i with u < cdf[i+1]
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (u < __ldg(&cdf[mid + 1])) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Same rule with a guide table: the search is confined to [guide[g], guide[g+1]].
__device__ __forceinline__ int cdf_pick_guided(const float* __restrict__ cdf, const int* __restrict__ guide, int G,
                                               float u) {
  const int g = min((int)(u * (float)G), G - 1);
  int lo = __ldg(&guide[g]), hi = __ldg(&guide[g + 1]);
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (u < __ldg(&cdf[mid + 1])) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ float power_heuristic(float a, float b) {
  float a2 = a * a, b2 = b * b;
  return (a2 + b2) > 0.0f ? a2 / (a2 + b2) : 0.0f;
}

__device__ __forceinline__ void env_pixel(const DevScene& S, float3 d, int& x, int& y) {
  float phi = atan2f(d.z, d.x);
  if (phi < 0.0f) phi += 2.0f * PT_PI;
  float theta = acosf(fminf(1.0f, fmaxf(-1.0f, d.y)));
  x = min((int)(phi * (0.5f * PT_INV_PI) * S.env_w), S.env_w - 1);
  y = min((int)(theta * PT_INV_PI * S.env_h), S.env_h - 1);
}
__device__ __forceinline__ float env_pdf_at(const DevScene& S, int x, int y, float sin_t) {
  if (!(sin_t > 0.0f)) return 0.0f;
  float p = __ldg(&S.env_p[y * S.env_w + x]) * (float)S.env_w * (float)S.env_h;
  return p / (2.0f * PT_PI * PT_PI * sin_t);
}

// ---------------------------------------------------------------- gradient scatter

__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  // smallest p with popc(m & bits[0..p]) > n
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    int p = lo + step - 1;
    unsigned upto = (p >= 31) ? 0xffffffffu : ((2u << p) - 1u);
    if (__popc(m & upto) <= n) lo += step;
  }
  return lo;
}

// Warp-aggregated reduction: lanes with equal `key` (among the currently
// converged lanes) sum their values with a segmented tree of shuffles; the
// group's first lane returns true and holds the sum.
template <int NV>
__device__ __forceinline__ bool warp_aggregate(unsigned key, float (&v)[NV]) {
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
    for (int k = 0; k < NV; ++k) {
      float x = __shfl_sync(active, v[k], src);
      if ((rank & (2 * s - 1)) == 0 && src_rank < n) v[k] += x;
    }
  }
  return rank == 0;
}

}  // namespace ptgb
