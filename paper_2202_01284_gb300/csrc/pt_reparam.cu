// Reparameterized Path Replay Backpropagation for geometry (Sec. 4.7,
// "Reparameterizations"; Sec. 4.8 on the derivative terms of adjacent vertices;
// Sec. 4.10's vertex-position benchmark; warp field after Bangaru et al. 2020).
//
// Parameters: one translation per shape, or every triangle corner's position; a
// surface point keeps its barycentric coordinates.  Every ray the path tracer
// traces -- the camera ray and, at diffuse, GGX-conductor and blend vertices, the
// light-sample ray and the BSDF-sampled ray -- is reparameterized: in the primal
// nothing changes, in the derivative the ray turns by a warp field V and its
// integrand is multiplied by the Jacobian determinant 1 + div V.  A ray therefore
// contributes  M . V(u) + R div V(u),  where R = dLoss/dI . (radiance the ray
// carries) and M the radiance-weighted covector of its integrand's log-derivative
// in the ray direction: R times its measure or cosine term (camera: the pinhole's
// image-plane density, -3 f / f.u; a vertex: the cosine, n / n.u), plus at a glossy
// vertex the BSDF's outgoing-direction gradient, and for the ray that arrives at a
// glossy vertex minus that vertex's incident-direction gradient (so the arriving
// ray is posted one vertex later).
//
// The warp of a ray (origin o, direction u) comes from N auxiliary rays in a von
// Mises-Fisher lobe around u (uniforms from the sample's auxiliary PCG32 stream,
// initseq | 2^62): each one that hits a triangle of plane n_i.(x - o) = d_i says
// that, seen along w, the plane point at distance d_i / (n_i.w) moves relative to
// the origin with Delta_i = tau'(shape_i) - tau'(shape_o) (vertex positions: the
// barycentric combination of the hit triangle's corner velocities at that point,
// minus the origin's).  With per-sample weights
//     alpha_i = exp((kk - kappa)(u.w_i - 1)) g_i,   g_i = (t0 / t_i)^m (1 if the
// ray itself escapes; `miss` for escaping auxiliary rays, which do not move),
// the normalised average C(w) = sum alpha_i(w) Delta_i (n_i.w)/d_i / (sum alpha_i(w)
// + N eps) with alpha_i(w) proportional to exp(kk (w.w_i - 1)) gives the warp
// V = (I - w w^T) C, and differentiating it at u (samples fixed) in closed form:
//     M.V + R div V = sum_i alpha_i / (D d_i) * H_i . Delta_i,
//     H_i = (n_i.u)(M_perp + R (kk p_i - 2u - kk P / D)) + R (I - u u^T) n_i,
// with p_i = (I - u u^T) w_i, P = sum alpha_j p_j, D = sum alpha_j + N eps.  The
// ratio's O(1/N) bias is removed by the leave-one-out (jackknife) combination
// N f(all) - (N-1)/N sum_j f(all but j), evaluated with two extra sums.  For the
// camera ray the warp may be multiplied by a window b that reaches 0 at the image
// border (option), adding R grad(b) . C.  Because every term is linear in the velocities,
// the reverse-mode gradient of a ray is the coefficient vector of each Delta_i: it
// is added to the hit's shape (or triangle corners) and subtracted from the
// origin's.
//
// Launch: the split-PRB radiance pass (each sample's radiance), then one thread per
// (pixel, lane) replays its samples in lockstep with the other lanes of its warp,
// which trace the auxiliary rays of the posted rays together.  Translation
// gradients are accumulated per CTA in shared memory when the shape table fits.
// Then one thread per (pixel edge, sample) adds the pixel-edge term: the camera
// warp moves the box-filtered pixels' footprints too.  The forward mode (at the end
// of the file) runs the same warps in one pass along a direction of translations.
#include "pt_mega.cuh"

namespace ptgb {
namespace {

constexpr int kMaxAux = 32;

struct RpOpts {
  int n_aux, jackknife, smem, group;  // group: lanes per cooperative warp, a power of two >= n_aux
  float kappa, kk, power, miss, eps, border, e2k;
  int edge_spp;
};

// One out-of-line traversal shared by all call sites (path, shadow, center and
// auxiliary rays): inlining it at each of them multiplied the kernel's code and
// its instruction-cache misses.
template <int LAYOUT, bool INSTR>
__device__ __noinline__ Hit closest(const DevScene& S, float3 o, float3 d, float tmax, bool any,
                                    Counters<INSTR>& cnt) {
  return LAYOUT == PT_BVH_WIDE ? trace_wide<INSTR>(S, o, d, tmax, any, cnt)
                               : trace_binary<INSTR>(S, o, d, tmax, any, cnt);
}

__device__ __forceinline__ int tri_shape(const DevScene& S, int pos) {
  return __float_as_int(__ldg(&S.tri_a[2 * pos + 1]).z);
}
__device__ __forceinline__ float3 tri_normal(const DevScene& S, int pos) {
  return normalize3(cross3(xyz(__ldg(&S.tri_v[3 * pos + 1])), xyz(__ldg(&S.tri_v[3 * pos + 2]))));
}

// vMF direction around u (Jakob 2012): cos(theta) - 1 = log(xi + (1 - xi) e^{-2 kappa})
// / kappa with xi = 1 - u0, phi = 2 pi u1; returns the direction and cos(theta) - 1.
__device__ __forceinline__ float3 vmf_dir(const Frame& fr, float u0, float u1, const RpOpts& K, float& c1) {
  const float xi = 1.0f - u0;
  c1 = logf(xi + (1.0f - xi) * K.e2k) / K.kappa;
  const float st = sqrtf(fmaxf(0.0f, -c1 * (2.0f + c1)));
  float sp, cp;
  sincospif(2.0f * u1, &sp, &cp);
  return normalize3(fr.s * (st * cp) + fr.t * (st * sp) + fr.n * (1.0f + c1));
}

// Image-plane coordinates (pixels, y down) of direction u and their gradients with
// respect to u (the camera's right / up vectors carry the half-extents of the
// image plane at unit distance).
__device__ __forceinline__ void pixel_coords(const LaunchArgs& A, const DevCamera& c, float3 u, float& px, float& py,
                                             float3& gpx, float3& gpy) {
  const float3 f = f3(c.fx, c.fy, c.fz), rs = f3(c.rx, c.ry, c.rz), us = f3(c.ux, c.uy, c.uz);
  const float fw = dot3(f, u), rr = dot3(rs, rs), uu = dot3(us, us);
  const float sx = dot3(rs, u) / (fw * rr), sy = dot3(us, u) / (fw * uu);
  const float W = (float)A.width, H = (float)A.height;
  px = (sx + 1.0f) * 0.5f * W;
  py = (1.0f - sy) * 0.5f * H;
  gpx = (rs - f * (dot3(rs, u) / fw)) * (0.5f * W / (rr * fw));
  gpy = (us - f * (dot3(us, u) / fw)) * (-0.5f * H / (uu * fw));
}

// Window of the camera warp: smoothstep of the distance in pixels to the nearest
// image border over `border` pixels; b and its gradient on the sphere at u.  No
// window (b = 1) for border = 0: the pixel-edge term then carries the flux through
// the image border.
__device__ __forceinline__ float cam_window(const LaunchArgs& A, const DevCamera& c, float3 u, float border,
                                            float3& grad) {
  if (border <= 0.0f) {
    grad = f3(0.f, 0.f, 0.f);
    return 1.0f;
  }
  const float W = (float)A.width, H = (float)A.height;
  float px, py;
  float3 gpx, gpy;
  pixel_coords(A, c, u, px, py, gpx, gpy);
  float d = px;
  float3 gd = gpx;
  if (W - px < d) { d = W - px; gd = -gpx; }
  if (py < d) { d = py; gd = gpy; }
  if (H - py < d) { d = H - py; gd = -gpy; }
  const float t = d / border;
  if (t >= 1.0f || t <= 0.0f) {
    grad = f3(0.f, 0.f, 0.f);
    return t >= 1.0f ? 1.0f : 0.0f;
  }
  const float3 g = gd * (6.0f * t * (1.0f - t) / border);
  grad = g - u * dot3(u, g);
  return t * t * (3.0f - 2.0f * t);
}

// (t0 / t)^power of the warp's depth weight; the default power 2 as one product (the
// correctly rounded square; powf is only guaranteed within a few ulp of it)
__device__ __forceinline__ float depth_weight(float q, float power) { return power == 2.0f ? q * q : powf(q, power); }

struct GradOut {
  float* dst;  // shared (per CTA) or global [n_shapes][3]
  __device__ __forceinline__ void add(int s, float3 g) {
    atomicAdd(&dst[3 * s], g.x);
    atomicAdd(&dst[3 * s + 1], g.y);
    atomicAdd(&dst[3 * s + 2], g.z);
  }
};

constexpr unsigned kFull = 0xffffffffu;

// Jump a PCG32 stream ahead by `delta` draws in O(log delta) (Brown 1994,
// "Random number generation with arbitrary strides": compose the LCG step).
__device__ __forceinline__ void pcg_advance(Pcg32& r, unsigned long long delta) {
  unsigned long long acc_mult = 1ull, acc_plus = 0ull, cur_mult = 6364136223846793005ull, cur_plus = r.inc;
  while (delta) {
    if (delta & 1ull) {
      acc_mult *= cur_mult;
      acc_plus = acc_plus * cur_mult + cur_plus;
    }
    cur_plus = (cur_mult + 1ull) * cur_plus;
    cur_mult *= cur_mult;
    delta >>= 1;
  }
  r.state = acc_mult * r.state + acc_plus;
}

// A reparameterized ray waiting for its warp: origin, direction, the covector M of
// its integrand's log-derivative in the ray direction weighted by the radiance it
// carries (R times the cosine / measure term, plus the BSDF's directional terms),
// origin shape (-1: camera), camera index for the window (-1: none), weight R =
// dLoss/dI . radiance, its own hit distance and the auxiliary stream at its first
// uniform.  Its derivative is M . V + R div V.
struct WarpRay {
  float3 o, u, m;
  int s_o, cam;
  float R, t0;
  unsigned long long st, inc;
  int o_tri;         // vertex mode: original id of the origin's triangle (-1: camera)
  float o_bu, o_bv;  // and the origin's barycentric coordinates on it
};

// Vertex mode output: corner k of original triangle t at [t][k][0..2].
struct VertOut {
  float* dst;
  __device__ __forceinline__ void add(int t, const float3 (&g)[3]) {
    float* d = dst + 9 * (size_t)t;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(d + 3 * k, g[k].x);
      atomicAdd(d + 3 * k + 1, g[k].y);
      atomicAdd(d + 3 * k + 2, g[k].z);
    }
  }
};
__device__ __forceinline__ int tri_orig(const DevScene& S, int pos) {
  return (int)__float_as_uint(__ldg(&S.tri_v[3 * pos]).w);
}

__device__ __forceinline__ float3 shfl3(float3 v, int src) {
  return f3(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src), __shfl_sync(kFull, v.z, src));
}
// sum over the aligned group of `gs` lanes (gs a power of two)
__device__ __forceinline__ float group_sum(float v, int gs) {
  for (int off = gs >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}
__device__ __forceinline__ float3 group_sum3(float3 v, int gs) {
  return f3(group_sum(v.x, gs), group_sum(v.y, gs), group_sum(v.z, gs));
}

// Warp-cooperative warps: called by all 32 lanes together.  The lanes form
// 32 / gs groups of gs >= N lanes; each round every group takes one pending ray
// of some lane, and its lane j traces auxiliary ray j of that ray (the rays of a
// lobe are coherent), so the reductions of the warp estimator are shuffles.
template <int LAYOUT, bool INSTR, bool VERT>
__device__ __noinline__ unsigned process_warps(const LaunchArgs& A, const RpOpts& K, bool has, const WarpRay& mine,
                                               GradOut& G, VertOut& GV, Counters<INSTR>& cnt) {
  const DevScene& S = A.scene;
  const int lane = lane_id(), gs = K.group, grp = lane / gs, j = lane % gs;
  const int ng = 32 / gs;
  const float dk = K.kk - K.kappa, n = (float)K.n_aux;
  unsigned rays = 0;
  unsigned pend = __ballot_sync(kFull, has);
  while (pend) {
    unsigned p = pend;
    for (int g = 0; g < grp && p; ++g) p &= p - 1;
    const int src = p ? __ffs(p) - 1 : -1;
    for (int g = 0; g < ng && pend; ++g) pend &= pend - 1;
    const int sl = src >= 0 ? src : lane;
    WarpRay w;
    w.o = shfl3(mine.o, sl);
    w.u = shfl3(mine.u, sl);
    w.m = shfl3(mine.m, sl);
    w.s_o = __shfl_sync(kFull, mine.s_o, sl);
    w.cam = __shfl_sync(kFull, mine.cam, sl);
    w.R = __shfl_sync(kFull, mine.R, sl);
    w.t0 = __shfl_sync(kFull, mine.t0, sl);
    w.st = __shfl_sync(kFull, mine.st, sl);
    w.inc = __shfl_sync(kFull, mine.inc, sl);
    if constexpr (VERT) {
      w.o_tri = __shfl_sync(kFull, mine.o_tri, sl);
      w.o_bu = __shfl_sync(kFull, mine.o_bu, sl);
      w.o_bv = __shfl_sync(kFull, mine.o_bv, sl);
    }
    const bool on = src >= 0 && j < K.n_aux;
    float alpha = 0.0f, t = 0.0f;
    int pos = -1;
    float3 wi = w.u, pi = f3(0.f, 0.f, 0.f);
    if (on) {
      Pcg32 r;
      r.state = w.st;
      r.inc = w.inc;
      pcg_advance(r, 2ull * (unsigned long long)j);
      const float a0 = r.uniform(), a1 = r.uniform();
      float c1;
      wi = vmf_dir(make_frame(w.u), a0, a1, K, c1);
      const Hit h = closest<LAYOUT, INSTR>(S, w.o, wi, INFINITY, false, cnt);
      ++rays;
      float g = K.miss;
      if (h.pos >= 0) g = w.t0 < INFINITY ? depth_weight(__fdiv_rn(w.t0, fmaxf(h.t, 1e-3f * w.t0)), K.power) : 1.0f;
      alpha = expf(dk * c1) * g;
      pos = h.pos;
      t = h.t;
      pi = wi - w.u * dot3(w.u, wi);
    }
    const float D = group_sum(alpha, gs) + n * K.eps;
    const float3 P = group_sum3(pi * alpha, gs);
    float S1 = 0.0f;
    float3 SP = f3(0.f, 0.f, 0.f);
    if (K.jackknife) {
      const float Dj = D - alpha - K.eps;
      const float3 Pj = P - pi * alpha;
      S1 = group_sum(on ? PT_RCP(Dj) : 0.0f, gs);
      SP = group_sum3(on ? Pj * PT_RCP(Dj * Dj) : f3(0.f, 0.f, 0.f), gs);
    }
    float3 gv = f3(0.f, 0.f, 0.f);  // coefficient of the relative translation (origin part)
    int si = -1;
    if (on && pos >= 0) si = tri_shape(S, pos);
    const bool contrib = VERT ? pos >= 0 : (si >= 0 && si != w.s_o);
    if (contrib) {
      float b = 1.0f;
      float3 gb = f3(0.f, 0.f, 0.f);
      if (w.cam >= 0) b = cam_window(A, A.cams[w.cam], w.u, K.border, gb);
      const float3 mp = w.m - w.u * dot3(w.u, w.m);
      const float3 nrm = tri_normal(S, pos);
      const float di = dot3(nrm, wi) * t;
      const float3 base = (mp + (pi * K.kk - w.u * 2.0f) * w.R) * b;  // M_perp + R (kk p - 2u), windowed
      float Dm = 0.0f;
      float3 Pm = f3(0.f, 0.f, 0.f);
      if (K.jackknife) {
        Dm = D - alpha - K.eps;
        Pm = P - pi * alpha;
      }
      // coefficient of a velocity field s(w) Delta with s linear in w: gradient g = (I - uu^T) grad s
      auto coef_of = [&](float sv, float3 g) {
        const float3 Ai = base * sv + (g * b + gb * sv) * w.R;
        const float kb = K.kk * b * sv * w.R;
        float3 c = Ai * PT_RCP(D) - P * __fdiv_rn(kb, D * D);
        if (K.jackknife) {
          const float3 loo = Ai * (S1 - PT_RCP(Dm)) - (SP - Pm * PT_RCP(Dm * Dm)) * kb;
          c = c * n - loo * __fdiv_rn(n - 1.0f, n);
        }
        return c * alpha;
      };
      // plane point seen along w: 1/t(w) = (n.w)/d; the origin moves as a whole
      gv = coef_of(__fdiv_rn(dot3(nrm, w.u), di), (nrm - w.u * dot3(nrm, w.u)) * PT_RCP(di));
      if constexpr (VERT) {
        // corner j of the hit triangle carries b_j(w)/t(w) = beta_j (n.w)/d + a_j.w with
        // a_1 = (e2 x c)/c.c, a_2 = (c x e1)/c.c, a_0 = -(a_1 + a_2), beta_j = a_j.(o - v0) + [j = 0]
        const float3 v0 = xyz(__ldg(&S.tri_v[3 * pos]));
        const float3 e1 = xyz(__ldg(&S.tri_v[3 * pos + 1])), e2 = xyz(__ldg(&S.tri_v[3 * pos + 2]));
        const float3 c = cross3(e1, e2);
        const float icc = PT_RCP(dot3(c, c));
        const float3 a1 = cross3(e2, c) * icc, a2 = cross3(c, e1) * icc;
        const float3 a0 = -(a1 + a2);
        const float3 ov = w.o - v0;
        const float nu = __fdiv_rn(dot3(nrm, w.u), di);
        const float3 nperp = (nrm - w.u * dot3(nrm, w.u)) * PT_RCP(di);
        float3 gc[3];
        const float3 aj[3] = {a0, a1, a2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float beta = dot3(aj[k], ov) + (k == 0 ? 1.0f : 0.0f);
          gc[k] = coef_of(beta * nu + dot3(aj[k], w.u), nperp * beta + (aj[k] - w.u * dot3(aj[k], w.u)));
        }
        float v[9] = {gc[0].x, gc[0].y, gc[0].z, gc[1].x, gc[1].y, gc[1].z, gc[2].x, gc[2].y, gc[2].z};
        const int to = tri_orig(S, pos);
        if (warp_aggregate<9>((unsigned)to, v)) {
          const float3 g3[3] = {f3(v[0], v[1], v[2]), f3(v[3], v[4], v[5]), f3(v[6], v[7], v[8])};
          GV.add(to, g3);
        }
      } else {
        float v[3] = {gv.x, gv.y, gv.z};
        if (warp_aggregate<3>((unsigned)si, v)) G.add(si, f3(v[0], v[1], v[2]));
      }
    }
    // the origin moves with its own shape (or triangle corners): minus the group's total
    const float3 go = group_sum3(gv, gs);
    if (j == 0 && src >= 0 && (go.x != 0.0f || go.y != 0.0f || go.z != 0.0f)) {
      if constexpr (VERT) {
        if (w.o_tri >= 0) {
          const float bo[3] = {1.0f - w.o_bu - w.o_bv, w.o_bu, w.o_bv};
          const float3 g3[3] = {-go * bo[0], -go * bo[1], -go * bo[2]};
          GV.add(w.o_tri, g3);
        }
      } else if (w.s_o >= 0) {
        G.add(w.s_o, -go);
      }
    }
  }
  return rays;
}

// Gradients of log f_c with respect to the outgoing (go) and incident (gi)
// directions, local frame (n = +z), for the glossy BSDFs: GGX conductor, and the
// blend w albedo/pi + (1 - w) GGX; zero for diffuse.  With h = (wi + wo)/|wi + wo|,
// f = F(c_d) D(c_h) G1(c_i) G1(c_o) / (4 c_i c_o), c_d = wi.h = |wi + wo|/2:
// d log D / d c_h = -4 c_h (a^2 - 1) / (c_h^2 (a^2 - 1) + 1), d c_h / d w = (z - h c_h)/|wi + wo|,
// d log G1 / d c = a^2 / (r c^3 (1 + r)) with r = sqrt(1 + a^2 (1 - c^2)/c^2),
// d log F_c / d c_d = -5 (1 - F0_c)(1 - c_d)^4 / F_c with d c_d / d w = h/2 (tangentially).
__device__ void glossy_log_grad(int type, float alpha, float3 f0, float wd, float3 albedo, float3 wi, float3 wo,
                                float3 (&go)[3], float3 (&gi)[3]) {
  for (int c = 0; c < 3; ++c) go[c] = gi[c] = f3(0.f, 0.f, 0.f);
  if (type != PT_BSDF_CONDUCTOR && type != PT_BSDF_BLEND) return;
  if (!(wi.z > 0.0f) || !(wo.z > 0.0f)) return;
  const float3 zz = f3(0.f, 0.f, 1.f);
  const float3 sv = wi + wo;
  const float sl = sqrtf(dot3(sv, sv));
  const float3 h = sv * (1.0f / sl);
  const float ch = h.z, cd = 0.5f * sl, a2 = alpha * alpha;
  const float den = ch * ch * (a2 - 1.0f) + 1.0f;
  const float3 common = (zz - h * ch) * (-4.0f * ch * (a2 - 1.0f) / (den * sl));
  auto G1 = [&](float c, float& dlog) {
    const float r = sqrtf(1.0f + a2 * (1.0f - c * c) / (c * c));
    dlog = a2 / (r * c * c * c * (1.0f + r));
    return 2.0f / (1.0f + r);
  };
  float dgi, dgo;
  const float G = G1(wi.z, dgi) * G1(wo.z, dgo);
  const float3 bo = common + zz * (dgo - 1.0f / wo.z);
  const float3 bi = common + zz * (dgi - 1.0f / wi.z);
  const float k = a2 / (PT_PI * den * den) * G / (4.0f * wi.z * wo.z);
  const float m = 1.0f - cd, m4 = m * m * m * m;
  const float f0c[3] = {f0.x, f0.y, f0.z}, alb[3] = {albedo.x, albedo.y, albedo.z};
  for (int c = 0; c < 3; ++c) {
    const float F = f0c[c] + (1.0f - f0c[c]) * m4 * m;
    const float3 gF = h * (F > 0.0f ? -2.5f * (1.0f - f0c[c]) * m4 / F : 0.0f);
    float share = 1.0f;  // fraction of f_c that depends on the directions
    if (type == PT_BSDF_BLEND) {
      const float fg = (1.0f - wd) * k * F;
      const float f = wd * alb[c] * PT_INV_PI + fg;
      share = f > 0.0f ? fg / f : 0.0f;
    }
    go[c] = (bo + gF) * share;
    gi[c] = (bi + gF) * share;
  }
}

// The glossy parameters of the material at a hit (as path_shade resolves them).
struct Gloss {
  int type;
  float alpha, wd;
  float3 f0, albedo;
};
__device__ Gloss gloss_at(const LaunchArgs& A, const Hit& hit) {
  const DevScene& S = A.scene;
  Gloss g;
  const float4 ta0 = __ldg(&S.tri_a[2 * hit.pos]);
  const float4 ta1 = __ldg(&S.tri_a[2 * hit.pos + 1]);
  const int4* shp = reinterpret_cast<const int4*>(&S.shapes[__float_as_int(ta1.z)]);
  const int4 sw0 = __ldg(shp);
  const float4 sw1 = __ldg(reinterpret_cast<const float4*>(shp + 1));
  g.type = sw0.x;
  g.alpha = sw0.w >= 0 ? __ldg(&A.params.rough[sw0.w]) : sw1.x;
  g.wd = sw1.z;
  g.f0 = xyz(__ldg(reinterpret_cast<const float4*>(shp + 2)));
  g.albedo = f3(0.f, 0.f, 0.f);
  if (g.type == PT_BSDF_BLEND) {
    if (sw0.y >= 0) {
      const float b0 = 1.0f - hit.u - hit.v;
      const float tu = b0 * ta0.x + hit.u * ta0.z + hit.v * ta1.x;
      const float tv = b0 * ta0.y + hit.u * ta0.w + hit.v * ta1.y;
      const int w = A.params.tex_w[sw0.y], h = A.params.tex_h[sw0.y];
      const int x = min((int)(fmaxf(tu, 0.0f) * (float)w), w - 1);
      const int y = min((int)(fmaxf(tv, 0.0f) * (float)h), h - 1);
      g.albedo = xyz(__ldg(&A.params.tex[sw0.y][y * w + x]));
    } else if (sw0.z >= 0) {
      const float* a = &A.params.albedo[3 * sw0.z];
      g.albedo = f3(__ldg(a), __ldg(a + 1), __ldg(a + 2));
    }
  }
  return g;
}

// Vertex mode: gradient with respect to the corners of the triangle at leaf position
// pos of scale log|n . u| + q . n, n its unit geometric normal (q: a covector on the
// normal's change, here from a glossy BSDF).  With c = e1 x e2 and w = (p - n (n.p))
// / |c|, p = scale u / (n.u) + q: d(...) = dn . p = de1.(e2 x w) + de2.(w x e1).
__device__ __forceinline__ void normal_log_grad(const DevScene& S, int pos, float3 u, float scale, float3 q,
                                                float3 (&g)[3]) {
  const float3 e1 = xyz(__ldg(&S.tri_v[3 * pos + 1])), e2 = xyz(__ldg(&S.tri_v[3 * pos + 2]));
  const float3 c = cross3(e1, e2);
  const float len = sqrtf(dot3(c, c));
  const float3 nn = c * (1.0f / len);
  const float3 p = u * (scale / dot3(nn, u)) + q;
  const float3 w = (p - nn * dot3(nn, p)) * (1.0f / len);
  g[1] = cross3(e2, w);
  g[2] = cross3(w, e1);
  g[0] = -(g[1] + g[2]);
}

// Lockstep loop: each iteration every lane advances the PRB replay of its current
// sample by one vertex (its radiance comes from the radiance pass launched before,
// as in split PRB), then the whole warp processes the reparameterized rays the
// lanes posted.
// VERT: gradients of every triangle corner's position (grad_v [n_tris][3][3]);
// otherwise of one translation per shape (grad_t [n_shapes][3]).  Capped at 64
// registers (8 CTAs of 128 per SM): on the sphere workload the occupancy gained
// outweighs the spills (uncapped 168 registers: 173 ms; 128: 148; 96: 135; 80: 130;
// 64: 127).
template <int LAYOUT, bool INSTR, bool VERT>
__global__ void __launch_bounds__(128, 8) reparam_kernel(const __grid_constant__ LaunchArgs A, const RpOpts K,
                                                      float* __restrict__ grad_t, float* __restrict__ grad_v,
                                                      unsigned long long* rays_out) {
  extern __shared__ float s_grad[];
  const int n3 = 3 * A.scene.n_shapes;
  if (K.smem) {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) s_grad[i] = 0.0f;
    __syncthreads();
  }
  GradOut G{K.smem ? s_grad : grad_t};
  VertOut GV{grad_v};
  const DevScene& S = A.scene;
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PixelOf px{};
  const bool valid = unit_pixel(A, unit, crop_tile(A), px);
  unsigned rays = 0;
  Counters<INSTR> cnt;
  if constexpr (INSTR)
    for (int i = 0; i < kCounters; ++i) cnt.c[i] = 0;
  const float3 z = f3(0.f, 0.f, 0.f);
  float3 dl = z, fwd = z;
  if (valid) {
    const float inv = 1.0f / (float)A.spp;
    dl = f3(A.grad_image[3 * px.pix] * inv, A.grad_image[3 * px.pix + 1] * inv, A.grad_image[3 * px.pix + 2] * inv);
    const DevCamera& cam = A.cams[px.cam];
    fwd = f3(cam.fx, cam.fy, cam.fz);
  }
  bool live = false;
  int si = (int)(unit & (A.lanes_per_pixel - 1));
  GradSink sink;
  PathState P;
  Pcg32 aux;
  aux.state = aux.inc = 0ull;
  bool cached = false;
  Hit next{};
  // The ray that arrives at the lane's next vertex (camera or BSDF ray): posted after
  // that vertex, whose glossy BSDF may add terms for its incident direction.
  WarpRay arr{};
  bool has_arr = false;
  const unsigned long long n2 = 2ull * (unsigned long long)K.n_aux;
  for (;;) {
    WarpRay w0{}, w1{};
    bool h0 = false, h1 = false;
    if (!live && valid && si < A.spp) {
      // start the replay of sample si: primary stream as the radiance pass,
      // auxiliary stream initseq | 2^62; the camera ray is the first warp
      path_start<INSTR>(A, P, A.seed, px.cam, px.px, px.py, si, px.pix, cnt);
      const float* Ls = A.sample_L + 3 * P.slot;
      P.Lrem = f3(Ls[0], Ls[1], Ls[2]);
      const unsigned long long pixel = (unsigned long long)px.py * (unsigned long long)A.width + px.px;
      aux.seed(A.seed, ((unsigned long long)px.cam << 40) | (pixel << 12) | (unsigned long long)si | (1ull << 62));
      next = closest<LAYOUT, INSTR>(S, P.ro, P.rd, INFINITY, false, cnt);
      ++rays;
      cached = true;
      const float R = dot3(dl, P.Lrem);
      arr = WarpRay{P.ro, P.rd, fwd * (-3.0f * R / dot3(fwd, P.rd)), -1, px.cam, R,
                    next.pos >= 0 ? next.t : INFINITY, aux.state, aux.inc, -1, 0.0f, 0.0f};
      has_arr = true;
      pcg_advance(aux, n2);
      live = true;
    } else if (live) {
      Hit hit;
      if (cached) {  // traced already as the center ray of the previous warp
        hit = next;
        cached = false;
      } else {
        hit = closest<LAYOUT, INSTR>(S, P.ro, P.rd, INFINITY, false, cnt);
        ++rays;
      }
      ++rays;  // its twin in the radiance pass
      const bool block = hit.pos >= 0 && P.depth < A.max_depth;
      int s_o = -1, o_tri = -1;
      float3 n_s = z, ng = z;
      const float3 wi_w = -P.rd;
      if (hit.pos >= 0) {
        s_o = tri_shape(S, hit.pos);
        o_tri = tri_orig(S, hit.pos);
        ng = tri_normal(S, hit.pos);
        n_s = dot3(ng, P.rd) < 0.0f ? ng : -ng;
      }
      bool more = path_shade<false, false, INSTR, PT_DISPATCH_SWITCH, FEAT_NOHASH>(A, P, hit, false, z, sink, cnt);
      Pcg32 aux_nee = aux, aux_bsdf = aux;
      if (block) {
        pcg_advance(aux_bsdf, n2);
        pcg_advance(aux, 2ull * n2);
      }
      float3 inc = z;  // covector of this vertex's terms in its incident direction (weighted)
      WarpRay out{};
      bool has_out = false;
      if (more) {
        bool occ = false;
        if (P.has_shadow) {
          occ = closest<LAYOUT, INSTR>(S, P.so, P.sd, P.stmax, true, cnt).pos >= 0;
          rays += 2;
        }
        const int mt = P.mtype;
        const bool warp = block && (mt == PT_BSDF_DIFFUSE || mt == PT_BSDF_CONDUCTOR || mt == PT_BSDF_BLEND);
        const bool glossy = warp && mt != PT_BSDF_DIFFUSE;
        Gloss gl{};
        Frame fr{};
        float3 wi_l = z;
        if (glossy) {
          gl = gloss_at(A, hit);
          fr = make_frame(n_s);
          wi_l = fr.to_local(wi_w);
        }
        // covector of the term C (per channel) leaving along d: R n/(n.d) plus, at a
        // glossy vertex, sum_c dl_c C_c grad_out log f_c; adds to `inc` the incident part.
        // Vertex mode: the glossy value also depends on the turning normal; f is
        // unchanged when n, wi and wo turn together, so for a turn n' = w x n (w = n x n')
        // d log f = -w . (wi x grad_in + wo x grad_out) = n' . (n x J): qn = ng x J, the
        // same for either orientation of the normal.
        float3 qn = z;
        auto covector = [&](float3 d, float3 C, float R) {
          float3 M = n_s * (R / dot3(n_s, d));
          qn = z;
          if (glossy) {
            float3 go[3], gi[3];
            glossy_log_grad(gl.type, gl.alpha, gl.f0, gl.wd, gl.albedo, wi_l, fr.to_local(d), go, gi);
            const float wc[3] = {dl.x * C.x, dl.y * C.y, dl.z * C.z};
            float3 Go = z, Gi = z;
            for (int c = 0; c < 3; ++c) {
              Go = Go + fr.to_world(go[c]) * wc[c];
              Gi = Gi + fr.to_world(gi[c]) * wc[c];
            }
            M = M + Go;
            inc = inc + Gi;
            if constexpr (VERT) qn = cross3(ng, cross3(wi_w, Gi) + cross3(d, Go));
          }
          return M;
        };
        if (warp && P.has_shadow && !occ) {
          const float R = dot3(dl, P.c_nee);
          const float3 M = covector(P.sd, P.c_nee, R);
          if (R != 0.0f || M.x != 0.0f || M.y != 0.0f || M.z != 0.0f) {
            const Hit hl = closest<LAYOUT, INSTR>(S, P.so, P.sd, INFINITY, false, cnt);
            ++rays;
            w0 = WarpRay{P.so, P.sd, M, s_o, -1, R, hl.pos >= 0 ? hl.t : INFINITY, aux_nee.state, aux_nee.inc,
                         o_tri, hit.u, hit.v};
            h0 = true;
            if constexpr (VERT) {
              float3 gn[3];
              normal_log_grad(S, hit.pos, P.sd, R, qn, gn);
              GV.add(o_tri, gn);
            }
          }
        }
        more = path_finish<false, false, INSTR, FEAT_NOHASH>(A, P, occ, false, z, sink, cnt);
        if (more && warp) {
          const float3 C = f3(fmaxf(P.Lrem.x, 0.f), fmaxf(P.Lrem.y, 0.f), fmaxf(P.Lrem.z, 0.f));
          const float R = dot3(dl, C);
          const float3 M = covector(P.rd, C, R);
          next = closest<LAYOUT, INSTR>(S, P.ro, P.rd, INFINITY, false, cnt);
          ++rays;
          cached = true;
          out = WarpRay{P.ro, P.rd, M, s_o, -1, R, next.pos >= 0 ? next.t : INFINITY, aux_bsdf.state,
                        aux_bsdf.inc, o_tri, hit.u, hit.v};
          has_out = true;
          if constexpr (VERT) {
            if (R != 0.0f || qn.x != 0.0f || qn.y != 0.0f || qn.z != 0.0f) {
              float3 gn[3];
              normal_log_grad(S, hit.pos, P.rd, R, qn, gn);
              GV.add(o_tri, gn);
            }
          }
        }
      }
      // the ray that arrived here: its direction is minus this vertex's incident one
      if (has_arr) {
        arr.m = arr.m - inc;
        if (arr.R != 0.0f || arr.m.x != 0.0f || arr.m.y != 0.0f || arr.m.z != 0.0f) {
          w1 = arr;
          h1 = true;
        }
      }
      arr = out;
      has_arr = has_out;
      if (!more) {
        live = false;
        si += A.lanes_per_pixel;
      }
    }
    if (!__any_sync(kFull, live || h0 || h1 || (valid && si < A.spp))) break;
    rays += process_warps<LAYOUT, INSTR, VERT>(A, K, h0, w0, G, GV, cnt);
    rays += process_warps<LAYOUT, INSTR, VERT>(A, K, h1, w1, G, GV, cnt);
  }
  if (K.smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x)
      if (s_grad[i] != 0.0f) atomicAdd(&grad_t[i], s_grad[i]);
  }
  if (rays_out) {
    unsigned long long r = rays;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
    if (lane_id() == 0 && r) atomicAdd(rays_out, r);
  }
  flush_counters<INSTR>(A, cnt);
}

// Edges of the crop that carry the pixel-edge term, per camera: vertical edges
// x = xlo .. xlo + nvx - 1 of every crop row, then horizontal edges y = ylo .. ylo +
// nhy - 1 of every crop column (all edges of the crop's pixels).
struct EdgeGrid {
  int xlo, nvx, ylo, nhy;
  long long per_cam;
};

// The edge and sample of a unit of the edge kernels (per camera: the vertical
// edges row by row, then the horizontal ones), its PCG32 stream and the pixel
// index of (x, y) in the crop (-1 outside).
struct EdgeSample {
  int ci, X, Y;
  bool vertical;
  unsigned long long stream;
};
__device__ __forceinline__ EdgeSample edge_of(const LaunchArgs& A, const RpOpts& K, const EdgeGrid& E,
                                              long long unit) {
  EdgeSample es;
  const int k = (int)(unit % K.edge_spp);
  const long long ea = unit / K.edge_spp;
  es.ci = (int)(ea / E.per_cam);
  long long e = ea - (long long)es.ci * E.per_cam;
  const long long nv = (long long)A.crop_h * E.nvx;
  es.vertical = e < nv;
  unsigned long long id;
  if (es.vertical) {
    es.Y = A.crop_y0 + (int)(e / E.nvx);
    es.X = E.xlo + (int)(e % E.nvx);
    id = (unsigned long long)es.Y * (unsigned long long)(A.width + 1) + (unsigned long long)es.X;
  } else {
    e -= nv;
    es.Y = E.ylo + (int)(e / A.crop_w);
    es.X = A.crop_x0 + (int)(e % A.crop_w);
    id = (unsigned long long)(A.width + 1) * (unsigned long long)A.height +
         (unsigned long long)es.Y * (unsigned long long)A.width + (unsigned long long)es.X;
  }
  es.stream = ((unsigned long long)es.ci << 40) | (id << 12) | (unsigned long long)k | (1ull << 61);
  return es;
}
__device__ __forceinline__ long long crop_pixel(const LaunchArgs& A, int ci, int x, int y) {
  if (x < A.crop_x0 || x >= A.crop_x0 + A.crop_w || y < A.crop_y0 || y >= A.crop_y0 + A.crop_h) return -1;
  return ((long long)ci * A.crop_h + (y - A.crop_y0)) * A.crop_w + (x - A.crop_x0);
}

// The path through a uniform point of the edge (the point's uniform first, then
// the unused second one, then the path's): its radiance, its camera ray (o, u) and
// that ray's hit distance (infinite if it escapes).
template <int LAYOUT, bool INSTR>
__device__ __forceinline__ float3 edge_path(const LaunchArgs& A, const EdgeSample& es, float3& o, float3& u,
                                            float& t0, unsigned& rays, Counters<INSTR>& cnt) {
  const float3 z = f3(0.f, 0.f, 0.f);
  PathState P;
  P.slot = 0;
  P.cache_done = false;
  P.rng.seed(A.seed, es.stream);
  P.fh.h = 2166136261u;
  const float j0 = P.rng.uniform();
  P.rng.uniform();
  path_start_at<INSTR>(A, P, es.ci, es.vertical ? (float)es.X : (float)es.X + j0,
                       es.vertical ? (float)es.Y + j0 : (float)es.Y, cnt);
  o = P.ro;
  u = P.rd;
  t0 = INFINITY;
  GradSink sink;
  for (bool first = true;; first = false) {
    const Hit hit = closest<LAYOUT, INSTR>(A.scene, P.ro, P.rd, INFINITY, false, cnt);
    ++rays;
    if (first && hit.pos >= 0) t0 = hit.t;
    if (!path_shade<false, false, INSTR, PT_DISPATCH_SWITCH, FEAT_NOHASH>(A, P, hit, false, z, sink, cnt)) break;
    bool occ = false;
    if (P.has_shadow) {
      occ = closest<LAYOUT, INSTR>(A.scene, P.so, P.sd, P.stmax, true, cnt).pos >= 0;
      ++rays;
    }
    if (!path_finish<false, false, INSTR, FEAT_NOHASH>(A, P, occ, false, z, sink, cnt)) break;
  }
  return P.L;
}

// Pixel-edge term of the camera-ray warp (box pixel filter).  The warp that holds
// the discontinuities still also moves every pixel's footprint, a unit box in pixel
// coordinates: its boundary moves with minus the warp's image-plane velocity v, so
// pixel p gains -integral over its boundary of L (v . n_out) ds.  An edge between
// pixels a (left / above) and b (right / below) thus adds (dLoss/dI_b - dLoss/dI_a)
// . integral of L v_e ds, v_e the velocity along +x (+y).  One thread per (edge,
// sample): the path through a uniform point of the edge (PCG32 stream camera << 40
// | edge << 12 | sample | 2^61) gives L, and its camera ray is posted as a warp with
// R = 0 and M = (dLoss/dI_b - dLoss/dI_a) . L grad(px) (grad(py)), whose M . V is the
// integrand.  On the crop's (or image's) border only the inside pixel's loss
// gradient counts; with a border window the image-border edges carry nothing.
template <int LAYOUT, bool INSTR, bool VERT>
__global__ void __launch_bounds__(128, 8) edge_kernel(const __grid_constant__ LaunchArgs A, const RpOpts K,
                                                   const EdgeGrid E, float* __restrict__ grad_t,
                                                   float* __restrict__ grad_v, unsigned long long* rays_out) {
  extern __shared__ float s_grad[];
  const int n3 = 3 * A.scene.n_shapes;
  if (K.smem) {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) s_grad[i] = 0.0f;
    __syncthreads();
  }
  GradOut G{K.smem ? s_grad : grad_t};
  VertOut GV{grad_v};
  Counters<INSTR> cnt;
  if constexpr (INSTR)
    for (int i = 0; i < kCounters; ++i) cnt.c[i] = 0;
  const float3 z = f3(0.f, 0.f, 0.f);
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned rays = 0;
  WarpRay w{};
  bool has = false;
  if (unit < (long long)A.n_cams * E.per_cam * K.edge_spp) {
    const EdgeSample es = edge_of(A, K, E, unit);
    auto dl_at = [&](int x, int y) {
      const long long pix = crop_pixel(A, es.ci, x, y);
      return pix < 0 ? z : f3(A.grad_image[3 * pix], A.grad_image[3 * pix + 1], A.grad_image[3 * pix + 2]);
    };
    const float3 gd = dl_at(es.X, es.Y) - (es.vertical ? dl_at(es.X - 1, es.Y) : dl_at(es.X, es.Y - 1));
    if (gd.x != 0.0f || gd.y != 0.0f || gd.z != 0.0f) {
      float3 o, u;
      float t0;
      const float3 L = edge_path<LAYOUT, INSTR>(A, es, o, u, t0, rays, cnt);
      const float R = dot3(gd, L) / (float)K.edge_spp;
      if (R != 0.0f) {
        float px, py;
        float3 gpx, gpy;
        pixel_coords(A, A.cams[es.ci], u, px, py, gpx, gpy);
        Pcg32 aux;
        aux.seed(A.seed, es.stream | (1ull << 62));
        w = WarpRay{o, u, (es.vertical ? gpx : gpy) * R, -1, es.ci, 0.0f, t0, aux.state, aux.inc, -1, 0.0f, 0.0f};
        has = true;
      }
    }
  }
  rays += process_warps<LAYOUT, INSTR, VERT>(A, K, has, w, G, GV, cnt);
  if (K.smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x)
      if (s_grad[i] != 0.0f) atomicAdd(&grad_t[i], s_grad[i]);
  }
  if (rays_out) {
    unsigned long long r = rays;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
    if (lane_id() == 0 && r) atomicAdd(rays_out, r);
  }
  flush_counters<INSTR>(A, cnt);
}

// ---------------------------------------------------------------- forward mode
// Forward-mode derivative images along a direction of shape translations (the
// paper's forward derivative of a translated mesh, Fig. "bunny": without the
// reparameterization the silhouettes' derivative is missing).  Every ray is
// reparameterized as in the reverse mode; a posted ray gets back its warp's
// tangential value V at u (windowed for camera rays) and div V, both linear in
// the direction's relative velocities Delta_i = dir[shape_i] - dir[shape_o]:
//     V = (I - u u^T) sum_i alpha_i b sv_i J Delta_i,  J = 1/D (jackknife:
//         N/D - (N-1)/N (S1 - 1/D_-i)),
//     div V = sum_i c_i . Delta_i, c_i the reverse mode's coefficient for M = 0,
//         R = 1.
// The path carries r = d(beta)/beta per channel (derivative of the log
// throughput): a camera ray starts it at m.V + div V (m = -3 f / f.u); a term
// C leaving a vertex along d adds its ray's m.V + div V with m = n / n.d, plus at a
// glossy vertex grad_out log f_c . V + grad_in log f_c . (-V_arriving); emitted
// radiance c adds r (.) c, a light sample c_nee adds (r + its term) (.) c_nee, the
// sampled continuation adds its term to r.

// Warps of the rays the lanes posted (called by all lanes together, as
// process_warps): the lane that posted a ray receives V (tangential) and div V.
// dir: [n_shapes][3] translation velocities, or (VERT) [n_tris][3][3] corner
// velocities by original triangle id; a plane point then moves with the
// barycentric combination of its triangle's corners (b_k(w) / t(w) = beta_k (n.w)
// / d + a_k . w, as in the reverse mode) and the origin with its own.
template <int LAYOUT, bool VERT>
__device__ __noinline__ unsigned warp_forward(const LaunchArgs& A, const RpOpts& K, bool has, const WarpRay& mine,
                                              const float* __restrict__ dir, float3& V_out, float& div_out,
                                              Counters<false>& cnt) {
  const DevScene& S = A.scene;
  const int lane = lane_id(), gs = K.group, grp = lane / gs, j = lane % gs;
  const int ng = 32 / gs;
  const float dk = K.kk - K.kappa, n = (float)K.n_aux;
  unsigned rays = 0;
  V_out = f3(0.f, 0.f, 0.f);
  div_out = 0.0f;
  unsigned pend = __ballot_sync(kFull, has);
  while (pend) {
    unsigned p = pend;
    for (int g = 0; g < grp && p; ++g) p &= p - 1;
    const int src = p ? __ffs(p) - 1 : -1;
    // this lane's own ray is served this round by group `rank` if it is among the first ng pending
    const int rank = __popc(pend & ((1u << lane) - 1u));
    const bool served = ((pend >> lane) & 1u) && rank < ng;
    for (int g = 0; g < ng && pend; ++g) pend &= pend - 1;
    const int sl = src >= 0 ? src : lane;
    WarpRay w;
    w.o = shfl3(mine.o, sl);
    w.u = shfl3(mine.u, sl);
    w.s_o = __shfl_sync(kFull, mine.s_o, sl);
    w.cam = __shfl_sync(kFull, mine.cam, sl);
    w.t0 = __shfl_sync(kFull, mine.t0, sl);
    w.st = __shfl_sync(kFull, mine.st, sl);
    w.inc = __shfl_sync(kFull, mine.inc, sl);
    if constexpr (VERT) {
      w.o_tri = __shfl_sync(kFull, mine.o_tri, sl);
      w.o_bu = __shfl_sync(kFull, mine.o_bu, sl);
      w.o_bv = __shfl_sync(kFull, mine.o_bv, sl);
    }
    const bool on = src >= 0 && j < K.n_aux;
    float alpha = 0.0f, t = 0.0f;
    int pos = -1;
    float3 wi = w.u, pi = f3(0.f, 0.f, 0.f);
    if (on) {
      Pcg32 r;
      r.state = w.st;
      r.inc = w.inc;
      pcg_advance(r, 2ull * (unsigned long long)j);
      const float a0 = r.uniform(), a1 = r.uniform();
      float c1;
      wi = vmf_dir(make_frame(w.u), a0, a1, K, c1);
      const Hit h = closest<LAYOUT, false>(S, w.o, wi, INFINITY, false, cnt);
      ++rays;
      float g = K.miss;
      if (h.pos >= 0) g = w.t0 < INFINITY ? depth_weight(__fdiv_rn(w.t0, fmaxf(h.t, 1e-3f * w.t0)), K.power) : 1.0f;
      alpha = expf(dk * c1) * g;
      pos = h.pos;
      t = h.t;
      pi = wi - w.u * dot3(w.u, wi);
    }
    const float D = group_sum(alpha, gs) + n * K.eps;
    const float3 P = group_sum3(pi * alpha, gs);
    float S1 = 0.0f;
    float3 SP = f3(0.f, 0.f, 0.f);
    if (K.jackknife) {
      const float Dj = D - alpha - K.eps;
      const float3 Pj = P - pi * alpha;
      S1 = group_sum(on ? PT_RCP(Dj) : 0.0f, gs);
      SP = group_sum3(on ? Pj * PT_RCP(Dj * Dj) : f3(0.f, 0.f, 0.f), gs);
    }
    float3 vs = f3(0.f, 0.f, 0.f);
    float dv = 0.0f;
    int si = -1;
    if (on && pos >= 0) si = tri_shape(S, pos);
    const bool contrib = VERT ? (on && pos >= 0) : (si >= 0 && si != w.s_o);
    if (contrib) {
      float b = 1.0f;
      float3 gb = f3(0.f, 0.f, 0.f);
      if (w.cam >= 0) b = cam_window(A, A.cams[w.cam], w.u, K.border, gb);
      const float3 nrm = tri_normal(S, pos);
      const float di = dot3(nrm, wi) * t;
      const float nu = __fdiv_rn(dot3(nrm, w.u), di);
      const float3 nperp = (nrm - w.u * dot3(nrm, w.u)) * PT_RCP(di);
      float Dm = 0.0f;
      float3 Pm = f3(0.f, 0.f, 0.f);
      if (K.jackknife) {
        Dm = D - alpha - K.eps;
        Pm = P - pi * alpha;
      }
      const float Jm = K.jackknife ? __fdiv_rn(n, D) - __fdiv_rn(n - 1.0f, n) * (S1 - PT_RCP(Dm)) : PT_RCP(D);
      // a velocity field s(w) Delta with s linear in w (gradient g on the sphere):
      // its weight in V at u, and the reverse coefficient with M = 0, R = 1 (div part)
      auto parts = [&](float sv, float3 g, float& vw, float3& cr) {
        vw = alpha * b * sv * Jm;
        const float3 Ai = (pi * K.kk - w.u * 2.0f) * (b * sv) + g * b + gb * sv;
        const float kb = K.kk * b * sv;
        float3 c = Ai * PT_RCP(D) - P * __fdiv_rn(kb, D * D);
        if (K.jackknife) {
          const float3 loo = Ai * (S1 - PT_RCP(Dm)) - (SP - Pm * PT_RCP(Dm * Dm)) * kb;
          c = c * n - loo * __fdiv_rn(n - 1.0f, n);
        }
        cr = c * alpha;
      };
      auto vel = [&](int base) { return f3(__ldg(&dir[base]), __ldg(&dir[base + 1]), __ldg(&dir[base + 2])); };
      float vw;
      float3 cr;
      parts(nu, nperp, vw, cr);
      if constexpr (VERT) {
        float3 vo = f3(0.f, 0.f, 0.f);  // the origin's velocity
        if (w.o_tri >= 0) {
          const size_t ob = 9 * (size_t)w.o_tri;
          vo = vel(ob) * (1.0f - w.o_bu - w.o_bv) + vel(ob + 3) * w.o_bu + vel(ob + 6) * w.o_bv;
        }
        vs = -vo * vw;
        dv = -dot3(cr, vo);
        const float3 v0 = xyz(__ldg(&S.tri_v[3 * pos]));
        const float3 e1 = xyz(__ldg(&S.tri_v[3 * pos + 1])), e2 = xyz(__ldg(&S.tri_v[3 * pos + 2]));
        const float3 c = cross3(e1, e2);
        const float icc = PT_RCP(dot3(c, c));
        const float3 a1 = cross3(e2, c) * icc, a2 = cross3(c, e1) * icc;
        const float3 aj[3] = {-(a1 + a2), a1, a2};
        const float3 ov = w.o - v0;
        const size_t tb = 9 * (size_t)tri_orig(S, pos);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float beta = dot3(aj[k], ov) + (k == 0 ? 1.0f : 0.0f);
          parts(beta * nu + dot3(aj[k], w.u), nperp * beta + (aj[k] - w.u * dot3(aj[k], w.u)), vw, cr);
          const float3 vk = vel(tb + 3 * k);
          vs = vs + vk * vw;
          dv += dot3(cr, vk);
        }
      } else {
        const float3 delta = vel(3 * si) - (w.s_o >= 0 ? vel(3 * w.s_o) : f3(0.f, 0.f, 0.f));
        vs = delta * vw;
        dv = dot3(cr, delta);
      }
    }
    vs = group_sum3(vs, gs);
    dv = group_sum(dv, gs);
    const int server = (rank < ng ? rank : 0) * gs;
    const float3 vr = shfl3(vs, server);
    const float dr = __shfl_sync(kFull, dv, server);
    if (served) {
      V_out = vr - mine.u * dot3(mine.u, vr);
      div_out = dr;
    }
  }
  return rays;
}

// Per-channel log-derivative of a term leaving a vertex along d: its ray's m.V +
// div V, plus at a glossy vertex the BSDF's directional terms (V of this ray,
// -V of the ray that arrived).  Vertex mode: ndot = the turn of the vertex's
// unit geometric normal ng; the cosine adds ndot.d / ng.d and a glossy value
// ndot . (ng x J_c), J_c = wi x grad_in log f_c + d x grad_out log f_c (f is
// unchanged when the normal and both directions turn together).
__device__ __forceinline__ float3 fwd_term(float3 n_s, float3 d, float3 V, float dvg, bool glossy, const Gloss& gl,
                                           const Frame& fr, float3 wi_l, float3 v_prev, float3 ng, float3 ndot,
                                           float3 wi_w) {
  const bool turns = ndot.x != 0.0f || ndot.y != 0.0f || ndot.z != 0.0f;
  const float l = dot3(n_s, V) / dot3(n_s, d) + dvg + (turns ? dot3(ndot, d) / dot3(ng, d) : 0.0f);
  float3 t = f3(l, l, l);
  if (glossy) {
    float3 go[3], gi[3];
    glossy_log_grad(gl.type, gl.alpha, gl.f0, gl.wd, gl.albedo, wi_l, fr.to_local(d), go, gi);
    float tc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float3 gow = fr.to_world(go[c]), giw = fr.to_world(gi[c]);
      tc[c] = dot3(gow, V) - dot3(giw, v_prev) + dot3(ndot, cross3(ng, cross3(wi_w, giw) + cross3(d, gow)));
    }
    t = t + f3(tc[0], tc[1], tc[2]);
  }
  return t;
}

// Vertex mode: the turn of the unit geometric normal of the triangle at leaf
// position pos when its corners move with dir[orig][k] (zero in translation mode).
template <bool VERT>
__device__ __forceinline__ float3 normal_turn(const DevScene& S, int pos, const float* __restrict__ dir) {
  if constexpr (!VERT) {
    return f3(0.f, 0.f, 0.f);
  } else {
    const float3 e1 = xyz(__ldg(&S.tri_v[3 * pos + 1])), e2 = xyz(__ldg(&S.tri_v[3 * pos + 2]));
    const size_t b = 9 * (size_t)tri_orig(S, pos);
    auto vel = [&](size_t i) { return f3(__ldg(&dir[i]), __ldg(&dir[i + 1]), __ldg(&dir[i + 2])); };
    const float3 v0 = vel(b), d1 = vel(b + 3) - v0, d2 = vel(b + 6) - v0;
    const float3 c = cross3(e1, e2), cd = cross3(d1, e2) + cross3(e1, d2);
    const float il = 1.0f / sqrtf(dot3(c, c));
    const float3 nn = c * il;
    return (cd - nn * dot3(nn, cd)) * il;
  }
}

// One thread per (pixel, lane) as the reverse kernel; samples in lockstep, the
// warps processed together after each vertex.  image / image_dot accumulate (the
// caller zeroes them): the mean over the pixel's samples.
template <int LAYOUT, bool VERT>
__global__ void __launch_bounds__(128, 8) reparam_jvp_kernel(const __grid_constant__ LaunchArgs A, const RpOpts K,
                                                          const float* __restrict__ dir_t, float* __restrict__ image,
                                                          float* __restrict__ image_dot,
                                                          unsigned long long* rays_out) {
  const DevScene& S = A.scene;
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PixelOf px{};
  const bool valid = unit_pixel(A, unit, crop_tile(A), px);
  unsigned rays = 0;
  Counters<false> cnt;
  const float3 z = f3(0.f, 0.f, 0.f);
  float3 fwd = z;
  if (valid) {
    const DevCamera& cam = A.cams[px.cam];
    fwd = f3(cam.fx, cam.fy, cam.fz);
  }
  bool live = false;
  int si = (int)(unit & (A.lanes_per_pixel - 1));
  GradSink sink;
  PathState P;
  Pcg32 aux;
  aux.state = aux.inc = 0ull;
  bool cached = false;
  Hit next{};
  float3 r = z, v_prev = z, ldot = z, sum_L = z, sum_dot = z;
  const unsigned long long n2 = 2ull * (unsigned long long)K.n_aux;
  for (;;) {
    WarpRay w0{}, w1{};
    bool h0 = false, h1 = false, start = false, done = false, glossy = false;
    float3 n_s = z, c_nee = z, wi_l = z, ng = z, ndot = z, wi_w = z;
    Gloss gl{};
    Frame fr{};
    if (!live && valid && si < A.spp) {
      path_start<false>(A, P, A.seed, px.cam, px.px, px.py, si, px.pix, cnt);
      const unsigned long long pixel = (unsigned long long)px.py * (unsigned long long)A.width + px.px;
      aux.seed(A.seed, ((unsigned long long)px.cam << 40) | (pixel << 12) | (unsigned long long)si | (1ull << 62));
      next = closest<LAYOUT, false>(S, P.ro, P.rd, INFINITY, false, cnt);
      ++rays;
      cached = true;
      w0 = WarpRay{P.ro, P.rd, fwd * (-3.0f / dot3(fwd, P.rd)), -1, px.cam, 0.0f,
                   next.pos >= 0 ? next.t : INFINITY, aux.state, aux.inc, -1, 0.0f, 0.0f};
      h0 = true;
      start = true;
      pcg_advance(aux, n2);
      live = true;
    } else if (live) {
      Hit hit;
      if (cached) {
        hit = next;
        cached = false;
      } else {
        hit = closest<LAYOUT, false>(S, P.ro, P.rd, INFINITY, false, cnt);
        ++rays;
      }
      const bool block = hit.pos >= 0 && P.depth < A.max_depth;
      int s_o = -1, o_tri = -1;
      wi_w = -P.rd;
      if (hit.pos >= 0) {
        s_o = tri_shape(S, hit.pos);
        o_tri = tri_orig(S, hit.pos);
        ng = tri_normal(S, hit.pos);
        n_s = dot3(ng, P.rd) < 0.0f ? ng : -ng;
        ndot = normal_turn<VERT>(S, hit.pos, dir_t);
      }
      float3 L0 = P.L;
      bool more = path_shade<false, false, false, PT_DISPATCH_SWITCH, FEAT_NOHASH>(A, P, hit, false, z, sink, cnt);
      ldot = ldot + r * (P.L - L0);  // emission reaching this vertex
      Pcg32 aux_nee = aux, aux_bsdf = aux;
      if (block) {
        pcg_advance(aux_bsdf, n2);
        pcg_advance(aux, 2ull * n2);
      }
      if (more) {
        bool occ = false;
        if (P.has_shadow) {
          occ = closest<LAYOUT, false>(S, P.so, P.sd, P.stmax, true, cnt).pos >= 0;
          ++rays;
        }
        const int mt = P.mtype;
        const bool warp = block && (mt == PT_BSDF_DIFFUSE || mt == PT_BSDF_CONDUCTOR || mt == PT_BSDF_BLEND);
        glossy = warp && mt != PT_BSDF_DIFFUSE;
        if (glossy) {
          gl = gloss_at(A, hit);
          fr = make_frame(n_s);
          wi_l = fr.to_local(wi_w);
        }
        if (warp && P.has_shadow && !occ) {
          const Hit hl = closest<LAYOUT, false>(S, P.so, P.sd, INFINITY, false, cnt);
          ++rays;
          c_nee = P.c_nee;
          w0 = WarpRay{P.so, P.sd, z, s_o, -1, 0.0f, hl.pos >= 0 ? hl.t : INFINITY, aux_nee.state, aux_nee.inc,
                       o_tri, hit.u, hit.v};
          h0 = true;
        }
        L0 = P.L;
        more = path_finish<false, false, false, FEAT_NOHASH>(A, P, occ, false, z, sink, cnt);
        ldot = ldot + r * (P.L - L0);  // the light sample, with the path's tangent so far
        if (more && warp) {
          next = closest<LAYOUT, false>(S, P.ro, P.rd, INFINITY, false, cnt);
          ++rays;
          cached = true;
          w1 = WarpRay{P.ro, P.rd, z, s_o, -1, 0.0f, next.pos >= 0 ? next.t : INFINITY, aux_bsdf.state,
                       aux_bsdf.inc, o_tri, hit.u, hit.v};
          h1 = true;
        }
      }
      if (!more) done = true;
    }
    if (!__any_sync(kFull, live || h0 || h1 || (valid && si < A.spp))) break;
    float3 V0, V1;
    float d0, d1;
    rays += warp_forward<LAYOUT, VERT>(A, K, h0, w0, dir_t, V0, d0, cnt);
    rays += warp_forward<LAYOUT, VERT>(A, K, h1, w1, dir_t, V1, d1, cnt);
    if (start) {
      const float l = dot3(w0.m, V0) + d0;  // m: the pinhole's image-plane density term
      r = f3(l, l, l);
      v_prev = V0;
    } else if (live) {
      if (h0) ldot = ldot + c_nee * fwd_term(n_s, w0.u, V0, d0, glossy, gl, fr, wi_l, v_prev, ng, ndot, wi_w);
      if (h1) {
        r = r + fwd_term(n_s, w1.u, V1, d1, glossy, gl, fr, wi_l, v_prev, ng, ndot, wi_w);
        v_prev = V1;
      } else {
        v_prev = z;  // a delta vertex: its continuation is not reparameterized
      }
      if (done) {
        sum_L = sum_L + P.L;
        sum_dot = sum_dot + ldot;
        ldot = r = v_prev = z;
        live = false;
        si += A.lanes_per_pixel;
      }
    }
  }
  if (valid) {
    const float inv = 1.0f / (float)A.spp;
    if (image) {
      atomicAdd(&image[3 * px.pix], sum_L.x * inv);
      atomicAdd(&image[3 * px.pix + 1], sum_L.y * inv);
      atomicAdd(&image[3 * px.pix + 2], sum_L.z * inv);
    }
    atomicAdd(&image_dot[3 * px.pix], sum_dot.x * inv);
    atomicAdd(&image_dot[3 * px.pix + 1], sum_dot.y * inv);
    atomicAdd(&image_dot[3 * px.pix + 2], sum_dot.z * inv);
  }
  if (rays_out) {
    unsigned long long rr = rays;
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
    if (lane_id() == 0 && rr) atomicAdd(rays_out, rr);
  }
}

// Forward mode of the pixel-edge term: per (edge, sample) the path's radiance L and
// its camera warp's velocity across the edge v_e; the pixel left of / above the
// edge loses L v_e / edge_spp, the one right of / below it gains it (pixels of the
// crop only).
template <int LAYOUT, bool VERT>
__global__ void __launch_bounds__(128, 8) edge_jvp_kernel(const __grid_constant__ LaunchArgs A, const RpOpts K,
                                                       const EdgeGrid E, const float* __restrict__ dir_t,
                                                       float* __restrict__ image_dot,
                                                       unsigned long long* rays_out) {
  Counters<false> cnt;
  const float3 z = f3(0.f, 0.f, 0.f);
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned rays = 0;
  WarpRay w{};
  bool has = false;
  EdgeSample es{};
  float3 L = z;
  if (unit < (long long)A.n_cams * E.per_cam * K.edge_spp) {
    es = edge_of(A, K, E, unit);
    float3 o, u;
    float t0;
    L = edge_path<LAYOUT, false>(A, es, o, u, t0, rays, cnt);
    if (L.x != 0.0f || L.y != 0.0f || L.z != 0.0f) {
      Pcg32 aux;
      aux.seed(A.seed, es.stream | (1ull << 62));
      w = WarpRay{o, u, z, -1, es.ci, 0.0f, t0, aux.state, aux.inc, -1, 0.0f, 0.0f};
      has = true;
    }
  }
  float3 V;
  float dv;
  rays += warp_forward<LAYOUT, VERT>(A, K, has, w, dir_t, V, dv, cnt);
  if (has) {
    float pxc, pyc;
    float3 gpx, gpy;
    pixel_coords(A, A.cams[es.ci], w.u, pxc, pyc, gpx, gpy);
    const float3 d = L * (dot3(es.vertical ? gpx : gpy, V) / (float)K.edge_spp);
    auto add = [&](int x, int y, float3 v) {
      const long long pix = crop_pixel(A, es.ci, x, y);
      if (pix < 0) return;
      atomicAdd(&image_dot[3 * pix], v.x);
      atomicAdd(&image_dot[3 * pix + 1], v.y);
      atomicAdd(&image_dot[3 * pix + 2], v.z);
    };
    add(es.vertical ? es.X - 1 : es.X, es.vertical ? es.Y : es.Y - 1, -d);
    add(es.X, es.Y, d);
  }
  if (rays_out) {
    unsigned long long rr = rays;
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_xor_sync(kFull, rr, off);
    if (lane_id() == 0 && rr) atomicAdd(rays_out, rr);
  }
}

}  // namespace
}  // namespace ptgb

using namespace ptgb;

extern "C" void pt_reparam_defaults(pt_reparam_opts* o) {
  if (!o) return;
  o->n_aux = 16;
  o->kappa = 1000.0f;
  o->kernel_scale = 8.0f;
  o->power = 2.0f;
  o->miss = 0.01f;
  o->eps = 1e-4f;
  o->border = 0.0f;
  o->jackknife = 1;
  o->edge_spp = 1;
}

namespace {
// Options (NULL: defaults) checked and converted to the kernels' form.
int rp_opts(const pt_reparam_opts* opts, RpOpts& K) {
  pt_reparam_opts o;
  pt_reparam_defaults(&o);
  if (opts) o = *opts;
  if (!(o.n_aux >= 2 && o.n_aux <= kMaxAux) || !(o.kappa > 0.0f && o.kappa <= 1e6f) || !(o.kernel_scale >= 1.0f) ||
      !(o.power >= 0.0f && o.power <= 16.0f) || !(o.miss >= 0.0f) || !(o.eps > 0.0f) ||
      !(o.border >= 0.0f && o.border <= 1e6f) || (o.jackknife != 0 && o.jackknife != 1) ||
      !(o.edge_spp >= 0 && o.edge_spp <= 4096))
    return PT_ERR_ARG;
  K.n_aux = o.n_aux;
  K.jackknife = o.jackknife;
  K.kappa = o.kappa;
  K.kk = o.kappa * o.kernel_scale;
  K.power = o.power;
  K.miss = o.miss;
  K.eps = o.eps;
  K.border = o.border;
  K.edge_spp = o.edge_spp;
  K.e2k = expf(-2.0f * o.kappa);
  K.group = 2;
  while (K.group < o.n_aux) K.group *= 2;
  K.smem = 0;
  return PT_OK;
}

// The pixel-edge term's edges (all edges of the crop's pixels); PT_ERR_ARG if the
// edge ids do not fit their 28 bits.
int edge_grid(const LaunchArgs& A, EdgeGrid& E) {
  E.xlo = A.crop_x0;
  E.nvx = A.crop_w + 1;
  E.ylo = A.crop_y0;
  E.nhy = A.crop_h + 1;
  E.per_cam = (long long)A.crop_h * E.nvx + (long long)E.nhy * A.crop_w;
  if ((unsigned long long)(A.width + 1) * A.height + (unsigned long long)A.width * (A.height + 1) >= (1ull << 28))
    return PT_ERR_ARG;
  return PT_OK;
}

int reparam_launch(pt_scene* s, const pt_render_desc* r, const pt_params* p, const pt_reparam_opts* opts,
                   const float* grad_image, float* grad_t, float* grad_v, unsigned long long* rays, void* stream) {
  RpOpts K;
  if (rp_opts(opts, K) != PT_OK) return PT_ERR_ARG;
  if (!s || !r || !p || !grad_image || (!grad_t && !grad_v)) return PT_ERR_ARG;
  LaunchArgs A;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (r->cache || r->dbg_sample_L || r->dbg_sample_hash) return PT_ERR_ARG;
  A.grad_image = grad_image;
  EdgeGrid E;
  if (K.edge_spp > 0 && edge_grid(A, E) != PT_OK) return PT_ERR_ARG;
  const bool vert = grad_v != nullptr;
  const size_t smem = (size_t)s->n_shapes * 3 * sizeof(float);
  K.smem = (!vert && smem <= 32768) ? 1 : 0;
  pt_render_desc rd = *r;
  if (rd.block_size == 0) rd.block_size = 128;
  if (rd.block_size != 128) return PT_ERR_ARG;
  int block;
  long long grid;
  if ((st = launch_dims(&rd, A, block, grid)) != PT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t sm = K.smem ? smem : 0;
  if ((st = radiance_pass(s, &rd, A, cs)) != PT_OK) return st;
  const dim3 gd((unsigned)grid), bd(block);
  const int v = (s->dev.layout == PT_BVH_WIDE ? 4 : 0) | (A.counters ? 2 : 0) | (vert ? 1 : 0);
  switch (v) {
    case 0: reparam_kernel<PT_BVH_BINARY, false, false><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 1: reparam_kernel<PT_BVH_BINARY, false, true><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 2: reparam_kernel<PT_BVH_BINARY, true, false><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 3: reparam_kernel<PT_BVH_BINARY, true, true><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 4: reparam_kernel<PT_BVH_WIDE, false, false><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 5: reparam_kernel<PT_BVH_WIDE, false, true><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    case 6: reparam_kernel<PT_BVH_WIDE, true, false><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
    default: reparam_kernel<PT_BVH_WIDE, true, true><<<gd, bd, sm, cs>>>(A, K, grad_t, grad_v, rays); break;
  }
  if (cudaGetLastError() != cudaSuccess) return PT_ERR_CUDA;
  if (K.edge_spp > 0) {
    const long long units = (long long)A.n_cams * E.per_cam * K.edge_spp;
    if (units > 0) {
      const dim3 eg((unsigned)((units + 127) / 128)), eb(128);
      auto go = [&](auto kernel) { kernel<<<eg, eb, sm, cs>>>(A, K, E, grad_t, grad_v, rays); };
      switch (v) {
        case 0: go(edge_kernel<PT_BVH_BINARY, false, false>); break;
        case 1: go(edge_kernel<PT_BVH_BINARY, false, true>); break;
        case 2: go(edge_kernel<PT_BVH_BINARY, true, false>); break;
        case 3: go(edge_kernel<PT_BVH_BINARY, true, true>); break;
        case 4: go(edge_kernel<PT_BVH_WIDE, false, false>); break;
        case 5: go(edge_kernel<PT_BVH_WIDE, false, true>); break;
        case 6: go(edge_kernel<PT_BVH_WIDE, true, false>); break;
        default: go(edge_kernel<PT_BVH_WIDE, true, true>); break;
      }
    }
  }
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
}  // namespace

extern "C" int pt_render_backward_reparam(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                          const pt_reparam_opts* opts, const float* grad_image,
                                          float* grad_translation, unsigned long long* rays, void* stream) {
  if (!grad_translation) return PT_ERR_ARG;
  return reparam_launch(s, r, p, opts, grad_image, grad_translation, nullptr, rays, stream);
}

extern "C" int pt_render_backward_reparam_vertices(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                                   const pt_reparam_opts* opts, const float* grad_image,
                                                   float* grad_vertices, unsigned long long* rays, void* stream) {
  if (!grad_vertices) return PT_ERR_ARG;
  return reparam_launch(s, r, p, opts, grad_image, nullptr, grad_vertices, rays, stream);
}

namespace {
int jvp_reparam_launch(pt_scene* s, const pt_render_desc* r, const pt_params* p, const pt_reparam_opts* opts,
                       const float* dir, bool vert, float* image, float* image_dot, unsigned long long* rays,
                       void* stream) {
  RpOpts K;
  if (rp_opts(opts, K) != PT_OK) return PT_ERR_ARG;
  if (!s || !r || !p || !dir || !image_dot) return PT_ERR_ARG;
  LaunchArgs A;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (r->cache || r->dbg_sample_L || r->dbg_sample_hash || r->counters) return PT_ERR_ARG;
  EdgeGrid E;
  if (K.edge_spp > 0 && edge_grid(A, E) != PT_OK) return PT_ERR_ARG;
  pt_render_desc rd = *r;
  if (rd.block_size == 0) rd.block_size = 128;
  if (rd.block_size != 128) return PT_ERR_ARG;
  int block;
  long long grid;
  if ((st = launch_dims(&rd, A, block, grid)) != PT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t bytes = (size_t)A.n_cams * A.crop_w * A.crop_h * 3 * sizeof(float);
  if (image && cudaMemsetAsync(image, 0, bytes, cs) != cudaSuccess) return PT_ERR_CUDA;
  if (cudaMemsetAsync(image_dot, 0, bytes, cs) != cudaSuccess) return PT_ERR_CUDA;
  const int v = (s->dev.layout == PT_BVH_WIDE ? 2 : 0) | (vert ? 1 : 0);
  const dim3 gd((unsigned)grid), bd(block);
  auto main = [&](auto kernel) { kernel<<<gd, bd, 0, cs>>>(A, K, dir, image, image_dot, rays); };
  switch (v) {
    case 0: main(reparam_jvp_kernel<PT_BVH_BINARY, false>); break;
    case 1: main(reparam_jvp_kernel<PT_BVH_BINARY, true>); break;
    case 2: main(reparam_jvp_kernel<PT_BVH_WIDE, false>); break;
    default: main(reparam_jvp_kernel<PT_BVH_WIDE, true>); break;
  }
  if (cudaGetLastError() != cudaSuccess) return PT_ERR_CUDA;
  if (K.edge_spp > 0) {
    const long long units = (long long)A.n_cams * E.per_cam * K.edge_spp;
    if (units > 0) {
      const dim3 eg((unsigned)((units + 127) / 128)), eb(128);
      auto edges = [&](auto kernel) { kernel<<<eg, eb, 0, cs>>>(A, K, E, dir, image_dot, rays); };
      switch (v) {
        case 0: edges(edge_jvp_kernel<PT_BVH_BINARY, false>); break;
        case 1: edges(edge_jvp_kernel<PT_BVH_BINARY, true>); break;
        case 2: edges(edge_jvp_kernel<PT_BVH_WIDE, false>); break;
        default: edges(edge_jvp_kernel<PT_BVH_WIDE, true>); break;
      }
    }
  }
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
}  // namespace

extern "C" int pt_render_jvp_reparam(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                     const pt_reparam_opts* opts, const float* dir_translation, float* image,
                                     float* image_dot, unsigned long long* rays, void* stream) {
  return jvp_reparam_launch(s, r, p, opts, dir_translation, false, image, image_dot, rays, stream);
}

extern "C" int pt_render_jvp_reparam_vertices(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                              const pt_reparam_opts* opts, const float* dir_vertices, float* image,
                                              float* image_dot, unsigned long long* rays, void* stream) {
  return jvp_reparam_launch(s, r, p, opts, dir_vertices, true, image, image_dot, rays, stream);
}
