// Reparameterized Path Replay Backpropagation for shape translations (Sec. 4.7,
// "Reparameterizations"; Sec. 4.8 on the derivative terms a moving vertex adds;
// warp field after Bangaru et al. 2020).
//
// Parameters: one translation per shape (all of its vertices move together); a
// surface point keeps its barycentric coordinates.  Every ray the path tracer
// traces -- the camera ray and, at diffuse vertices, the light-sample ray and the
// BSDF-sampled ray -- is reparameterized: in the primal nothing changes, in the
// derivative the ray turns by a warp field V and its integrand is multiplied by
// the Jacobian determinant 1 + div V.  A ray therefore contributes
//     R * (m_perp . V(u) + div V(u))
// to the derivative, where R = dLoss/dI . (radiance the ray carries) and m is the
// covector of the ray's own measure or cosine term (camera: the pinhole's
// image-plane density, -3 f / f.u; diffuse vertex: the cosine, n / n.u).
//
// The warp of a ray (origin o, direction u) comes from N auxiliary rays in a von
// Mises-Fisher lobe around u (uniforms from the sample's auxiliary PCG32 stream,
// initseq | 2^62): each one that hits a triangle of plane n_i.(x - o) = d_i says
// that, seen along w, the plane point at distance d_i / (n_i.w) moves relative to
// the origin with Delta_i = tau'(shape_i) - tau'(shape_o).  With per-sample weights
//     alpha_i = exp((kk - kappa)(u.w_i - 1)) g_i,   g_i = (t0 / t_i)^m (1 if the
// ray itself escapes; `miss` for escaping auxiliary rays, which do not move),
// the normalised average C(w) = sum alpha_i(w) Delta_i (n_i.w)/d_i / (sum alpha_i(w)
// + N eps) with alpha_i(w) proportional to exp(kk (w.w_i - 1)) gives the warp
// V = (I - w w^T) C, and differentiating it at u (samples fixed) in closed form:
//     m_perp.V + div V = sum_i alpha_i / (D d_i) * H_i . Delta_i,
//     H_i = (n_i.u)(m_perp - 2u + kk p_i - kk P / D) + (I - u u^T) n_i,
// with p_i = (I - u u^T) w_i, P = sum alpha_j p_j, D = sum alpha_j + N eps.  The
// ratio's O(1/N) bias is removed by the leave-one-out (jackknife) combination
// N f(all) - (N-1)/N sum_j f(all but j), evaluated with two extra sums.  For the
// camera ray the warp is multiplied by a window b that reaches 0 at the image
// border, adding grad(b) . C.  Because every term is linear in the translation
// velocities, the reverse-mode gradient of a ray is the coefficient vector of
// each Delta_i: it is added to shape_i's gradient and subtracted from the
// origin shape's.
//
// Launch: one thread per (pixel, lane) as in the megakernel; each sample is
// traced once for its radiance and replayed (PRB) with the warps.  Gradients
// are accumulated per CTA in shared memory when the shape table fits.
#include "pt_mega.cuh"

namespace ptgb {
namespace {

constexpr int kMaxAux = 32;

struct RpOpts {
  int n_aux, jackknife, smem;
  float kappa, kk, power, miss, eps, border, e2k;
};

template <int LAYOUT>
__device__ __forceinline__ Hit closest(const DevScene& S, float3 o, float3 d, float tmax, bool any,
                                       Counters<false>& cnt) {
  return LAYOUT == PT_BVH_WIDE ? trace_wide<false>(S, o, d, tmax, any, cnt)
                               : trace_binary<false>(S, o, d, tmax, any, cnt);
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

// Window of the camera warp: smoothstep of the distance in pixels to the nearest
// image border over `border` pixels; b and its gradient on the sphere at u.
__device__ __forceinline__ float cam_window(const LaunchArgs& A, const DevCamera& c, float3 u, float border,
                                            float3& grad) {
  const float3 f = f3(c.fx, c.fy, c.fz), rs = f3(c.rx, c.ry, c.rz), us = f3(c.ux, c.uy, c.uz);
  const float fw = dot3(f, u), rr = dot3(rs, rs), uu = dot3(us, us);
  const float sx = dot3(rs, u) / (fw * rr), sy = dot3(us, u) / (fw * uu);
  const float W = (float)A.width, H = (float)A.height;
  const float px = (sx + 1.0f) * 0.5f * W, py = (1.0f - sy) * 0.5f * H;
  const float3 gpx = (rs - f * (dot3(rs, u) / fw)) * (0.5f * W / (rr * fw));
  const float3 gpy = (us - f * (dot3(us, u) / fw)) * (-0.5f * H / (uu * fw));
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

struct GradOut {
  float* dst;  // shared (per CTA) or global [n_shapes][3]
  __device__ __forceinline__ void add(int s, float3 g) {
    atomicAdd(&dst[3 * s], g.x);
    atomicAdd(&dst[3 * s + 1], g.y);
    atomicAdd(&dst[3 * s + 2], g.z);
  }
};

// One reparameterized ray: trace its N auxiliary rays and scatter R times the
// coefficient of every shape's translation velocity.  Consumes 2N uniforms of
// `rng` whether or not R is zero.  Returns the rays traced.
template <int LAYOUT>
__device__ __noinline__ unsigned warp_scatter(const LaunchArgs& A, const RpOpts& K, Pcg32& rng, float3 o, float3 u,
                                              int s_o, float3 m, int cam, float R, GradOut& G) {
  const Pcg32 r0 = rng;
  for (int i = 0; i < 2 * K.n_aux; ++i) rng.next();
  if (R == 0.0f) return 0;
  const DevScene& S = A.scene;
  Counters<false> cnt;
  const Hit h0 = closest<LAYOUT>(S, o, u, INFINITY, false, cnt);
  const float t0 = h0.pos >= 0 ? h0.t : INFINITY;
  const Frame fr = make_frame(u);
  const float dk = K.kk - K.kappa;
  float alpha[kMaxAux], dist[kMaxAux];
  int pos[kMaxAux];
  float D = 0.0f;
  float3 P = f3(0.f, 0.f, 0.f);
  Pcg32 r = r0;
  for (int i = 0; i < K.n_aux; ++i) {
    const float a0 = r.uniform(), a1 = r.uniform();
    float c1;
    const float3 w = vmf_dir(fr, a0, a1, K, c1);
    const Hit h = closest<LAYOUT>(S, o, w, INFINITY, false, cnt);
    float g = K.miss;
    if (h.pos >= 0) g = t0 < INFINITY ? powf(t0 / fmaxf(h.t, 1e-3f * t0), K.power) : 1.0f;
    const float a = expf(dk * c1) * g;
    alpha[i] = a;
    pos[i] = h.pos;
    dist[i] = h.t;
    D += a;
    P = P + (w - u * dot3(u, w)) * a;
  }
  D += K.n_aux * K.eps;
  // leave-one-out sums: S1 = sum_j 1 / D_{-j}, SP = sum_j P_{-j} / D_{-j}^2
  float S1 = 0.0f;
  float3 SP = f3(0.f, 0.f, 0.f);
  if (K.jackknife) {
    r = r0;
    for (int j = 0; j < K.n_aux; ++j) {
      const float a0 = r.uniform(), a1 = r.uniform();
      float c1;
      const float3 w = vmf_dir(fr, a0, a1, K, c1);
      const float Dj = D - alpha[j] - K.eps;
      const float3 Pj = P - (w - u * dot3(u, w)) * alpha[j];
      S1 += 1.0f / Dj;
      SP = SP + Pj * (1.0f / (Dj * Dj));
    }
  }
  float b = 1.0f;
  float3 gb = f3(0.f, 0.f, 0.f);
  if (cam >= 0) b = cam_window(A, A.cams[cam], u, K.border, gb);
  const float3 mp = m - u * dot3(u, m);
  const float n = (float)K.n_aux;
  r = r0;
  for (int i = 0; i < K.n_aux; ++i) {
    const float a0 = r.uniform(), a1 = r.uniform();
    if (pos[i] < 0) continue;
    const int si = tri_shape(S, pos[i]);
    if (si == s_o) continue;
    float c1;
    const float3 w = vmf_dir(fr, a0, a1, K, c1);
    const float3 nrm = tri_normal(S, pos[i]);
    const float nu = dot3(nrm, u);
    const float di = dot3(nrm, w) * dist[i];
    const float3 p = w - u * dot3(u, w);
    // A_i: the part of H_i that does not depend on the sample set
    const float3 Ai = (mp - u * 2.0f + p * K.kk) * (nu * b) + (nrm - u * nu) * b + gb * nu;
    const float kb = K.kk * b * nu;
    float3 coef = Ai * (1.0f / D) - P * (kb / (D * D));
    if (K.jackknife) {
      const float Dm = D - alpha[i] - K.eps;
      const float3 Pm = P - p * alpha[i];
      const float3 loo = Ai * (S1 - 1.0f / Dm) - (SP - Pm * (1.0f / (Dm * Dm))) * kb;
      coef = coef * n - loo * ((n - 1.0f) / n);
    }
    const float3 g = coef * (R * alpha[i] / di);
    G.add(si, g);
    if (s_o >= 0) G.add(s_o, -g);
  }
  return 1u + (unsigned)K.n_aux;
}

template <int LAYOUT>
__device__ __forceinline__ float3 sample_radiance(const LaunchArgs& A, PathState& P, const PixelOf& px, int si,
                                                  GradSink& sink, Counters<false>& cnt, unsigned& rays) {
  path_start<false>(A, P, A.seed, px.cam, px.px, px.py, si, px.pix, cnt);
  P.Lrem = f3(0.f, 0.f, 0.f);
  const float3 z = f3(0.f, 0.f, 0.f);
  for (;;) {
    const Hit hit = closest<LAYOUT>(A.scene, P.ro, P.rd, INFINITY, false, cnt);
    ++rays;
    if (!path_shade<false, false, false, PT_DISPATCH_SWITCH>(A, P, hit, false, z, sink, cnt)) break;
    bool occ = false;
    if (P.has_shadow) {
      occ = closest<LAYOUT>(A.scene, P.so, P.sd, P.stmax, true, cnt).pos >= 0;
      ++rays;
    }
    if (!path_finish<false, false, false>(A, P, occ, false, z, sink, cnt)) break;
  }
  return P.L;
}

template <int LAYOUT>
__global__ void __launch_bounds__(128) reparam_kernel(const __grid_constant__ LaunchArgs A, const RpOpts K,
                                                      float* __restrict__ grad_t, unsigned long long* rays_out) {
  extern __shared__ float s_grad[];
  const int n3 = 3 * A.scene.n_shapes;
  if (K.smem) {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) s_grad[i] = 0.0f;
    __syncthreads();
  }
  GradOut G{K.smem ? s_grad : grad_t};
  const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PixelOf px{};
  const bool valid = unit_pixel(A, unit, crop_tile(A), px);
  unsigned rays = 0;
  if (valid) {
    const int lane = (int)(unit & (A.lanes_per_pixel - 1));
    const float inv = 1.0f / (float)A.spp;
    const float3 dl = f3(A.grad_image[3 * px.pix] * inv, A.grad_image[3 * px.pix + 1] * inv,
                         A.grad_image[3 * px.pix + 2] * inv);
    const DevCamera& cam = A.cams[px.cam];
    const float3 fwd = f3(cam.fx, cam.fy, cam.fz);
    const float3 z = f3(0.f, 0.f, 0.f);
    Counters<false> cnt;
    GradSink sink;
    PathState P;
    for (int si = lane; si < A.spp; si += A.lanes_per_pixel) {
      const float3 L = sample_radiance<LAYOUT>(A, P, px, si, sink, cnt, rays);
      // replay with the same primary stream; auxiliary stream initseq | 2^62
      path_start<false>(A, P, A.seed, px.cam, px.px, px.py, si, px.pix, cnt);
      P.Lrem = L;
      const unsigned long long pixel = (unsigned long long)px.py * (unsigned long long)A.width + px.px;
      Pcg32 aux;
      aux.seed(A.seed, ((unsigned long long)px.cam << 40) | (pixel << 12) | (unsigned long long)si | (1ull << 62));
      rays += warp_scatter<LAYOUT>(A, K, aux, P.ro, P.rd, -1, fwd * (-3.0f / dot3(fwd, P.rd)), px.cam,
                                   dot3(dl, L), G);
      for (;;) {
        const Hit hit = closest<LAYOUT>(A.scene, P.ro, P.rd, INFINITY, false, cnt);
        ++rays;
        const bool block = hit.pos >= 0 && P.depth < A.max_depth;
        int s_o = -1;
        float3 n_s = z;
        if (hit.pos >= 0) {
          s_o = tri_shape(A.scene, hit.pos);
          const float3 ng = tri_normal(A.scene, hit.pos);
          n_s = dot3(ng, P.rd) < 0.0f ? ng : -ng;
        }
        const bool alive = path_shade<false, false, false, PT_DISPATCH_SWITCH>(A, P, hit, false, z, sink, cnt);
        Pcg32 aux_nee = aux, aux_bsdf = aux;
        if (block) {
          for (int i = 0; i < 2 * K.n_aux; ++i) aux_bsdf.next();
          aux = aux_bsdf;
          for (int i = 0; i < 2 * K.n_aux; ++i) aux.next();
        }
        if (!alive) break;
        bool occ = false;
        if (P.has_shadow) {
          occ = closest<LAYOUT>(A.scene, P.so, P.sd, P.stmax, true, cnt).pos >= 0;
          ++rays;
        }
        const bool diffuse = P.mtype == PT_BSDF_DIFFUSE;
        if (block && diffuse && P.has_shadow && !occ)
          rays += warp_scatter<LAYOUT>(A, K, aux_nee, P.so, P.sd, s_o, n_s * (1.0f / dot3(n_s, P.sd)), -1,
                                       dot3(dl, P.c_nee), G);
        const bool cont = path_finish<false, false, false>(A, P, occ, false, z, sink, cnt);
        if (!cont) break;
        if (block && diffuse) {
          const float3 lr = f3(fmaxf(P.Lrem.x, 0.f), fmaxf(P.Lrem.y, 0.f), fmaxf(P.Lrem.z, 0.f));
          rays += warp_scatter<LAYOUT>(A, K, aux_bsdf, P.ro, P.rd, s_o, n_s * (1.0f / dot3(n_s, P.rd)), -1,
                                       dot3(dl, lr), G);
        }
      }
    }
  }
  if (K.smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x)
      if (s_grad[i] != 0.0f) atomicAdd(&grad_t[i], s_grad[i]);
  }
  if (rays_out && rays) atomicAdd(rays_out, (unsigned long long)rays);
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
  o->border = 4.0f;
  o->jackknife = 1;
}

extern "C" int pt_render_backward_reparam(pt_scene* s, const pt_render_desc* r, const pt_params* p,
                                          const pt_reparam_opts* opts, const float* grad_image,
                                          float* grad_translation, unsigned long long* rays, void* stream) {
  pt_reparam_opts o;
  pt_reparam_defaults(&o);
  if (opts) o = *opts;
  if (!(o.n_aux >= 2 && o.n_aux <= kMaxAux) || !(o.kappa > 0.0f && o.kappa <= 1e6f) || !(o.kernel_scale >= 1.0f) ||
      !(o.power >= 0.0f && o.power <= 16.0f) || !(o.miss >= 0.0f) || !(o.eps > 0.0f) || !(o.border > 0.0f) ||
      (o.jackknife != 0 && o.jackknife != 1))
    return PT_ERR_ARG;
  if (!s || !r || !p || !grad_image || !grad_translation) return PT_ERR_ARG;
  LaunchArgs A;
  int st = fill_launch(s, r, p, A);
  if (st != PT_OK) return st;
  if (r->cache || r->counters || r->dbg_sample_L || r->dbg_sample_hash) return PT_ERR_ARG;
  A.grad_image = grad_image;
  RpOpts K;
  K.n_aux = o.n_aux;
  K.jackknife = o.jackknife;
  K.kappa = o.kappa;
  K.kk = o.kappa * o.kernel_scale;
  K.power = o.power;
  K.miss = o.miss;
  K.eps = o.eps;
  K.border = o.border;
  K.e2k = expf(-2.0f * o.kappa);
  const size_t smem = (size_t)s->n_shapes * 3 * sizeof(float);
  K.smem = smem <= 32768 ? 1 : 0;
  pt_render_desc rd = *r;
  if (rd.block_size == 0) rd.block_size = 128;
  if (rd.block_size != 128) return PT_ERR_ARG;
  int block;
  long long grid;
  if ((st = launch_dims(&rd, A, block, grid)) != PT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t sm = K.smem ? smem : 0;
  if (s->dev.layout == PT_BVH_WIDE)
    reparam_kernel<PT_BVH_WIDE><<<(unsigned)grid, block, sm, cs>>>(A, K, grad_translation, rays);
  else
    reparam_kernel<PT_BVH_BINARY><<<(unsigned)grid, block, sm, cs>>>(A, K, grad_translation, rays);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
