// FP64 CPU oracle for the path-tracing megakernel and its reverse-mode derivative.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code with
// the CUDA path: its own PCG32, camera, BVH, intersection, BSDFs, emitter
// sampling and gradient code, all in double precision, written for clarity.
//
// What it computes (Dr.Jit paper, Sec. 4.1 and Fig. 7): the Monte Carlo
// estimate of a unidirectional path tracer with next-event estimation and
// multiple importance sampling, pixel by pixel, with the same random numbers
// the GPU kernel draws; and the derivative of that estimate with respect to
// albedos, texels and roughness values with every random number fixed and the
// sampling detached (Sec. 4.9: only BSDF *values* carry derivatives).  The
// derivative is computed two ways, neither of which uses path replay:
//   * oracle_grad_tape : reverse mode over a stored per-path vertex tape
//                        (the "shadow memory" approach that PRB avoids, Sec. 2),
//                        derivative factors written out analytically;
//   * oracle_render_jvp: image and its derivative along one parameter direction
//   * oracle_grad_dual : forward mode with dual numbers, derivative factors
//                        obtained by automatic differentiation of the BSDF code.
// The conventions the paper leaves open (RNG seeding, random-number layout,
// depth convention, ray offsets, Fresnel, MIS, roulette) are fixed in
// `render_sample` below and restated on the GPU side independently.
//
// Parity notes: no function here is "parity unpinned"; the pins are the
// closed forms and finite-difference tests under tests/.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- vectors
struct V3 {
  double x = 0, y = 0, z = 0;
  V3() = default;
  V3(double a, double b, double c) : x(a), y(b), z(c) {}
  double operator[](int i) const { return i == 0 ? x : (i == 1 ? y : z); }
  double& operator[](int i) { return i == 0 ? x : (i == 1 ? y : z); }
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator*(double s, V3 a) { return a * s; }
inline V3 mul(V3 a, V3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double length(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return a * (1.0 / length(a)); }
inline double max3(V3 a) { return std::max(a.x, std::max(a.y, a.z)); }

// ---------------------------------------------------------------- PCG32
// O'Neill (2014), "PCG: A family of simple fast space-efficient statistically
// good algorithms for random number generation": 64-bit LCG state with the
// XSH-RR output function; the paper uses it as its per-lane sampler (Sec. 3.1).
struct Pcg32 {
  uint64_t state = 0, inc = 0;
  void seed(uint64_t initstate, uint64_t initseq) {
    state = 0;
    inc = (initseq << 1u) | 1u;
    next_u32();
    state += initstate;
    next_u32();
  }
  uint32_t next_u32() {
    uint64_t old = state;
    state = old * 6364136223846793005ULL + inc;
    uint32_t xorshifted = (uint32_t)(((old >> 18u) ^ old) >> 27u);
    uint32_t rot = (uint32_t)(old >> 59u);
    return (xorshifted >> rot) | (xorshifted << ((0u - rot) & 31u));
  }
  // 24 high bits -> [0,1): exact in both single and double precision.
  double uniform() { return (double)(next_u32() >> 8) * (1.0 / 16777216.0); }
};

// ---------------------------------------------------------------- dual numbers
// Forward-mode AD value with a fixed number of tangent slots.
struct Dual {
  double v = 0;
  std::vector<double> d;
  Dual() = default;
  Dual(double val, size_t n) : v(val), d(n, 0.0) {}
};
inline size_t nd(const Dual& a, const Dual& b) { return std::max(a.d.size(), b.d.size()); }
inline double tg(const Dual& a, size_t i) { return i < a.d.size() ? a.d[i] : 0.0; }
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v, nd(a, b));
  for (size_t i = 0; i < r.d.size(); ++i) r.d[i] = tg(a, i) + tg(b, i);
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v, nd(a, b));
  for (size_t i = 0; i < r.d.size(); ++i) r.d[i] = tg(a, i) - tg(b, i);
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v, nd(a, b));
  for (size_t i = 0; i < r.d.size(); ++i) r.d[i] = tg(a, i) * b.v + a.v * tg(b, i);
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v, nd(a, b));
  for (size_t i = 0; i < r.d.size(); ++i) r.d[i] = (tg(a, i) * b.v - a.v * tg(b, i)) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
inline Dual operator+(double b, const Dual& a) { return a + b; }
inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
inline Dual operator-(double b, const Dual& a) { Dual r = a; r.v = b - a.v; for (auto& x : r.d) x = -x; return r; }
inline Dual operator*(const Dual& a, double b) { Dual r = a; r.v *= b; for (auto& x : r.d) x *= b; return r; }
inline Dual operator*(double b, const Dual& a) { return a * b; }
inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
inline Dual operator/(double b, const Dual& a) { return Dual(b, a.d.size()) / a; }
inline Dual dsqrt(const Dual& a) {
  Dual r = a;
  r.v = std::sqrt(a.v);
  for (auto& x : r.d) x = x / (2.0 * r.v);
  return r;
}
inline double dsqrt(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }

// ---------------------------------------------------------------- scene
enum { BSDF_NONE = 0, BSDF_DIFFUSE = 1, BSDF_CONDUCTOR = 2, BSDF_DIELECTRIC = 3, BSDF_BLEND = 4 };

struct Shape {
  int bsdf, tex, albedo_index, rough_index;
  double alpha, eta, diffuse_weight;
  V3 f0, emission;
  bool emitter;
};

struct Texture {
  int w = 0, h = 0;
  std::vector<double> rgba;  // [h][w][4]
};

struct Node {  // binary BVH node of the oracle's own (median-split) tree
  V3 lo, hi;
  int left = -1, right = -1;  // children, or -1 for a leaf
  int first = 0, count = 0;   // leaf: range into `order`
};

struct Scene {
  int n_tris = 0;
  std::vector<V3> v0, v1, v2;        // vertices (FP32 inputs widened to FP64)
  std::vector<double> uv;            // [n][3][2]
  std::vector<int> tri_shape;
  std::vector<Shape> shapes;
  std::vector<double> albedo;        // [A][3]
  std::vector<Texture> tex;
  std::vector<double> roughness;
  // emitters (area lights): triangle ids and area CDF
  std::vector<int> light_tris;
  std::vector<double> light_cdf;     // normalised, size n+1
  double light_area = 0;
  // environment map
  int env_w = 0, env_h = 0;
  std::vector<double> env;           // [h][w][4]
  std::vector<double> env_marg;      // normalised, size h+1
  std::vector<double> env_cond;      // normalised per row, [h][w+1]
  std::vector<double> env_p;         // pixel probability [h][w]
  // BVH
  std::vector<Node> nodes;
  std::vector<int> order;
};

// oracle-side input record (plain pointers, host memory)
}  // namespace

extern "C" {
typedef struct {
  int n_tris;
  const float* vertices;   // [n][3][3]
  const float* uvs;        // [n][3][2]
  const int* tri_shape;    // [n]
  int n_shapes;
  const int* bsdf;
  const int* tex;
  const int* albedo_index;
  const int* rough_index;
  const float* alpha;
  const float* f0;         // [s][3]
  const float* eta;
  const float* emission;   // [s][3]
  const float* diffuse_weight;
  int n_albedo;
  const float* albedo;     // [a][3]
  int n_tex;
  const float* const* tex_data;  // each [h][w][4]
  const int* tex_w;
  const int* tex_h;
  int n_rough;
  const float* roughness;
  int env_w, env_h;
  const float* env;        // [h][w][4] or NULL
} oracle_scene_in;

typedef struct {
  double origin[3], target[3], up[3];
  double vfov_deg;
  int width, height;
  int spp, max_depth, rr_depth, nee;
  uint64_t seed;
  int cam_index;
  int crop_x0, crop_y0, crop_w, crop_h;  // crop_w == 0: whole image
  // Environment radiance used for shading, [env_h][env_w][4], or NULL for the
  // scene's map.  Sampling always uses the scene's map (detached sampling).
  const double* env_radiance;
} oracle_render_in;

// Options of the reparameterized translation derivative (see ReparamOpts).
typedef struct {
  int n_aux;
  double kappa, kernel_scale, power, miss, eps;
  int jackknife;
  double border;
  int edge_spp;
} oracle_reparam_opts;
}

namespace {

// ---------------------------------------------------------------- BVH (own, simple)
// Object-median split on the longest centroid axis, leaves of <= 4 triangles.
// Quality is irrelevant here; it only has to find the same closest hit as
// brute force (pinned by tests).
void tri_bounds(const Scene& s, int t, V3& lo, V3& hi) {
  for (int k = 0; k < 3; ++k) {
    double a = s.v0[t][k], b = s.v1[t][k], c = s.v2[t][k];
    lo[k] = std::min(a, std::min(b, c));
    hi[k] = std::max(a, std::max(b, c));
  }
}

int build_node(Scene& s, int first, int count) {
  Node n;
  n.lo = V3(1e300, 1e300, 1e300);
  n.hi = V3(-1e300, -1e300, -1e300);
  for (int i = first; i < first + count; ++i) {
    V3 lo, hi;
    tri_bounds(s, s.order[i], lo, hi);
    for (int k = 0; k < 3; ++k) {
      n.lo[k] = std::min(n.lo[k], lo[k]);
      n.hi[k] = std::max(n.hi[k], hi[k]);
    }
  }
  // inflate slightly so that slab tests never reject a boundary hit
  for (int k = 0; k < 3; ++k) {
    double pad = 1e-9 * (1.0 + std::fabs(n.lo[k]) + std::fabs(n.hi[k]));
    n.lo[k] -= pad;
    n.hi[k] += pad;
  }
  int id = (int)s.nodes.size();
  s.nodes.push_back(n);
  if (count <= 4) {
    s.nodes[id].first = first;
    s.nodes[id].count = count;
    return id;
  }
  V3 clo(1e300, 1e300, 1e300), chi(-1e300, -1e300, -1e300);
  auto centroid = [&](int t) { return (s.v0[t] + s.v1[t] + s.v2[t]) * (1.0 / 3.0); };
  for (int i = first; i < first + count; ++i) {
    V3 c = centroid(s.order[i]);
    for (int k = 0; k < 3; ++k) {
      clo[k] = std::min(clo[k], c[k]);
      chi[k] = std::max(chi[k], c[k]);
    }
  }
  V3 ext = chi - clo;
  int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
  int mid = first + count / 2;
  std::nth_element(s.order.begin() + first, s.order.begin() + mid, s.order.begin() + first + count,
                   [&](int a, int b) {
                     double ca = centroid(a)[axis], cb = centroid(b)[axis];
                     return ca < cb || (ca == cb && a < b);
                   });
  int l = build_node(s, first, mid - first);
  int r = build_node(s, mid, first + count - mid);
  s.nodes[id].left = l;
  s.nodes[id].right = r;
  return id;
}

bool hit_box(const Node& n, V3 o, V3 inv_d, double tmax) {
  double t0 = 0.0, t1 = tmax;
  for (int k = 0; k < 3; ++k) {
    double a = (n.lo[k] - o[k]) * inv_d[k];
    double b = (n.hi[k] - o[k]) * inv_d[k];
    if (std::isnan(a) || std::isnan(b)) {  // 0 * inf: ray parallel and on the slab plane
      if (o[k] < n.lo[k] || o[k] > n.hi[k]) return false;
      continue;
    }
    if (a > b) std::swap(a, b);
    t0 = std::max(t0, a);
    t1 = std::min(t1, b);
    if (t0 > t1) return false;
  }
  return true;
}

// Moller-Trumbore ray/triangle test in FP64.  Edges inclusive; det == 0 misses.
bool intersect_tri(const Scene& s, int t, V3 o, V3 d, double& th, double& bu, double& bv) {
  V3 e1 = s.v1[t] - s.v0[t];
  V3 e2 = s.v2[t] - s.v0[t];
  V3 p = cross(d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  V3 sv = o - s.v0[t];
  double u = dot(sv, p) * inv;
  if (u < 0.0 || u > 1.0) return false;
  V3 q = cross(sv, e1);
  double v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  double tt = dot(e2, q) * inv;
  if (!(tt > 0.0)) return false;
  th = tt;
  bu = u;
  bv = v;
  return true;
}

thread_local uint64_t g_rays = 0;  // rays traced by this thread (closest-hit + shadow)

struct Hit {
  int prim = -1;
  double t = 0, u = 0, v = 0;
};

// Closest hit with t in (0, tmax); ties broken by the smaller triangle index.
Hit closest_hit(const Scene& s, V3 o, V3 d, double tmax, bool brute) {
  ++g_rays;
  Hit h;
  double best = tmax;
  auto test = [&](int t) {
    double th, u, v;
    if (!intersect_tri(s, t, o, d, th, u, v)) return;
    if (th < best || (h.prim >= 0 && th == best && t < h.prim)) {
      best = th;
      h.prim = t;
      h.t = th;
      h.u = u;
      h.v = v;
    }
  };
  if (brute || s.nodes.empty()) {
    for (int t = 0; t < s.n_tris; ++t) test(t);
    return h;
  }
  V3 inv(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
  std::vector<int> stack;
  stack.push_back(0);
  while (!stack.empty()) {
    int ni = stack.back();
    stack.pop_back();
    const Node& n = s.nodes[ni];
    if (!hit_box(n, o, inv, best)) continue;
    if (n.left < 0) {
      for (int i = n.first; i < n.first + n.count; ++i) test(s.order[i]);
    } else {
      stack.push_back(n.left);
      stack.push_back(n.right);
    }
  }
  return h;
}

bool occluded(const Scene& s, V3 o, V3 d, double tmax) {
  Hit h = closest_hit(s, o, d, tmax, false);
  return h.prim >= 0;
}

V3 geo_normal(const Scene& s, int t) { return normalize(cross(s.v1[t] - s.v0[t], s.v2[t] - s.v0[t])); }

// Ray origin offset: p + n_g * sign(n_g . d) * eps, eps = 1e-4 * max(1, max|p_i|).
V3 offset_origin(V3 p, V3 ng, V3 d) {
  double eps = 1e-4 * std::max(1.0, std::max(std::fabs(p.x), std::max(std::fabs(p.y), std::fabs(p.z))));
  return p + ng * (dot(ng, d) >= 0.0 ? eps : -eps);
}

// ---------------------------------------------------------------- frames
// Orthonormal basis around n (Duff et al. 2017, "Building an orthonormal basis,
// revisited"), with the branch taken on n.z >= 0 so that +0 and -0 agree.
struct Frame {
  V3 s, t, n;
  V3 to_local(V3 w) const { return {dot(w, s), dot(w, t), dot(w, n)}; }
  V3 to_world(V3 v) const { return s * v.x + t * v.y + n * v.z; }
};
Frame make_frame(V3 n) {
  double sign = n.z >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  Frame f;
  f.n = n;
  f.s = V3(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  f.t = V3(b, sign + n.y * n.y * a, -n.y);
  return f;
}

// ---------------------------------------------------------------- BSDFs
// Local shading space: the normal is +z and faces the incident direction wi.
// Derivative-carrying inputs (albedo, alpha) are templated on T = double/Dual.
template <class T>
T ggx_D(const T& alpha, double cos_h) {
  T a2 = alpha * alpha;
  T den = (cos_h * cos_h) * (a2 - 1.0) + 1.0;
  return a2 / (kPi * (den * den));
}
template <class T>
T ggx_G1(const T& alpha, double cos_w) {
  double tan2 = (1.0 - cos_w * cos_w) / (cos_w * cos_w);
  return 2.0 / (1.0 + dsqrt(1.0 + (alpha * alpha) * tan2));
}
double schlick(double f0, double cos_d) {
  double m = 1.0 - cos_d;
  return f0 + (1.0 - f0) * m * m * m * m * m;
}
template <class T>
void ggx_eval(const T& alpha, V3 f0, V3 wi, V3 wo, T out[3]) {
  V3 h = normalize(wi + wo);
  T D = ggx_D(alpha, h.z);
  T G = ggx_G1(alpha, wi.z) * ggx_G1(alpha, wo.z);
  double cd = dot(wi, h);
  for (int c = 0; c < 3; ++c) out[c] = D * G * (schlick(f0[c], cd) / (4.0 * wi.z * wo.z));
}
double ggx_pdf(double alpha, V3 wi, V3 wo) {
  V3 h = normalize(wi + wo);
  double D = ggx_D<double>(alpha, h.z);
  return D * h.z / (4.0 * std::fabs(dot(wo, h)));
}
// Walter et al. 2007 half-vector sampling: phi = 2 pi u4, tan^2 theta_h = a^2 u5 / (1 - u5)
bool ggx_sample(double alpha, V3 wi, double u4, double u5, V3& wo) {
  double phi = 2.0 * kPi * u4;
  double tan2 = alpha * alpha * u5 / (1.0 - u5);
  double cos_t = 1.0 / std::sqrt(1.0 + tan2);
  double sin_t = std::sqrt(std::max(0.0, 1.0 - cos_t * cos_t));
  V3 h(sin_t * std::cos(phi), sin_t * std::sin(phi), cos_t);
  wo = h * (2.0 * dot(wi, h)) - wi;
  return wo.z > 0.0;
}

// Cosine-weighted hemisphere, mapping of the ambient-occlusion example (Sec. 3.1):
// phi = 2 pi u4, sin^2 theta = u5.
V3 cosine_sample(double u4, double u5) {
  double phi = 2.0 * kPi * u4;
  double r = std::sqrt(u5);
  return {std::cos(phi) * r, std::sin(phi) * r, std::sqrt(1.0 - u5)};
}

// The material seen at one vertex, with its differentiable inputs resolved.
struct Mat {
  int bsdf;
  V3 albedo;        // diffuse / blend albedo
  double alpha;     // GGX roughness
  V3 f0;
  double eta, wd;
  // parameter references for gradients
  int alb_kind;     // 0 none, 1 constant row, 2 texel
  int alb_row, tex_id;
  long long texel;  // linear texel index y*w + x
  int rough;        // roughness entry or -1
};

template <class T>
void bsdf_eval_t(const Mat& m, const T alb[3], const T& alpha, V3 wi, V3 wo, T out[3]) {
  for (int c = 0; c < 3; ++c) out[c] = alb[c] * 0.0;
  if (wi.z <= 0.0 || wo.z <= 0.0) return;
  if (m.bsdf == BSDF_DIFFUSE) {
    for (int c = 0; c < 3; ++c) out[c] = alb[c] * (1.0 / kPi);
  } else if (m.bsdf == BSDF_CONDUCTOR) {
    ggx_eval(alpha, m.f0, wi, wo, out);
  } else if (m.bsdf == BSDF_BLEND) {
    T g[3];
    ggx_eval(alpha, m.f0, wi, wo, g);
    for (int c = 0; c < 3; ++c) out[c] = alb[c] * (m.wd / kPi) + g[c] * (1.0 - m.wd);
  }
}
V3 bsdf_eval(const Mat& m, V3 wi, V3 wo) {
  double alb[3] = {m.albedo.x, m.albedo.y, m.albedo.z}, out[3];
  bsdf_eval_t<double>(m, alb, m.alpha, wi, wo, out);
  return {out[0], out[1], out[2]};
}
double bsdf_pdf(const Mat& m, V3 wi, V3 wo) {
  if (wi.z <= 0.0 || wo.z <= 0.0) return 0.0;
  if (m.bsdf == BSDF_DIFFUSE) return wo.z / kPi;
  if (m.bsdf == BSDF_CONDUCTOR) return ggx_pdf(m.alpha, wi, wo);
  if (m.bsdf == BSDF_BLEND) return m.wd * wo.z / kPi + (1.0 - m.wd) * ggx_pdf(m.alpha, wi, wo);
  return 0.0;
}

// Analytic derivative factors (d f_c / d theta) / f_c for the stored-tape method.
struct DFactors {
  V3 d_alb;    // per channel: (d f_c / d albedo_c) / f_c
  V3 d_alpha;  // per channel: (d f_c / d alpha) / f_c
};
DFactors bsdf_dfactors(const Mat& m, V3 wi, V3 wo) {
  DFactors r;
  V3 f = bsdf_eval(m, wi, wo);
  if (wi.z <= 0.0 || wo.z <= 0.0) return r;
  // d ln f_ggx / d alpha = 2/a - 4 a c^2 / (c^2 (a^2-1) + 1) - sum_w (a T_w / s_w) / (1 + s_w)
  auto dlog_ggx = [&](double a) {
    V3 h = normalize(wi + wo);
    double c2 = h.z * h.z;
    double r0 = 2.0 / a - 4.0 * a * c2 / (c2 * (a * a - 1.0) + 1.0);
    for (double cw : {wi.z, wo.z}) {
      double T = (1.0 - cw * cw) / (cw * cw);
      double sw = std::sqrt(1.0 + a * a * T);
      r0 -= (a * T / sw) / (1.0 + sw);
    }
    return r0;
  };
  if (m.bsdf == BSDF_DIFFUSE) {
    for (int c = 0; c < 3; ++c) r.d_alb[c] = f[c] > 0 ? (1.0 / kPi) / f[c] : 0.0;
  } else if (m.bsdf == BSDF_CONDUCTOR) {
    double dl = dlog_ggx(m.alpha);
    for (int c = 0; c < 3; ++c) r.d_alpha[c] = f[c] > 0 ? dl : 0.0;
  } else if (m.bsdf == BSDF_BLEND) {
    double alb0[3] = {0, 0, 0}, g[3];
    Mat mg = m;
    mg.bsdf = BSDF_CONDUCTOR;
    bsdf_eval_t<double>(mg, alb0, m.alpha, wi, wo, g);
    double dl = dlog_ggx(m.alpha);
    for (int c = 0; c < 3; ++c) {
      if (f[c] <= 0) continue;
      r.d_alb[c] = (m.wd / kPi) / f[c];
      r.d_alpha[c] = (1.0 - m.wd) * g[c] * dl / f[c];
    }
  }
  return r;
}

// Exact unpolarised Fresnel reflectance of a smooth dielectric interface.
// eta = n_t / n_i, cos_i >= 0.  Returns F and cos_t (0 on total internal reflection).
double fresnel_dielectric(double cos_i, double eta, double& cos_t) {
  double sin2_t = (1.0 - cos_i * cos_i) / (eta * eta);
  if (sin2_t >= 1.0) {
    cos_t = 0.0;
    return 1.0;
  }
  cos_t = std::sqrt(1.0 - sin2_t);
  double rs = (cos_i - eta * cos_t) / (cos_i + eta * cos_t);
  double rp = (eta * cos_i - cos_t) / (eta * cos_i + cos_t);
  return 0.5 * (rs * rs + rp * rp);
}

// One scattering event at a smooth dielectric interface with geometric normal ng
// (oriented outward, so that a ray arriving against it enters the medium of
// relative index eta_shape) and incident direction wi_w (pointing away from the
// surface).  Reflection is chosen with probability F (uniform u3 < F) and keeps
// the radiance; refraction follows Snell's law and scales radiance by 1/eta^2,
// eta being the index of the far side over the near side (radiance mode).
// Returns true if the ray refracted; wo is the outgoing direction.
bool dielectric_scatter(V3 ng, V3 wi_w, double eta_shape, double u3, V3& wo, double& weight) {
  bool entering = dot(ng, wi_w) > 0.0;
  V3 n = entering ? ng : -ng;
  double eta = entering ? eta_shape : 1.0 / eta_shape;
  double cos_i = dot(n, wi_w), cos_t;
  double F = fresnel_dielectric(cos_i, eta, cos_t);
  if (u3 < F) {
    wo = n * (2.0 * cos_i) - wi_w;
    weight = 1.0;
    return false;
  }
  wo = -wi_w * (1.0 / eta) + n * (cos_i / eta - cos_t);
  weight = 1.0 / (eta * eta);
  return true;
}

// ---------------------------------------------------------------- emitters
V3 env_lookup(const Scene& s, V3 d, int& px, int& py) {
  double phi = std::atan2(d.z, d.x);
  if (phi < 0.0) phi += 2.0 * kPi;
  double theta = std::acos(std::min(1.0, std::max(-1.0, d.y)));
  double u = phi / (2.0 * kPi), v = theta / kPi;
  px = std::min((int)(u * s.env_w), s.env_w - 1);
  py = std::min((int)(v * s.env_h), s.env_h - 1);
  const double* e = &s.env[((size_t)py * s.env_w + px) * 4];
  return {e[0], e[1], e[2]};
}
// Radiance of env pixel (x, y): the render's override, else the scene's map.
V3 env_value(const Scene& s, const oracle_render_in& r, int x, int y) {
  const double* e = r.env_radiance ? &r.env_radiance[((size_t)y * s.env_w + x) * 4]
                                   : &s.env[((size_t)y * s.env_w + x) * 4];
  return {e[0], e[1], e[2]};
}
// Solid-angle density of the environment sampler at direction d.
double env_pdf(const Scene& s, V3 d) {
  int px, py;
  env_lookup(s, d, px, py);
  double sin_t = std::sqrt(std::max(0.0, 1.0 - d.y * d.y));
  if (sin_t == 0.0) return 0.0;
  double p = s.env_p[(size_t)py * s.env_w + px] * s.env_w * s.env_h;
  return p / (2.0 * kPi * kPi * sin_t);
}
// first index i with u < cdf[i+1]; cdf normalised, size n+1
int cdf_pick(const double* cdf, int n, double u) {
  int i = (int)(std::upper_bound(cdf + 1, cdf + n + 1, u) - (cdf + 1));
  return std::min(std::max(i, 0), n - 1);
}

double power_heuristic(double a, double b) {
  double a2 = a * a, b2 = b * b;
  return (a2 + b2) > 0.0 ? a2 / (a2 + b2) : 0.0;
}

Mat resolve_material(const Scene& s, int shape, double tu, double tv) {
  const Shape& sh = s.shapes[shape];
  Mat m{};
  m.bsdf = sh.bsdf;
  m.alpha = sh.rough_index >= 0 ? s.roughness[sh.rough_index] : sh.alpha;
  m.rough = sh.rough_index;
  m.f0 = sh.f0;
  m.eta = sh.eta;
  m.wd = sh.diffuse_weight;
  m.alb_kind = 0;
  if (sh.bsdf == BSDF_DIFFUSE || sh.bsdf == BSDF_BLEND) {
    if (sh.tex >= 0) {
      // nearest lookup as in the paper's closure example (App. B):
      // pos = min(uint(uv * res), res - 1), texel [pos.y, pos.x]
      const Texture& t = s.tex[sh.tex];
      int x = std::min((int)(std::max(tu, 0.0) * t.w), t.w - 1);
      int y = std::min((int)(std::max(tv, 0.0) * t.h), t.h - 1);
      const double* p = &t.rgba[((size_t)y * t.w + x) * 4];
      m.albedo = V3(p[0], p[1], p[2]);
      m.alb_kind = 2;
      m.tex_id = sh.tex;
      m.texel = (long long)y * t.w + x;
    } else if (sh.albedo_index >= 0) {
      const double* p = &s.albedo[(size_t)sh.albedo_index * 3];
      m.albedo = V3(p[0], p[1], p[2]);
      m.alb_kind = 1;
      m.alb_row = sh.albedo_index;
    }
  }
  return m;
}

// ---------------------------------------------------------------- integrator
// FNV-1a over 32-bit words: a fingerprint of the discrete decisions of a path
// (hit triangles, light picks, visibility, lobes, texels, roulette).
struct DecisionHash {
  uint32_t h = 2166136261u;
  void add(uint32_t w) { h = (h ^ w) * 16777619u; }
};

struct Camera {
  V3 o, fwd, right, up;
  double tan_half, aspect;
  int w, h;
};
Camera make_camera(const oracle_render_in& r) {
  Camera c;
  c.o = V3(r.origin[0], r.origin[1], r.origin[2]);
  V3 t(r.target[0], r.target[1], r.target[2]);
  V3 up(r.up[0], r.up[1], r.up[2]);
  c.fwd = normalize(t - c.o);
  c.right = normalize(cross(c.fwd, up));
  c.up = cross(c.right, c.fwd);
  c.tan_half = std::tan(0.5 * r.vfov_deg * kPi / 180.0);
  c.w = r.width;
  c.h = r.height;
  c.aspect = (double)r.width / (double)r.height;
  return c;
}

// Events reported by the integrator to an accumulator.  `scatter` is called
// for every continued vertex with the throughput factor of the sampled
// direction; the accumulators decide what to do with derivative information.
// The ray events (camera ray, the block of auxiliary random numbers a vertex
// draws, the unoccluded light-sample ray and the sampled continuation ray) are
// only used by the reparameterized derivative; the others inherit no-ops.
struct NoRayEvents {
  void camera_ray(uint64_t, V3, V3, V3) {}
  void vertex_block() {}
  void nee_ray(V3, V3, int, double, double, V3, int) {}
  void bsdf_ray(V3, V3, int, double, double, V3, int) {}
};
struct VertexInfo {
  Mat m;
  V3 wi;        // local incident direction (toward the previous vertex)
};

// Radiance-cache termination for the oracle: the MLP of mlp.cpp evaluated on
// the raw features of the termination vertex (same definition as the kernels:
// paths end at the first non-delta vertex reached by segment >= bounce).
struct CacheModel {
  const double* W = nullptr;  // NULL: no cache
  double box[6];
  int bounce = 0;
};
struct TrainRecord {
  double raw[10];
  V3 beta, L_before;
  int depth;
};

}  // namespace
extern "C" void oracle_nrc_encode(int n, const double* raw, const double* box, double* enc_out);
extern "C" void oracle_mlp_forward(const double* W, int n, const double* enc, double* out);
namespace {

// A path started on a pixel edge instead of inside a pixel (the reparameterized
// derivative's pixel-edge term): its own stream, and the image-plane point (X, Y +
// j0) on a vertical edge or (X + j0, Y) on a horizontal one, in pixel coordinates.
struct EdgeStart {
  uint64_t stream;
  bool vertical;
  int X, Y;
};

template <class Acc>
V3 render_sample(const Scene& s, const Camera& cam, const oracle_render_in& r, int px, int py,
                 int spp_index, Acc& acc, uint32_t* hash_out, const CacheModel* cache = nullptr,
                 std::vector<TrainRecord>* records = nullptr, const EdgeStart* edge = nullptr) {
  // RNG stream of this sample: (camera << 40) | (pixel << 12) | sample
  Pcg32 rng;
  uint64_t pixel = (uint64_t)py * (uint64_t)r.width + (uint64_t)px;
  uint64_t stream = ((uint64_t)r.cam_index << 40) | (pixel << 12) | (uint64_t)spp_index;
  if (edge) stream = edge->stream;
  rng.seed(r.seed, stream);
  DecisionHash dh;

  double j0 = rng.uniform(), j1 = rng.uniform();
  double fx = px + j0, fy = py + j1;
  if (edge) {
    fx = edge->vertical ? edge->X : edge->X + j0;
    fy = edge->vertical ? edge->Y + j0 : edge->Y;
  }
  double sx = (2.0 * fx / cam.w - 1.0) * cam.tan_half * cam.aspect;
  double sy = (1.0 - 2.0 * fy / cam.h) * cam.tan_half;
  V3 ro = cam.o;
  V3 rd = normalize(cam.fwd + cam.right * sx + cam.up * sy);
  acc.camera_ray(stream, ro, rd, cam.fwd);

  bool has_area = !s.light_tris.empty();
  bool has_env = s.env_w > 0;
  double p_env = has_env ? (has_area ? 0.5 : 1.0) : 0.0;
  double p_area = has_area ? 1.0 - p_env : 0.0;

  V3 beta(1, 1, 1), L(0, 0, 0);
  bool prev_delta = true;
  double prev_pdf = 0.0;
  for (int depth = 1;; ++depth) {
    Hit hit = closest_hit(s, ro, rd, INFINITY, false);
    dh.add(hit.prim < 0 ? 0xffffffffu : (uint32_t)hit.prim);
    if (hit.prim < 0) {
      if (has_env) {
        int ex, ey;
        env_lookup(s, rd, ex, ey);
        V3 Le = env_value(s, r, ex, ey);
        double w = (prev_delta || !r.nee) ? 1.0 : power_heuristic(prev_pdf, p_env * env_pdf(s, rd));
        V3 c = mul(beta, Le) * w;
        L = L + c;
        acc.emission(c, Le * w, ey * s.env_w + ex, beta * w, w);
      }
      break;
    }
    int t = hit.prim;
    const Shape& sh = s.shapes[s.tri_shape[t]];
    V3 ng = geo_normal(s, t);
    V3 wi_w = -rd;
    double cos_front = dot(ng, wi_w);
    if (sh.emitter && cos_front > 0.0) {
      double w = 1.0;  // no MIS without light sampling or after a delta lobe
      if (!prev_delta && r.nee) {
        double pdf_l = p_area * hit.t * hit.t / (cos_front * s.light_area);
        w = power_heuristic(prev_pdf, pdf_l);
      }
      V3 c = mul(beta, sh.emission) * w;
      L = L + c;
      acc.emission(c, sh.emission * w, -1, V3(), 0.0);
    }
    if (depth >= r.max_depth) break;
    double u[8];
    for (int k = 0; k < 8; ++k) u[k] = rng.uniform();
    acc.vertex_block();
    if (sh.bsdf == BSDF_NONE) break;

    V3 p = ro + rd * hit.t;
    const double* tuv = &s.uv[(size_t)t * 6];
    double b0 = 1.0 - hit.u - hit.v;
    double tu = b0 * tuv[0] + hit.u * tuv[2] + hit.v * tuv[4];
    double tv = b0 * tuv[1] + hit.u * tuv[3] + hit.v * tuv[5];
    VertexInfo vi;
    vi.m = resolve_material(s, s.tri_shape[t], tu, tv);
    dh.add(vi.m.alb_kind == 2 ? (uint32_t)vi.m.texel : 0xffffffffu);
    if ((cache && cache->W) || records) {
      if (sh.bsdf != BSDF_DIELECTRIC) {
        V3 n = cos_front > 0.0 ? ng : -ng;
        double rough = (sh.bsdf == BSDF_CONDUCTOR || sh.bsdf == BSDF_BLEND) ? vi.m.alpha : 1.0;
        double raw[10] = {p.x, p.y, p.z, wi_w.x, wi_w.y, wi_w.z, n.x, n.y, n.z, rough};
        if (records) {
          TrainRecord rec;
          std::memcpy(rec.raw, raw, sizeof raw);
          rec.beta = beta;
          rec.L_before = L;
          rec.depth = depth;
          records->push_back(rec);
        } else if (depth >= cache->bounce) {
          double enc[64], y[3];
          oracle_nrc_encode(1, raw, cache->box, enc);
          oracle_mlp_forward(cache->W, 1, enc, y);
          V3 Lc(std::max(y[0], 0.0), std::max(y[1], 0.0), std::max(y[2], 0.0));
          V3 c = mul(beta, Lc);
          L = L + c;
          acc.emission(c, Lc, -1, V3(), 0.0);
          break;
        }
      }
    }

    if (sh.bsdf == BSDF_DIELECTRIC) {
      V3 wo;
      double weight;
      bool refracted = dielectric_scatter(ng, wi_w, sh.eta, u[3], wo, weight);
      dh.add(refracted ? 3 : 2);
      dh.add(0xfffffffeu);  // no light sample at a delta vertex
      beta = beta * weight;
      acc.scatter_delta(weight);
      prev_delta = true;
      prev_pdf = 0.0;
      ro = offset_origin(p, ng, wo);
      rd = wo;
    } else {
      V3 n = cos_front > 0.0 ? ng : -ng;
      Frame fr = make_frame(n);
      vi.wi = fr.to_local(wi_w);
      // ---- next-event estimation
      if (r.nee && (has_area || has_env)) {
        bool pick_env = has_env && (!has_area || u[7] < 0.5);
        V3 dir, Le;
        double pdf_l = 0.0, dist = INFINITY;
        bool valid = false;
        int env_texel = -1;
        if (pick_env) {
          int y = cdf_pick(s.env_marg.data(), s.env_h, u[1]);
          const double* cond = &s.env_cond[(size_t)y * (s.env_w + 1)];
          int x = cdf_pick(cond, s.env_w, u[2]);
          double fv = (u[1] - s.env_marg[y]) / (s.env_marg[y + 1] - s.env_marg[y]);
          double fu = (u[2] - cond[x]) / (cond[x + 1] - cond[x]);
          double theta = kPi * (y + fv) / s.env_h, phi = 2.0 * kPi * (x + fu) / s.env_w;
          double st = std::sin(theta);
          dir = V3(st * std::cos(phi), std::cos(theta), st * std::sin(phi));
          Le = env_value(s, r, x, y);
          env_texel = y * s.env_w + x;
          double pdf_uv = s.env_p[(size_t)y * s.env_w + x] * s.env_w * s.env_h;
          pdf_l = st > 0.0 ? p_env * pdf_uv / (2.0 * kPi * kPi * st) : 0.0;
          valid = pdf_l > 0.0;
          dh.add(0x80000000u | (uint32_t)(y * s.env_w + x));
        } else {
          int k = cdf_pick(s.light_cdf.data(), (int)s.light_tris.size(), u[0]);
          int lt = s.light_tris[k];
          double su = std::sqrt(u[1]);
          double lb0 = 1.0 - su, lb1 = u[2] * su;
          V3 q = s.v0[lt] * lb0 + s.v1[lt] * lb1 + s.v2[lt] * (1.0 - lb0 - lb1);
          V3 dv = q - p;
          dist = length(dv);
          dir = dv * (1.0 / dist);
          V3 nl = geo_normal(s, lt);
          double cos_l = -dot(nl, dir);
          Le = s.shapes[s.tri_shape[lt]].emission;
          if (cos_l > 0.0 && dist > 0.0) {
            pdf_l = p_area * dist * dist / (cos_l * s.light_area);
            valid = true;
          }
          dh.add((uint32_t)lt);
        }
        V3 wl = fr.to_local(dir);
        V3 f = bsdf_eval(vi.m, vi.wi, wl);
        uint32_t vis_code = 2;
        if (valid && wl.z > 0.0 && max3(f) > 0.0) {
          V3 so = offset_origin(p, ng, dir);
          double tmax = pick_env ? INFINITY : dist * (1.0 - 1e-3);
          bool occ = occluded(s, so, dir, tmax);
          vis_code = occ ? 1 : 0;
          if (!occ) {
            double w = power_heuristic(pdf_l, bsdf_pdf(vi.m, vi.wi, wl));
            double s_env = wl.z * w / pdf_l;   // d scale / d Le
            V3 scale = Le * s_env;             // everything but beta and f
            V3 c = mul(mul(beta, f), scale);
            L = L + c;
            acc.nee_ray(so, dir, t, hit.u, hit.v, n, vi.m.bsdf);
            acc.nee(vi, wl, scale, c, env_texel, mul(beta, f) * s_env, s_env);
          }
        }
        dh.add(vis_code);
      }
      // ---- BSDF sampling
      V3 wo_l;
      bool ok = true;
      int lobe;
      if (vi.m.bsdf == BSDF_DIFFUSE) {
        wo_l = cosine_sample(u[4], u[5]);
        lobe = 0;
      } else if (vi.m.bsdf == BSDF_CONDUCTOR) {
        ok = ggx_sample(vi.m.alpha, vi.wi, u[4], u[5], wo_l);
        lobe = 1;
      } else {  // blend
        if (u[3] < vi.m.wd) {
          wo_l = cosine_sample(u[4], u[5]);
          lobe = 0;
        } else {
          ok = ggx_sample(vi.m.alpha, vi.wi, u[4], u[5], wo_l);
          lobe = 1;
        }
      }
      dh.add((uint32_t)lobe);
      if (!ok) break;
      double pdf = bsdf_pdf(vi.m, vi.wi, wo_l);
      V3 f = bsdf_eval(vi.m, vi.wi, wo_l);
      if (!(pdf > 0.0) || max3(f) <= 0.0) break;
      double k = wo_l.z / pdf;
      beta = mul(beta, f) * k;
      V3 wo = fr.to_world(wo_l);
      V3 ro_next = offset_origin(p, ng, wo);
      acc.bsdf_ray(ro_next, wo, t, hit.u, hit.v, n, vi.m.bsdf);
      acc.scatter(vi, wo_l, k);
      prev_delta = false;
      prev_pdf = pdf;
      ro = ro_next;
      rd = wo;
    }
    // ---- Russian roulette from depth rr_depth on
    if (r.rr_depth >= 0 && depth >= r.rr_depth) {
      double q = std::min(max3(beta), 0.95);
      bool cont = u[6] < q;
      dh.add(cont ? 1u : 0u);
      if (!cont) break;
      beta = beta * (1.0 / q);
      acc.roulette(q);
    }
  }
  if (hash_out) *hash_out = dh.h;
  return L;
}

// Accumulator for the plain render: ignores events.
struct NullAcc : NoRayEvents {
  void emission(V3, V3, int, V3, double) {}
  void nee(const VertexInfo&, V3, V3, V3, int, V3, double) {}
  void scatter(const VertexInfo&, V3, double) {}
  void scatter_delta(double) {}
  void roulette(double) {}
};

// Stored-tape accumulator: keeps every vertex record, then runs a reverse sweep.
struct TapeAcc : NoRayEvents {
  struct Rec {
    int kind;      // 0 emission, 1 nee, 2 scatter
    V3 c;          // contribution (emission / nee)
    Mat m;
    V3 wi, wo;
    int env_texel;  // emission / nee from the environment: its pixel, else -1
    V3 d_env;       // d contribution / d env radiance, per channel
  };
  std::vector<Rec> recs;
  void emission(V3 c, V3, int env_texel, V3 d_env, double) {
    recs.push_back({0, c, Mat{}, V3(), V3(), env_texel, d_env});
  }
  void nee(const VertexInfo& v, V3 wl, V3, V3 c, int env_texel, V3 d_env, double) {
    recs.push_back({1, c, v.m, v.wi, wl, env_texel, d_env});
  }
  void scatter(const VertexInfo& v, V3 wo, double) { recs.push_back({2, V3(), v.m, v.wi, wo, -1, V3()}); }
  void scatter_delta(double) {}
  void roulette(double) {}
};

struct GradOut {
  std::vector<double> albedo;                 // [A][3]
  std::vector<std::vector<double>> tex;       // each [h][w][4]
  std::vector<double> rough;                  // [R]
  std::vector<double> env;                    // [env_h][env_w][4]
};

void add_param_grad(GradOut& g, const Mat& m, V3 contrib, const DFactors& df, V3 dl) {
  if (m.alb_kind == 1) {
    for (int c = 0; c < 3; ++c) g.albedo[(size_t)m.alb_row * 3 + c] += dl[c] * contrib[c] * df.d_alb[c];
  } else if (m.alb_kind == 2) {
    for (int c = 0; c < 3; ++c) g.tex[m.tex_id][(size_t)m.texel * 4 + c] += dl[c] * contrib[c] * df.d_alb[c];
  }
  if (m.rough >= 0 && (m.bsdf == BSDF_CONDUCTOR || m.bsdf == BSDF_BLEND)) {
    double s = 0.0;
    for (int c = 0; c < 3; ++c) s += dl[c] * contrib[c] * df.d_alpha[c];
    g.rough[m.rough] += s;
  }
}

// Forward-mode accumulator: RGB dual throughput, dual radiance.
struct SelParam {
  int kind, a, b, c;  // 0: albedo (row a, channel b); 1: texel (tex a, texel b, channel c); 2: roughness a;
                      // 3: environment pixel a, channel b
};
struct DualAcc : NoRayEvents {
  const std::vector<SelParam>* sel;
  Dual beta[3], L[3];
  size_t n;
  void init(const std::vector<SelParam>* s) {
    sel = s;
    n = s->size();
    for (int c = 0; c < 3; ++c) {
      beta[c] = Dual(1.0, n);
      L[c] = Dual(0.0, n);
    }
  }
  void seeded_inputs(const Mat& m, Dual alb[3], Dual& alpha) const {
    for (int c = 0; c < 3; ++c) alb[c] = Dual(m.albedo[c], n);
    alpha = Dual(m.alpha, n);
    for (size_t i = 0; i < n; ++i) {
      const SelParam& p = (*sel)[i];
      if (p.kind == 0 && m.alb_kind == 1 && m.alb_row == p.a) alb[p.b].d[i] = 1.0;
      if (p.kind == 1 && m.alb_kind == 2 && m.tex_id == p.a && m.texel == p.b) alb[p.c].d[i] = 1.0;
      if (p.kind == 2 && m.rough == p.a) alpha.d[i] = 1.0;
    }
  }
  // le_w (or scale) as duals: derivative `k` in the slots of environment pixel `texel`
  void env_seeded(V3 v, int texel, double k, Dual out[3]) const {
    for (int c = 0; c < 3; ++c) out[c] = Dual(v[c], n);
    if (texel < 0) return;
    for (size_t i = 0; i < n; ++i) {
      const SelParam& p = (*sel)[i];
      if (p.kind == 3 && p.a == texel) out[p.b].d[i] = k;
    }
  }
  void emission(V3, V3 le_w, int env_texel, V3, double w_env) {
    Dual e[3];
    env_seeded(le_w, env_texel, w_env, e);
    for (int c = 0; c < 3; ++c) L[c] = L[c] + beta[c] * e[c];
  }
  void nee(const VertexInfo& v, V3 wl, V3 scale, V3, int env_texel, V3, double s_env) {
    Dual alb[3], alpha, f[3], sc[3];
    seeded_inputs(v.m, alb, alpha);
    bsdf_eval_t<Dual>(v.m, alb, alpha, v.wi, wl, f);
    env_seeded(scale, env_texel, s_env, sc);
    for (int c = 0; c < 3; ++c) L[c] = L[c] + beta[c] * f[c] * sc[c];
  }
  void scatter(const VertexInfo& v, V3 wo, double k) {
    Dual alb[3], alpha, f[3];
    seeded_inputs(v.m, alb, alpha);
    bsdf_eval_t<Dual>(v.m, alb, alpha, v.wi, wo, f);
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * f[c] * k;
  }
  void scatter_delta(double w) {
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * w;
  }
  void roulette(double q) {
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * (1.0 / q);
  }
};

// Forward-mode accumulator along one direction v of parameter space: one tangent
// slot holds d/d eps at eps = 0 of the estimator evaluated at (params + eps v).
// Sampling stays detached (the sampled directions do not move with eps), the
// same convention as the adjoint (Sec. 4.9).
struct Direction {
  const double* albedo = nullptr;         // [A][3] or null (zero)
  std::vector<const double*> tex;         // per texture [h][w][4] or null
  const double* rough = nullptr;          // [R] or null
  const double* env = nullptr;            // [env_h][env_w][4] or null
};
struct JvpAcc : NoRayEvents {
  const Direction* v;
  Dual beta[3], L[3];
  void init(const Direction* dir) {
    v = dir;
    for (int c = 0; c < 3; ++c) {
      beta[c] = Dual(1.0, 1);
      L[c] = Dual(0.0, 1);
    }
  }
  void seeded_inputs(const Mat& m, Dual alb[3], Dual& alpha) const {
    for (int c = 0; c < 3; ++c) alb[c] = Dual(m.albedo[c], 1);
    alpha = Dual(m.alpha, 1);
    if (m.alb_kind == 1 && v->albedo)
      for (int c = 0; c < 3; ++c) alb[c].d[0] = v->albedo[(size_t)m.alb_row * 3 + c];
    if (m.alb_kind == 2 && m.tex_id < (int)v->tex.size() && v->tex[m.tex_id])
      for (int c = 0; c < 3; ++c) alb[c].d[0] = v->tex[m.tex_id][(size_t)m.texel * 4 + c];
    if (m.rough >= 0 && v->rough) alpha.d[0] = v->rough[m.rough];
  }
  // le_w (or scale) as duals: tangent k * v_env at environment pixel `texel`
  void env_seeded(V3 val, int texel, double k, Dual out[3]) const {
    for (int c = 0; c < 3; ++c) {
      out[c] = Dual(val[c], 1);
      if (texel >= 0 && v->env) out[c].d[0] = k * v->env[(size_t)texel * 4 + c];
    }
  }
  void emission(V3, V3 le_w, int env_texel, V3, double w_env) {
    Dual e[3];
    env_seeded(le_w, env_texel, w_env, e);
    for (int c = 0; c < 3; ++c) L[c] = L[c] + beta[c] * e[c];
  }
  void nee(const VertexInfo& vi, V3 wl, V3 scale, V3, int env_texel, V3, double s_env) {
    Dual alb[3], alpha, f[3], sc[3];
    seeded_inputs(vi.m, alb, alpha);
    bsdf_eval_t<Dual>(vi.m, alb, alpha, vi.wi, wl, f);
    env_seeded(scale, env_texel, s_env, sc);
    for (int c = 0; c < 3; ++c) L[c] = L[c] + beta[c] * f[c] * sc[c];
  }
  void scatter(const VertexInfo& vi, V3 wo, double k) {
    Dual alb[3], alpha, f[3];
    seeded_inputs(vi.m, alb, alpha);
    bsdf_eval_t<Dual>(vi.m, alb, alpha, vi.wi, wo, f);
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * f[c] * k;
  }
  void scatter_delta(double w) {
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * w;
  }
  void roulette(double q) {
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * (1.0 / q);
  }
};

// ---------------------------------------------------------------- reparameterized derivatives
// Derivatives with respect to shape translations through visibility (Sec. 4.7,
// "Reparameterizations"; warp field after Bangaru et al. 2020).  Every ray the
// integrator traces is reparameterized: in the primal the warp is the identity;
// its derivative turns the ray direction by V(u) and multiplies the integrand by
// the Jacobian determinant 1 + div V.  The parameters are one translation per
// shape (all its vertices move together) or every triangle corner's position; a
// surface point keeps its barycentric coordinates, so path vertices move with
// their shape (or their triangle's corners).
//
// The warp field of a ray (origin o, primal direction u, origin shape s_o; the
// camera counts as static) is built from N auxiliary rays w_i drawn from the von
// Mises-Fisher lobe of concentration kappa around u (Jakob 2012, "Numerically
// stable sampling of the von Mises-Fisher distribution on S^2"), in the frame of u
// (Duff et al. 2017), with uniforms from the sample's auxiliary PCG32 stream.  An
// auxiliary ray that hits triangle i (plane n_i . (x - o) = d_i) says how a point
// of that plane moves relative to the origin: seen along w, the plane point at
// distance d_i / (n_i . w) moves with Delta_i = tau'(shape_i) - tau'(s_o), i.e. its
// direction turns by (I - w w^T) Delta_i (n_i . w) / d_i.  The warp is the
// kernel-weighted average of these velocities,
//   V(w) = sum_i k(w, w_i) g_i c_i(w) / q_i  /  ( sum_i k(w, w_i) g_i / q_i + N eps K ),
// with the vMF kernel k(w, w') = exp(kernel_scale kappa (w.w' - 1)) (narrower
// than the sampling density q), depth weights g_i = (t0 / t_i)^m relative to the
// ray's own hit distance t0 (1 if the ray escapes) so that the closer surface
// dominates near its silhouette, and escaping auxiliary rays weighted `miss` with
// velocity 0 (the environment does not move).  The samples are held fixed while V
// is evaluated at other w, so V is smooth; its divergence on the sphere is taken
// in the gnomonic chart around u with two-component dual numbers.  The ratio of
// sample sums is biased by O(1/N); the leave-one-out (jackknife) combination
// N f(all) - (N-1)/N sum_j f(all but j) removes the leading term.
//
// Each traced ray multiplies the integrand it carries by
//   camera ray: 1 + theta (div(bV) - 3 f.(bV) / f.u), the image-plane measure of
//               the pinhole (f = optical axis); b = 1, or with border > 0 a window
//               that takes the warp to 0 within `border` pixels of the image
//               border (an option: the pixel-edge term below makes it unneeded);
//   light and BSDF rays at diffuse, GGX-conductor and blend vertices:
//               1 + theta (div V + n.V / n.u), the cosine term; at the glossy
//               ones the BSDF value also turns with both of its directions
//               (grad_out log f_c . V of this ray, grad_in log f_c . -V of the
//               ray that arrived) and, with vertex positions as parameters, with
//               the triangle's normal.
// Rays leaving dielectric (delta) vertices are not reparameterized.  The warp of
// the camera rays also moves the pixels' own footprints: the pixel-edge term
// (paths through pixel edges) carries that flux.  The tangent of a sample is
// propagated forward along the path like the throughput (no replay): the
// oracle's independent route to the reverse-mode kernel's gradients, and its
// forward-mode image derivative.

struct ReparamOpts {
  int n_aux = 16;
  double kappa = 1000.0;      // concentration of the auxiliary-ray lobe
  double kernel_scale = 8.0;  // the weighting kernel is kernel_scale x narrower
  double power = 2.0;         // depth-weight exponent m
  double miss = 0.01;         // weight of an auxiliary ray that escapes (velocity 0)
  double eps = 1e-4;          // floor of the normaliser
  int jackknife = 1;          // leave-one-out correction of the ratio's 1/N bias
  double border = 0.0;        // camera-ray warp window at the image border, pixels (0: none)
  int edge_spp = 1;           // samples per pixel edge of the pixel-edge term (0: off)
};

// value and gradient in the two chart coordinates
struct D2 {
  double v = 0, a = 0, b = 0;
};
inline D2 operator+(D2 x, D2 y) { return {x.v + y.v, x.a + y.a, x.b + y.b}; }
inline D2 operator-(D2 x, D2 y) { return {x.v - y.v, x.a - y.a, x.b - y.b}; }
inline D2 operator*(D2 x, D2 y) { return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b}; }
inline D2 operator*(D2 x, double k) { return {x.v * k, x.a * k, x.b * k}; }
inline D2 operator/(D2 x, D2 y) {
  double q = x.v / y.v;
  return {q, (x.a - q * y.a) / y.v, (x.b - q * y.b) / y.v};
}
inline D2 d2exp(D2 x) {
  double e = std::exp(x.v);
  return {e, e * x.a, e * x.b};
}
inline D2 d2sqrt(D2 x) {
  double r = std::sqrt(x.v);
  return {r, x.a / (2.0 * r), x.b / (2.0 * r)};
}
struct VD {
  D2 x, y, z;
};
inline D2 dotd(VD p, V3 q) { return p.x * q.x + p.y * q.y + p.z * q.z; }
inline D2 dotd(VD p, VD q) { return p.x * q.x + p.y * q.y + p.z * q.z; }
inline VD scaled(V3 q, D2 k) { return {k * q.x, k * q.y, k * q.z}; }
inline VD operator+(VD p, VD q) { return {p.x + q.x, p.y + q.y, p.z + q.z}; }
inline VD divided(VD p, D2 k) { return {p.x / k, p.y / k, p.z / k}; }
inline VD constant(V3 q) { return {D2{q.x, 0, 0}, D2{q.y, 0, 0}, D2{q.z, 0, 0}}; }

// Divergence on the unit sphere at u of the field F (a functor VD -> VD taking a
// unit direction): in gnomonic coordinates x around u, w(x) = normalize(u + x1
// t1 + x2 t2), the field's coordinates are U_a = d x_a / d theta =
// [t_a.V (u.w) - (t_a.w)(u.V)] / (u.w)^2, and the chart's metric is Euclidean to
// first order at x = 0, so div = dU_1/dx1 + dU_2/dx2 there.
template <class F>
double sphere_div(V3 u, F field) {
  Frame fr = make_frame(u);
  VD wr{D2{u.x, fr.s.x, fr.t.x}, D2{u.y, fr.s.y, fr.t.y}, D2{u.z, fr.s.z, fr.t.z}};
  D2 len = d2sqrt(dotd(wr, wr));
  VD w = divided(wr, len);
  VD V = field(w);
  D2 uw = dotd(w, u), uV = dotd(V, u);
  D2 den = uw * uw;
  D2 U1 = (dotd(V, fr.s) * uw - dotd(w, fr.s) * uV) / den;
  D2 U2 = (dotd(V, fr.t) * uw - dotd(w, fr.t) * uV) / den;
  return U1.a + U2.b;
}

// Auxiliary rays of one warp, traced once at the primal center u.
struct AuxHit {
  V3 w;
  double t, g_over_q;
  int shape;
  V3 n;       // geometric normal of the hit triangle
  double d;   // n . (hit point - origin): the plane is {x : n.(x - o) = d}
  int tri;    // hit triangle (-1: escaped)
};
struct WarpSamples {
  V3 u;
  std::vector<AuxHit> hits;
  int n = 0;
  double kappa = 0, eps = 0, K = 0, kscale = 1.0;
  int jackknife = 0;
};

// vMF direction (local z = lobe axis) from two uniforms: cos(theta) = 1 + log(xi +
// (1 - xi) e^{-2 kappa}) / kappa with xi = 1 - u0 in (0, 1], phi = 2 pi u1.
V3 vmf_local(double u0, double u1, double kappa) {
  double xi = 1.0 - u0;
  double c1 = std::log(xi + (1.0 - xi) * std::exp(-2.0 * kappa)) / kappa;  // cos(theta) - 1
  double sin2 = std::max(0.0, -c1 * (2.0 + c1));
  double st = std::sqrt(sin2), phi = 2.0 * kPi * u1;
  return V3(st * std::cos(phi), st * std::sin(phi), 1.0 + c1);
}

WarpSamples warp_samples(const Scene& s, const ReparamOpts& op, V3 o, V3 u, const double* uni) {
  WarpSamples ws;
  ws.u = u;
  ws.n = op.n_aux;
  ws.kappa = op.kappa;
  ws.eps = op.eps;
  ws.kscale = op.kernel_scale;
  ws.jackknife = op.jackknife;
  ws.K = 2.0 * kPi * (1.0 - std::exp(-2.0 * op.kappa)) / op.kappa;  // integral of k
  const double Cq = 1.0 / ws.K;                                       // vMF normalisation
  Frame fr = make_frame(u);
  for (int i = 0; i < op.n_aux; ++i) {
    V3 w = normalize(fr.to_world(vmf_local(uni[2 * i], uni[2 * i + 1], op.kappa)));
    Hit h = closest_hit(s, o, w, INFINITY, false);
    if (h.prim < 0) {
      if (op.miss > 0)
        ws.hits.push_back({w, INFINITY, op.miss / (Cq * std::exp(op.kappa * (dot(u, w) - 1.0))), -1, V3(), 1.0, -1});
      continue;
    }
    double q = Cq * std::exp(op.kappa * (dot(u, w) - 1.0));
    V3 n = geo_normal(s, h.prim);
    ws.hits.push_back({w, h.t, 1.0 / q, s.tri_shape[h.prim], n, dot(n, w) * h.t, h.prim});
  }
  // depth weights relative to the ray's own hit distance t0: g = (t0 / t)^m, so
  // a closer surface dominates a farther one near its silhouette; if the ray
  // itself escapes, every hit has g = 1
  Hit h0 = closest_hit(s, o, u, INFINITY, false);
  if (h0.prim >= 0)
    for (AuxHit& h : ws.hits)
      if (h.shape >= 0) h.g_over_q *= std::pow(h0.t / std::max(h.t, 1e-3 * h0.t), op.power);
  return ws;
}

// Parameters: one translation per shape (param = 3 shape + axis) or every triangle
// corner's position (param = 9 triangle + 3 corner + axis).  A surface point moves
// with its barycentric coordinates: by tau[shape] or by sum_j b_j v'_j.
struct Param {
  bool vertex;
  int index, corner, axis;  // shape or triangle; corner (vertex mode); axis
};
Param param_of(bool vertex, int p) {
  return vertex ? Param{true, p / 9, (p / 3) % 3, p % 3} : Param{false, p / 3, 0, p % 3};
}
V3 axis_vec(int a, D2) { return a == 0 ? V3(1, 0, 0) : a == 1 ? V3(0, 1, 0) : V3(0, 0, 1); }

// The ray's origin: the camera (tri < 0) or a point of triangle `tri` with
// barycentric coordinates (1 - bu - bv, bu, bv) on shape `shape`.
struct Origin {
  int shape = -1, tri = -1;
  double bu = 0, bv = 0;
};

// Motion of the origin for the unit tangent of parameter P.
V3 origin_motion(const Origin& og, const Param& P) {
  if (og.tri < 0) return V3();
  V3 e = axis_vec(P.axis, D2{});
  if (!P.vertex) return og.shape == P.index ? e : V3();
  if (og.tri != P.index) return V3();
  const double b[3] = {1.0 - og.bu - og.bv, og.bu, og.bv};
  return e * b[P.corner];
}

// Barycentric coordinate `corner` of the point x(w) = o + t(w) w where the ray meets
// the plane of triangle t (extended beyond its edges), divided by t(w).  From the
// definition with signed areas, b1 = ((x - v0) x e2).c / c.c = (x - v0).a1 and b2 =
// (e1 x (x - v0)).c / c.c = (x - v0).a2 with a1 = (e2 x c) / c.c, a2 = (c x e1) / c.c,
// b0 = 1 - b1 - b2; dividing by t(w), with 1 / t(w) = (w.c) / (c.(v0 - o)), gives
// b_j / t = (o - v0).a_j / t + w.a_j, finite also where w runs parallel to the plane
// (where b_j and t are not).
D2 plane_barycentric_over_t(const Scene& s, int t, V3 o, VD w, int corner) {
  V3 v0 = s.v0[t], e1 = s.v1[t] - s.v0[t], e2 = s.v2[t] - s.v0[t];
  V3 c = cross(e1, e2);
  D2 inv_t = dotd(w, c) * (1.0 / dot(c, v0 - o));
  V3 a1 = cross(e2, c) * (1.0 / dot(c, c)), a2 = cross(c, e1) * (1.0 / dot(c, c));
  D2 b1 = inv_t * dot(o - v0, a1) + dotd(w, a1);
  D2 b2 = inv_t * dot(o - v0, a2) + dotd(w, a2);
  if (corner == 1) return b1;
  if (corner == 2) return b2;
  return inv_t - b1 - b2;
}

// Velocity, seen along w, of the point where w meets the plane of auxiliary hit h
// (distance d_h / (n_h . w)), relative to the origin, for the unit tangent of P.
VD aux_velocity(const Scene& s, const AuxHit& h, V3 o, const Origin& og, const Param& P, VD w) {
  if (h.tri < 0) return constant(V3());
  V3 e = axis_vec(P.axis, D2{});
  D2 inv_t = dotd(w, h.n) * (1.0 / h.d);
  D2 mt{0, 0, 0};  // motion of the plane point along e, divided by its distance t(w)
  if (!P.vertex) {
    if (h.shape == P.index) mt = inv_t;
  } else if (h.tri == P.index) {
    mt = plane_barycentric_over_t(s, h.tri, o, w, P.corner);
  }
  V3 om = origin_motion(og, P);
  VD rel{mt * e.x - inv_t * om.x, mt * e.y - inv_t * om.y, mt * e.z - inv_t * om.z};  // relative motion / t(w)
  D2 wr = dotd(w, rel);
  return VD{rel.x - w.x * wr, rel.y - w.y * wr, rel.z - w.z * wr};
}

// The warp field of parameter P at direction w (fixed samples; `skip` >= 0 leaves
// that sample out, -2 leaves out an escaped sample that carries no weight).
VD warp_field(const Scene& s, const WarpSamples& ws, V3 o, const Origin& og, const Param& P, VD w, int skip = -1) {
  VD num = constant(V3());
  D2 den{0, 0, 0};
  int idx = -1;
  for (const AuxHit& h : ws.hits) {
    if (++idx == skip) continue;
    D2 a = d2exp((dotd(w, h.w) - D2{1.0, 0, 0}) * (ws.kappa * ws.kscale)) * h.g_over_q;
    VD pc = aux_velocity(s, h, o, og, P, w);
    num = num + VD{pc.x * a, pc.y * a, pc.z * a};
    den = den + a;
  }
  const double inv_n = 1.0 / (skip != -1 ? ws.n - 1 : ws.n);
  D2 d = den * inv_n + D2{ws.eps * ws.K, 0, 0};
  return divided(VD{num.x * inv_n, num.y * inv_n, num.z * inv_n}, d);
}

// Derivative of log|n . u| for the unit tangent of P, n the unit geometric normal of
// the origin's triangle (vertex mode only; a translation does not turn a normal).
double normal_derivative(const Scene& s, const Origin& og, const Param& P, V3 u) {
  if (!P.vertex || og.tri < 0 || og.tri != P.index) return 0.0;
  V3 e = axis_vec(P.axis, D2{});
  VD v[3] = {constant(s.v0[og.tri]), constant(s.v1[og.tri]), constant(s.v2[og.tri])};
  v[P.corner] = VD{D2{v[P.corner].x.v, e.x, 0}, D2{v[P.corner].y.v, e.y, 0}, D2{v[P.corner].z.v, e.z, 0}};
  VD e1{v[1].x - v[0].x, v[1].y - v[0].y, v[1].z - v[0].z}, e2{v[2].x - v[0].x, v[2].y - v[0].y, v[2].z - v[0].z};
  VD c{e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x};
  D2 nu = dotd(c, u) / d2sqrt(dotd(c, c));
  return nu.a / nu.v;
}

// Window of the camera-ray warp (border > 0): 1 inside the image, falling to 0 at
// its border over `border` pixels (smoothstep of the distance in pixels to the
// nearest image edge), so that no sample is moved across the border of the image;
// border = 0: no window (samples near the border move across it, and the
// pixel-edge term on the image-border edges accounts for the flux).
struct CamWindow {
  V3 fwd, right, up;
  double tan_half = 1, aspect = 1, border = 4;
  int w = 1, h = 1;
};
D2 window(const CamWindow& c, VD w) {
  if (c.border <= 0.0) return D2{1, 0, 0};
  D2 fw = dotd(w, c.fwd);
  D2 sx = dotd(w, c.right) / fw * (1.0 / (c.tan_half * c.aspect));
  D2 sy = dotd(w, c.up) / fw * (1.0 / c.tan_half);
  D2 px = (sx + D2{1, 0, 0}) * (0.5 * c.w), py = (D2{1, 0, 0} - sy) * (0.5 * c.h);
  D2 d = px;
  for (D2 x : {D2{c.w - px.v, -px.a, -px.b}, py, D2{c.h - py.v, -py.a, -py.b}})
    if (x.v < d.v) d = x;
  D2 t = d * (1.0 / c.border);
  if (t.v >= 1.0) return D2{1, 0, 0};
  if (t.v <= 0.0) return D2{0, 0, 0};
  return t * t * (D2{3, 0, 0} - t * 2.0);
}

// Log-derivative factor of one reparameterized ray for every parameter that can
// move it: d/dtheta log(integrand * det) = m.(P_u V) + div V (+ the derivative of
// the cosine's normal, (n' . u) / (n . u), when m is a cosine covector n / n.u and
// the vertices move).  `out` gets (param, value).
struct LogDeriv {
  double l;   // m . (tangential V) + div V
  V3 wdot;    // tangential V: how the ray direction turns
};
void warp_log_derivs(const Scene& s, const WarpSamples& ws, V3 o, const Origin& og, bool vertex, V3 m, V3 n_cos,
                     std::vector<std::pair<int, double>>& out, const CamWindow* win = nullptr,
                     std::vector<std::pair<int, V3>>* wdot_out = nullptr) {
  out.clear();
  if (wdot_out) wdot_out->clear();
  // the parameters that can move this ray: those of the hit shapes / triangles and the origin
  std::vector<int> ids;
  auto add = [&](int id) {
    if (id >= 0 && std::find(ids.begin(), ids.end(), id) == ids.end()) ids.push_back(id);
  };
  bool moving_hit = false;
  for (const AuxHit& h : ws.hits) {
    if (h.tri < 0) continue;
    if (vertex) {
      add(h.tri);
      moving_hit = true;
    } else if (h.shape != og.shape) {
      add(h.shape);
      moving_hit = true;
    }
  }
  if (og.tri >= 0 && (moving_hit || vertex)) add(vertex ? og.tri : og.shape);
  const V3 u = ws.u;
  const int per = vertex ? 9 : 3;
  for (int id : ids)
    for (int k = 0; k < per; ++k) {
      const int p = per * id + k;
      const Param P = param_of(vertex, p);
      auto ld = [&](int skip) {
        auto field = [&](VD w) {
          VD V = warp_field(s, ws, o, og, P, w, skip);
          if (!win) return V;
          D2 b = window(*win, w);
          return VD{V.x * b, V.y * b, V.z * b};
        };
        double div = sphere_div(u, field);
        VD V = field(constant(u));
        V3 v(V.x.v, V.y.v, V.z.v);
        V3 wdot = v - u * dot(u, v);
        return LogDeriv{dot(m, wdot) + div, wdot};
      };
      LogDeriv fv = ld(-1);
      double full = fv.l;
      V3 wd = fv.wdot;
      if (ws.jackknife && ws.n > 1) {
        // leave-one-out over all N samples (misses without weight contribute the full value)
        double loo = 0.0;
        V3 wloo;
        int nh = (int)ws.hits.size();
        for (int j = 0; j < nh; ++j) {
          LogDeriv r = ld(j);
          loo += r.l;
          wloo = wloo + r.wdot;
        }
        LogDeriv r2 = ld(-2);
        loo += (ws.n - nh) * r2.l;
        wloo = wloo + r2.wdot * (double)(ws.n - nh);
        full = ws.n * full - (ws.n - 1.0) / ws.n * loo;
        wd = wd * (double)ws.n - wloo * ((ws.n - 1.0) / ws.n);
      }
      if (dot(n_cos, n_cos) > 0) full += normal_derivative(s, og, P, u);
      out.push_back({p, full});
      if (wdot_out) wdot_out->push_back({p, wd});
    }
}

// BSDF value with a direction in dual numbers (local frame, normal +z): diffuse,
// GGX conductor and blend, the same formulas as bsdf_eval_t.
void bsdf_value_dirs(const Mat& m, VD wi, VD wo, D2 out[3]) {
  for (int c = 0; c < 3; ++c) out[c] = D2{};
  if (m.bsdf == BSDF_DIFFUSE || m.bsdf == BSDF_BLEND) {
    const double w = m.bsdf == BSDF_DIFFUSE ? 1.0 : m.wd;
    for (int c = 0; c < 3; ++c) out[c] = D2{m.albedo[c] * w / kPi, 0, 0};
  }
  if (m.bsdf == BSDF_CONDUCTOR || m.bsdf == BSDF_BLEND) {
    VD sv{wi.x + wo.x, wi.y + wo.y, wi.z + wo.z};
    VD h = divided(sv, d2sqrt(dotd(sv, sv)));
    const double a2 = m.alpha * m.alpha;
    D2 den = h.z * h.z * (a2 - 1.0) + D2{1, 0, 0};
    D2 D = D2{a2 / kPi, 0, 0} / (den * den);
    auto G1 = [&](D2 c) {
      D2 tan2 = (D2{1, 0, 0} - c * c) / (c * c);
      return D2{2, 0, 0} / (D2{1, 0, 0} + d2sqrt(D2{1, 0, 0} + tan2 * a2));
    };
    D2 G = G1(wi.z) * G1(wo.z);
    D2 cd = dotd(wi, h);
    D2 mcd = D2{1, 0, 0} - cd;
    D2 m5 = mcd * mcd * mcd * mcd * mcd;
    const double w = m.bsdf == BSDF_CONDUCTOR ? 1.0 : 1.0 - m.wd;
    for (int c = 0; c < 3; ++c) {
      D2 F = D2{m.f0[c], 0, 0} + m5 * (1.0 - m.f0[c]);
      out[c] = out[c] + D * G * F / (wi.z * wo.z * 4.0) * w;
    }
  }
}

// Gradient (tangential, local frame) of log f_c with respect to the outgoing
// (wrt_out) or incident direction, by chart duals around that direction.
void bsdf_log_grad(const Mat& m, V3 wi, V3 wo, bool wrt_out, V3 g[3]) {
  V3 d = wrt_out ? wo : wi;
  Frame fr = make_frame(d);
  VD dr{D2{d.x, fr.s.x, fr.t.x}, D2{d.y, fr.s.y, fr.t.y}, D2{d.z, fr.s.z, fr.t.z}};
  VD dd = divided(dr, d2sqrt(dotd(dr, dr)));
  D2 f[3];
  bsdf_value_dirs(m, wrt_out ? constant(wi) : dd, wrt_out ? dd : constant(wo), f);
  for (int c = 0; c < 3; ++c)
    g[c] = f[c].v > 0 ? fr.s * (f[c].a / f[c].v) + fr.t * (f[c].b / f[c].v) : V3();
}

// Derivative of log f_c (per channel) at a glossy vertex with respect to the 9
// coordinates of its triangle's corners v0, v1, v2 (index 3 corner + axis), through
// the unit normal they define (oriented like n): the Duff et al. 2017 frame of the
// normal in dual numbers gives the local directions of the fixed world directions
// wi, wo, and f is evaluated on them (vertex mode: a non-rigid motion turns n).
void bsdf_normal_log_derivs(V3 v0, V3 v1, V3 v2, V3 n, const Mat& m, V3 wi, V3 wo, V3 out[9]) {
  for (int p = 0; p < 9; ++p) {
    out[p] = V3();
    if (m.bsdf == BSDF_DIFFUSE) continue;
    const int k = p / 3;
    const V3 e = axis_vec(p % 3, D2{});
    VD v[3] = {constant(v0), constant(v1), constant(v2)};
    v[k] = VD{D2{v[k].x.v, e.x, 0}, D2{v[k].y.v, e.y, 0}, D2{v[k].z.v, e.z, 0}};
    VD e1{v[1].x - v[0].x, v[1].y - v[0].y, v[1].z - v[0].z}, e2{v[2].x - v[0].x, v[2].y - v[0].y, v[2].z - v[0].z};
    VD c{e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x};
    const double orient = dot(V3(c.x.v, c.y.v, c.z.v), n) < 0.0 ? -1.0 : 1.0;
    VD nn = divided(c, d2sqrt(dotd(c, c)) * orient);
    const double sg = nn.z.v >= 0.0 ? 1.0 : -1.0;
    const D2 a = D2{-1, 0, 0} / (nn.z + D2{sg, 0, 0});
    const D2 b = nn.x * nn.y * a;
    VD fs{D2{1, 0, 0} + nn.x * nn.x * a * sg, b * sg, nn.x * (-sg)};
    VD ft{b, D2{sg, 0, 0} + nn.y * nn.y * a, nn.y * -1.0};
    VD wil{dotd(fs, wi), dotd(ft, wi), dotd(nn, wi)}, wol{dotd(fs, wo), dotd(ft, wo), dotd(nn, wo)};
    D2 f[3];
    bsdf_value_dirs(m, wil, wol, f);
    for (int ch = 0; ch < 3; ++ch) out[p][ch] = f[ch].v > 0 ? f[ch].a / f[ch].v : 0.0;
  }
}

bool reparameterized(int bsdf) { return bsdf == BSDF_DIFFUSE || bsdf == BSDF_CONDUCTOR || bsdf == BSDF_BLEND; }

// Forward-mode accumulator of the translation derivatives (all shapes at once).
struct ReparamAcc {
  const Scene* s = nullptr;
  const ReparamOpts* op = nullptr;
  uint64_t seed = 0;
  int np = 0;
  Pcg32 aux;
  std::vector<double> block;  // 4N uniforms of the current vertex: light ray, then BSDF ray
  V3 beta;
  std::vector<V3> bdot, ldot;
  using Sparse = std::vector<std::pair<int, double>>;
  using SparseV = std::vector<std::pair<int, V3>>;
  Sparse lnee, lbsdf, tmp;
  SparseV wnee, wbsdf, wprev;  // tangential direction change of the light ray, the BSDF ray, the previous ray
  V3 nee_n, bsdf_n;            // world normal of the vertex the rays leave
  int nee_tri = -1, bsdf_tri = -1;  // and its triangle
  CamWindow win;
  bool vertex = false;
  void init(const Scene* sc, const ReparamOpts* o, uint64_t sd, const Camera& cam, bool vert) {
    vertex = vert;
    win.fwd = cam.fwd;
    win.right = cam.right;
    win.up = cam.up;
    win.tan_half = cam.tan_half;
    win.aspect = cam.aspect;
    win.w = cam.w;
    win.h = cam.h;
    win.border = o->border;
    s = sc;
    op = o;
    seed = sd;
    np = vert ? 9 * sc->n_tris : 3 * (int)sc->shapes.size();
    bdot.assign(np, V3());
    ldot.assign(np, V3());
    block.assign(4 * o->n_aux, 0.0);
  }
  void camera_ray(uint64_t stream, V3 o, V3 d, V3 fwd) {
    aux.seed(seed, stream | (1ull << 62));
    std::vector<double> uni(2 * op->n_aux);
    for (double& x : uni) x = aux.uniform();
    WarpSamples ws = warp_samples(*s, *op, o, d, uni.data());
    warp_log_derivs(*s, ws, o, Origin{}, vertex, fwd * (-3.0 / dot(fwd, d)), V3(), tmp, &win, &wprev);
    beta = V3(1, 1, 1);
    for (auto& pv : tmp) bdot[pv.first] = V3(1, 1, 1) * pv.second;
  }
  void vertex_block() {
    for (double& x : block) x = aux.uniform();
  }
  void ray(V3 o, V3 d, int tri, double bu, double bv, V3 n, int bsdf, const double* uni, Sparse& out, SparseV& wout) {
    out.clear();
    wout.clear();
    if (!reparameterized(bsdf)) return;
    WarpSamples ws = warp_samples(*s, *op, o, d, uni);
    Origin og{s->tri_shape[tri], tri, bu, bv};
    warp_log_derivs(*s, ws, o, og, vertex, n * (1.0 / dot(n, d)), n, out, nullptr, &wout);
  }
  void nee_ray(V3 o, V3 d, int tri, double bu, double bv, V3 n, int bsdf) {
    nee_n = n;
    nee_tri = tri;
    ray(o, d, tri, bu, bv, n, bsdf, block.data(), lnee, wnee);
  }
  void bsdf_ray(V3 o, V3 d, int tri, double bu, double bv, V3 n, int bsdf) {
    bsdf_n = n;
    bsdf_tri = tri;
    ray(o, d, tri, bu, bv, n, bsdf, block.data() + 2 * op->n_aux, lbsdf, wbsdf);
  }
  // Per-channel log-derivative of one term of vertex `vi` (on triangle tri) leaving
  // along wl (local): the ray's warp terms, plus the BSDF's dependence on the
  // outgoing direction (turned by this ray's warp), on the incident one (turned by
  // the previous ray's warp; it points back along that ray) and, with vertex
  // positions as parameters, on the triangle's turning normal.
  std::vector<std::pair<int, V3>> term(const VertexInfo& vi, V3 wl, V3 n, int tri, const Sparse& l,
                                       const SparseV& w) {
    std::vector<std::pair<int, V3>> out;
    for (auto& pv : l) out.push_back({pv.first, V3(1, 1, 1) * pv.second});
    if (vi.m.bsdf == BSDF_DIFFUSE) return out;
    Frame fr = make_frame(n);
    V3 go[3], gi[3];
    bsdf_log_grad(vi.m, vi.wi, wl, true, go);
    bsdf_log_grad(vi.m, vi.wi, wl, false, gi);
    V3 gow[3], giw[3];
    for (int c = 0; c < 3; ++c) {
      gow[c] = fr.to_world(go[c]);
      giw[c] = fr.to_world(gi[c]);
    }
    auto add = [&](int p, V3 v) {
      for (auto& q : out)
        if (q.first == p) {
          q.second = q.second + v;
          return;
        }
      out.push_back({p, v});
    };
    for (auto& pw : w) add(pw.first, V3(dot(gow[0], pw.second), dot(gow[1], pw.second), dot(gow[2], pw.second)));
    for (auto& pw : wprev) {
      V3 di = -pw.second;  // the incident direction points back along the previous ray
      add(pw.first, V3(dot(giw[0], di), dot(giw[1], di), dot(giw[2], di)));
    }
    if (vertex && tri >= 0) {
      V3 nd[9];
      bsdf_normal_log_derivs(s->v0[tri], s->v1[tri], s->v2[tri], n, vi.m, fr.to_world(vi.wi), fr.to_world(wl), nd);
      for (int q = 0; q < 9; ++q) add(9 * tri + q, nd[q]);
    }
    return out;
  }
  void emission(V3, V3 le_w, int, V3, double) {
    for (int p = 0; p < np; ++p) ldot[p] = ldot[p] + mul(bdot[p], le_w);
  }
  void nee(const VertexInfo& vi, V3 wl, V3 scale, V3 c, int, V3, double) {
    V3 f = bsdf_eval(vi.m, vi.wi, wl);
    for (int p = 0; p < np; ++p) ldot[p] = ldot[p] + mul(mul(bdot[p], f), scale);
    for (auto& pv : term(vi, wl, nee_n, nee_tri, lnee, wnee)) ldot[pv.first] = ldot[pv.first] + mul(c, pv.second);
  }
  void scatter(const VertexInfo& vi, V3 wo, double k) {
    V3 f = bsdf_eval(vi.m, vi.wi, wo);
    V3 nb = mul(beta, f) * k;
    for (int p = 0; p < np; ++p) bdot[p] = mul(bdot[p], f) * k;
    for (auto& pv : term(vi, wo, bsdf_n, bsdf_tri, lbsdf, wbsdf)) bdot[pv.first] = bdot[pv.first] + mul(nb, pv.second);
    beta = nb;
    wprev = wbsdf;
  }
  void scatter_delta(double w) {
    beta = beta * w;
    for (auto& b : bdot) b = b * w;
    wprev.clear();  // a delta lobe's outgoing ray is not reparameterized
  }
  void roulette(double q) {
    beta = beta * (1.0 / q);
    for (auto& b : bdot) b = b * (1.0 / q);
  }
};

// ---------------------------------------------------------------- parallel driver
// A path through a pixel edge: only its camera ray's warp is needed (the radiance
// it carries enters the edge term as a value, not differentiated).  The warp is
// the camera-ray warp of ReparamAcc (windowed or not), from the same auxiliary
// stream rule.
struct EdgeAcc : NullAcc {
  const Scene* s = nullptr;
  const ReparamOpts* op = nullptr;
  uint64_t seed = 0;
  CamWindow win;
  bool vertex = false;
  V3 u;
  std::vector<std::pair<int, double>> tmp;
  std::vector<std::pair<int, V3>> wdot;  // per parameter: the tangential turn of the camera ray
  void camera_ray(uint64_t stream, V3 o, V3 d, V3) {
    Pcg32 aux;
    aux.seed(seed, stream | (1ull << 62));
    std::vector<double> uni(2 * op->n_aux);
    for (double& x : uni) x = aux.uniform();
    WarpSamples ws = warp_samples(*s, *op, o, d, uni.data());
    u = d;
    warp_log_derivs(*s, ws, o, Origin{}, vertex, V3(), V3(), tmp, &win, &wdot);
  }
};

// Gradient of the image-plane pixel coordinate (px if `x`, else py) with respect
// to the ray direction w of a pinhole camera: px = (w.right / w.fwd / (tan_half *
// aspect) + 1) w / 2, py = (1 - w.up / w.fwd / tan_half) h / 2.
V3 pixel_coord_grad(const Camera& c, V3 w, bool x) {
  const double f = dot(w, c.fwd);
  if (x) return (c.right * (1.0 / f) - c.fwd * (dot(w, c.right) / (f * f))) * (0.5 * c.w / (c.tan_half * c.aspect));
  return (c.up * (1.0 / f) - c.fwd * (dot(w, c.up) / (f * f))) * (-0.5 * c.h / c.tan_half);
}

template <class F>
void parallel_rows(int y0, int rows, int n_threads, F fn) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  std::atomic<int> next(0);
  std::vector<std::thread> ts;
  for (int i = 0; i < n_threads; ++i)
    ts.emplace_back([&]() {
      for (;;) {
        int r = next.fetch_add(1);
        if (r >= rows) break;
        fn(y0 + r);
      }
    });
  for (auto& t : ts) t.join();
}

CacheModel make_cache(const double* W, const double* box, int bounce) {
  CacheModel c;
  c.W = W;
  if (box) std::memcpy(c.box, box, sizeof c.box);
  c.bounce = bounce;
  return c;
}

void crop_of(const oracle_render_in& r, int& x0, int& y0, int& cw, int& ch) {
  x0 = r.crop_w > 0 ? r.crop_x0 : 0;
  y0 = r.crop_w > 0 ? r.crop_y0 : 0;
  cw = r.crop_w > 0 ? r.crop_w : r.width;
  ch = r.crop_w > 0 ? r.crop_h : r.height;
}

}  // namespace

extern "C" {

// Copy the scene into FP64, build the oracle's BVH, the area-light CDF and the
// environment-map distribution (luminance x sin(theta), marginal/conditional).
void* oracle_scene_new(const oracle_scene_in* in) {
  Scene* s = new Scene();
  s->n_tris = in->n_tris;
  for (int t = 0; t < in->n_tris; ++t) {
    const float* v = in->vertices + (size_t)t * 9;
    s->v0.emplace_back(v[0], v[1], v[2]);
    s->v1.emplace_back(v[3], v[4], v[5]);
    s->v2.emplace_back(v[6], v[7], v[8]);
    for (int k = 0; k < 6; ++k) s->uv.push_back(in->uvs ? in->uvs[(size_t)t * 6 + k] : 0.0);
    s->tri_shape.push_back(in->tri_shape[t]);
  }
  for (int i = 0; i < in->n_shapes; ++i) {
    Shape sh;
    sh.bsdf = in->bsdf[i];
    sh.tex = in->tex[i];
    sh.albedo_index = in->albedo_index[i];
    sh.rough_index = in->rough_index[i];
    sh.alpha = in->alpha[i];
    sh.eta = in->eta[i];
    sh.diffuse_weight = in->diffuse_weight[i];
    sh.f0 = V3(in->f0[i * 3], in->f0[i * 3 + 1], in->f0[i * 3 + 2]);
    sh.emission = V3(in->emission[i * 3], in->emission[i * 3 + 1], in->emission[i * 3 + 2]);
    sh.emitter = max3(sh.emission) > 0.0;
    s->shapes.push_back(sh);
  }
  s->albedo.assign(in->albedo, in->albedo + (size_t)in->n_albedo * 3);
  for (int i = 0; i < in->n_tex; ++i) {
    Texture t;
    t.w = in->tex_w[i];
    t.h = in->tex_h[i];
    t.rgba.assign(in->tex_data[i], in->tex_data[i] + (size_t)t.w * t.h * 4);
    s->tex.push_back(std::move(t));
  }
  s->roughness.assign(in->roughness, in->roughness + in->n_rough);
  // area lights: every triangle of an emitting shape, picked proportionally to area
  s->light_cdf.push_back(0.0);
  for (int t = 0; t < s->n_tris; ++t) {
    if (!s->shapes[s->tri_shape[t]].emitter) continue;
    double a = 0.5 * length(cross(s->v1[t] - s->v0[t], s->v2[t] - s->v0[t]));
    s->light_tris.push_back(t);
    s->light_cdf.push_back(s->light_cdf.back() + a);
  }
  s->light_area = s->light_cdf.back();
  for (auto& c : s->light_cdf) c = s->light_area > 0 ? c / s->light_area : 0.0;
  // environment map
  if (in->env && in->env_w > 0) {
    s->env_w = in->env_w;
    s->env_h = in->env_h;
    size_t n = (size_t)s->env_w * s->env_h;
    s->env.assign(in->env, in->env + n * 4);
    std::vector<double> w(n);
    double total = 0.0;
    s->env_marg.assign(s->env_h + 1, 0.0);
    s->env_cond.assign((size_t)s->env_h * (s->env_w + 1), 0.0);
    for (int y = 0; y < s->env_h; ++y) {
      double st = std::sin(kPi * (y + 0.5) / s->env_h);
      double row = 0.0;
      double* cond = &s->env_cond[(size_t)y * (s->env_w + 1)];
      for (int x = 0; x < s->env_w; ++x) {
        const double* e = &s->env[((size_t)y * s->env_w + x) * 4];
        double lum = 0.2126 * e[0] + 0.7152 * e[1] + 0.0722 * e[2];
        w[(size_t)y * s->env_w + x] = lum * st;
        row += lum * st;
        cond[x + 1] = row;
      }
      for (int x = 0; x <= s->env_w; ++x) cond[x] = row > 0 ? cond[x] / row : 0.0;
      s->env_marg[y + 1] = s->env_marg[y] + row;
      total += row;
    }
    for (auto& m : s->env_marg) m /= total;
    s->env_p.resize(n);
    for (size_t i = 0; i < n; ++i) s->env_p[i] = w[i] / total;
  }
  // BVH
  s->order.resize(s->n_tris);
  for (int t = 0; t < s->n_tris; ++t) s->order[t] = t;
  if (s->n_tris > 0) build_node(*s, 0, s->n_tris);
  return s;
}

void oracle_scene_free(void* sc) { delete (Scene*)sc; }

// Mean over `spp` samples per pixel of the crop -> image [ch][cw][3].
// Optional per-sample radiance [ch][cw][spp][3] and decision hashes [ch][cw][spp].
int oracle_render(void* sc, const oracle_render_in* r, double* image, double* sample_L,
                  uint32_t* sample_hash, int n_threads, uint64_t* n_rays) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  std::atomic<uint64_t> rays(0);
  parallel_rows(y0, ch, n_threads, [&](int py) {
    g_rays = 0;
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      V3 sum(0, 0, 0);
      for (int k = 0; k < r->spp; ++k) {
        NullAcc acc;
        uint32_t h;
        V3 L = render_sample(s, cam, *r, px, py, k, acc, &h);
        sum = sum + L;
        size_t si = pi * r->spp + k;
        if (sample_L)
          for (int c = 0; c < 3; ++c) sample_L[si * 3 + c] = L[c];
        if (sample_hash) sample_hash[si] = h;
      }
      for (int c = 0; c < 3; ++c) image[pi * 3 + c] = sum[c] / r->spp;
    }
    rays += g_rays;
  });
  if (n_rays) *n_rays = rays.load();
  return 0;
}

// Gradient of sum(grad_image * image) by reverse mode over a stored per-path tape.
// grad_image [ch][cw][3] is dLoss/dImage; each sample gets 1/spp of it.
// Outputs are *overwritten*: g_albedo [A][3], g_tex[i] [h][w][4], g_rough [R] (any may be NULL).
int oracle_grad_tape(void* sc, const oracle_render_in* r, const double* grad_image, double* g_albedo,
                     double* const* g_tex, double* g_rough, double* g_env, int n_threads, uint64_t* n_rays) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  GradOut total;
  total.albedo.assign(s.albedo.size(), 0.0);
  for (auto& t : s.tex) total.tex.emplace_back(t.rgba.size(), 0.0);
  total.rough.assign(s.roughness.size(), 0.0);
  total.env.assign((size_t)s.env_w * s.env_h * 4, 0.0);
  std::mutex mu;
  std::atomic<uint64_t> rays(0);
  parallel_rows(y0, ch, n_threads, [&](int py) {
    g_rays = 0;
    // one row's contributions, merged under the lock (texture buffers are shared)
    GradOut row;
    row.albedo.assign(s.albedo.size(), 0.0);
    row.rough.assign(s.roughness.size(), 0.0);
    struct TexAdd { int tex; size_t idx; double v; };
    std::vector<TexAdd> tex_adds;  // tex = -1: environment pixel
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      V3 dl(grad_image[pi * 3] / r->spp, grad_image[pi * 3 + 1] / r->spp, grad_image[pi * 3 + 2] / r->spp);
      for (int k = 0; k < r->spp; ++k) {
        TapeAcc tape;
        render_sample(s, cam, *r, px, py, k, tape, nullptr);
        // reverse sweep: suffix sums of the recorded contributions give the
        // radiance that flows through each sampled BSDF value (no subtraction);
        // texel gradients go through a sparse list to keep per-row memory small
        V3 suffix(0, 0, 0);
        for (int i = (int)tape.recs.size() - 1; i >= 0; --i) {
          const auto& rc = tape.recs[i];
          // environment radiance: the contribution is linear in it (local term)
          if (rc.env_texel >= 0)
            for (int c = 0; c < 3; ++c) tex_adds.push_back({-1, (size_t)rc.env_texel * 4 + c, dl[c] * rc.d_env[c]});
          if (rc.kind == 0) {
            suffix = suffix + rc.c;
            continue;
          }
          V3 contrib = rc.kind == 1 ? rc.c : suffix;
          DFactors df = bsdf_dfactors(rc.m, rc.wi, rc.wo);
          if (rc.m.alb_kind == 2) {
            for (int c = 0; c < 3; ++c)
              tex_adds.push_back({rc.m.tex_id, (size_t)rc.m.texel * 4 + c, dl[c] * contrib[c] * df.d_alb[c]});
            Mat m2 = rc.m;
            m2.alb_kind = 0;
            add_param_grad(row, m2, contrib, df, dl);
          } else {
            add_param_grad(row, rc.m, contrib, df, dl);
          }
          if (rc.kind == 1) suffix = suffix + rc.c;
        }
      }
    }
    rays += g_rays;
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < row.albedo.size(); ++i) total.albedo[i] += row.albedo[i];
    for (size_t i = 0; i < row.rough.size(); ++i) total.rough[i] += row.rough[i];
    for (const auto& a : tex_adds) (a.tex < 0 ? total.env : total.tex[a.tex])[a.idx] += a.v;
  });
  if (n_rays) *n_rays = rays.load();
  if (g_albedo) std::memcpy(g_albedo, total.albedo.data(), total.albedo.size() * sizeof(double));
  if (g_rough) std::memcpy(g_rough, total.rough.data(), total.rough.size() * sizeof(double));
  if (g_env) std::memcpy(g_env, total.env.data(), total.env.size() * sizeof(double));
  if (g_tex)
    for (size_t i = 0; i < total.tex.size(); ++i)
      if (g_tex[i]) std::memcpy(g_tex[i], total.tex[i].data(), total.tex[i].size() * sizeof(double));
  return 0;
}

// Gradient of sum(grad_image * image) w.r.t. a list of selected parameters by
// forward-mode dual numbers.  sel: n_sel records of 4 ints (kind, a, b, c):
//   kind 0 = albedo row a channel b; 1 = texture a, texel b, channel c; 2 = roughness a.
int oracle_grad_dual(void* sc, const oracle_render_in* r, const double* grad_image, int n_sel,
                     const int* sel, double* out, int n_threads) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  std::vector<SelParam> params;
  for (int i = 0; i < n_sel; ++i) params.push_back({sel[i * 4], sel[i * 4 + 1], sel[i * 4 + 2], sel[i * 4 + 3]});
  std::vector<double> total(n_sel, 0.0);
  std::mutex mu;
  parallel_rows(y0, ch, n_threads, [&](int py) {
    std::vector<double> acc_row(n_sel, 0.0);
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      for (int k = 0; k < r->spp; ++k) {
        DualAcc acc;
        acc.init(&params);
        render_sample(s, cam, *r, px, py, k, acc, nullptr);
        for (int c = 0; c < 3; ++c) {
          double dl = grad_image[pi * 3 + c] / r->spp;
          for (int i = 0; i < n_sel; ++i) acc_row[i] += dl * tg(acc.L[c], i);
        }
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n_sel; ++i) total[i] += acc_row[i];
  });
  std::memcpy(out, total.data(), n_sel * sizeof(double));
  return 0;
}

// Forward-mode image derivative: image (as oracle_render) and image_dot =
// d image / d eps of the render at params + eps v.  t_tex: n_tex pointers
// (entries may be null), each [h][w][4] like the scene's textures; t_env:
// tangent of the environment radiance [env_h][env_w][4] or null.
int oracle_render_jvp(void* sc, const oracle_render_in* r, const double* t_albedo, const double* const* t_tex,
                      int n_tex, const double* t_rough, const double* t_env, double* image, double* image_dot,
                      int n_threads) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  Direction dir;
  dir.albedo = t_albedo;
  for (int i = 0; i < n_tex; ++i) dir.tex.push_back(t_tex ? t_tex[i] : nullptr);
  dir.rough = t_rough;
  dir.env = t_env;
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  parallel_rows(y0, ch, n_threads, [&](int py) {
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      double sum[3] = {0, 0, 0}, sum_dot[3] = {0, 0, 0};
      for (int k = 0; k < r->spp; ++k) {
        JvpAcc acc;
        acc.init(&dir);
        V3 l = render_sample(s, cam, *r, px, py, k, acc, nullptr);
        for (int c = 0; c < 3; ++c) {
          sum[c] += l[c];
          sum_dot[c] += tg(acc.L[c], 0);
        }
      }
      for (int c = 0; c < 3; ++c) {
        image[pi * 3 + c] = sum[c] / r->spp;
        image_dot[pi * 3 + c] = sum_dot[c] / r->spp;
      }
    }
  });
  return 0;
}

// Cache-terminated render (W: MLP weights [20672], box: lo[3], hi[3]).
int oracle_render_cached(void* sc, const oracle_render_in* r, const double* W, const double* box, int bounce,
                         double* image, int n_threads) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  CacheModel cm = make_cache(W, box, bounce);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  parallel_rows(y0, ch, n_threads, [&](int py) {
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      V3 sum(0, 0, 0);
      for (int k = 0; k < r->spp; ++k) {
        NullAcc acc;
        sum = sum + render_sample(s, cam, *r, px, py, k, acc, nullptr, &cm);
      }
      for (int c = 0; c < 3; ++c) image[pi * 3 + c] = sum[c] / r->spp;
    }
  });
  return 0;
}

// Albedo gradient (rows [A][3]) of the cache-terminated estimator by forward-mode
// duals; the cache radiance is a detached incident radiance.
int oracle_grad_dual_cached(void* sc, const oracle_render_in* r, const double* W, const double* box, int bounce,
                            const double* grad_image, int n_sel, const int* sel, double* out, int n_threads) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  CacheModel cm = make_cache(W, box, bounce);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  std::vector<SelParam> params;
  for (int i = 0; i < n_sel; ++i) params.push_back({sel[i * 4], sel[i * 4 + 1], sel[i * 4 + 2], sel[i * 4 + 3]});
  std::vector<double> total(n_sel, 0.0);
  std::mutex mu;
  parallel_rows(y0, ch, n_threads, [&](int py) {
    std::vector<double> acc_row(n_sel, 0.0);
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      for (int k = 0; k < r->spp; ++k) {
        DualAcc acc;
        acc.init(&params);
        render_sample(s, cam, *r, px, py, k, acc, nullptr, &cm);
        for (int c = 0; c < 3; ++c) {
          double dl = grad_image[pi * 3 + c] / r->spp;
          for (int i = 0; i < n_sel; ++i) acc_row[i] += dl * tg(acc.L[c], i);
        }
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n_sel; ++i) total[i] += acc_row[i];
  });
  std::memcpy(out, total.data(), n_sel * sizeof(double));
  return 0;
}

// Training records of full-length paths: per non-delta vertex below max_depth,
// raw features and the target (L_path - L_up_to_vertex) / beta.  Returns the
// number of records (<= cap); out_raw [cap][10], out_target [cap][3],
// out_meta [cap][2] = (sample index pixel*spp + s within the crop, depth).
int oracle_train_records(void* sc, const oracle_render_in* r, int cap, double* out_raw, double* out_target,
                         int* out_meta) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  int n = 0;
  for (int py = y0; py < y0 + ch; ++py)
    for (int px = x0; px < x0 + cw; ++px)
      for (int k = 0; k < r->spp; ++k) {
        NullAcc acc;
        std::vector<TrainRecord> recs;
        V3 L = render_sample(s, cam, *r, px, py, k, acc, nullptr, nullptr, &recs);
        long long slot = ((long long)(py - y0) * cw + (px - x0)) * r->spp + k;
        for (const auto& rc : recs) {
          if (n >= cap) return n;
          std::memcpy(out_raw + 10 * (size_t)n, rc.raw, sizeof rc.raw);
          for (int c = 0; c < 3; ++c)
            out_target[3 * (size_t)n + c] = rc.beta[c] > 1e-12 ? std::max(L[c] - rc.L_before[c], 0.0) / rc.beta[c] : 0.0;
          out_meta[2 * n] = (int)slot;
          out_meta[2 * n + 1] = rc.depth;
          ++n;
        }
      }
  return n;
}

static bool reparam_opts(const oracle_reparam_opts* o, ReparamOpts& op) {
  if (!o || o->n_aux < 2 || !(o->kappa > 0) || !(o->kernel_scale >= 1) || !(o->eps > 0) || !(o->miss >= 0))
    return false;
  op.n_aux = o->n_aux;
  op.kappa = o->kappa;
  op.kernel_scale = o->kernel_scale;
  op.power = o->power;
  op.miss = o->miss;
  op.eps = o->eps;
  op.jackknife = o->jackknife;
  op.border = o->border;
  op.edge_spp = o->edge_spp;
  return o->border >= 0 && o->edge_spp >= 0;
}

// Reverse-mode-equivalent gradient by forward mode: g[p] = sum over pixels and
// channels of grad_image * d image / d theta_p for every translation parameter
// (vertex = 0: p = 3 shape + axis, g [n_shapes][3]) or every triangle corner
// position (vertex = 1: p = 9 triangle + 3 corner + axis, g [n_tris][3][3]), by
// the reparameterized estimator above (every random number fixed, auxiliary ones
// from the stream initseq | 2^62).  Optionally the image and its derivative along
// parameter `dot_param`, or (dot_dir non-NULL, one weight per parameter) along the
// direction sum_p dot_dir[p] e_p.
int oracle_grad_reparam(void* sc, const oracle_render_in* r, const double* grad_image, const oracle_reparam_opts* o,
                        int vertex, double* g_out, double* image, int dot_param, double* image_dot, int n_threads,
                        const double* dot_dir) {
  const Scene& s = *(Scene*)sc;
  Camera cam = make_camera(*r);
  ReparamOpts op;
  if (!reparam_opts(o, op)) return -1;
  int x0, y0, cw, ch;
  crop_of(*r, x0, y0, cw, ch);
  const int np = vertex ? 9 * s.n_tris : 3 * (int)s.shapes.size();
  std::vector<double> rows((size_t)(ch + 1) * np, 0.0);
  // weight of parameter p in the image derivative
  auto dot_w = [&](int p) { return dot_dir ? dot_dir[p] : (p == dot_param ? 1.0 : 0.0); };
  const bool want_dot = image_dot && (dot_dir || (dot_param >= 0 && dot_param < np));
  // Pixel-edge term.  The warp that fixes the discontinuities also moves the
  // footprint of every pixel (a box of unit area in pixel coordinates): its
  // boundary moves with minus the warp's image-plane velocity, so pixel p gains
  // -integral over its boundary of L (v . n_out) ds.  An edge between pixels a
  // (left / above) and b (right / below) adds -L v_n to a and +L v_n to b, v_n
  // the velocity along +x (+y); one path through a uniform point of the edge
  // estimates the integral.  Every edge of every pixel of the crop: on the crop's
  // (or the image's) border only the inside pixel counts; with a border window the
  // image-border edges carry nothing (the warp vanishes there).
  std::vector<double> edge_dot((size_t)(ch + 1) * cw * 3, 0.0);  // horizontal edges: L v_n of dot_param
  if (image_dot) std::fill(image_dot, image_dot + (size_t)cw * ch * 3, 0.0);
  if (op.edge_spp > 0 && (grad_image || want_dot)) {
    const double* gimg = grad_image;
    parallel_rows(y0, ch + 1, n_threads, [&](int Y) {
      double* grow = &rows[(size_t)(Y - y0) * np];
      auto pixel_grad = [&](int X, int Yp) -> const double* {
        if (!gimg || X < x0 || X >= x0 + cw || Yp < y0 || Yp >= y0 + ch) return nullptr;
        return gimg + ((size_t)(Yp - y0) * cw + (X - x0)) * 3;
      };
      auto edge = [&](bool vertical, int X, int Yy, uint64_t id) {
        const double* ga = vertical ? pixel_grad(X - 1, Yy) : pixel_grad(X, Yy - 1);
        const double* gb = pixel_grad(X, Yy);
        V3 sum_dot;
        for (int k = 0; k < op.edge_spp; ++k) {
          EdgeStart e{((uint64_t)r->cam_index << 40) | (id << 12) | (uint64_t)k | (1ull << 61), vertical, X, Yy};
          EdgeAcc acc;
          acc.s = &s;
          acc.op = &op;
          acc.seed = r->seed;
          acc.vertex = vertex != 0;
          acc.win = CamWindow{cam.fwd, cam.right, cam.up, cam.tan_half, cam.aspect, op.border, cam.w, cam.h};
          V3 l = render_sample(s, cam, *r, 0, 0, k, acc, nullptr, nullptr, nullptr, &e);
          V3 gp = pixel_coord_grad(cam, acc.u, vertical);
          for (auto& pw : acc.wdot) {
            const double vn = dot(gp, pw.second) / op.edge_spp;
            double gl = 0.0;
            for (int c = 0; c < 3; ++c) gl += ((gb ? gb[c] : 0.0) - (ga ? ga[c] : 0.0)) * l[c];
            grow[pw.first] += gl * vn;
            sum_dot = sum_dot + l * (vn * dot_w(pw.first));
          }
        }
        return sum_dot;
      };
      const uint64_t nv = (uint64_t)(r->width + 1) * r->height;  // vertical edges first, then horizontal
      if (Y < y0 + ch)
        for (int X = x0; X <= x0 + cw; ++X) {
          V3 d = edge(true, X, Y, (uint64_t)Y * (r->width + 1) + X);
          if (!image_dot) continue;
          double* row = image_dot + (size_t)(Y - y0) * cw * 3;
          for (int c = 0; c < 3; ++c) {
            if (X - 1 >= x0) row[(X - 1 - x0) * 3 + c] -= d[c];
            if (X < x0 + cw) row[(X - x0) * 3 + c] += d[c];
          }
        }
      for (int X = x0; X < x0 + cw; ++X) {
        V3 d = edge(false, X, Y, nv + (uint64_t)Y * r->width + X);
        for (int c = 0; c < 3; ++c) edge_dot[((size_t)(Y - y0) * cw + (X - x0)) * 3 + c] = d[c];
      }
    });
    if (image_dot)
      for (int Y = y0; Y <= y0 + ch; ++Y)
        for (int X = x0; X < x0 + cw; ++X)
          for (int c = 0; c < 3; ++c) {
            const double d = edge_dot[((size_t)(Y - y0) * cw + (X - x0)) * 3 + c];
            if (Y - 1 >= y0) image_dot[((size_t)(Y - 1 - y0) * cw + (X - x0)) * 3 + c] -= d;
            if (Y < y0 + ch) image_dot[((size_t)(Y - y0) * cw + (X - x0)) * 3 + c] += d;
          }
  }
  parallel_rows(y0, ch, n_threads, [&](int py) {
    double* grow = &rows[(size_t)(py - y0) * np];
    for (int px = x0; px < x0 + cw; ++px) {
      size_t pi = (size_t)(py - y0) * cw + (px - x0);
      double sum[3] = {0, 0, 0}, sum_dot[3] = {0, 0, 0};
      const double* gi = grad_image ? grad_image + pi * 3 : nullptr;
      for (int k = 0; k < r->spp; ++k) {
        ReparamAcc acc;
        acc.init(&s, &op, r->seed, cam, vertex != 0);
        V3 l = render_sample(s, cam, *r, px, py, k, acc, nullptr);
        for (int c = 0; c < 3; ++c) sum[c] += l[c];
        if (want_dot)
          for (int p = 0; p < np; ++p) {
            const double wp = dot_w(p);
            if (wp != 0.0)
              for (int c = 0; c < 3; ++c) sum_dot[c] += wp * acc.ldot[p][c];
          }
        if (gi)
          for (int p = 0; p < np; ++p) grow[p] += (gi[0] * acc.ldot[p].x + gi[1] * acc.ldot[p].y +
                                                   gi[2] * acc.ldot[p].z) / r->spp;
      }
      for (int c = 0; c < 3; ++c) {
        if (image) image[pi * 3 + c] = sum[c] / r->spp;
        if (image_dot) image_dot[pi * 3 + c] += sum_dot[c] / r->spp;
      }
    }
  });
  if (g_out)
    for (int p = 0; p < np; ++p) {
      double t = 0.0;
      for (int y = 0; y <= ch; ++y) t += rows[(size_t)y * np + p];
      g_out[p] = t;
    }
  return 0;
}

// ---------------------------------------------------------------- unit-test hooks
void oracle_pcg32(uint64_t initstate, uint64_t initseq, int n, uint32_t* out) {
  Pcg32 r;
  r.seed(initstate, initseq);
  for (int i = 0; i < n; ++i) out[i] = r.next_u32();
}

// Closest hits for n rays (o,d: [n][3]); prim = -1 on a miss.
void oracle_trace(void* sc, int n, const double* o, const double* d, int brute, double* t_out, int* prim_out) {
  const Scene& s = *(Scene*)sc;
  for (int i = 0; i < n; ++i) {
    Hit h = closest_hit(s, V3(o[i * 3], o[i * 3 + 1], o[i * 3 + 2]), V3(d[i * 3], d[i * 3 + 1], d[i * 3 + 2]),
                        INFINITY, brute != 0);
    t_out[i] = h.prim >= 0 ? h.t : INFINITY;
    prim_out[i] = h.prim;
  }
}

// BSDF hooks in local space (normal +z).  params: albedo[3], alpha, f0[3], eta, wd.
static Mat hook_mat(int bsdf, const double* p) {
  Mat m{};
  m.bsdf = bsdf;
  m.albedo = V3(p[0], p[1], p[2]);
  m.alpha = p[3];
  m.f0 = V3(p[4], p[5], p[6]);
  m.eta = p[7];
  m.wd = p[8];
  m.rough = -1;
  return m;
}
void oracle_bsdf_eval(int bsdf, const double* params, const double* wi, const double* wo, double* f_out,
                      double* pdf_out) {
  Mat m = hook_mat(bsdf, params);
  V3 a(wi[0], wi[1], wi[2]), b(wo[0], wo[1], wo[2]);
  V3 f = bsdf_eval(m, a, b);
  for (int c = 0; c < 3; ++c) f_out[c] = f[c];
  *pdf_out = bsdf_pdf(m, a, b);
}
// d log f_c / d (corner k, axis a) at [3 (3 k + a) + c] through the normal of the
// triangle v (9 doubles), oriented like n; wi, wo world directions.
void oracle_bsdf_normal_dlog(int bsdf, const double* params, const double* v, const double* n, const double* wi,
                             const double* wo, double* out27) {
  Mat m = hook_mat(bsdf, params);
  V3 d[9];
  bsdf_normal_log_derivs(V3(v[0], v[1], v[2]), V3(v[3], v[4], v[5]), V3(v[6], v[7], v[8]), V3(n[0], n[1], n[2]), m,
                         V3(wi[0], wi[1], wi[2]), V3(wo[0], wo[1], wo[2]), d);
  for (int p = 0; p < 9; ++p)
    for (int c = 0; c < 3; ++c) out27[3 * p + c] = d[p][c];
}
// The dual-number classes on the paper's two toy programs (Fig. 1: x^n by repeated
// multiplication; Fig. 6: the exponential density a exp(-a x) with x detached):
// out = {x^n, d x^n / dx (Dual), a exp(-a x), d / da (D2)}.
void oracle_dual_toys(double x, int n, double a, double* out) {
  Dual dx(x, 1);
  dx.d[0] = 1.0;
  Dual y(1.0, 1);
  for (int i = 0; i < n; ++i) y = y * dx;
  out[0] = y.v;
  out[1] = y.d[0];
  D2 da{a, 1.0, 0.0};
  D2 e = da * d2exp(da * (-x));
  out[2] = e.v;
  out[3] = e.a;
}
// Returns 1 and wo if sampling succeeded (non-delta BSDFs).
int oracle_bsdf_sample(int bsdf, const double* params, const double* wi, double u3, double u4, double u5,
                       double* wo_out) {
  Mat m = hook_mat(bsdf, params);
  V3 a(wi[0], wi[1], wi[2]), wo;
  bool ok = true;
  if (bsdf == BSDF_DIFFUSE || (bsdf == BSDF_BLEND && u3 < m.wd)) {
    wo = cosine_sample(u4, u5);
  } else {
    ok = ggx_sample(m.alpha, a, u4, u5, wo);
  }
  wo_out[0] = wo.x;
  wo_out[1] = wo.y;
  wo_out[2] = wo.z;
  return ok ? 1 : 0;
}
// Analytic derivative factors: d_alb[3], d_alpha[3].
void oracle_bsdf_dfactors(int bsdf, const double* params, const double* wi, const double* wo, double* out6) {
  Mat m = hook_mat(bsdf, params);
  DFactors df = bsdf_dfactors(m, V3(wi[0], wi[1], wi[2]), V3(wo[0], wo[1], wo[2]));
  for (int c = 0; c < 3; ++c) {
    out6[c] = df.d_alb[c];
    out6[3 + c] = df.d_alpha[c];
  }
}
// The dielectric scattering event of the integrator: returns 1 on refraction,
// 0 on reflection; wo_out the outgoing direction, *weight_out the radiance factor.
int oracle_dielectric_sample(const double* ng, const double* wi, double eta, double u3, double* wo_out,
                             double* weight_out) {
  V3 wo;
  double w;
  bool refr = dielectric_scatter(V3(ng[0], ng[1], ng[2]), V3(wi[0], wi[1], wi[2]), eta, u3, wo, w);
  wo_out[0] = wo.x;
  wo_out[1] = wo.y;
  wo_out[2] = wo.z;
  *weight_out = w;
  return refr ? 1 : 0;
}
// The GGX terms of the conductor lobe: out2 = {D(cos_h), G1(cos_w)} (no sign tests).
void oracle_ggx_terms(double alpha, double cos_h, double cos_w, double* out2) {
  out2[0] = ggx_D<double>(alpha, cos_h);
  out2[1] = ggx_G1<double>(alpha, cos_w);
}
double oracle_fresnel(double cos_i, double eta) {
  double ct;
  return fresnel_dielectric(cos_i, eta, ct);
}
double oracle_env_pdf(void* sc, const double* d) { return env_pdf(*(Scene*)sc, V3(d[0], d[1], d[2])); }
int oracle_frame(const double* n, double* s_out, double* t_out) {
  Frame f = make_frame(V3(n[0], n[1], n[2]));
  for (int k = 0; k < 3; ++k) {
    s_out[k] = f.s[k];
    t_out[k] = f.t[k];
  }
  return 0;
}


// The auxiliary-ray sampler: local vMF direction (lobe axis +z) for uniforms (u0, u1).
void oracle_vmf(double u0, double u1, double kappa, double* out) {
  V3 w = vmf_local(u0, u1, kappa);
  out[0] = w.x;
  out[1] = w.y;
  out[2] = w.z;
}

// Divergence on the sphere (gnomonic-chart duals) of analytic fields at u:
// kind 0: V = e (constant ambient vector), 1: V = w x e, 2: V = (I - w w^T) e.
double oracle_sphere_div(int kind, const double* u, const double* e) {
  V3 uu(u[0], u[1], u[2]), ee(e[0], e[1], e[2]);
  auto field = [&](VD w) -> VD {
    if (kind == 0) return constant(ee);
    if (kind == 1) return VD{w.z * ee.y * -1.0 + w.y * ee.z, w.x * ee.z * -1.0 + w.z * ee.x,
                             w.y * ee.x * -1.0 + w.x * ee.y};
    D2 we = dotd(w, ee);
    return VD{D2{ee.x, 0, 0} - w.x * we, D2{ee.y, 0, 0} - w.y * we, D2{ee.z, 0, 0} - w.z * we};
  };
  return sphere_div(uu, field);
}

// One warp field at origin o and center u (uniforms: 2 n_aux values): the
// field of parameter (param / 3, param % 3) for origin shape s_o evaluated at the
// unit direction `at` (NULL: u) into V_out, its divergence at u, and the log
// derivative with covector m (NULL: zero).  Returns the number of auxiliary hits.
int oracle_warp(void* sc, const double* o, const double* u, int s_o, const double* uni, const oracle_reparam_opts* opt,
                int param, const double* at, const double* m, double* V_out, double* div_out, double* logd_out) {
  const Scene& s = *(Scene*)sc;
  ReparamOpts op;
  if (!reparam_opts(opt, op)) return -1;
  V3 uu(u[0], u[1], u[2]);
  WarpSamples ws = warp_samples(s, op, V3(o[0], o[1], o[2]), uu, uni);
  const int ps = param / 3, pa = param % 3;
  V3 w = at ? V3(at[0], at[1], at[2]) : uu;
  Origin og{s_o, s_o >= 0 ? 0 : -1, 0.0, 0.0};
  const Param P{false, ps, 0, pa};
  const V3 oo(o[0], o[1], o[2]);
  VD V = warp_field(s, ws, oo, og, P, constant(w));
  V_out[0] = V.x.v;
  V_out[1] = V.y.v;
  V_out[2] = V.z.v;
  *div_out = sphere_div(uu, [&](VD x) { return warp_field(s, ws, oo, og, P, x); });
  if (logd_out) {
    std::vector<std::pair<int, double>> ld;
    warp_log_derivs(s, ws, oo, og, false, m ? V3(m[0], m[1], m[2]) : V3(), V3(), ld);
    *logd_out = 0.0;
    for (auto& pv : ld)
      if (pv.first == param) *logd_out = pv.second;
  }
  return (int)ws.hits.size();
}
}  // extern "C"
