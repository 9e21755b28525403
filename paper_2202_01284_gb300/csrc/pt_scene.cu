// Scene creation, emitter tables, BVH upload and status handling (host side of the C ABI).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bvh_build.h"
#include "pt_internal.h"

using namespace ptgb;

namespace {

template <class T>
int upload(void** dst, const T* src, size_t count) {
  if (*dst) {
    cudaFree(*dst);
    *dst = nullptr;
  }
  if (count == 0) return PT_OK;
  if (cudaMalloc(dst, count * sizeof(T)) != cudaSuccess) {
    *dst = nullptr;
    cudaGetLastError();
    return PT_ERR_OOM;
  }
  if (cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return PT_ERR_CUDA;
  return PT_OK;
}

// Guide table of a normalised CDF (Chen & Asau 1974 style "cutpoints"):
// guide[g] = the index the inversion rule (first i with u < cdf[i+1]) picks for
// u = g / G.  The pick for any u in [g/G, (g+1)/G) lies in [guide[g], guide[g+1]],
// so a binary search in that range returns exactly the full search's answer.
int guide_size(int n) {
  int g = 1;
  while (g < n && g < 4096) g <<= 1;
  return g;
}
void make_guide(const float* cdf, int n, int G, int* guide) {
  int i = 0;
  for (int g = 0; g <= G; ++g) {
    float u = (float)g / (float)G;
    while (i < n - 1 && !(u < cdf[i + 1])) ++i;
    guide[g] = i;
  }
}

void free_dev(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void scene_free_all(pt_scene* s) {
  free_dev(s->d_tri_v);
  free_dev(s->d_tri_a);
  free_dev(s->d_nodes);
  free_dev(s->d_shapes);
  free_dev(s->d_lights);
  free_dev(s->d_light_cdf);
  free_dev(s->d_env);
  free_dev(s->d_env_marg);
  free_dev(s->d_env_cond);
  free_dev(s->d_env_p);
  free_dev(s->d_light_guide);
  free_dev(s->d_env_marg_guide);
  free_dev(s->d_env_cond_guide);
  free_dev(s->d_status);
  free_dev(s->d_wf);
  free_dev(s->d_sample_L);
  std::free(s->h_vertices);
  std::free(s->h_uvs);
  std::free(s->h_tri_shape);
}

}  // namespace

extern "C" int pt_scene_create(const pt_scene_desc* d, pt_scene** out) {
  if (!d || !out || d->n_tris <= 0 || !d->vertices || !d->tri_shape || d->n_shapes <= 0 || !d->shapes)
    return PT_ERR_ARG;
  if (d->n_tris > (1 << 27)) return PT_ERR_ARG;
  if ((d->env_w > 0) != (d->env_h > 0) || (d->env_w > 0 && !d->env)) return PT_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < d->n_tris; ++i)
    if (d->tri_shape[i] < 0 || d->tri_shape[i] >= d->n_shapes) return PT_ERR_ARG;
  for (int i = 0; i < 9 * d->n_tris; ++i)
    if (!std::isfinite(d->vertices[i])) return PT_ERR_ARG;
  if (d->uvs)
    for (int i = 0; i < 6 * d->n_tris; ++i)
      if (!std::isfinite(d->uvs[i])) return PT_ERR_ARG;
  for (int i = 0; i < d->n_shapes; ++i) {
    const pt_shape& p = d->shapes[i];
    for (int c = 0; c < 3; ++c)
      if (!(p.emission[c] >= 0.0f) || !std::isfinite(p.emission[c]) || !std::isfinite(p.f0[c])) return PT_ERR_ARG;
    if (!std::isfinite(p.alpha) || !std::isfinite(p.eta) || !std::isfinite(p.diffuse_weight)) return PT_ERR_ARG;
  }
  if (d->env_w > 0)
    for (size_t i = 0; i < 4 * (size_t)d->env_w * d->env_h; ++i)
      if (!(d->env[i] >= 0.0f) || !std::isfinite(d->env[i])) return PT_ERR_ARG;
  {
    // emitters must have some area: light sampling divides by the total
    bool any_emitter = false;
    double area = 0.0;
    for (int t = 0; t < d->n_tris; ++t) {
      const pt_shape& p = d->shapes[d->tri_shape[t]];
      if (!(p.emission[0] > 0 || p.emission[1] > 0 || p.emission[2] > 0)) continue;
      any_emitter = true;
      const float* v = d->vertices + 9 * (size_t)t;
      const double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
      const double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
      const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      area += std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
    if (any_emitter && !(area > 0.0)) return PT_ERR_ARG;
  }
  pt_scene* s = new (std::nothrow) pt_scene();
  if (!s) return PT_ERR_OOM;
  s->n_tris = d->n_tris;
  s->n_shapes = d->n_shapes;
  // shape table
  std::vector<DevShape> shapes(d->n_shapes);
  for (int i = 0; i < d->n_shapes; ++i) {
    const pt_shape& p = d->shapes[i];
    if (p.bsdf < PT_BSDF_NONE || p.bsdf > PT_BSDF_BLEND || p.tex >= PT_MAX_TEX) {
      delete s;
      return PT_ERR_ARG;
    }
    DevShape& q = shapes[i];
    std::memset(&q, 0, sizeof q);
    q.bsdf = p.bsdf;
    q.tex = (p.bsdf == PT_BSDF_DIFFUSE || p.bsdf == PT_BSDF_BLEND) ? p.tex : -1;
    q.albedo_index = p.albedo_index;
    q.rough_index = (p.bsdf == PT_BSDF_CONDUCTOR || p.bsdf == PT_BSDF_BLEND) ? p.rough_index : -1;
    q.alpha = p.alpha;
    q.eta = p.eta;
    q.wd = p.diffuse_weight;
    q.emitter = (p.emission[0] > 0 || p.emission[1] > 0 || p.emission[2] > 0) ? 1.0f : 0.0f;
    q.f0x = p.f0[0];
    q.f0y = p.f0[1];
    q.f0z = p.f0[2];
    q.lex = p.emission[0];
    q.ley = p.emission[1];
    q.lez = p.emission[2];
    if (q.tex >= 0) s->max_tex_slot = std::max(s->max_tex_slot, q.tex);
    if (q.tex < 0 && (p.bsdf == PT_BSDF_DIFFUSE || p.bsdf == PT_BSDF_BLEND) && p.albedo_index >= 0)
      s->max_albedo_row = std::max(s->max_albedo_row, p.albedo_index);
    if (q.rough_index >= 0) s->max_rough = std::max(s->max_rough, q.rough_index);
    if ((p.bsdf == PT_BSDF_CONDUCTOR || p.bsdf == PT_BSDF_BLEND) && q.rough_index < 0 && !(p.alpha > 0)) {
      delete s;
      return PT_ERR_ARG;
    }
    if (p.bsdf == PT_BSDF_DIELECTRIC && !(p.eta > 0)) {
      delete s;
      return PT_ERR_ARG;
    }
  }
  // host copies for BVH builds
  size_t nv = 9 * (size_t)d->n_tris, nu = 6 * (size_t)d->n_tris;
  s->h_vertices = (float*)std::malloc(nv * sizeof(float));
  s->h_uvs = (float*)std::malloc(nu * sizeof(float));
  s->h_tri_shape = (int*)std::malloc((size_t)d->n_tris * sizeof(int));
  if (!s->h_vertices || !s->h_uvs || !s->h_tri_shape) {
    scene_free_all(s);
    delete s;
    return PT_ERR_OOM;
  }
  std::memcpy(s->h_vertices, d->vertices, nv * sizeof(float));
  if (d->uvs) std::memcpy(s->h_uvs, d->uvs, nu * sizeof(float));
  else std::memset(s->h_uvs, 0, nu * sizeof(float));
  std::memcpy(s->h_tri_shape, d->tri_shape, (size_t)d->n_tris * sizeof(int));

  int st = upload(&s->d_shapes, shapes.data(), shapes.size());
  // area lights: all triangles of emitting shapes, area-proportional CDF (FP64 -> FP32)
  std::vector<float4> lights;
  std::vector<double> cdf{0.0};
  for (int t = 0; t < d->n_tris && st == PT_OK; ++t) {
    const DevShape& q = shapes[d->tri_shape[t]];
    if (q.emitter == 0.0f) continue;
    const float* v = d->vertices + 9 * (size_t)t;
    double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
    double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
    double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double area = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    float4 a;
    a.x = v[0]; a.y = v[1]; a.z = v[2];
    uint32_t tid = (uint32_t)t;
    std::memcpy(&a.w, &tid, 4);
    lights.push_back(a);
    lights.push_back(make_float4(v[3], v[4], v[5], 0.f));
    lights.push_back(make_float4(v[6], v[7], v[8], 0.f));
    lights.push_back(make_float4(q.lex, q.ley, q.lez, 0.f));
    cdf.push_back(cdf.back() + area);
  }
  double total_area = cdf.back();
  std::vector<float> cdf_f(cdf.size());
  for (size_t i = 0; i < cdf.size(); ++i) cdf_f[i] = total_area > 0 ? (float)(cdf[i] / total_area) : 0.0f;
  if (!cdf_f.empty()) cdf_f.back() = 1.0f;
  if (st == PT_OK) st = upload(&s->d_lights, lights.data(), lights.size());
  if (st == PT_OK && !lights.empty()) st = upload(&s->d_light_cdf, cdf_f.data(), cdf_f.size());
  if (st == PT_OK && !lights.empty()) {
    int n = (int)(lights.size() / 4), G = guide_size(n);
    std::vector<int> guide(G + 1);
    make_guide(cdf_f.data(), n, G, guide.data());
    st = upload(&s->d_light_guide, guide.data(), guide.size());
    s->dev.light_g = G;
  }
  s->dev.n_lights = (int)(lights.size() / 4);
  s->dev.light_area = (float)total_area;
  // environment map: pixel weights luminance x sin(theta_center), marginal + conditional CDFs
  if (st == PT_OK && d->env_w > 0) {
    int W = d->env_w, H = d->env_h;
    size_t n = (size_t)W * H;
    std::vector<double> w(n);
    std::vector<float> marg(H + 1), cond((size_t)H * (W + 1)), prob(n);
    std::vector<double> rows(H);
    double total = 0.0;
    for (int y = 0; y < H; ++y) {
      double st_ = std::sin(3.14159265358979323846 * (y + 0.5) / H);
      double acc = 0.0;
      std::vector<double> c(W + 1, 0.0);
      for (int x = 0; x < W; ++x) {
        const float* e = d->env + 4 * ((size_t)y * W + x);
        double lum = 0.2126 * e[0] + 0.7152 * e[1] + 0.0722 * e[2];
        w[(size_t)y * W + x] = lum * st_;
        acc += lum * st_;
        c[x + 1] = acc;
      }
      for (int x = 0; x <= W; ++x) cond[(size_t)y * (W + 1) + x] = acc > 0 ? (float)(c[x] / acc) : 0.0f;
      if (acc > 0) cond[(size_t)y * (W + 1) + W] = 1.0f;
      rows[y] = acc;
      total += acc;
    }
    if (!(total > 0)) {
      scene_free_all(s);
      delete s;
      return PT_ERR_ARG;
    }
    double m = 0.0;
    marg[0] = 0.0f;
    for (int y = 0; y < H; ++y) {
      m += rows[y];
      marg[y + 1] = (float)(m / total);
    }
    marg[H] = 1.0f;
    for (size_t i = 0; i < n; ++i) prob[i] = (float)(w[i] / total);
    int gm = guide_size(H), gc = guide_size(W);
    std::vector<int> mguide(gm + 1), cguide((size_t)H * (gc + 1));
    make_guide(marg.data(), H, gm, mguide.data());
    for (int y = 0; y < H; ++y) make_guide(&cond[(size_t)y * (W + 1)], W, gc, &cguide[(size_t)y * (gc + 1)]);
    s->dev.env_gm = gm;
    s->dev.env_gc = gc;
    st = upload(&s->d_env, reinterpret_cast<const float4*>(d->env), n);
    if (st == PT_OK) st = upload(&s->d_env_marg_guide, mguide.data(), mguide.size());
    if (st == PT_OK) st = upload(&s->d_env_cond_guide, cguide.data(), cguide.size());
    if (st == PT_OK) st = upload(&s->d_env_marg, marg.data(), marg.size());
    if (st == PT_OK) st = upload(&s->d_env_cond, cond.data(), cond.size());
    if (st == PT_OK) st = upload(&s->d_env_p, prob.data(), prob.size());
    s->dev.env_w = W;
    s->dev.env_h = H;
    s->info.env_bytes = (int64_t)(n * 16 + marg.size() * 4 + cond.size() * 4 + n * 4);
  }
  if (st == PT_OK) {
    // status word at byte 0, the persistent launches' work counter at byte 128
    if (cudaMalloc(&s->d_status, 256) != cudaSuccess) st = PT_ERR_OOM;
    else if (cudaMemset(s->d_status, 0, 256) != cudaSuccess) st = PT_ERR_CUDA;
  }
  if (st != PT_OK) {
    cudaGetLastError();
    scene_free_all(s);
    delete s;
    return st;
  }
  s->dev.shapes = (const DevShape*)s->d_shapes;
  s->dev.n_shapes = d->n_shapes;
  s->dev.lights = (const float4*)s->d_lights;
  s->dev.light_cdf = (const float*)s->d_light_cdf;
  s->dev.light_guide = (const int*)s->d_light_guide;
  s->dev.env_marg_guide = (const int*)s->d_env_marg_guide;
  s->dev.env_cond_guide = (const int*)s->d_env_cond_guide;
  s->dev.env = (const float4*)s->d_env;
  s->dev.env_marg = (const float*)s->d_env_marg;
  s->dev.env_cond = (const float*)s->d_env_cond;
  s->dev.env_p = (const float*)s->d_env_p;
  s->dev.status = (int*)s->d_status;
  s->queue = reinterpret_cast<unsigned long long*>(static_cast<char*>(s->d_status) + 128);
  s->dev.n_tris = d->n_tris;
  s->info.n_tris = d->n_tris;
  *out = s;
  return PT_OK;
}

extern "C" void pt_scene_destroy(pt_scene* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  scene_free_all(s);
  delete s;
}

extern "C" int pt_bvh_build(pt_scene* s, const pt_bvh_opts* o) {
  if (!s) return PT_ERR_ARG;
  pt_bvh_opts opts{PT_BVH_BINARY, 0, 0};
  if (o) opts = *o;
  if (opts.layout != PT_BVH_BINARY && opts.layout != PT_BVH_WIDE) return PT_ERR_ARG;
  int max_leaf = opts.max_leaf_tris > 0 ? opts.max_leaf_tris : (opts.layout == PT_BVH_WIDE ? 3 : 4);
  int n_bins = opts.n_bins > 0 ? opts.n_bins : 32;
  if (n_bins < 4 || n_bins > 64) return PT_ERR_ARG;
  if (opts.layout == PT_BVH_BINARY && max_leaf > 8) return PT_ERR_ARG;
  if (opts.layout == PT_BVH_WIDE && max_leaf > 3) return PT_ERR_ARG;
  BuildTree tree = build_sah(s->h_vertices, s->n_tris, opts.layout == PT_BVH_WIDE ? wide_build_leaf(max_leaf) : max_leaf,
                             n_bins);
  std::vector<int> order = tree.order;
  std::vector<float> node_words;
  std::vector<uint32_t> wide_words;
  if (opts.layout == PT_BVH_BINARY) {
    layout_binary(tree, node_words);
  } else {
    layout_wide(tree, wide_words, order, max_leaf);
    if ((int)order.size() != s->n_tris) return PT_ERR_BVH;
  }
  // triangles and attributes in layout order
  std::vector<float4> tv(3 * (size_t)s->n_tris), ta(2 * (size_t)s->n_tris);
  for (int i = 0; i < s->n_tris; ++i) {
    int t = order[i];
    const float* v = s->h_vertices + 9 * (size_t)t;
    const float* uv = s->h_uvs + 6 * (size_t)t;
    float4 a;
    a.x = v[0]; a.y = v[1]; a.z = v[2];
    uint32_t tid = (uint32_t)t;
    std::memcpy(&a.w, &tid, 4);
    tv[3 * (size_t)i] = a;
    tv[3 * (size_t)i + 1] = make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], 0.f);
    tv[3 * (size_t)i + 2] = make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], 0.f);
    ta[2 * (size_t)i] = make_float4(uv[0], uv[1], uv[2], uv[3]);
    float4 b = make_float4(uv[4], uv[5], 0.f, 0.f);
    int shp = s->h_tri_shape[t];
    std::memcpy(&b.z, &shp, 4);
    ta[2 * (size_t)i + 1] = b;
  }
  int st = upload(&s->d_tri_v, tv.data(), tv.size());
  if (st == PT_OK) st = upload(&s->d_tri_a, ta.data(), ta.size());
  if (st == PT_OK) {
    if (opts.layout == PT_BVH_BINARY) st = upload(&s->d_nodes, node_words.data(), node_words.size());
    else st = upload(&s->d_nodes, wide_words.data(), wide_words.size());
  }
  if (st != PT_OK) {
    cudaGetLastError();
    s->has_bvh = 0;
    return st;
  }
  s->dev.tri_v = (const float4*)s->d_tri_v;
  s->dev.tri_a = (const float4*)s->d_tri_a;
  s->dev.nodes = (const float4*)s->d_nodes;
  s->dev.layout = opts.layout;
  s->has_bvh = 1;
  s->info.layout = opts.layout;
  s->info.depth = tree.depth;
  s->info.sah_cost = tree.sah_cost;
  s->info.n_nodes = opts.layout == PT_BVH_BINARY ? (int64_t)(node_words.size() / 16) : (int64_t)(wide_words.size() / 20);
  s->info.node_bytes = opts.layout == PT_BVH_BINARY ? (int64_t)node_words.size() * 4 : (int64_t)wide_words.size() * 4;
  s->info.tri_bytes = (int64_t)(tv.size() + ta.size()) * 16;
  return PT_OK;
}

extern "C" int pt_scene_get_info(const pt_scene* s, pt_scene_info* info) {
  if (!s || !info) return PT_ERR_ARG;
  *info = s->info;
  return PT_OK;
}

extern "C" int pt_last_device_status(pt_scene* s, void* stream, int* out) {
  if (!s || !out) return PT_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PT_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, s->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PT_ERR_CUDA;
  if (cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) return PT_ERR_CUDA;
  *out = v;
  return PT_OK;
}

extern "C" const char* pt_status_string(int st) {
  switch (st) {
    case PT_OK: return "ok";
    case PT_ERR_ARG: return "invalid argument";
    case PT_ERR_CUDA: return "CUDA runtime error";
    case PT_ERR_OOM: return "out of device memory";
    case PT_ERR_TIMEOUT: return "device-side wait timed out";
    case PT_ERR_BVH: return "BVH missing or traversal stack overflow";
    case PT_ERR_STATE: return "call order violated";
    default: return "unknown status";
  }
}
