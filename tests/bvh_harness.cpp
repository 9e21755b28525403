// Host-side checks of the library's BVH builder (test harness, CPU only).
//
// Builds the 2-wide and 8-wide layouts with the library's own builder source
// and checks, without a GPU: every child / triangle index stays inside its
// buffer, the triangle order is a permutation, every decoded child box contains
// the triangles below it, and a host replay of the kernels' traversal rules
// (FP32, same decode) finds the same closest triangle as brute force.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "bvh_build.h"

using namespace ptgb;

namespace {

struct Tri {
  float v0[3], e1[3], e2[3];
  int orig;
};

bool mt(const Tri& T, const float* o, const float* d, float& t_out) {
  auto cross = [](const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
  };
  auto dot = [](const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  float p[3], q[3], s[3];
  cross(d, T.e2, p);
  float det = dot(T.e1, p);
  if (det == 0.0f) return false;
  float inv = 1.0f / det;
  for (int k = 0; k < 3; ++k) s[k] = o[k] - T.v0[k];
  float u = dot(s, p) * inv;
  if (u < 0.0f || u > 1.0f) return false;
  cross(s, T.e1, q);
  float v = dot(d, q) * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  float t = dot(T.e2, q) * inv;
  if (!(t > 0.0f)) return false;
  t_out = t;
  return true;
}

struct Ctx {
  std::vector<Tri> tris;  // in layout order
  int bad = 0;            // index / containment violations
};

void test_tri(const Ctx& c, int pos, const float* o, const float* d, float& best, int& best_orig) {
  float t;
  if (mt(c.tris[pos], o, d, t)) {
    int orig = c.tris[pos].orig;
    if (t < best || (best_orig >= 0 && t == best && orig < best_orig)) {
      best = t;
      best_orig = orig;
    }
  }
}

int trace_wide(Ctx& c, const std::vector<uint32_t>& W, const float* o, const float* d, int& visits) {
  int n_nodes = (int)(W.size() / 20);
  float inv[3];
  for (int k = 0; k < 3; ++k) {
    float dk = std::fabs(d[k]) > 1e-20f ? d[k] : std::copysign(1e-20f, d[k]);
    inv[k] = 1.0f / dk;
  }
  uint32_t flip = (d[0] >= 0 ? 1u : 0u) | (d[1] >= 0 ? 2u : 0u) | (d[2] >= 0 ? 4u : 0u);
  std::vector<std::pair<uint32_t, uint32_t>> stack;
  int node = 0;
  float best = INFINITY;
  int best_orig = -1;
  for (;;) {
    if (node < 0 || node >= n_nodes) {
      c.bad++;
      break;
    }
    ++visits;
    const uint32_t* w = &W[(size_t)node * 20];
    uint32_t e = w[3], imask = e >> 24;
    float p[3];
    std::memcpy(p, w, 12);
    // as the kernel: plane q enters as 1 + q 2^-15 against A = 2^15 a (the stored
    // exponent is that of 2^15 times the step) and B = b - A in one FMA
    float A[3], B[3];
    for (int k = 0; k < 3; ++k) {
      uint32_t bits = ((e >> (8 * k)) & 0xffu) << 23;
      float sc;
      std::memcpy(&sc, &bits, 4);
      A[k] = sc * inv[k];
      B[k] = std::fma(p[k] - o[k], inv[k], -A[k]);
    }
    auto byte_of = [&](int word0, int sl) { return (w[word0 + (sl >> 2)] >> (8 * (sl & 3))) & 0xffu; };
    const int lo_w[3] = {8, 10, 12}, hi_w[3] = {14, 16, 18};
    uint32_t inner_hits = 0;
    for (int sl = 0; sl < 8; ++sl) {
      uint32_t meta = byte_of(6, sl);
      float tn = 0.0f, tf = best;
      for (int k = 0; k < 3; ++k) {
        float qn = (float)byte_of(d[k] >= 0 ? lo_w[k] : hi_w[k], sl);
        float qf = (float)byte_of(d[k] >= 0 ? hi_w[k] : lo_w[k], sl);
        tn = std::max(tn, std::fma(1.0f + qn * (1.0f / 32768.0f), A[k], B[k]));
        tf = std::min(tf, std::fma(1.0f + qf * (1.0f / 32768.0f), A[k], B[k]));
      }
      if (!(tn <= tf)) continue;  // as the kernel: an empty slot that passes is a leaf of zero triangles
      if ((imask >> sl) & 1u) {
        inner_hits |= 1u << (sl ^ flip);
      } else {
        int count = (int)(meta >> 5), first = (int)w[5] + (int)(meta & 31u);
        for (int i = 0; i < count; ++i) {
          if (first + i < 0 || first + i >= (int)c.tris.size()) {
            c.bad++;
            continue;
          }
          test_tri(c, first + i, o, d, best, best_orig);
        }
      }
    }
    uint32_t base = w[4], gmask = imask, hits = inner_hits;
    if (hits == 0u) {
      if (stack.empty()) break;
      base = stack.back().first;
      gmask = stack.back().second & 0xffu;
      hits = stack.back().second >> 8;
      stack.pop_back();
    }
    int k = __builtin_ctz(hits);
    hits &= hits - 1;
    int sl = k ^ (int)flip;
    node = (int)base + __builtin_popcount(gmask & ((1u << sl) - 1u));
    if (hits) {
      if (stack.size() >= 32) {
        c.bad++;
        break;
      }
      stack.push_back({base, gmask | (hits << 8)});
    }
  }
  return best_orig;
}

}  // namespace

extern "C" {

// Returns the number of violations (0 = ok).  stats: [n_wide_nodes, mismatches vs brute force,
// mean node visits x 1000, binary node count].
int check_bvh(const float* V, int n, const float* rays, int n_rays, int max_leaf, long long* stats) {
  BuildTree t = build_sah(V, n, max_leaf, 32);
  std::vector<float> bin;
  layout_binary(t, bin);
  // the 8-wide tree as pt_bvh_build makes it: collapsed from its own binary build
  BuildTree tw = build_sah(V, n, wide_build_leaf(max_leaf), 32);
  std::vector<uint32_t> W;
  std::vector<int> order;
  layout_wide(tw, W, order, max_leaf);
  int bad = 0;
  // permutation
  std::vector<int> seen(n, 0);
  if ((int)order.size() != n) bad++;
  for (int x : order) {
    if (x < 0 || x >= n || seen[x]++) bad++;
  }
  Ctx c;
  c.tris.resize(order.size());
  for (size_t i = 0; i < order.size(); ++i) {
    const float* v = V + 9 * (size_t)order[i];
    Tri& T = c.tris[i];
    for (int k = 0; k < 3; ++k) {
      T.v0[k] = v[k];
      T.e1[k] = v[3 + k] - v[k];
      T.e2[k] = v[6 + k] - v[k];
    }
    T.orig = order[i];
  }
  // containment: every triangle lies inside the decoded box of each slot on its path
  int n_wide = (int)(W.size() / 20);
  for (int node = 0; node < n_wide; ++node) {
    const uint32_t* w = &W[(size_t)node * 20];
    uint32_t e = w[3], imask = e >> 24;
    float p[3], sc[3];
    std::memcpy(p, w, 12);
    for (int k = 0; k < 3; ++k) {
      uint32_t bits = ((e >> (8 * k)) & 0xffu) << 23;
      std::memcpy(&sc[k], &bits, 4);
      sc[k] *= 1.0f / 32768.0f;  // the step itself
    }
    for (int sl = 0; sl < 8; ++sl) {
      uint32_t meta = (w[6 + (sl >> 2)] >> (8 * (sl & 3))) & 0xffu;
      if (!meta) continue;
      if ((imask >> sl) & 1u) {
        int child = (int)w[4] + __builtin_popcount(imask & ((1u << sl) - 1u));
        if (child <= node || child >= n_wide) bad++;
      } else {
        int count = (int)(meta >> 5), first = (int)w[5] + (int)(meta & 31u);
        if (count < 1 || count > 3 || first < 0 || first + count > n) {
          bad++;
          continue;
        }
        for (int i = 0; i < count; ++i) {
          const float* v = V + 9 * (size_t)order[first + i];
          for (int k = 0; k < 3; ++k) {
            float lo = p[k] + (float)((w[8 + 2 * k + (sl >> 2)] >> (8 * (sl & 3))) & 0xffu) * sc[k];
            float hi = p[k] + (float)((w[14 + 2 * k + (sl >> 2)] >> (8 * (sl & 3))) & 0xffu) * sc[k];
            for (int j = 0; j < 3; ++j)
              if (v[3 * j + k] < lo || v[3 * j + k] > hi) bad++;
          }
        }
      }
    }
  }
  // traversal replay vs brute force
  long long mism = 0, visits = 0;
  for (int r = 0; r < n_rays; ++r) {
    const float* o = rays + 6 * (size_t)r;
    const float* d = o + 3;
    int v = 0;
    int got = trace_wide(c, W, o, d, v);
    visits += v;
    float best = INFINITY;
    int want = -1;
    for (int i = 0; i < n; ++i) test_tri(c, i, o, d, best, want);
    if (got != want) mism++;
  }
  bad += c.bad;
  stats[0] = n_wide;
  stats[1] = mism;
  stats[2] = n_rays ? visits * 1000 / n_rays : 0;
  stats[3] = (long long)(bin.size() / 16);
  return bad;
}

}  // extern "C"
