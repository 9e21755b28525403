// Binned-SAH BVH builder and GPU layouts (host C++).
//
// The paper delegates ray tracing to Embree/OptiX (Sec. 3.1); on GB300 the
// RT cores are not reachable from CUDA, so the acceleration structure is our
// own: a binned surface-area-heuristic build (cost = 1 per traversal step + 1
// per triangle test), laid out either as a 2-wide tree with float boxes or as
// an 8-wide tree with 8-bit quantised child boxes (80-byte nodes, five
// 16-byte loads per node).  The 8-wide tree is collapsed from a binary tree
// built down to single triangles by a cost-optimal dynamic programme that also
// forms its leaves (up to three triangles).
#include "bvh_build.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>

namespace ptgb {
namespace {

struct Box {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const float* l, const float* h) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], l[k]);
      hi[k] = std::max(hi[k], h[k]);
    }
  }
  void grow_pt(const float* p) { grow(p, p); }
  double area() const {
    if (!(hi[0] >= lo[0])) return 0.0;
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

struct Job {
  int node, first, count, depth;
};

}  // namespace

BuildTree build_sah(const float* V, int n, int max_leaf, int n_bins) {
  BuildTree t;
  std::vector<float> tlo(3 * (size_t)n), thi(3 * (size_t)n), cen(3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const float* v = V + (size_t)i * 9;
    for (int k = 0; k < 3; ++k) {
      float a = v[k], b = v[3 + k], c = v[6 + k];
      tlo[3 * i + k] = std::min(a, std::min(b, c));
      thi[3 * i + k] = std::max(a, std::max(b, c));
      cen[3 * i + k] = 0.5f * (tlo[3 * i + k] + thi[3 * i + k]);
    }
  }
  t.order.resize(n);
  for (int i = 0; i < n; ++i) t.order[i] = i;
  auto bounds_of = [&](int first, int count, Box& b) {
    for (int i = first; i < first + count; ++i) {
      int tri = t.order[i];
      b.grow(&tlo[3 * tri], &thi[3 * tri]);
    }
  };
  t.nodes.reserve(2 * (size_t)n);
  t.nodes.emplace_back();
  {
    Box b;
    bounds_of(0, n, b);
    std::memcpy(t.nodes[0].lo, b.lo, sizeof b.lo);
    std::memcpy(t.nodes[0].hi, b.hi, sizeof b.hi);
  }
  double root_area = std::max(Box{}.area(), 0.0);
  {
    Box b;
    std::memcpy(b.lo, t.nodes[0].lo, sizeof b.lo);
    std::memcpy(b.hi, t.nodes[0].hi, sizeof b.hi);
    root_area = std::max(b.area(), 1e-30);
  }
  std::vector<Job> stack;
  stack.push_back({0, 0, n, 1});
  std::vector<int> bin_count(n_bins);
  std::vector<Box> bin_box(n_bins);
  std::vector<double> right_area(n_bins);
  std::vector<int> right_count(n_bins);
  double sah = 0.0;
  while (!stack.empty()) {
    Job j = stack.back();
    stack.pop_back();
    t.depth = std::max(t.depth, j.depth);
    BuildNode& nd = t.nodes[j.node];
    Box nb;
    std::memcpy(nb.lo, nd.lo, sizeof nb.lo);
    std::memcpy(nb.hi, nd.hi, sizeof nb.hi);
    double a_node = std::max(nb.area(), 1e-30);
    auto make_leaf = [&]() {
      t.nodes[j.node].first = j.first;
      t.nodes[j.node].count = j.count;
      sah += a_node / root_area * j.count;
    };
    if (j.count <= 1) {
      make_leaf();
      continue;
    }
    Box cb;
    for (int i = j.first; i < j.first + j.count; ++i) cb.grow_pt(&cen[3 * t.order[i]]);
    double best_cost = INFINITY;
    int best_axis = -1, best_split = -1;
    bool force_median = j.depth >= 48;  // keeps the tree shallow enough for a 64-entry stack
    if (!force_median) {
      for (int axis = 0; axis < 3; ++axis) {
        float ext = cb.hi[axis] - cb.lo[axis];
        if (!(ext > 0.0f)) continue;
        float scale = (float)n_bins / ext;
        std::fill(bin_count.begin(), bin_count.end(), 0);
        std::fill(bin_box.begin(), bin_box.end(), Box{});
        for (int i = j.first; i < j.first + j.count; ++i) {
          int tri = t.order[i];
          int b = std::min((int)((cen[3 * tri + axis] - cb.lo[axis]) * scale), n_bins - 1);
          bin_count[b]++;
          bin_box[b].grow(&tlo[3 * tri], &thi[3 * tri]);
        }
        Box acc;
        int cnt = 0;
        for (int b = n_bins - 1; b > 0; --b) {
          acc.grow(bin_box[b].lo, bin_box[b].hi);
          cnt += bin_count[b];
          right_area[b] = acc.area();
          right_count[b] = cnt;
        }
        Box lacc;
        int lcnt = 0;
        for (int b = 0; b < n_bins - 1; ++b) {
          lacc.grow(bin_box[b].lo, bin_box[b].hi);
          lcnt += bin_count[b];
          if (lcnt == 0 || right_count[b + 1] == 0) continue;
          double cost = 1.0 + (lacc.area() * lcnt + right_area[b + 1] * right_count[b + 1]) / a_node;
          if (cost < best_cost) {
            best_cost = cost;
            best_axis = axis;
            best_split = b;
          }
        }
      }
      if (j.count <= max_leaf && (best_axis < 0 || (double)j.count <= best_cost)) {
        make_leaf();
        continue;
      }
    } else if (j.count <= max_leaf) {
      make_leaf();
      continue;
    }
    int mid;
    if (best_axis >= 0) {
      float ext = cb.hi[best_axis] - cb.lo[best_axis];
      float scale = (float)n_bins / ext;
      auto it = std::partition(t.order.begin() + j.first, t.order.begin() + j.first + j.count, [&](int tri) {
        int b = std::min((int)((cen[3 * tri + best_axis] - cb.lo[best_axis]) * scale), n_bins - 1);
        return b <= best_split;
      });
      mid = (int)(it - t.order.begin());
    } else {
      // all centroids coincide (or forced): split by object median on the widest axis
      int axis = 0;
      float e0 = cb.hi[0] - cb.lo[0], e1 = cb.hi[1] - cb.lo[1], e2 = cb.hi[2] - cb.lo[2];
      axis = (e0 >= e1 && e0 >= e2) ? 0 : (e1 >= e2 ? 1 : 2);
      mid = j.first + j.count / 2;
      std::nth_element(t.order.begin() + j.first, t.order.begin() + mid, t.order.begin() + j.first + j.count,
                       [&](int a, int b) { return cen[3 * a + axis] < cen[3 * b + axis] || (cen[3 * a + axis] == cen[3 * b + axis] && a < b); });
    }
    if (mid <= j.first || mid >= j.first + j.count) mid = j.first + j.count / 2;
    sah += a_node / root_area * 1.0;
    int l = (int)t.nodes.size();
    t.nodes.emplace_back();
    t.nodes.emplace_back();
    int r = l + 1;
    Box lb, rb;
    bounds_of(j.first, mid - j.first, lb);
    bounds_of(mid, j.first + j.count - mid, rb);
    std::memcpy(t.nodes[l].lo, lb.lo, sizeof lb.lo);
    std::memcpy(t.nodes[l].hi, lb.hi, sizeof lb.hi);
    std::memcpy(t.nodes[r].lo, rb.lo, sizeof rb.lo);
    std::memcpy(t.nodes[r].hi, rb.hi, sizeof rb.hi);
    t.nodes[j.node].left = l;
    t.nodes[j.node].right = r;
    stack.push_back({r, mid, j.first + j.count - mid, j.depth + 1});
    stack.push_back({l, j.first, mid - j.first, j.depth + 1});
  }
  t.sah_cost = sah;
  return t;
}

namespace {
// Conservative outward padding of a box coordinate for FP32 slab tests.
float pad_lo(float v, float abs_pad) { return v - (std::fabs(v) * 3.0e-6f + abs_pad); }
float pad_hi(float v, float abs_pad) { return v + (std::fabs(v) * 3.0e-6f + abs_pad); }
float scene_abs_pad(const BuildTree& t) {
  const BuildNode& r = t.nodes[0];
  float e = std::max(r.hi[0] - r.lo[0], std::max(r.hi[1] - r.lo[1], r.hi[2] - r.lo[2]));
  return std::max(e, 1e-20f) * 1.0e-6f;
}
}  // namespace

void layout_binary(const BuildTree& t, std::vector<float>& words) {
  const float ap = scene_abs_pad(t);
  std::vector<int> gidx(t.nodes.size(), -1);
  std::vector<int> inner;
  std::vector<int> st{0};
  while (!st.empty()) {
    int i = st.back();
    st.pop_back();
    if (t.nodes[i].left < 0) continue;
    gidx[i] = (int)inner.size();
    inner.push_back(i);
    st.push_back(t.nodes[i].right);
    st.push_back(t.nodes[i].left);
  }
  auto leaf_ref = [&](const BuildNode& n) { return ~((n.first << 3) | (n.count - 1)); };
  auto child_ref = [&](int c) { return t.nodes[c].left < 0 ? leaf_ref(t.nodes[c]) : gidx[c]; };
  auto put = [&](float* w, int c0, int c1, int r0, int r1) {
    const BuildNode& a = t.nodes[c0];
    const BuildNode& b = t.nodes[c1];
    w[0] = pad_lo(a.lo[0], ap); w[1] = pad_hi(a.hi[0], ap); w[2] = pad_lo(a.lo[1], ap); w[3] = pad_hi(a.hi[1], ap);
    w[4] = pad_lo(b.lo[0], ap); w[5] = pad_hi(b.hi[0], ap); w[6] = pad_lo(b.lo[1], ap); w[7] = pad_hi(b.hi[1], ap);
    w[8] = pad_lo(a.lo[2], ap); w[9] = pad_hi(a.hi[2], ap); w[10] = pad_lo(b.lo[2], ap); w[11] = pad_hi(b.hi[2], ap);
    int32_t refs[4] = {r0, r1, 0, 0};
    std::memcpy(&w[12], refs, sizeof refs);
  };
  if (inner.empty()) {  // the whole scene is one leaf: root with the leaf in both slots
    words.assign(16, 0.0f);
    int r = leaf_ref(t.nodes[0]);
    put(words.data(), 0, 0, r, r);
    return;
  }
  words.assign(inner.size() * 16, 0.0f);
  for (size_t g = 0; g < inner.size(); ++g) {
    const BuildNode& n = t.nodes[inner[g]];
    put(&words[g * 16], n.left, n.right, child_ref(n.left), child_ref(n.right));
  }
}

namespace {

// Children of one 8-wide node: collapse the binary tree greedily by opening the
// inner child with the largest surface area while at most 8 children result.
void collapse_children(const BuildTree& t, int b, std::vector<int>& out) {
  out.clear();
  const BuildNode& n = t.nodes[b];
  if (n.left < 0) {  // a leaf as the whole (root) node
    out.push_back(b);
    return;
  }
  out.push_back(n.left);
  out.push_back(n.right);
  while (out.size() < 8) {
    int best = -1;
    double best_area = -1.0;
    for (size_t i = 0; i < out.size(); ++i) {
      const BuildNode& c = t.nodes[out[i]];
      if (c.left < 0) continue;
      Box bx;
      std::memcpy(bx.lo, c.lo, sizeof bx.lo);
      std::memcpy(bx.hi, c.hi, sizeof bx.hi);
      double a = bx.area();
      if (a > best_area) {
        best_area = a;
        best = (int)i;
      }
    }
    if (best < 0) break;
    int c = out[best];
    out[best] = t.nodes[c].left;
    out.push_back(t.nodes[c].right);
  }
}

// Cost-optimal collapse of the binary tree into 8-wide nodes (dynamic programming
// after Ylitie, Karras and Laine 2017).  A ray that reaches a box pays c_node if the
// box is a wide node (its eight child tests) or c_tri per triangle if it is a leaf;
// the chance of reaching a box is proportional to its surface area.  For a binary
// node m and i = 1..8, slots(m, i) is the cheapest way to put m's subtree into at
// most i child slots of the parent: one slot holding m itself (a leaf of all its
// triangles if they are at most max_leaf, or a new wide node), or the slots split
// between m's two children.  A wide node at m costs c_node A(m) plus the cheapest
// split of its two children over 8 slots.
#ifndef PT_WIDE_NODE_COST
#define PT_WIDE_NODE_COST 1.0
#endif
#ifndef PT_WIDE_TRI_COST
#define PT_WIDE_TRI_COST 0.5
#endif
#ifndef PT_WIDE_COLLAPSE_DP
#define PT_WIDE_COLLAPSE_DP 1
#endif
#ifndef PT_WIDE_BUILD_LEAF
#define PT_WIDE_BUILD_LEAF 1
#endif
struct WidePlan {
  std::vector<int> first, count;           // subtree triangle range in t.order
  std::vector<float> slots;                // [node][8]: slots(m, i + 1)
  std::vector<int8_t> how;                 // [node][8]: 0 = m in one slot, k > 0 = k slots left
  std::vector<uint8_t> leaf;               // m as one slot is a leaf (else a wide node)
  std::vector<int8_t> split;               // wide node at m: slots given to the left child
};

WidePlan plan_wide(const BuildTree& t, int max_leaf) {
  const int n = (int)t.nodes.size();
  WidePlan p;
  p.first.assign(n, 0);
  p.count.assign(n, 0);
  p.slots.assign((size_t)n * 8, 0.0f);
  p.how.assign((size_t)n * 8, 0);
  p.leaf.assign(n, 0);
  p.split.assign(n, 0);
  const double cn = PT_WIDE_NODE_COST, ct = PT_WIDE_TRI_COST;
  // children are created after their parent, so a reverse sweep visits them first
  for (int m = n - 1; m >= 0; --m) {
    const BuildNode& b = t.nodes[m];
    Box bx;
    std::memcpy(bx.lo, b.lo, sizeof bx.lo);
    std::memcpy(bx.hi, b.hi, sizeof bx.hi);
    const double a = bx.area();
    float* S = &p.slots[(size_t)m * 8];
    int8_t* H = &p.how[(size_t)m * 8];
    if (b.left < 0) {
      p.first[m] = b.first;
      p.count[m] = b.count;
      p.leaf[m] = 1;
      for (int i = 0; i < 8; ++i) S[i] = (float)(ct * b.count * a);
      continue;
    }
    const int l = b.left, r = b.right;
    p.first[m] = p.first[l];
    p.count[m] = p.count[l] + p.count[r];
    const float* SL = &p.slots[(size_t)l * 8];
    const float* SR = &p.slots[(size_t)r * 8];
    // wide node at m: the two children over at most 8 slots
    double best = INFINITY;
    int bk = 1;
    for (int k = 1; k < 8; ++k) {
      const double c = (double)SL[k - 1] + SR[8 - k - 1];
      if (c < best) {
        best = c;
        bk = k;
      }
    }
    const double inner = cn * a + best;
    const double as_leaf = p.count[m] <= max_leaf ? ct * p.count[m] * a : INFINITY;
    p.split[m] = (int8_t)bk;
    p.leaf[m] = as_leaf <= inner ? 1 : 0;
    const double one = std::min(as_leaf, inner);
    S[0] = (float)one;
    H[0] = 0;
    for (int i = 2; i <= 8; ++i) {
      double c = S[i - 2];
      int h = H[i - 2];
      for (int k = 1; k < i; ++k) {
        const double d = (double)SL[k - 1] + SR[i - k - 1];
        if (d < c) {
          c = d;
          h = k;
        }
      }
      S[i - 1] = (float)c;
      H[i - 1] = (int8_t)h;
    }
  }
  return p;
}

// The child slots of the wide node at binary node m under plan p.
void plan_slots(const BuildTree& t, const WidePlan& p, int m, int i, std::vector<int>& out) {
  const int h = p.how[(size_t)m * 8 + i - 1];
  if (h == 0 || t.nodes[m].left < 0) {
    out.push_back(m);
    return;
  }
  plan_slots(t, p, t.nodes[m].left, h, out);
  plan_slots(t, p, t.nodes[m].right, i - h, out);
}
void plan_children(const BuildTree& t, const WidePlan& p, int m, std::vector<int>& out) {
  out.clear();
  if (t.nodes[m].left < 0) {
    out.push_back(m);
    return;
  }
  const int k = p.split[m];
  plan_slots(t, p, t.nodes[m].left, k, out);
  plan_slots(t, p, t.nodes[m].right, 8 - k, out);
}
// Depth of the wide tree the plan makes (levels of wide nodes).
int plan_depth(const BuildTree& t, const WidePlan& p) {
  int depth = 0;
  std::vector<std::pair<int, int>> st{{0, 1}};
  std::vector<int> kids;
  while (!st.empty()) {
    auto [m, d] = st.back();
    st.pop_back();
    depth = std::max(depth, d);
    plan_children(t, p, m, kids);
    for (int c : kids)
      if (t.nodes[c].left >= 0 && !p.leaf[c]) st.push_back({c, d + 1});
  }
  return depth;
}

uint32_t pack4(const uint8_t* b) {
  return (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24);
}

}  // namespace

int wide_build_leaf(int max_leaf) { return PT_WIDE_COLLAPSE_DP ? std::min(PT_WIDE_BUILD_LEAF, max_leaf) : max_leaf; }

void layout_wide(const BuildTree& t, std::vector<uint32_t>& words, std::vector<int>& order_out, int max_leaf) {
  (void)max_leaf;
  const float ap = scene_abs_pad(t);
  struct Item {
    int b, w;
  };
  std::vector<Item> queue{{0, 0}};
  size_t head = 0;
  int n_wide = 1;
  words.assign(20, 0u);
  order_out.clear();
  std::vector<int> kids;
  const WidePlan plan = plan_wide(t, max_leaf);
  // the traversal keeps one stack entry per wide level: the greedy collapse (at
  // least two binary levels per wide level) stays the fallback for deep trees
  const bool use_plan = PT_WIDE_COLLAPSE_DP && plan_depth(t, plan) <= 30;
  auto inner = [&](int c) { return t.nodes[c].left >= 0 && !(use_plan && plan.leaf[c]); };
  while (head < queue.size()) {
    Item it = queue[head++];
    if (use_plan)
      plan_children(t, plan, it.b, kids);
    else
      collapse_children(t, it.b, kids);
    // node box = union of the (padded) child boxes
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    std::vector<std::array<float, 6>> cb(kids.size());
    for (size_t i = 0; i < kids.size(); ++i) {
      const BuildNode& c = t.nodes[kids[i]];
      for (int k = 0; k < 3; ++k) {
        cb[i][k] = pad_lo(c.lo[k], ap);
        cb[i][3 + k] = pad_hi(c.hi[k], ap);
        lo[k] = std::min(lo[k], cb[i][k]);
        hi[k] = std::max(hi[k], cb[i][3 + k]);
      }
    }
    // slot assignment: slot bit k set = child centroid on the negative side of axis k
    float ctr[3] = {0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2])};
    int slot_of[8];
    bool used[8] = {false, false, false, false, false, false, false, false};
    std::vector<bool> done(kids.size(), false);
    for (size_t round = 0; round < kids.size(); ++round) {
      double best = -INFINITY;
      int bc = -1, bs = -1;
      for (size_t i = 0; i < kids.size(); ++i) {
        if (done[i]) continue;
        double off[3];
        for (int k = 0; k < 3; ++k) off[k] = 0.5 * ((double)cb[i][k] + cb[i][3 + k]) - ctr[k];
        for (int sl = 0; sl < 8; ++sl) {
          if (used[sl]) continue;
          double score = 0.0;
          for (int k = 0; k < 3; ++k) score += ((sl >> k) & 1) ? -off[k] : off[k];
          if (score > best) {
            best = score;
            bc = (int)i;
            bs = sl;
          }
        }
      }
      done[bc] = true;
      used[bs] = true;
      slot_of[bc] = bs;
    }
    int slot_child[8];
    for (int sl = 0; sl < 8; ++sl) slot_child[sl] = -1;
    for (size_t i = 0; i < kids.size(); ++i) slot_child[slot_of[i]] = (int)i;
    // quantisation frame: power-of-two step per axis, 8-bit coordinates
    int ebits[3];
    float scale[3];
    for (int k = 0; k < 3; ++k) {
      float ext = std::max(hi[k] - lo[k], 1e-30f);
      int e = (int)std::ceil(std::log2(ext / 254.0f));
      e = std::min(std::max(e, -126), 112);
      ebits[k] = e + 127 + 15;  // stored as the FP32 exponent of 2^15 times the step
      scale[k] = std::ldexp(1.0f, e);
      // keep 1/256 of a step between each child box and its quantised planes (the
      // traversal's plane decode rounds by up to 1/512 of a step): the origin moves out
      // by that much (where FP32 can represent the move; otherwise the step is below
      // 2^-15 of the coordinate and the boxes' relative padding covers the rounding)
      lo[k] -= std::ldexp(1.0f, e - 8);
    }
    // empty slots get inverted boxes (low planes 255, high planes 0), which every slab
    // test rejects: the traversal needs no separate empty-slot test
    uint8_t meta[8] = {0}, qlo[3][8], qhi[3][8];
    std::memset(qlo, 0xff, sizeof qlo);
    std::memset(qhi, 0, sizeof qhi);
    uint8_t imask = 0;
    uint32_t child_base = (uint32_t)n_wide;
    uint32_t tri_base = (uint32_t)order_out.size();
    int inner_rank = 0;
    for (int sl = 0; sl < 8; ++sl) {
      int i = slot_child[sl];
      if (i < 0) continue;
      for (int k = 0; k < 3; ++k) {
        int q0 = (int)std::floor((cb[i][k] - lo[k]) / scale[k]);
        int q1 = (int)std::ceil((cb[i][3 + k] - lo[k]) / scale[k]);
        q0 = std::min(std::max(q0, 0), 255);
        q1 = std::min(std::max(q1, 0), 255);
        const float margin = std::ldexp(scale[k], -8);
        while (q0 > 0 && lo[k] + (float)q0 * scale[k] > cb[i][k] - margin) --q0;
        while (q1 < 255 && lo[k] + (float)q1 * scale[k] < cb[i][3 + k] + margin) ++q1;
        qlo[k][sl] = (uint8_t)q0;
        qhi[k][sl] = (uint8_t)q1;
      }
      if (inner(kids[i])) {
        imask |= (uint8_t)(1u << sl);
        meta[sl] = (uint8_t)(0x20 | sl);  // non-zero marker; the child index comes from imask ranks
        queue.push_back({kids[i], (int)child_base + inner_rank});
        ++inner_rank;
      } else {
        int off = (int)(order_out.size() - tri_base);
        const int first = plan.first[kids[i]], count = plan.count[kids[i]];
        for (int k = 0; k < count; ++k) order_out.push_back(t.order[first + k]);
        meta[sl] = (uint8_t)((count << 5) | off);
      }
    }
    n_wide += inner_rank;
    words.resize((size_t)n_wide * 20, 0u);
    uint32_t* w = &words[(size_t)it.w * 20];
    std::memcpy(&w[0], &lo[0], 4);
    std::memcpy(&w[1], &lo[1], 4);
    std::memcpy(&w[2], &lo[2], 4);
    w[3] = (uint32_t)ebits[0] | ((uint32_t)ebits[1] << 8) | ((uint32_t)ebits[2] << 16) | ((uint32_t)imask << 24);
    w[4] = child_base;
    w[5] = tri_base;
    w[6] = pack4(meta);
    w[7] = pack4(meta + 4);
    w[8] = pack4(qlo[0]);
    w[9] = pack4(qlo[0] + 4);
    w[10] = pack4(qlo[1]);
    w[11] = pack4(qlo[1] + 4);
    w[12] = pack4(qlo[2]);
    w[13] = pack4(qlo[2] + 4);
    w[14] = pack4(qhi[0]);
    w[15] = pack4(qhi[0] + 4);
    w[16] = pack4(qhi[1]);
    w[17] = pack4(qhi[1] + 4);
    w[18] = pack4(qhi[2]);
    w[19] = pack4(qhi[2] + 4);
  }
}

}  // namespace ptgb
