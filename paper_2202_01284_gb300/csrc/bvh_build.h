// Host-side BVH construction: binned SAH over triangle centroids, then either
// a 2-wide layout with float child boxes or an 8-wide layout with 8-bit
// quantised child boxes (compressed wide BVH).
#pragma once

#include <cstdint>
#include <vector>

namespace ptgb {

struct BuildNode {
  float lo[3], hi[3];
  int left = -1, right = -1;  // children (build-node indices), -1 for a leaf
  int first = 0, count = 0;   // leaf: range into the triangle order
};

struct BuildTree {
  std::vector<BuildNode> nodes;  // nodes[0] = root
  std::vector<int> order;        // triangle ids in leaf order
  int depth = 0;
  double sah_cost = 0.0;
};

// tri_vertices: [n][3][3] float.  max_leaf >= 1, n_bins in [4, 64].
BuildTree build_sah(const float* tri_vertices, int n, int max_leaf, int n_bins);

// 2-wide GPU layout: per inner node four 16-byte words
//   w0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   w1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   w2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   w3 = (child0, child1, 0, 0) as int32: >= 0 inner node, < 0 leaf ~((first << 3) | (count - 1))
// Boxes are padded outward so that FP32 slab tests stay conservative.
// `order` (leaf order of triangles) is the one of the build tree.
void layout_binary(const BuildTree& t, std::vector<float>& words /* 16 floats per node */);

// Leaf size of the binary build that layout_wide collapses (the collapse forms the
// wide tree's leaves of up to max_leaf triangles itself).
int wide_build_leaf(int max_leaf);

// 8-wide compressed layout (80 bytes per node = five 16-byte words):
//   w0 = (origin.x, origin.y, origin.z, exps)  exps = e_x | e_y << 8 | e_z << 16 | imask << 24
//   w1 = (child_base, tri_base, meta[0..3], meta[4..7])
//   w2 = (qlo_x[0..3], qlo_x[4..7], qlo_y[0..3], qlo_y[4..7])
//   w3 = (qlo_z[0..3], qlo_z[4..7], qhi_x[0..3], qhi_x[4..7])
//   w4 = (qhi_y[0..3], qhi_y[4..7], qhi_z[0..3], qhi_z[4..7])
// The exponent byte e of an axis is the FP32 exponent of 2^15 times its step: a
// child box is origin + [q_lo, q_hi] * 2^(e - 142) per axis (conservative, with
// 2^-8 of a step between the planes and the padded child box where FP32 allows).
// meta[k] = 0 for an empty slot; inner child: (1 << 5) | k (non-zero; the child is
// node child_base + the number of inner slots below k, from imask); leaf child:
// count << 5 | tri_offset (count 1..3, tri_offset < 32 relative to tri_base: the
// triangles of all leaf children of a node are consecutive).  imask bit k set = slot
// k is an inner node.  The children come from a cost-optimal collapse of the binary
// tree (plan_wide), or the greedy largest-area collapse where that plan's tree would
// be deeper than the traversal stack.  Reorders `order_out` into the layout's
// triangle order.
void layout_wide(const BuildTree& t, std::vector<uint32_t>& words /* 20 words per node */,
                 std::vector<int>& order_out, int max_leaf);

}  // namespace ptgb
