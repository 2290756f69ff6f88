// Host plan of the treecode far field (see tree_plan.h).  No device code: the file builds with
// nvcc into the library and with a plain C++ compiler in the host tests.
#include "tree_plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace pbfb {

namespace {

void node_box(const double* xyz, const std::vector<int>& perm, int b, int e, double* box) {
  for (int d = 0; d < 3; ++d) {
    box[d] = 1e300;
    box[3 + d] = -1e300;
  }
  for (int q = b; q < e; ++q)
    for (int d = 0; d < 3; ++d) {
      const double v = xyz[3 * (size_t)perm[q] + d];
      box[d] = std::min(box[d], v);
      box[3 + d] = std::max(box[3 + d], v);
    }
}

double radius(const double* box) {
  const double dx = box[3] - box[0], dy = box[4] - box[1], dz = box[5] - box[2];
  return 0.5 * std::sqrt(dx * dx + dy * dy + dz * dz);
}

double centre_distance(const double* a, const double* b) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double t = 0.5 * (a[d] + a[3 + d]) - 0.5 * (b[d] + b[3 + d]);
    s += t * t;
  }
  return std::sqrt(s);
}

}  // namespace

int build_tree_plan(const double* xyz, int n, int leaf, double theta, int min_size, TreePlan* out) {
  if (!xyz || !out || n < 1 || leaf < 1 || !(theta > 0.0 && theta < 1.0)) return 1;
  for (size_t i = 0; i < 3 * (size_t)n; ++i)
    if (!std::isfinite(xyz[i])) return 1;
  TreePlan& t = *out;
  t = TreePlan();
  t.n = n;
  t.leaf = leaf;
  t.perm.resize(n);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  // breadth-first: children of a node are stored consecutively
  t.begin.push_back(0);
  t.end.push_back(n);
  t.child.push_back(-1);
  t.box.resize(6);
  node_box(xyz, t.perm, 0, n, t.box.data());
  for (size_t k = 0; k < t.begin.size(); ++k) {
    const int b = t.begin[k], e = t.end[k];
    if (e - b <= leaf) continue;
    const double* bx = &t.box[6 * k];
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (bx[3 + d] - bx[d] > bx[3 + ax] - bx[ax]) ax = d;
    const int mid = b + (e - b) / 2;
    std::stable_sort(t.perm.begin() + b, t.perm.begin() + e, [&](int i, int j) {
      return xyz[3 * (size_t)i + ax] < xyz[3 * (size_t)j + ax];
    });
    const int c = (int)t.begin.size();
    t.child[k] = c;
    for (int h = 0; h < 2; ++h) {
      const int cb = h == 0 ? b : mid, ce = h == 0 ? mid : e;
      t.begin.push_back(cb);
      t.end.push_back(ce);
      t.child.push_back(-1);
      t.box.resize(t.box.size() + 6);
      node_box(xyz, t.perm, cb, ce, &t.box[t.box.size() - 6]);
    }
  }
  for (size_t k = 0; k < t.begin.size(); ++k)
    if (t.child[k] < 0) t.leaves.push_back((int)k);
  std::sort(t.leaves.begin(), t.leaves.end(), [&](int a, int b) { return t.begin[a] < t.begin[b]; });
  // interaction lists, one root-to-leaf walk per target leaf
  t.far_ptr.assign(1, 0);
  t.near_ptr.assign(1, 0);
  std::vector<int> stack;
  for (int B : t.leaves) {
    const double* bb = &t.box[6 * (size_t)B];
    const double rb = radius(bb);
    stack.assign(1, 0);
    while (!stack.empty()) {
      const int C = stack.back();
      stack.pop_back();
      const double* cb = &t.box[6 * (size_t)C];
      const int size = t.end[C] - t.begin[C];
      if (C != B && size > min_size && rb + radius(cb) < theta * centre_distance(bb, cb)) {
        t.far_node.push_back(C);
      } else if (t.child[C] < 0) {
        t.near_node.push_back(C);
      } else {
        stack.push_back(t.child[C] + 1);  // the first child is visited first
        stack.push_back(t.child[C]);
      }
    }
    t.far_ptr.push_back((int)t.far_node.size());
    t.near_ptr.push_back((int)t.near_node.size());
  }
  return 0;
}

}  // namespace pbfb
