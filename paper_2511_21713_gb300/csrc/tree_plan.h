// Host plan of a hierarchical (treecode) far field over a set of points: a binary tree and, per
// leaf (a batch of targets), the clusters whose interaction with it may be approximated through
// interpolation proxies and the leaves it must sum directly.  Plain C++ (no CUDA), deterministic.
#pragma once

#include <vector>

namespace pbfb {

struct TreePlan {
  int n = 0;                           // points
  int leaf = 0;                        // largest leaf
  std::vector<int> perm;               // tree position -> point index
  std::vector<int> begin, end;         // per node: its points are perm[begin, end)
  std::vector<int> child;              // per node: first of its two consecutive children, -1 for a leaf
  std::vector<double> box;             // per node: lo x, y, z, hi x, y, z of its points
  std::vector<int> leaves;             // leaf node ids, in tree order (they tile [0, n))
  std::vector<int> far_ptr, far_node;  // per leaf (CSR): clusters taken through their proxies
  std::vector<int> near_ptr, near_node;  // per leaf (CSR): leaves summed point by point (itself included)
};

// Builds the tree by bisection of each node's longest box side at the median (ties kept in input
// order), down to leaves of at most `leaf` points, then walks it once per leaf from the root: a
// cluster C is accepted for leaf B when it holds more than min_size points and
// r_B + r_C < theta * |c_B - c_C| (r: half the box diagonal, c: the box centre); otherwise a leaf
// cluster joins B's near list and an inner one is opened.  xyz: 3 n doubles (x, y, z per point).
// Returns 0, or 1 for bad arguments (n < 1, leaf < 1, theta not in (0, 1), non-finite coordinates).
int build_tree_plan(const double* xyz, int n, int leaf, double theta, int min_size, TreePlan* out);

}  // namespace pbfb
