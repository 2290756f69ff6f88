// Host plan of the treecode far field (see tree_plan.h).  No device code: the file builds with
// nvcc into the library and with a plain C++ compiler in the host tests.
#include "tree_plan.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
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
  return build_tree_plan(xyz, n, leaf, theta, min_size, 1, out);
}

int build_tree_plan(const double* xyz, int n, int leaf, double theta, int min_size, int granule, TreePlan* out) {
  if (!xyz || !out || n < 1 || leaf < 1 || granule < 1 || !(theta > 0.0 && theta < 1.0)) return 1;
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
    int half = (e - b) / 2;
    if (granule > 1) half = std::max(granule, (int)(((int64_t)half + granule / 2) / granule) * granule);
    const int mid = b + std::min(half, e - b - 1);
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

int plan_tree_tiles(const double* xyz, int n, int leaf, double theta, int npx, int tile, int tiles_per_chunk,
                    TreeTiles* out) {
  if (!out || tile < 1 || tiles_per_chunk < 1 || npx < 1) return 1;
  TreePlan P;
  if (build_tree_plan(xyz, n, leaf, theta, npx, leaf, &P)) return 1;
  TreeTiles& T = *out;
  T = TreeTiles();
  T.n = n;
  T.nleaf = (int)P.leaves.size();
  T.perm = P.perm;
  std::vector<int> cidx(P.begin.size(), -1), cnode;
  for (int C : P.far_node)
    if (cidx[C] < 0) {
      cidx[C] = (int)cnode.size();
      cnode.push_back(C);
    }
  T.nclus = (int)cnode.size();
  T.clus_seg.assign(1, 0);
  for (int C : cnode) {
    T.clus_beg.push_back(P.begin[C]);
    T.clus_end.push_back(P.end[C]);
    for (int b = P.begin[C]; b < P.end[C]; b += leaf) {
      T.seg_clus.push_back((int)T.clus_seg.size() - 1);
      T.seg_beg.push_back(b);
      T.seg_cnt.push_back(std::min(leaf, P.end[C] - b));
    }
    T.clus_seg.push_back((int)T.seg_beg.size());
    const double* bx = &P.box[6 * (size_t)C];
    double side = 0.0;
    for (int d = 0; d < 3; ++d) side = std::max(side, bx[3 + d] - bx[d]);
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      const double pad = std::max(0.0, 1e-3 * side - (bx[3 + d] - bx[d])) * 0.5;
      lo[d] = bx[d] - pad;
      hi[d] = bx[3 + d] + pad;
    }
    T.clus_box.insert(T.clus_box.end(), {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]});
  }
  T.pos_leaf.assign(n, 0);
  T.chunk_tile.assign(1, 0);
  T.leaf_chunk.assign(1, 0);
  for (int i = 0; i < T.nleaf; ++i) {
    const int B = P.leaves[i];
    T.leaf_beg.push_back(P.begin[B]);
    T.leaf_end.push_back(P.end[B]);
    for (int q = P.begin[B]; q < P.end[B]; ++q) T.pos_leaf[q] = i;
    const int nt_leaf = P.end[B] - P.begin[B];
    std::vector<int> ls, lc;
    auto add_range = [&](int b, int e) {
      for (int s0 = b; s0 < e; s0 += tile) {
        ls.push_back(s0);
        lc.push_back(std::min(tile, e - s0));
      }
      T.pairs += (double)nt_leaf * (e - b);
    };
    for (int k = P.near_ptr[i]; k < P.near_ptr[i + 1]; ++k) add_range(P.begin[P.near_node[k]], P.end[P.near_node[k]]);
    for (int k = P.far_ptr[i]; k < P.far_ptr[i + 1]; ++k) {
      const int o = n + cidx[P.far_node[k]] * npx;
      add_range(o, o + npx);
    }
    for (size_t t0 = 0; t0 < ls.size(); t0 += tiles_per_chunk) {
      T.chunk_leaf.push_back(i);
      for (size_t t = t0; t < std::min(ls.size(), t0 + (size_t)tiles_per_chunk); ++t) {
        T.tile_start.push_back(ls[t]);
        T.tile_count.push_back(lc[t]);
      }
      T.chunk_tile.push_back((int)T.tile_start.size());
    }
    T.leaf_chunk.push_back((int)T.chunk_leaf.size());
  }
  return 0;
}

}  // namespace pbfb
