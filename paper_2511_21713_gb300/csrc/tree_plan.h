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

// As above, with the split point of a node of m points at the multiple of `granule` nearest to m / 2
// (at least one granule) instead of the median: with granule = leaf every leaf holds exactly `leaf`
// points except the remainders, which fills fixed-size blocks of targets on the GPU.  granule = 1
// is the median split.
int build_tree_plan(const double* xyz, int n, int leaf, double theta, int min_size, int granule, TreePlan* out);

// Work plan of the treecode far field on the GPU, from a TreePlan built with leaf = granule =
// `leaf`: the clusters taken through proxies (numbered in order of first use; proxy records of
// cluster k are npx consecutive source records from n + k npx), and per target leaf its source
// tiles -- runs of at most `tile` consecutive source records: the points of each near leaf (in tree
// order) and the proxies of each accepted cluster -- grouped into chunks of at most
// tiles_per_chunk tiles (one GPU block each).
struct TreeTiles {
  int n = 0, nleaf = 0, nclus = 0;
  double pairs = 0.0;                    // target-source pair evaluations per application
  std::vector<int> perm;                 // tree position -> point index
  std::vector<int> pos_leaf;             // tree position -> leaf
  std::vector<int> leaf_beg, leaf_end;   // per leaf: its targets [beg, end) in tree order
  std::vector<int> leaf_chunk;           // per leaf: its chunks [leaf_chunk[L], leaf_chunk[L + 1])
  std::vector<int> chunk_leaf;           // per chunk: its leaf
  std::vector<int> chunk_tile;           // per chunk: its tiles [chunk_tile[c], chunk_tile[c + 1])
  std::vector<int> tile_start, tile_count;  // per tile: first source record, records (<= tile)
  std::vector<int> clus_beg, clus_end;   // per cluster: its points [beg, end) in tree order
  std::vector<double> clus_box;          // per cluster: lo x, y, z, hi x, y, z (a flat side widened
                                         // to 1e-3 of the longest one)
  // each cluster cut into segments of at most `leaf` consecutive points (the work of an upward pass
  // that sums every cluster from its points; the device pass interpolates leaf proxies instead,
  // one (cluster, leaf) pair per segment when the leaves are full)
  std::vector<int> seg_clus, seg_beg, seg_cnt;  // per segment: cluster, first point, points
  std::vector<int> clus_seg;             // per cluster: its segments [clus_seg[k], clus_seg[k + 1])
};

// Builds the tree plan (leaves and granule `leaf`, clusters accepted with more than npx points)
// and the work plan above.  Returns 0, or 1 for bad arguments.
int plan_tree_tiles(const double* xyz, int n, int leaf, double theta, int npx, int tile, int tiles_per_chunk,
                    TreeTiles* out);

}  // namespace pbfb
