"""Host logic of the treecode plan (paper_2511_21713_gb300/csrc/tree_plan.cu), compiled with the host
C++ compiler and checked on CPU: the tree tiles the points, every leaf's accepted clusters and near
leaves cover every point exactly once, the acceptance criterion holds for every accepted cluster,
the build is deterministic, and bad arguments are refused."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_21713_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include "tree_plan.h"
template <class T> static void put(FILE* f, const std::vector<T>& v) {
  int64_t n = (int64_t)v.size();
  fwrite(&n, sizeof(n), 1, f);
  if (n) fwrite(v.data(), sizeof(T), v.size(), f);
}
int main(int argc, char** argv) {
  int n = atoi(argv[1]), leaf = atoi(argv[2]), min_size = atoi(argv[4]);
  double theta = atof(argv[3]);
  int granule = argc > 7 ? atoi(argv[7]) : 1;
  std::vector<double> xyz(3 * (size_t)n);
  FILE* fi = fopen(argv[5], "rb");
  if (fread(xyz.data(), sizeof(double), xyz.size(), fi) != xyz.size()) return 3;
  fclose(fi);
  pbfb::TreePlan t;
  int st = granule == 1 ? pbfb::build_tree_plan(xyz.data(), n, leaf, theta, min_size, &t)
                        : pbfb::build_tree_plan(xyz.data(), n, leaf, theta, min_size, granule, &t);
  FILE* fo = fopen(argv[6], "wb");
  fwrite(&st, sizeof(st), 1, fo);
  put(fo, t.perm); put(fo, t.begin); put(fo, t.end); put(fo, t.child); put(fo, t.box);
  put(fo, t.leaves); put(fo, t.far_ptr); put(fo, t.far_node); put(fo, t.near_ptr); put(fo, t.near_node);
  fclose(fo);
  return 0;
}
"""

NAMES = ["perm", "begin", "end", "child", "box", "leaves", "far_ptr", "far_node", "near_ptr", "near_node"]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("tree_plan")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-x", "c++", os.path.join(CSRC, "tree_plan.cu"),
                    "-o", str(exe)], check=True)
    return exe, d


def plan(driver, xyz, leaf, theta, min_size, granule=1):
    exe, d = driver
    xyz = np.ascontiguousarray(xyz, np.float64)
    pin, pout = d / "pts.bin", d / "plan.bin"
    xyz.tofile(pin)
    subprocess.run([str(exe), str(len(xyz)), str(leaf), repr(theta), str(min_size), str(pin), str(pout),
                    str(granule)], check=True)
    raw = pout.read_bytes()
    st = struct.unpack_from("i", raw, 0)[0]
    off = 4
    out = {"status": st}
    for name in NAMES:
        (cnt,) = struct.unpack_from("q", raw, off)
        off += 8
        dt = np.float64 if name == "box" else np.int32
        out[name] = np.frombuffer(raw, dt, cnt, off).copy()
        off += cnt * np.dtype(dt).itemsize
    return out


def surface_points(nu=12):
    """Quadrature-like points: the vertices and edge midpoints of a stretched geodesic sphere."""
    from paper_2511_21713_gb300 import inputs
    v, t = inputs.icosphere(nu)
    mid = 0.5 * (v[t[:, 0]] + v[t[:, 1]])
    p = np.concatenate([v, mid]) * np.array([11.0, 11.0, 36.6])
    return p


def check(p, xyz, leaf, theta, min_size, granule=1):
    n = len(xyz)
    assert p["status"] == 0
    perm, begin, end, child = p["perm"], p["begin"], p["end"], p["child"]
    box = p["box"].reshape(-1, 6)
    assert np.array_equal(np.sort(perm), np.arange(n))
    # children: consecutive, splitting the parent's range at its middle; boxes enclose the points
    for k in range(len(begin)):
        pts = xyz[perm[begin[k]:end[k]]]
        assert np.array_equal(box[k, :3], pts.min(0)) and np.array_equal(box[k, 3:], pts.max(0))
        if child[k] >= 0:
            a, b = child[k], child[k] + 1
            assert begin[a] == begin[k] and end[a] == begin[b] and end[b] == end[k]
            m = end[k] - begin[k]
            if granule == 1:
                assert end[a] - begin[a] == m // 2
            else:
                # the multiple of the granule nearest to half (at least one granule, one point right)
                want = min(max(granule, ((m // 2 + granule // 2) // granule) * granule), m - 1)
                assert end[a] - begin[a] == want
        else:
            assert end[k] - begin[k] <= leaf
    leaves = p["leaves"]
    assert np.array_equal(np.concatenate([np.arange(begin[l], end[l]) for l in leaves]), np.arange(n))
    rad = lambda k: 0.5 * np.linalg.norm(box[k, 3:] - box[k, :3])
    cen = lambda k: 0.5 * (box[k, 3:] + box[k, :3])
    fp, fn, np_, nn = p["far_ptr"], p["far_node"], p["near_ptr"], p["near_node"]
    assert len(fp) == len(np_) == len(leaves) + 1
    work = 0
    for i, B in enumerate(leaves):
        cover = np.zeros(n, np.int32)
        for C in fn[fp[i]:fp[i + 1]]:
            assert C != B and end[C] - begin[C] > min_size
            assert rad(B) + rad(C) < theta * np.linalg.norm(cen(B) - cen(C))
            cover[begin[C]:end[C]] += 1
        near = nn[np_[i]:np_[i + 1]]
        assert B in near and all(child[C] < 0 for C in near)
        for C in near:
            cover[begin[C]:end[C]] += 1
            work += (end[B] - begin[B]) * (end[C] - begin[C])
        assert np.all(cover == 1), i
    return work


@pytest.mark.parametrize("leaf,theta", [(64, 0.5), (256, 0.7), (100, 0.6)])
def test_plan_invariants(driver, leaf, theta):
    xyz = surface_points(12)
    p = plan(driver, xyz, leaf, theta, 343)
    check(p, xyz, leaf, theta, 343)


def test_plan_saves_pairs_on_larger_surfaces(driver):
    """17,282 points, leaves of 256, theta 0.7, proxies of 7^3: about a third of the pairs remain
    direct (two thirds at 4,322 points), and the share falls as the surface grows."""
    fr = []
    for nu in (12, 24):
        xyz = surface_points(nu)
        fr.append(check(plan(driver, xyz, 256, 0.7, 343), xyz, 256, 0.7, 343) / len(xyz) ** 2)
    assert fr[1] < 0.4 and fr[1] < 0.6 * fr[0], fr


def test_plan_edge_cases(driver):
    rng = np.random.default_rng(3)
    # one point, fewer points than a leaf, coincident points, ragged sizes
    for xyz in (np.zeros((1, 3)), rng.standard_normal((7, 3)), np.zeros((50, 3)), rng.standard_normal((1001, 3))):
        p = plan(driver, xyz, 16, 0.5, 27)
        check(p, xyz, 16, 0.5, 27)
    xyz = rng.standard_normal((500, 3))
    a, b = plan(driver, xyz, 32, 0.6, 64), plan(driver, xyz, 32, 0.6, 64)
    assert all(np.array_equal(a[k], b[k]) for k in NAMES)
    bad = xyz.copy()
    bad[3, 1] = np.nan
    assert plan(driver, bad, 32, 0.6, 64)["status"] == 1
    assert plan(driver, xyz, 32, 1.0, 64)["status"] == 1
    assert plan(driver, xyz, 0, 0.5, 64)["status"] == 1


def test_granule_split_fills_fixed_size_leaves(driver):
    """Split at multiples of the leaf size: every leaf holds exactly `leaf` points but for the
    remainders (at most one short leaf per right spine here), and the plan keeps its invariants."""
    for nu in (12, 20):
        xyz = surface_points(nu)
        p = plan(driver, xyz, 256, 0.5, 343, granule=256)
        check(p, xyz, 256, 0.5, 343, granule=256)
        sizes = np.array([p["end"][l] - p["begin"][l] for l in p["leaves"]])
        assert (sizes == 256).sum() >= len(sizes) - 2 and sizes.sum() == len(xyz)


TILES_DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include "tree_plan.h"
template <class T> static void put(FILE* f, const std::vector<T>& v) {
  int64_t n = (int64_t)v.size();
  fwrite(&n, sizeof(n), 1, f);
  if (n) fwrite(v.data(), sizeof(T), v.size(), f);
}
int main(int argc, char** argv) {
  int n = atoi(argv[1]), leaf = atoi(argv[2]), npx = atoi(argv[4]), tile = atoi(argv[5]), tpc = atoi(argv[6]);
  double theta = atof(argv[3]);
  std::vector<double> xyz(3 * (size_t)n);
  FILE* fi = fopen(argv[7], "rb");
  if (fread(xyz.data(), sizeof(double), xyz.size(), fi) != xyz.size()) return 3;
  fclose(fi);
  pbfb::TreeTiles t;
  int st = pbfb::plan_tree_tiles(xyz.data(), n, leaf, theta, npx, tile, tpc, &t);
  FILE* fo = fopen(argv[8], "wb");
  fwrite(&st, sizeof(st), 1, fo);
  fwrite(&t.nclus, sizeof(int), 1, fo);
  fwrite(&t.pairs, sizeof(double), 1, fo);
  put(fo, t.perm); put(fo, t.pos_leaf); put(fo, t.leaf_beg); put(fo, t.leaf_end); put(fo, t.leaf_chunk);
  put(fo, t.chunk_leaf); put(fo, t.chunk_tile); put(fo, t.tile_start); put(fo, t.tile_count);
  put(fo, t.clus_beg); put(fo, t.clus_end); put(fo, t.clus_box);
  put(fo, t.seg_clus); put(fo, t.seg_beg); put(fo, t.seg_cnt); put(fo, t.clus_seg);
  fclose(fo);
  return 0;
}
"""

TILE_NAMES = ["perm", "pos_leaf", "leaf_beg", "leaf_end", "leaf_chunk", "chunk_leaf", "chunk_tile",
              "tile_start", "tile_count", "clus_beg", "clus_end", "clus_box", "seg_clus", "seg_beg", "seg_cnt",
              "clus_seg"]


@pytest.fixture(scope="module")
def tiles_driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("tree_tiles")
    src = d / "tiles.cpp"
    src.write_text(TILES_DRIVER)
    exe = d / "tiles"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-x", "c++", os.path.join(CSRC, "tree_plan.cu"),
                    "-o", str(exe)], check=True)
    return exe, d


def tiles_plan(drv, xyz, leaf=256, theta=0.5, npx=343, tile=128, tpc=8):
    exe, d = drv
    xyz = np.ascontiguousarray(xyz, np.float64)
    pin, pout = d / "pts.bin", d / "tiles.bin"
    xyz.tofile(pin)
    subprocess.run([str(exe), str(len(xyz)), str(leaf), repr(theta), str(npx), str(tile), str(tpc), str(pin),
                    str(pout)], check=True)
    raw = pout.read_bytes()
    st, nclus = struct.unpack_from("ii", raw, 0)
    (pairs,) = struct.unpack_from("d", raw, 8)
    off = 16
    out = {"status": st, "nclus": nclus, "pairs": pairs}
    for name in TILE_NAMES:
        (cnt,) = struct.unpack_from("q", raw, off)
        off += 8
        dt = np.float64 if name == "clus_box" else np.int32
        out[name] = np.frombuffer(raw, dt, cnt, off).copy()
        off += cnt * np.dtype(dt).itemsize
    return out


def quadrature_like_points(nu, a=12.0):
    """Six interior points per triangle of a radius-a geodesic sphere (as the surface quadrature)."""
    from paper_2511_21713_gb300 import inputs
    v, t = inputs.icosphere(nu)
    v = a * v / np.linalg.norm(v, axis=1, keepdims=True)
    bary = np.array([[0.66, 0.17, 0.17], [0.17, 0.66, 0.17], [0.17, 0.17, 0.66],
                     [0.1, 0.45, 0.45], [0.45, 0.1, 0.45], [0.45, 0.45, 0.1]])
    return np.einsum("qa,tad->tqd", bary, v[t]).reshape(-1, 3)


@pytest.mark.parametrize("nu", [8, 20])
def test_tree_tiles_plan_bounds_and_coverage(tiles_driver, nu):
    """Every index the treecode kernels read stays inside the buffers they are given, and each
    leaf's tiles cover every point exactly once, directly or through its clusters' proxies: perm a
    permutation; leaves of at most 256 consecutive tree positions tiling [0, n); each leaf one or more
    chunks, each chunk at most 8 tiles of 1..128 records within [0, n + nclus * 343); a proxy tile
    inside one cluster's block of 343 records; cluster boxes enclosing their points."""
    xyz = quadrature_like_points(nu)
    n = len(xyz)
    p = tiles_plan(tiles_driver, xyz)
    assert p["status"] == 0
    perm, pos_leaf = p["perm"], p["pos_leaf"]
    lb, le, lc = p["leaf_beg"], p["leaf_end"], p["leaf_chunk"]
    cl, ct, ts, tc = p["chunk_leaf"], p["chunk_tile"], p["tile_start"], p["tile_count"]
    cb, ce, box = p["clus_beg"], p["clus_end"], p["clus_box"].reshape(-1, 6)
    nclus, npx = p["nclus"], 343
    assert np.array_equal(np.sort(perm), np.arange(n))
    nleaf = len(lb)
    assert lb[0] == 0 and le[-1] == n and np.array_equal(lb[1:], le[:-1])
    assert np.all(le - lb >= 1) and np.all(le - lb <= 256)
    assert np.array_equal(pos_leaf, np.repeat(np.arange(nleaf), le - lb))
    assert len(lc) == nleaf + 1 and lc[0] == 0 and np.all(np.diff(lc) >= 1) and lc[-1] == len(cl)
    assert np.array_equal(cl, np.repeat(np.arange(nleaf), np.diff(lc)))
    assert len(ct) == len(cl) + 1 and ct[0] == 0 and ct[-1] == len(ts)
    assert np.all(np.diff(ct) >= 1) and np.all(np.diff(ct) <= 8)
    assert np.all(tc >= 1) and np.all(tc <= 128)
    assert np.all(ts >= 0) and np.all(ts + tc <= n + nclus * npx)
    assert len(cb) == len(ce) == nclus and np.all(ce - cb > npx) and np.all(cb >= 0) and np.all(ce <= n)
    for k in range(nclus):
        pts = xyz[perm[cb[k]:ce[k]]]
        assert np.all(pts >= box[k, :3] - 1e-12) and np.all(pts <= box[k, 3:] + 1e-12)
    # upward-pass segments: each cluster's points in consecutive runs of at most 256
    sc, sb, sn, cs = p["seg_clus"], p["seg_beg"], p["seg_cnt"], p["clus_seg"]
    assert len(cs) == nclus + 1 and cs[0] == 0 and cs[-1] == len(sb) == len(sc) == len(sn)
    assert np.all(sn >= 1) and np.all(sn <= 256)
    for k in range(nclus):
        g = np.arange(cs[k], cs[k + 1])
        assert np.all(sc[g] == k) and sb[g[0]] == cb[k] and sb[g[-1]] + sn[g[-1]] == ce[k]
        assert np.array_equal(sb[g[1:]], sb[g[:-1]] + sn[g[:-1]])
    pairs = 0.0
    for L in range(nleaf):
        cover = np.zeros(n, np.int32)
        for c in range(lc[L], lc[L + 1]):
            for t in range(ct[c], ct[c + 1]):
                s0, cnt = ts[t], tc[t]
                pairs += (le[L] - lb[L]) * cnt
                if s0 < n:
                    assert s0 + cnt <= n
                    cover[s0:s0 + cnt] += 1
                else:
                    k = (s0 - n) // npx
                    assert s0 + cnt <= n + (k + 1) * npx
                    if (s0 - n) % npx == 0:
                        cover[cb[k]:ce[k]] += 1
        assert np.all(cover == 1), L
    assert abs(pairs - p["pairs"]) < 1e-6 * pairs
    if nu == 20:
        # the bench-sized surface: proxies replace a good share of the direct pairs
        assert nclus > 0 and p["pairs"] < 0.7 * n * n


def test_proxy_tiles_well_separated_from_their_leaf(tiles_driver):
    """The evaluation kernel forms r^2 on proxy tiles as |t'|^2 + |y'|^2 - 2 t'.y' about the centre
    of the target leaf's box, which is accurate only while every proxy stays well away from every
    target of the leaf: with the acceptance rule r_B + r_C < theta D the targets lie within theta D
    of the leaf centre, the proxies (tensor Chebyshev points of the cluster box, corners included)
    within (1 + theta) D, and each target-proxy distance exceeds (1 - theta) D, so
    (|t'| + |y'|) / |t - y| < (1 + 2 theta) / (1 - theta).  Checked point by point on the bench-sized
    surface at theta = 0.6 (the kernel's), with the leaf boxes widened as the device plan widens them."""
    theta = 0.6
    xyz = quadrature_like_points(20)
    n = len(xyz)
    p = tiles_plan(tiles_driver, xyz, theta=theta)
    assert p["status"] == 0 and p["nclus"] > 0
    perm, lb, le, lc = p["perm"], p["leaf_beg"], p["leaf_end"], p["leaf_chunk"]
    ct, ts, tc = p["chunk_tile"], p["tile_start"], p["tile_count"]
    box = p["clus_box"].reshape(-1, 6)
    cheb = np.cos(np.pi * np.arange(7) / 6)
    worst = 0.0
    ntile = 0
    for L in range(len(lb)):
        t = xyz[perm[lb[L]:le[L]]]
        lo, hi = t.min(0), t.max(0)
        pad = np.maximum(0.0, 1e-3 * (hi - lo).max() - (hi - lo)) * 0.5
        c = 0.5 * ((lo - pad) + (hi + pad))
        for ch in range(lc[L], lc[L + 1]):
            for k in range(ct[ch], ct[ch + 1]):
                if ts[k] < n:
                    continue
                ntile += 1
                C = (ts[k] - n) // 343
                bl, bh = box[C, :3], box[C, 3:]
                g = [0.5 * (bl[d] + bh[d]) + 0.5 * (bh[d] - bl[d]) * cheb for d in range(3)]
                y = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
                y = y[(ts[k] - n) % 343:(ts[k] - n) % 343 + tc[k]]
                r = np.linalg.norm(t[:, None, :] - y[None, :, :], axis=2)
                ratio = (np.linalg.norm(t - c, axis=1)[:, None] + np.linalg.norm(y - c, axis=1)[None, :]) / r
                worst = max(worst, ratio.max())
    assert ntile > 0
    assert worst < (1 + 2 * theta) / (1 - theta), worst
