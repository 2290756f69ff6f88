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
  std::vector<double> xyz(3 * (size_t)n);
  FILE* fi = fopen(argv[5], "rb");
  if (fread(xyz.data(), sizeof(double), xyz.size(), fi) != xyz.size()) return 3;
  fclose(fi);
  pbfb::TreePlan t;
  int st = pbfb::build_tree_plan(xyz.data(), n, leaf, theta, min_size, &t);
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


def plan(driver, xyz, leaf, theta, min_size):
    exe, d = driver
    xyz = np.ascontiguousarray(xyz, np.float64)
    pin, pout = d / "pts.bin", d / "plan.bin"
    xyz.tofile(pin)
    subprocess.run([str(exe), str(len(xyz)), str(leaf), repr(theta), str(min_size), str(pin), str(pout)], check=True)
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


def check(p, xyz, leaf, theta, min_size):
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
            assert end[a] - begin[a] == (end[k] - begin[k]) // 2
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
