"""The C ABI library builds, loads and exports every declared symbol; host-side
validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21713_gb300 import build, pbfb
    build.build()
    return pbfb.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pbfb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pbfb_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2511_21713_gb300 import pbfb
    names = declared_symbols()
    assert len(names) >= 19
    assert sorted(pbfb.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_default_options_are_the_papers(lib):
    from paper_2511_21713_gb300 import pbfb
    o = pbfb.default_opts()
    assert (o.tol_nl, o.tol_gmres, o.tol_gmres0, o.tol_omega, o.L_e) == (1e-3, 1e-6, 1e-3, 0.1, 0.35)
    assert (o.omega0_first, o.omega0_rest, o.omega_max) == (2.0, 1.0, 4.0)
    assert o.n_taylor == 1 and o.taylor[0] == pbfb.T3 and o.method == pbfb.NEWTON and o.R_e == 1.4
    assert o.omega_search == 1 and o.precision == pbfb.FP64 and o.precond == pbfb.BLOCK_DENSE
    assert o.accept_ratio == 1.0          # the global convergence condition ||d(omega)|| < ||d(0)||
    assert o.residual_update == 0.0 and o.residual_far == pbfb.FLOAT2


def _create(lib, xyz, tets, gm, gs):
    h = ctypes.c_void_p()
    xyz = np.ascontiguousarray(xyz, np.float64)
    tets = np.ascontiguousarray(tets, np.int32)
    gm = np.ascontiguousarray(gm, np.int32)
    gs = np.ascontiguousarray(gs, np.int32)
    code = lib.pbfb_mesh_create(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, tets.shape[0],
                                gm.ctypes.data, gm.shape[0], gs.ctypes.data, gs.shape[0], 0, ctypes.byref(h))
    return code, h


def test_mesh_validation_on_host(lib, tiny_case):
    from paper_2511_21713_gb300 import pbfb
    c = tiny_case
    # out-of-range vertex id
    bad = c.tets.copy()
    bad[0, 0] = c.n_v
    code, _ = _create(lib, c.xyz, bad, c.gm_tris, c.gs_tris)
    assert code == 1 and b"out of range" in lib.pbfb_last_error()
    # a missing surface triangle: the boundary is not covered
    code, _ = _create(lib, c.xyz, c.tets, c.gm_tris[1:], c.gs_tris)
    assert code == 1
    # wrong orientation of Gamma_m
    code, _ = _create(lib, c.xyz, c.tets, c.gm_tris[:, [0, 2, 1]], c.gs_tris)
    assert code == 1 and b"orientation" in lib.pbfb_last_error()
    # surfaces swapped: both orientations wrong
    code, _ = _create(lib, c.xyz, c.tets, c.gs_tris, c.gm_tris)
    assert code == 1
    # degenerate tetrahedron
    xyz = c.xyz.copy()
    t0 = c.tets[0]
    xyz[t0[3]] = xyz[t0[0]] + 0.5 * (xyz[t0[1]] - xyz[t0[0]]) + 0.5 * (xyz[t0[2]] - xyz[t0[0]])
    code, _ = _create(lib, xyz, c.tets, c.gm_tris, c.gs_tris)
    assert code == 1
    # NaN coordinate
    xyz = c.xyz.copy()
    xyz[5, 1] = np.nan
    code, _ = _create(lib, xyz, c.tets, c.gm_tris, c.gs_tris)
    assert code == 1 and b"non-finite" in lib.pbfb_last_error()
    assert pbfb.ERRORS[1] == "INVALID"


def _create_full(lib, xyz, tets, region, gm, gs):
    h = ctypes.c_void_p()
    xyz = np.ascontiguousarray(xyz, np.float64)
    tets = np.ascontiguousarray(tets, np.int32)
    region = np.ascontiguousarray(region, np.int32)
    gm = np.ascontiguousarray(gm, np.int32)
    gs = np.ascontiguousarray(gs, np.int32)
    code = lib.pbfb_mesh_create_full(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, tets.shape[0],
                                     region.ctypes.data, gm.ctypes.data, gm.shape[0], gs.ctypes.data,
                                     gs.shape[0], 0, ctypes.byref(h))
    return code, h


def test_full_mesh_validation_on_host(lib, tiny_solute_case):
    import torch
    c = tiny_solute_case
    r = c.tet_region
    # Gamma_m is interior here: as a shell mesh the boundary does not match the surfaces
    code, _ = _create(lib, c.xyz, c.tets, c.gm_tris, c.gs_tris)
    assert code == 1
    bad = r.copy()
    bad[3] = 2
    code, _ = _create_full(lib, c.xyz, c.tets, bad, c.gm_tris, c.gs_tris)
    assert code == 1 and b"region" in lib.pbfb_last_error()
    code, _ = _create_full(lib, c.xyz, c.tets, np.ones_like(r), c.gm_tris, c.gs_tris)
    assert code == 1 and b"both" in lib.pbfb_last_error()
    # Gamma_m pointing into Omega_m, a missing interface triangle, a region flip that moves the
    # interface, and the surfaces swapped
    code, _ = _create_full(lib, c.xyz, c.tets, r, c.gm_tris[:, [0, 2, 1]], c.gs_tris)
    assert code == 1 and b"orientation" in lib.pbfb_last_error()
    code, _ = _create_full(lib, c.xyz, c.tets, r, c.gm_tris[1:], c.gs_tris)
    assert code == 1
    flip = r.copy()
    flip[np.nonzero(r == 0)[0][-1]] = 1
    code, _ = _create_full(lib, c.xyz, c.tets, flip, c.gm_tris, c.gs_tris)
    assert code == 1
    code, _ = _create_full(lib, c.xyz, c.tets, r, c.gs_tris, c.gm_tris)
    assert code == 1
    if not torch.cuda.is_available():
        # the valid mesh passes validation and then needs the GPU: no CPU fallback
        code, h = _create_full(lib, c.xyz, c.tets, r, c.gm_tris, c.gs_tris)
        assert code == 2 and not h.value


def test_valid_mesh_without_gpu_reports_cuda_error(lib, tiny_case):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = tiny_case
    code, h = _create(lib, c.xyz, c.tets, c.gm_tris, c.gs_tris)
    assert code == 2 and not h.value          # PBFB_ERR_CUDA, no handle, no CPU fallback


def test_null_handle_calls_fail_cleanly(lib):
    z = np.zeros(8)
    assert lib.pbfb_apply(None, z.ctypes.data, z.ctypes.data) == 1
    assert lib.pbfb_solve(None, 1.0, 1.0, 0.1, 300.0, None, None, None, None, None) == 1
    assert lib.pbfb_mesh_destroy(None) == 0


def test_ctypes_mirrors_match_the_header(tmp_path):
    """Every struct the binding mirrors has the C header's size and field offsets (a plain C
    program compiled against include/pbfb.h prints them), so arrays of them index alike."""
    import shutil
    import subprocess
    from paper_2511_21713_gb300 import pbfb
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pbfb_newton_opts": pbfb.NewtonOpts, "pbfb_result": pbfb.Result, "pbfb_request": pbfb.Request,
               "pbfb_response": pbfb.Response, "pbfb_tuning": pbfb.Tuning, "pbfb_batch_params": pbfb.BatchParams}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pbfb.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sizes"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_charges_must_lie_strictly_inside_gamma_m(lib, tiny_case):
    """pbfb_check_charges (the host check pbfb_charges_set runs before any GPU work): the winding
    number of the closed Gamma_m is 1 at a point inside, 0 outside and 1/2 on a face, and a charge
    on Gamma_m or outside it is refused with PBFB_ERR_INVALID naming that charge."""
    c = tiny_case
    xyz = np.ascontiguousarray(c.xyz, np.float64)
    gm = np.ascontiguousarray(c.gm_tris, np.int32)

    def check(q):
        q = np.ascontiguousarray(q, np.float64).reshape(-1, 3)
        w = np.full(q.shape[0], np.nan)
        code = lib.pbfb_check_charges(xyz.ctypes.data, xyz.shape[0], gm.ctypes.data, gm.shape[0],
                                      q.ctypes.data, q.shape[0], w.ctypes.data)
        return code, w

    # radius of the largest ball about the centre inside the polyhedron (distance to the face planes)
    P = xyz[gm]
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    r_in = np.abs(np.einsum("ij,ij->i", nrm, P[:, 0]) / np.linalg.norm(nrm, axis=1)).min()
    inside = np.array([[0.0, 0.0, 0.0], [0.5 * r_in, 0.1, -0.2], [0.0, 0.0, 0.999 * r_in]])
    code, w = check(inside)
    assert code == 0 and np.allclose(w, 1.0, atol=1e-12, rtol=0)
    face = xyz[gm[7]].mean(axis=0)                       # the centroid of a Gamma_m triangle
    outside = 0.5 * (c.xyz[c.gs_tris[0, 0]] + face)      # in the shell, between the surfaces
    code, w = check(np.vstack([inside, face, outside]))
    assert code == 1 and b"charge 3" in lib.pbfb_last_error()
    assert abs(w[3] - 0.5) < 1e-12 and abs(w[4]) < 1e-12 and np.allclose(w[:3], 1.0, atol=1e-12, rtol=0)
    code, _ = check(outside)
    assert code == 1 and b"charge 0" in lib.pbfb_last_error()
    # the oracle's seeded workloads all pass
    assert check(c.q_xyz)[0] == 0
    bad = gm.copy()
    bad[0, 0] = xyz.shape[0]
    q = np.zeros(3)
    assert lib.pbfb_check_charges(xyz.ctypes.data, xyz.shape[0], bad.ctypes.data, bad.shape[0],
                                  q.ctypes.data, 1, None) == 1
