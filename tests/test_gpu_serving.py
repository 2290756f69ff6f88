"""Serving and batching through the C ABI: results are identical alone and in the mix,
admission respects the HBM budget, failures stay local (GPU)."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mix():
    """Seeded spheres of three sizes with different charges, salt and dielectrics."""
    from paper_2511_21713_gb300 import inputs
    cases = []
    for i, (nu, layers) in enumerate([(3, 5), (4, 6), (5, 8), (3, 4), (4, 5), (6, 8)]):
        q, z = inputs.ball_charges(1 + 3 * i, 3.0, (1 + 3 * i) // 2 + 1, 100 + i)
        c = inputs.sphere_case(nu=nu, a=4.0, R=9.0, layers=layers, q_xyz=q, q_z=z,
                               eps_in=(2.0, 4.0)[i % 2], eps_out=80.0, ionic=(0.05, 0.15, 0.5)[i % 3],
                               name=f"mix{i}")
        cases.append(c)
    return cases


def _collect(sv, n, timeout_s=300):
    out, t0 = {}, time.time()
    while len(out) < n and time.time() - t0 < timeout_s:
        for r in sv.poll(64, 200000):
            out[r["id"]] = r
    assert len(out) == n
    return out


def test_results_identical_alone_and_in_the_mix():
    from paper_2511_21713_gb300 import pbfb
    cases = _mix()
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=4)
    for i, c in enumerate(cases):
        sv.submit(c, i)
    mixed = _collect(sv, len(cases))
    assert sv.stats()["completed"] == len(cases)
    sv.close()
    for i, c in enumerate(cases):
        alone = pbfb.Server(budget_bytes=8 << 30, max_inflight=1)
        alone.submit(c, 0)
        a = _collect(alone, 1)[0]
        alone.close()
        r = mixed[i]
        assert r["status"] == 0 and a["status"] == 0
        assert r["total"] == a["total"] and r["gmres"] == a["gmres"] and r["omega"] == a["omega"]
    # and, at tight tolerances, the same solution as the single-solve entry point (which takes the
    # cooperative inner PCG: another rounding of the same preconditioner)
    tight = pbfb.default_opts(tol_gmres0=1e-11, tol_gmres=1e-11, tol_nl=1e-9)
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=3)
    for i, c in enumerate(cases):
        sv.submit(c, i, opts=tight)
    tres = _collect(sv, len(cases))
    sv.close()
    for i, c in enumerate(cases):
        m = pbfb.Mesh.from_case(c)
        m.charges_set(c.q_xyz, c.q_z)
        _, s = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, tight)
        m.close()
        assert tres[i]["status"] == 0
        assert abs(s["total"] - tres[i]["total"]) < 1e-9 * abs(s["total"])


def test_budget_admission_and_failures():
    from paper_2511_21713_gb300 import pbfb
    cases = _mix()[:3]
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=3)
    # a request larger than the whole budget is refused at submission
    small = pbfb.Server(budget_bytes=1 << 20, max_inflight=1)
    with pytest.raises(pbfb.PbfbError) as e:
        small.submit(cases[0], 0)
    assert e.value.code == 7
    small.close()
    # a failing request (no charges inside: NaN charge) reports its error; the others complete
    bad = cases[1]
    import dataclasses
    bad = dataclasses.replace(bad, q_z=np.array([np.nan] * bad.q_z.size))
    sv.submit(cases[0], 0)
    sv.submit(bad, 1)
    sv.submit(cases[2], 2)
    out = _collect(sv, 3)
    assert out[0]["status"] == 0 and out[2]["status"] == 0 and out[1]["status"] == 1
    assert "non-finite" in out[1]["error"]
    sv.close()


def test_tight_budget_serialises_but_completes():
    from paper_2511_21713_gb300 import pbfb
    cases = _mix()[:4]
    # a budget below any request refuses them
    sv = pbfb.Server(budget_bytes=1, max_inflight=4)
    with pytest.raises(pbfb.PbfbError):
        sv.submit(cases[0], 0)
    sv.close()
    est = 150 << 20   # each of these small requests is estimated near 70 MB: about two fit at once
    sv = pbfb.Server(budget_bytes=est, max_inflight=4)
    for i, c in enumerate(cases):
        sv.submit(c, i)
    out = _collect(sv, 4)
    st = sv.stats()
    sv.close()
    assert all(r["status"] == 0 for r in out.values())
    assert st["peak"] <= est
    # admitted in arrival order
    starts = [out[i]["t_start_ms"] for i in range(4)]
    assert starts == sorted(starts)


def test_solve_batch_matches_individual_solves():
    import torch
    from paper_2511_21713_gb300 import pbfb
    cases = _mix()[:4]
    streams = [torch.cuda.Stream() for _ in cases]
    meshes = []
    for c, s in zip(cases, streams):
        m = pbfb.Mesh.from_case(c, stream=s.cuda_stream)
        m.charges_set(c.q_xyz, c.q_z)
        meshes.append(m)
    res = pbfb.solve_batch(meshes, [(c.eps_in, c.eps_out, c.kappa, c.T, None) for c in cases], 4)
    # the batch results equal a sequential batch of one (same kernels, same path)
    for c, m, r in zip(cases, meshes, res):
        r1 = pbfb.solve_batch([m], [(c.eps_in, c.eps_out, c.kappa, c.T, None)], 1)[0]
        assert r["status"] == 0 and r1["total"] == r["total"] and r1["gmres"] == r["gmres"]
        m.close()


def test_resident_meshes_reused_with_identical_results():
    """A server that keeps meshes resident serves repeated geometries without rebuilding them;
    every result equals the one of a server that builds each mesh afresh."""
    from paper_2511_21713_gb300 import inputs, pbfb
    base = _mix()
    cases = []
    for k in range(8):                      # three geometries, new charges and salt each time
        c = base[k % 3]
        q, z = inputs.ball_charges(2 + k, 3.0, 1 + k // 2, 500 + k)
        cases.append(inputs.Case(f"rep{k}", c.xyz, c.tets, c.gm_tris, c.gs_tris, q, z, c.eps_in,
                                 c.eps_out, inputs.kappa_from_ionic_strength((0.05, 0.3)[k % 2], 80.0, 300.0),
                                 c.T))
    fresh = pbfb.Server(budget_bytes=8 << 30, max_inflight=2)
    for i, c in enumerate(cases):
        fresh.submit(c, i)
    ref = _collect(fresh, len(cases))
    fresh.close()
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=2, cached_meshes=2)
    for i, c in enumerate(cases):
        sv.submit(c, i)
    got = _collect(sv, len(cases))
    st = sv.stats()
    sv.close()
    assert st["mesh_hits"] >= 3 and st["resident_meshes"] <= 2
    for i in range(len(cases)):
        assert got[i]["status"] == 0
        assert got[i]["total"] == ref[i]["total"] and got[i]["gmres"] == ref[i]["gmres"]
    # a budget of about two meshes: resident meshes are evicted to admit new geometries
    sv = pbfb.Server(budget_bytes=150 << 20, max_inflight=2, cached_meshes=8)
    for i, c in enumerate(cases):
        sv.submit(c, i)
    got = _collect(sv, len(cases))
    st = sv.stats()
    sv.close()
    assert all(got[i]["status"] == 0 and got[i]["total"] == ref[i]["total"] for i in range(len(cases)))
    assert st["peak"] <= 150 << 20


def test_meshes_of_omega_m_and_omega_i_served_and_batched():
    """Requests carrying tet regions are built as meshes of Omega_m and Omega_i (the paper's own
    formulation) and give the single-solve entry point's result; so does pbfb_solve_batch."""
    import torch
    from paper_2511_21713_gb300 import inputs, pbfb
    cases = []
    for i in range(3):
        q, z = inputs.ball_charges(2 + 2 * i, 3.0, 1 + i, 700 + i)
        cases.append(inputs.solute_sphere_case(nu=3 + i % 2, layers=5, core_layers=6, q_xyz=q, q_z=z,
                                               ionic=(0.05, 0.15, 0.5)[i], name=f"solute{i}"))
    tight = pbfb.default_opts(tol_gmres0=1e-11, tol_gmres=1e-11, tol_nl=1e-8)
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=3, cached_meshes=4)
    for i, c in enumerate(cases):
        sv.submit(c, i, opts=tight)
    got = _collect(sv, len(cases))
    sv.submit(cases[0], len(cases), opts=tight)          # served on the resident mesh
    got.update(_collect(sv, 1))
    st = sv.stats()
    sv.close()
    assert st["mesh_hits"] == 1
    streams = [torch.cuda.Stream() for _ in cases]
    meshes = []
    for c, s in zip(cases, streams):
        m = pbfb.Mesh.from_case(c, stream=s.cuda_stream)
        m.charges_set(c.q_xyz, c.q_z)
        meshes.append(m)
    batch = pbfb.solve_batch(meshes, [(c.eps_in, c.eps_out, c.kappa, c.T, tight) for c in cases], 3)
    for m in meshes:
        m.close()
    for i, c in enumerate(cases):
        m = pbfb.Mesh.from_case(c)
        assert m.full
        m.charges_set(c.q_xyz, c.q_z)
        _, s = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, tight)
        m.close()
        for r in (got[i], batch[i]):
            assert r["status"] == 0 and abs(r["total"] - s["total"]) < 1e-9 * abs(s["total"])
    assert got[len(cases)]["total"] == got[0]["total"]


def test_poll_times_out_without_a_response():
    """pbfb_server_poll's bounded wait: with nothing submitted a 20 ms wait ends with
    PBFB_ERR_TIMEOUT and no response; the server then serves a request normally."""
    import ctypes
    from paper_2511_21713_gb300 import pbfb
    sv = pbfb.Server(budget_bytes=8 << 30, max_inflight=1)
    buf = (pbfb.Response * 4)()
    n = ctypes.c_int(-1)
    t0 = time.time()
    code = pbfb.load().pbfb_server_poll(sv.h, buf, 4, 20000, ctypes.byref(n))
    assert code == pbfb.ERR_TIMEOUT and n.value == 0 and time.time() - t0 >= 0.015
    assert b"no response" in pbfb.load().pbfb_last_error()
    assert pbfb.load().pbfb_server_poll(sv.h, buf, 4, 0, ctypes.byref(n)) == 0 and n.value == 0
    c = _mix()[0]
    sv.submit(c, 7)
    r = _collect(sv, 1)[7]
    assert r["status"] == 0
    sv.close()
