"""Parity on the synthetic double helix at full size (24 base pairs, 40,500 triangles per
surface, 344,284 vertices, 1,944,000 tets, 1548 charges, 0.15 M), where the oracle can only
compute rows one by one:

* boundary-operator rows of sampled vertices (float64 and float-float far field), 1e-11;
* every FEM row of A + J and the load N, 1e-12;
* the mixed-precision solve: its nonlinear residual d = b - Acal(0) Phi - N(Phi), evaluated by the
  oracle on every FEM row and on the sampled boundary rows, is small against the right-hand side,
  and the energy terms are consistent.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


@pytest.fixture(scope="module")
def helix():
    from paper_2511_21713_gb300 import inputs, pbfb
    case = inputs.double_helix()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    yield case, m
    m.close()


@pytest.fixture(scope="module")
def sampled_rows(helix):
    """Complete oracle rows (V, K) of 10 sampled vertices per surface."""
    from oracle import bem
    case, _ = helix
    out = {}
    for name, tris, kap in (("m", case.gm_tris, 0.0), ("s", case.gs_tris, case.kappa)):
        s = bem.Surface(case.xyz, tris)
        rows = np.sort(np.random.default_rng(31).choice(s.n, 10, replace=False))
        tt = np.unique(np.nonzero(np.isin(s.tl, rows).any(axis=1))[0])
        V, K = bem.assemble(s, kap, test_tris=tt)
        out[name] = (s, rows, V[rows], K[rows], kap)
        del V, K
    return out


def test_helix_realised_sizes(helix):
    case, m = helix
    assert (case.n_v, case.n_t) == (344284, 1944000)
    assert (m.n_m, m.n_s) == (20252, 20252) and len(case.q_z) == 1548
    assert abs(case.q_z.sum() + 48.0) < 1e-9


@pytest.mark.parametrize("precision,treecode", [(0, 0), (2, 0), (1, 2)])
def test_helix_boundary_operator_rows(helix, sampled_rows, precision, treecode):
    """float64 and float-float 1e-11 of the largest entry; the float32 treecode (built in at this
    size: 243,000 points per surface) 3e-6."""
    from paper_2511_21713_gb300 import pbfb
    case, m = helix
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    base = m.get_tuning()
    m.apply_tuning(dict(base, treecode=treecode))
    tol = 3e-6 if precision == pbfb.MIXED else 1e-11
    try:
        _helix_rows(case, m, sampled_rows, tol)
    finally:
        m.apply_tuning(base)


def _helix_rows(case, m, sampled_rows, tol):
    from paper_2511_21713_gb300 import pbfb
    rng = np.random.default_rng(7)
    for which, key in ((pbfb.GAMMA_M, "m"), (pbfb.GAMMA_S, "s")):
        s, rows, Vr, Kr, _ = sampled_rows[key]
        x = rng.standard_normal(s.n) + 1.0
        for op, Mr in ((0, Vr), (1, Kr)):
            y = dev(np.zeros(s.n))
            m.bem_apply(which, op, dev(x), y)
            ref = Mr @ x
            got = y.cpu().numpy()[rows]
            assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (which, op)


def test_helix_fem_rows_and_load(helix):
    from paper_2511_21713_gb300 import pbfb
    from oracle import fem
    case, m = helix
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.MIXED)
    r = np.linalg.norm(case.xyz, axis=1)
    u = 8.0 * np.exp(-0.2 * (r - r.min())) * np.cos(0.3 * case.xyz[:, 2])
    N = dev(np.zeros(case.n_v))
    m.assemble(pbfb.HS, dev(u), N)
    rp, col, val = m.fem_rows()
    coef = case.eps_out * case.kappa ** 2
    A = fem.stiffness(case.xyz, case.tets, case.eps_out) + fem.jacobian(case.xyz, case.tets, u, "HS", coef)
    G = sp.csr_matrix((val, col, rp), shape=(case.n_v, m.n))[:, :case.n_v]
    assert abs(G - A).max() <= 1e-12 * abs(A).max()
    Nref = fem.nonlinear_load(case.xyz, case.tets, u, "HS", coef)
    assert np.linalg.norm(N.cpu().numpy() - Nref) < 1e-13 * np.linalg.norm(Nref)


def test_helix_mixed_solve_residual(helix, sampled_rows):
    """Mixed solve (Newton to Tol_NL = 1e-8): the oracle's residual rows of the solution."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import bem, fem
    case, m = helix
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                     pbfb.default_opts(precision=pbfb.MIXED, tol_nl=1e-8))
    assert res["status"] == 0 and res["NC"] < 0 and res["dG_ion"] > 0
    assert abs(res["total"] - (res["LC"] + res["NC"] + res["dG_ion"])) < 1e-12 * abs(res["total"])
    nv = case.n_v
    sm, ss = sampled_rows["m"][0], sampled_rows["s"][0]
    u, lm, ls = x[:nv], x[nv:nv + sm.n], x[nv + sm.n:]
    assert np.array_equal(m.surface_vertices(pbfb.GAMMA_M), sm.verts)
    # FEM rows: 0 - (A u + N(u) + eps_m Rm^T Mm lam_m - eps_s Rs^T Ms lam_s)
    coef = case.eps_out * case.kappa ** 2
    Mm, Ms = bem.mass_matrix(sm), bem.mass_matrix(ss)
    yu = fem.stiffness(case.xyz, case.tets, case.eps_out) @ u + fem.nonlinear_load(case.xyz, case.tets, u, "HS", coef)
    np.add.at(yu, sm.verts, case.eps_in * (Mm @ lm))
    np.add.at(yu, ss.verts, -case.eps_out * (Ms @ ls))
    # boundary rows of the sampled vertices
    lB = 332.0637 / (0.0019872043 * case.T)
    _, rows_m, Vm, Km, _ = sampled_rows["m"]
    # Coulomb right-hand side of the sampled Gamma_m rows: the oracle's rule on the triangles
    # incident to them (the full surface's point-charge table would take 9 GB)
    tt = np.unique(np.nonzero(np.isin(sm.tl, rows_m).any(axis=1))[0])
    sub = bem.Surface(case.xyz, case.gm_tris[tt])
    bsub = (lB / case.eps_in) * bem.coulomb_rhs(sub, case.q_xyz, case.q_z)
    bm_rows = bsub[np.searchsorted(sub.verts, sm.verts[rows_m])]
    _, rows_s, Vs, Ks, _ = sampled_rows["s"]
    um, us = u[sm.verts], u[ss.verts]
    dm = bm_rows - (0.5 * (Mm @ um)[rows_m] + Km @ um - Vm @ lm)
    ds = -(0.5 * (Ms @ us)[rows_s] - Ks @ us + Vs @ ls)
    scale = np.abs(bm_rows).max()
    print("helix residual / max|b|: FEM rows %.3e, Gamma_m rows %.3e, Gamma_s rows %.3e; Newton %d, GMRES %s"
          % (np.abs(yu).max() / scale, np.abs(dm).max() / scale, np.abs(ds).max() / scale,
             res["newton_iters"], res["gmres"]))
    assert np.abs(yu).max() < 1e-10 * scale
    assert np.abs(dm).max() < 1e-10 * scale and np.abs(ds).max() < 1e-10 * scale
