"""Parity of the paper's own formulation at the bench's size (the multi-charge sphere meshed inside
Gamma_m as well: 168,085 vertices, 992,000 tets of which 584,000 in Omega_m, 8000 + 8000
triangles, 200 charges), where the oracle computes rows one by one:

* every FEM row of A~ + J and the load N against the oracle's sparse assembly, 1e-12;
* the mixed-precision solve (Newton to Tol_NL = 1e-7): the oracle's residual of Eq. fembem_matrix on
  every FEM row and on sampled Gamma_s rows, and of the Gamma_m equation of Sec. 2.3.1 (which fills
  lam_m) on sampled Gamma_m rows, small against the right-hand side; the energy terms consistent.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


@pytest.fixture(scope="module")
def big():
    from paper_2511_21713_gb300 import inputs, pbfb
    case = inputs.multi_charge_solute_sphere()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    yield case, m
    m.close()


def _sampled_rows(s, kappa, k=10, seed=41):
    """Rows (V, K) of k sampled vertices of surface s (the oracle assembles only their triangles)."""
    from oracle import bem
    rows = np.sort(np.random.default_rng(seed).choice(s.n, k, replace=False))
    tt = np.unique(np.nonzero(np.isin(s.tl, rows).any(axis=1))[0])
    V, K = bem.assemble(s, kappa, test_tris=tt)
    return rows, tt, V[rows], K[rows]


def test_fem_rows_and_load(big):
    from paper_2511_21713_gb300 import pbfb
    from oracle import fem
    case, m = big
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.MIXED)
    r = np.linalg.norm(case.xyz, axis=1)
    u = 6.0 * np.exp(-0.2 * np.abs(r - 12.0)) * np.cos(0.3 * case.xyz[:, 2])
    N = dev(np.zeros(case.n_v))
    m.assemble(pbfb.HS, dev(u), N)
    rp, col, val = m.fem_rows()
    ti, tm = case.tets[case.tet_region == 1], case.tets[case.tet_region == 0]
    coef = case.eps_out * case.kappa ** 2
    A = (fem.stiffness(case.xyz, ti, case.eps_out) + fem.stiffness(case.xyz, tm, case.eps_in)
         + fem.jacobian(case.xyz, ti, u, "HS", coef))
    G = sp.csr_matrix((val, col, rp), shape=(case.n_v, m.n))[:, :case.n_v]
    assert abs(G - A).max() <= 1e-12 * abs(A).max()
    Nref = fem.nonlinear_load(case.xyz, ti, u, "HS", coef)
    assert np.linalg.norm(N.cpu().numpy() - Nref) < 1e-13 * np.linalg.norm(Nref)
    m.clear_jacobian()


def test_mixed_solve_residual(big):
    from paper_2511_21713_gb300 import pbfb
    from oracle import bem, fem, solute
    from oracle.pb import COULOMB, KB
    case, m = big
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                     pbfb.default_opts(precision=pbfb.MIXED, tol_nl=1e-7))
    assert res["status"] == 0 and res["NC"] < 0 and res["dG_ion"] > 0
    assert abs(res["total"] - (res["LC"] + res["NC"] + res["dG_ion"])) < 1e-12 * abs(res["total"])
    nv = case.n_v
    sm, ss = bem.Surface(case.xyz, case.gm_tris), bem.Surface(case.xyz, case.gs_tris)
    u, lm, ls = x[:nv], x[nv:nv + sm.n], x[nv + sm.n:]
    lB = COULOMB / (KB * case.T)
    ti, tm = case.tets[case.tet_region == 1], case.tets[case.tet_region == 0]
    coef = case.eps_out * case.kappa ** 2
    # FEM rows: rho - (A~ u + N(u) - eps_s R_s^T M_s lam_s)
    rho = 4.0 * np.pi * lB * solute.point_load(case.xyz, tm, case.q_xyz, case.q_z)
    Ms, Mm = bem.mass_matrix(ss), bem.mass_matrix(sm)
    yu = (fem.stiffness(case.xyz, ti, case.eps_out) @ u + fem.stiffness(case.xyz, tm, case.eps_in) @ u
          + fem.nonlinear_load(case.xyz, ti, u, "HS", coef))
    np.add.at(yu, ss.verts, -case.eps_out * (Ms @ ls))
    scale = np.abs(rho).max()
    # Gamma_s rows at sampled vertices: (M_s/2 - K_Y) u + V_Y lam_s = 0
    rows_s, _, Vs, Ks = _sampled_rows(ss, case.kappa)
    us = u[ss.verts]
    ds = 0.5 * (Ms @ us)[rows_s] - Ks @ us + Vs @ ls
    # Gamma_m equation at sampled vertices: V_L lam_m - (M_m/2 + K_L) u + (l_B/eps_m) <u_coul, psi> = 0,
    # the Coulomb rows from the triangles incident to the sampled vertices
    rows_m, tt, Vm, Km = _sampled_rows(sm, 0.0)
    sub = bem.Surface(case.xyz, case.gm_tris[tt])
    coul = (lB / case.eps_in) * bem.coulomb_rhs(sub, case.q_xyz, case.q_z)
    coul_rows = coul[np.searchsorted(sub.verts, sm.verts[rows_m])]
    um = u[sm.verts]
    dm = Vm @ lm - (0.5 * (Mm @ um)[rows_m] + Km @ um) + coul_rows
    print("solute full size residual: FEM rows %.3e of max|rho|, Gamma_s rows %.3e, Gamma_m rows %.3e "
          "of max|coul|; Newton %d, GMRES %s"
          % (np.abs(rho - yu).max() / scale, np.abs(ds).max() / np.abs(coul_rows).max(),
             np.abs(dm).max() / np.abs(coul_rows).max(), res["newton_iters"], res["gmres"]))
    assert np.abs(rho - yu).max() < 1e-9 * scale
    assert np.abs(ds).max() < 1e-9 * np.abs(coul_rows).max()
    assert np.abs(dm).max() < 1e-9 * np.abs(coul_rows).max()
