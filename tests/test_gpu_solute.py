"""Parity of the paper's own formulation on the GPU (FEM over Omega_m and Omega_i with the charges
as point loads and the Yukawa BEM on Gamma_s, Eq. fembem_matrix; lam_m from the Gamma_m equation
of Sec. 2.3.1) against the oracle's SoluteProblem, through the C ABI.

Inputs: the tiny single-charge solute sphere (nu = 3, 5 shell and 6 core layers) and a
multi-charge one (nu = 5, 13 shell and 12 core layers, 12 charges of both signs off the centre,
so the point loads fall inside tets).  Tolerances as for the three-region path: 1e-11 relative
per step in float64, 1e-8 relative L2 on the converged potentials, 1e-9 on the energy; the mixed
path 1e-5 on the energy.  The Newton tolerance is 1e-9 absolute: next to a point charge the
potential reaches 1e4 kT/e.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-9)
_CASES = {}


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _multi_case():
    from paper_2511_21713_gb300 import inputs
    if "multi" not in _CASES:
        q, z = inputs.ball_charges(12, 3.0, 5, seed=77)
        _CASES["multi"] = inputs.solute_sphere_case(nu=5, layers=13, core_layers=12, q_xyz=q, q_z=z,
                                                    eps_in=2.0, ionic=0.1, name="multi_charge_solute_nu5")
    return _CASES["multi"]


@pytest.fixture(scope="module", params=["tiny", "multi"])
def solute_pair(request, tiny_solute_case, bem_cache):
    from paper_2511_21713_gb300 import pbfb
    from oracle import solute
    case = tiny_solute_case if request.param == "tiny" else _multi_case()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    P = solute.SoluteProblem(case, bem_cache=bem_cache)
    yield case, m, P
    m.close()


def _full(P, x2, lam_m=None):
    """[u; lam_m; lam_s] from the oracle's [u; lam_s]."""
    return np.concatenate([x2[:P.nv], np.zeros(P.nm) if lam_m is None else lam_m, x2[P.nv:]])


def test_sizes_and_surface_order(solute_pair):
    from paper_2511_21713_gb300 import pbfb
    case, m, P = solute_pair
    assert m.full and (m.n_v, m.n_t, m.n_m, m.n_s) == (P.nv, case.n_t, P.nm, P.ns)
    assert m.n == P.nv + P.nm + P.ns
    assert np.array_equal(m.surface_vertices(pbfb.GAMMA_M), P.sm.verts)
    assert np.array_equal(m.surface_vertices(pbfb.GAMMA_S), P.ss.verts)


def test_fem_rows_and_load(solute_pair):
    """Rows of A~ + J (eps_m on Omega_m tets, eps_s and J on Omega_i tets) and N."""
    from paper_2511_21713_gb300 import pbfb
    case, m, P = solute_pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    r = np.linalg.norm(P.xyz, axis=1)
    u = 4.0 * np.exp(-0.3 * np.abs(r - 4.0)) + 0.2 * np.random.default_rng(1).standard_normal(P.nv)
    N_dev = dev(np.zeros(P.nv))
    m.assemble(pbfb.HS, dev(u), N_dev)
    rp, col, val = m.fem_rows()
    G = sp.csr_matrix((val, col, rp), shape=(P.nv, m.n))
    O = sp.hstack([P.A + P.J(u, "HS"), sp.csr_matrix((P.nv, P.nm)), P.B_us]).tocsr()
    assert np.abs((G - O).toarray()).max() <= 1e-12 * np.abs(O).max()
    assert rel(host(N_dev), P.N(u, "HS")) < 1e-13
    m.clear_jacobian()


@pytest.mark.parametrize("precision", [0, 1])
def test_coupled_apply(solute_pair, precision):
    """Acal(J) x: the oracle's operator on [u; lam_s], the identity on the lam_m rows."""
    from paper_2511_21713_gb300 import pbfb
    case, m, P = solute_pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    u = 3.0 * np.exp(-0.3 * np.abs(np.linalg.norm(P.xyz, axis=1) - 4.0))
    m.assemble(pbfb.HS, dev(u))
    x = np.random.default_rng(4).standard_normal(m.n)
    y = dev(np.zeros(m.n))
    m.apply(dev(x), y)
    x2 = np.concatenate([x[:P.nv], x[P.nv + P.nm:]])
    ref = P.apply(x2, P.J(u, "HS"))
    got = host(y)
    tol = 3e-6 if precision == pbfb.MIXED else 1e-11
    assert rel(got[:P.nv], ref[:P.nv]) < tol
    assert rel(got[P.nv + P.nm:], ref[P.nv:]) < tol
    assert np.array_equal(got[P.nv:P.nv + P.nm], x[P.nv:P.nv + P.nm])
    m.clear_jacobian()


@pytest.mark.parametrize("precision", [0, 1])
def test_gamma_m_flux(solute_pair, precision):
    """lam_m from a given u (float64 and float-float far fields) equals the oracle's dense solve."""
    case, m, P = solute_pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    r = np.linalg.norm(P.xyz, axis=1)
    u = 5.0 * np.exp(-0.2 * r) + 0.1 * np.cos(P.xyz[:, 2])
    x = dev(_full(P, np.concatenate([u, np.zeros(P.ns)])))
    for coulomb in (1, 0):
        lam = dev(np.zeros(P.nm))
        m.gamma_m_flux(x, coulomb, lam)
        assert rel(host(lam), P.lam_m(u, bool(coulomb))) < 1e-11, coulomb


def test_solve_fp64_tight(solute_pair):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = solute_pair
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(**TIGHT))
    R = pb.solve(P, pb.Opts(tol_gmres0=1e-13, tol_gmres=1e-13, tol_nl=1e-9, linear_solver="direct"))
    ref = P.expand(R.x)
    assert rel(x[:P.nv], ref[:P.nv]) < 1e-8
    assert rel(x[P.nv:P.nv + P.nm], ref[P.nv:P.nv + P.nm]) < 1e-8
    assert rel(x[P.nv + P.nm:], ref[P.nv + P.nm:]) < 1e-8
    for key, val in (("total", R.total), ("LC", R.LC), ("NC", R.NC), ("dG_ion", R.dG_ion)):
        assert abs(res[key] - val) < 1e-9 * abs(R.total), key
    assert res["status"] == 0 and abs(res["newton_iters"] - R.newton_iters) <= 1


def test_solve_mixed(solute_pair):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = solute_pair
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                     pbfb.default_opts(precision=pbfb.MIXED, tol_gmres0=1e-7, tol_gmres=1e-7, tol_nl=1e-6))
    R = pb.solve(P, pb.Opts(tol_gmres0=1e-13, tol_gmres=1e-13, tol_nl=1e-9, linear_solver="direct"))
    assert abs(res["total"] - R.total) < 1e-5 * abs(R.total)
    assert rel(x, P.expand(R.x)) < 1e-4


def test_flux_reproduces_a_shell_solution(tiny_case):
    """On a three-region mesh the Gamma_m row of the solve is the same equation: the flux of the
    converged trace equals the solve's own lam_m."""
    from paper_2511_21713_gb300 import pbfb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, c.q_z)
    x, _ = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(tol_gmres0=1e-12, tol_gmres=1e-12,
                                                                         tol_nl=1e-11))
    lam = dev(np.zeros(m.n_m))
    m.gamma_m_flux(dev(x), 1, lam)
    assert rel(host(lam), x[m.n_v:m.n_v + m.n_m]) < 1e-9
    m.close()


def test_zero_charges(tiny_solute_case):
    """No charge: no point load, a zero first residual, the solution and every energy term zero."""
    from paper_2511_21713_gb300 import pbfb
    c = tiny_solute_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, 0.0 * c.q_z)
    x, res = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(precision=pbfb.MIXED))
    assert res["status"] == 0 and res["newton_iters"] == 1 and not np.any(x)
    assert (res["total"], res["LC"], res["NC"], res["dG_ion"]) == (0.0, 0.0, 0.0, 0.0)
    m.close()


def test_charge_outside_omega_m(tiny_solute_case):
    from paper_2511_21713_gb300 import pbfb
    c = tiny_solute_case
    m = pbfb.Mesh.from_case(c)
    with pytest.raises(pbfb.PbfbError) as e:
        m.charges_set(np.array([[0.0, 0.0, 4.5]]), np.array([1.0]))
    assert e.value.code == 1 and "Omega_m" in str(e.value)
    with pytest.raises(pbfb.PbfbError) as e:
        m.gamma_m_flux(dev(np.zeros(m.n)), 1, dev(np.zeros(m.n_m)))
    assert e.value.code == 8                       # STATE: no parameters yet
    m.close()
