"""Pins for the oracle's FEM(Omega_m and Omega_i)-BEM(Gamma_s) formulation with the Gamma_m
post-process (Sec. 2.2, Eq. fembem_matrix; Sec. 2.3.1), no GPU.

Independent references: the partition of unity and linear precision of the P1 hat functions
(point load), the exact discrete Gauss law (row sums of the stiffness vanish), the continuum
Gauss law on Gamma_m, Kirkwood's closed form, the radial boundary-value solve of the nonlinear
sphere, and the separately pinned three-region formulation on the same surfaces and shell.
"""
import numpy as np
import pytest

from oracle import pb, solute
from test_oracle_solver import kirkwood, radial_nonlinear

TIGHT = pb.Opts(tol_gmres0=1e-13, tol_gmres=1e-13, tol_nl=1e-9, linear_solver="direct")


@pytest.fixture(scope="module")
def small_solute(small_solute_case, bem_cache):
    P = solute.SoluteProblem(small_solute_case, bem_cache=bem_cache)
    return P, pb.solve(P, TIGHT)


@pytest.fixture(scope="module")
def small_shell(small_case, bem_cache):
    P = pb.Problem(small_case, bem_cache=bem_cache)
    return P, pb.solve(P, pb.Opts(tol_gmres0=1e-13, tol_gmres=1e-13, tol_nl=1e-11, linear_solver="direct"))


def test_mesh_regions(tiny_solute_case):
    from oracle import fem
    c = tiny_solute_case
    vol, _ = fem.tet_geometry(c.xyz, c.tets)
    # the tets inside Gamma_m fill the polyhedron Gamma_m bounds (divergence theorem on its faces)
    x = c.xyz[c.gm_tris]
    enclosed = np.einsum("ij,ij->i", x[:, 0], np.cross(x[:, 1], x[:, 2])).sum() / 6.0
    assert abs(vol[c.tet_region == 0].sum() - enclosed) < 1e-12 * enclosed


def test_point_load_moments(tiny_solute_case):
    from paper_2511_21713_gb300 import inputs
    c = tiny_solute_case
    tm = c.tets[c.tet_region == 0]
    q, z = inputs.ball_charges(25, 3.0, 10, seed=5)
    z = z * np.linspace(0.5, 1.5, z.size)
    load = solute.point_load(c.xyz, tm, q, z)
    # partition of unity and linear precision of the P1 hat functions
    assert abs(load.sum() - z.sum()) < 1e-12 * np.abs(z).sum()
    assert np.abs(load @ c.xyz - z @ q).max() < 1e-12 * np.abs(z).sum() * 4.0
    # a charge on a vertex loads that vertex alone; one outside Omega_m is refused
    v = int(tm[7, 2])
    one = solute.point_load(c.xyz, tm, c.xyz[v][None], [2.0])
    assert abs(one[v] - 2.0) < 1e-12 and np.abs(np.delete(one, v)).max() < 1e-12
    with pytest.raises(ValueError):
        solute.point_load(c.xyz, tm, np.array([[0.0, 0.0, 5.0]]), [1.0])


def test_discrete_gauss_law(small_solute):
    """Summing every FEM row of the converged system: the stiffness rows sum to zero, so
    eps_s kappa^2 int F(u) - eps_s int_Gamma_s lam_s = 4 pi l_B sum z (to solver precision)."""
    P, R = small_solute
    u, ls = P.split(R.x)
    lhs = P.N(u, "HS").sum() - P.eps_s * (P.Ms @ ls).sum()
    rhs = 4.0 * np.pi * P.lB * P.case.q_z.sum()
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
    assert R.newton_iters <= 8 and R.trace["e"][-1] < 1e-9


def test_linear_energy_near_kirkwood(small_solute):
    P, _ = small_solute
    R = pb.solve(P, TIGHT, linear_only=True)
    ref = kirkwood(5.0, 4.0, P.eps_m, P.eps_s, P.kappa)
    assert abs(R.total / ref - 1) < 1e-2     # nu = 5 surfaces: discretisation error 0.8 %


def test_nonlinear_energy_near_radial_solution(small_solute):
    P, R = small_solute
    total, dG = radial_nonlinear(5.0, 4.0, 10.0, P.eps_m, P.eps_s, P.kappa, P.T)
    assert abs(R.total / total - 1) < 1.5e-2
    assert abs(R.dG_ion / dG - 1) < 3e-2
    assert abs(R.total - (R.LC + R.NC + R.dG_ion)) < 1e-12 * abs(R.total)


def test_formulations_agree(small_solute, small_shell):
    """Same surfaces and shell; Omega_m by FEM with a point load here, by the Laplace BIE there:
    the energies agree to a few parts in 1e6, far inside either's discretisation error."""
    P, R = small_solute
    Ps, Rs = small_shell
    assert abs(R.LC / Rs.LC - 1) < 1e-4
    assert abs(R.NC / Rs.NC - 1) < 1e-3
    assert abs(R.dG_ion / Rs.dG_ion - 1) < 1e-3
    # the potentials on the shell differ by the two discretisations of Omega_m (1.4 % of the
    # largest; the energies, Galerkin functionals, much less), lam_m by 0.09 %
    off = P.nv - Ps.nv - 1                  # core vertices come first, the centre last
    u = R.x[:P.nv]
    us = Rs.x[:Ps.nv]
    assert np.abs(u[off:off + Ps.nv] - us).max() < 2e-2 * np.abs(us).max()
    lm = P.lam_m(u)
    lms = Rs.x[Ps.nv:Ps.nv + Ps.nm]
    assert np.linalg.norm(lm - lms) < 2e-3 * np.linalg.norm(lms)


def test_post_processed_flux(small_solute):
    """eps_m int_Gamma_m lam_m = -4 pi l_B sum z (Gauss's law in Omega_m), within the
    discretisation error; without the Coulomb term the nonlinear part's flux is small."""
    P, R = small_solute
    u = R.x[:P.nv]
    lm = P.lam_m(u)
    ref = -4.0 * np.pi * P.lB * P.case.q_z.sum()
    assert abs(P.eps_m * (P.Mm @ lm).sum() / ref - 1) < 1e-3
    x = P.expand(R.x)
    assert np.array_equal(x[P.nv:P.nv + P.nm], lm) and np.array_equal(x[P.nv + P.nm:], R.x[P.nv:])


def test_picard_reaches_the_newton_solution(small_solute):
    """Picard (Sec. 2.4.1) on the same system converges to the same discrete solution."""
    P, R = small_solute
    Rp = pb.solve(P, pb.Opts(tol_gmres0=1e-13, tol_gmres=1e-13, tol_nl=1e-9, linear_solver="direct",
                             method="picard", max_newton=200))
    assert np.linalg.norm(Rp.x - R.x) < 1e-9 * np.linalg.norm(R.x)
    assert abs(Rp.total - R.total) < 1e-10 * abs(R.total)


def test_born_limit(small_solute_case, bem_cache):
    """kappa = 0: no ions (Delta G_Omega_i = 0, no nonlinear part) and Born's energy of a central
    charge within the nu = 5 discretisation error (measured 0.77 %, as for Kirkwood; bound 0.9 %)."""
    P = solute.SoluteProblem(small_solute_case, kappa=0.0, bem_cache=bem_cache)
    R = pb.solve(P, TIGHT)
    born = 332.0637 * 25.0 / (2 * 4.0) * (1 / P.eps_s - 1 / P.eps_m)
    assert abs(R.total / born - 1) < 9e-3
    assert R.dG_ion == 0.0 and abs(R.NC) < 1e-9 * abs(R.total)


def test_uniform_dielectric_has_no_reaction_field(small_solute_case, bem_cache):
    """eps_m = eps_s and no salt: the potential is the charge's own Coulomb field, so the reaction
    potential and the energy vanish up to the discretisation (measured 0.41 % of the Born scale
    C z^2 / (2 a eps) on nu = 5; bound 0.5 %)."""
    P = solute.SoluteProblem(small_solute_case, eps_in=80.0, eps_out=80.0, kappa=0.0, bem_cache=bem_cache)
    R = pb.solve(P, TIGHT, linear_only=True)
    assert abs(R.total) < 5e-3 * 332.0637 * 25.0 / (2 * 4.0) / 80.0
