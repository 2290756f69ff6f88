"""Pins for the oracle's coupled solve, Newton iteration, omega search and
energy (no GPU).

Independent references: the Kirkwood / Debye-Hueckel closed form for a
central charge in a sphere, Born's formula at kappa = 0, a high-resolution
radial boundary-value solve of the nonlinear spherical problem
(scipy.integrate.solve_bvp), a sparse direct solve for GMRES, Gauss's law,
finite differences for f_d', quadratic Newton convergence and the small-charge
scaling of the nonlinear terms.
"""
import numpy as np
import pytest
from scipy.integrate import solve_bvp, quad

from oracle import pb

C_KCAL = 332.0637
KB = 0.0019872043


def kirkwood(z, a, eps_m, eps_s, kappa):
    """Linear solvation energy of a central charge z in a sphere of radius a (kcal/mol)."""
    return C_KCAL * z * z / (2 * a) * (1 / (eps_s * (1 + kappa * a)) - 1 / eps_m)


def radial_nonlinear(z, a, R, eps_m, eps_s, kappa, T):
    """(Total, dG_ion) of the nonlinear spherical three-region problem by a radial BVP:
    u'' + 2u'/r = kappa^2 sinh u on [a, R], eps_s u'(a) = -l_B z / a^2,
    u'(R) = -(kappa + 1/R) u(R) (the linear Yukawa far field)."""
    kT = KB * T
    lB = C_KCAL / kT
    r = np.linspace(a, R, 4001)
    B = lB * z * np.exp(kappa * a) / (eps_s * (1 + kappa * a))
    y0 = np.vstack([B * np.exp(-kappa * r) / r, -B * np.exp(-kappa * r) / r * (1 / r + kappa)])
    f = lambda r, y: np.vstack([y[1], kappa ** 2 * np.sinh(y[0]) - 2 * y[1] / r])
    bc = lambda ya, yb: np.array([eps_s * ya[1] + lB * z / a ** 2, yb[1] + (kappa + 1 / R) * yb[0]])
    sol = solve_bvp(f, bc, r, y0, tol=1e-10, max_nodes=200000)
    assert sol.success
    ur = sol.sol(a)[0] - lB * z / (eps_m * a)
    c0 = eps_s * kappa ** 2 / (8 * np.pi * lB)
    g = lambda s: (lambda u: 4 * np.pi * s * s * (u * np.sinh(u) - 2 * np.cosh(u) + 2))(sol.sol(s)[0])
    ion, _ = quad(g, a, R, epsabs=1e-300, epsrel=1e-10, limit=400)
    dG = kT * c0 * ion
    return 0.5 * kT * z * ur + dG, dG


TIGHT = pb.Opts(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-11)


@pytest.fixture(scope="module")
def tiny_problem(tiny_case, bem_cache):
    return pb.Problem(tiny_case, bem_cache=bem_cache)


@pytest.fixture(scope="module")
def small_problem(small_case, bem_cache):
    return pb.Problem(small_case, bem_cache=bem_cache)


def test_radial_reference_matches_kirkwood_in_linear_limit():
    # the BVP machinery itself: tiny charge -> ion term ~ z^4, energy -> Kirkwood
    tot, dG = radial_nonlinear(0.01, 4.0, 10.0, 4.0, 80.0, 0.125, 300.0)
    assert abs(tot - kirkwood(0.01, 4.0, 4.0, 80.0, 0.125)) < 1e-6 * abs(tot)
    # the radial BVP's nonlinear value for this geometry (kappa = 0.125), recorded once: -251.7472 kcal/mol
    tot5, dG5 = radial_nonlinear(5.0, 4.0, 10.0, 4.0, 80.0, 0.125, 300.0)
    assert abs(tot5 + 251.7472) < 1e-3 and abs(dG5 - 0.7964) < 1e-4


def test_linear_energy_converges_to_kirkwood(tiny_problem, small_problem):
    errs = []
    for P in (tiny_problem, small_problem):
        R = pb.solve(P, TIGHT, linear_only=True)
        ref = kirkwood(5.0, 4.0, 4.0, 80.0, P.kappa)
        errs.append(abs(R.LC - ref) / abs(ref))
    assert errs[1] < 1e-2          # nu = 5, 13 layers
    assert errs[1] < errs[0]       # refinement reduces the error


def test_born_limit_kappa_zero(tiny_case, bem_cache):
    P = pb.Problem(tiny_case, kappa=0.0, bem_cache=bem_cache)
    R = pb.solve(P, TIGHT)
    born = C_KCAL * 25 / (2 * 4.0) * (1 / 80.0 - 1 / 4.0)
    assert abs(R.total - born) / abs(born) < 2.5e-2
    assert R.dG_ion == 0.0 and abs(R.NC) < 1e-9 * abs(R.LC)


def test_nonlinear_energy_against_radial_bvp(tiny_problem, small_problem):
    errs = []
    for P in (tiny_problem, small_problem):
        R = pb.solve(P, TIGHT)
        tot, dG = radial_nonlinear(5.0, 4.0, 10.0, 4.0, 80.0, P.kappa, 300.0)
        errs.append(abs(R.total - tot) / abs(tot))
        assert abs(R.total - (R.LC + R.NC + R.dG_ion)) < 1e-12 * abs(R.total)
        assert R.dG_ion > 0 and R.NC < 0
        if P is small_problem:
            assert abs(R.dG_ion - dG) / dG < 3e-2
    assert errs[1] < 1e-2 and errs[1] < errs[0]


def test_gmres_matches_direct_solve(tiny_problem):
    P = tiny_problem
    Jm = P.J(np.linspace(-1, 1, P.nv), 'HS')
    rhs = np.random.default_rng(3).standard_normal(P.n)
    x_it, its, rel = pb.gmres(lambda v: P.apply(v, Jm), rhs, 1e-12, 200, 2000, P.jacobi(Jm))
    x_d = pb.linear_solve(P, Jm, rhs, 0, pb.Opts(linear_solver='direct'))[0]
    assert rel < 1e-12 and its > 10
    assert np.linalg.norm(x_it - x_d) < 1e-9 * np.linalg.norm(x_d)
    # the operator apply agrees with the assembled matrix
    assert np.linalg.norm(P.apply(rhs, Jm) - P.matrix(Jm) @ rhs) < 1e-12 * np.linalg.norm(P.apply(rhs, Jm))


def test_newton_gauss_law_and_quadratic_convergence(tiny_problem):
    P = tiny_problem
    R = pb.solve(P, TIGHT)
    u, lm, ls = P.split(R.x)
    # discrete Gauss law: the FEM rows sum to zero at convergence (A has zero row sums)
    flux = P.N(u, 'HS').sum() + P.eps_m * (P.Mm @ lm).sum() - P.eps_s * (P.Ms @ ls).sum()
    scale = P.eps_m * abs((P.Mm @ lm).sum())
    assert abs(flux) < 1e-8 * scale
    # continuum Gauss law for the flux through Gamma_m: eps_m int lam_m = -4 pi l_B sum z
    tot = P.eps_m * (P.Mm @ lm).sum()
    assert abs(tot / (-4 * np.pi * P.lB * 5.0) - 1) < 3e-2
    e = R.trace['e']
    assert len(e) >= 4 and e[-1] < 1e-10
    # quadratic: e_{k+1} <= C e_k^2 once in the basin
    k = next(i for i in range(len(e)) if e[i] < 1.0)
    assert e[k + 1] < 0.1 * e[k] ** 2 * 10 and e[k + 1] < e[k] ** 1.8


def test_residual_of_converged_solution(tiny_problem):
    P = tiny_problem
    R = pb.solve(P, TIGHT)
    u = R.x[:P.nv]
    res = P.apply(R.x) + P.pad(P.N(u, 'HS')) - P.b
    assert np.linalg.norm(res) < 1e-9 * np.linalg.norm(P.b)


def test_fd_derivative_and_search_conditions(tiny_problem):
    P = tiny_problem
    xL = pb.solve(P, TIGHT, linear_only=True).x
    u = xL[:P.nv]
    c = P.b - P.apply(xL)
    d = c - P.pad(P.N(u, 'T3'))
    Jm = P.J(u, 'T3')
    du = pb.linear_solve(P, Jm, d, 1e-12, TIGHT)[0]
    p = -P.apply(du)
    for om in (0.7, 1.3, 2.0):
        D = pb.omega_dots(P, u, du[:P.nv], c, p, om, 'T3')
        f, fp = pb.fd_and_derivative(D, om)
        h = 1e-5
        fpl = pb.fd_and_derivative(pb.omega_dots(P, u, du[:P.nv], c, p, om + h, 'T3'), om + h)[0]
        fmi = pb.fd_and_derivative(pb.omega_dots(P, u, du[:P.nv], c, p, om - h, 'T3'), om - h)[0]
        assert abs(fp - (fpl - fmi) / (2 * h)) < 1e-6 * max(1.0, abs(fp))
        # ||d(omega)||^2 from the dots equals the direct residual norm
        w = xL + om * du
        dv = P.b - P.apply(w) - P.pad(P.N(w[:P.nv], 'T3'))
        assert abs(pb.dnorm2(D, om) - dv @ dv) < 1e-9 * (dv @ dv)
    # d(0) . d'(0) = -||d||^2 (Delta solves the Newton system): g_d(0) < 0
    D0 = pb.omega_dots(P, u, du[:P.nv], c, p, 0.0, 'T3')
    assert abs(D0['PR'] + d @ d) < 1e-8 * (d @ d)
    tr = dict(omega_evals=[])
    om = pb.omega_search(P, u, du[:P.nv], c, p, float(d @ d), 'T3', 2.0, pb.Opts(tol_omega=1e-8), tr)
    D = pb.omega_dots(P, u, du[:P.nv], c, p, om, 'T3')
    assert abs(pb.fd_and_derivative(D, om)[0]) < 1e-8
    assert pb.dnorm2(D, om) < d @ d
    # omega minimises ||d(omega)||: neighbours are not better
    for dom in (-0.05, 0.05):
        Dn = pb.omega_dots(P, u, du[:P.nv], c, p, om + dom, 'T3')
        assert pb.dnorm2(Dn, om + dom) >= pb.dnorm2(D, om)


def test_small_charge_scaling(tiny_case, bem_cache):
    import dataclasses
    out = {}
    for zs in (0.5, 0.05):
        c = dataclasses.replace(tiny_case, q_z=tiny_case.q_z * zs / 5.0)
        P = pb.Problem(c, bem_cache=bem_cache)
        out[zs] = pb.solve(P, TIGHT)
    # LC ~ z^2, NC ~ z^4, dG_ion ~ z^4 in the weakly nonlinear limit
    assert abs(out[0.5].LC / out[0.05].LC / 100 - 1) < 1e-9
    assert abs(out[0.5].NC / out[0.05].NC / 1e4 - 1) < 2e-2
    assert abs(out[0.5].dG_ion / out[0.05].dG_ion / 1e4 - 1) < 2e-2


def test_zero_charges_give_the_zero_solution(tiny_case, bem_cache):
    """With no charge the system Acal(0) Phi + N(Phi) = 0 is homogeneous and sinh is monotone, so
    Phi = 0 is its only solution: the linear part is zero, the first Newton residual is exactly
    zero and the iteration stops there with e_0 = 0 and every energy term zero."""
    import dataclasses
    c = dataclasses.replace(tiny_case, q_z=0.0 * tiny_case.q_z)
    r = pb.solve(pb.Problem(c, bem_cache=bem_cache), TIGHT)
    assert not r.x.any() and r.newton_iters == 1
    assert r.trace["e"] == [0.0] and r.trace["gmres"] == [0] and r.trace["linear_gmres"] == 0
    assert (r.total, r.LC, r.NC, r.dG_ion) == (0.0, 0.0, 0.0, 0.0)


def test_paper_default_options_trace(small_problem):
    """Paper-default tolerances: converges in a handful of Newton steps with omega > 0
    and the final energy within Tol-level of the tight solve."""
    R = pb.solve(small_problem, pb.Opts())
    Rt = pb.solve(small_problem, TIGHT)
    assert 3 <= R.newton_iters <= 8
    assert all(0 < w <= 4 for w in R.trace['omega'])
    assert R.trace['scheme'][0] == 'T3' and set(R.trace['scheme'][1:]) == {'HS'}
    assert abs(R.total - Rt.total) / abs(Rt.total) < 1e-4


def test_taylor_schedules_and_picard_reach_the_newton_solution(tiny_problem):
    """T3-T5-HS, T3-T5-T7-T7-HS (Sec. 3.2) and Picard (Sec. 2.4.1) iterate to the same discrete
    fixed point as T3-HS Newton: the nonlinear system does not depend on the path."""
    P = tiny_problem
    ref = pb.solve(P, TIGHT)
    tight = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-10)
    for o in (pb.Opts(taylor=('T3', 'T5'), **tight), pb.Opts(taylor=('T3', 'T5', 'T7', 'T7'), **tight),
              pb.Opts(taylor=(), **tight), pb.Opts(omega_warm_start=True, **tight),
              pb.Opts(method='picard', omega0_first=0.5, omega0_rest=0.5, **tight)):
        R = pb.solve(P, o)
        assert abs(R.total - ref.total) < 1e-10 * abs(ref.total), (o.method, o.taylor)
        assert np.linalg.norm(R.x - ref.x) < 1e-8 * np.linalg.norm(ref.x)


def test_omega_warm_start_steps(tiny_problem):
    """Sec. 3.5 warm start: three bisection midpoints of [2, 3] (2.5 first), then secant steps;
    the returned guess is a secant iterate of f_d."""
    P = tiny_problem
    xL = pb.solve(P, TIGHT, linear_only=True).x
    u = xL[:P.nv]
    c = P.b - P.apply(xL)
    d = c - P.pad(P.N(u, 'T3'))
    du = pb.linear_solve(P, P.J(u, 'T3'), d, 1e-12, TIGHT)[0]
    p = -P.apply(du)
    tr = {}
    om0 = pb.warm_start_omega(P, u, du[:P.nv], c, p, 'T3', pb.Opts(), tr)
    assert tr['omega_evals_warm'] >= 3 and np.isfinite(om0)
    f = lambda o: pb.fd_and_derivative(pb.omega_dots(P, u, du[:P.nv], c, p, o, 'T3'), o)[0]
    # the first bisection point is the midpoint and the search moves towards the root of f_d
    f25 = f(2.5)
    assert (om0 < 2.5) == (f25 < 0)
    # near the returned guess f_d is small compared with its value at the start of the bracket
    assert abs(f(om0)) < abs(f25)


def test_picard_defaults_converge_slower_than_newton(tiny_problem):
    P = tiny_problem
    Rn = pb.solve(P, pb.Opts())
    Rp = pb.solve(P, pb.Opts(method='picard', omega0_first=0.5, omega0_rest=0.5))
    assert Rp.newton_iters > Rn.newton_iters
    assert all(0 < w < 1.0 for w in Rp.trace['omega'])
    assert abs(Rp.total - Rn.total) < 1e-5 * abs(Rn.total)


def test_taylor_schemes_are_sinh_series():
    from oracle import fem
    import math
    u = np.linspace(-2, 2, 9)
    for name, deg in (('T3', 3), ('T5', 5), ('T7', 7)):
        F, Fp, Fpp = fem.F_scheme(name, u)
        assert np.allclose(F, sum(u ** k / math.factorial(k) for k in range(1, deg + 1, 2)), rtol=0, atol=1e-14)
        assert np.allclose(Fp, sum(u ** k / math.factorial(k) for k in range(0, deg, 2)), rtol=0, atol=1e-14)
        assert np.allclose(Fpp, sum(u ** k / math.factorial(k) for k in range(1, deg - 1, 2)), rtol=0, atol=1e-14)
    # higher degree is closer to sinh
    errs = [np.abs(fem.F_scheme(n, u)[0] - np.sinh(u)).max() for n in ('T3', 'T5', 'T7')]
    assert errs[0] > errs[1] > errs[2]
