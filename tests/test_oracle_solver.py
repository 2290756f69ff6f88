"""Pins for the oracle's coupled solve, Newton iteration, omega search and
energy (no GPU).

Independent references: the Kirkwood / Debye-Hueckel closed form for a
central charge in a sphere, Born's formula at kappa = 0, a high-resolution
radial boundary-value solve of the nonlinear spherical problem
(scipy.integrate.solve_bvp), a sparse direct solve for GMRES, Gauss's law,
finite differences for f_d', quadratic Newton convergence and the small-charge
scaling of the nonlinear terms.  The omega search's fallback is pinned by a
brute-force minimisation of the residual norm itself, Picard's first secant step
by Eq. SEC_FD and f_d(0) = 1, and the reuse rules (R_e, L_e) and the GMRES
tolerance schedule on the recorded traces.
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


def test_automatic_omega_beats_every_constant_omega(small_problem):
    """The paper's case for the automatic relaxation factor (Sec. 3.3, the 1AJF tables with a constant
    and with a variable omega: 7 Newton iterations at the best constant omega, 1.0 or 1.1, against 4
    with omega from f_d(omega) = 0): on the single-charge sphere at the paper's default options the
    automatic omega converges in fewer Newton iterations than every constant omega from 0.5 to 1.5
    (the best constants, 1.0 and 1.1, take 5 against 4; the iteration count grows away from them on
    both sides, as in the paper's table), and every run reaches the same energy to the nonlinear
    tolerance.  A wrong sign or term in f_d or f_d' would give worse factors than the constants."""
    auto = pb.solve(small_problem, pb.Opts())
    runs = {w: pb.solve(small_problem, pb.Opts(omega_search=False, omega0_first=w, omega0_rest=w))
            for w in (0.5, 0.8, 1.0, 1.1, 1.2, 1.5)}
    its = {w: r.newton_iters for w, r in runs.items()}
    assert auto.newton_iters < min(its.values()), (auto.newton_iters, its)
    assert its[0.5] > its[0.8] > its[1.0] and its[1.5] > its[1.2] > its[1.1], its
    for r in runs.values():
        assert abs(r.total - auto.total) < 1e-6 * abs(auto.total)


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


def _step_inputs(P, Phi, scheme, picard=False):
    """u, c = b - Acal(0) Phi, d = c - [N(u); 0; 0], the exact increment Delta (sparse direct solve
    of Acal(J) Delta = d, J = 0 for Picard) and p = -Acal(0) Delta at the iterate Phi."""
    u = Phi[:P.nv]
    c = P.b - P.apply(Phi)
    d = c - P.pad(P.N(u, scheme))
    J = None if picard else P.J(u, scheme)
    du = pb.linear_solve(P, J, d, 0.0, pb.Opts(linear_solver="direct"))[0]
    return u, c, d, du, -P.apply(du)


def _golden_min(f, a, b, tol=1e-10):
    """Minimiser of a unimodal f on [a, b] by golden-section search (function values only)."""
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = f(x1), f(x2)
    while b - a > tol:
        if f1 < f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - g * (b - a)
            f1 = f(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (b - a)
            f2 = f(x2)
    return 0.5 * (a + b)


@pytest.mark.parametrize("k", [0, 1])
def test_fallback_returns_the_minimiser_of_the_residual_norm(tiny_problem, k):
    """The scan-and-bisect fallback of the omega search (reading R10 of the global convergence
    condition of Sec. 2.5.2) returns the minimiser of ||d(omega)||^2 on (0, omega_max]: checked
    against a brute-force search on the residual itself, d(omega) = b - Acal(0)(Phi + omega Delta)
    - [N(u + omega Delta_u); 0; 0] (a 1000-point grid, then golden section), not on the dot
    products the fallback uses.  k = 0: the T3 step from x_L; k = 1: the sinh step after it."""
    P = tiny_problem
    Phi = pb.solve(P, TIGHT, linear_only=True).x
    if k == 1:
        u, c, d, du, p = _step_inputs(P, Phi, "T3")
        om = pb.omega_search(P, u, du[:P.nv], c, p, float(d @ d), "T3", 2.0, pb.Opts(), dict(omega_evals=[]))
        Phi = Phi + om * du
    scheme = "T3" if k == 0 else "HS"
    u, c, d, du, p = _step_inputs(P, Phi, scheme)
    om_fb = pb._fallback(P, u, du[:P.nv], c, p, float(d @ d), scheme, pb.Opts())
    ADelta = P.apply(du)

    def dn2(o):
        dv = c - o * ADelta - P.pad(P.N(u + o * du[:P.nv], scheme))
        return float(dv @ dv)

    grid = np.linspace(0.0, 4.0, 1001)[1:]
    vals = np.array([dn2(o) for o in grid])
    j = int(np.argmin(vals))
    om_bf = _golden_min(dn2, grid[max(j - 1, 0)], grid[min(j + 1, grid.size - 1)])
    # bisection accuracy (omega_max / 16) / 2^20 = 2.4e-7; the minimum is flat, so golden section
    # on function values locates it to about sqrt(rounding) of the curvature scale
    assert abs(om_fb - om_bf) < 2e-6, (om_fb, om_bf)
    assert dn2(om_fb) < dn2(0.0) and dn2(om_fb) <= vals.min() * (1 + 1e-12)


def test_forced_fallback_solves_reach_the_same_solution(tiny_problem):
    """max_omega_iters = 1 with an unreachable Tol_omega sends every omega search to the
    fallback (Newton and Picard); the iteration still converges to the discrete solution."""
    P = tiny_problem
    ref = pb.solve(P, TIGHT)
    tight = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-10, max_omega_iters=1, tol_omega=1e-14)
    for o in (pb.Opts(**tight), pb.Opts(method="picard", omega0_first=0.5, omega0_rest=0.5, **tight)):
        R = pb.solve(P, o)
        searches = sum(1 for n in R.trace["omega_evals"] if n > 0)
        assert R.trace.get("fallback", 0) == searches >= 1
        assert abs(R.total - ref.total) < 1e-10 * abs(ref.total)


def test_picard_direct_secant(tiny_problem):
    """Appendix A for Picard: f_d(0) = 1 (Delta solves Acal(0) Delta = d, so p + r(0) = 0), and the
    first secant step through (0, f_d(0) = 1) and (omega0, f_d(omega0)) is the direct formula
    Eq. SEC_FD, omega = omega0 / (1 - f_d(omega0)).  With Tol_omega between |f_d(omega0)| and
    |f_d| at that point, picard_omega returns exactly that omega after two evaluations."""
    P = tiny_problem
    xL = pb.solve(P, TIGHT, linear_only=True).x
    u, c, d, du, p = _step_inputs(P, xL, "T3", picard=True)
    f = lambda o: pb.fd_and_derivative(pb.omega_dots(P, u, du[:P.nv], c, p, o, "T3"), o)[0]
    assert abs(f(0.0) - 1.0) < 1e-12
    om0 = 0.5
    f0 = f(om0)
    om1 = om0 / (1.0 - f0)
    f1 = f(om1)
    assert abs(f1) < 0.5 * abs(f0)
    tr = dict(omega_evals=[])
    om = pb.picard_omega(P, u, du[:P.nv], c, p, float(d @ d), "T3", om0,
                         pb.Opts(tol_omega=np.sqrt(abs(f0 * f1))), tr)
    assert om == om1 and tr["omega_evals"] == [2] and "fallback" not in tr


@pytest.mark.parametrize("R_e", [1.4, 3.0])
def test_picard_R_e_rule_on_the_trace(tiny_problem, R_e):
    """Appendix B: a Picard step keeps the previous omega exactly when the last two errors fell by
    at least R_e (e_{k-1} / e_k >= R_e in the paper's indexing; with trace index j, e[j-2] / e[j-1]),
    and recomputes it otherwise (always in the first two steps, which have no such ratio)."""
    P = tiny_problem
    R = pb.solve(P, pb.Opts(method="picard", omega0_first=0.5, omega0_rest=0.5, R_e=R_e))
    e, ev, om = R.trace["e"], R.trace["omega_evals"], R.trace["omega"]
    kinds = set()
    for j in range(len(e)):
        reuse = j >= 2 and e[j - 2] / e[j - 1] >= R_e
        kinds.add(reuse)
        assert (ev[j] == 0) == reuse, (j, e[j - 2:j], ev[j])
        if reuse:
            assert om[j] == om[j - 1]
    assert kinds == {True, False}


def test_accept_ratio_zero_fails_the_search(tiny_problem):
    """accept_ratio = 0 leaves no omega satisfying ||d(omega)||^2 < 0: the search and its fallback
    both refuse, which is how the omega-search failure is forced on the host."""
    P = tiny_problem
    with pytest.raises(RuntimeError, match="omega search failed"):
        pb.solve(P, pb.Opts(accept_ratio=0.0))


def test_newton_L_e_rule_and_tolerance_schedule_on_the_trace(small_problem):
    """Appendix B: once the last update e_{k-1} < L_e the Newton step reuses the previous omega
    without a search, and otherwise searches; the GMRES tolerance starts at Tol_GR0 and after a
    step with e < 1250 tol drops tenfold, not below Tol_GR (reading R12)."""
    P = small_problem
    o = pb.Opts()
    R = pb.solve(P, o)
    e, ev, om, tol = R.trace["e"], R.trace["omega_evals"], R.trace["omega"], R.trace["tol_gmres"]
    kinds = set()
    for k in range(len(e)):
        reuse = k > 0 and e[k - 1] < o.L_e
        kinds.add(reuse)
        assert (ev[k] == 0) == reuse, (k, e[k - 1:k + 1], ev[k])
        if reuse:
            assert om[k] == om[k - 1]
    assert kinds == {True, False}
    assert tol[0] == o.tol_gmres0
    for k in range(1, len(tol)):
        expect = max(0.1 * tol[k - 1], o.tol_gmres) if e[k - 1] < 1250.0 * tol[k - 1] else tol[k - 1]
        assert tol[k] == expect
    assert tol[-1] < tol[0]
