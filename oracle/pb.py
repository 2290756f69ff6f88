"""Coupled three-region problem, Newton-Raphson with the optimal relaxation
factor, and the solvation energy (oracle; test infrastructure only).

Formulation (three-region model, Eq. pbe_vp, discretised BEM(Omega_m) -
FEM(Omega_i) - BEM(Omega_s)).  Unknowns x = [u (shell vertices), lam_m
(Gamma_m vertices), lam_s (Gamma_s vertices)] in reduced units
u = e phi / (kB T).  Block operator (the three-region analogue of
Eq. fembem_matrix; FEM row from the weak form of Sec. 2.2 with the flux
conditions of Eq. pbe_vp, Gamma_m row from Sec. 2.3.1, Gamma_s row from the
Yukawa BIE of Sec. 2.2):

  [ A + J          eps_m R_m^T M_m     -eps_s R_s^T M_s ] [u    ]   [ 0           ]
  [ (M_m/2 + K_L) R_m    -V_L                0          ] [lam_m] = [ <u_coul,psi> ]
  [ (M_s/2 - K_Y) R_s     0                 V_Y         ] [lam_s]   [ 0           ]

with u_coul(x) = (l_B / eps_m) sum_k z_k / |x - x_k|, l_B = C / (kB T).

Nonlinear system (Eq. general_nonlinear): Acal(0) x + [N(u); 0; 0] = b.
Solve order (Sec. 2.4): linear part x_L (Eq. Ec_phi_T with N = u), then Newton
(Eqs. NR_main, Ec_NL_NR, Norma_Newton-Raphson) on x_NL with the T3 scheme in
the first iteration and sinh afterwards, the relaxation factor chosen by
Newton's method on f_d (Eq. fd=0, Appendix A), the L_e skip rule and the
adjustable GMRES tolerance (Appendix B).  Energy: Eq. Esolv with the reaction
potential of Eq. Potential_in_Omega_m and the Delta G_{Omega_i} integral.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, bem

# e^2 / (4 pi eps0) in kcal mol^-1 Angstrom, and kB in kcal mol^-1 K^-1.
COULOMB = 332.0637
KB = 0.0019872043


@dataclasses.dataclass
class Opts:
    """Solver options (defaults: the paper's best Newton configuration, Appendix B)."""
    tol_nl: float = 1e-3          # Tol_NL on e_k = omega ||Delta||_2 (Eq. Norma_Newton-Raphson)
    tol_gmres: float = 1e-6       # final Tol_GR
    tol_gmres0: float = 1e-3      # Tol_GR0 (linear part and early iterations)
    tol_omega: float = 0.1        # Tol_omega on |f_d|
    L_e: float = 0.35             # skip the omega search when e_k < L_e
    omega0_first: float = 2.0     # initial omega for the T3 iteration
    omega0_rest: float = 1.0      # initial omega afterwards
    omega_max: float = 4.0
    max_newton: int = 50
    max_gmres: int = 1000
    restart: int = 200
    max_omega_iters: int = 30
    taylor: tuple = ('T3',)       # schemes of the first iterations, then sinh (Sec. 3.2: T3-HS)
    linear_solver: str = 'gmres'  # 'gmres' (the paper's) or 'direct' (sparse LU)
    omega_search: bool = True     # False: constant omega = omega0_* every iteration
    method: str = 'newton'        # 'newton' (Sec. 2.4.2) or 'picard' (Sec. 2.4.1)
    omega_warm_start: bool = False  # Newton, first iteration: bisection + secant start (Sec. 3.5)
    R_e: float = 1.4              # Picard: recompute omega only when e_{k-1} / e_k < R_e (0 = always)
    accept_ratio: float = 1.0     # accept omega when ||d(omega)||^2 < accept_ratio ||d(0)||^2 (1: Sec. 2.5.2)


class Problem:
    """Assembled three-region problem for one mesh and one parameter set."""

    def __init__(self, case, eps_in=None, eps_out=None, kappa=None, T=None, bem_cache=None):
        self.case = case
        self.eps_m = case.eps_in if eps_in is None else eps_in
        self.eps_s = case.eps_out if eps_out is None else eps_out
        self.kappa = case.kappa if kappa is None else kappa
        self.T = case.T if T is None else T
        self.kT = KB * self.T
        self.lB = COULOMB / self.kT
        self.coef = self.eps_s * self.kappa ** 2            # eps_s kappa^2
        xyz, tets = case.xyz, case.tets
        self.xyz, self.tets = xyz, tets
        self.nv = xyz.shape[0]
        self.sm = bem.Surface(xyz, case.gm_tris)
        self.ss = bem.Surface(xyz, case.gs_tris)
        self.nm, self.ns = self.sm.n, self.ss.n
        self.n = self.nv + self.nm + self.ns
        self.A = fem.stiffness(xyz, tets, self.eps_s)
        self.Mm = bem.mass_matrix(self.sm)
        self.Ms = bem.mass_matrix(self.ss)
        self.Rm = sp.csr_matrix((np.ones(self.nm), (np.arange(self.nm), self.sm.verts)), shape=(self.nm, self.nv))
        self.Rs = sp.csr_matrix((np.ones(self.ns), (np.arange(self.ns), self.ss.verts)), shape=(self.ns, self.nv))
        if bem_cache is not None and ('L', id(case)) in bem_cache:
            self.VL, self.KL = bem_cache[('L', id(case))]
        else:
            self.VL, self.KL = bem.assemble(self.sm, 0.0)
            if bem_cache is not None:
                bem_cache[('L', id(case))] = (self.VL, self.KL)
        key = ('Y', id(case), self.kappa)
        if bem_cache is not None and key in bem_cache:
            self.VY, self.KY = bem_cache[key]
        else:
            self.VY, self.KY = bem.assemble(self.ss, self.kappa)
            if bem_cache is not None:
                bem_cache[key] = (self.VY, self.KY)
        # right-hand side: <u_coul, psi_i> on Gamma_m
        self.b = np.zeros(self.n)
        self.b[self.nv:self.nv + self.nm] = (self.lB / self.eps_m) * bem.coulomb_rhs(
            self.sm, case.q_xyz, case.q_z)
        # constant coupling blocks
        self.B_um = self.eps_m * (self.Rm.T @ self.Mm)
        self.B_us = -self.eps_s * (self.Rs.T @ self.Ms)

    # ---- pieces of the vector
    def split(self, x):
        return x[:self.nv], x[self.nv:self.nv + self.nm], x[self.nv + self.nm:]

    def apply(self, x, Jmat=None):
        """y = Acal(J) x; Jmat None means J = 0 (the operator Acal of Eq. general_nonlinear)."""
        u, lm, ls = self.split(x)
        yu = self.A @ u + self.B_um @ lm + self.B_us @ ls
        if Jmat is not None:
            yu = yu + Jmat @ u
        um, us = u[self.sm.verts], u[self.ss.verts]
        ym = 0.5 * (self.Mm @ um) + self.KL @ um - self.VL @ lm
        ys = 0.5 * (self.Ms @ us) - self.KY @ us + self.VY @ ls
        return np.concatenate([yu, ym, ys])

    def matrix(self, Jmat=None):
        """Assembled sparse Acal(J) (BEM blocks dense inside a sparse container)."""
        Auu = self.A if Jmat is None else self.A + Jmat
        Rm, Rs = self.Rm, self.Rs
        Bmu = sp.csr_matrix(0.5 * self.Mm.toarray() + self.KL) @ Rm
        Bsu = sp.csr_matrix(0.5 * self.Ms.toarray() - self.KY) @ Rs
        return sp.bmat([[Auu, self.B_um, self.B_us],
                        [Bmu, sp.csr_matrix(-self.VL), None],
                        [Bsu, None, sp.csr_matrix(self.VY)]], format='csc')

    def jacobi(self, Jmat=None):
        """Diagonal of Acal(J): the right preconditioner used by GMRES."""
        dA = self.A.diagonal() + (0.0 if Jmat is None else Jmat.diagonal())
        return np.concatenate([dA, -np.diag(self.VL), np.diag(self.VY)])

    # ---- nonlinear pieces (zero outside the FEM rows)
    def N(self, u, scheme):
        return fem.nonlinear_load(self.xyz, self.tets, u, scheme, self.coef)

    def J(self, u, scheme):
        return fem.jacobian(self.xyz, self.tets, u, scheme, self.coef)

    def N2(self, u, d, scheme):
        return fem.second_derivative_load(self.xyz, self.tets, u, d, scheme, self.coef)

    def pad(self, vu):
        out = np.zeros(self.n)
        out[:self.nv] = vu
        return out


def gmres(apply, b, tol, restart=200, maxit=1000, diag=None):
    """Restarted GMRES, x0 = 0, stop when ||b - A x|| <= tol ||b||.

    Right preconditioned by diag (x = z / diag).  Arnoldi uses classical
    Gram-Schmidt applied twice; the least-squares problem is updated with
    Givens rotations.  Returns (x, iterations, relative residual).
    """
    n = b.size
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    dinv = np.ones(n) if diag is None else 1.0 / diag
    its = 0
    r = b.copy()
    rel = 1.0
    while its < maxit:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for k in range(restart):
            w = apply(dinv * V[k])
            h = V[:k + 1] @ w
            w = w - V[:k + 1].T @ h
            h2 = V[:k + 1] @ w
            w = w - V[:k + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:k + 1, k] = h
            H[k + 1, k] = hn
            if hn > 0:
                V[k + 1] = w / hn
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            rel = abs(g[k + 1]) / bn
            if rel <= tol or its >= maxit:
                break
        m = k + 1
        y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
        x = x + dinv * (V[:m].T @ y)
        r = b - apply(x)
        rel = np.linalg.norm(r) / bn
        if rel <= tol:
            break
    return x, its, rel


def linear_solve(P: Problem, Jmat, rhs, tol, opts: Opts):
    """Solve Acal(J) x = rhs at relative tolerance tol; returns (x, iterations)."""
    if opts.linear_solver == 'direct':
        return spla.spsolve(P.matrix(Jmat), rhs), 0
    x, its, rel = gmres(lambda v: P.apply(v, Jmat), rhs, tol, opts.restart, opts.max_gmres,
                        P.jacobi(Jmat))
    if rel > tol:
        raise RuntimeError(f'GMRES did not converge: rel {rel:.3e} > {tol:.1e} after {its}')
    return x, its


def omega_dots(P: Problem, u, du, c, p, omega, scheme):
    """Scalars of the omega search at one omega (Eq. ab_pic, Eq. fd=0, Appendix A).

    r = c - [N(u + omega du); 0; 0], r' = -[J(u + omega du) du; 0; 0],
    r'' = -[N''(u + omega du)[du, du]; 0; 0].
    Returns dict with PR=(p+r').r, PP=(p+r').p, PRp=(p+r').r', RRpp=r.r'',
    PRpp=p.r'', RR=r.r, pp=p.p.
    """
    w = u + omega * du
    r = c - P.pad(P.N(w, scheme))
    rp = -P.pad(P.J(w, scheme) @ du)
    rpp = -P.pad(P.N2(w, du, scheme))
    Pv = p + rp
    return dict(PR=Pv @ r, PP=Pv @ p, PRp=Pv @ rp, RRpp=r @ rpp, PRpp=p @ rpp, RR=r @ r, pp=p @ p, pr=p @ r)


def fd_and_derivative(D, omega):
    """f_d(omega) (Eq. fd=0) and its derivative (Appendix A) from the omega_dots scalars."""
    f = -D['PR'] / D['PP'] - omega
    fp = -(D['PRp'] + D['RRpp']) / D['PP'] + D['PR'] * D['PRpp'] / D['PP'] ** 2 - 1.0
    return f, fp


def dnorm2(D, omega):
    """||d(omega)||^2 = ||omega p + r(omega)||^2 from the dot products."""
    return omega * omega * D['pp'] + 2.0 * omega * D['pr'] + D['RR']


def omega_search(P: Problem, u, du, c, p, d0n2, scheme, omega0, opts: Opts, trace):
    """Optimal relaxation factor: Newton on f_d from omega0 until |f_d| < Tol_omega
    (Appendix A), accepted only if 0 < omega <= omega_max and ||d(omega)|| < ||d(0)||
    (the global convergence condition of Sec. 2.5.2).  Otherwise: scan
    g_d = d.d' = -(p+r').p f_d at omega_max j / 16 (j = 1..16), bisect the first
    sign change 20 times, and accept on the same decrease test."""
    om = omega0
    ok = False
    evals = 0
    for _ in range(opts.max_omega_iters):
        D = omega_dots(P, u, du, c, p, om, scheme)
        evals += 1
        if not np.isfinite(D['PP']) or abs(D['PP']) < 1e-300:
            break
        f, fp = fd_and_derivative(D, om)
        if not np.isfinite(f):
            break
        if abs(f) < opts.tol_omega:
            ok = 0.0 < om <= opts.omega_max and np.isfinite(dnorm2(D, om)) and dnorm2(D, om) < d0n2
            break
        if not np.isfinite(fp) or fp == 0.0:
            break
        om = om - f / fp
        if not np.isfinite(om):
            break
    if not ok:
        om = _fallback(P, u, du, c, p, d0n2, scheme, opts)
        evals += 38
        trace['fallback'] = trace.get('fallback', 0) + 1
    trace['omega_evals'].append(evals)
    return om


def warm_start_omega(P: Problem, u, du, c, p, scheme, opts: Opts, trace):
    """Initial guess of the first Newton iteration's omega (Sec. 3.5, the 1HC8 optimisation):
    three bisection steps of f_d on [2, 3] (f_d decreases through its root, so f_d > 0 moves
    right), then secant steps (Eq. Met_Secante, standard form) until two iterates differ by less
    than 0.05.  Returns omega0_first when a step is not finite."""
    def fd(o):
        return fd_and_derivative(omega_dots(P, u, du, c, p, o, scheme), o)[0]
    lo, hi = 2.0, 3.0
    pts = []
    for _ in range(3):
        mid = 0.5 * (lo + hi)
        f = fd(mid)
        pts.append((mid, f))
        if not np.isfinite(f):
            trace['omega_evals_warm'] = len(pts)
            return opts.omega0_first
        if f > 0.0:
            lo = mid
        else:
            hi = mid
    (o_prev, f_prev), (o_cur, f_cur) = pts[-2], pts[-1]
    evals = 3
    o_next = o_cur
    for _ in range(opts.max_omega_iters):
        den = f_prev - f_cur
        if den == 0.0 or not np.isfinite(den):
            break
        o_next = o_prev - (o_prev - o_cur) * f_prev / den
        if not np.isfinite(o_next):
            o_next = opts.omega0_first
            break
        if abs(o_next - o_cur) < 0.05:
            break
        o_prev, f_prev, o_cur = o_cur, f_cur, o_next
        f_cur = fd(o_cur)
        evals += 1
        if not np.isfinite(f_cur):
            o_next = opts.omega0_first
            break
    trace['omega_evals_warm'] = evals
    return o_next


def picard_omega(P: Problem, u, du, c, p, d0n2, scheme, omega0, opts: Opts, trace):
    """Relaxation factor of a Picard step: the direct secant of Appendix A (Eq. SEC_FD) through
    (0, f_d(0) = 1) and (omega0, f_d(omega0)), continued by secant steps (Eq. Met_Secante) until
    |f_d| < Tol_omega; accepted under the same decrease test as the Newton search, else the same
    scan-and-bisect fallback."""
    o_prev, f_prev = 0.0, 1.0
    o_cur = omega0
    D = omega_dots(P, u, du, c, p, o_cur, scheme)
    f_cur = fd_and_derivative(D, o_cur)[0]
    evals = 1
    ok = False
    for _ in range(opts.max_omega_iters):
        if not np.isfinite(f_cur):
            break
        if abs(f_cur) < opts.tol_omega:
            dn = dnorm2(D, o_cur)
            ok = 0.0 < o_cur <= opts.omega_max and np.isfinite(dn) and dn < d0n2
            break
        den = f_prev - f_cur
        if den == 0.0 or not np.isfinite(den):
            break
        o_next = o_prev - (o_prev - o_cur) * f_prev / den
        if not np.isfinite(o_next):
            break
        o_prev, f_prev, o_cur = o_cur, f_cur, o_next
        D = omega_dots(P, u, du, c, p, o_cur, scheme)
        f_cur = fd_and_derivative(D, o_cur)[0]
        evals += 1
    if ok:
        trace['omega_evals'].append(evals)
        return o_cur
    om = _fallback(P, u, du, c, p, d0n2, scheme, opts)
    trace['fallback'] = trace.get('fallback', 0) + 1
    trace['omega_evals'].append(evals + 38)
    return om


def _fallback(P, u, du, c, p, d0n2, scheme, opts):
    """Scan g_d at omega_max j / 16 and bisect the first sign change (reading R10)."""
    def gd(o):
        D = omega_dots(P, u, du, c, p, o, scheme)
        return o * D['PP'] + D['PR']
    lo, hi = 0.0, None
    for j in range(1, 17):
        o = opts.omega_max * j / 16.0
        g = gd(o)
        if not np.isfinite(g) or g >= 0.0:
            hi = o
            break
        lo = o
    if hi is None:
        om = opts.omega_max
    else:
        for _ in range(20):
            mid = 0.5 * (lo + hi)
            g = gd(mid)
            if np.isfinite(g) and g < 0.0:
                lo = mid
            else:
                hi = mid
        om = 0.5 * (lo + hi)
    D = omega_dots(P, u, du, c, p, om, scheme)
    if not (np.isfinite(dnorm2(D, om)) and dnorm2(D, om) < d0n2):
        raise RuntimeError('omega search failed')
    return om


@dataclasses.dataclass
class Result:
    x: np.ndarray
    xL: np.ndarray
    xNL: np.ndarray
    total: float
    LC: float
    NC: float
    dG_ion: float
    newton_iters: int
    trace: dict


def reaction_potential(P: Problem, x):
    """u_r(x_k) = (V_L lam_m)(x_k) - (K_L u)(x_k) at the charges (Eq. Potential_in_Omega_m)."""
    u, lm, _ = P.split(x)
    return bem.layer_potentials_at(P.sm, P.case.q_xyz, lm, u[P.sm.verts])


def energy(P: Problem, xL, xNL):
    """(Total, LC, NC, dG_ion) in kcal/mol (Eq. Esolv, Eq. Esolv_Lineal).

    LC = kT/2 sum z_k u_r[x_L](x_k), NC = kT/2 sum z_k u_r[x_NL](x_k),
    dG_ion = kT c0 int (u sinh u - 2 cosh u + 2), c0 = eps_s kappa^2 / (8 pi l_B)
    (the paper's (1/2) eps_s kappa^2 prefactor expressed in reduced units).
    """
    z = P.case.q_z
    if hasattr(P, 'reaction_potentials'):
        # a problem whose unknowns hold no lam_m computes u_r itself (solute.SoluteProblem)
        urL, urNL = P.reaction_potentials(xL, xNL)
    else:
        urL, urNL = reaction_potential(P, xL), reaction_potential(P, xNL)
    LC = 0.5 * P.kT * float(z @ urL)
    NC = 0.5 * P.kT * float(z @ urNL)
    c0 = P.coef / (8.0 * np.pi * P.lB)
    u = (xL + xNL)[:P.nv]
    dG = P.kT * c0 * fem.ion_energy_integral(P.xyz, P.tets, u)
    return LC + NC + dG, LC, NC, dG


def solve(P: Problem, opts: Opts = None, linear_only=False):
    """Full solve: linear part, Newton loop with the omega search, energy."""
    opts = opts or Opts()
    trace = dict(gmres=[], omega=[], e=[], omega_evals=[], scheme=[], dnorm=[], tol_gmres=[])
    tol = opts.tol_gmres0
    Mlin = P.J(np.zeros(P.nv), 'linear')                      # eps_s kappa^2 M (F' = 1)
    xL, its = linear_solve(P, Mlin, P.b, tol, opts)
    trace['linear_gmres'] = its
    xNL = np.zeros(P.n)
    if linear_only:
        # Eq. Esolv_Lineal: the linear energy is the reaction-potential term alone
        _, LC, _, _ = energy(P, xL, xNL)
        return Result(xL, xL, xNL, LC, LC, 0.0, 0.0, 0, trace)
    om_last = None
    e_prev = None
    k = 0
    picard = opts.method == 'picard'
    e_prev2 = None
    for k in range(opts.max_newton):
        scheme = opts.taylor[k] if k < len(opts.taylor) else 'HS'
        Phi = xL + xNL
        u = Phi[:P.nv]
        Nu = P.N(u, scheme)
        c = P.b - P.apply(Phi)                                  # b - Acal(0) Phi
        d = c - P.pad(Nu)
        if not d.any():
            # the iterate solves Eq. NR_main's system exactly (e.g. no charges): Delta = 0 for every
            # omega, so e_k = 0 < Tol_NL (Sec. 3.5) and no relaxation factor is searched for
            for key, v in (('gmres', 0), ('scheme', scheme), ('dnorm', 0.0), ('omega', 0.0), ('e', 0.0),
                           ('omega_evals', 0), ('tol_gmres', tol)):
                trace[key].append(v)
            break
        # Newton: Acal(J) Delta = d (Eq. NR_main); Picard: Acal(0) Delta = d, Delta = Phi~ - Phi_NL
        # (Eq. Ec_NL_Previo2 written for the increment)
        Jm = None if picard else P.J(u, scheme)
        du, its = linear_solve(P, Jm, d, tol, opts)
        trace['gmres'].append(its)
        trace['tol_gmres'].append(tol)
        trace['scheme'].append(scheme)
        trace['dnorm'].append(float(np.linalg.norm(d)))
        if not opts.omega_search:
            om = opts.omega0_first if k == 0 else opts.omega0_rest
        elif (not picard) and k > 0 and e_prev is not None and e_prev < opts.L_e and om_last is not None:
            om = om_last
            trace['omega_evals'].append(0)
        elif picard and om_last is not None and e_prev2 is not None and opts.R_e > 0 \
                and not (e_prev2 / e_prev < opts.R_e):
            # R_e rule (Appendix B): keep omega while the error still falls by R_e per step
            om = om_last
            trace['omega_evals'].append(0)
        else:
            p = -P.apply(du)
            om0 = opts.omega0_first if k == 0 else opts.omega0_rest
            if k == 0 and opts.omega_warm_start and not picard:
                om0 = warm_start_omega(P, u, du[:P.nv], c, p, scheme, opts, trace)
            # the global convergence condition of Sec. 2.5.2, ||d(omega)|| < ||d(0)||, scaled by
            # accept_ratio (1: the paper's condition; below 1 a sufficient decrease)
            d0n2 = opts.accept_ratio * float(d @ d)
            if picard:
                om = picard_omega(P, u, du[:P.nv], c, p, d0n2, scheme, om0, opts, trace)
            else:
                om = omega_search(P, u, du[:P.nv], c, p, d0n2, scheme, om0, opts, trace)
        om_last = om
        xNL = xNL + om * du
        e = om * float(np.linalg.norm(du))
        trace['omega'].append(om)
        trace['e'].append(e)
        e_prev2 = e_prev
        e_prev = e
        if e < 1250.0 * tol:
            tol = max(0.1 * tol, opts.tol_gmres)
        if e < opts.tol_nl:
            break
    else:
        raise RuntimeError('nonlinear iteration did not converge')
    t, LC, NC, dG = energy(P, xL, xNL)
    return Result(xL + xNL, xL, xNL, t, LC, NC, dG, k + 1, trace)
