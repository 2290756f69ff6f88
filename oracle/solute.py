"""The paper's own formulation: FEM over Omega_m and Omega_i, Yukawa BEM on Gamma_s, and the
reaction potential from a Laplace boundary integral equation on Gamma_m (oracle; test
infrastructure only).

Discrete system (Sec. 2.2, Eq. fembem_matrix), unknowns x = [u (all vertices of the mesh of
Omega_m and Omega_i), lam_s (Gamma_s vertices)], reduced units u = e phi / (kB T):

  [ A~ + J          -eps_s R_s^T M_s ] [u    ]   [ rho ]
  [ (M_s/2 - K_Y) R_s      V_Y       ] [lam_s] = [ 0   ]

with A~_ij = sum_T eps_T int_T grad v_i . grad v_j (eps_m in Omega_m, eps_s in Omega_i), the
nonlinear term N, J only on the tets of Omega_i (kappa = 0 in Omega_m), and the point charges as
the load rho_i = 4 pi l_B sum_k z_k v_i(x_k) (the weak form's int rho_c v for
rho_c = 4 pi l_B sum_k z_k delta(x - x_k) in reduced units).

Reaction potential (Sec. 2.3.1, Eq. Potential_in_Omega_m and the Gamma_m trace equation after
it): with the trace of u on Gamma_m, lam_m solves

  V_L lam_m = (M_m/2 + K_L) u|Gamma_m - <u_coul, psi>,   u_coul = (l_B / eps_m) sum_k z_k / |x - x_k|,

and u_r(x_k) = (V_L lam_m)(x_k) - (K_L u)(x_k).  The energy splits as in Eq. Esolv: LC from the
linear part x_L (lam_m with the Coulomb term), NC from x_NL (lam_m of its trace alone, the map
being affine), and Delta G_{Omega_i} over the tets of Omega_i.

``SoluteProblem`` offers the interface ``pb.solve`` uses, so the linear part, the Newton (or
Picard) iteration and the relaxation-factor search run unchanged on it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bem, fem
from .pb import COULOMB, KB


def point_load(xyz, tets, q_xyz, q_z):
    """sum_k z_k v_i(x_k) for the P1 hat functions v_i: each charge is located in a tet whose
    barycentric coordinates of it are all >= -1e-12 (any of them where it lies on a shared face,
    the hat functions being continuous) and adds z_k lambda_a(x_k) to the tet's vertex a.
    Raises ValueError when a charge lies in none of the tets."""
    vol, g = fem.tet_geometry(xyz, tets)
    x0 = xyz[tets[:, 0]]
    out = np.zeros(xyz.shape[0])
    for x, z in zip(np.asarray(q_xyz).reshape(-1, 3), q_z):
        lam = np.einsum('tad,td->ta', g, x[None, :] - x0)
        lam[:, 0] += 1.0
        inside = np.nonzero(lam.min(axis=1) >= -1e-12)[0]
        if inside.size == 0:
            raise ValueError('charge outside the tets of Omega_m')
        t = inside[0]
        out[tets[t]] += z * lam[t]
    return out


class SoluteProblem:
    """Assembled FEM(Omega_m and Omega_i)-BEM(Gamma_s) problem for one mesh and parameter set."""

    def __init__(self, case, eps_in=None, eps_out=None, kappa=None, T=None, bem_cache=None):
        if case.tet_region is None:
            raise ValueError('the case has no Omega_m tets')
        self.case = case
        self.eps_m = case.eps_in if eps_in is None else eps_in
        self.eps_s = case.eps_out if eps_out is None else eps_out
        self.kappa = case.kappa if kappa is None else kappa
        self.T = case.T if T is None else T
        self.kT = KB * self.T
        self.lB = COULOMB / self.kT
        self.coef = self.eps_s * self.kappa ** 2
        region = np.asarray(case.tet_region)
        self.xyz = case.xyz
        self.tets = case.tets[region == 1]          # Omega_i: the nonlinear term and Delta G_{Omega_i}
        self.tets_m = case.tets[region == 0]        # Omega_m: eps_m, no ions
        self.nv = self.xyz.shape[0]
        self.sm = bem.Surface(self.xyz, case.gm_tris)
        self.ss = bem.Surface(self.xyz, case.gs_tris)
        self.nm, self.ns = self.sm.n, self.ss.n
        self.n = self.nv + self.ns
        self.A = fem.stiffness(self.xyz, self.tets, self.eps_s) + fem.stiffness(self.xyz, self.tets_m, self.eps_m)
        self.Mm = bem.mass_matrix(self.sm)
        self.Ms = bem.mass_matrix(self.ss)
        self.Rs = sp.csr_matrix((np.ones(self.ns), (np.arange(self.ns), self.ss.verts)), shape=(self.ns, self.nv))
        key_l, key_y = ('SL', id(case)), ('SY', id(case), self.kappa)
        if bem_cache is not None and key_l in bem_cache:
            self.VL, self.KL = bem_cache[key_l]
        else:
            self.VL, self.KL = bem.assemble(self.sm, 0.0)
            if bem_cache is not None:
                bem_cache[key_l] = (self.VL, self.KL)
        if bem_cache is not None and key_y in bem_cache:
            self.VY, self.KY = bem_cache[key_y]
        else:
            self.VY, self.KY = bem.assemble(self.ss, self.kappa)
            if bem_cache is not None:
                bem_cache[key_y] = (self.VY, self.KY)
        self.rho = 4.0 * np.pi * self.lB * point_load(self.xyz, self.tets_m, case.q_xyz, case.q_z)
        self.b = np.concatenate([self.rho, np.zeros(self.ns)])
        self.coul = (self.lB / self.eps_m) * bem.coulomb_rhs(self.sm, case.q_xyz, case.q_z)
        self.B_us = -self.eps_s * (self.Rs.T @ self.Ms)

    def split(self, x):
        return x[:self.nv], x[self.nv:]

    def apply(self, x, Jmat=None):
        """y = Acal(J) x (Eq. fembem_matrix); Jmat None means J = 0."""
        u, ls = self.split(x)
        yu = self.A @ u + self.B_us @ ls
        if Jmat is not None:
            yu = yu + Jmat @ u
        us = u[self.ss.verts]
        ys = 0.5 * (self.Ms @ us) - self.KY @ us + self.VY @ ls
        return np.concatenate([yu, ys])

    def matrix(self, Jmat=None):
        Auu = self.A if Jmat is None else self.A + Jmat
        Bsu = sp.csr_matrix(0.5 * self.Ms.toarray() - self.KY) @ self.Rs
        return sp.bmat([[Auu, self.B_us], [Bsu, sp.csr_matrix(self.VY)]], format='csc')

    def jacobi(self, Jmat=None):
        dA = self.A.diagonal() + (0.0 if Jmat is None else Jmat.diagonal())
        return np.concatenate([dA, np.diag(self.VY)])

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

    # ---- reaction potential (Sec. 2.3.1)
    def lam_m(self, u, coulomb=True):
        """lam_m from V_L lam_m = (M_m/2 + K_L) u|Gamma_m - <u_coul, psi> (dense solve); without
        the Coulomb term for the nonlinear part of an affine split."""
        um = u[self.sm.verts]
        rhs = 0.5 * (self.Mm @ um) + self.KL @ um
        if coulomb:
            rhs = rhs - self.coul
        return np.linalg.solve(self.VL, rhs)

    def expand(self, x, coulomb=True):
        """[u, lam_m, lam_s]: the vector with the post-processed lam_m inserted (the layout of
        the three-region unknowns)."""
        u, ls = self.split(x)
        return np.concatenate([u, self.lam_m(u, coulomb), ls])

    def reaction_potentials(self, xL, xNL):
        """u_r at the charges of the linear part (with the Coulomb term) and of the nonlinear
        part (without it): Eq. Potential_in_Omega_m."""
        out = []
        for x, coulomb in ((xL, True), (xNL, False)):
            u = x[:self.nv]
            out.append(bem.layer_potentials_at(self.sm, self.case.q_xyz, self.lam_m(u, coulomb), u[self.sm.verts]))
        return out[0], out[1]
