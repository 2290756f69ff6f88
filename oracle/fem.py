"""P1 finite elements on the solvent shell Omega_i (oracle; test infrastructure only).

Follows the weak form of the Omega_i equation (Sec. 2.2, the integration by
parts that precedes Eq. fembem_matrix) with test function v (the printed
"N(phi) grad v" is read as "N(phi) v"), and the operator split of
Eqs. general_nonlinear / Vector_c:

  A_ij       = eps_s  int grad v_i . grad v_j                (stiffness)
  N(u)_i     = eps_s kappa^2 int F(u_h) v_i                  (nonlinear load)
  J(u)_ij    = eps_s kappa^2 int F'(u_h) v_i v_j             (Jacobian of N, Eq. NR_main)
  N2(u)[D,D]_i = eps_s kappa^2 int F''(u_h) D_h^2 v_i        (Appendix A, [Delta]^2 d^2 N)

with F = u (linear), the Taylor polynomials of sinh of degree 3, 5, 7 (T3, T5,
T7: the schemes of the first iterations) or sinh u (HS), Sec. 3.2 "Gradually
incorporating sinh".
Volume integrals of F use the 14-point rule; stiffness is exact for P1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import tet14


def F_scheme(scheme: str, u: np.ndarray):
    """(F, F', F'') for the nonlinearity of the given scheme at values u."""
    if scheme == 'linear':
        return u, np.ones_like(u), np.zeros_like(u)
    if scheme == 'T3':
        return u + u ** 3 / 6.0, 1.0 + 0.5 * u * u, u
    if scheme == 'T5':
        return (u + u ** 3 / 6.0 + u ** 5 / 120.0, 1.0 + 0.5 * u * u + u ** 4 / 24.0,
                u + u ** 3 / 6.0)
    if scheme == 'T7':
        return (u + u ** 3 / 6.0 + u ** 5 / 120.0 + u ** 7 / 5040.0,
                1.0 + 0.5 * u * u + u ** 4 / 24.0 + u ** 6 / 720.0,
                u + u ** 3 / 6.0 + u ** 5 / 120.0)
    if scheme == 'HS':
        s = np.sinh(u)
        return s, np.cosh(u), s
    raise ValueError(scheme)


def tet_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Volumes (n_t,) and barycentric gradients (n_t, 4, 3) of P1 tets."""
    x = xyz[tets]                                   # (n_t, 4, 3)
    E = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=1)  # rows = edges
    det = np.linalg.det(E)
    vol = np.abs(det) / 6.0
    # grad lambda_{1..3} are the columns of E^{-1}; grad lambda_0 = -sum
    Einv = np.linalg.inv(E)                         # (n_t, 3, 3)
    g123 = np.transpose(Einv, (0, 2, 1))            # row k = grad lambda_{k+1}
    g0 = -g123.sum(axis=1, keepdims=True)
    return vol, np.concatenate([g0, g123], axis=1)


def _scatter_matrix(tets, local, n_v):
    """Sparse (n_v x n_v) sum of element matrices local (n_t, 4, 4)."""
    rows = np.repeat(tets, 4, axis=1).reshape(-1)
    cols = np.tile(tets, (1, 4)).reshape(-1)
    return sp.csr_matrix((local.reshape(-1), (rows, cols)), shape=(n_v, n_v))


def stiffness(xyz, tets, eps_s):
    """A_ij = eps_s sum_T |T| grad l_i . grad l_j (exact for P1)."""
    vol, g = tet_geometry(xyz, tets)
    loc = eps_s * vol[:, None, None] * np.einsum('tik,tjk->tij', g, g)
    return _scatter_matrix(tets, loc, xyz.shape[0])


def _qp_values(tets, lam, u):
    """u_h at the 14 quadrature points of every tet: (n_t, 14)."""
    return u[tets] @ lam.T


def nonlinear_load(xyz, tets, u, scheme, coef):
    """N(u)_i = coef * int F(u_h) v_i, coef = eps_s kappa^2."""
    lam, w = tet14()
    vol, _ = tet_geometry(xyz, tets)
    F, _, _ = F_scheme(scheme, _qp_values(tets, lam, u))
    loc = coef * vol[:, None] * ((F * w[None, :]) @ lam)          # (n_t, 4)
    return np.bincount(tets.reshape(-1), loc.reshape(-1), minlength=xyz.shape[0])


def jacobian(xyz, tets, u, scheme, coef):
    """J(u)_ij = coef * int F'(u_h) v_i v_j (sparse)."""
    lam, w = tet14()
    vol, _ = tet_geometry(xyz, tets)
    _, Fp, _ = F_scheme(scheme, _qp_values(tets, lam, u))
    g = coef * vol[:, None] * Fp * w[None, :]                      # (n_t, 14)
    loc = np.einsum('tq,qi,qj->tij', g, lam, lam)
    return _scatter_matrix(tets, loc, xyz.shape[0])


def second_derivative_load(xyz, tets, u, d, scheme, coef):
    """N2(u)[d,d]_i = coef * int F''(u_h) d_h^2 v_i."""
    lam, w = tet14()
    vol, _ = tet_geometry(xyz, tets)
    _, _, Fpp = F_scheme(scheme, _qp_values(tets, lam, u))
    dq = _qp_values(tets, lam, d)
    loc = coef * vol[:, None] * ((Fpp * dq * dq * w[None, :]) @ lam)
    return np.bincount(tets.reshape(-1), loc.reshape(-1), minlength=xyz.shape[0])


def ion_energy_integral(xyz, tets, u):
    """int_{Omega_i} (u sinh u - 2 cosh u + 2) dx by the 14-point rule
    (the Delta G_{Omega_i} integrand of Sec. 2.3)."""
    lam, w = tet14()
    vol, _ = tet_geometry(xyz, tets)
    uq = _qp_values(tets, lam, u)
    g = uq * np.sinh(uq) - 2.0 * np.cosh(uq) + 2.0
    return float(np.sum(vol * (g @ w)))
