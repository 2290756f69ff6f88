"""Pins for the oracle's P1 finite-element pieces (no GPU).

Independent checks: the exact Dirichlet energy and second moments of linear
fields over the polyhedral shell (closed-form per-tet formulas), the shell
volume by the divergence theorem over its two boundary surfaces, and
central finite differences for the Jacobian and the second derivative.
"""
import numpy as np
import pytest

from oracle import fem


def _poly_volume(xyz, tris):
    """Signed volume enclosed by an outward-oriented triangulated surface."""
    P = xyz[tris]
    return np.sum(np.einsum('ij,ij->i', P[:, 0], np.cross(P[:, 1], P[:, 2]))) / 6.0


def test_stiffness_symmetric_rowsums_and_linear_energy(tiny_case):
    c = tiny_case
    A = fem.stiffness(c.xyz, c.tets, 80.0)
    assert abs(A - A.T).max() < 1e-12 * abs(A).max()
    assert np.abs(A @ np.ones(c.n_v)).max() < 1e-12 * abs(A).max()
    vol = _poly_volume(c.xyz, c.gs_tris) - _poly_volume(c.xyz, c.gm_tris)
    for k in range(3):
        x = c.xyz[:, k]
        # |grad x|^2 = 1 everywhere: x^T A x = eps * volume
        assert abs(x @ (A @ x) - 80.0 * vol) < 1e-10 * 80 * vol
    # positive semi-definite on a random vector
    r = np.random.default_rng(0).standard_normal(c.n_v)
    assert r @ (A @ r) > 0


def test_mass_from_jacobian_matches_closed_forms(tiny_case):
    c = tiny_case
    coef = 3.0
    M = fem.jacobian(c.xyz, c.tets, np.zeros(c.n_v), 'linear', coef) / coef
    one = np.ones(c.n_v)
    vol = _poly_volume(c.xyz, c.gs_tris) - _poly_volume(c.xyz, c.gm_tris)
    assert abs(one @ M @ one - vol) < 1e-12 * vol
    # int x^2 over each tet = |T|/20 (sum x_i^2 + (sum x_i)^2)   (exact for P1 geometry)
    x = c.xyz[:, 0]
    X = x[c.tets]
    vols, _ = fem.tet_geometry(c.xyz, c.tets)
    exact = np.sum(vols / 20.0 * (np.sum(X * X, 1) + np.sum(X, 1) ** 2))
    assert abs(x @ M @ x - exact) < 1e-12 * exact
    assert abs(M - M.T).max() < 1e-15


def test_linear_scheme_load_is_mass_times_u(tiny_case):
    c = tiny_case
    u = np.sin(c.xyz[:, 0] / 3.0) + 0.1 * c.xyz[:, 2]
    N = fem.nonlinear_load(c.xyz, c.tets, u, 'linear', 2.0)
    M = fem.jacobian(c.xyz, c.tets, u, 'linear', 2.0)
    assert np.abs(N - M @ u).max() < 1e-12 * np.abs(N).max()


def test_scheme_functions():
    u = np.linspace(-3, 3, 13)
    F, Fp, Fpp = fem.F_scheme('T3', u)
    assert np.allclose(F, u + u ** 3 / 6) and np.allclose(Fp, 1 + u ** 2 / 2) and np.allclose(Fpp, u)
    F, Fp, Fpp = fem.F_scheme('HS', u)
    assert np.allclose(F, (np.exp(u) - np.exp(-u)) / 2) and np.allclose(Fp, (np.exp(u) + np.exp(-u)) / 2)
    # T3 is the cubic Taylor polynomial of sinh: error O(u^5 / 120)
    small = np.linspace(-0.1, 0.1, 5)
    assert np.abs(fem.F_scheme('T3', small)[0] - np.sinh(small)).max() < 1e-7


@pytest.mark.parametrize("scheme", ["T3", "T5", "T7", "HS"])
def test_jacobian_and_second_derivative_by_finite_differences(tiny_case, scheme):
    c = tiny_case
    rng = np.random.default_rng(1)
    r = np.linalg.norm(c.xyz, axis=1)
    u = 4.0 * np.exp(-0.3 * (r - 4.0)) + 0.1 * rng.standard_normal(c.n_v)
    d = rng.standard_normal(c.n_v)
    coef = 1.26
    h = 1e-5
    Np = fem.nonlinear_load(c.xyz, c.tets, u + h * d, scheme, coef)
    Nm = fem.nonlinear_load(c.xyz, c.tets, u - h * d, scheme, coef)
    Jd = fem.jacobian(c.xyz, c.tets, u, scheme, coef) @ d
    fd = (Np - Nm) / (2 * h)
    assert np.linalg.norm(Jd - fd) < 1e-7 * np.linalg.norm(Jd)
    Jp = fem.jacobian(c.xyz, c.tets, u + h * d, scheme, coef) @ d
    Jm = fem.jacobian(c.xyz, c.tets, u - h * d, scheme, coef) @ d
    N2 = fem.second_derivative_load(c.xyz, c.tets, u, d, scheme, coef)
    assert np.linalg.norm(N2 - (Jp - Jm) / (2 * h)) < 1e-6 * np.linalg.norm(N2)


def test_ion_energy_integrand_nonnegative_and_small_u_limit(tiny_case):
    c = tiny_case
    vol = _poly_volume(c.xyz, c.gs_tris) - _poly_volume(c.xyz, c.gm_tris)
    assert fem.ion_energy_integral(c.xyz, c.tets, np.zeros(c.n_v)) == 0.0
    # constant u: integrand is exactly u sinh u - 2 cosh u + 2 times the volume
    for u0 in (0.5, 3.0, -2.0):
        g = u0 * np.sinh(u0) - 2 * np.cosh(u0) + 2
        got = fem.ion_energy_integral(c.xyz, c.tets, np.full(c.n_v, u0))
        assert got > 0 and abs(got - g * vol) < 1e-11 * g * vol
