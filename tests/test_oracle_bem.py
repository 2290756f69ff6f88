"""Pins for the oracle's Galerkin boundary operators (no GPU).

Independent checks on spheres: the constant-density double-layer jump of
-1/2 (Gauss), the closed-form single- and double-layer potentials of a
uniform density on a sphere (Laplace and Yukawa), Green's representation
identities for exact harmonic / Yukawa fields (interior Laplace row and
exterior Yukawa row of the coupled system), the surface area, and the
Coulomb right-hand side against its continuum value.
"""
import numpy as np
import pytest

from oracle import bem


@pytest.fixture(scope="module")
def sphere_ops(tiny_case, bem_cache):
    c = tiny_case
    out = {}
    for name, tris, kap in (("m", c.gm_tris, 0.0), ("s", c.gs_tris, 0.125)):
        s = bem.Surface(c.xyz, tris)
        key = ("oracle-bem-test", name, c.name, kap)
        if key not in bem_cache:
            bem_cache[key] = bem.assemble(s, kap)
        V, K = bem_cache[key]
        out[name] = (s, bem.mass_matrix(s), V, K, kap)
    return out


def test_mass_matrix_sums_to_area(sphere_ops):
    s, M, _, _, _ = sphere_ops["m"]
    assert abs(M.sum() - s.area.sum()) < 1e-12 * s.area.sum()
    assert abs(M - M.T).max() == 0.0


def test_double_layer_constant_jump(sphere_ops):
    s, M, _, K, _ = sphere_ops["m"]
    one = np.ones(s.n)
    ratio = (K @ one) / (M @ one)
    assert np.abs(ratio + 0.5).max() < 5e-5


def test_uniform_density_on_sphere_closed_forms(sphere_ops):
    # Laplace: V 1 = a (M 1);  Yukawa: V 1 = (1 - e^{-2 k a})/(2k) M 1,
    # K 1 = -(1/(4a)) [2/k - (2a + 2/k) e^{-2 k a}] M 1   (integrals over the sphere)
    s, M, V, _, _ = sphere_ops["m"]
    one = np.ones(s.n)
    a = np.linalg.norm(s.P[0, 0])
    assert np.abs((V @ one) / (M @ one) / a - 1).max() < 2.5e-2        # O(h^2) polyhedral error at nu = 3
    s, M, V, K, k = sphere_ops["s"]
    one = np.ones(s.n)
    a = np.linalg.norm(s.P[0, 0])
    v_ex = (1 - np.exp(-2 * k * a)) / (2 * k)
    k_ex = -(1 / (4 * a)) * (2 / k - (2 * a + 2 / k) * np.exp(-2 * k * a))
    assert np.abs((V @ one) / (M @ one) / v_ex - 1).max() < 2.5e-2
    assert np.abs((K @ one) / (M @ one) / k_ex - 1).max() < 2.5e-2


def test_single_layer_nearly_symmetric(sphere_ops):
    for name in ("m", "s"):
        _, _, V, _, _ = sphere_ops[name]
        assert abs(V - V.T).max() < 1e-4 * abs(V).max()
        assert np.all(np.linalg.eigvalsh(0.5 * (V + V.T)) > 0)


def test_interior_laplace_row_on_harmonic_field(sphere_ops):
    """1/2 phi + K phi - V dphi/dn = 0 for phi = x (harmonic inside Gamma_m)."""
    s, M, V, K, _ = sphere_ops["m"]
    from paper_2511_21713_gb300 import inputs
    xyz = inputs.single_charge_sphere(nu=3, layers=5).xyz[s.verts]
    r = np.linalg.norm(xyz, axis=1)
    phi, lam = xyz[:, 0], xyz[:, 0] / r
    res = 0.5 * (M @ phi) + K @ phi - V @ lam
    assert np.linalg.norm(res) < 2e-2 * np.linalg.norm(M @ phi)
    # a wrong sign of K fails by O(1)
    bad = 0.5 * (M @ phi) - K @ phi - V @ lam
    assert np.linalg.norm(bad) > 0.3 * np.linalg.norm(M @ phi)


def test_exterior_yukawa_row_on_decaying_field(sphere_ops):
    """1/2 phi - K phi + V dphi/dn = 0 for phi = e^{-k r}/r (outward normal into Omega_s)."""
    s, M, V, K, k = sphere_ops["s"]
    from paper_2511_21713_gb300 import inputs
    xyz = inputs.single_charge_sphere(nu=3, layers=5).xyz[s.verts]
    r = np.linalg.norm(xyz, axis=1)
    phi = np.exp(-k * r) / r
    lam = -(1 / r + k) * phi
    res = 0.5 * (M @ phi) - K @ phi + V @ lam
    assert np.linalg.norm(res) < 1e-2 * np.linalg.norm(M @ phi)


def test_coulomb_rhs_central_charge(sphere_ops):
    s, M, _, _, _ = sphere_ops["m"]
    b = bem.coulomb_rhs(s, np.zeros((1, 3)), np.array([2.0]))
    a = np.linalg.norm(s.P[0, 0])
    # int over the polyhedron of 2/|x| psi_i ~ (2/a) (M 1)_i
    assert np.abs(b / (M @ np.ones(s.n)) / (2 / a) - 1).max() < 3e-2
    assert np.all(b > 0)


def test_layer_potential_inside_reproduces_harmonic_field(sphere_ops):
    """Green's representation inside: (V dphi/dn)(x) - (K phi)(x) = phi(x) for harmonic phi."""
    s, _, _, _, _ = sphere_ops["m"]
    from paper_2511_21713_gb300 import inputs
    xyz = inputs.single_charge_sphere(nu=3, layers=5).xyz[s.verts]
    r = np.linalg.norm(xyz, axis=1)
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.3]])
    phi = 1.0 + xyz[:, 0]
    lam = xyz[:, 0] / r
    got = bem.layer_potentials_at(s, pts, lam, phi)
    assert np.abs(got - (1.0 + pts[:, 0])).max() < 2e-2


def test_classification_restricted_to_test_triangles():
    """The classification of a subset of test triangles lists exactly the pairs of the full
    classification whose test triangle is in the subset (used for sampled rows of large
    surfaces)."""
    from paper_2511_21713_gb300 import inputs
    c = inputs.double_helix(n_bp=6, nu=10, layers=3, n_interior=375)
    s = bem.Surface(c.xyz, c.gm_tris)
    full = bem.classify_pairs(s)
    tt = np.sort(np.random.default_rng(4).choice(s.nt, 40, replace=False))
    part = bem.classify_pairs(s, test_tris=tt)
    keep = np.isin(np.arange(s.nt), tt)
    assert np.array_equal(part['identical'], tt)
    for k in ('edge', 'vertex', 'near'):
        ref = full[k][keep[full[k][:, 0]]]
        assert np.array_equal(part[k], ref), k
    assert len(full['near']) > 0 and len(part['near']) > 0
