"""The seeded input generators (no GPU): the double helix's atoms, surfaces and shell."""
import numpy as np

from paper_2511_21713_gb300 import inputs


def test_helix_atoms_geometry_and_charges():
    cen, rad, q = inputs.helix_atoms(n_bp=24, seed=3000, n_interior=1500)
    assert cen.shape == (1548, 3) and rad.shape == (1548,) and q.shape == (1548,)
    ph, core = slice(0, 48), slice(48, None)
    assert np.all(q[ph] == -1.0) and np.all(rad[ph] == 1.9)
    assert np.allclose(np.hypot(cen[ph, 0], cen[ph, 1]), 9.0)
    z = cen[:24, 2]
    assert np.allclose(np.diff(z), 2.8) and abs(z.mean()) < 1e-12
    ang = np.unwrap(np.arctan2(cen[:24, 1], cen[:24, 0]))
    assert np.allclose(np.diff(ang), np.deg2rad(32.727))
    off = np.angle(np.exp(1j * (np.arctan2(cen[24, 1], cen[24, 0]) - np.arctan2(cen[0, 1], cen[0, 0]))))
    assert abs(off - np.deg2rad(144.0)) < 1e-12
    assert np.all(np.hypot(cen[core, 0], cen[core, 1]) < 8.0) and np.all(np.abs(cen[core, 2]) <= 33.6)
    assert np.all((rad[core] >= 1.4) & (rad[core] < 1.9))
    assert abs(q[core].sum()) < 1e-12 and abs(q.sum() + 48.0) < 1e-12
    assert 0.25 < q[core].std() < 0.35


def _closed(tris):
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    return np.all(cnt == 2)


def test_small_helix_mesh_is_a_valid_shell():
    nu, L, nbp = 10, 3, 6
    c = inputs.double_helix(n_bp=nbp, nu=nu, layers=L, n_interior=375)
    ns = 10 * nu * nu + 2
    assert c.n_v == (L + 1) * ns and c.n_t == 3 * 20 * nu * nu * L
    assert c.gm_tris.shape == (20 * nu * nu, 3) and c.gs_tris.shape == (20 * nu * nu, 3)
    assert _closed(c.gm_tris) and _closed(c.gs_tris)
    # every tet has a volume of the same sign, bounded away from zero
    X = c.xyz[c.tets]
    det = np.einsum('ij,ij->i', X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))
    assert np.all(det > 0) or np.all(det < 0)
    assert np.abs(det).min() > 1e-9 * np.abs(det).max()
    # Gamma_m faces point away from the centre (into the shell), Gamma_s is the outer sphere
    P = c.xyz[c.gm_tris]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    assert np.all(np.einsum('ij,ij->i', n, P.sum(axis=1)) > 0)
    r_out = np.linalg.norm(c.xyz[c.gs_tris.ravel()], axis=1)
    r_in = np.linalg.norm(c.xyz[:ns], axis=1)
    assert np.allclose(r_out, r_in.max() + 3.0 / c.kappa)
    assert abs(c.q_z.sum() + 2 * nbp) < 1e-12 and abs(c.kappa - 0.1257259) < 1e-6


def test_mixed_cases_follow_their_recipe():
    """The batched / served mix: seeded (the same seed gives the same instance), triangles within the
    requested ranges (log-uniform draw, rounded to an icosphere frequency), at most 2M tets, salt in
    0.01-1 M, eps_in 2 or 4, and every charge strictly inside Gamma_m."""
    kinds = set()
    for seed in range(4000, 4012):
        c = inputs.mixed_case(seed, sphere_tri=(2000.0, 3000.0), helix_tri=(2000.0, 3000.0), n_bp=(6, 8))
        again = inputs.mixed_case(seed, sphere_tri=(2000.0, 3000.0), helix_tri=(2000.0, 3000.0), n_bp=(6, 8))
        assert np.array_equal(c.xyz, again.xyz) and np.array_equal(c.q_z, again.q_z)
        kinds.add("helix" in c.name)
        nt = c.gm_tris.shape[0]
        assert 1700 <= nt <= 3400 and c.n_t <= 2_000_000
        assert c.eps_in in (2.0, 4.0)
        k01 = inputs.kappa_from_ionic_strength(0.01, 80.0, 300.0)
        k1 = inputs.kappa_from_ionic_strength(1.0, 80.0, 300.0)
        assert k01 <= c.kappa <= k1
        # winding number of Gamma_m at every charge (1 inside)
        P = c.xyz[c.gm_tris]
        for x in c.q_xyz[:20]:
            a, b, d = P[:, 0] - x, P[:, 1] - x, P[:, 2] - x
            la, lb, ld = (np.linalg.norm(v, axis=1) for v in (a, b, d))
            det = np.einsum("ij,ij->i", a, np.cross(b, d))
            den = la * lb * ld + np.einsum("ij,ij->i", a, b) * ld + np.einsum("ij,ij->i", b, d) * la \
                + np.einsum("ij,ij->i", d, a) * lb
            assert abs(np.sum(2 * np.arctan2(det, den)) / (4 * np.pi) - 1.0) < 1e-9
    assert kinds == {True, False}
