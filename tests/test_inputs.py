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
