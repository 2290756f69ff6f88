"""Seeded synthetic inputs for the three-region FEM-BEM Poisson-Boltzmann solve.

This module is the only code shared by the CUDA library's callers (tests,
bench) and the CPU oracle.  It builds geometry and charges only: it holds none
of the method's arithmetic (no quadrature, no operators, no physics).

Workloads (lengths in Angstrom, charges in units of e):

* ``sphere_case(nu, a, R, layers, ...)``: a geodesic icosphere of frequency
  ``nu`` (20 nu^2 triangles, 10 nu^2 + 2 vertices) of radius ``a`` for the
  molecular surface Gamma_m, the same sphere scaled to ``R`` for the outer
  surface Gamma_s, and a P1 tetrahedral shell between them made of
  ``layers`` radial layers with geometric radii r_l = a (R/a)^(l/layers).
  Each triangular prism is cut into 3 tetrahedra by choosing each quad
  diagonal from the quad's lowest global vertex id, which makes neighbouring
  prisms conform.
* The small single-charge sphere (radius 4, shell to 10, nu = 5, 13 layers:
  3528 vertices, 19,500 tets, +5 e at the centre).
* The multi-charge sphere (radius 12, shell to 24, nu = 20, 17 layers:
  72,036 vertices, 408,000 tets, 200 charges of +-1 e uniform in r < 10,
  90 positive and 110 negative).

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), seeded per case.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator; ``uniform()`` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) by rejection (unbiased)."""
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            v = self.next_u64()
            if v < lim:
                return v % n


@dataclasses.dataclass
class Case:
    """A complete solve input.

    xyz: (n_v, 3) float64 shell vertex coordinates.
    tets: (n_t, 4) int32 shell tetrahedra.
    gm_tris: (n_gm, 3) int32 Gamma_m faces (shell vertex ids), normal into the shell.
    gs_tris: (n_gs, 3) int32 Gamma_s faces (shell vertex ids), normal out of the shell.
    q_xyz: (n_q, 3) float64 charge positions, q_z: (n_q,) charges in e.
    eps_in, eps_out, kappa (1/Angstrom), T (K).
    """
    name: str
    xyz: np.ndarray
    tets: np.ndarray
    gm_tris: np.ndarray
    gs_tris: np.ndarray
    q_xyz: np.ndarray
    q_z: np.ndarray
    eps_in: float
    eps_out: float
    kappa: float
    T: float

    @property
    def n_v(self):
        return self.xyz.shape[0]

    @property
    def n_t(self):
        return self.tets.shape[0]


_ICO_V = None


def _icosahedron():
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosphere(nu: int):
    """Unit geodesic sphere of frequency ``nu``: returns (verts (n,3), tris (m,3)).

    Each icosahedron face is cut into nu^2 triangles; shared edge and corner
    points are merged by their integer lattice key, so the result is a closed
    2-manifold with 10 nu^2 + 2 vertices and 20 nu^2 outward-oriented faces.
    """
    v0, f0 = _icosahedron()
    key_to_id = {}
    pts = []
    tris = []

    def vid(face, i, j):
        # lattice point ((nu-i-j) A + i B + j C) / nu, keyed by the corner ids and weights
        a, b, c = face
        w = {a: nu - i - j, b: i, c: j}
        key = tuple(sorted((k, wt) for k, wt in w.items() if wt > 0))
        if key not in key_to_id:
            key_to_id[key] = len(pts)
            pnt = (w[a] * v0[a] + w[b] * v0[b] + w[c] * v0[c]) / nu
            pts.append(pnt / np.linalg.norm(pnt))
        return key_to_id[key]

    for face in f0:
        for i in range(nu):
            for j in range(nu - i):
                t1 = (vid(face, i, j), vid(face, i + 1, j), vid(face, i, j + 1))
                tris.append(t1)
                if i + j < nu - 1:
                    t2 = (vid(face, i + 1, j), vid(face, i + 1, j + 1), vid(face, i, j + 1))
                    tris.append(t2)
    verts = np.array(pts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int64)
    # orient every face outward (the sphere is centred at the origin)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    s = np.einsum('ij,ij->i', np.cross(b - a, c - a), a + b + c)
    flip = s < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris


def _prism_tets(v):
    """Cut prism (v0,v1,v2 bottom; v3,v4,v5 top, v[i+3] above v[i]) into 3 tets.

    Diagonals of the three quad faces start at the quad's lowest global id.
    Bottom ids are always below top ids here, so the lowest id of a quad is a
    bottom vertex.
    """
    b = list(v[:3])
    t = list(v[3:])
    r = int(np.argmin(b))
    b = b[r:] + b[:r]
    t = t[r:] + t[:r]
    # b[0] is the smallest id: quads (b0,b1,t1,t0) and (b0,b2,t2,t0) take diagonals b0-t1, b0-t2
    if b[1] < b[2]:
        # quad (b1,b2,t2,t1): diagonal b1-t2
        return [(b[0], b[1], b[2], t[2]), (b[0], b[1], t[2], t[1]), (b[0], t[1], t[2], t[0])]
    # diagonal b2-t1
    return [(b[0], b[1], b[2], t[1]), (b[0], t[1], b[2], t[2]), (b[0], t[1], t[2], t[0])]


def spherical_shell(nu: int, a: float, R: float, layers: int):
    """Shell mesh between spheres of radius a and R (see module docstring)."""
    u, tri = icosphere(nu)
    ns = u.shape[0]
    radii = a * (R / a) ** (np.arange(layers + 1) / layers)
    xyz = (radii[:, None, None] * u[None, :, :]).reshape(-1, 3)
    tets = []
    for lay in range(layers):
        off0, off1 = lay * ns, (lay + 1) * ns
        for f in tri:
            v = [off0 + f[0], off0 + f[1], off0 + f[2], off1 + f[0], off1 + f[1], off1 + f[2]]
            tets.extend(_prism_tets(v))
    tets = np.array(tets, dtype=np.int32)
    gm = tri.astype(np.int32)                     # outward of the inner sphere = into the shell
    gs = (tri + layers * ns).astype(np.int32)     # outward of the outer sphere = into the far field
    # fix xyz radii exactly on the two surfaces (already exact by construction)
    return xyz, tets, gm, gs


def ball_charges(n: int, radius: float, n_pos: int, seed: int):
    """``n`` unit charges uniform in the ball r < radius (rejection sampling),
    ``n_pos`` of them +1 and the rest -1 by a seeded Fisher-Yates permutation."""
    rng = SplitMix64(seed)
    pts = []
    while len(pts) < n:
        p = np.array([2 * rng.uniform() - 1, 2 * rng.uniform() - 1, 2 * rng.uniform() - 1])
        if p @ p < 1.0:
            pts.append(radius * p)
    z = np.array([1.0] * n_pos + [-1.0] * (n - n_pos))
    for i in range(n - 1, 0, -1):
        j = rng.below(i + 1)
        z[i], z[j] = z[j], z[i]
    return np.array(pts, dtype=np.float64), z


# Physical-input helpers: ionic strength (mol/L) -> inverse Debye length.
AVOGADRO = 6.02214076e23
COULOMB_KCAL_A = 332.0637          # e^2 / (4 pi eps0) in kcal mol^-1 Angstrom
KB_KCAL = 0.0019872043             # Boltzmann constant in kcal mol^-1 K^-1


def kappa_from_ionic_strength(I_molar: float, eps_out: float, T: float) -> float:
    """Inverse Debye length of a 1:1 salt: kappa^2 = 8 pi l_B c0 / eps_out,
    l_B = e^2/(4 pi eps0 kB T) and c0 = I N_A / 1e27 per cubic Angstrom."""
    lB = COULOMB_KCAL_A / (KB_KCAL * T)
    c0 = I_molar * AVOGADRO * 1e-27
    return float(np.sqrt(8.0 * np.pi * lB * c0 / eps_out))


def sphere_case(nu=5, a=4.0, R=10.0, layers=13, q_xyz=None, q_z=None,
                eps_in=4.0, eps_out=80.0, kappa=None, ionic=0.15, T=300.0, name=None):
    xyz, tets, gm, gs = spherical_shell(nu, a, R, layers)
    if q_xyz is None:
        q_xyz = np.zeros((1, 3))
        q_z = np.array([5.0])
    if kappa is None:
        kappa = kappa_from_ionic_strength(ionic, eps_out, T)
    return Case(name or f"sphere_nu{nu}_L{layers}", xyz, tets, gm, gs,
                np.asarray(q_xyz, np.float64).reshape(-1, 3), np.asarray(q_z, np.float64),
                eps_in, eps_out, kappa, T)


def single_charge_sphere(nu=5, layers=13, kappa=None):
    """Radius-4 solute, shell to 10, +5 e at the centre, eps 4/80, 0.15 M, 300 K."""
    return sphere_case(nu=nu, a=4.0, R=10.0, layers=layers, eps_in=4.0, eps_out=80.0,
                       kappa=kappa, ionic=0.15, T=300.0, name=f"single_charge_sphere_nu{nu}_L{layers}")


def multi_charge_sphere(nu=20, layers=17, seed=2000, n_charges=200, n_pos=90):
    """Radius-12 solute, shell to 24, 200 +-1 e charges in r < 10 (net -20 e), eps 2/80, 0.1 M."""
    q, z = ball_charges(n_charges, 10.0, n_pos, seed)
    return sphere_case(nu=nu, a=12.0, R=24.0, layers=layers, q_xyz=q, q_z=z,
                       eps_in=2.0, eps_out=80.0, ionic=0.1, T=300.0,
                       name=f"multi_charge_sphere_nu{nu}_L{layers}")
