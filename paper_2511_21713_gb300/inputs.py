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
    tet_region: np.ndarray = None   # (n_t,) int32 for a mesh of Omega_m and Omega_i: 0 in Omega_m,
                                    # 1 in Omega_i (Gamma_m interior); None for a shell mesh

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


def spherical_solute(nu: int, a: float, R: float, layers: int, core_layers: int, r_core: float):
    """Mesh of the ball r < R with the interface Gamma_m at r = a inside it.

    Layers of the same icosphere at radii r_core (a / r_core)^(l / core_layers), l = 0..core_layers,
    then a (R / a)^(l / layers), cut into prisms and tets as in ``spherical_shell``, and a core of
    one tet per icosphere triangle of the innermost layer with apex at the centre.  Returns
    (xyz, tets, region, gm, gs): region 0 for the tets inside Gamma_m (Omega_m), 1 outside
    (Omega_i); gm oriented away from the centre (into Omega_i), gs out of the ball.
    """
    u, tri = icosphere(nu)
    ns = u.shape[0]
    r_in = r_core * (a / r_core) ** (np.arange(core_layers + 1) / core_layers)
    r_out = a * (R / a) ** (np.arange(1, layers + 1) / layers)
    radii = np.concatenate([r_in, r_out])
    nl = radii.size
    xyz = np.concatenate([(radii[:, None, None] * u[None, :, :]).reshape(-1, 3), np.zeros((1, 3))])
    centre = nl * ns
    tets, region = [], []
    for f in tri:
        tets.append((centre, f[0], f[1], f[2]))
        region.append(0)
    for lay in range(nl - 1):
        off0, off1 = lay * ns, (lay + 1) * ns
        for f in tri:
            v = [off0 + f[0], off0 + f[1], off0 + f[2], off1 + f[0], off1 + f[1], off1 + f[2]]
            tets.extend(_prism_tets(v))
            region.extend([0 if lay < core_layers else 1] * 3)
    gm = (tri + core_layers * ns).astype(np.int32)
    gs = (tri + (nl - 1) * ns).astype(np.int32)
    return xyz, np.array(tets, dtype=np.int32), np.array(region, dtype=np.int32), gm, gs


def solute_sphere_case(nu=5, a=4.0, R=10.0, layers=13, core_layers=12, r_core=None, q_xyz=None,
                       q_z=None, eps_in=4.0, eps_out=80.0, kappa=None, ionic=0.15, T=300.0, name=None):
    """A sphere case meshed inside Gamma_m too (FEM over Omega_m and Omega_i).  The core layers
    are graded geometrically towards r_core (default a / 16), where the central cone starts."""
    r_core = a / 16.0 if r_core is None else r_core
    xyz, tets, region, gm, gs = spherical_solute(nu, a, R, layers, core_layers, r_core)
    if q_xyz is None:
        q_xyz = np.zeros((1, 3))
        q_z = np.array([5.0])
    if kappa is None:
        kappa = kappa_from_ionic_strength(ionic, eps_out, T)
    return Case(name or f"solute_sphere_nu{nu}_L{layers}_C{core_layers}", xyz, tets, gm, gs,
                np.asarray(q_xyz, np.float64).reshape(-1, 3), np.asarray(q_z, np.float64),
                eps_in, eps_out, kappa, T, tet_region=region)


def single_charge_solute_sphere(nu=5, layers=13, core_layers=12, kappa=None):
    """The single-charge sphere (radius 4, shell to 10, +5 e at the centre, eps 4/80, 0.15 M),
    meshed inside Gamma_m as well."""
    return solute_sphere_case(nu=nu, a=4.0, R=10.0, layers=layers, core_layers=core_layers, kappa=kappa,
                              name=f"single_charge_solute_sphere_nu{nu}_L{layers}_C{core_layers}")


def multi_charge_solute_sphere(nu=20, layers=17, core_layers=24, seed=2000, n_charges=200, n_pos=90):
    """The multi-charge sphere (radius 12, shell to 24, 200 +-1 e charges in r < 10, eps 2/80,
    0.1 M), meshed inside Gamma_m as well."""
    q, z = ball_charges(n_charges, 10.0, n_pos, seed)
    return solute_sphere_case(nu=nu, a=12.0, R=24.0, layers=layers, core_layers=core_layers, q_xyz=q, q_z=z,
                              eps_in=2.0, eps_out=80.0, ionic=0.1,
                              name=f"multi_charge_solute_sphere_nu{nu}_L{layers}_C{core_layers}")


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


# ----------------------------------------------------------------------------- double helix
#
# A synthetic, highly charged double helix standing in for the paper's RNA structures:
# phosphate charges of -1 e on two backbone strands and interior partial charges, a molecular
# surface at the level set 1 of a Gaussian density of the atoms, and a graded P1 shell from it to
# a sphere three Debye lengths further out.
#
# Surface and shell are built radially: ray directions d_i are the vertices of a geodesic
# icosphere stretched along the helix axis (so that triangles spread evenly over the elongated
# surface) and renormalised; along each ray the surface radius R_i is the outermost crossing of
# the density level set (which makes the enclosed region star-shaped around the centre, filling
# any overhang or interior cavity), after crevices narrower than a few rays are filled the way a
# rolling probe sphere fills them; layer l of the shell sits at R_i (R_out / R_i)^(l / L).  Every
# tetrahedron of the prism split has two vertices on one ray, so its volume has the sign of the
# ray triangle's orientation: the shell is valid for any radial profile.


def _normal(rng: SplitMix64) -> float:
    """Standard normal deviate by the Box-Muller transform of two splitmix64 uniforms."""
    u1 = 1.0 - rng.uniform()
    u2 = rng.uniform()
    return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


def helix_atoms(n_bp=24, seed=3000, n_interior=1500, twist_deg=32.727, rise=2.8, r_phos=9.0,
                strand_offset_deg=144.0, r_core=8.0):
    """Atom centres (N,3), radii (N,) and charges (N,) of the synthetic double helix.

    Phosphates: two strands, one per base pair each, at radius r_phos, rotated by twist_deg per
    base pair and offset by strand_offset_deg between strands, rise per base pair along z (the
    helix is centred at the origin); radius 1.9, charge -1.  Interior atoms: uniform in the
    cylinder of radius r_core over the helix length (rejection sampling), radii U(1.4, 1.9),
    charges N(0, 0.3) shifted to zero sum.  Net charge -2 n_bp.
    """
    rng = SplitMix64(seed)
    z0 = -0.5 * (n_bp - 1) * rise
    cen, rad, q = [], [], []
    for s in range(2):
        for k in range(n_bp):
            ang = np.deg2rad(k * twist_deg + s * strand_offset_deg)
            cen.append([r_phos * np.cos(ang), r_phos * np.sin(ang), z0 + k * rise])
            rad.append(1.9)
            q.append(-1.0)
    half = 0.5 * n_bp * rise
    qi = []
    while len(qi) < n_interior:
        x, y = (2 * rng.uniform() - 1) * r_core, (2 * rng.uniform() - 1) * r_core
        z = (2 * rng.uniform() - 1) * half
        if x * x + y * y < r_core * r_core:
            cen.append([x, y, z])
            rad.append(1.4 + 0.5 * rng.uniform())
            qi.append(0.3 * _normal(rng))
    qi = np.array(qi) - np.mean(qi)
    return np.array(cen), np.array(rad), np.concatenate([np.array(q), qi])


def _gaussian_density_grid(cen, rad, spacing, pad):
    """rho = sum_i exp(-2 (|x - c_i|^2 / r_i^2 - 1)) sampled on a regular grid (each atom summed
    within 3 r_i, where its term is below 1e-6).  Returns (origin, spacing, rho)."""
    lo = cen.min(axis=0) - pad
    hi = cen.max(axis=0) + pad
    shape = np.ceil((hi - lo) / spacing).astype(int) + 1
    rho = np.zeros(shape)
    for c, r in zip(cen, rad):
        w = 3.0 * r
        i0 = np.maximum(np.floor((c - w - lo) / spacing).astype(int), 0)
        i1 = np.minimum(np.ceil((c + w - lo) / spacing).astype(int) + 1, shape)
        ax = [lo[d] + spacing * np.arange(i0[d], i1[d]) - c[d] for d in range(3)]
        d2 = ax[0][:, None, None] ** 2 + ax[1][None, :, None] ** 2 + ax[2][None, None, :] ** 2
        rho[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] += np.exp(-2.0 * (d2 / (r * r) - 1.0))
    return lo, spacing, rho


def _outermost_crossing(dirs, lo, spacing, rho, level=1.0, step=0.2, iters=40):
    """Largest t with rho(t d) = level along each unit direction d (trilinear rho).  A ray that meets
    the level set nowhere (it leaves through a gap between atoms near the centre) gets t = step;
    the crevice closing that follows raises it to its neighbours' smoothed radius."""
    from scipy.ndimage import map_coordinates
    shape = np.array(rho.shape)
    hi = lo + spacing * (shape - 1)
    t_max = float(np.linalg.norm(np.maximum(np.abs(lo), np.abs(hi)))) + step

    def f(t):
        p = (t[:, None] * dirs - lo) / spacing
        return map_coordinates(rho, p.T, order=1, mode='constant', cval=0.0) - level

    n = dirs.shape[0]
    t_in = np.full(n, np.nan)
    t = t_max
    while t > 0 and np.isnan(t_in).any():
        todo = np.isnan(t_in)
        hit = f(np.full(n, t))[todo] >= 0
        idx = np.nonzero(todo)[0][hit]
        t_in[idx] = t
        t -= step
    t_in[np.isnan(t_in)] = step
    a, b = t_in.copy(), t_in + step          # f(a) >= 0 > f(b) where the ray met the level set
    for _ in range(iters):
        m = 0.5 * (a + b)
        inside = f(m) >= 0
        a = np.where(inside, m, a)
        b = np.where(inside, b, m)
    return 0.5 * (a + b)


def _close_crevices(r, tri, k_close=40, k_soft=3):
    """Fill narrow crevices of a radial surface, as a probe sphere rolling over the atoms would:
    r <- max(r, r smoothed by k_close Laplacian passes), then k_soft light passes.  Raising r only
    enlarges the enclosed region; the light passes move peaks by a fraction of an Angstrom."""
    import scipy.sparse as sp
    n = r.shape[0]
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    A = sp.csr_matrix((np.ones(2 * len(e)), (np.r_[e[:, 0], e[:, 1]], np.r_[e[:, 1], e[:, 0]])), shape=(n, n))
    A.data[:] = 1.0
    deg = np.asarray(A.sum(axis=1)).ravel()

    def smooth(x, k, w):
        for _ in range(k):
            x = (1.0 - w) * x + w * (A @ x) / deg
        return x

    return smooth(np.maximum(r, smooth(r, k_close, 0.5)), k_soft, 0.3)


def _radial_shell(dirs, tri, r_in, r_out, layers):
    """Shell between the star-shaped surfaces r_in(d) and r_out(d) over the ray triangulation
    (dirs, tri): layer radii r_in (r_out / r_in)^(l / layers), prisms cut as in spherical_shell."""
    ns = dirs.shape[0]
    big = 4 * ns
    pattern = []                              # per triangle: 3 tets of (local id + big * top)
    for f in tri:
        pattern.append(_prism_tets([f[0], f[1], f[2], f[0] + big, f[1] + big, f[2] + big]))
    pattern = np.array(pattern, dtype=np.int64)             # (m, 3, 4)
    top = pattern >= big
    local = np.where(top, pattern - big, pattern)
    frac = np.arange(layers + 1) / layers
    radii = r_in[None, :] * (r_out / r_in)[None, :] ** frac[:, None]        # (layers+1, ns)
    xyz = (radii[:, :, None] * dirs[None, :, :]).reshape(-1, 3)
    tets = np.concatenate([local + ns * (lay + top) for lay in range(layers)], axis=0).reshape(-1, 4)
    gm = tri.astype(np.int32)
    gs = (tri + layers * ns).astype(np.int32)
    return xyz, tets.astype(np.int32), gm, gs


def double_helix(n_bp=24, nu=45, layers=16, seed=3000, n_interior=1500, ionic=0.15, eps_in=2.0,
                 eps_out=80.0, T=300.0, grid=0.35):
    """Synthetic double helix (see above): 24 base pairs, nu = 45 (40,500 triangles per surface,
    20,252 rays), 16 shell layers (1.94M tets, 344,284 vertices), 0.15 M, outer sphere at the
    largest surface radius + 3 Debye lengths."""
    cen, rad, q = helix_atoms(n_bp, seed, n_interior)
    u, tri = icosphere(nu)
    half = 0.5 * n_bp * 2.8
    stretch = np.array([11.0, 11.0, half + 3.0])
    dirs = u * stretch
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    lo, h, rho = _gaussian_density_grid(cen, rad, grid, 6.0)
    r_in = _close_crevices(_outermost_crossing(dirs, lo, h, rho), tri)
    r_in = _enclose_charges(cen, dirs, tri, r_in, margin=0.3)
    kappa = kappa_from_ionic_strength(ionic, eps_out, T)
    R_out = float(r_in.max()) + 3.0 / kappa
    xyz, tets, gm, gs = _radial_shell(dirs, tri, r_in, np.full_like(r_in, R_out), layers)
    _check_charges_inside(cen, xyz, gm, dirs, tri, r_in, margin=0.3)
    return Case(f"double_helix_{n_bp}bp_nu{nu}_L{layers}", xyz, tets, gm, gs, cen, q,
                eps_in, eps_out, kappa, T)


def mixed_case(seed, sphere_tri=(2000.0, 8000.0), helix_tri=(5000.0, 40000.0), n_bp=(8, 48),
               max_tets=2_000_000):
    """One instance of the batched and served mixes, drawn from `seed`: a sphere or a double helix by
    a fair coin; surface triangles log-uniform in sphere_tri or helix_tri (icosphere frequency
    nu = round(sqrt(triangles / 20))); ionic strength U(0.01, 1) M; eps_in 2 or 4.  Spheres: radius
    12, shell to 24, 1-200 unit charges uniform in r < 9.6 with a random number of them positive.
    Helices: n_bp uniform in n_bp (62 interior atoms per base pair), shell to three Debye lengths
    beyond the surface.  Shell layers max(8, 0.85 nu) (spheres) or max(8, 0.6 nu) (helices), fewer
    where needed to keep the shell at most max_tets tets (4 at least)."""
    rng = SplitMix64(seed)
    sphere = rng.below(2) == 0
    lo, hi = sphere_tri if sphere else helix_tri
    tri = lo * (hi / lo) ** rng.uniform()
    nu = max(3, int(round((tri / 20.0) ** 0.5)))
    ionic = 0.01 + 0.99 * rng.uniform()
    eps_in = (2.0, 4.0)[rng.below(2)]
    cap = int(max_tets // (60 * nu * nu))
    if sphere:
        layers = max(4, min(max(8, int(0.85 * nu)), cap))
        nq = 1 + rng.below(200)
        q, z = ball_charges(nq, 9.6, rng.below(nq + 1), seed + 17)
        return sphere_case(nu=nu, a=12.0, R=24.0, layers=layers, q_xyz=q, q_z=z, eps_in=eps_in, eps_out=80.0,
                           ionic=ionic, T=300.0, name=f"mix{seed}_sphere_nu{nu}_L{layers}")
    nbp = n_bp[0] + rng.below(n_bp[1] - n_bp[0] + 1)
    layers = max(4, min(max(8, int(0.6 * nu)), cap))
    return double_helix(n_bp=nbp, nu=nu, layers=layers, seed=seed + 31, n_interior=62 * nbp, ionic=ionic,
                        eps_in=eps_in)


def _ray_triangle_of(d, dirs, tri):
    """Index of the ray triangle containing each unit direction d (first match)."""
    A, B, C = dirs[tri[:, 0]], dirs[tri[:, 1]], dirs[tri[:, 2]]
    nAB, nBC, nCA = np.cross(A, B), np.cross(B, C), np.cross(C, A)
    out = np.empty(d.shape[0], dtype=np.int64)
    for k in range(0, d.shape[0], 64):
        dk = d[k:k + 64]
        inside = (dk @ nAB.T >= -1e-12) & (dk @ nBC.T >= -1e-12) & (dk @ nCA.T >= -1e-12)
        if not inside.any(axis=1).all():
            raise ValueError("a charge direction is in no ray triangle")
        out[k:k + 64] = np.argmax(inside, axis=1)
    return out


def _enclose_charges(pts, dirs, tri, r, margin, iters=50):
    """Raise the ray radii of the triangles that would cut a charge off (a coarse triangle over an
    atom's bump) until every charge lies ``margin`` inside the surface along its ray."""
    rho = np.linalg.norm(pts, axis=1)
    d = pts / rho[:, None]
    t = _ray_triangle_of(d, dirs, tri)
    r = r.copy()
    for _ in range(iters):
        P = r[tri[t]][:, :, None] * dirs[tri[t]]                   # (nq, 3, 3) triangle corners
        n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        t_surf = np.einsum('ij,ij->i', n, P[:, 0]) / np.einsum('ij,ij->i', n, d)
        short = rho + margin - t_surf
        if not (short > 0).any():
            break
        for q in np.nonzero(short > 0)[0]:
            f = tri[t[q]]
            r[f] = np.maximum(r[f], r[f] * (rho[q] + margin + 1e-3) / t_surf[q])
    return r


def _check_charges_inside(pts, xyz, gm, dirs, tri, r_in, margin):
    """Every charge lies inside Gamma_m, at least ``margin`` below it along its own ray."""
    d = pts / np.linalg.norm(pts, axis=1)[:, None]
    A, B, C = dirs[tri[:, 0]], dirs[tri[:, 1]], dirs[tri[:, 2]]
    nAB, nBC, nCA = np.cross(A, B), np.cross(B, C), np.cross(C, A)
    for k in range(0, d.shape[0], 64):
        dk = d[k:k + 64]
        inside = (dk @ nAB.T >= -1e-12) & (dk @ nBC.T >= -1e-12) & (dk @ nCA.T >= -1e-12)
        for j in range(dk.shape[0]):
            t = np.nonzero(inside[j])[0]
            if t.size == 0:
                raise ValueError("a charge direction is in no ray triangle")
            f = tri[t[0]]
            P = xyz[gm[t[0]]]
            n = np.cross(P[1] - P[0], P[2] - P[0])
            t_surf = (n @ P[0]) / (n @ dk[j])
            if not np.linalg.norm(pts[k + j]) < t_surf - margin:
                raise ValueError(f"charge {k + j} is not inside the molecular surface by {margin} A")
