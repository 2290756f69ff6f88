"""Dense Galerkin boundary operators on a closed triangulated surface
(oracle; test infrastructure only).

Follows Sec. 2.2 (the Yukawa operators V_Y, K_Y on Gamma_s and the kernel
g_Y = exp(-kappa r) / (4 pi r)) and Sec. 2.3.1 (Eq. KV: the Laplace operators
V_L, K_L on Gamma_m with g_L = 1 / (4 pi r)).  With P1 hat functions psi_i
(Sec. 3: "piecewise-linear (P1) basis functions") the Galerkin matrices are

  V_ij = int int psi_i(x) g(x, y) psi_j(y) dy dx
  K_ij = int int psi_i(x) dg/dn_y(x, y) psi_j(y) dy dx,
  dg/dn_y = n_y . (x - y) (1 + kappa r) exp(-kappa r) / (4 pi r^3),

and the Laplace operators are the kappa = 0 case.  Each triangle pair
(tau test, sigma trial) is integrated by a rule chosen by its class:

  identical / common edge / common vertex : Sauter-Schwab, n = 5 per variable
  near (no shared vertex, centroid distance < 2 max(h_tau, h_sigma),
        h = longest edge)                 : 6-point test x 6-point rule on
                                            the 16 sub-triangles of sigma
  all other pairs                         : 6-point x 6-point

The matrices are formed densely (the paper's own choice for small meshes,
Sec. 3 discretisation paragraph) and applied by plain matrix products.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from .quadrature import tri6, subdivided_tri6, sauter_schwab, ss_basis

FOUR_PI = 4.0 * np.pi


class Surface:
    """A closed surface given by triangles over a global vertex array.

    verts: sorted global ids of the surface vertices (local index = position).
    tl: (n_tri, 3) local vertex ids; P: (n_tri, 3, 3) corner coordinates.
    area, normal (unit, from the stored orientation), h (longest edge), cen.
    """

    def __init__(self, xyz: np.ndarray, tris: np.ndarray):
        tris = np.asarray(tris, dtype=np.int64)
        self.verts = np.unique(tris)
        loc = -np.ones(xyz.shape[0], dtype=np.int64)
        loc[self.verts] = np.arange(self.verts.size)
        self.tl = loc[tris]
        self.tris = tris
        self.P = xyz[tris]
        cr = np.cross(self.P[:, 1] - self.P[:, 0], self.P[:, 2] - self.P[:, 0])
        nrm = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * nrm
        self.normal = cr / nrm[:, None]
        e = [np.linalg.norm(self.P[:, (k + 1) % 3] - self.P[:, k], axis=1) for k in range(3)]
        self.h = np.maximum(np.maximum(e[0], e[1]), e[2])
        self.cen = self.P.mean(axis=1)
        self.n = self.verts.size
        self.nt = tris.shape[0]
        b6, w6 = tri6()
        self.b6, self.w6 = b6, w6
        self.qp = np.einsum('qa,tad->tqd', b6, self.P)            # (n_tri, 6, 3)
        self.qw = self.area[:, None] * w6[None, :]                # (n_tri, 6)
        # Q maps P1 coefficients to values at quadrature points: (6 n_tri, n)
        rows = np.repeat(np.arange(6 * self.nt), 3)
        cols = np.repeat(self.tl, 6, axis=0).reshape(-1)
        vals = np.tile(b6, (self.nt, 1)).reshape(-1)
        self.Q = sp.csr_matrix((vals, (rows, cols)), shape=(6 * self.nt, self.n))


def mass_matrix(s: Surface):
    """P1 surface mass matrix M_ij = int psi_i psi_j (exact: |t|/12 [[2,1,1],[1,2,1],[1,1,2]])."""
    loc = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0
    vals = s.area[:, None, None] * loc[None]
    rows = np.repeat(s.tl, 3, axis=1).reshape(-1)
    cols = np.tile(s.tl, (1, 3)).reshape(-1)
    return sp.csr_matrix((vals.reshape(-1), (rows, cols)), shape=(s.n, s.n))


def kernels(x, y, ny, kappa):
    """Single-layer g(x,y) and double-layer dg/dn_y(x,y) for arrays of points."""
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    e = np.exp(-kappa * r)
    g = e / (FOUR_PI * r)
    dl = np.sum(ny * d, axis=-1) * (1.0 + kappa * r) * e / (FOUR_PI * r ** 3)
    return g, dl


def classify_pairs(s: Surface, near_factor: float = 2.0, test_tris=None):
    """Ordered triangle pairs by class.

    Returns dict with 'identical' (m,), 'edge' (m,2), 'vertex' (m,2) and
    'near' (m,2) arrays of (test, trial) triangle indices.  Pairs in none of
    these lists are regular.  With test_tris (a subset of test triangles) only
    the pairs whose test triangle is in the subset are listed: the same lists
    as the full classification filtered to those rows.
    """
    nt = s.nt
    rows = np.arange(nt) if test_tris is None else np.unique(np.asarray(test_tris, dtype=np.int64))
    # triangles incident to each vertex
    inc = [[] for _ in range(s.n)]
    for t in range(nt):
        for v in s.tl[t]:
            inc[v].append(t)
    shared = {}
    for t in rows:
        for v in s.tl[t]:
            for u in inc[v]:
                shared[(t, u)] = shared.get((t, u), 0) + 1
    edge, vert = [], []
    for (t, u), c in shared.items():
        if t == u:
            continue
        if c == 2:
            edge.append((t, u))
        elif c == 1:
            vert.append((t, u))
    tree = cKDTree(s.cen)
    rad = near_factor * s.h.max()
    near = []
    for a, cand in zip(rows, tree.query_ball_point(s.cen[rows], rad)):
        for b in cand:
            if (a, b) in shared:
                continue
            d = s.cen[a] - s.cen[b]
            lim = near_factor * max(s.h[a], s.h[b])
            if d @ d < lim * lim:
                near.append((a, b))
    ident = rows if test_tris is not None else np.arange(nt)
    srt = lambda L: np.array(sorted(L), dtype=np.int64).reshape(-1, 2)
    return {'identical': ident, 'edge': srt(edge), 'vertex': srt(vert), 'near': srt(near)}


def _pair_local(Pt, Ps, ns, bx, by, w, kappa):
    """Local 3x3 SL and DL matrices of a batch of pairs for one rule.

    Pt, Ps: (m, 3, 3) corners in the rule's vertex order; ns: (m, 3) trial
    normals; bx, by: (K, 3) barycentric points; w: (K,) weights on the
    reference pair (measure of the reference pair domain included).
    Returns SL, DL of shape (m, 3, 3) *without* the Jacobian factor.
    """
    x = np.einsum('ka,mad->mkd', bx, Pt)
    y = np.einsum('ka,mad->mkd', by, Ps)
    g, dl = kernels(x, y, ns[:, None, :], kappa)
    SL = np.einsum('mk,k,ka,kb->mab', g, w, bx, by)
    DL = np.einsum('mk,k,ka,kb->mab', dl, w, bx, by)
    return SL, DL


def _order_edge(tt, ts):
    """Vertex orders placing the shared edge at reference vertices 0, 1 in both."""
    sh = [v for v in tt if v in ts]
    pt = [list(tt).index(sh[0]), list(tt).index(sh[1])]
    pt.append(3 - pt[0] - pt[1])
    ps = [list(ts).index(sh[0]), list(ts).index(sh[1])]
    ps.append(3 - ps[0] - ps[1])
    return pt, ps


def _order_vertex(tt, ts):
    """Vertex orders placing the shared vertex at reference vertex 0 in both."""
    v = [x for x in tt if x in ts][0]
    it, is_ = list(tt).index(v), list(ts).index(v)
    return [it, (it + 1) % 3, (it + 2) % 3], [is_, (is_ + 1) % 3, (is_ + 2) % 3]


def assemble(s: Surface, kappa: float, n_ss: int = 5, chunk: int = 64, classes=None, test_tris=None):
    """Dense Galerkin (V, K) on surface s for the kernel with inverse length kappa.

    test_tris: optional sorted subset of test triangles; only their contributions are
    added (the rows of the other vertices are then incomplete).  Used to time or check
    a sample of rows of a large surface.
    """
    if classes is None:
        classes = classify_pairs(s, test_tris=test_tris)
    if test_tris is not None:
        test_tris = np.asarray(test_tris, dtype=np.int64)
        keep = np.zeros(s.nt, dtype=bool)
        keep[test_tris] = True
        classes = {'identical': classes['identical'][keep[classes['identical']]],
                   **{k: classes[k][keep[classes[k][:, 0]]] for k in ('edge', 'vertex', 'near')}}
    n, nt = s.n, s.nt
    V = np.zeros((n, n))
    K = np.zeros((n, n))
    # --- regular pairs: 6 x 6 points over the pairs not in any special class
    special = sp.coo_matrix((np.ones(nt), (np.arange(nt), np.arange(nt))), shape=(nt, nt)).tocsr()
    for key in ('edge', 'vertex', 'near'):
        pr = classes[key]
        if pr.size:
            special = special + sp.csr_matrix((np.ones(len(pr)), (pr[:, 0], pr[:, 1])), shape=(nt, nt))
    Y = s.qp.reshape(-1, 3)
    NY = np.repeat(s.normal, 6, axis=0)
    WY = s.qw.reshape(-1)
    rows = np.arange(nt) if test_tris is None else test_tris
    for c0 in range(0, rows.size, chunk):
        tc = rows[c0:c0 + chunk]
        q6 = (6 * tc[:, None] + np.arange(6)[None, :]).reshape(-1)
        X = s.qp[tc].reshape(-1, 3)
        WX = s.qw[tc].reshape(-1)
        mask = np.asarray(special[tc].todense()) == 0                        # (c, nt) regular pairs
        m6 = np.repeat(np.repeat(mask, 6, axis=0), 6, axis=1)
        with np.errstate(divide='ignore', invalid='ignore'):
            g, dl = kernels(X[:, None, :], Y[None, :, :], NY[None, :, :], kappa)
        g = np.where(m6, g, 0.0) * WX[:, None] * WY[None, :]
        dl = np.where(m6, dl, 0.0) * WX[:, None] * WY[None, :]
        Qc = s.Q[q6]
        V += (Qc.T @ (s.Q.T @ g.T).T)
        K += (Qc.T @ (s.Q.T @ dl.T).T)
    # --- special pairs
    def scatter(tt, ts, pt, ps, SL, DL):
        gi = s.tl[tt[:, None], pt]           # (m,3) local ids of test rule vertices
        gj = s.tl[ts[:, None], ps]
        I = np.repeat(gi[:, :, None], 3, axis=2)
        J = np.repeat(gj[:, None, :], 3, axis=1)
        np.add.at(V, (I.reshape(-1), J.reshape(-1)), SL.reshape(-1))
        np.add.at(K, (I.reshape(-1), J.reshape(-1)), DL.reshape(-1))

    for case in ('identical', 'edge', 'vertex'):
        pr = classes[case]
        if case == 'identical':
            tt = ts = pr
            pt = ps = np.tile(np.arange(3), (len(pr), 1))
        else:
            tt, ts = pr[:, 0], pr[:, 1]
            orders = [(_order_edge if case == 'edge' else _order_vertex)(s.tl[a], s.tl[b])
                      for a, b in zip(tt, ts)]
            pt = np.array([o[0] for o in orders], dtype=np.int64).reshape(-1, 3)
            ps = np.array([o[1] for o in orders], dtype=np.int64).reshape(-1, 3)
        if len(tt) == 0:
            continue
        xh, yh, w = sauter_schwab(case, n_ss)
        bx, by = ss_basis(xh), ss_basis(yh)
        for c0 in range(0, len(tt), 256):
            sl = slice(c0, c0 + 256)
            Pt = np.take_along_axis(s.P[tt[sl]], pt[sl][:, :, None], axis=1)
            Ps = np.take_along_axis(s.P[ts[sl]], ps[sl][:, :, None], axis=1)
            SL, DL = _pair_local(Pt, Ps, s.normal[ts[sl]], bx, by, w, kappa)
            jac = (4.0 * s.area[tt[sl]] * s.area[ts[sl]])[:, None, None]
            scatter(tt[sl], ts[sl], pt[sl], ps[sl], SL * jac, DL * jac)
    pr = classes['near']
    if len(pr):
        bt, wt = tri6()
        bs, ws = subdivided_tri6(4)
        bx = np.repeat(bt, len(ws), axis=0)
        by = np.tile(bs, (len(wt), 1))
        w = np.outer(wt, ws).reshape(-1)
        idx = np.tile(np.arange(3), (len(pr), 1))
        for c0 in range(0, len(pr), 256):
            p = pr[c0:c0 + 256]
            SL, DL = _pair_local(s.P[p[:, 0]], s.P[p[:, 1]], s.normal[p[:, 1]], bx, by, w, kappa)
            jac = (s.area[p[:, 0]] * s.area[p[:, 1]])[:, None, None]
            scatter(p[:, 0], p[:, 1], idx[:len(p)], idx[:len(p)], SL * jac, DL * jac)
    return V, K


def coulomb_rhs(s: Surface, q_xyz, q_z):
    """<sum_k z_k / |x - x_k|, psi_i> on s by the 6-point rule (Sec. 2.3.1, phi_coul,
    without the l_B / eps_m factor)."""
    X = s.qp.reshape(-1, 3)
    d = X[:, None, :] - q_xyz[None, :, :]
    pot = np.sum(q_z[None, :] / np.sqrt(np.sum(d * d, axis=-1)), axis=1)
    return s.Q.T @ (s.qw.reshape(-1) * pot)


def layer_potentials_at(s: Surface, pts, lam, u_surf):
    """(V_L lam)(x) - (K_L u)(x) at points off the surface, 6-point rule
    (Eq. Potential_in_Omega_m for the reaction potential)."""
    Y = s.qp.reshape(-1, 3)
    NY = np.repeat(s.normal, 6, axis=0)
    wl = s.qw.reshape(-1) * (s.Q @ lam)
    wu = s.qw.reshape(-1) * (s.Q @ u_surf)
    g, dl = kernels(pts[:, None, :], Y[None, :, :], NY[None, :, :], 0.0)
    return g @ wl - dl @ wu
