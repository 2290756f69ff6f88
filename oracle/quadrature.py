"""Quadrature rules used by the oracle (test infrastructure only).

The paper states P1 elements with fourth-order Gaussian quadrature (Sec. 3,
Results, discretisation paragraph) without naming rules.  The oracle fixes:

* tetrahedra: the symmetric 14-point rule exact for polynomials of degree 5
  (orbits S31 x2 and S22, Walkington 2014 / Keast-type);
* triangles: the symmetric 6-point rule exact for degree 4 (Dunavant 1985);
* singular and adjacent triangle pairs: the Sauter-Schwab regularising
  transformations (Sauter & Schwab, Boundary Element Methods, 2011, Sec. 5.2)
  with an n-point Gauss-Legendre rule in each of the four variables.

All rules here return barycentric or reference coordinates and weights that
sum to the measure of the reference domain they integrate over.
"""
from __future__ import annotations

import numpy as np


def tet14():
    """14-point degree-5 rule on a tetrahedron.

    Returns (lam (14,4) barycentric coordinates, w (14,) weights summing to 1);
    the integral over a tet of volume |T| is |T| * sum_q w_q f(x_q).
    """
    a1, w1 = 0.0927352503108912264023, 0.0734930431163619495437
    a2, w2 = 0.3108859192633006097973, 0.1126879257180158507992
    c3, w3 = 0.0455037041256496494918, 0.0425460207770814664380
    pts, wts = [], []
    for a, w in ((a1, w1), (a2, w2)):
        for k in range(4):
            lam = np.full(4, a)
            lam[k] = 1.0 - 3.0 * a
            pts.append(lam)
            wts.append(w)
    b3 = 0.5 - c3
    for i in range(4):
        for j in range(i + 1, 4):
            lam = np.full(4, c3)
            lam[i] = b3
            lam[j] = b3
            pts.append(lam)
            wts.append(w3)
    return np.array(pts), np.array(wts)


def tri6():
    """6-point degree-4 rule on a triangle.

    Returns (beta (6,3) barycentric coordinates, w (6,) weights summing to 1);
    the integral over a triangle of area |t| is |t| * sum_q w_q f(y_q).
    """
    a1, w1 = 0.44594849091596488632, 0.22338158967801146570
    a2, w2 = 0.09157621350977074346, 0.10995174365532186764
    pts, wts = [], []
    for a, w in ((a1, w1), (a2, w2)):
        for k in range(3):
            b = np.full(3, a)
            b[k] = 1.0 - 2.0 * a
            pts.append(b)
            wts.append(w)
    return np.array(pts), np.array(wts)


def subdivided_tri6(m: int = 4):
    """The 6-point rule on each of the m^2 congruent sub-triangles of a triangle.

    Returns (beta (6 m^2, 3) barycentric coordinates in the parent, w summing to 1).
    Used for near (non-touching but close) triangle pairs on the trial side.
    """
    beta6, w6 = tri6()
    subs = []
    for i in range(m):
        for j in range(m - i):
            subs.append(((i, j), (i + 1, j), (i, j + 1)))
            if i + j < m - 1:
                subs.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    pts, wts = [], []
    for tri in subs:
        # corner barycentrics in the parent: lattice (i, j) -> (1 - (i+j)/m, i/m, j/m)
        corners = np.array([[1.0 - (i + j) / m, i / m, j / m] for (i, j) in tri])
        for q in range(6):
            pts.append(beta6[q] @ corners)
            wts.append(w6[q] / (m * m))
    return np.array(pts), np.array(wts)


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (library nodes, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _grid4(n):
    t, w = gauss_legendre01(n)
    X = np.stack(np.meshgrid(t, t, t, t, indexing='ij'), -1).reshape(-1, 4)
    W = np.einsum('i,j,k,l->ijkl', w, w, w, w).reshape(-1)
    return X, W


def sauter_schwab(case: str, n: int = 5):
    """Sauter-Schwab rule for a pair of triangles on the reference triangle
    That = {(s1, s2): 0 <= s2 <= s1 <= 1} (area 1/2) in both variables.

    case: 'identical' (same triangle, same vertex order), 'edge' (shared
    vertices at reference (0,0) and (1,0) in both triangles), or 'vertex'
    (shared vertex at reference (0,0) in both).

    Returns (xh (K,2), yh (K,2), w (K,)) with sum_k w_k f(xh_k, yh_k)
    approximating the double integral over That x That of f; the weights carry
    the Jacobians of the regularising maps (Sauter & Schwab 2011, Sec. 5.2).
    """
    X, W = _grid4(n)
    xi, e1, e2, e3 = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    xs, ys, ws = [], [], []
    if case == 'identical':
        jac = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * (1 - e1 + e1 * e2)), (xi * (1 - e1 * e2 * e3), xi * (1 - e1))),
            ((xi * (1 - e1 * e2 * e3), xi * (1 - e1)), (xi, xi * (1 - e1 + e1 * e2))),
            ((xi, xi * e1 * (1 - e2 + e2 * e3)), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * (1 - e2 + e2 * e3))),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * (1 - e2))),
            ((xi, xi * e1 * (1 - e2)), (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3))),
        ]
        jacs = [jac] * 6
    elif case == 'edge':
        j1 = xi ** 3 * e1 ** 2
        j2 = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * e1 * e3), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            ((xi, xi * e1), (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3))),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * e2 * e3)),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), (xi, xi * e1)),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * e2)),
        ]
        jacs = [j1, j2, j2, j2, j2]
    elif case == 'vertex':
        jac = xi ** 3 * e2
        regions = [
            ((xi, xi * e1), (xi * e2, xi * e2 * e3)),
            ((xi * e2, xi * e2 * e3), (xi, xi * e1)),
        ]
        jacs = [jac, jac]
    else:
        raise ValueError(case)
    for ((x1, x2), (y1, y2)), jac in zip(regions, jacs):
        xs.append(np.stack([x1, x2], -1))
        ys.append(np.stack([y1, y2], -1))
        ws.append(W * jac)
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ws)


def ss_basis(sh):
    """P1 basis on the Sauter-Schwab reference triangle at points sh (K,2):
    vertex 0 at (0,0), vertex 1 at (1,0), vertex 2 at (1,1)."""
    s1, s2 = sh[:, 0], sh[:, 1]
    return np.stack([1.0 - s1, s1 - s2, s2], -1)
