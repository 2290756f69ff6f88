"""Pins for the oracle's quadrature rules (no GPU).

Each rule is checked against exact integrals of monomials (closed form
a! b! c! / (a+b+c+d)! on the unit simplex), and the Sauter-Schwab rules
against exact polynomial double integrals and an independent semi-analytic
value of the weakly singular 1/r integral.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def test_tet14_exact_to_degree5_and_not_6():
    lam, w = Q.tet14()
    assert lam.shape == (14, 4) and np.allclose(lam.sum(1), 1.0)
    assert np.all(w > 0) and abs(w.sum() - 1.0) < 1e-15
    P = lam[:, 1:]
    worst, deg6 = 0.0, 0.0
    for a, b, c in itertools.product(range(7), repeat=3):
        d = a + b + c
        if d > 6:
            continue
        exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(d + 3)
        got = np.sum(w * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c) / 6.0
        err = abs(got - exact) / exact
        if d <= 5:
            worst = max(worst, err)
        else:
            deg6 = max(deg6, err)
    assert worst < 1e-14
    assert deg6 > 1e-6          # a degree-5 rule, not a higher one mislabelled


def test_tri6_exact_to_degree4():
    b, w = Q.tri6()
    assert np.all(w > 0) and abs(w.sum() - 1.0) < 1e-15
    P = b[:, 1:]
    for a, c in itertools.product(range(6), repeat=2):
        d = a + c
        if d > 5:
            continue
        exact = math.factorial(a) * math.factorial(c) / math.factorial(d + 2)
        got = 0.5 * np.sum(w * P[:, 0] ** a * P[:, 1] ** c)
        if d <= 4:
            assert abs(got - exact) < 1e-15 * max(1.0, exact) * 10
        if (a, c) == (5, 0):
            assert abs(got - exact) / exact > 1e-6


def test_subdivided_rule_covers_parent():
    b, w = Q.subdivided_tri6(4)
    assert b.shape == (96, 3) and abs(w.sum() - 1.0) < 1e-14
    assert np.all(b >= -1e-15)
    P = b[:, 1:]
    for a, c in [(4, 0), (2, 2), (1, 3), (3, 1)]:
        exact = math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
        assert abs(0.5 * np.sum(w * P[:, 0] ** a * P[:, 1] ** c) - exact) < 1e-15


def _tri_ref(a, b):
    # int over {0 <= s2 <= s1 <= 1} of s1^a s2^b
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("case", ["identical", "edge", "vertex"])
def test_sauter_schwab_integrates_polynomials(case):
    xh, yh, w = Q.sauter_schwab(case, 5)
    assert abs(w.sum() - 0.25) < 1e-14
    for a, b, c, d in itertools.product(range(3), repeat=4):
        if a + b + c + d > 4:
            continue
        exact = _tri_ref(a, b) * _tri_ref(c, d)
        got = np.sum(w * xh[:, 0] ** a * xh[:, 1] ** b * yh[:, 0] ** c * yh[:, 1] ** d)
        assert abs(got - exact) / exact < 1e-13


def _chi(P, s):
    return P[0] + s[:, :1] * (P[1] - P[0]) + s[:, 1:2] * (P[2] - P[1])


def _area(P):
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def _inner_1_over_r(P, x):
    """int_T 1/|x - y| dy for x in the plane of triangle T (closed form: sum over
    the edges of h_e [asinh(t1/h_e) - asinh(t0/h_e)], the polar-coordinate
    integral of each sub-triangle (x, v_i, v_{i+1}))."""
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    tot = np.zeros(len(x))
    for i in range(3):
        A, B = P[i], P[(i + 1) % 3]
        e = (B - A) / np.linalg.norm(B - A)
        m = np.cross(e, n)                       # in-plane normal to the edge (outward for ccw)
        h = (A - x) @ m                          # signed distance from x to the edge line
        t0 = (A - x) @ e
        t1 = (B - x) @ e
        ok = np.abs(h) > 1e-14
        tot[ok] += h[ok] * (np.arcsinh(t1[ok] / np.abs(h[ok])) - np.arcsinh(t0[ok] / np.abs(h[ok])))
    return tot


def test_sauter_schwab_singular_identical_panel():
    """Identical-panel int int 1/|x-y| vs analytic inner integral + fine outer rule."""
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.9, 0.0]])
    # outer: Gauss-Legendre on the collapsed square (Duffy), 80 x 80 points
    t, wt = Q.gauss_legendre01(80)
    S1, S2 = np.meshgrid(t, t, indexing='ij')
    s = np.stack([S1.reshape(-1), (S1 * S2).reshape(-1)], -1)       # point in That
    W = (np.outer(wt, wt) * S1).reshape(-1)                          # Duffy Jacobian s1
    ref = 2 * _area(P) * np.sum(W * _inner_1_over_r(P, _chi(P, s)))
    vals = {}
    for n in (5, 12):
        xh, yh, w = Q.sauter_schwab('identical', n)
        r = np.linalg.norm(_chi(P, xh) - _chi(P, yh), axis=1)
        vals[n] = 4 * _area(P) ** 2 * np.sum(w / r)
    assert abs(vals[12] - ref) / ref < 1e-7
    assert abs(vals[5] - ref) / ref < 1e-5


@pytest.mark.parametrize("case", ["edge", "vertex"])
def test_sauter_schwab_adjacent_converges(case):
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.9, 0.0]])
    Q2 = (np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.6, -0.8, 0.2]]) if case == 'edge'
          else np.array([[0.0, 0.0, 0.0], [-0.7, 0.2, 0.1], [-0.4, -0.8, -0.3]]))
    vals = []
    for n in (5, 8, 16):
        xh, yh, w = Q.sauter_schwab(case, n)
        r = np.linalg.norm(_chi(P, xh) - _chi(Q2, yh), axis=1)
        vals.append(4 * _area(P) * _area(Q2) * np.sum(w / r))
    assert abs(vals[1] - vals[2]) / vals[2] < 1e-7       # exponential convergence
    assert abs(vals[0] - vals[2]) / vals[2] < 1e-5
    # brute force: fine product Gauss on the two triangles (no singular point in common
    # interior, so a plain rule converges slowly but to the same value)
    t, wt = Q.gauss_legendre01(24)
    S1, S2 = np.meshgrid(t, t, indexing='ij')
    s = np.stack([S1.reshape(-1), (S1 * S2).reshape(-1)], -1)
    W = (np.outer(wt, wt) * S1).reshape(-1)
    X, Y = _chi(P, s), _chi(Q2, s)
    r = np.linalg.norm(X[:, None] - Y[None], axis=-1)
    brute = 4 * _area(P) * _area(Q2) * (W @ (1 / r) @ W)
    assert abs(brute - vals[2]) / vals[2] < 2e-3
