"""Pins for the oracle's touching-pair quadrature rules.

Flat squares: the self-interaction of an a x b rectangle,
    I(a, b) = int_R int_R |x - y|^-1 = 4 int_0^a int_0^b (a-u)(b-v) / sqrt(u^2+v^2),
is additive over a split of R into unit squares, which isolates the identical,
common-edge and common-vertex pieces:
    I(1,1) = identical,  I(2,1) = 2 identical + 2 edge,
    I(2,2) = 4 identical + 8 edge + 4 vertex.
The reduced integrals are computed with scipy's adaptive quadrature, and the
unit square also has the closed form (4/3)(1 - sqrt 2) + 4 ln(1 + sqrt 2).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import singular


def _rect(a, b):
    f = lambda v, u: (a - u) * (b - v) / np.hypot(u, v)
    val, _ = integrate.dblquad(f, 0, a, 0, b, epsabs=1e-14, epsrel=1e-14)
    return 4 * val


@pytest.fixture(scope="module")
def pieces():
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        i11, i21, i22 = _rect(1, 1), _rect(2, 1), _rect(2, 2)
    edge = (i21 - 2 * i11) / 2
    vertex = (i22 - 4 * i11 - 8 * edge) / 4
    return i11, edge, vertex


def test_identical_unit_square_closed_form(pieces):
    X, Y, W = singular.identical_rule(8)
    val = np.sum(W / np.linalg.norm(X - Y, axis=1))
    closed = (4 / 3) * (1 - np.sqrt(2)) + 4 * np.log(1 + np.sqrt(2))
    assert abs(pieces[0] - closed) < 1e-12
    assert abs(val - closed) < 1e-10


def test_common_edge_flat(pieces):
    # A = [0,1]^2 at local (x1, x2); B = [-1,0] x [0,1] with local (y1, y2) -> (-y1, y2)
    X, Y, W = singular.edge_rule(8)
    PB = np.stack((-Y[:, 0], Y[:, 1]), axis=1)
    assert abs(np.sum(W / np.linalg.norm(X - PB, axis=1)) - pieces[1]) < 1e-10


def test_common_vertex_flat(pieces):
    X, Y, W = singular.vertex_rule(8)
    assert abs(np.sum(W / np.linalg.norm(X + Y, axis=1)) - pieces[2]) < 1e-10


@pytest.mark.parametrize("rule", [singular.identical_rule, singular.edge_rule, singular.vertex_rule])
def test_rules_integrate_polynomials_exactly(rule):
    # a smooth integrand: the rule must reproduce int x1^a x2^b y1^c y2^d = prod 1/(k+1)
    X, Y, W = rule(8)
    for a, b, c, d in [(0, 0, 0, 0), (1, 0, 2, 0), (0, 3, 1, 2), (2, 2, 2, 1)]:
        val = np.sum(W * X[:, 0] ** a * X[:, 1] ** b * Y[:, 0] ** c * Y[:, 1] ** d)
        assert abs(val - 1 / ((a + 1) * (b + 1) * (c + 1) * (d + 1))) < 1e-13


def test_rules_map_into_unit_cubes():
    for rule in (singular.identical_rule, singular.edge_rule, singular.vertex_rule,
                 singular.near_singular_rule):
        X, Y, W = rule(4)
        assert np.all((X >= 0) & (X <= 1) & (Y >= 0) & (Y <= 1)) and np.all(W > 0)


def test_dihedral_table_is_the_square_group():
    pts = np.array([[0.2, 0.7], [0.9, 0.1], [0.5, 0.5]])
    imgs = set()
    for k in range(8):
        out = singular.apply_dihedral(k, pts)
        assert np.all((out >= 0) & (out <= 1))
        corners = {singular.dihedral_corner(k, s, t) for s, t in [(0, 0), (1, 0), (1, 1), (0, 1)]}
        assert corners == {0, 1, 2, 3}
        imgs.add(tuple(np.round(out.ravel(), 12)))
    assert len(imgs) == 8
