"""Pins for the oracle's Gauss rules, B-splines and space dimensions."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bspline
from oracle.gauss import gauss_legendre

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 20, 40])
def test_gauss_exact_for_monomials(n):
    # Gauss with n points integrates x^k on [0, 1] exactly for k <= 2n - 1.
    x, w = gauss_legendre(n)
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1))
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14 * max(1, k)
    # and not for 2n: the rule has a non-zero error there (visible for small n)
    if n <= 8:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-15


def _frac(s):
    return float(Fraction(s))


def _fig_pieces():
    out = []
    with open(os.path.join(GOLDEN, "fig_splines.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, j, lo, hi, expr = (t.strip() for t in line.split("|"))
            out.append((int(p), int(j), _frac(lo), _frac(hi), expr))
    return out


def test_bsplines_match_figure_pieces():
    # Fig. fig::splines: open knot vectors with interior knots 1/3, 2/3.
    for p, j, lo, hi, expr in _fig_pieces():
        knots = [0.0] * (p + 1) + [1 / 3, 2 / 3] + [1.0] * (p + 1)
        x = np.linspace(lo, hi, 23)[1:-1]
        got = bspline.basis_values(knots, p, x)[:, j]
        want = np.array([eval(expr, {"x": xi}) for xi in x])
        np.testing.assert_allclose(got, want, atol=1e-14)


def test_bsplines_vanish_outside_printed_pieces():
    pieces = _fig_pieces()
    for p in (1, 2):
        knots = [0.0] * (p + 1) + [1 / 3, 2 / 3] + [1.0] * (p + 1)
        x = np.linspace(0, 1, 301)
        b = bspline.basis_values(knots, p, x)
        for j in range(b.shape[1]):
            inside = np.zeros_like(x, dtype=bool)
            for pp, jj, lo, hi, _ in pieces:
                if pp == p and jj == j:
                    inside |= (x >= lo) & (x <= hi)
            assert np.all(b[~inside, j] == 0.0)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("m", [0, 1, 3])
def test_partition_of_unity_and_support(p, m):
    knots = bspline.open_uniform_knots(p, m)
    assert len(knots) == 2 ** m + 2 * p + 1
    x = np.concatenate([np.random.default_rng(p + 7 * m).random(200), [0.0, 1.0]])
    b = bspline.basis_values(knots, p, x)
    assert b.shape[1] == 2 ** m + p
    np.testing.assert_allclose(b.sum(axis=1), 1.0, atol=1e-14)
    assert np.all(b >= -1e-15)
    # on element i only b_i..b_{i+p} are non-zero
    for xi, row in zip(x, b):
        i = min(int(xi * 2 ** m), 2 ** m - 1)
        nz = np.nonzero(np.abs(row) > 0)[0]
        assert set(nz) <= set(range(i, i + p + 1))


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_single_element_bsplines_are_bernstein(p):
    # With m = 0 the B-splines of Xi_{p,0} are the Bernstein polynomials (Sec. 4.3).
    from math import comb
    x = np.linspace(0, 1, 41)
    b = bspline.basis_values(bspline.open_uniform_knots(p, 0), p, x)
    for i in range(p + 1):
        np.testing.assert_allclose(b[:, i], comb(p, i) * x ** i * (1 - x) ** (p - i), atol=1e-14)


def test_derivatives_against_finite_differences():
    knots = bspline.open_uniform_knots(3, 2)
    x = np.random.default_rng(3).random(50) * 0.98 + 0.01
    hstep = 1e-6
    fd = (bspline.basis_values(knots, 3, x + hstep) - bspline.basis_values(knots, 3, x - hstep)) / (2 * hstep)
    np.testing.assert_allclose(bspline.basis_derivatives(knots, 3, x), fd, atol=2e-7)


def test_space_dimensions_match_table():
    # dim S* = n (2^m (p+1))^2 against Table tab::mat::sph; dim S = n (2^m + p)^2.
    typos = {("torus", 1, 4)}
    with open(os.path.join(GOLDEN, "superspace_dims.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            geo, n, p, vals = (t.strip() for t in line.split("|"))
            for m, v in enumerate(vals.split(), start=1):
                got = bspline.superspace_dimension(int(n), int(p), m)
                if (geo, int(p), m) in typos:
                    assert got != int(v) and got == 16384
                else:
                    assert got == int(v), (geo, p, m)
    assert bspline.space_dimension(6, 2, 2) == 216
    assert bspline.space_dimension(6, 3, 5) == 7350
    assert bspline.space_dimension(6, 2, 6) == 26136
    assert bspline.space_dimension(6, 2, 7) == 101400


def test_local_window_equals_full_knot_vector(sphere):
    # the element-local evaluation used by the mesh equals the full recursion
    from oracle.mesh import Mesh
    me = Mesh(sphere, 3, 3)
    rng = np.random.default_rng(9)
    for e in (0, 5, 27, 63):
        st = rng.random((40, 2))
        uv = me.to_patch(e, st)
        _, ix, iy = me.element(e)
        full_u = bspline.basis_values(me.knots, 3, uv[:, 0])[:, ix:ix + 4]
        full_v = bspline.basis_values(me.knots, 3, uv[:, 1])[:, iy:iy + 4]
        want = (full_v[:, :, None] * full_u[:, None, :]).reshape(40, -1)
        assert np.array_equal(me.local_basis(e, uv), want)
