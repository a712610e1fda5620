"""Pins for the graded Gauss orders of near pairs (Sec. 4 item 4: the order is
raised logarithmically towards the singularity, up to 40).  The rule is a
reading: a non-touching pair takes n_regular + grading * k points per
direction, k the number of halvings of rho = dist / diam below 3/4.

Flat pin: on the unit square refined to level m (element size h), two elements
of a row with one element between them are the outer squares A, B of three
consecutive h x h squares A G B.  For p = 0 (indicator basis) and the Laplace
kernel their Galerkin entry is, by inclusion-exclusion over the rectangles
AGB, AG, GB and G,
    X = [I(3h, h) - 2 I(2h, h) + I(h, h)] / (2 * 4 pi),
I(a, b) the self-interaction of an a x b rectangle (computed as in
tests/test_oracle_singular.py).  The pair is near-singular (rho < 1/2: both
elements split 2 x 2); the graded order, used on every sub-square pair, must
bring the oracle's entry to this value where the base order does not.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import galerkin, geometry

_K1 = [0.0, 0.0, 1.0, 1.0]


def _rect(a, b):
    f = lambda v, u: (a - u) * (b - v) / np.hypot(u, v)
    val, _ = integrate.dblquad(f, 0, a, 0, b, epsabs=1e-15, epsrel=1e-14)
    return 4 * val


def _unit_square():
    ctrl = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0], [1.0, 1.0, 0.0]]])
    return [geometry.NurbsPatch(1, 1, _K1, _K1, ctrl, np.ones((2, 2)))]


def test_order_is_logarithmic_in_the_distance():
    base, g, diam = 4, 3, 1.0
    # at and above 3/4 of the diameter: the base order; zero distance: the cap
    assert galerkin.graded_order(base, g, 0.75, diam) == base
    assert galerkin.graded_order(base, g, 5.0, diam) == base
    assert galerkin.graded_order(base, g, 0.0, diam) == 40
    # grading 0: the base order everywhere
    assert all(galerkin.graded_order(base, 0, d, diam) == base for d in (0.0, 1e-9, 0.3, 2.0))
    # every halving of the distance below 3/4 diam adds `g` points, up to 40
    prev = galerkin.graded_order(base, g, 0.7, diam)
    assert prev == base + g
    d = 0.7
    for _ in range(30):
        d /= 2.0
        n = galerkin.graded_order(base, g, d, diam)
        assert n == min(prev + g, 40)
        prev = n
    assert prev == 40
    # scale invariance: only the ratio matters
    for d in (0.05, 0.2, 0.5, 0.74):
        assert galerkin.graded_order(base, g, d, diam) == galerkin.graded_order(base, g, 8 * d, 8 * diam)


@pytest.fixture(scope="module")
def flat_pair():
    m = 2
    h = 0.5 ** m
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            exact = (_rect(3 * h, h) - 2 * _rect(2 * h, h) + _rect(h, h)) / (2 * 4 * np.pi)
    return m, exact


def _entry(m, n_regular, grading):
    disc = galerkin.Discretisation(_unit_square(), 0, m, galerkin.LaplaceKernel(), n_regular=n_regular,
                                   grading=grading)
    me = disc.mesh
    # elements (ix, iy) = (0, 0) and (2, 0) of the patch
    eA = next(e for e in range(me.n_elements) if me.element(e) == (0, 0, 0))
    eB = next(e for e in range(me.n_elements) if me.element(e) == (0, 2, 0))
    assert disc.pair_class(eA, eB)[0] == "nearsing"      # rho < 1/2: 2 x 2 sub-squares
    return disc.pair_block(eA, eB)[0, 0], disc.pair_order(eA, eB)


def test_graded_pair_reaches_the_inclusion_exclusion_value(flat_pair):
    m, exact = flat_pair
    base, n0 = _entry(m, 2, 0)
    graded, n1 = _entry(m, 2, 6)
    # rho = (2 - sqrt 2) / sqrt 2 = 0.414: one halving below 3/4
    assert n0 == 2 and n1 == 8
    err0 = abs(base - exact) / exact
    err1 = abs(graded - exact) / exact
    assert err0 > 1e-5, err0
    assert err1 < 1e-9, err1
    # the same order given as the base order gives the same entry
    same, n2 = _entry(m, 8, 0)
    assert n2 == 8 and abs(same - graded) <= 1e-15 * abs(exact)


def test_cap_reaches_forty_points(flat_pair):
    m, exact = flat_pair
    val, n = _entry(m, 4, 40)
    assert n == 40
    assert abs(val - exact) / exact < 1e-12
