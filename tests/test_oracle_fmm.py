"""Pins for the oracle's cluster tree and interpolation far field."""
import numpy as np
import pytest

from oracle import fmm, galerkin, tree


class PolynomialKernel:
    """A localised kernel that is a polynomial of degree < 6 in each parameter
    variable: the degree-(q-1) interpolant reproduces it exactly for q >= 6."""
    is_complex = False

    def __call__(self, FA, kA, uvA, pA, FB, kB, uvB, pB):
        a, b = uvA[..., 0], uvA[..., 1]
        c, d = uvB[..., 0], uvB[..., 1]
        return (1 + a * c + b * d + 0.1 * pA - 0.05 * pB) ** 2 + a ** 3 * d ** 2 - b * c ** 4


def test_block_tree_partitions_all_element_pairs(sphere):
    m, eta = 2, 1.6
    cg = tree.ClusterGeometry(sphere)
    near, far = tree.block_cluster_tree(sphere, m, eta, cg)
    E = len(sphere) * 4 ** m
    cover = np.zeros((E, E), dtype=int)

    def leaves(cl):
        patch, level, ix, iy = cl
        s = 2 ** (m - level)
        return [patch * 4 ** m + (iy * s + dy) * 2 ** m + ix * s + dx
                for dy in range(s) for dx in range(s)]

    for s, t in near + far:
        for a in leaves(s):
            for b in leaves(t):
                cover[a, b] += 1
    assert np.all(cover == 1)
    for s, t in far:
        assert cg.admissible(s, t, eta)
        if s[1] > 0:
            ps = (s[0], s[1] - 1, s[2] // 2, s[3] // 2)
            pt = (t[0], t[1] - 1, t[2] // 2, t[3] // 2)
            assert not cg.admissible(ps, pt, eta)
    for s, t in near:
        assert s[1] == m and not cg.admissible(s, t, eta)
    # symmetric structure: (s, t) far iff (t, s) far
    assert set(far) == {(t, s) for s, t in far}


def test_fmm_exact_for_polynomial_kernel(sphere):
    disc = galerkin.Discretisation(sphere, 1, 2, PolynomialKernel())
    A = disc.dense_matrix()
    F = fmm.FMMOperator(disc, 6, 1.6)
    assert len(F.far) > 0
    x = np.random.default_rng(1).normal(size=disc.mesh.n_dofs)
    y, y0 = F.matvec(x), A @ x
    assert np.max(np.abs(y - y0)) < 1e-13 * np.max(np.abs(y0))
    rows = [0, 7, 33, disc.mesh.n_dofs - 1]
    np.testing.assert_allclose(F.rows(rows, x)[:, 0], y[rows], rtol=0, atol=1e-13 * np.max(np.abs(y0)))


def test_fmm_error_decays_with_q(laplace_p2m2):
    disc, A = laplace_p2m2
    x = np.random.default_rng(2).normal(size=disc.mesh.n_dofs)
    y0 = A @ x
    errs, cache = [], {}
    for q in (2, 4, 6, 8):
        y = fmm.FMMOperator(disc, q, 1.6, near_block_cache=cache).matvec(x)
        errs.append(np.max(np.abs(y - y0)) / np.max(np.abs(y0)))
    assert all(e2 < 0.05 * e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[2] < 1e-7


def test_chebyshev_lagrange():
    z = fmm.chebyshev_nodes(6)
    np.testing.assert_allclose(fmm.lagrange_values(z, z), np.eye(6), atol=1e-14)
    x = np.linspace(0, 1, 17)
    np.testing.assert_allclose(fmm.lagrange_values(z, x).sum(axis=1), 1.0, atol=1e-13)
    # reproduces polynomials of degree 5 exactly
    L = fmm.lagrange_values(z, x)
    np.testing.assert_allclose(L @ (z ** 5 - 2 * z ** 2), x ** 5 - 2 * x ** 2, atol=1e-13)
