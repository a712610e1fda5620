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


def _potential_points():
    from conftest import seeded_ball_points
    rng = np.random.default_rng(61)
    far = rng.normal(size=(8, 3))
    far *= 3.0 / np.linalg.norm(far, axis=1)[:, None]
    close = rng.normal(size=(4, 3))
    close *= 1.08 / np.linalg.norm(close, axis=1)[:, None]
    return np.concatenate([far, close, seeded_ball_points(4, 0.5, 62)])


def test_fmm_potential_exact_for_polynomial_point_kernel(sphere):
    # a point kernel of degree < q in each parameter variable is interpolated
    # exactly, so the tree sum equals the direct Gauss sum over all elements
    disc = galerkin.Discretisation(sphere, 2, 2, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, 6, 1.6)

    def pk(X, F, k, uv, patch):
        u, v = uv[:, 0], uv[:, 1]
        s = 1.0 + X @ np.array([0.3, -0.2, 0.1])
        return s[:, None] * ((1 + u * v + 0.1 * patch) ** 2 + u ** 3 * v ** 2 - v * u ** 4)[None, :]

    w = np.random.default_rng(63).normal(size=(op.mesh.n_dofs, 2))
    P = _potential_points()
    u = op.potential(w, P, point_kernel=pk)
    counts = np.array(op.potential_counts)
    assert counts[:, 0].sum() > 0 and counts[:, 1].sum() > 0
    me = op.mesh
    direct = np.zeros_like(u)
    for e in range(me.n_elements):
        uvq, F, k, wq, b, patch = disc._product_points(e, "regular")
        direct += pk(P, F, k, uvq, patch) @ (wq[:, None] * (b @ w[me.local_dofs(e)]))
    assert np.max(np.abs(u - direct)) < 1e-13 * np.max(np.abs(direct))


def test_fmm_potential_without_admissible_clusters_is_direct(sphere):
    from oracle import solve
    disc = galerkin.Discretisation(sphere, 1, 2, galerkin.HelmholtzKernel(3.0))
    op = fmm.FMMOperator(disc, 4, 1e9)
    rng = np.random.default_rng(64)
    w = rng.normal(size=op.mesh.n_dofs) + 1j * rng.normal(size=op.mesh.n_dofs)
    P = _potential_points()
    u = op.potential(w, P)
    assert all(c == (0, op.mesh.n_elements) for c in op.potential_counts)
    u0 = solve.potential(disc, w, P)
    assert np.max(np.abs(u - u0)) < 1e-14 * np.max(np.abs(u0))


@pytest.mark.parametrize("kernel", [galerkin.LaplaceKernel(), galerkin.HelmholtzKernel(3.0)], ids=["laplace", "helmholtz"])
def test_fmm_potential_error_decays_with_q(sphere, kernel):
    from oracle import solve
    disc = galerkin.Discretisation(sphere, 2, 2, kernel)
    rng = np.random.default_rng(65)
    w = rng.normal(size=disc.mesh.n_dofs)
    P = _potential_points()
    u0 = solve.potential(disc, w, P)
    errs = []
    for q in (4, 6, 8):
        u = fmm.FMMOperator(disc, q, 1.6).potential(w, P)
        errs.append(np.max(np.abs(u - u0)) / np.max(np.abs(u0)))
    assert errs[0] > errs[1] > errs[2]
    # measured: Laplace 3.8e-3, 2.2e-4, 9.5e-7; Helmholtz (kappa = 3, so
    # kappa diam reaches ~3 on the largest admissible clusters) 1.1e-2, 9.2e-4,
    # 1.9e-5; the points 0.08 outside the sphere set these figures
    assert errs[2] < (1e-4 if kernel.is_complex else 1e-5), errs
