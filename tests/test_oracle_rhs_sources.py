"""Pins for the oracle's FMM-compressed right-hand side of point sources,
FMMOperator.rhs_sources: b_i = int g b_i with g = sum_j c_j u*(., y_j) and the
far field of each source interpolated on the clusters admissible for it
(Sec. 3.2 right-hand side, Sec. 4.2 interpolation).

* Adjointness: u* is symmetric, so for every density w
      w . b(Y, c) = sum_j c_j u_w(y_j),
  u_w the interpolated potential of w (FMMOperator.potential, pinned in
  tests/test_oracle_fmm.py) - the same clusters, nodes and Gauss points.
* Nothing admissible (eta huge): the direct Galerkin right-hand side
  Discretisation.rhs of g.
* A point kernel polynomial of degree < q in the parameters: interpolation is
  exact, so the result equals the direct Gauss sums with that kernel.
* The true kernel: the error against the direct right-hand side falls as q
  grows.
"""
import numpy as np
import pytest

from oracle import fmm, galerkin, geometry


def _sources(n, seed, radii):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * np.asarray(radii)[rng.integers(0, len(radii), size=n)][:, None]


@pytest.fixture(scope="module")
def lap_q5():
    disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 2, galerkin.LaplaceKernel())
    return fmm.FMMOperator(disc, 5, 1.6)


def _g(kernel, Y, c):
    def g(F):
        return sum(galerkin.fundamental_solution(kernel, F, y[None, :])[:, None] * c[j][None, :]
                   for j, y in enumerate(Y))
    return g


def test_adjoint_of_interpolated_potential(lap_q5):
    op = lap_q5
    Y = _sources(12, 1, [0.4, 2.5, 4.0])
    c = np.random.default_rng(2).normal(size=(12, 2))
    b = op.rhs_sources(Y, c)
    assert sum(n for n, _ in op.rhs_counts) > 0 and sum(n for _, n in op.rhs_counts) > 0
    w = np.random.default_rng(3).normal(size=(op.mesh.n_dofs, 3))
    u = op.potential(w, Y)                                  # (nsrc, 3)
    lhs = w.T @ b                                           # (3, 2)
    rhs = u.T @ c
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))


def test_helmholtz_adjoint_without_conjugation():
    disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 2, galerkin.HelmholtzKernel(2.5))
    op = fmm.FMMOperator(disc, 5, 1.6)
    Y = _sources(8, 4, [0.3, 3.0])
    rng = np.random.default_rng(5)
    c = rng.normal(size=(8, 1)) + 1j * rng.normal(size=(8, 1))
    w = rng.normal(size=(op.mesh.n_dofs, 1)) + 1j * rng.normal(size=(op.mesh.n_dofs, 1))
    b = op.rhs_sources(Y, c)
    u = op.potential(w, Y)
    lhs = (w.T @ b)[0, 0]
    rhs = (u.T @ c)[0, 0]
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_nothing_admissible_is_the_direct_rhs():
    disc = galerkin.Discretisation(geometry.unit_sphere(), 2, 1, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, 4, 1e9)
    Y = _sources(5, 6, [0.5, 3.0])
    c = np.random.default_rng(7).normal(size=(5, 2))
    b = op.rhs_sources(Y, c)
    assert all(n == 0 for n, _ in op.rhs_counts)
    ref = disc.rhs(_g(disc.kernel, Y, c))
    assert np.max(np.abs(b - ref)) < 1e-13 * np.max(np.abs(ref))


def test_parameter_polynomial_kernel_is_exact(lap_q5):
    op = lap_q5
    me = op.mesh

    def pk(X, F, k, uv, patch):
        # replaces u* k: degree 4 < q = 5 in each parameter, different per patch and point
        s = 1.0 + 0.1 * patch + 0.05 * X[:, :1]
        return s * (uv[None, :, 0] ** 4 - 2 * uv[None, :, 0] * uv[None, :, 1] ** 3 + uv[None, :, 1])

    Y = _sources(6, 8, [0.5, 3.0])
    c = np.random.default_rng(9).normal(size=(6, 1))
    b = op.rhs_sources(Y, c, point_kernel=pk)
    assert sum(n for n, _ in op.rhs_counts) > 0
    ref = np.zeros_like(b)
    for e in range(me.n_elements):
        uvq, F, k, wq, bq, patch = op.disc._product_points(e, "regular")
        for j, y in enumerate(Y):
            ref[me.local_dofs(e)] += bq.T @ np.outer(wq * pk(y[None, :], F, k, uvq, patch)[0], c[j])
    assert np.max(np.abs(b - ref)) < 1e-12 * np.max(np.abs(ref))


def test_error_against_direct_falls_with_q():
    Y = _sources(6, 10, [0.3, 2.0])
    c = np.random.default_rng(11).normal(size=(6, 1))
    errs = []
    for q in (3, 5, 7):
        disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 2, galerkin.LaplaceKernel())
        op = fmm.FMMOperator(disc, q, 1.6)
        b = op.rhs_sources(Y, c)
        ref = disc.rhs(_g(disc.kernel, Y, c))
        errs.append(np.max(np.abs(b - ref)) / np.max(np.abs(ref)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5, errs
