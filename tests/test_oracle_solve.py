"""Pins for the oracle's right-hand side, solvers and potential evaluation."""
import numpy as np
import pytest

from conftest import seeded_ball_points
from oracle import galerkin, solve

X0 = np.array([0.9, 0.9, 0.9])


def _point_source(F, src):
    return 1.0 / (4 * np.pi * np.linalg.norm(F - src, axis=1))


def test_interior_laplace_point_source(laplace_p2m2):
    # Harmonic data from a source outside the unit ball: u = g inside (Eq. repform).
    disc, A = laplace_p2m2
    b = disc.rhs(lambda F: _point_source(F, X0))[:, 0]
    w = solve.dense_solve(A, b)
    P = seeded_ball_points(100, 0.5, 170809162)
    u = solve.potential(disc, w, P)[:, 0]
    assert np.max(np.abs(u - _point_source(P, X0))) < 2e-6


def test_cg_matches_direct(laplace_p2m2):
    disc, A = laplace_p2m2
    b = disc.rhs(lambda F: _point_source(F, X0))[:, 0]
    w0 = solve.dense_solve(A, b)
    w, it = solve.cg(lambda v: A @ v, b, rtol=1e-10, diag=np.diag(A).copy())
    assert it < 200
    assert np.linalg.norm(b - A @ w) <= 1e-10 * np.linalg.norm(b) * 1.0001
    assert np.linalg.norm(w - w0) < 1e-6 * np.linalg.norm(w0)


def test_exterior_helmholtz_point_source(sphere):
    k = 2.0
    v = np.array([0.1, 0.2, -0.1])
    disc = galerkin.Discretisation(sphere, 2, 1, galerkin.HelmholtzKernel(k))
    A = disc.dense_matrix()

    def g(F):
        r = np.linalg.norm(F - v, axis=1)
        return np.exp(1j * k * r) / (4 * np.pi * r)

    b = disc.rhs(g)[:, 0]
    w = solve.dense_solve(A, b)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(40, 3))
    P = 3.0 * d / np.linalg.norm(d, axis=1)[:, None]
    u = solve.potential(disc, w, P)[:, 0]
    assert np.max(np.abs(u - g(P))) < 2e-4 * np.max(np.abs(g(P)))
    wg, it = solve.gmres(lambda x: A @ x, b, rtol=1e-10, restart=30, diag=np.diag(A).copy())
    assert np.linalg.norm(b - A @ wg) <= 1.0001e-10 * np.linalg.norm(b)
    assert np.linalg.norm(wg - w) < 1e-7 * np.linalg.norm(w)


def test_perturbed_mapping_rate_drop():
    # Sec. 5 (perturbed mappings): with the kinked reparametrisation the interior
    # point-source potential converges only like h^3 (the lowest-order rate), and
    # at equal (p, m) its error is orders of magnitude above the plain sphere's
    from conftest import seeded_ball_points
    from oracle import geometry
    x0 = np.array([0.9, 0.9, 0.9])
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - x0, axis=1))
    P = seeded_ball_points(50, 0.5, 170809162)
    err = {}
    for name, pats in (("plain", geometry.unit_sphere()), ("perturbed", geometry.perturbed_sphere())):
        for m in (1, 2):
            disc = galerkin.Discretisation(pats, 1, m, galerkin.LaplaceKernel())
            w = solve.dense_solve(disc.dense_matrix(), disc.rhs(g)[:, 0])
            err[name, m] = np.max(np.abs(solve.potential(disc, w, P)[:, 0] - g(P)))
    assert 6.0 < err["perturbed", 1] / err["perturbed", 2] < 12.0      # h^3 gives 8
    assert err["perturbed", 2] > 100 * err["plain", 2]


def test_mie_series_cancels_the_plane_wave_on_the_sphere():
    # the closed form itself: u_i + u_s = 0 on the unit sphere
    from closed_forms import mie_sound_soft
    rng = np.random.default_rng(11)
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    X = rng.normal(size=(50, 3))
    X /= np.linalg.norm(X, axis=1)[:, None]
    for k in (1.0, 4.0):
        assert np.max(np.abs(np.exp(1j * k * (X @ d)) + mie_sound_soft(k, d, X))) < 1e-12


def test_sound_soft_plane_wave_matches_mie_series(sphere):
    # Helmholtz, sound-soft sphere: g = -e^{i k d.x} on the boundary, V w = g,
    # scattered field u_s = V~ w outside (Eq. repform) against the Mie series at
    # 30 points on r = 3; degree 2 beats degree 1 on the same mesh
    from closed_forms import mie_sound_soft
    k = 2.0
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    rng = np.random.default_rng(7)
    P = rng.normal(size=(30, 3))
    P = 3.0 * P / np.linalg.norm(P, axis=1)[:, None]
    ue = mie_sound_soft(k, d, P)
    err = {}
    for p in (1, 2):
        disc = galerkin.Discretisation(sphere, p, 1, galerkin.HelmholtzKernel(k))
        b = disc.rhs(lambda F: -np.exp(1j * k * (F @ d)))[:, 0]
        w = solve.dense_solve(disc.dense_matrix(), b)
        err[p] = np.max(np.abs(solve.potential(disc, w, P)[:, 0] - ue)) / np.max(np.abs(ue))
    assert err[1] < 6e-3 and err[2] < 1e-3, err
    assert err[2] < err[1] / 4.0, err
