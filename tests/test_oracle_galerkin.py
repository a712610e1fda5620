"""Pins for the oracle's dense Galerkin single-layer matrix on the unit sphere.

On the unit sphere the single-layer operator is diagonal in spherical harmonics:
V Y_l = Y_l / (2l + 1) (Laplace) and V Y_l = i k j_l(k) h_l(k) Y_l (Helmholtz).
For l = 0 that gives V 1 = 1 and V 1 = sin(k) e^{ik} / k; since the B-splines sum
to one, A @ ones must equal lambda_0 times the row integrals of the basis.
"""
import numpy as np
import pytest

from oracle import galerkin, solve


def _row_integrals(disc):
    return disc.rhs(lambda F: np.ones(len(F)))[:, 0]


def test_laplace_constant_eigenfunction_p0(sphere):
    disc = galerkin.Discretisation(sphere, 0, 1, galerkin.LaplaceKernel())
    A = disc.dense_matrix()
    mass = _row_integrals(disc)
    assert np.max(np.abs(A @ np.ones(len(mass)) - mass)) < 1e-9 * np.max(mass)


def test_laplace_constant_eigenfunction_p2(laplace_p2m2):
    disc, A = laplace_p2m2
    mass = _row_integrals(disc)
    assert np.max(np.abs(A @ np.ones(len(mass)) - mass)) < 1e-11 * np.max(mass)


def test_laplace_matrix_symmetric_positive(laplace_p2m2):
    _, A = laplace_p2m2
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_helmholtz_constant_eigenfunction_and_symmetry(sphere):
    k = 2.0
    disc = galerkin.Discretisation(sphere, 0, 1, galerkin.HelmholtzKernel(k))
    A = disc.dense_matrix()
    mass = _row_integrals(disc)
    lam = np.sin(k) * np.exp(1j * k) / k
    # 8-point Gauss on the oscillatory factor over m = 1 elements limits this to ~1e-8
    assert np.max(np.abs(A @ np.ones(len(mass)) - lam * mass)) < 2e-8 * np.max(mass)
    # complex-symmetric (no conjugation in the bilinear form), not Hermitian
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A - A.conj().T)) > 1e-3 * np.max(np.abs(A))


def _density_error_y1(disc, A, scale=3.0):
    # L2 error of the computed density against scale * z for data g = z
    b = disc.rhs(lambda F: F[:, 2])[:, 0]
    w = solve.dense_solve(A, b)
    me = disc.mesh
    err2, nrm2 = 0.0, 0.0
    for e in range(me.n_elements):
        _, F, k, wq, bas, _ = disc._product_points(e, "regular")
        dens = bas @ w[me.local_dofs(e)]
        err2 += np.sum(wq * k * np.abs(dens - scale * F[:, 2]) ** 2)
        nrm2 += np.sum(wq * k * np.abs(scale * F[:, 2]) ** 2)
    return np.sqrt(err2 / nrm2), w


def test_laplace_density_of_first_harmonic(sphere, laplace_p2m2):
    # g = z = Y_1 on the sphere -> density w = 3 z (eigenvalue 1/3), potential u = z
    # inside; the L2 density error falls like h^{p+1} (Lemma 3.1).
    disc, A = laplace_p2m2
    err2, w = _density_error_y1(disc, A)
    disc1 = galerkin.Discretisation(sphere, 2, 1, galerkin.LaplaceKernel())
    err1, _ = _density_error_y1(disc1, disc1.dense_matrix())
    assert err2 < 5e-3
    assert err1 / err2 > 4.0          # h^3 would give 8
    from conftest import seeded_ball_points
    P = seeded_ball_points(50, 0.5, 3)
    u = solve.potential(disc, w, P)[:, 0]
    assert np.max(np.abs(u - P[:, 2])) < 5e-6


def test_helmholtz_density_of_first_harmonic(sphere):
    # On the unit sphere the Helmholtz single layer maps Y_l to i k j_l(k) h_l(k) Y_l
    # (spherical Bessel and first-kind Hankel functions); for g = z the density is
    # z / (i k j_1(k) h_1(k)).  A sign or phase error in the kernel, a dropped
    # Jacobian or a conjugated bilinear form changes this l = 1 eigenvalue.
    from scipy.special import spherical_jn, spherical_yn
    k = 2.0
    lam = 1j * k * spherical_jn(1, k) * (spherical_jn(1, k) + 1j * spherical_yn(1, k))
    errs = []
    for m in (1, 2):
        disc = galerkin.Discretisation(sphere, 2, m, galerkin.HelmholtzKernel(k))
        err, _ = _density_error_y1(disc, disc.dense_matrix(), scale=1.0 / lam)
        errs.append(err)
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 4.0


def test_pair_classes_counts(laplace_p2m2):
    disc, _ = laplace_p2m2
    from collections import Counter
    E = disc.mesh.n_elements
    c = Counter(disc.pair_class(a, b)[0] for a in range(E) for b in range(E))
    # 96 elements: each has itself; 4 edge neighbours; 4 vertex neighbours except
    # the 24 cube-corner elements, which have 3 (three faces meet there).
    assert c["identical"] == 96
    assert c["edge"] == 96 * 4
    assert c["vertex"] == 96 * 4 - 24
