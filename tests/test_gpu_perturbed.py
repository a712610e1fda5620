"""Perturbed mappings (Sec. 5): the sphere's face maps composed with the
piecewise-linear f in both parameters.  FP64 library against the FP64 oracle
at 1e-12 (dense and FMM operator, right-hand side, potential), and the
solution's potential error against the plain parametrisation."""
import numpy as np
import pytest

from gpu_common import gpu_matvec, lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
X0 = np.array([0.9, 0.9, 0.9])


def _handle(p, m, q, kernel=0, kappa=0.0, perturbed=True):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(perturbed=perturbed),
                         ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kernel, kappa=kappa))
    ibem.ibem_assemble(h)
    return h


@pytest.fixture(scope="module")
def pert_fmm_p2m2():
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.perturbed_sphere(), 2, 2, galerkin.LaplaceKernel())
    return fmm.FMMOperator(disc, 6, 1.6)


def test_fmm_and_dense_operator(pert_fmm_p2m2):
    op = pert_fmm_p2m2
    x = np.random.default_rng(51).normal(size=(2, op.mesh.n_dofs))
    h = _handle(2, 2, 6)
    assert rel_err(gpu_matvec(h, x), np.stack([op.matvec(xi) for xi in x])) < TOL64
    lib().ibem_destroy(h)
    # dense mode (no far field) against the oracle's dense matrix
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.perturbed_sphere(), 1, 1, galerkin.LaplaceKernel())
    A = disc.dense_matrix()
    h = _handle(1, 1, 0)
    x = np.random.default_rng(52).normal(size=(2, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    lib().ibem_destroy(h)


def test_dense_helmholtz():
    import torch
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.perturbed_sphere(), 1, 1, galerkin.HelmholtzKernel(2.0))
    A = disc.dense_matrix()
    ibem = lib()
    h = _handle(1, 1, 0, kernel=1, kappa=2.0)
    rng = np.random.default_rng(53)
    x = rng.normal(size=(2, A.shape[0])) + 1j * rng.normal(size=(2, A.shape[0]))
    xd = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, 2, 0)
    y = yd.cpu().numpy()
    assert rel_err(y[..., 0] + 1j * y[..., 1], x @ A.T) < TOL64
    ibem.ibem_destroy(h)


def test_rhs_and_potential(pert_fmm_p2m2):
    import torch
    from oracle import solve
    ibem = lib()
    op = pert_fmm_p2m2
    disc = op.disc
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - X0, axis=1))
    b0 = disc.rhs(g)[:, 0]
    h = _handle(2, 2, 6)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gq = torch.from_numpy(g(qp.cpu().numpy())).cuda()
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    assert rel_err(b.cpu().numpy(), b0) < TOL64
    w = np.random.default_rng(54).normal(size=info.ndof)
    from conftest import seeded_ball_points
    P = seeded_ball_points(20, 0.5, 55)
    u0 = solve.potential(disc, w, P)[:, 0]
    u = torch.empty(20, dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, torch.from_numpy(w).cuda(), 1, torch.from_numpy(P).cuda(), u)
    assert rel_err(u.cpu().numpy(), u0) < TOL64
    ibem.ibem_destroy(h)


def _potential_error(p, m, q, perturbed):
    """Interior Laplace problem with a point source outside the sphere: the
    max-norm potential error at 100 seeded points of the ball r = 0.5."""
    import torch
    ibem = lib()
    h = _handle(p, m, q, perturbed=perturbed)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - X0, axis=1))
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, torch.from_numpy(g(qp.cpu().numpy())).cuda(), 1, b)
    w = torch.zeros_like(b)
    s = ibem.ibem_solve(h, b, w, 1, rtol=1e-12, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    assert s.rel_residual <= 1e-12
    from conftest import seeded_ball_points
    P = seeded_ball_points(100, 0.5, 170809162)
    u = torch.empty(100, dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 1, torch.from_numpy(P).cuda(), u)
    ibem.ibem_destroy(h)
    return float(np.max(np.abs(u.cpu().numpy() - g(P))))


def test_perturbation_costs_accuracy_uncompressed():
    # Sec. 5: the kinked parametrisation lowers the regularity of the discrete
    # space; without compression (q = 0) the perturbed sphere's potential error
    # at p = 2 stays orders of magnitude above the plain sphere's at equal
    # (p, m).  (The oracle checks the h^3 rate at p = 1 from m = 1 to 2; at
    # m = 3 the 8-point rules on the elements that contain a kink, where the
    # surface measure jumps, set the error: 2.2e-3 at m = 2, 5.9e-3 at m = 3.)
    plain = [_potential_error(2, m, 0, False) for m in (2, 3)]
    pert = [_potential_error(2, m, 0, True) for m in (2, 3)]
    assert plain[1] < plain[0]
    assert min(pert) > 100 * max(plain), (plain, pert)


def test_interpolation_stalls_across_kinks():
    # The FMM interpolates the localised kernel, which carries the surface
    # measure; across the kinks of f that measure jumps (slopes 1/2 and 7/4), so
    # the interpolation error of the operator stops falling with q, while on the
    # plain sphere it falls geometrically
    def op_err(perturbed, q):
        x = np.random.default_rng(56).normal(size=(2, 150))
        hd, hf = _handle(1, 2, 0, perturbed=perturbed), _handle(1, 2, q, perturbed=perturbed)
        y0, y = gpu_matvec(hd, x), gpu_matvec(hf, x)
        lib().ibem_destroy(hd)
        lib().ibem_destroy(hf)
        return rel_err(y, y0)
    assert op_err(False, 8) < 1e-8 < 1e-6 < op_err(True, 8)
    assert op_err(True, 8) > 0.1 * op_err(True, 4)
