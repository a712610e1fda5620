"""The paper's torus (16 rational biquadratic patches) and Fichera cube (24
bilinear squares with re-entrant edges and corner), Sec. 5: the FP64 library
against the FP64 oracle at 1e-12 (dense, FMM, sampled FMM rows at full size,
Laplace and Helmholtz), and the interior Laplace problem with a point source
outside the solid."""
import numpy as np
import pytest

import shapes
from gpu_common import gpu_matvec, lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _oracle_patches(name):
    from oracle import geometry
    return [geometry.NurbsPatch(*s) for s in getattr(shapes, name)()]


def _handle(name, p, m, q, kernel=0, kappa=0.0, assemble=True):
    ibem = lib()
    h = ibem.ibem_create(ibem.nurbs_patches(getattr(shapes, name)()),
                         ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kernel, kappa=kappa))
    if assemble:
        ibem.ibem_assemble(h)
    return h


def _cmatvec(h, x):
    import torch
    ibem = lib()
    xd = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], 0)
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1]


def test_dense_torus():
    from oracle import galerkin
    disc = galerkin.Discretisation(_oracle_patches("torus"), 1, 1, galerkin.LaplaceKernel())
    A = disc.dense_matrix()
    h = _handle("torus", 1, 1, 0)
    x = np.random.default_rng(81).normal(size=(2, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    lib().ibem_destroy(h)


def test_fmm_fichera():
    # m = 1 already has 3,522 admissible blocks on the L-shaped surface
    from oracle import fmm, galerkin
    disc = galerkin.Discretisation(_oracle_patches("fichera"), 1, 1, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, 6, 1.6)
    assert len(op.far) == 3522
    h = _handle("fichera", 1, 1, 6)
    x = np.random.default_rng(82).normal(size=(2, op.mesh.n_dofs))
    assert rel_err(gpu_matvec(h, x), np.stack([op.matvec(xi) for xi in x])) < TOL64
    lib().ibem_destroy(h)


@pytest.mark.parametrize("name,p,kernel", [("torus", 2, 0), ("fichera", 1, 1)])
def test_fmm_rows(name, p, kernel):
    # m = 2: sampled rows of the FMM operator (each exact in the oracle) against
    # the library's full product
    from oracle import fmm, galerkin
    kern = galerkin.HelmholtzKernel(2.0) if kernel else galerkin.LaplaceKernel()
    disc = galerkin.Discretisation(_oracle_patches(name), p, 2, kern)
    op = fmm.FMMOperator(disc, 6, 1.6)
    N = op.mesh.n_dofs
    rng = np.random.default_rng(83 + kernel)
    x = rng.normal(size=N) + (1j * rng.normal(size=N) if kernel else 0.0)
    rows = np.sort(rng.choice(N, size=6, replace=False))
    y0 = op.rows(rows, x)[:, 0]
    h = _handle(name, p, 2, 6, kernel=kernel, kappa=2.0 if kernel else 0.0)
    y = _cmatvec(h, x[None, :])[0] if kernel else gpu_matvec(h, x[None, :])[0]
    assert np.max(np.abs(y[rows] - y0)) < TOL64 * np.max(np.abs(y))
    lib().ibem_destroy(h)


def _interior_error(name, p, m, q, x0, P):
    import torch
    ibem = lib()
    h = _handle(name, p, m, q)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - x0, axis=1))
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, torch.from_numpy(g(qp.cpu().numpy())).cuda(), 1, b)
    w = torch.zeros_like(b)
    s = ibem.ibem_solve(h, b, w, 1, rtol=1e-10, maxit=5000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    assert s.rel_residual <= 1e-10
    u = torch.empty(len(P), dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 1, torch.from_numpy(P).cuda(), u)
    ibem.ibem_destroy(h)
    return float(np.max(np.abs(u.cpu().numpy() - g(P)) / np.max(np.abs(g(P)))))


def test_interior_point_source():
    # u = the point source's field inside the solid (Eq. repform with the
    # Dirichlet data g = u* (., x0), x0 outside): the potential error falls
    # with refinement on both geometries
    rng = np.random.default_rng(85)
    # torus: source in the hole, points inside the tube
    phi, rho = rng.uniform(0, 2 * np.pi, 30), rng.uniform(0, 0.25, 30)
    th = rng.uniform(0, 2 * np.pi, 30)
    Pt = np.stack([(2 + rho * np.cos(th)) * np.cos(phi), (2 + rho * np.cos(th)) * np.sin(phi), rho * np.sin(th)], 1)
    et = [_interior_error("torus", 2, m, 8, np.array([0.0, 0.0, 0.3]), Pt) for m in (1, 2, 3)]
    # Fichera: source in the removed corner, points in the solid's far octant
    Pf = rng.uniform(-0.8, -0.2, size=(30, 3))
    ef = [_interior_error("fichera", 1, m, 6, np.array([0.5, 0.5, 0.5]), Pf) for m in (1, 2, 3)]
    assert et[2] < et[1] < et[0] and et[2] < 1e-3, et
    assert ef[2] < ef[1] < ef[0] and ef[2] < 5e-2, ef
