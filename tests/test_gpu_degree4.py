"""Degree p = 4 (the highest degree of the paper's experiments, Sec. 5): the
FP64 library against the FP64 oracle at 1e-12 (dense Laplace and Helmholtz,
FMM Laplace at equal q), and the FP32 paths against the FP64 library.  At p = 4
an element carries 25 Bernstein functions, so every near block has 625 entries
and the near product runs 640 threads per element."""
import numpy as np
import pytest

from gpu_common import gpu_matvec, handle, lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _helm(p, m, q, kappa):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=1, kappa=kappa))
    ibem.ibem_assemble(h)
    return h


def _cmatvec(h, x, precision=0):
    import torch
    ibem = lib()
    xd = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], precision)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1]


def test_dense_laplace_p4():
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 4, 1, galerkin.LaplaceKernel())
    A = disc.dense_matrix()
    h = handle(4, 1, q=0)
    assert lib().ibem_get_info(h).ndof == A.shape[0] == 216
    x = np.random.default_rng(41).normal(size=(2, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    # FP32 near blocks: single-precision rounding of the entries and sums
    assert rel_err(gpu_matvec(h, x, 1), x @ A.T) < 1e-5
    lib().ibem_destroy(h)


def test_dense_helmholtz_p4():
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 4, 1, galerkin.HelmholtzKernel(2.0))
    A = disc.dense_matrix()
    h = _helm(4, 1, 0, 2.0)
    rng = np.random.default_rng(42)
    x = rng.normal(size=(2, A.shape[0])) + 1j * rng.normal(size=(2, A.shape[0]))
    assert rel_err(_cmatvec(h, x), x @ A.T) < TOL64
    lib().ibem_destroy(h)


def test_fmm_laplace_p4_m2():
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 4, 2, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, 6, 1.6)
    h = handle(4, 2, q=6)
    x = np.random.default_rng(43).normal(size=(1, op.mesh.n_dofs))
    assert rel_err(gpu_matvec(h, x), op.matvec(x[0])[None, :]) < TOL64
    lib().ibem_destroy(h)


@pytest.mark.parametrize("kernel", [0, 1], ids=["laplace", "helmholtz"])
def test_many_rhs_p4_matches_fp64(kernel):
    # 16 right-hand sides: generic many-right-hand-side near product (25 rows
    # per element) and the tensor-core coupling, against the FP64 operator
    # applied to each right-hand side; BF16 coupling bounds the error
    ibem = lib()
    kappa = 3.0 if kernel else 0.0
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(4, 3, q_cheb=6, eta=1.6, kernel=kernel, kappa=kappa))
    ibem.ibem_assemble(h)
    N = ibem.ibem_get_info(h).ndof
    rng = np.random.default_rng(44 + kernel)
    x = rng.normal(size=(16, N)) + (1j * rng.normal(size=(16, N)) if kernel else 0.0)
    if kernel:
        y = _cmatvec(h, x, 1)
        y64 = np.concatenate([_cmatvec(h, x[r:r + 1]) for r in range(16)])
    else:
        y = gpu_matvec(h, x, 1)
        y64 = np.concatenate([gpu_matvec(h, x[r:r + 1]) for r in range(16)])
    err = rel_err(y, y64)
    assert 1e-7 < err < 5e-3, err
    ibem.ibem_destroy(h)


def test_block_jacobi_cg_p4():
    # Laplace, point-source data: block-Jacobi CG reaches the FP64 true residual
    import torch
    ibem = lib()
    h = handle(4, 3, q=6)
    nq = ibem.ibem_get_info(h).n_quad_points
    qp = torch.empty((nq, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    x0 = torch.tensor([0.9, 0.9, 0.9], dtype=torch.float64, device="cuda")
    g = 1.0 / (4 * np.pi * torch.linalg.norm(qp - x0, dim=1))
    N = ibem.ibem_get_info(h).ndof
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, g.contiguous(), 1, b)
    w = torch.zeros_like(b)
    info = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=2000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    assert info.rel_residual <= 1e-8
    r = torch.empty_like(b)
    ibem.ibem_matvec(h, w, r, 1, 0)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.01e-8
    ibem.ibem_destroy(h)
