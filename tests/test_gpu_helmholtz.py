"""GPU parity of the Helmholtz (complex) path against the FP64 oracle:
operator (dense and FMM, stored double-float and on-the-fly FP64 coupling),
FP32 operator error, right-hand side, GMRES solves and potentials."""
import numpy as np
import pytest

from gpu_common import lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _handle(p, m, q, kappa, coupling=0, assemble=True):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=1, kappa=kappa,
                                                                 fp64_coupling=coupling))
    if assemble:
        ibem.ibem_assemble(h)
    return h


def _cmatvec(h, x, precision=0):
    """x complex numpy [R, N] -> y complex through ibem_matvec (interleaved)."""
    import torch
    ibem = lib()
    xi = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))
    xd = torch.from_numpy(xi).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], precision)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1]


def _x(n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(r, n)) + 1j * rng.normal(size=(r, n))


@pytest.fixture(scope="module")
def helm_p1m1():
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 1, galerkin.HelmholtzKernel(2.0))
    return disc, disc.dense_matrix()


@pytest.fixture(scope="module")
def helm_fmm_p2m2():
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 2, 2, galerkin.HelmholtzKernel(4.0))
    return fmm.FMMOperator(disc, 6, 1.6)


def test_dense_helmholtz_matvec(helm_p1m1):
    disc, A = helm_p1m1
    h = _handle(1, 1, 0, 2.0)
    x = _x(A.shape[0], 2, 1)
    assert rel_err(_cmatvec(h, x), x @ A.T) < TOL64
    lib().ibem_destroy(h)


@pytest.mark.parametrize("coupling", [0, 1], ids=["stored-double-float", "on-the-fly-fp64"])
def test_fmm_helmholtz_matvec(helm_fmm_p2m2, coupling):
    op = helm_fmm_p2m2
    h = _handle(2, 2, 6, 4.0, coupling)
    info = lib().ibem_get_info(h)
    assert (info.bytes_far == 0) == (coupling == 1)
    x = _x(op.mesh.n_dofs, 2, 3)
    y0 = np.stack([op.matvec(xi) for xi in x])
    assert rel_err(_cmatvec(h, x), y0) < TOL64
    lib().ibem_destroy(h)


def test_fp32_helmholtz_operator_error():
    h = _handle(2, 4, 6, 4.0)
    x = _x(lib().ibem_get_info(h).ndof, 1, 5)
    y64 = _cmatvec(h, x, 0)
    y32 = _cmatvec(h, x, 1)
    assert rel_err(y32, y64) < 2e-5
    lib().ibem_destroy(h)


def test_rhs_gmres_potential_exterior_point_source(helm_p1m1):
    import torch
    from oracle import solve
    ibem = lib()
    k = 2.0
    v = np.array([0.1, 0.2, -0.1])

    def g(F):
        r = np.linalg.norm(F - v, axis=1)
        return np.exp(1j * k * r) / (4 * np.pi * r)

    disc, A = helm_p1m1
    h = _handle(1, 1, 0, k)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gv = g(qp.cpu().numpy())
    gq = torch.from_numpy(np.ascontiguousarray(np.stack([gv.real, gv.imag], axis=-1))).cuda()
    b = torch.empty((info.ndof, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    bc = b.cpu().numpy()
    b0 = disc.rhs(g)[:, 0]
    assert rel_err(bc[:, 0] + 1j * bc[:, 1], b0) < TOL64
    w = torch.empty_like(b)
    for prec in (0, 1):
        si = ibem.ibem_solve(h, b, w, 1, rtol=1e-10, maxit=500, precision=prec)
        assert si.rel_residual <= 1e-10
    wc = w.cpu().numpy()
    wc = wc[:, 0] + 1j * wc[:, 1]
    w0 = solve.dense_solve(A, b0)
    assert rel_err(wc, w0) < 1e-7
    rng = np.random.default_rng(7)
    d = rng.normal(size=(30, 3))
    P = 3.0 * d / np.linalg.norm(d, axis=1)[:, None]
    u = torch.empty((30, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 1, torch.from_numpy(P).cuda(), u)
    uc = u.cpu().numpy()
    uc = uc[:, 0] + 1j * uc[:, 1]
    u_or = solve.potential(disc, wc, P)[:, 0]
    assert rel_err(uc, u_or) < TOL64
    assert np.max(np.abs(uc - g(P))) < 2e-3 * np.max(np.abs(g(P)))
    ibem.ibem_destroy(h)


def test_gmres_fmm_fp64_and_mixed():
    import torch
    ibem = lib()
    h = _handle(2, 4, 6, 4.0)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    dvec = np.array([0.0, 0.6, 0.8])
    gv = -np.exp(1j * 4.0 * (qp.cpu().numpy() @ dvec))      # sound-soft plane wave
    gq = torch.from_numpy(np.ascontiguousarray(np.stack([gv.real, gv.imag], axis=-1))).cuda()
    b = torch.empty((info.ndof, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    w = torch.empty_like(b)
    s64 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precision=0)
    s32 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precision=1)
    assert s64.rel_residual <= 1e-8 and s32.rel_residual <= 1e-8
    ibem.ibem_destroy(h)


def test_gmres_block_jacobi():
    import torch
    ibem = lib()
    h = _handle(2, 4, 6, 4.0)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gv = -np.exp(1j * 4.0 * (qp.cpu().numpy() @ np.array([0.6, 0.0, 0.8])))
    gq = torch.from_numpy(np.ascontiguousarray(np.stack([gv.real, gv.imag], axis=-1))).cuda()
    b = torch.empty((info.ndof, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    w = torch.empty_like(b)
    sj = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_JACOBI)
    sb = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    sm = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=1)
    assert sb.rel_residual <= 1e-8 and sm.rel_residual <= 1e-8
    assert sb.iterations <= sj.iterations
    ibem.ibem_destroy(h)


def test_potential_many_densities(helm_p1m1):
    """Potentials of 20 densities at once (one chunk of 16 sharing each kernel
    evaluation, then a ragged chunk of 4) against the oracle, column by column."""
    import torch
    from oracle import solve
    ibem = lib()
    disc, _ = helm_p1m1
    h = _handle(1, 1, 0, 2.0)
    N = disc.mesh.n_dofs
    w = _x(N, 20, 41)
    rng = np.random.default_rng(42)
    d = rng.normal(size=(25, 3))
    pts = 2.5 * d / np.linalg.norm(d, axis=1)[:, None]
    wd = torch.from_numpy(np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1))).cuda()
    u = torch.empty((20, 25, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, wd, 20, torch.from_numpy(pts).cuda(), u)
    uc = u.cpu().numpy()
    uc = uc[..., 0] + 1j * uc[..., 1]
    u0 = solve.potential(disc, w.T, pts).T
    assert rel_err(uc, u0) < TOL64
    ibem.ibem_destroy(h)
