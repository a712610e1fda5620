"""GPU parity: libibem (FP64) against the FP64 CPU oracle, element by element.

Tolerance: 1e-12 relative (max-norm of the difference over max-norm of the
oracle result) for the FP64 operator at equal FMM parameters; both sides use
the same quadrature rules, interpolation nodes, admissibility arithmetic and
pair classification, so only rounding order differs."""
import numpy as np
import pytest

from gpu_common import gpu_matvec, handle, lib, oracle_fmm, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _x(n, r, seed):
    return np.random.default_rng(seed).normal(size=(r, n))


def test_dense_matvec_p2_m2(laplace_p2m2):
    # p = 2, m = 2, no compression: y = A x with A the oracle's dense matrix
    disc, A = laplace_p2m2
    h = handle(2, 2, q=0)
    x = _x(A.shape[0], 3, 1)
    y = gpu_matvec(h, x)
    assert rel_err(y, x @ A.T) < TOL64
    lib().ibem_destroy(h)


def test_dense_matvec_minimal_mesh():
    # m = 0: one element per patch (6 elements), p = 0 and p = 1
    from oracle import galerkin, geometry
    for p in (0, 1):
        disc = galerkin.Discretisation(geometry.unit_sphere(), p, 0, galerkin.LaplaceKernel())
        A = disc.dense_matrix()
        h = handle(p, 0, q=0)
        x = _x(A.shape[0], 2, 3)
        assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
        lib().ibem_destroy(h)


@pytest.mark.parametrize("coupling", [0, 1], ids=["double-float", "native-fp64"])
def test_fmm_matvec_p2_m2(coupling):
    op = oracle_fmm(2, 2, 6, 1.6)
    h = handle(2, 2, q=6, fp64_coupling=coupling)
    x = _x(op.mesh.n_dofs, 2, 5)
    y0 = np.stack([op.matvec(xi) for xi in x])
    assert rel_err(gpu_matvec(h, x), y0) < TOL64
    lib().ibem_destroy(h)


_NEAR_CACHE = {}


@pytest.mark.parametrize("q", [3, 4, 5, 8])
def test_fmm_matvec_double_float_other_q(q):
    """The double-float coupling for odd q (bounds-checked lanes, fixed ring
    depth) and for even q other than 6 (specialised lanes, ring depth chosen by
    the autotuner at assembly) against the oracle FMM at equal q."""
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 2, 2, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, q, 1.6, near_block_cache=_NEAR_CACHE)
    h = handle(2, 2, q=q, fp64_coupling=0)
    x = _x(op.mesh.n_dofs, 2, 30 + q)
    y0 = np.stack([op.matvec(xi) for xi in x])
    assert rel_err(gpu_matvec(h, x), y0) < TOL64
    lib().ibem_destroy(h)


def test_native_and_double_float_coupling_agree_p3_m5():
    hd = handle(3, 5, q=6, fp64_coupling=0)
    x = _x(7350, 1, 19)
    yd = gpu_matvec(hd, x)
    lib().ibem_destroy(hd)
    hn = handle(3, 5, q=6, fp64_coupling=1)
    yn = gpu_matvec(hn, x)
    lib().ibem_destroy(hn)
    assert rel_err(yd, yn) < 1e-13


def test_fmm_rows_p3_m3():
    op = oracle_fmm(3, 3, 6, 1.6)
    h = handle(3, 3, q=6)
    x = _x(op.mesh.n_dofs, 1, 7)
    y = gpu_matvec(h, x)[0]
    N = op.mesh.n_dofs
    rows = [0, 13, N // 2 + 5, N - 1]          # patch corners, interior, last patch
    y0 = op.rows(rows, x[0])[:, 0]
    assert np.max(np.abs(y[rows] - y0)) < TOL64 * np.max(np.abs(y))
    lib().ibem_destroy(h)


def test_fmm_rows_p3_m5_full_size():
    # the benchmark workload: p = 3, m = 5, q = 6, eta = 1.6 (7350 dofs)
    op = oracle_fmm(3, 5, 6, 1.6)
    h = handle(3, 5, q=6)
    info = lib().ibem_get_info(h)
    assert info.ndof == 7350 and info.ndof_super == 98304
    assert info.n_near == len(op.near) and info.n_far == len(op.far)
    x = _x(7350, 1, 11)
    y = gpu_matvec(h, x)[0]
    rows = [0, 1224, 3675, 7349]
    y0 = op.rows(rows, x[0])[:, 0]
    assert np.max(np.abs(y[rows] - y0)) < TOL64 * np.max(np.abs(y))
    lib().ibem_destroy(h)


def test_fp32_operator_error_bound():
    # FP32 near blocks + FP32 on-the-fly coupling: error against FP64 <= 1e-5
    h = handle(3, 5, q=6)
    x = _x(7350, 1, 13)
    y64 = gpu_matvec(h, x, 0)
    y32 = gpu_matvec(h, x, 1)
    assert rel_err(y32, y64) < 1e-5
    lib().ibem_destroy(h)


def test_multi_rhs_matches_columns_and_host_entry():
    h = handle(2, 3, q=6)
    ibem = lib()
    N = ibem.ibem_get_info(h).ndof
    x = _x(N, 4, 17)
    y = gpu_matvec(h, x)
    for r in range(4):
        assert np.array_equal(gpu_matvec(h, x[r:r + 1])[0], y[r])
    yh = np.zeros_like(x)
    ibem.ibem_matvec_host(h, np.ascontiguousarray(x), yh, 4)
    assert np.array_equal(yh, y)
    ibem.ibem_destroy(h)


def test_rhs_solve_potential_p2_m2(laplace_p2m2):
    import torch
    from conftest import seeded_ball_points
    from oracle import solve
    ibem = lib()
    disc, A = laplace_p2m2
    x0 = np.array([0.9, 0.9, 0.9])
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - x0, axis=1))
    h = handle(2, 2, q=0)
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gq = torch.from_numpy(g(qp.cpu().numpy())).cuda()
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    b0 = disc.rhs(g)[:, 0]
    assert rel_err(b.cpu().numpy(), b0) < TOL64
    w = torch.empty_like(b)
    si = ibem.ibem_solve(h, b, w, 1, rtol=1e-12, maxit=500)
    assert si.rel_residual <= 1e-12
    w0 = solve.dense_solve(A, b0)
    assert rel_err(w.cpu().numpy(), w0) < 1e-8
    P = seeded_ball_points(100, 0.5, 170809162)
    pts = torch.from_numpy(P).cuda()
    u = torch.empty(100, dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 1, pts, u)
    u_or = solve.potential(disc, w.cpu().numpy(), P)[:, 0]
    assert rel_err(u.cpu().numpy(), u_or) < TOL64
    assert np.max(np.abs(u.cpu().numpy() - g(P))) < 2e-6
    ibem.ibem_destroy(h)


def test_solve_p3_m5_fp64_and_mixed():
    import torch
    ibem = lib()
    h = handle(3, 5, q=6)
    x0 = np.array([0.9, 0.9, 0.9])
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - x0, axis=1))
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gq = torch.from_numpy(g(qp.cpu().numpy())).cuda()
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    w64 = torch.empty_like(b)
    w32 = torch.empty_like(b)
    s64 = ibem.ibem_solve(h, b, w64, 1, rtol=1e-8, maxit=2000, precision=0)
    s32 = ibem.ibem_solve(h, b, w32, 1, rtol=1e-8, maxit=2000, precision=1)
    assert s64.rel_residual <= 1e-8 and s32.rel_residual <= 1e-8
    # The first-kind operator is ill-conditioned, so densities at equal residual
    # differ by up to cond * 1e-8; potentials off the surface are insensitive.
    from conftest import seeded_ball_points
    P = seeded_ball_points(100, 0.5, 170809162)
    pts = torch.from_numpy(P).cuda()
    u64 = torch.empty(100, dtype=torch.float64, device="cuda")
    u32 = torch.empty(100, dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w64, 1, pts, u64)
    ibem.ibem_potential(h, w32, 1, pts, u32)
    exact = g(P)
    e64 = np.max(np.abs(u64.cpu().numpy() - exact))
    e32 = np.max(np.abs(u32.cpu().numpy() - exact))
    assert e64 < 1e-7 * np.max(np.abs(exact)) and e32 < 1e-7 * np.max(np.abs(exact)), (e64, e32)
    ibem.ibem_destroy(h)


def test_argument_and_state_errors():
    import torch
    ibem = lib()
    h = handle(1, 1, q=0, assemble=False)
    N = ibem.ibem_get_info(h).ndof
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_matvec(h, x, y, 1)
    assert ei.value.status == "IBEM_ERR_STATE"
    ibem.ibem_assemble(h)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_matvec(h, x, x, 1)
    assert ei.value.status == "IBEM_ERR_ARG"
    with pytest.raises(ibem.IbemError):
        ibem.ibem_matvec(h, x, y, 1, precision=7)
    ibem.ibem_matvec(h, x, y, 0)              # empty batch: no-op
    ibem.ibem_matvec(h, x, y, 1)
    torch.cuda.synchronize()
    assert torch.all(y == 0)                  # A 0 = 0
    ibem.ibem_destroy(h)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(2, 2, kernel=1, kappa=0.0))
    assert "kappa" in str(ei.value)


def test_bounded_wait_failure_path_and_recovery():
    # A wait limit of 0 makes every mbarrier wait of the streaming coupling
    # kernel fail at once: the kernel must record the timeout, drain its copies
    # and return; the context stays usable and the next application is exact.
    ibem = lib()
    h = handle(2, 3, q=6)
    N = ibem.ibem_get_info(h).ndof
    x = _x(N, 1, 23)
    y_ok = gpu_matvec(h, x)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    ibem.ibem_set_wait_limit(h, 0)
    gpu_matvec(h, x)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_TIMEOUT
    ibem.ibem_set_wait_limit(h, 1 << 26)
    y2 = gpu_matvec(h, x)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    assert np.array_equal(y2, y_ok)
    ibem.ibem_destroy(h)


def test_block_jacobi_cg_p3_m5():
    # block-Jacobi CG (FP64 and mixed) reaches 1e-8 in fewer iterations than point Jacobi
    import torch
    ibem = lib()
    h = handle(3, 5, q=6)
    info = ibem.ibem_get_info(h)
    x0 = np.array([0.9, 0.9, 0.9])
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    gq = torch.from_numpy(1.0 / (4 * np.pi * np.linalg.norm(qp.cpu().numpy() - x0, axis=1))).cuda()
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    w = torch.empty_like(b)
    sj = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_JACOBI)
    sb = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    sm = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=1)
    assert sb.rel_residual <= 1e-8 and sm.rel_residual <= 1e-8
    assert sb.iterations < sj.iterations
    ibem.ibem_destroy(h)


def test_potential_accuracy_floor_p2_m4():
    # interior Laplace problem, point source outside the unit sphere, p = 2,
    # m = 4 without compression, fixed 8-point rules: the potential error in
    # the ball r = 0.5 reaches the 1e-10 level the paper's high-order
    # experiments aim at (measured 1.0e-11; 3.4e-9 at m = 3)
    import torch
    from conftest import seeded_ball_points
    ibem = lib()
    h = handle(2, 4, q=0)
    x0 = np.array([0.9, 0.9, 0.9])
    g = lambda F: 1.0 / (4 * np.pi * np.linalg.norm(F - x0, axis=1))
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    b = torch.empty(info.ndof, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, torch.from_numpy(g(qp.cpu().numpy())).cuda(), 1, b)
    w = torch.zeros_like(b)
    s = ibem.ibem_solve(h, b, w, 1, rtol=1e-12, maxit=5000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI)
    assert s.rel_residual <= 1e-12
    P = seeded_ball_points(100, 0.5, 170809162)
    u = torch.empty(100, dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 1, torch.from_numpy(P).cuda(), u)
    assert np.max(np.abs(u.cpu().numpy() - g(P))) < 1e-10
    ibem.ibem_destroy(h)
