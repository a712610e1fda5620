"""Lock-step solves of many right-hand sides (ibem_solve with nrhs > 1):
Helmholtz GMRES(100) on sound-soft plane-wave data and Laplace CG, with the
FP64 operator and with the FP32 operator inside iterative refinement (the
tensor-core coupling from 16 columns on).  Checked against the oracle: the
discrete solution of the oracle's FMM operator (assembled densely from its
matvec and solved directly) and the residual with that operator."""
import numpy as np
import pytest

from gpu_common import lib, oracle_fmm_kernel

pytestmark = pytest.mark.gpu


def _handle(p, m, q, kappa, coupling=0):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        p, m, q_cheb=q, eta=1.6, kernel=1 if kappa else 0, kappa=kappa or 0.0, fp64_coupling=coupling))
    ibem.ibem_assemble(h)
    return h


def _dirs(R, seed):
    d = np.random.default_rng(seed).normal(size=(R, 3))
    return d / np.linalg.norm(d, axis=1)[:, None]


def _plane_wave_rhs(h, kappa, dirs):
    """b = T g* for g = -exp(i kappa d.x) (sound-soft), complex [R][N]."""
    import torch
    ibem = lib()
    info = ibem.ibem_get_info(h)
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    X = qp.cpu().numpy()
    g = -np.exp(1j * kappa * (dirs @ X.T))                      # [R][nq]
    gd = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], -1))).cuda()
    b = torch.empty((len(dirs), info.ndof, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gd, len(dirs), b)
    return b


def _dense_fmm(op):
    N = op.mesh.n_dofs
    return op.matvec(np.eye(N, dtype=complex if op.disc.kernel.is_complex else float))


@pytest.mark.parametrize("precision,R", [(0, 16), (1, 16), (0, 5)])
def test_block_gmres_plane_waves_vs_oracle(precision, R):
    import torch
    ibem = lib()
    kappa = 4.0
    op = oracle_fmm_kernel(2, 2, 8, 1.6, kappa)
    A = _dense_fmm(op)
    h = _handle(2, 2, 8, kappa, ibem.IBEM_COUPLING_GENERATE)
    b = _plane_wave_rhs(h, kappa, _dirs(R, 17))
    w = torch.empty_like(b)
    info = ibem.ibem_solve(h, b, w, R, rtol=1e-10, maxit=2000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI,
                           precision=precision)
    assert info.rel_residual <= 1e-10
    bn = b.cpu().numpy()
    bn = bn[..., 0] + 1j * bn[..., 1]
    wn = w.cpu().numpy()
    wn = wn[..., 0] + 1j * wn[..., 1]
    cond = np.linalg.cond(A)
    for r in range(R):
        # residual with the oracle's operator, and the distance to its direct solution
        res = np.linalg.norm(bn[r] - A @ wn[r]) / np.linalg.norm(bn[r])
        assert res < 2e-10, (r, res)
        ws = np.linalg.solve(A, bn[r])
        assert np.linalg.norm(wn[r] - ws) <= 2e-10 * cond * np.linalg.norm(ws), r
    # one operator application per lock-step step serves all columns
    assert info.steps * R >= info.iterations
    if precision == 1:
        assert info.outer >= 2          # refinement sweeps with FP64 residuals
    ibem.ibem_destroy(h)


def test_block_cg_laplace_vs_oracle_and_single_rhs():
    import torch
    ibem = lib()
    op = oracle_fmm_kernel(2, 2, 6, 1.6, None)
    A = _dense_fmm(op)
    h = _handle(2, 2, 6, None)
    N = ibem.ibem_get_info(h).ndof
    R = 20
    rng = np.random.default_rng(4)
    bn = rng.normal(size=(R, N))
    bn[3] = 0.0                                                  # a zero column: w = 0
    b = torch.from_numpy(bn).cuda()
    for precision in (0, 1):
        w = torch.full_like(b, np.nan)
        info = ibem.ibem_solve(h, b, w, R, rtol=1e-10, maxit=3000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI,
                               precision=precision)
        wn = w.cpu().numpy()
        assert info.rel_residual <= 1e-10
        assert np.all(wn[3] == 0.0)
        for r in range(R):
            if r == 3:
                continue
            assert np.linalg.norm(bn[r] - A @ wn[r]) <= 2e-10 * np.linalg.norm(bn[r]), (precision, r)
        # the same columns one by one
        w1 = torch.empty((1, N), dtype=torch.float64, device="cuda")
        ibem.ibem_solve(h, b[5:6].contiguous(), w1, 1, rtol=1e-10, maxit=3000,
                        precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=0)
        ws = w1.cpu().numpy()[0]
        assert np.linalg.norm(wn[5] - ws) <= 1e-7 * np.linalg.norm(ws)
    ibem.ibem_destroy(h)


def test_block_gmres_noconv_and_maxit():
    import torch
    ibem = lib()
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_GENERATE)
    b = _plane_wave_rhs(h, 4.0, _dirs(3, 5))
    w = torch.empty_like(b)
    s, info = ibem.ibem_solve(h, b, w, 3, rtol=1e-12, maxit=3, precond=ibem.IBEM_PRECOND_JACOBI, check=False)
    assert s == ibem.IBEM_ERR_NOCONV and info.steps <= 3
    ibem.ibem_destroy(h)
