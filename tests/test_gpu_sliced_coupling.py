"""FP64-accurate Helmholtz coupling contracted on the tensor cores in BF16
digit slices (IBEM_COUPLING_SLICED): the operator against the FP64 oracle at
the 1e-12 parity tolerance per column, for right-hand side counts that fill one
chunk of 32, leave ragged chunks and span several chunks; against the
double-float generated coupling up to kappa = 14 (phases over several periods
of the reduction table); repeatable; bounded waits; and the fallbacks of the
mode (q != 8 takes the generated path, Laplace the stored double-float one)."""
import numpy as np
import pytest

from gpu_common import lib, oracle_fmm_kernel, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _handle(p, m, q, kappa, coupling, kernel=1):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kernel, kappa=kappa,
                                                                 fp64_coupling=coupling))
    ibem.ibem_assemble(h)
    return h


def _cmatvec(h, x):
    import torch
    ibem = lib()
    xi = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))
    xd = torch.from_numpy(xi).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], 0)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1]


def _x(n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(r, n)) + 1j * rng.normal(size=(r, n))


@pytest.mark.parametrize("R", [1, 5, 32, 33, 70])
def test_sliced_coupling_vs_oracle(R):
    ibem = lib()
    op = oracle_fmm_kernel(2, 2, 8, 1.6, 4.0)
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_SLICED)
    assert ibem.ibem_get_info(h).bytes_far == 0
    x = _x(op.mesh.n_dofs, R, 200 + R)
    y = _cmatvec(h, x)
    y_or = op.matvec(x.T).T
    for r in range(R):
        assert rel_err(y[r], y_or[r]) < TOL64, (r, rel_err(y[r], y_or[r]))
    ibem.ibem_destroy(h)


@pytest.mark.parametrize("kappa", [3.0, 14.0])
def test_sliced_equals_generated_coupling(kappa):
    ibem = lib()
    hs = _handle(2, 3, 8, kappa, ibem.IBEM_COUPLING_SLICED)
    hg = _handle(2, 3, 8, kappa, ibem.IBEM_COUPLING_GENERATE)
    x = _x(ibem.ibem_get_info(hs).ndof, 40, 11)
    ys, yg = _cmatvec(hs, x), _cmatvec(hg, x)
    errs = [rel_err(ys[r], yg[r]) for r in range(40)]
    assert max(errs) < TOL64, max(errs)
    # repeatable: a second application is bitwise identical
    assert np.array_equal(_cmatvec(hs, x), ys)
    ibem.ibem_destroy(hs)
    ibem.ibem_destroy(hg)


def test_sliced_coupling_bounded_wait():
    ibem = lib()
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_SLICED)
    x = _x(ibem.ibem_get_info(h).ndof, 8, 3)
    y_ok = _cmatvec(h, x)
    ibem.ibem_set_wait_limit(h, 0)
    _cmatvec(h, x)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_TIMEOUT
    ibem.ibem_set_wait_limit(h, 1 << 26)
    assert np.array_equal(_cmatvec(h, x), y_ok)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    ibem.ibem_destroy(h)


def test_sliced_mode_fallbacks():
    ibem = lib()
    # q = 6: the generated double-float path, bit for bit
    hs = _handle(2, 2, 6, 3.0, ibem.IBEM_COUPLING_SLICED)
    hg = _handle(2, 2, 6, 3.0, ibem.IBEM_COUPLING_GENERATE)
    x = _x(ibem.ibem_get_info(hs).ndof, 6, 5)
    assert np.array_equal(_cmatvec(hs, x), _cmatvec(hg, x))
    ibem.ibem_destroy(hs)
    ibem.ibem_destroy(hg)
    # Laplace: stored double-float matrices as with IBEM_COUPLING_DF
    hl = _handle(2, 3, 8, 0.0, ibem.IBEM_COUPLING_SLICED, kernel=0)
    hd = _handle(2, 3, 8, 0.0, ibem.IBEM_COUPLING_DF, kernel=0)
    assert ibem.ibem_get_info(hl).bytes_far == ibem.ibem_get_info(hd).bytes_far > 0
    xr = np.random.default_rng(6).normal(size=(3, ibem.ibem_get_info(hl).ndof))
    from gpu_common import gpu_matvec
    assert np.array_equal(gpu_matvec(hl, xr), gpu_matvec(hd, xr))
    ibem.ibem_destroy(hl)
    ibem.ibem_destroy(hd)
