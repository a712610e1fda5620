"""FP64-accurate Helmholtz coupling generated on the fly in double-float
arithmetic for many right-hand sides (IBEM_COUPLING_GENERATE): the operator
against the FP64 oracle at the 1e-12 parity tolerance, for right-hand side
counts that exercise each chunk width (16, 32, 64) and ragged chunks, and
against the stored double-float coupling of the same discretisation."""
import numpy as np
import pytest

from gpu_common import lib, oracle_fmm_kernel, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _handle(p, m, q, kappa, coupling):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=1, kappa=kappa,
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


@pytest.mark.parametrize("R", [1, 5, 16, 17, 40, 70])
def test_generated_coupling_vs_oracle(R):
    ibem = lib()
    op = oracle_fmm_kernel(2, 2, 8, 1.6, 4.0)
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_GENERATE)
    assert ibem.ibem_get_info(h).bytes_far == 0
    x = _x(op.mesh.n_dofs, R, 100 + R)
    y = _cmatvec(h, x)
    y_or = op.matvec(x.T).T
    for r in range(R):
        assert rel_err(y[r], y_or[r]) < TOL64, (r, rel_err(y[r], y_or[r]))
    ibem.ibem_destroy(h)


@pytest.mark.parametrize("q,kappa", [(6, 3.0), (8, 14.0)])
def test_generated_equals_stored_coupling(q, kappa):
    # same operator as the stored double-float matrices; kappa = 14 takes the
    # phase through several periods of the reduction table
    ibem = lib()
    hg = _handle(2, 3, q, kappa, ibem.IBEM_COUPLING_GENERATE)
    hs = _handle(2, 3, q, kappa, ibem.IBEM_COUPLING_DF)
    assert ibem.ibem_get_info(hs).bytes_far > 0
    x = _x(ibem.ibem_get_info(hg).ndof, 20, 7)
    yg, ys = _cmatvec(hg, x), _cmatvec(hs, x)
    for r in range(20):
        assert rel_err(yg[r], ys[r]) < TOL64, (r, rel_err(yg[r], ys[r]))
    # deterministic: a second application is bitwise identical
    assert np.array_equal(_cmatvec(hg, x), yg)
    ibem.ibem_destroy(hg)
    ibem.ibem_destroy(hs)


def test_generated_coupling_bounded_wait():
    ibem = lib()
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_GENERATE)
    x = _x(ibem.ibem_get_info(h).ndof, 16, 3)
    y_ok = _cmatvec(h, x)
    ibem.ibem_set_wait_limit(h, 0)
    _cmatvec(h, x)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_TIMEOUT
    ibem.ibem_set_wait_limit(h, 1 << 26)
    assert np.array_equal(_cmatvec(h, x), y_ok)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    ibem.ibem_destroy(h)


def test_matvec_host_helmholtz_many_rhs():
    # the host-buffer entry point with complex values: same result as the device one
    import torch
    ibem = lib()
    h = _handle(2, 2, 8, 4.0, ibem.IBEM_COUPLING_GENERATE)
    x = _x(ibem.ibem_get_info(h).ndof, 20, 9)
    xh = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], -1))).pin_memory()
    yh = torch.zeros_like(xh).pin_memory()
    ibem.ibem_matvec_host(h, xh, yh, 20, 0)
    y = yh.numpy()
    assert np.array_equal(y[..., 0] + 1j * y[..., 1], _cmatvec(h, x))
    ibem.ibem_destroy(h)
