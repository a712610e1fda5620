"""Many right-hand sides on the FP32 operator: the far-field coupling is
contracted on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation).
Checked against the FP64 operator applied to each right-hand side; the BF16
rounding of K and of the moments (2^-9 relative) bounds the error."""
import numpy as np
import pytest

from gpu_common import lib, rel_err

pytestmark = pytest.mark.gpu


def _handle(p, m, q, kernel=0, kappa=0.0):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kernel, kappa=kappa))
    ibem.ibem_assemble(h)
    return h


def _apply(h, x, precision, cplx):
    import torch
    ibem = lib()
    xr = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1)) if cplx else np.ascontiguousarray(x)
    xd = torch.from_numpy(xr).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], precision)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1] if cplx else y


def _per_rhs_fp64(h, x, cplx):
    return np.stack([_apply(h, x[r:r + 1], 0, cplx)[0] for r in range(x.shape[0])])


@pytest.mark.parametrize("R", [16, 40])
def test_laplace_tensor_core_coupling(R):
    h = _handle(2, 3, 6)
    N = lib().ibem_get_info(h).ndof
    x = np.random.default_rng(R).normal(size=(R, N))
    y = _apply(h, x, 1, False)
    y64 = _per_rhs_fp64(h, x, False)
    err = rel_err(y, y64)
    assert 1e-7 < err < 5e-3, err
    lib().ibem_destroy(h)


def test_helmholtz_tensor_core_coupling_q8():
    h = _handle(2, 3, 8, kernel=1, kappa=4.0)
    N = lib().ibem_get_info(h).ndof
    rng = np.random.default_rng(3)
    x = rng.normal(size=(32, N)) + 1j * rng.normal(size=(32, N))
    y = _apply(h, x, 1, True)
    y64 = _per_rhs_fp64(h, x, True)
    err = rel_err(y, y64)
    assert 1e-7 < err < 5e-3, err
    lib().ibem_destroy(h)


@pytest.mark.parametrize("p,kernel,R", [(1, 0, 16), (2, 0, 40), (3, 0, 16), (2, 1, 24), (3, 1, 16)])
def test_multi_rhs_near_only_matches_fp64(p, kernel, R):
    # no far field (dense mode): the many-RHS path is the FP32 near product alone
    # (generic kernel for p = 1; one thread per right-hand side for p = 2, 3)
    h = _handle(p, 2 if p < 3 else 1, 0, kernel=kernel, kappa=3.0 if kernel else 0.0)
    N = lib().ibem_get_info(h).ndof
    rng = np.random.default_rng(5 + p)
    x = rng.normal(size=(R, N)) + (1j * rng.normal(size=(R, N)) if kernel else 0.0)
    assert rel_err(_apply(h, x, 1, bool(kernel)), _per_rhs_fp64(h, x, bool(kernel))) < 1e-5
    lib().ibem_destroy(h)


def test_tensor_core_kernel_bounded_wait():
    ibem = lib()
    h = _handle(2, 3, 6)
    N = ibem.ibem_get_info(h).ndof
    x = np.random.default_rng(9).normal(size=(16, N))
    y_ok = _apply(h, x, 1, False)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    ibem.ibem_set_wait_limit(h, 0)
    _apply(h, x, 1, False)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_TIMEOUT
    ibem.ibem_set_wait_limit(h, 1 << 26)
    y2 = _apply(h, x, 1, False)
    assert ibem.ibem_device_status(h) == ibem.IBEM_DEVICE_OK
    assert np.array_equal(y2, y_ok)
    ibem.ibem_destroy(h)
