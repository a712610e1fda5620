"""Regular Gauss orders above what a CTA holds as a kernel matrix in shared
memory (Sec. 4 item 4: orders up to 40): the streaming near-field kernels
against the FP64 oracle with the same rule (1e-12), and the module-wide Gauss
rule of a handle surviving the creation of another handle with another order."""
import numpy as np
import pytest

from gpu_common import gpu_matvec, lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _handle(p, m, Q, kernel=0, kappa=0.0, assemble=True):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=0, kernel=kernel, kappa=kappa,
                                                                 gauss_regular=Q))
    if assemble:
        ibem.ibem_assemble(h)
    return h


@pytest.mark.parametrize("p,m,Q", [(1, 1, 16), (2, 0, 40)])
def test_laplace_high_order_against_oracle(p, m, Q):
    # p = 1, m = 1 has 120 regular and 264 subdivided pairs (both streamed at
    # Q = 16); p = 2, m = 0 takes the largest order on the regular pairs of
    # opposite faces
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), p, m, galerkin.LaplaceKernel(), n_regular=Q)
    A = disc.dense_matrix()
    h = _handle(p, m, Q)
    x = np.random.default_rng(90 + Q).normal(size=(2, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    lib().ibem_destroy(h)


def test_helmholtz_high_order_against_oracle():
    import torch
    from oracle import galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 1, galerkin.HelmholtzKernel(2.0), n_regular=12)
    A = disc.dense_matrix()
    ibem = lib()
    h = _handle(1, 1, 12, kernel=1, kappa=2.0)
    rng = np.random.default_rng(93)
    x = rng.normal(size=(2, A.shape[0])) + 1j * rng.normal(size=(2, A.shape[0]))
    xd = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, 2, 0)
    y = yd.cpu().numpy()
    assert rel_err(y[..., 0] + 1j * y[..., 1], x @ A.T) < TOL64
    ibem.ibem_destroy(h)


def test_gauss_rule_per_handle():
    # the rule is module-wide device state: a handle assembled after another
    # handle with another order was created must still use its own
    ibem = lib()
    x = np.random.default_rng(94).normal(size=(1, 150))
    ref = _handle(1, 2, 8)
    y_ref = gpu_matvec(ref, x)
    ibem.ibem_destroy(ref)
    a = _handle(1, 2, 8, assemble=False)
    b = _handle(1, 1, 12, assemble=False)
    ibem.ibem_assemble(a)
    assert np.array_equal(gpu_matvec(a, x), y_ref)
    ibem.ibem_destroy(a)
    ibem.ibem_destroy(b)
