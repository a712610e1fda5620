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


def _graded(p, m, base, grading, q=0, kernel=0, kappa=0.0, patches=None):
    ibem = lib()
    prm = ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kernel, kappa=kappa, gauss_regular=base,
                           gauss_singular=6, gauss_grading=grading)
    pats = patches if patches is not None else ibem.sphere_patches()
    h = ibem.ibem_create(pats, prm)
    ibem.ibem_assemble(h)
    return h, prm, pats


@pytest.mark.parametrize("p,m,base,grading", [(1, 2, 4, 3), (2, 1, 3, 4)])
def test_graded_orders_laplace_dense_against_oracle(p, m, base, grading):
    # every element pair near (q = 0): orders from the base up to 40 across
    # the distance ratios of the sphere, each group by the streaming kernel
    from oracle import galerkin, geometry
    ibem = lib()
    h, prm, pats = _graded(p, m, base, grading)
    info = ibem.ibem_get_info(h)
    orders = ibem.ibem_near_orders(pats, prm)
    near, _ = ibem.ibem_block_tree(pats, prm)
    nt = orders[near[:, 6] >= 3]
    assert info.max_gauss_order == int(nt.max()) and info.n_near_graded == int(np.sum(nt != base))
    assert info.n_near_graded > 0 and len(set(nt.tolist())) >= 3
    disc = galerkin.Discretisation(geometry.unit_sphere(), p, m, galerkin.LaplaceKernel(), n_regular=base,
                                   n_singular=6, grading=grading)
    A = disc.dense_matrix()
    x = np.random.default_rng(95 + grading).normal(size=(2, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    ibem.ibem_destroy(h)


def test_graded_orders_helmholtz_fmm_against_oracle():
    # near field of the compressed operator with graded orders (Helmholtz,
    # p = 1, m = 2, q = 4) against the oracle's FMM operator with the same reading
    import torch
    from oracle import fmm, galerkin, geometry
    ibem = lib()
    h, prm, pats = _graded(1, 2, 3, 3, q=4, kernel=1, kappa=3.0)
    assert ibem.ibem_get_info(h).n_near_graded > 0
    disc = galerkin.Discretisation(geometry.unit_sphere(), 1, 2, galerkin.HelmholtzKernel(3.0), n_regular=3,
                                   n_singular=6, grading=3)
    op = fmm.FMMOperator(disc, 4, 1.6)
    rng = np.random.default_rng(96)
    N = disc.mesh.n_dofs
    x = rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))
    xd = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, 2, 0)
    y = yd.cpu().numpy()
    ref = op.matvec(x.T).T
    assert rel_err(y[..., 0] + 1j * y[..., 1], ref) < TOL64
    ibem.ibem_destroy(h)


def test_graded_orders_fichera_against_oracle():
    # flat faces: the distance ratios of the lattice (0.414, 0.581, 1, ...) sit
    # away from the thresholds 3/4, 3/8, ..., so both sides take the same orders
    import shapes
    from oracle import galerkin, geometry
    ibem = lib()
    specs = shapes.fichera()
    h, prm, pats = _graded(1, 1, 2, 4, patches=ibem.nurbs_patches(specs))
    assert ibem.ibem_get_info(h).n_near_graded > 0
    disc = galerkin.Discretisation([geometry.NurbsPatch(*s) for s in specs], 1, 1, galerkin.LaplaceKernel(),
                                   n_regular=2, n_singular=6, grading=4)
    A = disc.dense_matrix()
    x = np.random.default_rng(97).normal(size=(1, A.shape[0]))
    assert rel_err(gpu_matvec(h, x), x @ A.T) < TOL64
    ibem.ibem_destroy(h)


def test_graded_pair_at_forty_points_against_inclusion_exclusion():
    # flat unit square, p = 0, m = 2: elements (0, 0) and (2, 0) have one
    # element between them (rho = 0.414, subdivided) and take 2 + 38 = 40
    # points per direction on every sub-square pair; their entry must equal
    # [I(3h, h) - 2 I(2h, h) + I(h, h)] / (8 pi) (inclusion-exclusion over
    # rectangle self-interactions, as in tests/test_oracle_grading.py)
    import warnings
    from test_oracle_grading import _rect
    ibem = lib()
    ctrl = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0], [1.0, 1.0, 0.0]]])
    k1 = [0.0, 0.0, 1.0, 1.0]
    pats = ibem.nurbs_patches([(1, 1, k1, k1, ctrl, np.ones((2, 2)))])
    h, prm, _ = _graded(0, 2, 2, 38, patches=pats)
    assert ibem.ibem_get_info(h).max_gauss_order == 40
    hh = 0.25
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        exact = (_rect(3 * hh, hh) - 2 * _rect(2 * hh, hh) + _rect(hh, hh)) / (8 * np.pi)
    # dofs of p = 0 on one patch: j_v * 4 + j_u; column (2, 0) -> dof 2, row (0, 0) -> dof 0
    x = np.zeros((1, 16))
    x[0, 2] = 1.0
    y = gpu_matvec(h, x)
    assert abs(y[0, 0] - exact) / exact < 1e-12, (y[0, 0], exact)
    ibem.ibem_destroy(h)
