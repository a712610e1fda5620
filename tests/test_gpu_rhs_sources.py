"""ibem_rhs_sources: the FMM-compressed right-hand side of a field of point
sources (Sec. 3.2 right-hand side, Sec. 4.2 interpolation on the clusters
admissible for each source) against the oracle's FMMOperator.rhs_sources
element by element (FP64, 1e-12), and at a size the oracle does not reach by
its adjointness with ibem_potential_fmm (u* is symmetric)."""
import numpy as np
import pytest

from gpu_common import lib, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _sources(n, seed, radii):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * np.asarray(radii)[rng.integers(0, len(radii), size=n)][:, None]


def _gpu_rhs(h, Y, c, cplx):
    """Y (nsrc, 3), c (nsrc, R) -> b (N, R) through ibem_rhs_sources."""
    import torch
    ibem = lib()
    R = c.shape[1]
    ct = np.ascontiguousarray(c.T)                                   # [R][nsrc]
    cd = np.stack([ct.real, ct.imag], axis=-1) if cplx else ct
    src = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    chg = torch.from_numpy(np.ascontiguousarray(cd)).cuda()
    N = ibem.ibem_get_info(h).ndof
    b = torch.full((R, N, 2) if cplx else (R, N), np.nan, dtype=torch.float64, device="cuda")
    nf, nn = ibem.ibem_rhs_sources(h, src, chg, R, b)
    torch.cuda.synchronize()
    out = b.cpu().numpy()
    out = out[..., 0] + 1j * out[..., 1] if cplx else out
    return out.T, nf, nn


@pytest.mark.parametrize("p,m,q", [(2, 2, 5), (1, 3, 4)])
def test_laplace_against_oracle(p, m, q):
    from oracle import fmm, galerkin, geometry
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6))
    disc = galerkin.Discretisation(geometry.unit_sphere(), p, m, galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, q, 1.6)
    Y = _sources(40, 20 + m, [0.3, 0.8, 1.3, 3.0])
    c = np.random.default_rng(21).normal(size=(40, 3))
    b, nf, nn = _gpu_rhs(h, Y, c, False)
    ref = op.rhs_sources(Y, c)
    counts = np.array(op.rhs_counts)
    assert nf == counts[:, 0].sum() and nn == counts[:, 1].sum() and nf > 0 and nn > 0
    assert rel_err(b, ref) < TOL64, rel_err(b, ref)
    ibem.ibem_destroy(h)


def test_helmholtz_against_oracle():
    from oracle import fmm, galerkin, geometry
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(2, 2, q_cheb=6, eta=1.6, kernel=1, kappa=3.0))
    disc = galerkin.Discretisation(geometry.unit_sphere(), 2, 2, galerkin.HelmholtzKernel(3.0))
    op = fmm.FMMOperator(disc, 6, 1.6)
    Y = _sources(25, 22, [0.4, 1.5, 2.5])
    rng = np.random.default_rng(23)
    c = rng.normal(size=(25, 11)) + 1j * rng.normal(size=(25, 11))    # 11 = 8 + 3: two charge chunks
    b, nf, nn = _gpu_rhs(h, Y, c, True)
    ref = op.rhs_sources(Y, c)
    assert nf > 0 and nn > 0
    assert rel_err(b, ref) < TOL64, rel_err(b, ref)
    ibem.ibem_destroy(h)


@pytest.mark.parametrize("kappa", [None, 5.0])
def test_adjoint_of_potential_fmm_at_level_5(kappa):
    # w . b(Y, c) = sum_j c_j u_w(y_j) with u_w from ibem_potential_fmm: the two
    # walk the same clusters and Gauss points, so the identity holds to rounding
    import torch
    ibem = lib()
    cplx = kappa is not None
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        2, 5, q_cheb=6, eta=1.6, kernel=1 if cplx else 0, kappa=kappa or 0.0))
    N = ibem.ibem_get_info(h).ndof
    Y = _sources(3000, 24, [0.2, 0.7, 0.97, 1.04, 2.0, 6.0])
    rng = np.random.default_rng(25)
    c = rng.normal(size=(3000, 2)) + (1j * rng.normal(size=(3000, 2)) if cplx else 0)
    b, nf, nn = _gpu_rhs(h, Y, c, cplx)
    assert nf > 0 and nn > 0
    w = rng.normal(size=(2, N)) + (1j * rng.normal(size=(2, N)) if cplx else 0)
    wd = torch.from_numpy(np.ascontiguousarray(np.stack([w.real, w.imag], -1) if cplx else w)).cuda()
    pts = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    u = torch.empty((2, 3000, 2) if cplx else (2, 3000), dtype=torch.float64, device="cuda")
    ibem.ibem_potential_fmm(h, wd, 2, pts, u)
    un = u.cpu().numpy()
    un = un[..., 0] + 1j * un[..., 1] if cplx else un                # (2, nsrc)
    lhs = w @ b                                                        # (2 densities, 2 charge vectors)
    rhs = un @ c
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(rhs)), np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))
    ibem.ibem_destroy(h)


def test_repeatable_and_empty():
    import torch
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(1, 4, q_cheb=5, eta=1.6))
    Y = _sources(500, 26, [0.5, 1.1, 4.0])
    c = np.random.default_rng(27).normal(size=(500, 9))
    b1, _, _ = _gpu_rhs(h, Y, c, False)
    b2, _, _ = _gpu_rhs(h, Y, c, False)
    assert np.array_equal(b1, b2)
    N = ibem.ibem_get_info(h).ndof
    b = torch.full((2, N), np.nan, dtype=torch.float64, device="cuda")
    src = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    chg = torch.empty((2, 0), dtype=torch.float64, device="cuda")
    assert ibem.ibem_rhs_sources(h, src, chg, 2, b) == (0, 0)
    torch.cuda.synchronize()
    assert torch.all(b == 0)
    h0 = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(1, 2, q_cheb=0))
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_rhs_sources(h0, torch.zeros((1, 3), dtype=torch.float64, device="cuda"),
                              torch.ones((1, 1), dtype=torch.float64, device="cuda"), 1,
                              torch.empty((1, 54), dtype=torch.float64, device="cuda"))
    assert ei.value.status == "IBEM_ERR_ARG"
    ibem.ibem_destroy(h0)
    ibem.ibem_destroy(h)
