"""Shared helpers of the GPU tests: build/load libibem, create handles, the
oracle reference operators (cached per session)."""
import functools

import numpy as np


def lib():
    from paper_1708_09162_gb300 import build
    build.build()
    from paper_1708_09162_gb300 import ibem
    return ibem


def handle(p, m, q, eta=1.6, assemble=True, fp64_coupling=0):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=eta,
                                                                 fp64_coupling=fp64_coupling))
    if assemble:
        ibem.ibem_assemble(h)
    return h


def gpu_matvec(h, x, precision=0):
    """x: numpy [R, N] -> y numpy [R, N] through ibem_matvec on device buffers."""
    import torch
    ibem = lib()
    xs = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ys = torch.empty_like(xs)
    ibem.ibem_matvec(h, xs, ys, x.shape[0], precision)
    torch.cuda.synchronize()
    return ys.cpu().numpy()


@functools.lru_cache(maxsize=None)
def oracle_fmm(p, m, q, eta):
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), p, m, galerkin.LaplaceKernel())
    return fmm.FMMOperator(disc, q, eta)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def oracle_fmm_kernel(p, m, q, eta, kappa=None):
    """Oracle FMM operator of the unit sphere, Laplace (kappa None) or Helmholtz."""
    return _oracle_fmm_cached(p, m, q, eta, kappa)


@functools.lru_cache(maxsize=None)
def _oracle_fmm_cached(p, m, q, eta, kappa):
    from oracle import fmm, galerkin, geometry
    kern = galerkin.LaplaceKernel() if kappa is None else galerkin.HelmholtzKernel(kappa)
    disc = galerkin.Discretisation(geometry.unit_sphere(), p, m, kern)
    return fmm.FMMOperator(disc, q, eta)


def oracle_abs_parts(op, x):
    """Magnitudes that bound rounding errors of the operator y = A x, per output:
    B = sum_s |M_s| sum_t |K_st| |x^_t|  (far field; x^_t the exact moments) and
    Nn = sum |A_e e'| |x_e'| over the near blocks.  x: (N, R); returns (B, Nn)."""
    me = op.mesh
    x2 = x.reshape(me.n_dofs, -1)
    B = np.zeros(x2.shape)
    Nn = np.zeros(x2.shape)
    dofs = [me.local_dofs(e) for e in range(me.n_elements)]
    ax = np.abs(x2)
    for eA, eB in op.near_elements:
        Nn[dofs[eA]] += np.abs(op.near_block(eA, eB)) @ ax[dofs[eB]]
    xh = op.forward_moments(x2)
    n1 = me.n1
    for s, targets in op.far_by_target.items():
        yh = sum(np.abs(op.coupling(s, t)) @ np.abs(xh[t]) for t in targets)
        patch, level, ix, iy = s
        mu_u = np.abs(op.moments_1d(level, ix))
        mu_v = np.abs(op.moments_1d(level, iy))
        B[patch * n1 * n1:(patch + 1) * n1 * n1] += np.einsum(
            "vb,uc,bcr->vur", mu_v, mu_u, yh.reshape(op.q, op.q, -1)).reshape(n1 * n1, -1)
    return B, Nn


def far_geometry_extent(op):
    """(min distance, max distance, max |F|) over the interpolation points of all
    far blocks: the cancellation factor of the FP32 differences X - Y and the
    largest phase kappa r."""
    dmin, dmax = np.inf, 0.0
    fmax = 0.0
    for s, t in op.far:
        _, FA, _, _ = op.interpolation_geometry(s)
        _, FB, _, _ = op.interpolation_geometry(t)
        d = np.sqrt(np.sum((FA[:, None, :] - FB[None, :, :]) ** 2, axis=-1))
        dmin = min(dmin, d.min())
        dmax = max(dmax, d.max())
        fmax = max(fmax, np.abs(FA).max(), np.abs(FB).max())
    return dmin, dmax, fmax
