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
