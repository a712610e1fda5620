"""Batched application of uneven instances (one launch per stage over all
instances, persistent coupling kernel, CUDA graph): every instance must match
its own FP64 operator to FP32 accuracy, and replays must be identical."""
import numpy as np
import pytest

from gpu_common import lib, rel_err

pytestmark = pytest.mark.gpu

SPECS = [  # (kernel, kappa, p, m, q, R, radius, center)
    (0, 0.0, 1, 3, 6, 3, 1.0, (0.0, 0.0, 0.0)),
    (1, 2.0, 2, 2, 6, 2, 1.0, (0.0, 0.0, 0.0)),
    (0, 0.0, 3, 2, 6, 1, 1.0, (0.0, 0.0, 0.0)),
    (1, 5.0, 1, 3, 8, 4, 0.7, (0.2, 0.0, -0.1)),
    (0, 0.0, 2, 4, 6, 5, 1.0, (0.0, 0.0, 0.0)),
    (0, 0.0, 2, 3, 8, 2, 1.8, (1.0, -2.0, 0.5)),
]


def test_batched_uneven_instances():
    import torch
    ibem = lib()
    handles = []
    for kern, kappa, p, m, q, R, rad, cen in SPECS:
        h = ibem.ibem_create(ibem.sphere_patches(rad, cen), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kern,
                                                                             kappa=kappa))
        ibem.ibem_assemble(h)
        handles.append(h)
    nrhs = [s[5] for s in SPECS]
    b = ibem.ibem_batch_create(handles, nrhs)
    off = ibem.ibem_batch_offsets(b, len(handles))
    rng = np.random.default_rng(42)
    x = torch.from_numpy(rng.normal(size=off[-1])).cuda()
    y1 = torch.zeros_like(x)
    y2 = torch.zeros_like(x)
    ibem.ibem_batch_matvec(b, x, y1)
    ibem.ibem_batch_matvec(b, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    info = ibem.ibem_batch_info(b)
    assert info["launches_per_apply"] <= 2 * max(s[3] for s in SPECS) + 8
    assert info["coupling_threads"] in (128, 256, 512)
    assert info["coupling_rhs_tile"] in (4, 8, 16)
    for i, (h, spec) in enumerate(zip(handles, SPECS)):
        R = spec[5]
        xi = x[off[i]:off[i + 1]].contiguous()
        y64 = torch.empty_like(xi)
        ibem.ibem_matvec(h, xi, y64, R, 0)
        torch.cuda.synchronize()
        yb = y1[off[i]:off[i + 1]].cpu().numpy()
        assert rel_err(yb, y64.cpu().numpy()) < 2e-5, (i, rel_err(yb, y64.cpu().numpy()))
    ibem.ibem_batch_destroy(b)
    for h in handles:
        ibem.ibem_destroy(h)


def test_coupling_none_refuses_fp64():
    import torch
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(1, 3, q_cheb=6, fp64_coupling=2))
    ibem.ibem_assemble(h)
    N = ibem.ibem_get_info(h).ndof
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_matvec(h, x, y, 1, 0)
    assert ei.value.status == "IBEM_ERR_STATE"
    ibem.ibem_matvec(h, x, y, 1, 1)        # FP32 operator still available
    ibem.ibem_destroy(h)


def test_batch_solve_against_single_instance_solves():
    # every instance of the uneven batch solved in lock step through the batched
    # operator (FP64 residual refinement), against each instance's own solve
    import torch
    ibem = lib()
    handles = []
    for kern, kappa, p, m, q, R, rad, cen in SPECS:
        h = ibem.ibem_create(ibem.sphere_patches(rad, cen), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=kern,
                                                                             kappa=kappa))
        ibem.ibem_assemble(h)
        handles.append(h)
    nrhs = [s[5] for s in SPECS]
    b = ibem.ibem_batch_create(handles, nrhs)
    off = ibem.ibem_batch_offsets(b, len(handles))
    rng = np.random.default_rng(7)
    rhs = torch.from_numpy(rng.normal(size=off[-1])).cuda()
    rhs[off[2]:off[3]] = 0.0                                   # an instance with a zero right-hand side
    x = torch.full_like(rhs, np.nan)
    for precond in (ibem.IBEM_PRECOND_JACOBI, ibem.IBEM_PRECOND_BLOCK_JACOBI):
        info = ibem.ibem_batch_solve(b, rhs, x, rtol=1e-9, maxit=3000, precond=precond)
        assert info.rel_residual <= 1e-9 and info.outer >= 2, (info.rel_residual, info.outer)
        assert torch.all(x[off[2]:off[3]] == 0.0)
        for i, (h, spec) in enumerate(zip(handles, SPECS)):
            if i == 2:
                continue
            R = spec[5]
            bi = rhs[off[i]:off[i + 1]].contiguous()
            xi = torch.empty_like(bi)
            ibem.ibem_solve(h, bi, xi, R, rtol=1e-11, maxit=3000, precond=precond)
            xb = x[off[i]:off[i + 1]]
            assert rel_err(xb.cpu().numpy(), xi.cpu().numpy()) < 1e-6, (i, rel_err(xb.cpu().numpy(), xi.cpu().numpy()))
            # residual of the batch solution with the instance's FP64 operator
            y = torch.empty_like(bi)
            ibem.ibem_matvec(h, xb.contiguous(), y, R, 0)
            res = (y - bi).reshape(R, -1).norm(dim=1) / bi.reshape(R, -1).norm(dim=1)
            assert float(res.max()) <= 1.0001e-9, (i, float(res.max()))
    ibem.ibem_batch_destroy(b)
    for h in handles:
        ibem.ibem_destroy(h)
