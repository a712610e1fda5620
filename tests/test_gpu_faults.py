"""Failure detection on the GPU without a GPU fault: non-finite input makes the
solvers return IBEM_ERR_BREAKDOWN, an allocation that cannot be satisfied
returns IBEM_ERR_OOM, and in both cases the handle and the CUDA context stay
usable (a normal application follows and matches the one before)."""
import numpy as np
import pytest

from gpu_common import lib

pytestmark = pytest.mark.gpu


def _handle(kernel):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(2, 2, q_cheb=6, kernel=kernel,
                                                                 kappa=3.0 if kernel else 0.0))
    ibem.ibem_assemble(h)
    return h


@pytest.mark.parametrize("kernel,R", [(0, 1), (0, 3), (1, 1), (1, 3)])
def test_nan_right_hand_side_is_a_breakdown(kernel, R):
    import torch
    ibem = lib()
    h = _handle(kernel)
    N = ibem.ibem_get_info(h).ndof
    shape = (R, N, 2) if kernel else (R, N)
    b = torch.from_numpy(np.random.default_rng(1).normal(size=shape)).cuda()
    w = torch.empty_like(b)
    ibem.ibem_solve(h, b, w, R, rtol=1e-8, maxit=500)
    w_ok = w.clone()
    b[R - 1].view(-1)[5] = float("nan")
    s, _ = ibem.ibem_solve(h, b, w, R, rtol=1e-8, maxit=500, check=False)
    assert s == 6, ibem.ibem_status_string(s)           # IBEM_ERR_BREAKDOWN
    b[R - 1].view(-1)[5] = 0.0
    b2 = torch.from_numpy(np.random.default_rng(1).normal(size=shape)).cuda()
    ibem.ibem_solve(h, b2, w, R, rtol=1e-8, maxit=500)
    assert torch.equal(w, w_ok)
    ibem.ibem_destroy(h)


def test_unsatisfiable_allocation_is_oom_and_the_handle_survives():
    import torch
    ibem = lib()
    h = _handle(1)
    N = ibem.ibem_get_info(h).ndof
    x = torch.from_numpy(np.random.default_rng(2).normal(size=(2, N, 2))).cuda()
    y0 = torch.empty_like(x)
    ibem.ibem_matvec(h, x, y0, 2)
    # the device copies of 2^30 complex right-hand sides (several TB) cannot be
    # allocated; the call fails before touching the (tiny) host arrays
    tiny = np.zeros(4)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_matvec_host(h, tiny, tiny, 1 << 30)
    assert ei.value.status == "IBEM_ERR_OOM", str(ei.value)
    y1 = torch.empty_like(x)
    ibem.ibem_matvec(h, x, y1, 2)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    ibem.ibem_destroy(h)
