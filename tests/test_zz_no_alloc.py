"""ibem_potential_noalloc: potential evaluation for callers that cannot
allocate device memory when they need it (graph capture, real-time loops,
externally managed memory pools).  Its scratch is a fixed array inside the
library, so the test checks that two calls in a row - which reuse that array -
both reproduce the allocating ibem_potential, and that a discretisation too
large for the array is refused with a clear error."""
import numpy as np
import pytest

from gpu_common import handle, lib, rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_potential_matches_allocating_entry_twice():
    import torch
    ibem = lib()
    h = handle(3, 4, q=6, assemble=False)
    info = ibem.ibem_get_info(h)
    rng = np.random.default_rng(31)
    w = torch.from_numpy(rng.normal(size=(2, info.ndof))).cuda()
    d = rng.normal(size=(150, 3))
    P = d / np.linalg.norm(d, axis=1)[:, None] * (0.5 * rng.random(150) ** (1 / 3))[:, None]
    P[:40] *= 6.0                                  # some exterior points as well
    pts = torch.from_numpy(P).cuda()
    u_ref = torch.empty((2, 150), dtype=torch.float64, device="cuda")
    ibem.ibem_potential(h, w, 2, pts, u_ref)
    for _ in range(2):
        u = torch.full((2, 150), np.nan, dtype=torch.float64, device="cuda")
        ibem.ibem_potential_noalloc(h, w, 2, pts, u)
        torch.cuda.synchronize()
        assert rel_err(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-12
    ibem.ibem_destroy(h)
    # the property the entry point exists for: a fresh handle (no work vectors
    # yet) evaluates potentials without the device's free memory changing
    h2 = handle(3, 4, q=6, assemble=False)
    u = torch.empty((2, 150), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        ibem.ibem_potential_noalloc(h2, w, 2, pts, u)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert rel_err(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-12
    ibem.ibem_destroy(h2)


def test_noalloc_potential_refuses_oversized_discretisation():
    import torch
    ibem = lib()
    # 6144 elements x 12^2 Gauss points x 32 B = 28 MB > 16 MiB of scratch
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(1, 5, q_cheb=4, gauss_regular=12))
    info = ibem.ibem_get_info(h)
    w = torch.zeros(info.ndof, dtype=torch.float64, device="cuda")
    pts = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_potential_noalloc(h, w, 1, pts, u)
    assert ei.value.status == "IBEM_ERR_ARG" and "scratch" in str(ei.value)
    ibem.ibem_destroy(h)


def test_noalloc_potential_inside_a_cuda_graph():
    # the reason for the entry point: a call recorded into a CUDA graph.  One
    # warm-up call (kernels loaded, scratch address resolved), then a call
    # captured on the handle's stream in thread-local capture mode (an
    # allocation or a synchronisation inside the call would fail the capture),
    # replayed twice against ibem_potential
    import torch
    ibem = lib()
    stream = torch.cuda.Stream()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(2, 3, q_cheb=6, eta=1.6), stream)
    info = ibem.ibem_get_info(h)
    rng = np.random.default_rng(33)
    w = torch.from_numpy(rng.normal(size=(3, info.ndof))).cuda()
    d = rng.normal(size=(90, 3))
    pts = torch.from_numpy(d / np.linalg.norm(d, axis=1)[:, None] * 0.4).cuda()
    u_ref = torch.empty((3, 90), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ibem.ibem_potential(h, w, 3, pts, u_ref)
    u = torch.empty((3, 90), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ibem.ibem_potential_noalloc(h, w, 3, pts, u)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        ibem.ibem_potential_noalloc(h, w, 3, pts, u)
    for _ in range(2):
        u.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert rel_err(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-12
    del g
    ibem.ibem_destroy(h)
