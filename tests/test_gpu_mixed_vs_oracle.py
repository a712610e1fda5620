"""The reduced-precision operators against the FP64 oracle (not against the
library's own FP64 path): the FP32 operator (one right-hand side), the
tensor-core coupling (16 and more right-hand sides; K and the moments rounded
to BF16, FP32 accumulation in TMEM) and the batched application of several
instances, on the unit sphere at p = 2, m = 2 (Laplace q = 6, Helmholtz
kappa = 4 with q = 8), element by element.

Tolerance per output component i (derived from the rounding, stated here):

    |y_i - y_i^oracle| <= eps_op B_i + 2 u32 Nn_i + lam sqrt(n) u32 (B_i + Nn_i)
                          + 1e-11 max|y^oracle|

* B_i  = (sum_s |M_s| sum_t |K_st| |x^_t|)_i, the far field taken in absolute
  values with the exact moments x^_t (the oracle's non-nested operator), and
  Nn_i = (sum |A_ee'| |x_e'|)_i over the near blocks; rounding a factor of a
  product by a relative delta perturbs the product by at most delta times its
  magnitude, and the downward pass is linear, so |Delta y_i| <= eps B_i.
* eps_op: rounding of the factors of each far-field product.  BF16 (unit
  roundoff u_bf = 2^-9) on both K and x^: 2 u_bf + u_bf^2 for a real product;
  for a complex product in the real form, |K_r||x_r| + |K_i||x_i| <= |K||x^|
  gives the same factor per real component.  Plus the FP32 generation error of
  K, eps_K = (2 sqrt(3) F_max / d_min + 10) u32 + 2^-22 (coordinates rounded to
  FP32 and their difference cancelling down to the smallest far distance d_min,
  r^2, rsqrt with at most 2 ulp), and for Helmholtz the phase error
  kappa d_max eps_K + 2 u32 kappa d_max + 2^-21.41 (hardware sine / cosine on
  [-pi, pi]) + (kappa d_max / 2 pi + 1) |2 pi - fl32(2 pi)|.  The FP32
  operator: eps_op = eps_K + 2 u32.
* 2 u32 Nn_i: near blocks and their inputs rounded to FP32.
* lam sqrt(n) u32 (B + Nn): FP32 accumulation of sums of at most n = 2e4 terms
  per output (near rows, far rows, transfers) with the probabilistic bound of
  Higham and Mary (SIAM J. Sci. Comput. 41, 2019), lam = 6.
* 1e-11 max|y|: the nested GPU operator against the oracle's non-nested one
  (equal in exact arithmetic; 1e-12 parity in FP64).

The tensor-core tests also require an error above 1e-6 of max|y| (far above
FP32 rounding), which shows that the BF16 path ran."""
import math

import numpy as np
import pytest

from gpu_common import far_geometry_extent, lib, oracle_abs_parts, oracle_fmm_kernel

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
UBF = 2.0 ** -9
LAM_SQRT_N = 6.0 * math.sqrt(2e4)
TWO_PI_ERR = abs(2 * math.pi - float(np.float32(2 * math.pi)))


def _eps_k32(op, kappa):
    dmin, dmax, fmax = far_geometry_extent(op)
    eps = (2 * math.sqrt(3) * fmax / dmin + 10) * U32 + 2.0 ** -22
    if kappa:
        th = kappa * dmax
        eps += th * eps + 2 * U32 * th + 2.0 ** -21.41 + (th / (2 * math.pi) + 1) * TWO_PI_ERR
    return eps


def _handle(p, m, q, kappa):
    ibem = lib()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        p, m, q_cheb=q, eta=1.6, kernel=1 if kappa else 0, kappa=kappa or 0.0))
    ibem.ibem_assemble(h)
    return h


def _apply(h, x, precision):
    """x numpy [R, N] (complex for Helmholtz) through ibem_matvec."""
    import torch
    ibem = lib()
    cplx = np.iscomplexobj(x)
    xr = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1)) if cplx else np.ascontiguousarray(x)
    xd = torch.from_numpy(xr).cuda()
    yd = torch.empty_like(xd)
    ibem.ibem_matvec(h, xd, yd, x.shape[0], precision)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    return y[..., 0] + 1j * y[..., 1] if cplx else y


def _check(y_gpu, op, x, eps_op):
    """Componentwise bound of the module docstring; returns (worst ratio, rel err)."""
    xt = x.T                                   # (N, R)
    y_or = op.matvec(xt).T
    B, Nn = oracle_abs_parts(op, xt)
    B, Nn = B.T, Nn.T
    tol = eps_op * B + 2 * U32 * Nn + LAM_SQRT_N * U32 * (B + Nn) + 1e-11 * np.max(np.abs(y_or))
    d = y_gpu - y_or
    if np.iscomplexobj(d):
        ratio = max(np.max(np.abs(d.real) / tol), np.max(np.abs(d.imag) / tol))
    else:
        ratio = np.max(np.abs(d) / tol)
    return ratio, float(np.max(np.abs(d)) / np.max(np.abs(y_or)))


def _x(N, R, seed, cplx, positive=False):
    rng = np.random.default_rng(seed)
    if positive:
        return rng.random(size=(R, N))
    x = rng.normal(size=(R, N))
    return x + 1j * rng.normal(size=(R, N)) if cplx else x


CASES = [(6, None), (8, 4.0)]   # (q, kappa): Laplace q = 6, Helmholtz kappa = 4 with q = 8


@pytest.mark.parametrize("q,kappa", CASES)
def test_fp32_operator_vs_oracle(q, kappa):
    op = oracle_fmm_kernel(2, 2, q, 1.6, kappa)
    h = _handle(2, 2, q, kappa)
    N = lib().ibem_get_info(h).ndof
    eps = _eps_k32(op, kappa) + 2 * U32
    for seed, pos in ((1, False), (2, True)):
        if pos and kappa:
            continue
        x = _x(N, 2, seed, bool(kappa), pos)
        ratio, err = _check(_apply(h, x, 1), op, x, eps)
        assert ratio <= 1.0, (ratio, err)
    lib().ibem_destroy(h)


@pytest.mark.parametrize("q,kappa,R", [(6, None, 16), (6, None, 40), (8, 4.0, 16), (8, 4.0, 32)])
def test_tensor_core_operator_vs_oracle(q, kappa, R):
    op = oracle_fmm_kernel(2, 2, q, 1.6, kappa)
    h = _handle(2, 2, q, kappa)
    N = lib().ibem_get_info(h).ndof
    eps = 2 * UBF + UBF * UBF + _eps_k32(op, kappa)
    x = _x(N, R, 10 + R, bool(kappa))
    ratio, err = _check(_apply(h, x, 1), op, x, eps)
    assert ratio <= 1.0 and err > 1e-6, (ratio, err)
    if not kappa:
        # positive inputs: no cancellation, so the bound is nearly attained in size
        xp = _x(N, R, 20 + R, False, True)
        ratio, err = _check(_apply(h, xp, 1), op, xp, eps)
        assert ratio <= 1.0 and err > 1e-6, (ratio, err)
    lib().ibem_destroy(h)


def test_batched_instances_vs_oracle():
    # a Laplace and a Helmholtz instance in one batched application (FP32 operator)
    import torch
    ibem = lib()
    specs = [(6, None, 3), (8, 4.0, 2)]
    handles = [_handle(2, 2, q, kappa) for q, kappa, _ in specs]
    b = ibem.ibem_batch_create(handles, [R for _, _, R in specs])
    off = ibem.ibem_batch_offsets(b, len(handles))
    N = ibem.ibem_get_info(handles[0]).ndof
    xs = [_x(N, R, 40 + i, bool(kappa)) for i, (_, kappa, R) in enumerate(specs)]
    flat = np.concatenate([np.stack([x.real, x.imag], -1).ravel() if np.iscomplexobj(x) else x.ravel() for x in xs])
    assert flat.size == off[-1]
    xd = torch.from_numpy(flat).cuda()
    yd = torch.zeros_like(xd)
    ibem.ibem_batch_matvec(b, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for i, (q, kappa, R) in enumerate(specs):
        op = oracle_fmm_kernel(2, 2, q, 1.6, kappa)
        yi = y[off[i]:off[i + 1]]
        yi = (yi.reshape(R, N, 2)[..., 0] + 1j * yi.reshape(R, N, 2)[..., 1]) if kappa else yi.reshape(R, N)
        ratio, err = _check(yi, op, xs[i], _eps_k32(op, kappa) + 2 * U32)
        assert ratio <= 1.0, (i, ratio, err)
    ibem.ibem_batch_destroy(b)
    for h in handles:
        ibem.ibem_destroy(h)


@pytest.mark.parametrize("R", [16, 40, 70])
def test_stored_bf16_coupling_vs_oracle(R):
    # IBEM_FP32_COUPLING_STORE: the BF16 blocks generated once at assembly and
    # streamed (stacked real / imaginary rows, one MMA group per block), same
    # bound as the generated tensor-core coupling; chunks of 64 right-hand sides
    # (70 = 64 + 6); close to the generating kernel, which rounds the same values
    import torch
    ibem = lib()
    op = oracle_fmm_kernel(2, 2, 8, 1.6, 4.0)
    hs = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        2, 2, q_cheb=8, eta=1.6, kernel=1, kappa=4.0, fp32_coupling=ibem.IBEM_FP32_COUPLING_STORE))
    ibem.ibem_assemble(hs)
    hg = _handle(2, 2, 8, 4.0)
    N = ibem.ibem_get_info(hs).ndof
    eps = 2 * UBF + UBF * UBF + _eps_k32(op, 4.0)
    x = _x(N, R, 50 + R, True)
    ys = _apply(hs, x, 1)
    ratio, err = _check(ys, op, x, eps)
    assert ratio <= 1.0 and err > 1e-6, (ratio, err)
    yg = _apply(hg, x, 1)
    assert float(np.max(np.abs(ys - yg)) / np.max(np.abs(yg))) < 1e-5
    ibem.ibem_destroy(hs)
    ibem.ibem_destroy(hg)


def test_switching_the_fp32_coupling_after_assembly():
    # ibem_set_fp32_coupling: STORE on a generating handle gives the stored
    # handle's result exactly, GENERATE releases the blocks and gives the
    # generating handle's result exactly; Laplace and unassembled handles refuse
    import torch
    ibem = lib()
    hs = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        2, 2, q_cheb=8, eta=1.6, kernel=1, kappa=4.0, fp32_coupling=ibem.IBEM_FP32_COUPLING_STORE))
    ibem.ibem_assemble(hs)
    hg = _handle(2, 2, 8, 4.0)
    N = ibem.ibem_get_info(hs).ndof
    x = _x(N, 24, 77, True)
    y_store, y_gen = _apply(hs, x, 1), _apply(hg, x, 1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ibem.ibem_set_fp32_coupling(hg, ibem.IBEM_FP32_COUPLING_STORE)
    assert torch.cuda.mem_get_info()[0] < free0
    assert np.array_equal(_apply(hg, x, 1), y_store)
    ibem.ibem_set_fp32_coupling(hg, ibem.IBEM_FP32_COUPLING_GENERATE)
    assert np.array_equal(_apply(hg, x, 1), y_gen)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_set_fp32_coupling(hg, 7)
    assert ei.value.status == "IBEM_ERR_ARG"
    hl = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(1, 2, q_cheb=8, eta=1.6))
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_set_fp32_coupling(hl, ibem.IBEM_FP32_COUPLING_STORE)
    assert ei.value.status == "IBEM_ERR_STATE"
    ibem.ibem_assemble(hl)
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_set_fp32_coupling(hl, ibem.IBEM_FP32_COUPLING_STORE)
    assert ei.value.status == "IBEM_ERR_ARG"
    for h in (hs, hg, hl):
        ibem.ibem_destroy(h)
