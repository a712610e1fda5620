"""The arithmetic of the digit-sliced FP64-accurate coupling, modelled on the
CPU (the GPU kernel is tested against the oracle in
tests/test_gpu_sliced_coupling.py; this file pins the scheme it rests on).

A far block's kernel values A (rows [Re K; Im K]) and a source's moments B
(rows Re x, Im x) are written as a power of two times 6 signed digits,
v = 2^E sum_s d_s 2^{-7 - 8 s}, |d_s| <= 128.  The level sums
D_k = sum_{s + t = k} A_s B_t^T (k <= 5) are then integer matrix products, and

    K x = 2^{E + F - 14} sum_k 2^{-8 k} D_k.

Checked here:
* digits are integers of at most 8 significant bits (exact in BF16);
* every level sum stays below 2^23 (the FP32 tensor-core accumulation keeps
  such sums exactly), by the worst-case bound and on random blocks;
* the recombination, with levels 3..5 combined in FP32 as the kernel does,
  reproduces the FP64 product to 2^-46 of the block's scale 64 2^{E + F}, and
  to 2^-45 of max_i sum_b |K_ib| |x_b| for blocks whose entries vary by a
  factor of 4.
"""
import math

import numpy as np

S = 6


def _digits(v):
    u = v * 128.0
    out = []
    for _ in range(S):
        d = np.rint(u)
        out.append(d)
        u = (u - d) * 256.0
    return out


def _sliced_product(K, x):
    A = np.vstack([K.real, K.imag])
    B = np.stack([x.real, x.imag])
    E = math.frexp(float(np.max(np.abs(A))))[1]
    F = [math.frexp(float(np.max(np.abs(B[c]))))[1] for c in range(2)]
    Ad = _digits(A * 2.0 ** -E)
    y = np.zeros((128, 2))
    dmax = 0
    for c in range(2):
        Bd = _digits(B[c] * 2.0 ** -F[c])
        Dk = [sum(Ad[s].astype(np.int64) @ Bd[k - s].astype(np.int64) for s in range(k + 1) if k - s < S)
              for k in range(S)]
        dmax = max(dmax, max(int(np.max(np.abs(d))) for d in Dk))
        # levels 5..3 in FP32 (as the kernel), then the rest in FP64
        inv = np.float32(2.0 ** -8)
        T = np.float32(Dk[5]) * inv + np.float32(Dk[4])
        T = T.astype(np.float32) * inv + np.float32(Dk[3])
        acc = T.astype(np.float32).astype(np.float64)
        for k in (2, 1, 0):
            acc = acc * 2.0 ** -8 + Dk[k].astype(np.float64)
        y[:, c] = acc * 2.0 ** (E + F[c] - 14)
    yr = y[:64, 0] - y[64:, 1]
    yi = y[:64, 1] + y[64:, 0]
    return yr + 1j * yi, E, F, Ad, dmax


def _block(rng, spread):
    mag = np.exp(rng.uniform(-math.log(spread), 0.0, size=(64, 64)))
    K = mag * np.exp(1j * rng.uniform(0, 2 * np.pi, size=(64, 64))) * 2.0 ** int(rng.integers(-3, 4))
    xm = np.exp(rng.uniform(-math.log(spread), 0.0, size=64))
    x = xm * np.exp(1j * rng.uniform(0, 2 * np.pi, size=64)) * 2.0 ** int(rng.integers(-20, -5))
    return K, x


def test_digits_are_small_integers():
    rng = np.random.default_rng(1)
    v = rng.uniform(-1.0, 1.0, size=10000)
    ds = _digits(v)
    for d in ds:
        assert np.all(d == np.rint(d)) and np.max(np.abs(d)) <= 128
        # exact in BF16: the low 16 bits of the FP32 pattern are zero
        bits = d.astype(np.float32).view(np.uint32)
        assert np.all((bits & 0xFFFF) == 0)
    # the digits reconstruct v to 2^-48 (6 digits: 7 + 5 x 8 = 47 bits and half a digit)
    rec = sum(d * 2.0 ** (-7 - 8 * s) for s, d in enumerate(ds))
    assert np.max(np.abs(rec - v)) <= 2.0 ** -48


def test_level_sums_stay_below_2_23():
    # worst case: at most 6 pairs per level, 64 terms, |d_s d_t| <= 128^2
    assert max((min(k, S - 1) + 1) * 64 * 128 * 128 for k in range(S)) < 2 ** 23
    rng = np.random.default_rng(2)
    for _ in range(20):
        K, x = _block(rng, 1000.0)
        _, _, _, _, dmax = _sliced_product(K, x)
        assert dmax < 2 ** 23


def test_recombination_reproduces_the_fp64_product():
    rng = np.random.default_rng(3)
    worst_scale = worst_rows = 0.0
    for _ in range(60):
        K, x = _block(rng, 4.0)
        y, E, F, _, _ = _sliced_product(K, x)
        err = np.max(np.abs(y - K @ x))
        worst_scale = max(worst_scale, err / (64 * 2.0 ** (E + max(F))))
        worst_rows = max(worst_rows, err / np.max(np.abs(K) @ np.abs(x)))
    assert worst_scale < 2.0 ** -46, math.log2(worst_scale)
    assert worst_rows < 2.0 ** -45, math.log2(worst_rows)
