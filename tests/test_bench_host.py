"""Host-side pieces of bench.py: the operation count of the generated coupling,
the resonance filter of the wavenumber draws, and the presence of every
section its flags select (no GPU)."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_sections_exist():
    import bench
    for name in ("oracle_child", "reference_arm", "laplace_section", "potentials_section", "batched_instances",
                 "config4_section", "fmm_error_study", "learned_preconditioner", "learned_config5",
                 "cnn_forward_timing", "ours"):
        assert callable(getattr(bench, name)), name


def test_generated_coupling_operation_count():
    import bench
    gen, mac = bench.gen_ops_per_launch(10, 8, 64)
    assert gen == 10 * 8 ** 4 * 247 and mac == 10 * 8 ** 4 * 48 * 64


def test_sliced_coupling_operation_count():
    # per far block and chunk of 32 right-hand sides: 4096 generated complex
    # values (247 each), 8192 sliced real values (58 each), 128 x 64
    # recombined accumulator entries (48 each); 21 slice-pair MMA groups
    import bench
    ops, flops = bench.sliced_ops_per_launch(10, 64)          # two chunks
    assert ops == 10 * 2 * (4096 * 247 + 8192 * 58 + 8192 * 48)
    assert flops == 10 * 2 * 21 * 2 * 128 * 64 * 64
    assert bench.sliced_ops_per_launch(10, 33) == bench.sliced_ops_per_launch(10, 64)
    assert bench.sliced_ops_per_launch(10, 32)[0] * 2 == ops


def test_bessel_zeros_and_resonance_filter():
    import bench
    z = bench.bessel_zeros(0, 1.0, 10.0)
    # j_0(x) = sin(x) / x vanishes at multiples of pi
    assert np.allclose(z, [math.pi, 2 * math.pi, 3 * math.pi], atol=1e-10)
    zs = bench.bessel_zeros(20, 7.0, 17.0)
    kept, rejected = bench.draw_wavenumbers(np.random.default_rng(3), 40)
    assert len(kept) == 40 and all(8.0 <= k <= 16.0 for k in kept)
    assert all(np.min(np.abs(zs - k)) >= 0.02 for k in kept)
    assert all(np.min(np.abs(zs - k)) < 0.02 for k in rejected)
