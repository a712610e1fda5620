import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sphere():
    from oracle import geometry
    return geometry.unit_sphere()


@pytest.fixture(scope="session")
def laplace_p2m2(sphere):
    """Dense Laplace Galerkin matrix, unit sphere, p = 2, m = 2 (216 dofs)."""
    from oracle import galerkin
    disc = galerkin.Discretisation(sphere, 2, 2, galerkin.LaplaceKernel())
    return disc, disc.dense_matrix()


def seeded_ball_points(n, radius, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * (radius * rng.random(n) ** (1.0 / 3.0))[:, None]
