"""Gauss-Legendre quadrature on [0, 1] (oracle; test infrastructure only).

The paper integrates regular element pairs with tensor Gauss rules and
implements Gauss rules up to order 40 (Sec. 4, item 4).  Nodes are the roots of
the Legendre polynomial P_n, found by Newton's method with P_n and P_n'
evaluated by the three-term recurrence
    (k+1) P_{k+1}(t) = (2k+1) t P_k(t) - k P_{k-1}(t),
and weights 2 / ((1 - t^2) P_n'(t)^2) on [-1, 1], then mapped affinely to
[0, 1].

Pinned by: exact integration of x^k, k <= 2n-1 (tests/test_oracle_basis.py).
"""
import numpy as np


def _legendre_and_derivative(n, t):
    p_prev = np.ones_like(t)
    p = t.copy()
    if n == 0:
        return p_prev, np.zeros_like(t)
    for k in range(1, n):
        p_prev, p = p, ((2 * k + 1) * t * p - k * p_prev) / (k + 1)
    # P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1)
    dp = n * (t * p - p_prev) / (t * t - 1.0)
    return p, dp


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (nodes ascending, weights)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    i = np.arange(1, n + 1, dtype=np.float64)
    # Chebyshev-like initial guesses for the roots, descending in t.
    t = np.cos(np.pi * (i - 0.25) / (n + 0.5))
    for _ in range(100):
        p, dp = _legendre_and_derivative(n, t)
        dt = p / dp
        t = t - dt
        if np.max(np.abs(dt)) < 1e-16:
            break
    p, dp = _legendre_and_derivative(n, t)
    w = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(t)
    t, w = t[order], w[order]
    return 0.5 * (t + 1.0), 0.5 * w
