"""B-splines by the Cox-de Boor recursion (oracle; test infrastructure only).

Follows Def. 2.1 (p-open knot vector, b_j^0 indicator functions and the
recursion for p > 0) and the uniform refined knot vector Xi_{p,m} of Sec. 2.2
(p+1 zeros, interior knots i/2^m, p+1 ones).

Readings where the paper is silent:
* b_j^0 is the indicator of [xi_j, xi_{j+1}); the last non-empty interval is
  closed at its right end so that the basis sums to one on all of [0, 1].
* A recursion term with a zero denominator (repeated knots) is taken as 0.

Pinned by: partition of unity, the closed-form pieces printed for
Fig. fig::splines (tests/golden/fig_splines.txt), and reduction to the Bernstein
polynomials for a single element (tests/test_oracle_basis.py).
"""
import numpy as np


def open_uniform_knots(p, m):
    """Xi_{p,m}: p+1 zeros, 1/2^m .. (2^m-1)/2^m, p+1 ones (Sec. 2.2)."""
    inner = [i / 2.0 ** m for i in range(1, 2 ** m)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1), dtype=np.float64)


def num_basis(knots, p):
    return len(knots) - p - 1


def basis_values(knots, p, x):
    """Values b_j^p(x) for all j: array of shape (len(x), k), k = #knots - p - 1."""
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nk = len(knots)
    # index of the last non-empty interval (closed at its right end)
    last = max(j for j in range(nk - 1) if knots[j] < knots[j + 1])
    b = np.zeros((len(x), nk - 1))
    for j in range(nk - 1):
        if knots[j] < knots[j + 1]:
            if j == last:
                b[:, j] = (knots[j] <= x) & (x <= knots[j + 1])
            else:
                b[:, j] = (knots[j] <= x) & (x < knots[j + 1])
    for d in range(1, p + 1):
        nb = nk - 1 - d
        bn = np.zeros((len(x), nb))
        for j in range(nb):
            den1 = knots[j + d] - knots[j]
            den2 = knots[j + d + 1] - knots[j + 1]
            t = np.zeros(len(x))
            if den1 > 0.0:
                t += (x - knots[j]) / den1 * b[:, j]
            if den2 > 0.0:
                t += (knots[j + d + 1] - x) / den2 * b[:, j + 1]
            bn[:, j] = t
        b = bn
    return b


def basis_derivatives(knots, p, x):
    """First derivatives d/dx b_j^p(x), from the degree-(p-1) basis."""
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    k = num_basis(knots, p)
    if p == 0:
        return np.zeros((len(x), k))
    lower = basis_values(knots, p - 1, x)  # shape (len(x), k + 1)
    d = np.zeros((len(x), k))
    for j in range(k):
        den1 = knots[j + p] - knots[j]
        den2 = knots[j + p + 1] - knots[j + 1]
        if den1 > 0.0:
            d[:, j] += p / den1 * lower[:, j]
        if den2 > 0.0:
            d[:, j] -= p / den2 * lower[:, j + 1]
    return d


def space_dimension(n_patches, p, m):
    """dim S_{p,m}(Gamma) = n (2^m + p)^2 (Sec. 2.2, after Eq. def::space)."""
    return n_patches * (2 ** m + p) ** 2


def superspace_dimension(n_patches, p, m):
    """dim S*_{p,m}(Gamma) = n (2^m (p+1))^2 (Sec. 4.3)."""
    return n_patches * (2 ** m * (p + 1)) ** 2
