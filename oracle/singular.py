"""Quadrature rules for element pairs (oracle; test infrastructure only).

Sec. 4, item 4: regular pairs use tensor Gauss rules; touching pairs need a
regularising transformation in the spirit of Sauter and Schwab.  The rules
below are derived here from the change of variables alone (no code is taken
from any book or library):

identical pair (singular on x^ = y^): per coordinate d, z_d = |y_d - x_d|,
  x_d = (1 - z_d) s_d (+ z_d for one of the two orderings), Jacobian (1 - z_d);
  the (z_1, z_2) square is cut into two triangles and each is mapped by the
  Duffy map (xi, xi*eta), Jacobian xi.  2 triangles x 4 orderings = 8 pieces.
common edge (canonical form: edge at x_1 = y_1 = 0, aligned in x_2 = y_2):
  z = |y_2 - x_2| with x_2 / y_2 as above; the cube (x_1, y_1, z) is cut into
  three pyramids by its largest coordinate and each is mapped by
  (xi, xi*eta_1, xi*eta_2), Jacobian xi^2.  3 pyramids x 2 orderings = 6 pieces.
common vertex (canonical form: vertex at x^ = y^ = 0): the 4-cube is cut into
  four pyramids by its largest coordinate, each mapped by
  (xi, xi*eta_1, xi*eta_2, xi*eta_3), Jacobian xi^3.  4 pieces.
After each map |F(x^) - F(y^)| = xi |G| with G smooth and non-zero, so the
integrand is smooth and every piece uses an 8-point Gauss rule per variable.

Pair classes (reading):
* same element -> identical;
* two physical corners in common -> common edge; one -> common vertex
  (corners match when |P - Q| <= 1e-10 * max diam);
* otherwise dist < 0.5 * max diam (bounding balls) -> both elements split 2 x 2,
  8 x 8 Gauss on each sub-square pair ("near-singular");
* otherwise 8 x 8 Gauss on each element ("regular").
The orders of the last two classes may be graded by the distance ratio of the
pair (``galerkin.graded_order``); the touching classes keep their rules.

Canonical orientation: the eight symmetries of the square are listed in
``DIHEDRAL`` in a fixed order; for a touching pair (A, B) the first (k_A, k_B)
in lexicographic order whose images of the canonical corners coincide is used.

Pinned by: the closed-form value of the self-interaction of the unit square and
of the 2 x 1 and 2 x 2 rectangles (edge and vertex pieces), and the constant
eigenfunction of the single-layer operator on the unit sphere
(tests/test_oracle_singular.py, tests/test_oracle_galerkin.py).
"""
import numpy as np

from .gauss import gauss_legendre

# rho_k(s, t) for the eight symmetries of [0,1]^2, as (a0, a1, a2, b0, b1, b2):
# rho(s, t) = (a0 + a1 s + a2 t, b0 + b1 s + b2 t).
DIHEDRAL = (
    (0, 1, 0, 0, 0, 1),     # (s, t)
    (1, 0, -1, 0, 1, 0),    # (1 - t, s)
    (1, -1, 0, 1, 0, -1),   # (1 - s, 1 - t)
    (0, 0, 1, 1, -1, 0),    # (t, 1 - s)
    (0, 0, 1, 0, 1, 0),     # (t, s)
    (1, -1, 0, 0, 0, 1),    # (1 - s, t)
    (1, 0, -1, 1, -1, 0),   # (1 - t, 1 - s)
    (0, 1, 0, 1, 0, -1),    # (s, 1 - t)
)

# local corner index of the point (s, t) for s, t in {0, 1}
_CORNER_ID = {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}


def apply_dihedral(k, st):
    a0, a1, a2, b0, b1, b2 = DIHEDRAL[k]
    s, t = st[:, 0], st[:, 1]
    return np.stack((a0 + a1 * s + a2 * t, b0 + b1 * s + b2 * t), axis=1)


def dihedral_corner(k, s, t):
    """Local corner index of rho_k(s, t) for a corner (s, t) of the square."""
    out = apply_dihedral(k, np.array([[float(s), float(t)]]))[0]
    return _CORNER_ID[(int(round(out[0])), int(round(out[1])))]


def _tensor4(n):
    g, w = gauss_legendre(n)
    a, b, c, d = np.meshgrid(g, g, g, g, indexing="ij")
    wa, wb, wc, wd = np.meshgrid(w, w, w, w, indexing="ij")
    return (a.ravel(), b.ravel(), c.ravel(), d.ravel(),
            (wa * wb * wc * wd).ravel())


def _split_coordinate(z, s, order):
    """Positions (x, y) with |y - x| = z, base (1 - z) s, for one ordering."""
    a = (1.0 - z) * s
    if order == 0:
        return a, a + z
    return a + z, a


def identical_rule(n=8):
    """(x^ (N,2), y^ (N,2), w (N)) on [0,1]^2 x [0,1]^2 for the identical pair."""
    xi, eta, s1, s2, W = _tensor4(n)
    X, Y, Wt = [], [], []
    for tri in (0, 1):
        z1, z2 = (xi, xi * eta) if tri == 0 else (xi * eta, xi)
        for o1 in (0, 1):
            for o2 in (0, 1):
                x1, y1 = _split_coordinate(z1, s1, o1)
                x2, y2 = _split_coordinate(z2, s2, o2)
                X.append(np.stack((x1, x2), axis=1))
                Y.append(np.stack((y1, y2), axis=1))
                Wt.append(W * xi * (1.0 - z1) * (1.0 - z2))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(Wt)


def edge_rule(n=8):
    """Rule for the canonical common-edge pair (edge x_1 = y_1 = 0, x_2 = y_2)."""
    xi, e1, e2, s, W = _tensor4(n)
    X, Y, Wt = [], [], []
    for pyr in (0, 1, 2):
        if pyr == 0:
            x1, y1, z = xi, xi * e1, xi * e2
        elif pyr == 1:
            x1, y1, z = xi * e1, xi, xi * e2
        else:
            x1, y1, z = xi * e1, xi * e2, xi
        for o in (0, 1):
            x2, y2 = _split_coordinate(z, s, o)
            X.append(np.stack((x1, x2), axis=1))
            Y.append(np.stack((y1, y2), axis=1))
            Wt.append(W * xi * xi * (1.0 - z))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(Wt)


def vertex_rule(n=8):
    """Rule for the canonical common-vertex pair (x^ = y^ = 0)."""
    xi, e1, e2, e3, W = _tensor4(n)
    X, Y, Wt = [], [], []
    for pyr in range(4):
        coords = [xi * e1, xi * e2, xi * e3]
        coords.insert(pyr, xi)
        x1, x2, y1, y2 = coords
        X.append(np.stack((x1, x2), axis=1))
        Y.append(np.stack((y1, y2), axis=1))
        Wt.append(W * xi ** 3)
    return np.concatenate(X), np.concatenate(Y), np.concatenate(Wt)


def regular_rule(n=8):
    g, w = gauss_legendre(n)
    a, b = np.meshgrid(g, g, indexing="xy")
    wa, wb = np.meshgrid(w, w, indexing="xy")
    st = np.stack((a.ravel(), b.ravel()), axis=1)
    return st, (wa * wb).ravel()


def near_singular_rule(n=8):
    """2 x 2 subdivision of both squares, n x n Gauss on each sub-square pair."""
    st, w = regular_rule(n)
    subs = [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]
    X, Y, Wt = [], [], []
    for ox, oy in subs:
        xs = np.stack((ox + 0.5 * st[:, 0], oy + 0.5 * st[:, 1]), axis=1)
        for px, py in subs:
            ys = np.stack((px + 0.5 * st[:, 0], py + 0.5 * st[:, 1]), axis=1)
            xx = np.repeat(xs, len(ys), axis=0)
            yy = np.tile(ys, (len(xs), 1))
            X.append(xx)
            Y.append(yy)
            Wt.append(np.outer(w, w).ravel() / 16.0)
    return np.concatenate(X), np.concatenate(Y), np.concatenate(Wt)


def match_corners(PA, PB, tol):
    """Pairs (i, j) of local corners with |PA[i] - PB[j]| <= tol."""
    out = []
    for i in range(4):
        for j in range(4):
            if np.sqrt(np.sum((PA[i] - PB[j]) ** 2)) <= tol:
                out.append((i, j))
    return out


def canonical_orientation(PA, PB, kind, tol):
    """First (kA, kB) mapping the canonical corner(s) of A and B onto each other."""
    need = [(0, 0)] if kind == "vertex" else [(0, 0), (0, 1)]
    for ka in range(8):
        for kb in range(8):
            ok = True
            for s, t in need:
                ca = dihedral_corner(ka, s, t)
                cb = dihedral_corner(kb, s, t)
                if np.sqrt(np.sum((PA[ca] - PB[cb]) ** 2)) > tol:
                    ok = False
                    break
            if ok:
                return ka, kb
    raise ValueError("no canonical orientation found for a touching pair")
