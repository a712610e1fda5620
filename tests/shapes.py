"""Patch descriptions of the paper's other test geometries (Sec. 5), as NURBS
control data shared by the oracle and the library tests: input geometry only,
none of the method's arithmetic.

Each patch is (deg_u, deg_v, knots_u, knots_v, ctrl [ncp_v][ncp_u][3],
weights [ncp_v][ncp_u]).

* Torus: major radius 2, tube radius 0.5 (the paper gives outer radius 2 and
  inner radius 0.5, read here as these two radii), 16 rational biquadratic
  patches: four quarters of the revolution times four quarters of the tube,
  each a pipe bent by 90 degrees.  A quarter circle is the rational quadratic
  with control points (1, 0), (1, 1), (0, 1) and weights 1, 1/sqrt(2), 1; the
  surface of revolution is the tensor product of the revolution arc and the
  profile arc (weights multiply).
* Fichera cube: the cube [-1, 1]^3 without the corner octant [0, 1]^3, 24
  bilinear unit squares, each oriented with the outward normal of the solid.
"""
import numpy as np

_S = np.sqrt(0.5)
_KNOTS2 = [0.0, 0.0, 0.0, 1.0, 1.0, 1.0]
_KNOTS1 = [0.0, 0.0, 1.0, 1.0]


def _quarter_arc(k):
    """Control points (3, 2) and weights (3,) of the unit-circle arc from angle
    k pi/2 to (k + 1) pi/2."""
    a = 0.5 * np.pi * k
    c, s = np.cos(a), np.sin(a)
    pts = np.array([[c, s], [c - s, s + c], [-s, c]])
    return pts, np.array([1.0, _S, 1.0])


def torus(major=2.0, minor=0.5):
    patches = []
    for i in range(4):                       # revolution quarter (u)
        rev, wr = _quarter_arc(i)
        for j in range(4):                   # tube quarter (v)
            tub, wt = _quarter_arc(j)
            ctrl = np.zeros((3, 3, 3))
            wts = np.zeros((3, 3))
            for b in range(3):               # v index
                rho = major + minor * tub[b, 0]
                z = minor * tub[b, 1]
                for a in range(3):           # u index
                    ctrl[b, a] = (rho * rev[a, 0], rho * rev[a, 1], z)
                    wts[b, a] = wr[a] * wt[b]
            patches.append((2, 2, _KNOTS2, _KNOTS2, ctrl, wts))
    return patches


def _square(origin, du, dv):
    o, du, dv = (np.asarray(v, dtype=np.float64) for v in (origin, du, dv))
    ctrl = np.array([[o, o + du], [o + dv, o + du + dv]])
    return (1, 1, _KNOTS1, _KNOTS1, ctrl, np.ones((2, 2)))


def fichera():
    """24 unit squares; du x dv points out of the solid."""
    patches = []
    for axis in range(3):
        for sign in (1.0, -1.0):
            e1, e2 = np.eye(3)[(axis + 1) % 3], np.eye(3)[(axis + 2) % 3]
            if sign < 0:
                e1, e2 = e2, e1                # keep du x dv = sign * e_axis
            for c1 in (-1.0, 0.0):
                for c2 in (-1.0, 0.0):
                    lo = np.zeros(3)
                    lo[axis] = sign
                    lo[(axis + 1) % 3] = c1 if sign > 0 else c2
                    lo[(axis + 2) % 3] = c2 if sign > 0 else c1
                    # the outer faces x, y, z = +1 lose the square over [0, 1]^2
                    if sign > 0 and c1 == 0.0 and c2 == 0.0:
                        continue
                    patches.append(_square(lo, e1, e2))
        # the three inner faces of the notch: axis = 0, other coordinates in
        # [0, 1]; the solid lies on the negative side, so the normal is +e_axis
        e1, e2 = np.eye(3)[(axis + 1) % 3], np.eye(3)[(axis + 2) % 3]
        patches.append(_square(np.zeros(3), e1, e2))
    return patches
