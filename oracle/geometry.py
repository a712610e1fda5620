"""Patch maps F_j : [0,1]^2 -> Gamma_j and surface measure (oracle; test only).

Sec. 2.2, Eq. def::geom: every patch is a NURBS map
    F(x, y) = sum c_{j1 j2} b_{j1}(x) b_{j2}(y) w_{j1 j2} / sum b b w,
and Sec. 3.2 defines the surface measure k(x^) = |d_x F x d_y F|.

Two kinds of patch are provided:
* ``NurbsPatch`` - the rational map above, evaluated by direct rational
  Cox-de Boor (``bspline.basis_values``) and the quotient rule for derivatives.
* ``SphereFace`` - the analytic cube-sphere face map
    F(u, v) = center + R c / |c|,  c = n + (2u-1) t1 + (2v-1) t2,
  used for the unit-sphere workloads: no exact rational biquadratic 6-patch
  sphere exists, so the closed-form sphere pins are run on this exact map.

* ``PerturbedPatch`` - either map composed with the piecewise-linear
  reparametrisation f of Sec. 5 (perturbed mappings) in both parameters.

Pinned by: |F| = R on the sphere, area 4 pi R^2, finite-difference derivatives,
and the exact area of a rational-quadratic quarter cylinder; for the perturbed
map, f against its three pieces and its continuity, the image on the sphere,
the corners of the unperturbed map, one-sided finite differences away from the
kinks, and the area 4 pi by a Gauss rule split at the kinks
(tests/test_oracle_geometry.py).
"""
import numpy as np

from . import bspline

# Face frames (n, t1, t2) with t1 x t2 = n, so every face is oriented outward.
SPHERE_FACE_FRAMES = (
    ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)),
    ((-1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)),
    ((0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)),
    ((0.0, -1.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)),
    ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)),
    ((0.0, 0.0, -1.0), (0.0, 1.0, 0.0), (1.0, 0.0, 0.0)),
)


class SphereFace:
    def __init__(self, face, radius=1.0, center=(0.0, 0.0, 0.0)):
        n, t1, t2 = (np.array(v) for v in SPHERE_FACE_FRAMES[face])
        self.n, self.t1, self.t2 = n, t1, t2
        self.radius = float(radius)
        self.center = np.asarray(center, dtype=np.float64)

    def eval(self, u, v):
        """Return F, dF/du, dF/dv, each of shape (len(u), 3)."""
        u = np.atleast_1d(np.asarray(u, dtype=np.float64))
        v = np.atleast_1d(np.asarray(v, dtype=np.float64))
        c = (self.n[None, :] + (2.0 * u - 1.0)[:, None] * self.t1[None, :]
             + (2.0 * v - 1.0)[:, None] * self.t2[None, :])
        r2 = np.sum(c * c, axis=1)
        r = np.sqrt(r2)
        F = self.center[None, :] + self.radius * c / r[:, None]
        # d/du (c/|c|) = (2 t1 - c (c . 2 t1) / |c|^2) / |c|
        ct1 = c @ self.t1
        ct2 = c @ self.t2
        Fu = self.radius * 2.0 * (self.t1[None, :] - c * (ct1 / r2)[:, None]) / r[:, None]
        Fv = self.radius * 2.0 * (self.t2[None, :] - c * (ct2 / r2)[:, None]) / r[:, None]
        return F, Fu, Fv


class NurbsPatch:
    """NURBS patch; ctrl has shape (ncp_v, ncp_u, 3), weights (ncp_v, ncp_u)."""

    def __init__(self, deg_u, deg_v, knots_u, knots_v, ctrl, weights):
        self.deg_u, self.deg_v = int(deg_u), int(deg_v)
        self.knots_u = np.asarray(knots_u, dtype=np.float64)
        self.knots_v = np.asarray(knots_v, dtype=np.float64)
        self.ctrl = np.asarray(ctrl, dtype=np.float64)
        self.weights = np.asarray(weights, dtype=np.float64)
        if self.ctrl.shape[:2] != self.weights.shape:
            raise ValueError("ctrl / weights shape mismatch")
        if np.any(self.weights <= 0.0):
            raise ValueError("NURBS weights must be positive")

    def eval(self, u, v):
        u = np.atleast_1d(np.asarray(u, dtype=np.float64))
        v = np.atleast_1d(np.asarray(v, dtype=np.float64))
        bu = bspline.basis_values(self.knots_u, self.deg_u, u)      # (n, ku)
        bv = bspline.basis_values(self.knots_v, self.deg_v, v)      # (n, kv)
        du = bspline.basis_derivatives(self.knots_u, self.deg_u, u)
        dv = bspline.basis_derivatives(self.knots_v, self.deg_v, v)
        w = self.weights                                             # (kv, ku)
        cw = self.ctrl * w[:, :, None]                               # (kv, ku, 3)
        W = np.einsum("nj,ni,ji->n", bv, bu, w)
        Wu = np.einsum("nj,ni,ji->n", bv, du, w)
        Wv = np.einsum("nj,ni,ji->n", dv, bu, w)
        P = np.einsum("nj,ni,jid->nd", bv, bu, cw)
        Pu = np.einsum("nj,ni,jid->nd", bv, du, cw)
        Pv = np.einsum("nj,ni,jid->nd", dv, bu, cw)
        F = P / W[:, None]
        Fu = (Pu - F * Wu[:, None]) / W[:, None]
        Fv = (Pv - F * Wv[:, None]) / W[:, None]
        return F, Fu, Fv


def perturbation(x):
    """The piecewise-linear f : [0, 1] -> [0, 1] of Sec. 5 (perturbed mappings),
    f(x) = x/2 on [0, 0.3], 1.75 x - 0.375 on (0.3, 0.7), (x + 1)/2 on [0.7, 1];
    returns f(x) and f'(x) (slope of the left piece at the two kinks)."""
    x = np.asarray(x, dtype=np.float64)
    f = np.where(x <= 0.3, 0.5 * x, np.where(x < 0.7, 1.75 * x - 0.375, 0.5 * (x + 1.0)))
    df = np.where(x <= 0.3, 0.5, np.where(x < 0.7, 1.75, 0.5))
    return f, df


class PerturbedPatch:
    """A patch map composed with f in each parameter (Sec. 5): G(u, v) =
    F(f(u), f(v)), dG/du = f'(u) dF/du, dG/dv = f'(v) dF/dv.  Same image and
    corners as F, but a parametrisation that is only H^1."""

    def __init__(self, patch):
        self.patch = patch

    def eval(self, u, v):
        fu, du = perturbation(np.atleast_1d(u))
        fv, dv = perturbation(np.atleast_1d(v))
        F, Fu, Fv = self.patch.eval(fu, fv)
        return F, Fu * du[:, None], Fv * dv[:, None]


def perturbed_sphere(radius=1.0, center=(0.0, 0.0, 0.0)):
    """The cube-sphere faces, each composed with the perturbation (Sec. 5)."""
    return [PerturbedPatch(p) for p in unit_sphere(radius, center)]


def surface_measure(Fu, Fv):
    """k = |dF/du x dF/dv| (Sec. 3.2)."""
    return np.linalg.norm(np.cross(Fu, Fv), axis=1)


def unit_sphere(radius=1.0, center=(0.0, 0.0, 0.0)):
    """Six cube-sphere faces covering the sphere of the given radius."""
    return [SphereFace(f, radius, center) for f in range(6)]


def quarter_cylinder(radius, height):
    """Rational-quadratic quarter cylinder: u along the arc, v along z (linear)."""
    s = np.sqrt(0.5)
    arc = [(radius, 0.0), (radius, radius), (0.0, radius)]
    wts = [1.0, s, 1.0]
    ctrl = np.zeros((2, 3, 3))
    weights = np.zeros((2, 3))
    for j, z in enumerate((0.0, height)):
        for i in range(3):
            ctrl[j, i] = (arc[i][0], arc[i][1], z)
            weights[j, i] = wts[i]
    return NurbsPatch(2, 1, [0, 0, 0, 1, 1, 1], [0, 0, 1, 1], ctrl, weights)
