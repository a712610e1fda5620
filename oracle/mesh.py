"""Uniform patch refinement, elements and the B-spline dofs on them (oracle).

Sec. 4.1: every patch is refined uniformly in its parameter domain, giving 4^m
elements per patch at level m.  Sec. 2.2: S_{p,m} is the patchwise tensor
product spline space on Xi_{p,m} with n (2^m + p)^2 dofs and no matching across
patches (Eq. def::space).

Public dof order (shared with the GPU path's interface, not with its code):
dof(patch, j_u, j_v) = patch * n1^2 + j_v * n1 + j_u, n1 = 2^m + p.
Oracle element order: e = patch * 4^m + iy * 2^m + ix.
On element (ix, iy) the non-zero B-splines are j_u = ix..ix+p, j_v = iy..iy+p.
"""
import numpy as np

from . import bspline
from .geometry import surface_measure


class Mesh:
    def __init__(self, patches, p, m):
        self.patches = list(patches)
        self.n_patches = len(self.patches)
        self.p, self.m = int(p), int(m)
        self.ne1 = 2 ** self.m
        self.n1 = self.ne1 + self.p
        self.knots = bspline.open_uniform_knots(self.p, self.m)
        self.n_elements = self.n_patches * self.ne1 ** 2
        self.n_dofs = self.n_patches * self.n1 ** 2
        self.h = 1.0 / self.ne1

    def element(self, e):
        """(patch, ix, iy) of element e."""
        patch, r = divmod(e, self.ne1 ** 2)
        iy, ix = divmod(r, self.ne1)
        return patch, ix, iy

    def local_dofs(self, e):
        """Global dof indices of the (p+1)^2 B-splines on element e, ordered
        (a_v, a_u) -> a_v * (p+1) + a_u with j_u = ix + a_u, j_v = iy + a_v."""
        patch, ix, iy = self.element(e)
        pp = self.p + 1
        out = np.empty(pp * pp, dtype=np.int64)
        for av in range(pp):
            for au in range(pp):
                out[av * pp + au] = patch * self.n1 ** 2 + (iy + av) * self.n1 + (ix + au)
        return out

    def to_patch(self, e, st):
        """Element-local coordinates st (N,2) in [0,1]^2 -> patch parameters."""
        _, ix, iy = self.element(e)
        return np.stack(((ix + st[:, 0]) * self.h, (iy + st[:, 1]) * self.h), axis=1)

    def local_basis(self, e, uv):
        """Values of the (p+1)^2 local B-splines of element e at patch params uv.

        b_{ix}..b_{ix+p} depend only on the knots xi_{ix}..xi_{ix+2p+1}, so the
        recursion is run on that window; for points inside the element (all
        quadrature points are) this is the same arithmetic as on the full
        knot vector."""
        _, ix, iy = self.element(e)
        w = 2 * self.p + 2
        bu = bspline.basis_values(self.knots[ix:ix + w], self.p, uv[:, 0])
        bv = bspline.basis_values(self.knots[iy:iy + w], self.p, uv[:, 1])
        return (bv[:, :, None] * bu[:, None, :]).reshape(len(uv), -1)

    def geometry(self, patch, uv):
        F, Fu, Fv = self.patches[patch].eval(uv[:, 0], uv[:, 1])
        return F, surface_measure(Fu, Fv)

    def element_corners(self, e):
        """Physical corners at local (0,0), (1,0), (1,1), (0,1)."""
        patch, _, _ = self.element(e)
        st = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
        F, _ = self.geometry(patch, self.to_patch(e, st))
        return F
