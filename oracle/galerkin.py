"""Dense Galerkin matrix of the single-layer operator in S_{p,m} (oracle).

Sec. 3.1, Eqs. fundament1/2 and varformdisc: the single-layer operator with
u*(x, y) = 1 / (4 pi |x - y|) (Laplace) or exp(i kappa |x - y|) / (4 pi |x - y|)
(Helmholtz).  Sec. 3.2 rewrites every entry on the reference domain:
    A[i, j] = sum over element pairs of
              int int k(x^) k(y^) u*(F(x^), F(y^)) b_i(x^) b_j(y^) dy^ dx^,
with b_i the patchwise tensor B-splines (row i = test function at x^).  The
bilinear form has no complex conjugation, so the Helmholtz matrix is
complex-symmetric.  Element pairs are integrated with the rules of
``singular``; the element parameter Jacobian is h^2 = 4^-m per element.

The "localised kernel" of Sec. 4.1 - the fundamental solution composed with the
patch maps and multiplied by both surface measures - is what ``LocalKernel``
objects evaluate, so a test can substitute another kernel (for example one that
is polynomial in the parameters).

Graded orders (Sec. 4 item 4: the order rises logarithmically towards the
singularity, up to 40; the rule is a reading): with grading > 0 a
non-touching pair takes graded_order(n_regular, grading, dist, diam) points per
direction (per sub-square pair when it is subdivided), dist and diam from the
elements' bounding balls as in the classification.  Pinned by the separated
flat squares of tests/test_oracle_grading.py (inclusion-exclusion over
rectangle self-interactions) and by the order being n_regular + grading per
halving of dist / diam below 3/4.

Pinned by: V 1 = 1 (Laplace) and V 1 = sin(k) e^{ik} / k (Helmholtz) on the unit
sphere, the Rayleigh quotients of Y_l against 1 / (2l + 1), the l = 1
densities 3 z (Laplace) and z / (i k j_1(k) h_1(k)) (Helmholtz), symmetry and
positivity of the Laplace matrix (tests/test_oracle_galerkin.py).
"""
import numpy as np

from . import singular
from .mesh import Mesh
from .tree import bounding_ball


MAX_GAUSS = 40


def graded_order(n_regular, grading, dist, diam):
    """Gauss order of a non-touching pair (Sec. 4 item 4: raised logarithmically
    towards the singularity, up to 40; reading): n_regular + grading * k with k
    the number of halvings of the ratio dist / diam below 3/4, i.e. the least
    k >= 0 with 2^k dist >= 3/4 diam; capped at 40, and 40 for dist = 0."""
    if grading == 0:
        return n_regular
    if not dist > 0.0:
        return MAX_GAUSS
    k = 0
    while dist * 2.0 ** k < 0.75 * diam and n_regular + grading * k < MAX_GAUSS:
        k += 1
    return min(n_regular + grading * k, MAX_GAUSS)


class LaplaceKernel:
    is_complex = False

    def __call__(self, FA, kA, uvA, pA, FB, kB, uvB, pB):
        r = np.sqrt(np.sum((FA - FB) ** 2, axis=-1))
        return kA * kB / (4.0 * np.pi * r)


class HelmholtzKernel:
    is_complex = True

    def __init__(self, kappa):
        self.kappa = float(kappa)

    def __call__(self, FA, kA, uvA, pA, FB, kB, uvB, pB):
        r = np.sqrt(np.sum((FA - FB) ** 2, axis=-1))
        return kA * kB * np.exp(1j * self.kappa * r) / (4.0 * np.pi * r)


def fundamental_solution(kernel, X, Y):
    """u*(X, Y) of the kernel's equation for physical points (no measures)."""
    r = np.sqrt(np.sum((X - Y) ** 2, axis=-1))
    if isinstance(kernel, HelmholtzKernel):
        return np.exp(1j * kernel.kappa * r) / (4.0 * np.pi * r)
    return 1.0 / (4.0 * np.pi * r)


class Discretisation:
    def __init__(self, patches, p, m, kernel, n_regular=8, n_singular=8, grading=0):
        self.mesh = Mesh(patches, p, m)
        self.kernel = kernel
        self.n_regular = n_regular
        self.n_singular = n_singular
        self.grading = grading
        me = self.mesh
        self.corners = [me.element_corners(e) for e in range(me.n_elements)]
        self.balls = []
        for e in range(me.n_elements):
            patch, ix, iy = me.element(e)
            self.balls.append(bounding_ball(me.patches[patch], me.m, ix, iy))
        self._regular_cache = {}
        self._nearsing_cache = {}
        self._rules = {}

    # ---- rules -------------------------------------------------------------
    def _rule(self, name):
        if name not in self._rules:
            fn = {"identical": singular.identical_rule, "edge": singular.edge_rule,
                  "vertex": singular.vertex_rule}[name]
            self._rules[name] = fn(self.n_singular)
        return self._rules[name]

    def _product_points(self, e, kind, n=None):
        n = self.n_regular if n is None else n
        cache = self._regular_cache if kind == "regular" else self._nearsing_cache
        if (e, n) not in cache:
            st, w = singular.regular_rule(n)
            if kind == "nearsing":
                subs = [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]
                st = np.concatenate([np.stack((ox + 0.5 * st[:, 0], oy + 0.5 * st[:, 1]), axis=1)
                                     for ox, oy in subs])
                w = np.concatenate([w / 4.0] * 4)
            me = self.mesh
            patch, _, _ = me.element(e)
            uv = me.to_patch(e, st)
            F, k = me.geometry(patch, uv)
            cache[(e, n)] = (uv, F, k, w * me.h ** 2, me.local_basis(e, uv), patch)
        return cache[(e, n)]

    # ---- classification ----------------------------------------------------
    def pair_class(self, eA, eB):
        """('identical'|'edge'|'vertex'|'nearsing'|'regular', kA, kB)."""
        if eA == eB:
            return "identical", 0, 0
        (cA, rA), (cB, rB) = self.balls[eA], self.balls[eB]
        diam = 2.0 * (rA if rA > rB else rB)
        tol = 1e-10 * diam
        matches = singular.match_corners(self.corners[eA], self.corners[eB], tol)
        if len(matches) >= 2:
            ka, kb = singular.canonical_orientation(self.corners[eA], self.corners[eB], "edge", tol)
            return "edge", ka, kb
        if len(matches) == 1:
            ka, kb = singular.canonical_orientation(self.corners[eA], self.corners[eB], "vertex", tol)
            return "vertex", ka, kb
        d = np.sqrt(np.sum((cA - cB) ** 2)) - rA - rB
        dist = d if d > 0.0 else 0.0
        if dist < 0.5 * diam:
            return "nearsing", 0, 0
        return "regular", 0, 0

    def pair_order(self, eA, eB):
        """Gauss points per direction of the pair: n_singular for touching pairs,
        else graded_order of the bounding-ball distance ratio."""
        cls, _, _ = self.pair_class(eA, eB)
        if cls in ("identical", "edge", "vertex"):
            return self.n_singular
        (cA, rA), (cB, rB) = self.balls[eA], self.balls[eB]
        diam = 2.0 * (rA if rA > rB else rB)
        d = np.sqrt(np.sum((cA - cB) ** 2)) - rA - rB
        return graded_order(self.n_regular, self.grading, d if d > 0.0 else 0.0, diam)

    # ---- element-pair block --------------------------------------------------
    def pair_block(self, eA, eB):
        """(p+1)^2 x (p+1)^2 block: rows = B-splines on eA, cols = on eB."""
        cls, ka, kb = self.pair_class(eA, eB)
        me = self.mesh
        if cls in ("regular", "nearsing"):
            n = self.pair_order(eA, eB)
            uvA, FA, kAv, wA, bA, pA = self._product_points(eA, cls, n)
            uvB, FB, kBv, wB, bB, pB = self._product_points(eB, cls, n)
            K = self.kernel(FA[:, None, :], kAv[:, None], uvA[:, None, :], pA,
                            FB[None, :, :], kBv[None, :], uvB[None, :, :], pB)
            return bA.T @ ((wA[:, None] * K * wB[None, :]) @ bB)
        X, Y, W = self._rule(cls)
        xa = singular.apply_dihedral(ka, X)
        yb = singular.apply_dihedral(kb, Y)
        pA, _, _ = me.element(eA)
        pB, _, _ = me.element(eB)
        uvA = me.to_patch(eA, xa)
        uvB = me.to_patch(eB, yb)
        FA, kAv = me.geometry(pA, uvA)
        FB, kBv = me.geometry(pB, uvB)
        K = self.kernel(FA, kAv, uvA, pA, FB, kBv, uvB, pB)
        bA = me.local_basis(eA, uvA)
        bB = me.local_basis(eB, uvB)
        wk = W * me.h ** 4 * K
        return bA.T @ (wk[:, None] * bB)

    def dense_matrix(self):
        me = self.mesh
        dt = np.complex128 if self.kernel.is_complex else np.float64
        A = np.zeros((me.n_dofs, me.n_dofs), dtype=dt)
        dofs = [me.local_dofs(e) for e in range(me.n_elements)]
        for eA in range(me.n_elements):
            for eB in range(me.n_elements):
                A[np.ix_(dofs[eA], dofs[eB])] += self.pair_block(eA, eB)
        return A

    # ---- right-hand side and mass-type quantities ------------------------------
    def rhs(self, g):
        """b_i = sum_e int k g(F) b_i with n_regular^2 Gauss (Sec. 3.2).

        ``g`` maps physical points (N, 3) to values (N,) or (N, R)."""
        me = self.mesh
        out = None
        for e in range(me.n_elements):
            uv, F, k, w, b, _ = self._product_points(e, "regular")
            gv = np.asarray(g(F))
            if gv.ndim == 1:
                gv = gv[:, None]
            if out is None:
                out = np.zeros((me.n_dofs, gv.shape[1]), dtype=np.result_type(gv, np.float64))
            out[me.local_dofs(e)] += b.T @ ((w * k)[:, None] * gv)
        return out

    def quadrature_points(self):
        """Physical Gauss points of every element (E * n^2, 3), element-major."""
        return np.concatenate([self._product_points(e, "regular")[1]
                               for e in range(self.mesh.n_elements)])
