"""Interpolation-based far field, non-nested (oracle; test infrastructure only).

Sec. 4.2: on an admissible block (sigma, tau) the localised kernel is replaced
by its tensor Lagrange interpolant,
    k(x^, y^) ~ sum_{a, b} k(z_a^sigma, z_b^tau) L_a^sigma(x^) L_b^tau(y^),
so the block becomes  M_sigma K_{sigma tau} M_tau^T  with moment matrices
M_sigma[i, a] = int_sigma L_a^sigma(x^) b_i(x^) dx^ that do not depend on the
geometry.  The oracle applies this formula literally: every cluster uses its own
q x q Lagrange basis, moments are integrated directly against the B-splines, and
there are no nested (M2M / L2L) transfers.

Readings: interpolation nodes are the Chebyshev points of the first kind,
z_a = (1 - cos((2a + 1) pi / (2q))) / 2, on each side of the cluster square; the
tensor index is a = a_v * q + a_u.  Moments are integrated per element with
ceil((q + p) / 2) + 1 Gauss points per direction, exact for the polynomial
integrand.  Near blocks are the element-pair blocks of ``galerkin``.

The potential (Eq. repform) takes the same interpolation on every cluster that
is admissible for the evaluation point (a reading: the point is a ball of radius
0 in the admissibility test) and the Gauss rule of ``solve.potential`` on the
remaining elements.

The right-hand side of a field of point sources (Sec. 3.2 with g = sum_j c_j
u*(., y_j)) takes the same walk per source: on an admissible cluster the
integrand k(x^) u*(F(x^), y_j) is interpolated, so the cluster contributes its
moments mu_tau times the values at its nodes; the other elements take the Gauss
rule of ``Discretisation.rhs``.  It is the transpose of the interpolated
potential (u* is symmetric).

Pinned by: with a kernel that is a polynomial of degree < q in each parameter
variable the far field is exact, so the FMM operator equals the dense one to
rounding; with the true kernel the error against the dense matrix falls as q
grows.  Potential: a point kernel polynomial of degree < q in the parameters
gives the direct quadrature to rounding with both branches taken; with nothing
admissible it is the direct potential; with the true kernel its error against
the direct potential falls as q grows (tests/test_oracle_fmm.py).  Point-source
right-hand side: adjointness with the interpolated potential (Laplace and
Helmholtz, no conjugation), the direct right-hand side when nothing is
admissible, exactness for a parameter-polynomial point kernel, error against
the direct right-hand side falling with q (tests/test_oracle_rhs_sources.py).
"""
import math
from collections import defaultdict

import numpy as np

from . import bspline
from .gauss import gauss_legendre
from .tree import ClusterGeometry, block_cluster_tree, element_index


def chebyshev_nodes(q):
    a = np.arange(q, dtype=np.float64)
    return 0.5 * (1.0 - np.cos((2.0 * a + 1.0) * np.pi / (2.0 * q)))


def lagrange_values(nodes, x):
    """L_a(x) for all a: shape (len(x), q)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    q = len(nodes)
    L = np.ones((len(x), q))
    for a in range(q):
        for b in range(q):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return L


class FMMOperator:
    def __init__(self, disc, q, eta, near_block_cache=None):
        self.disc = disc
        self.mesh = disc.mesh
        self.q = int(q)
        self.eta = float(eta)
        self.nodes = chebyshev_nodes(self.q)
        me = self.mesh
        self.cg = ClusterGeometry(me.patches)
        self.near, self.far = block_cluster_tree(me.patches, me.m, self.eta, self.cg)
        self.near_elements = [(element_index(s, me.m), element_index(t, me.m)) for s, t in self.near]
        self.far_by_target = defaultdict(list)
        for s, t in self.far:
            self.far_by_target[s].append(t)
        self._mom1d = {}
        self._interp = {}
        self._near_blocks = {} if near_block_cache is None else near_block_cache
        self.near_by_row = defaultdict(list)
        for eA, eB in self.near_elements:
            self.near_by_row[eA].append(eB)

    # ---- moments -----------------------------------------------------------
    def moments_1d(self, level, i):
        """mu[j, a] = int over [i, i+1] / 2^level of L_a b_j  (all j, shape (n1, q))."""
        key = (level, i)
        if key not in self._mom1d:
            me = self.mesh
            ng = math.ceil((self.q + me.p) / 2) + 1
            g, w = gauss_legendre(ng)
            hl = 1.0 / 2 ** level
            per = 2 ** (me.m - level)
            mu = np.zeros((me.n1, self.q))
            for k in range(per):
                lo = i * hl + k * me.h
                x = lo + me.h * g
                b = bspline.basis_values(me.knots, me.p, x)           # (ng, n1)
                L = lagrange_values(self.nodes, (x - i * hl) / hl)     # (ng, q)
                mu += b.T @ ((w * me.h)[:, None] * L)
            self._mom1d[key] = mu
        return self._mom1d[key]

    def interpolation_geometry(self, cl):
        if cl not in self._interp:
            patch, level, ix, iy = cl
            hl = 1.0 / 2 ** level
            zu, zv = np.meshgrid(self.nodes, self.nodes, indexing="xy")
            uv = np.stack(((ix + zu.ravel()) * hl, (iy + zv.ravel()) * hl), axis=1)
            F, k = self.mesh.geometry(patch, uv)
            self._interp[cl] = (uv, F, k, patch)
        return self._interp[cl]

    def coupling(self, s, t):
        """K[a, b] = localised kernel at (z_a^s, z_b^t), shape (q^2, q^2)."""
        uvA, FA, kA, pA = self.interpolation_geometry(s)
        uvB, FB, kB, pB = self.interpolation_geometry(t)
        return self.disc.kernel(FA[:, None, :], kA[:, None], uvA[:, None, :], pA,
                                FB[None, :, :], kB[None, :], uvB[None, :, :], pB)

    def near_block(self, eA, eB):
        key = (eA, eB)
        if key not in self._near_blocks:
            self._near_blocks[key] = self.disc.pair_block(eA, eB)
        return self._near_blocks[key]

    # ---- application -------------------------------------------------------
    def _grid(self, x, patch):
        me = self.mesh
        n1 = me.n1
        return x[patch * n1 * n1:(patch + 1) * n1 * n1].reshape(n1, n1, -1)  # [jv, ju, r]

    def forward_moments(self, x):
        """x^_tau = M_tau^T x for every cluster tau that is the source of a far block."""
        xh = {}
        for (_, t) in self.far:
            if t in xh:
                continue
            patch, level, ix, iy = t
            mu_u = self.moments_1d(level, ix)
            mu_v = self.moments_1d(level, iy)
            X = self._grid(x, patch)
            xh[t] = np.einsum("vb,uc,vur->bcr", mu_v, mu_u, X).reshape(self.q * self.q, -1)
        return xh

    def matvec(self, x):
        me = self.mesh
        x2 = x.reshape(me.n_dofs, -1)
        dt = np.result_type(x2, np.complex128 if self.disc.kernel.is_complex else np.float64)
        y = np.zeros(x2.shape, dtype=dt)
        dofs = [me.local_dofs(e) for e in range(me.n_elements)]
        for eA, eB in self.near_elements:
            y[dofs[eA]] += self.near_block(eA, eB) @ x2[dofs[eB]]
        xh = self.forward_moments(x2)
        for s, targets in self.far_by_target.items():
            yh = sum(self.coupling(s, t) @ xh[t] for t in targets)
            patch, level, ix, iy = s
            mu_u = self.moments_1d(level, ix)
            mu_v = self.moments_1d(level, iy)
            Yh = yh.reshape(self.q, self.q, -1)                       # [a_v, a_u, r]
            n1 = me.n1
            y[patch * n1 * n1:(patch + 1) * n1 * n1] += np.einsum(
                "vb,uc,bcr->vur", mu_v, mu_u, Yh).reshape(n1 * n1, -1)
        return y.reshape(x.shape) if x.ndim == 1 else y

    # ---- potential (Eq. repform) with the far field interpolated -----------
    def cluster_moments(self, x2, cl):
        """x^_tau[b] = int_tau L_b^tau(y^) w(y^) dy^ for one cluster (shape (q^2, R))."""
        patch, level, ix, iy = cl
        X = self._grid(x2, patch)
        mu_u = self.moments_1d(level, ix)
        mu_v = self.moments_1d(level, iy)
        return np.einsum("vb,uc,vur->bcr", mu_v, mu_u, X).reshape(self.q * self.q, -1)

    def point_admissible(self, x, cl):
        """Reading of Def. 4.1 for a point and a cluster (the point as a ball of
        radius 0): eta * diam(tau) < dist(x, tau) = max(0, |x - c_tau| - r_tau)."""
        c, r = self.cg.ball(cl)
        d = np.sqrt(np.sum((x - c) ** 2)) - r
        return self.eta * 2.0 * r < (d if d > 0.0 else 0.0)

    def potential(self, w, points, point_kernel=None):
        """u(x) = int_Gamma u*(x, y) w(y) dy (Eq. repform), with the interpolation
        of Sec. 4.2 on every cluster that is admissible for x:
            int_tau u*(x, F(y^)) k(y^) w(y^) dy^
              ~ sum_b u*(x, F(z_b^tau)) k(z_b^tau) x^_tau[b].
        For each point the clusters are visited from the patch roots down: an
        admissible cluster is taken in the far field, a non-admissible element
        with the n x n Gauss rule of ``solve.potential``, any other cluster is
        split into its four children.  ``point_kernel(X (P,3), F (n,3), k (n,),
        uv (n,2), patch)`` replaces u*(x, F) k (a test hook); w is (N,) or (N, R)."""
        from .galerkin import fundamental_solution
        from .tree import children, element_index
        me = self.mesh
        w2 = w.reshape(me.n_dofs, -1)
        if point_kernel is None:
            kern = self.disc.kernel

            def point_kernel(X, F, k, uv, patch):
                return fundamental_solution(kern, X[:, None, :], F[None, :, :]) * k[None, :]
        dt = np.result_type(w2, np.complex128 if self.disc.kernel.is_complex else np.float64)
        u = np.zeros((len(points), w2.shape[1]), dtype=dt)
        moments = {}
        self.potential_counts = []
        for i, x in enumerate(np.asarray(points, dtype=np.float64)):
            nfar = nnear = 0
            stack = [(patch, 0, 0, 0) for patch in range(len(me.patches))]
            while stack:
                cl = stack.pop()
                if self.point_admissible(x, cl):
                    if cl not in moments:
                        moments[cl] = self.cluster_moments(w2, cl)
                    uv, F, k, patch = self.interpolation_geometry(cl)
                    u[i] += point_kernel(x[None, :], F, k, uv, patch)[0] @ moments[cl]
                    nfar += 1
                elif cl[1] == me.m:
                    e = element_index(cl, me.m)
                    uvq, F, k, wq, b, patch = self.disc._product_points(e, "regular")
                    dens = b @ w2[me.local_dofs(e)]
                    u[i] += point_kernel(x[None, :], F, k, uvq, patch)[0] @ (wq[:, None] * dens)
                    nnear += 1
                else:
                    stack.extend(children(cl))
            self.potential_counts.append((nfar, nnear))
        return u

    def rhs_sources(self, sources, charges, point_kernel=None):
        """Right-hand side b_i = int_Gamma g b_i (Sec. 3.2) of the field of point
        sources, g(x) = sum_j charges[j] u*(x, y_j), with the interpolation of
        Sec. 4.2 on every cluster that is admissible for a source (the walk of
        ``potential`` with the source in the place of the point):
            int_tau u*(F(x^), y) k(x^) b_i(x^) dx^
              ~ sum_a u*(F(z_a^tau), y) k(z_a^tau) mu_tau[i, a],
        mu_tau[i, a] = int_tau L_a^tau b_i (``moments_1d`` in each direction).
        A non-admissible element takes the n x n Gauss rule of
        ``Discretisation.rhs``.  ``point_kernel`` as in ``potential``.
        charges: (nsrc,) or (nsrc, R); returns (N, R)."""
        from .galerkin import fundamental_solution
        from .tree import children, element_index
        me = self.mesh
        Q = np.asarray(charges).reshape(len(sources), -1)
        if point_kernel is None:
            kern = self.disc.kernel

            def point_kernel(X, F, k, uv, patch):
                return fundamental_solution(kern, X[:, None, :], F[None, :, :]) * k[None, :]
        dt = np.result_type(Q, np.complex128 if self.disc.kernel.is_complex else np.float64)
        b = np.zeros((me.n_dofs, Q.shape[1]), dtype=dt)
        ghat = {}                                   # cluster -> (q^2, R) values k(z_a) g_far(F(z_a))
        self.rhs_counts = []
        for j, y in enumerate(np.asarray(sources, dtype=np.float64)):
            nfar = nnear = 0
            stack = [(patch, 0, 0, 0) for patch in range(len(me.patches))]
            while stack:
                cl = stack.pop()
                if self.point_admissible(y, cl):
                    uv, F, k, patch = self.interpolation_geometry(cl)
                    g = point_kernel(y[None, :], F, k, uv, patch)[0]
                    ghat[cl] = ghat.get(cl, 0) + np.outer(g, Q[j])
                    nfar += 1
                elif cl[1] == me.m:
                    e = element_index(cl, me.m)
                    uvq, F, k, wq, bq, patch = self.disc._product_points(e, "regular")
                    g = point_kernel(y[None, :], F, k, uvq, patch)[0]
                    b[me.local_dofs(e)] += bq.T @ np.outer(wq * g, Q[j])
                    nnear += 1
                else:
                    stack.extend(children(cl))
            self.rhs_counts.append((nfar, nnear))
        n1 = me.n1
        for (patch, level, ix, iy), G in ghat.items():
            mu_u = self.moments_1d(level, ix)
            mu_v = self.moments_1d(level, iy)
            b[patch * n1 * n1:(patch + 1) * n1 * n1] += np.einsum(
                "vb,uc,bcr->vur", mu_v, mu_u, G.reshape(self.q, self.q, -1)).reshape(n1 * n1, -1)
        return b

    def rows(self, rows, x):
        """Selected rows of the FMM operator applied to x (exact per row).  The
        moments x^_t are formed only for the source clusters these rows use, by
        the same formula as ``forward_moments``."""
        me = self.mesh
        x2 = x.reshape(me.n_dofs, -1)
        dt = np.result_type(x2, np.complex128 if self.disc.kernel.is_complex else np.float64)
        out = np.zeros((len(rows), x2.shape[1]), dtype=dt)
        xh = {}

        def moments(t):
            if t not in xh:
                xh[t] = self.cluster_moments(x2, t)
            return xh[t]

        n1 = me.n1
        for r, i in enumerate(rows):
            patch, rem = divmod(int(i), n1 * n1)
            jv, ju = divmod(rem, n1)
            ex = [ix for ix in range(ju - me.p, ju + 1) if 0 <= ix < me.ne1]
            ey = [iy for iy in range(jv - me.p, jv + 1) if 0 <= iy < me.ne1]
            # near part
            for iy in ey:
                for ix in ex:
                    e = patch * me.ne1 ** 2 + iy * me.ne1 + ix
                    loc = list(me.local_dofs(e)).index(i)
                    for eB in self.near_by_row[e]:
                        out[r] += self.near_block(e, eB)[loc] @ x2[me.local_dofs(eB)]
            # far part: every cluster that contains an element of the support
            for level in range(me.m + 1):
                sh = me.m - level
                for cy in sorted({iy >> sh for iy in ey}):
                    for cx in sorted({ix >> sh for ix in ex}):
                        s = (patch, level, cx, cy)
                        targets = self.far_by_target.get(s, [])
                        if not targets:
                            continue
                        yh = sum(self.coupling(s, t) @ moments(t) for t in targets)
                        mrow = np.outer(self.moments_1d(level, cy)[jv],
                                        self.moments_1d(level, cx)[ju]).ravel()
                        out[r] += mrow @ yh
        return out
