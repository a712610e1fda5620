"""Cluster tree, admissibility and block cluster tree (oracle; test only).

Sec. 4.1: each patch is refined uniformly; a cluster lambda = (patch, level,
index) is a square of the patch parameter domain, and the hierarchy of all of
them is the cluster tree.  Def. 4.1: a block (lambda, lambda') is admissible
when the cluster diameters are small compared with their distance.

Readings (the printed definition uses 0 < mu < 1 with max diam < mu dist, and
its far/near sentence is garbled):
* admissible  iff  eta * max(diam_s, diam_t) < dist(s, t), eta = 1/mu (eta = 1.6
  in the workloads);
* diam = 2 r and dist = max(0, |c_s - c_t| - r_s - r_t), with c = F(midpoint) and
  r = max |F(x) - c| over a 5 x 5 uniform grid of parameter points including
  the corners;
* the block tree starts from all patch pairs at level 0; an admissible block is
  far field, a non-admissible block at the leaf level (elements) is near field,
  any other block is split into its 4 x 4 child pairs.

Clusters are identified by (patch, level, ix, iy).

Pinned by: near and far blocks partition all element pairs exactly once, every
far block is admissible with a non-admissible parent
(tests/test_oracle_fmm.py::test_block_tree_partitions_all_element_pairs).
"""
import numpy as np


def bounding_ball(patch, level, ix, iy):
    """(center, radius) of the cluster square [ix, ix+1] x [iy, iy+1] / 2^level."""
    h = 1.0 / 2 ** level
    g = np.linspace(0.0, 1.0, 5)
    su, sv = np.meshgrid(g, g, indexing="xy")
    u = (ix + su.ravel()) * h
    v = (iy + sv.ravel()) * h
    F, _, _ = patch.eval(u, v)
    c, _, _ = patch.eval(np.array([(ix + 0.5) * h]), np.array([(iy + 0.5) * h]))
    c = c[0]
    r = np.sqrt(np.max(np.sum((F - c[None, :]) ** 2, axis=1)))
    return c, r


class ClusterGeometry:
    """Bounding balls of every cluster, memoised."""

    def __init__(self, patches):
        self.patches = patches
        self._cache = {}

    def ball(self, cl):
        if cl not in self._cache:
            patch, level, ix, iy = cl
            self._cache[cl] = bounding_ball(self.patches[patch], level, ix, iy)
        return self._cache[cl]

    def admissible(self, s, t, eta, reading="eta_diam"):
        """reading "eta_diam": eta max(diam) < dist (eta = 1/mu, the default);
        "eta_dist": max(diam) < eta dist (the other way to fit eta = 1.6 into
        the printed max diam < mu dist)."""
        cs, rs = self.ball(s)
        ct, rt = self.ball(t)
        d = np.sqrt(np.sum((cs - ct) ** 2)) - rs - rt
        dist = d if d > 0.0 else 0.0
        diam = 2.0 * (rs if rs > rt else rt)
        if reading == "eta_dist":
            return diam < eta * dist
        return eta * diam < dist


def children(cl):
    patch, level, ix, iy = cl
    return [(patch, level + 1, 2 * ix + dx, 2 * iy + dy) for dy in (0, 1) for dx in (0, 1)]


def block_cluster_tree(patches, m, eta, cg=None, reading="eta_diam"):
    """Return (near, far): lists of (sigma, tau) cluster pairs."""
    cg = cg or ClusterGeometry(patches)
    near, far = [], []
    stack = [((i, 0, 0, 0), (j, 0, 0, 0))
             for i in range(len(patches)) for j in range(len(patches))]
    while stack:
        s, t = stack.pop()
        if cg.admissible(s, t, eta, reading):
            far.append((s, t))
        elif s[1] == m:
            near.append((s, t))
        else:
            for sc in children(s):
                for tc in children(t):
                    stack.append((sc, tc))
    return near, far


def element_index(cl, m):
    patch, level, ix, iy = cl
    assert level == m
    return patch * 4 ** m + iy * 2 ** m + ix
