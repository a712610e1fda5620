"""CPU tests of libibem: it builds, loads, exports every symbol of
include/ibem.h, and its host-side block cluster tree and pair classification
equal the oracle's exactly (no device calls)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ibem():
    from paper_1708_09162_gb300 import build
    build.build()
    from paper_1708_09162_gb300 import ibem as mod
    return mod


def test_exports_every_declared_symbol(ibem):
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "ibem.h")).read()
    declared = set(re.findall(r"\b(ibem_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(ibem.EXPORTED)
    lib = ctypes.CDLL(ibem.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def _oracle_lists(patches_py, p, m, eta, reading="eta_diam"):
    from oracle import galerkin, tree
    disc = galerkin.Discretisation(patches_py, p, m, galerkin.LaplaceKernel())
    near, far = tree.block_cluster_tree(patches_py, m, eta, reading=reading)
    cls_code = {"identical": 0, "edge": 1, "vertex": 2, "nearsing": 3, "regular": 4}
    rows = []
    for s, t in near:
        eA, eB = tree.element_index(s, m), tree.element_index(t, m)
        c, ka, kb = disc.pair_class(eA, eB)
        rows.append((s[0], s[2], s[3], t[0], t[2], t[3], cls_code[c], 8 * ka + kb))
    frows = [tuple(s) + tuple(t) for s, t in far]
    return sorted(rows), sorted(frows)


@pytest.mark.parametrize("p,m", [(2, 2), (1, 3)])
def test_block_tree_equals_oracle_sphere(ibem, sphere, p, m):
    near, far = ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=6, eta=1.6))
    onear, ofar = _oracle_lists(sphere, p, m, 1.6)
    assert sorted(map(tuple, near.tolist())) == onear
    assert sorted(map(tuple, far.tolist())) == ofar


def test_block_tree_alternative_admissibility_reading(ibem, sphere):
    # Def. 4.1 read as max(diam) < eta dist: many more far blocks, lists equal
    # the oracle's with the same reading
    prm = ibem.make_params(1, 3, q_cheb=6, eta=1.6, admissibility=ibem.IBEM_ADMISSIBLE_ETA_DIST)
    near, far = ibem.ibem_block_tree(ibem.sphere_patches(), prm)
    onear, ofar = _oracle_lists(sphere, 1, 3, 1.6, reading="eta_dist")
    assert sorted(map(tuple, near.tolist())) == onear
    assert sorted(map(tuple, far.tolist())) == ofar
    near0, _ = ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(1, 3, q_cheb=6, eta=1.6))
    assert len(near) < len(near0)


def test_block_tree_equals_oracle_perturbed_sphere(ibem):
    # the perturbed face maps of Sec. 5 move the bounding balls and the
    # near-singular pairs; lists still equal the oracle's exactly
    from oracle import geometry
    pert = geometry.perturbed_sphere()
    near, far = ibem.ibem_block_tree(ibem.sphere_patches(perturbed=True), ibem.make_params(2, 3, q_cheb=6, eta=1.6))
    onear, ofar = _oracle_lists(pert, 2, 3, 1.6)
    assert sorted(map(tuple, near.tolist())) == onear
    assert sorted(map(tuple, far.tolist())) == ofar
    plain, _ = ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(2, 3, q_cheb=6, eta=1.6))
    assert sorted(map(tuple, plain.tolist())) != onear


@pytest.mark.parametrize("name,p,m", [("torus", 2, 2), ("fichera", 1, 2)])
def test_block_tree_equals_oracle_torus_fichera(ibem, name, p, m):
    # rational biquadratic torus (16 patches) and Fichera cube (24 bilinear
    # squares, re-entrant edges): touching classes across patches in every
    # relative orientation, admissibility on non-spherical clusters
    import shapes
    from oracle import geometry
    specs = getattr(shapes, name)()
    near, far = ibem.ibem_block_tree(ibem.nurbs_patches(specs), ibem.make_params(p, m, q_cheb=6, eta=1.6))
    onear, ofar = _oracle_lists([geometry.NurbsPatch(*sp) for sp in specs], p, m, 1.6)
    assert sorted(map(tuple, near.tolist())) == onear
    assert sorted(map(tuple, far.tolist())) == ofar
    assert len(ofar) > 0 and {r[6] for r in onear} >= {0, 1, 2, 4}


def test_block_tree_dense_mode_has_all_pairs(ibem):
    near, far = ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(1, 1, q_cheb=0))
    assert far.shape[0] == 0 and near.shape[0] == 24 * 24


def test_block_tree_nurbs_cylinder(ibem):
    # two rational-quadratic quarter cylinders side by side (a half cylinder)
    from oracle import geometry
    R, H = 1.0, 1.5
    a = geometry.quarter_cylinder(R, H)
    ctrl2 = a.ctrl.copy()
    ctrl2[:, :, 0], ctrl2[:, :, 1] = -a.ctrl[:, :, 1], a.ctrl[:, :, 0]   # rotate by 90 degrees
    b = geometry.NurbsPatch(2, 1, a.knots_u, a.knots_v, ctrl2, a.weights)
    specs = [(2, 1, a.knots_u, a.knots_v, a.ctrl, a.weights), (2, 1, b.knots_u, b.knots_v, b.ctrl, b.weights)]
    pats = ibem.nurbs_patches(specs)
    near, far = ibem.ibem_block_tree(pats, ibem.make_params(1, 3, q_cheb=4, eta=1.0))
    onear, ofar = _oracle_lists([a, b], 1, 3, 1.0)
    assert sorted(map(tuple, far.tolist())) == ofar
    # classes must agree; orientation codes too
    assert sorted(map(tuple, near.tolist())) == onear


def test_invalid_arguments_rejected(ibem):
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(9, 2))
    assert "p must be" in str(ei.value)
    pats = ibem.sphere_patches()
    pats[0].face = 7
    with pytest.raises(ibem.IbemError):
        ibem.ibem_block_tree(pats, ibem.make_params(1, 1))
    bad = ibem.nurbs_patches([(2, 1, [0, 0, 0, 1, 1, 1], [0, 0, 1, 1], np.zeros((2, 3, 3)), -np.ones((2, 3)))])
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_block_tree(bad, ibem.make_params(1, 1))
    assert "weights" in str(ei.value)
    # regular Gauss orders up to 40 per direction (Sec. 4 item 4)
    ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(4, 1, kernel=1, kappa=1.0, gauss_regular=40))
    with pytest.raises(ibem.IbemError) as ei:
        ibem.ibem_block_tree(ibem.sphere_patches(), ibem.make_params(2, 1, gauss_regular=41))
    assert "gauss_regular" in str(ei.value)
    assert ibem.ibem_status_string(5) == "IBEM_ERR_NOCONV"


def test_block_tree_partitions_every_element_pair(ibem):
    # near element pairs plus the leaves of the far cluster pairs cover every
    # (target, source) element pair exactly once, for random eta on the four
    # geometries (the library's host tree alone, no oracle)
    import shapes
    rng = np.random.default_rng(97)
    geos = [(ibem.sphere_patches(), 6), (ibem.sphere_patches(perturbed=True), 6),
            (ibem.nurbs_patches(shapes.torus()), 16), (ibem.nurbs_patches(shapes.fichera()), 24)]
    for pats, npatch in geos:
        for m in (1, 2):
            eta = float(rng.uniform(0.3, 3.0))
            near, far = ibem.ibem_block_tree(pats, ibem.make_params(1, m, q_cheb=4, eta=eta))
            n1 = 2 ** m
            E = npatch * n1 * n1
            cover = np.zeros((E, E), dtype=np.int32)
            eid = lambda pa, ix, iy: (pa * n1 + iy) * n1 + ix
            for r in near:
                cover[eid(r[0], r[1], r[2]), eid(r[3], r[4], r[5])] += 1
            for r in far:
                s = 2 ** (m - r[1])
                ia = [eid(r[0], r[2] * s + dx, r[3] * s + dy) for dy in range(s) for dx in range(s)]
                t = 2 ** (m - r[5])
                ib = [eid(r[4], r[6] * t + dx, r[7] * t + dy) for dy in range(t) for dx in range(t)]
                cover[np.ix_(ia, ib)] += 1
            assert np.all(cover == 1), (npatch, m, eta)
            # identical pairs are near and classed as such
            diag = near[(near[:, 0] == near[:, 3]) & (near[:, 1] == near[:, 4]) & (near[:, 2] == near[:, 5])]
            assert len(diag) == E and np.all(diag[:, 6] == 0)


def test_corrupt_geometry_rejected_on_the_host(ibem):
    # failure detection without a GPU: corrupt patch descriptions and parameters
    # are refused by the host-side validation with IBEM_ERR_GEOMETRY / ARG
    from oracle import geometry
    a = geometry.quarter_cylinder(1.0, 1.5)

    def tree(spec, **kw):
        return ibem.ibem_block_tree(ibem.nurbs_patches([spec]), ibem.make_params(1, 1, **kw))

    good = (2, 1, a.knots_u, a.knots_v, a.ctrl, a.weights)
    tree(good)
    cases = [
        ((2, 1, a.knots_u[::-1], a.knots_v, a.ctrl, a.weights), "non-decreasing"),
        ((2, 1, 0.5 * np.asarray(a.knots_u), a.knots_v, a.ctrl, a.weights), "from 0 to 1"),
        ((2, 1, a.knots_u, a.knots_v, np.zeros_like(a.ctrl), a.weights), "degenerate"),
        ((2, 1, a.knots_u, a.knots_v, np.where(np.arange(a.ctrl.size).reshape(a.ctrl.shape) == 4, np.nan, a.ctrl),
          a.weights), "degenerate"),
    ]
    for spec, text in cases:
        with pytest.raises(ibem.IbemError) as ei:
            tree(spec)
        assert ei.value.status == "IBEM_ERR_GEOMETRY" and text in str(ei.value), str(ei.value)
    for kw, text in (({"kernel": 1, "kappa": float("nan")}, "kappa"), ({"q_cheb": 4, "eta": float("nan")}, "eta")):
        with pytest.raises(ibem.IbemError) as ei:
            tree(good, **kw)
        assert ei.value.status == "IBEM_ERR_ARG" and text in str(ei.value)


@pytest.mark.parametrize("shape,p,m,base,grading", [("sphere", 2, 3, 4, 3), ("fichera", 1, 2, 3, 5),
                                                     ("perturbed", 1, 3, 6, 2)])
def test_graded_orders_equal_oracle(ibem, shape, p, m, base, grading):
    # Gauss order of every near pair (Sec. 4 item 4, graded reading) equals the
    # oracle's pair_order exactly, in the order of the block tree's near list
    from oracle import galerkin, geometry, tree
    import shapes
    if shape == "sphere":
        lib_p, ora_p = ibem.sphere_patches(), geometry.unit_sphere()
    elif shape == "perturbed":
        lib_p, ora_p = ibem.sphere_patches(perturbed=True), geometry.perturbed_sphere()
    else:
        specs = shapes.fichera()
        lib_p, ora_p = ibem.nurbs_patches(specs), [geometry.NurbsPatch(*s) for s in specs]
    prm = ibem.make_params(p, m, q_cheb=4, eta=1.6, gauss_regular=base, gauss_singular=5, gauss_grading=grading)
    near, _ = ibem.ibem_block_tree(lib_p, prm)
    orders = ibem.ibem_near_orders(lib_p, prm)
    assert len(orders) == len(near)
    disc = galerkin.Discretisation(ora_p, p, m, galerkin.LaplaceKernel(), n_regular=base, n_singular=5,
                                   grading=grading)
    got = {}
    for row, o in zip(near.tolist(), orders.tolist()):
        s = (row[0], m, row[1], row[2])
        t = (row[3], m, row[4], row[5])
        eA, eB = tree.element_index(s, m), tree.element_index(t, m)
        assert o == disc.pair_order(eA, eB), (row, o, disc.pair_order(eA, eB))
        got[o] = got.get(o, 0) + 1
    # the grading is exercised: more than one order among the non-touching pairs
    assert len([k for k in got if k != 5]) >= 2, got
    # grading 0 gives the base order to every non-touching pair
    prm0 = ibem.make_params(p, m, q_cheb=4, eta=1.6, gauss_regular=base, gauss_singular=5)
    o0 = ibem.ibem_near_orders(lib_p, prm0)
    assert set(o0[near[:, 6] >= 3].tolist()) == {base}
    with pytest.raises(ibem.IbemError):
        ibem.ibem_near_orders(lib_p, ibem.make_params(p, m, gauss_grading=40))
