"""Pins for the oracle's patch maps and surface measure."""
import numpy as np
import pytest

from oracle import geometry, galerkin


def test_sphere_faces_lie_on_sphere_and_cover_it(sphere):
    rng = np.random.default_rng(11)
    u, v = rng.random(500), rng.random(500)
    for face in sphere:
        F, Fu, Fv = face.eval(u, v)
        np.testing.assert_allclose(np.linalg.norm(F, axis=1), 1.0, atol=1e-15)
        # outward orientation: (Fu x Fv) . F > 0
        assert np.all(np.sum(np.cross(Fu, Fv) * F, axis=1) > 0)
    # every direction is hit by exactly the face of its largest |coordinate|
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for x in d:
        ax = np.argmax(np.abs(x))
        face = 2 * ax + (0 if x[ax] > 0 else 1)
        n, t1, t2 = (np.array(t) for t in geometry.SPHERE_FACE_FRAMES[face])
        c = x / abs(x[ax])
        uu, vv = (c @ t1 + 1) / 2, (c @ t2 + 1) / 2
        F, _, _ = sphere[face].eval([uu], [vv])
        np.testing.assert_allclose(F[0], x, atol=1e-14)


def test_derivatives_against_finite_differences(sphere):
    u = np.array([0.1, 0.37, 0.5, 0.93])
    v = np.array([0.8, 0.21, 0.5, 0.07])
    h = 1e-6
    cyl = geometry.quarter_cylinder(1.3, 0.7)
    for patch in list(sphere) + [cyl]:
        _, Fu, Fv = patch.eval(u, v)
        fdu = (patch.eval(u + h, v)[0] - patch.eval(u - h, v)[0]) / (2 * h)
        fdv = (patch.eval(u, v + h)[0] - patch.eval(u, v - h)[0]) / (2 * h)
        np.testing.assert_allclose(Fu, fdu, atol=1e-8)
        np.testing.assert_allclose(Fv, fdv, atol=1e-8)


def test_sphere_area_by_gauss(sphere):
    # sum over elements of the 8 x 8 Gauss rule of k -> 4 pi (Sec. 3.2, surface measure)
    disc = galerkin.Discretisation(sphere, 0, 3, galerkin.LaplaceKernel())
    area = disc.rhs(lambda F: np.ones(len(F))).sum()
    assert abs(area - 4 * np.pi) < 1e-12


def test_sphere_area_radius_and_center():
    pats = geometry.unit_sphere(radius=1.7, center=(0.3, -1.0, 2.0))
    disc = galerkin.Discretisation(pats, 0, 2, galerkin.LaplaceKernel())
    area = disc.rhs(lambda F: np.ones(len(F))).sum()
    assert abs(area - 4 * np.pi * 1.7 ** 2) < 1e-9


def test_nurbs_quarter_cylinder_exact():
    # rational quadratic arcs are exact circles: |(x, y)| = R, area = (pi/2) R H
    R, H = 1.3, 0.7
    cyl = geometry.quarter_cylinder(R, H)
    u = np.linspace(0, 1, 37)
    F, Fu, Fv = cyl.eval(u, np.full_like(u, 0.4))
    np.testing.assert_allclose(np.hypot(F[:, 0], F[:, 1]), R, atol=1e-15)
    np.testing.assert_allclose(F[:, 2], 0.4 * H, atol=1e-15)
    disc = galerkin.Discretisation([cyl], 0, 2, galerkin.LaplaceKernel())
    area = disc.rhs(lambda F: np.ones(len(F))).sum()
    assert abs(area - 0.5 * np.pi * R * H) < 1e-12


def test_nurbs_rejects_nonpositive_weights():
    with pytest.raises(ValueError):
        geometry.NurbsPatch(1, 1, [0, 0, 1, 1], [0, 0, 1, 1], np.zeros((2, 2, 3)), np.array([[1, 1], [0, 1.0]]))


def test_perturbation_pieces_and_continuity():
    # Sec. 5 (perturbed mappings): slopes 1/2, 7/4, 1/2; f(0) = 0, f(1) = 1,
    # continuous at the kinks 0.3 (value 0.15) and 0.7 (value 0.85)
    f, df = geometry.perturbation(np.array([0.0, 0.1, 0.3, 0.5, 0.7, 0.9, 1.0]))
    np.testing.assert_allclose(f, [0.0, 0.05, 0.15, 0.5, 0.85, 0.95, 1.0], atol=1e-15)
    np.testing.assert_array_equal(df, [0.5, 0.5, 0.5, 1.75, 0.5, 0.5, 0.5])
    for k in (0.3, 0.7):
        lo, _ = geometry.perturbation(k - 1e-12)
        hi, _ = geometry.perturbation(k + 1e-12)
        assert abs(hi - lo) < 1e-11


def test_perturbed_sphere_image_corners_derivatives_area(sphere):
    pert = geometry.perturbed_sphere()
    rng = np.random.default_rng(12)
    u, v = rng.random(300), rng.random(300)
    c = np.array([0.0, 1.0])
    for face, pface in zip(sphere, pert):
        F, Fu, Fv = pface.eval(u, v)
        np.testing.assert_allclose(np.linalg.norm(F, axis=1), 1.0, atol=1e-15)
        assert np.all(np.sum(np.cross(Fu, Fv) * F, axis=1) > 0)
        # same corners, so the faces still meet edge to edge
        uu, vv = np.repeat(c, 2), np.tile(c, 2)
        np.testing.assert_allclose(pface.eval(uu, vv)[0], face.eval(uu, vv)[0], atol=1e-15)
    # central differences at points whose +-h stencil stays inside one piece
    uu = np.array([0.1, 0.45, 0.62, 0.85])
    vv = np.array([0.55, 0.2, 0.95, 0.4])
    h = 1e-6
    for pface in pert:
        _, Fu, Fv = pface.eval(uu, vv)
        fdu = (pface.eval(uu + h, vv)[0] - pface.eval(uu - h, vv)[0]) / (2 * h)
        fdv = (pface.eval(uu, vv + h)[0] - pface.eval(uu, vv - h)[0]) / (2 * h)
        np.testing.assert_allclose(Fu, fdu, atol=1e-8)
        np.testing.assert_allclose(Fv, fdv, atol=1e-8)
    # the area is invariant under reparametrisation: a Gauss rule split at the
    # kinks integrates the piecewise-smooth measure to 4 pi
    from oracle import gauss
    x, w = gauss.gauss_legendre(16)
    cuts = [0.0, 0.3, 0.7, 1.0]
    nodes = np.concatenate([a + (b - a) * x for a, b in zip(cuts, cuts[1:])])
    wts = np.concatenate([(b - a) * w for a, b in zip(cuts, cuts[1:])])
    U, V = np.meshgrid(nodes, nodes, indexing="ij")
    W = np.outer(wts, wts).ravel()
    area = 0.0
    for pface in pert:
        _, Fu, Fv = pface.eval(U.ravel(), V.ravel())
        area += np.sum(W * geometry.surface_measure(Fu, Fv))
    assert abs(area - 4 * np.pi) < 1e-12


def _nurbs(specs):
    return [geometry.NurbsPatch(*s) for s in specs]


def _area_and_volume(patches, m=3):
    """Area sum_e sum_g w k and volume (1/3) int x . n dA by the 8 x 8 Gauss rule
    per element (n = dF/du x dF/dv / k, so the sign follows the orientation)."""
    from oracle.mesh import Mesh
    from oracle import gauss
    me = Mesh(patches, 0, m)
    x, w = gauss.gauss_legendre(8)
    st = np.array([(a, b) for b in x for a in x])
    ww = np.outer(w, w).ravel()
    area = vol = 0.0
    for e in range(me.n_elements):
        patch, _, _ = me.element(e)
        uv = me.to_patch(e, st)
        F, Fu, Fv = patches[patch].eval(uv[:, 0], uv[:, 1])
        cr = np.cross(Fu, Fv)
        area += np.sum(ww * np.linalg.norm(cr, axis=1)) * me.h ** 2
        vol += np.sum(ww * np.sum(F * cr, axis=1)) * me.h ** 2 / 3.0
    return area, vol


def test_torus_patches():
    # (|(x, y)| - 2)^2 + z^2 = 1/4 everywhere; area 4 pi^2 R r, volume
    # 2 pi^2 R r^2 with outward normals; 16 patches meeting edge to edge
    import shapes
    pats = _nurbs(shapes.torus())
    assert len(pats) == 16
    rng = np.random.default_rng(13)
    u, v = rng.random(200), rng.random(200)
    for pt in pats:
        F, _, _ = pt.eval(u, v)
        np.testing.assert_allclose((np.hypot(F[:, 0], F[:, 1]) - 2.0) ** 2 + F[:, 2] ** 2, 0.25, atol=1e-14)
    area, vol = _area_and_volume(pats)
    assert abs(area - 4 * np.pi ** 2 * 2.0 * 0.5) < 1e-9
    assert abs(vol - 2 * np.pi ** 2 * 2.0 * 0.25) < 1e-9
    # every patch edge is shared with exactly one other patch's edge
    edges = []
    for pt in pats:
        for uu, vv in (((0.5,), (0.0,)), ((0.5,), (1.0,)), ((0.0,), (0.5,)), ((1.0,), (0.5,))):
            edges.append(pt.eval(uu, vv)[0][0])
    E = np.array(edges)
    d = np.linalg.norm(E[:, None, :] - E[None, :, :], axis=2)
    assert np.all(np.sum(d < 1e-12, axis=1) == 2)


def test_fichera_patches():
    # 24 unit squares, area 24, volume 8 - 1 with outward normals
    import shapes
    pats = _nurbs(shapes.fichera())
    assert len(pats) == 24
    area, vol = _area_and_volume(pats, m=1)
    assert abs(area - 24.0) < 1e-13
    assert abs(vol - 7.0) < 1e-13
    mids = np.array([pt.eval([0.5], [0.5])[0][0] for pt in pats])
    assert len({tuple(np.round(mm, 12)) for mm in mids}) == 24
    # no square lies on the removed corner's outer faces
    for mm in mids:
        assert not (np.max(mm) == 1.0 and np.all(mm >= 0.0))


def test_dimensions_on_torus_and_fichera_meshes():
    # n (2^m (p + 1))^2 superspace functions (Table tab::mat::sph) on the
    # built meshes, n (2^m + p)^2 B-splines
    import shapes
    from oracle.mesh import Mesh
    for specs, n in ((shapes.torus(), 16), (shapes.fichera(), 24)):
        for p, m in ((0, 1), (2, 2), (4, 1)):
            me = Mesh(_nurbs(specs), p, m)
            assert me.n_elements * (p + 1) ** 2 == n * (2 ** m * (p + 1)) ** 2
            assert me.n_dofs == n * (2 ** m + p) ** 2
