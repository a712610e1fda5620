"""Pins of the oracle network, flexible GMRES and the learned preconditioner."""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn, learned, solve


def _setup(C=3, B=2, H=5, W=6, seed=0):
    rng = np.random.default_rng(seed)
    params = rng.normal(0.0, 0.4, cnn.n_params(C))
    x = rng.normal(size=(B, 2, H, W))
    t = rng.normal(size=(B, 2, H, W))
    return params, x, t


def test_param_count_and_layout():
    assert cnn.n_params(32) == (2 * 32 * 9 + 32) + 2 * (32 * 32 * 9 + 32) + (32 * 2 * 9 + 2)
    p = np.arange(cnn.n_params(2), dtype=float)
    layers = cnn.unpack(p, 2)
    assert layers[0][0].shape == (2, 2, 3, 3) and layers[0][1][0] == 36.0
    assert layers[3][1][-1] == p[-1]


def test_single_channel_conv_is_correlate2d():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(7, 9))
    w = rng.normal(size=(3, 3))
    ref = scipy.signal.correlate2d(x, w, mode="same", boundary="fill", fillvalue=0.0) + 0.25
    out = cnn.conv3x3(x[None, None], w[None, None], np.array([0.25]))[0, 0]
    assert np.max(np.abs(out - ref)) < 1e-13


def test_impulse_response_is_flipped_kernel():
    w = np.arange(9, dtype=float).reshape(3, 3) + 1.0
    x = np.zeros((1, 1, 6, 6))
    x[0, 0, 3, 2] = 1.0
    out = cnn.conv3x3(x, w[None, None], np.zeros(1))[0, 0]
    for dy in range(3):
        for dx in range(3):
            assert out[3 - (dy - 1), 2 - (dx - 1)] == w[dy, dx]
    assert np.count_nonzero(out) == 9


def test_zero_weights_give_last_bias():
    C = 4
    p = np.zeros(cnn.n_params(C))
    p[-2:] = [0.5, -1.5]
    out = cnn.forward(p, np.random.default_rng(2).normal(size=(3, 2, 4, 5)), C)
    assert np.all(out[:, 0] == 0.5) and np.all(out[:, 1] == -1.5)


def test_gradient_matches_central_differences():
    C = 3
    params, x, t = _setup(C)
    loss, g = cnn.loss_and_grad(params, x, t, C)
    assert loss == pytest.approx(0.5 * np.sum((cnn.forward(params, x, C) - t) ** 2) / x.shape[0])
    rng = np.random.default_rng(3)
    eps = 1e-6
    # random directions
    for _ in range(3):
        d = rng.normal(size=params.shape)
        lp = cnn.loss_and_grad(params + eps * d, x, t, C)[0]
        lm = cnn.loss_and_grad(params - eps * d, x, t, C)[0]
        assert (lp - lm) / (2 * eps) == pytest.approx(g @ d, rel=1e-7)
    # single entries in every layer: a weight, a corner tap and the bias
    off = 0
    for ci, co in cnn.layer_channels(C):
        for i in (off, off + co * ci * 9 - 1, off + co * ci * 9):
            e = np.zeros_like(params)
            e[i] = 1.0
            lp = cnn.loss_and_grad(params + eps * e, x, t, C)[0]
            lm = cnn.loss_and_grad(params - eps * e, x, t, C)[0]
            assert (lp - lm) / (2 * eps) == pytest.approx(g[i], rel=1e-6, abs=1e-10)
        off += co * ci * 9 + co


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3])
    opt = cnn.Adam(3, lr=0.01)
    p = opt.step(np.zeros(3), g)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_reduces_loss():
    C = 4
    rng = np.random.default_rng(5)
    params = rng.normal(0.0, 0.3, cnn.n_params(C))
    x = rng.normal(size=(4, 2, 6, 6))
    t = 0.5 * x[:, ::-1]
    opt = cnn.Adam(len(params), lr=1e-2)
    l0 = cnn.loss_and_grad(params, x, t, C)[0]
    for _ in range(60):
        _, g = cnn.loss_and_grad(params, x, t, C)
        params = opt.step(params, g)
    assert cnn.loss_and_grad(params, x, t, C)[0] < 0.5 * l0


def _system(n=40, seed=7):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    return A, b


def test_fgmres_exact_inverse_one_step():
    A, b = _system()
    Ainv = np.linalg.inv(A)
    x, its = solve.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, rtol=1e-12)
    assert its == 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


def test_fgmres_fixed_preconditioner_equals_gmres():
    A, b = _system()
    d = np.diag(A).copy()
    x1, i1 = solve.fgmres(lambda v: A @ v, b, lambda v: v / d, rtol=1e-10, restart=15)
    x2, i2 = solve.gmres(lambda v: A @ v, b, rtol=1e-10, restart=15, diag=d)
    assert i1 == i2
    assert np.linalg.norm(x1 - x2) < 1e-9 * np.linalg.norm(x2)


def test_fgmres_variable_preconditioner_converges():
    A, b = _system()
    rng = np.random.default_rng(9)
    d = np.diag(A).copy()

    def varying(v):
        return v / d * (1.0 + 0.3 * rng.random()) + 0.05 * np.tanh(v.real)

    rec = []
    x, its = solve.fgmres(lambda v: A @ v, b, varying, rtol=1e-10, restart=60, record=rec)
    assert np.linalg.norm(b - A @ x) <= 1.0001e-10 * np.linalg.norm(b)
    res = [np.linalg.norm(b - A @ xk) for xk in rec]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))


def test_block_jacobi_groups(sphere):
    from oracle.mesh import Mesh
    for m, nblocks in ((1, 6), (2, 6), (3, 24)):
        me = Mesh(sphere, 2, m)
        groups = learned.block_jacobi_groups(me)
        assert len(groups) == nblocks
        allg = np.sort(np.concatenate(groups))
        assert np.array_equal(allg, np.arange(me.n_dofs))
    me = Mesh(sphere, 2, 3)
    g0 = learned.block_jacobi_groups(me)[0]
    # first cluster of patch 0 at level 1: anchors 0..3 in each direction
    assert set(g0.tolist()) == {jv * me.n1 + ju for jv in range(4) for ju in range(4)}


def test_learned_apply_and_pairs_identities():
    rng = np.random.default_rng(11)
    n1, npatch = 5, 2
    N = npatch * n1 * n1
    M = np.eye(N) * 3 + 0.2 * rng.normal(size=(N, N))
    groups = [np.arange(0, N // 2), np.arange(N // 2, N)]
    bj = learned.BlockJacobi(M, groups)
    C = 3
    params = rng.normal(0.0, 0.3, cnn.n_params(C))
    v = rng.normal(size=N) + 1j * rng.normal(size=N)
    # zero last layer: block-Jacobi alone
    p0 = params.copy()
    p0[-(2 * C * 9 + 2):] = 0.0
    assert np.allclose(learned.learned_apply(v, bj, p0, C, n1), bj(v), rtol=0, atol=1e-14)
    # homogeneous of degree one in positive scalings
    z1 = learned.learned_apply(v, bj, params, C, n1)
    z2 = learned.learned_apply(7.0 * v, bj, params, C, n1)
    assert np.allclose(z2, 7.0 * z1, rtol=1e-12, atol=0)
    # a pair reconstructs r and e
    e = rng.normal(size=N) + 1j * rng.normal(size=N)
    r = M @ e
    inp, tgt = learned.training_pair(r, e, bj, n1)
    s = bj(r)
    sig = learned.rms(s)
    assert inp.shape == (npatch, 2, n1, n1)
    assert np.allclose(sig * cnn.images_to_vector(inp + tgt), e, atol=1e-12)
    assert np.allclose(sig * cnn.images_to_vector(inp), s, atol=1e-12)
    assert np.sqrt(np.mean(inp ** 2)) == pytest.approx(1.0)


def test_operator_loss_gradient_matches_central_differences():
    """dL/dparams of the residual-norm objective against central differences,
    with a random complex A (A^H its conjugate transpose) and a block-Jacobi of
    its diagonal blocks."""
    rng = np.random.default_rng(13)
    n1, npatch, C = 4, 2, 3
    N = npatch * n1 * n1
    A = np.eye(N) * 2 + 0.3 * (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    bj = learned.BlockJacobi(A, [np.arange(0, N // 2), np.arange(N // 2, N)])
    rs = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    rs /= np.linalg.norm(rs, axis=1)[:, None]
    params = rng.normal(0.0, 0.3, cnn.n_params(C))
    f = lambda p: learned.operator_loss_and_grad(p, rs, lambda z: A @ z, lambda z: A.conj().T @ z, bj, C, n1)
    loss, g = f(params)
    # the loss is the residual of the preconditioned vectors
    z0 = [learned.learned_apply(r, bj, params, C, n1) for r in rs]
    assert loss == pytest.approx(sum(np.linalg.norm(A @ z - r) ** 2 for z, r in zip(z0, rs)) / 6.0, rel=1e-12)
    eps = 1e-6
    for _ in range(3):
        d = rng.normal(size=params.shape)
        fd = (f(params + eps * d)[0] - f(params - eps * d)[0]) / (2 * eps)
        assert fd == pytest.approx(g @ d, rel=1e-6)


def test_coarse_grid_restriction_and_prolongation():
    # ragged blocks (n1 = 7, f = 3 and 2): R P = identity on coarse images, P is
    # the adjoint of the block sum, f = 1 changes nothing
    rng = np.random.default_rng(17)
    for n1, f in ((7, 3), (7, 2), (6, 2)):
        nc = learned.coarse_size(n1, f)
        c = rng.normal(size=(2, 2, nc, nc))
        assert np.allclose(learned.restrict(learned.prolong(c, f, n1), f), c, rtol=0, atol=1e-14)
        y = rng.normal(size=(2, 2, n1, n1))
        assert np.isclose(np.sum(learned.prolong(c, f, n1) * y), np.sum(c * learned.prolong_adjoint(y, f, nc)))
        # mean of a block: a constant image stays constant, a single pixel is divided by the block size
        one = np.zeros((1, 1, n1, n1))
        one[0, 0, 0, 0] = 1.0
        assert learned.restrict(one, f)[0, 0, 0, 0] == pytest.approx(1.0 / (f * f))
    x = rng.normal(size=(1, 2, 5, 5))
    assert learned.restrict(x, 1) is x and learned.prolong(x, 1, 5) is x


def test_coarse_operator_loss_gradient_matches_central_differences():
    # the residual-norm objective of the coarse-grid variant (f = 2 on ragged
    # 5 x 5 patch images): loss = direct evaluation, gradient = differences
    rng = np.random.default_rng(19)
    n1, npatch, C, f = 5, 2, 3, 2
    N = npatch * n1 * n1
    A = np.eye(N) * 2 + 0.3 * (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    bj = learned.BlockJacobi(A, [np.arange(0, N // 2), np.arange(N // 2, N)])
    rs = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    rs /= np.linalg.norm(rs, axis=1)[:, None]
    params = rng.normal(0.0, 0.3, cnn.n_params(C))
    fn = lambda p: learned.operator_loss_and_grad(p, rs, lambda z: A @ z, lambda z: A.conj().T @ z, bj, C, n1, f)
    loss, g = fn(params)
    z0 = [learned.learned_apply(r, bj, params, C, n1, f) for r in rs]
    assert loss == pytest.approx(sum(np.linalg.norm(A @ z - r) ** 2 for z, r in zip(z0, rs)) / 6.0, rel=1e-12)
    eps = 1e-6
    for _ in range(3):
        d = rng.normal(size=params.shape)
        fd = (fn(params + eps * d)[0] - fn(params - eps * d)[0]) / (2 * eps)
        assert fd == pytest.approx(g @ d, rel=1e-6)
    # the zero last layer still gives block-Jacobi
    p0 = params.copy()
    p0[-(2 * C * 9 + 2):] = 0.0
    v = rs[0]
    assert np.allclose(learned.learned_apply(v, bj, p0, C, n1, f), bj(v), rtol=0, atol=1e-14)
