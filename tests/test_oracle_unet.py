"""Pins of the learned-preconditioner oracle (oracle/unet.py) against facts
that do not come from the oracle itself: brute-force loops, an independent
library correlation, adjoint identities, central finite differences and an
exactly constructed identity network."""
import numpy as np
import pytest

from oracle import unet


def _rng(seed):
    return np.random.default_rng(seed)


def test_param_count():
    # 3x3 convs of the stated widths plus biases, plus the 16 -> 1 head
    expect = (16 * 3 * 9 + 16) + (32 * 16 * 9 + 32) + (64 * 32 * 9 + 64) + (128 * 64 * 9 + 128) \
        + (64 * 192 * 9 + 64) + (32 * 96 * 9 + 32) + (16 * 48 * 9 + 16) + 17
    assert unet.param_count() == expect == 242721


def test_conv3x3_brute_force():
    rng = _rng(1)
    x = rng.standard_normal((2, 5, 4, 3))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = unet.conv3x3(x, W, b)
    B, H, Wd, C = x.shape
    for n in range(B):
        for i in range(H):
            for j in range(Wd):
                for o in range(2):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            ii, jj = i + ky - 1, j + kx - 1
                            if 0 <= ii < H and 0 <= jj < Wd:
                                for c in range(C):
                                    acc += W[o, c, ky, kx] * x[n, ii, jj, c]
                    assert abs(y[n, i, j, o] - acc) < 1e-12


def test_conv3x3_vs_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = _rng(2)
    x = rng.standard_normal((1, 9, 7, 2))
    W = rng.standard_normal((3, 2, 3, 3))
    y = unet.conv3x3(x, W, np.zeros(3))
    for o in range(3):
        ref = sum(signal.correlate2d(x[0, :, :, c], W[o, c], mode="same", boundary="fill")
                  for c in range(2))
        np.testing.assert_allclose(y[0, :, :, o], ref, rtol=0, atol=1e-12)


def test_conv_adjoint_identity():
    rng = _rng(3)
    x = rng.standard_normal((2, 6, 8, 4))
    W = rng.standard_normal((5, 4, 3, 3))
    dy = rng.standard_normal((2, 6, 8, 5))
    y = unet.conv3x3(x, W, np.zeros(5))
    dx, dW, db = unet.conv3x3_backward(x, W, dy)
    # <conv(x), dy> = <x, conv^T dy> = <W, dW>
    lhs = np.sum(y * dy)
    assert abs(lhs - np.sum(x * dx)) < 1e-9 * abs(lhs) + 1e-9
    assert abs(lhs - np.sum(W * dW)) < 1e-9 * abs(lhs) + 1e-9
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1, 2)))


def test_pool_up_adjoint():
    rng = _rng(4)
    x = rng.standard_normal((1, 8, 6, 3))
    z = rng.standard_normal((1, 4, 3, 3))
    assert abs(np.sum(unet.pool2(x) * z) - np.sum(x * unet.up2(z)) / 4.0) < 1e-12
    np.testing.assert_allclose(unet.pool2(unet.up2(z)), z)


def test_identity_network_is_exact():
    rng = _rng(5)
    r = rng.standard_normal((16, 24))
    U = rng.uniform(0, 1, (16, 24))
    V = rng.uniform(0, 1, (16, 24))
    x, rho = unet.network_input(r, U, V)
    y, _ = unet.forward(unet.identity_params(), x)
    np.testing.assert_allclose(y[0] * rho[0], r, rtol=1e-14, atol=1e-14)
    # the application adds the Jacobi step; masked pixels are zero
    s = unet.apply(unet.identity_params(), r, U, V)
    np.testing.assert_allclose(s, unet.jacobi(U, V, r) + r, rtol=1e-13, atol=1e-13)
    mask = np.zeros((16, 24), bool)
    mask[3:5, 7:9] = True
    s = unet.apply(unet.identity_params(), r, U, V, mask)
    assert np.all(s[mask] == 0)


def test_zero_residual_gives_zero_input():
    x, rho = unet.network_input(np.zeros((8, 8)), np.ones((8, 8)), np.ones((8, 8)))
    assert rho[0] == 0 and np.all(x[..., 0] == 0) and np.all(x[..., 1] == 1)


def test_zero_network_is_jacobi():
    rng = _rng(15)
    r = rng.standard_normal((20, 12))
    U = rng.uniform(0, 1, (20, 12))
    V = rng.uniform(0, 1, (20, 12))
    np.testing.assert_allclose(unet.apply(unet.zero_params(), r, U, V), unet.jacobi(U, V, r), rtol=0, atol=0)


def test_stencil_and_diag_match_the_csr_matrix():
    """The U-Net oracle's matrix-free A is the main oracle's CSR A of Eq. (Axb)."""
    import oracle
    rng = _rng(16)
    H, W = 7, 9
    U = rng.uniform(0, 1, (H, W))
    V = rng.uniform(0, 1, (H, W))
    U[:, -1] = 0.0
    V[-1, :] = 0.0
    z = np.zeros((H, W))
    A = oracle.assemble(U, V, z, z)
    x = rng.standard_normal((H, W))
    np.testing.assert_allclose(unet.stencil(U, V, x), A.matvec(x), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(unet.diag(U, V).ravel(), np.diag(A.dense()), rtol=1e-14)


def _consistent_pair(B, H, W, seed):
    rng = _rng(seed)
    U = rng.uniform(0.1, 1, (B, H, W))
    V = rng.uniform(0.1, 1, (B, H, W))
    U[..., :, -1] = 0.0
    V[..., -1, :] = 0.0
    e = rng.standard_normal((B, H, W))
    r = unet.stencil(U, V, e)
    return r, U, V, e


def test_direction_loss_closed_forms():
    r, U, V, e = _consistent_pair(2, 16, 16, 17)
    x, rho = unet.network_input(r, U, V)
    es = e / rho[:, None, None]
    # s parallel to the error: one line search is exact, L = 0
    y = 3.0 * es - unet.jacobi(U, V, x[..., 0])
    L, _ = unet.direction_loss(x[..., 0], U, V, es, y)
    np.testing.assert_allclose(L, 0.0, atol=1e-12)
    # any direction: 0 <= L <= 1 (Cauchy-Schwarz in the A inner product)
    rng = _rng(18)
    for _ in range(5):
        L, _ = unet.direction_loss(x[..., 0], U, V, es, rng.standard_normal(es.shape))
        assert np.all(L >= -1e-12) and np.all(L <= 1 + 1e-12)
    # a direction A-orthogonal to the error gives L = 1
    s0 = rng.standard_normal(es.shape)
    for b in range(2):
        As0 = unet.stencil(U[b], V[b], s0[b])
        s0[b] -= np.sum(s0[b] * x[b, ..., 0]) / np.sum(es[b] * x[b, ..., 0]) * es[b]
        assert abs(np.sum(s0[b] * x[b, ..., 0])) < 1e-9 * np.linalg.norm(As0)
    y = s0 - unet.jacobi(U, V, x[..., 0])
    L, _ = unet.direction_loss(x[..., 0], U, V, es, y)
    np.testing.assert_allclose(L, 1.0, atol=1e-9)


def _random_theta(seed, scale=1.0):
    rng = _rng(seed)
    p = {}
    for name, ci, co in unet.LAYERS:
        p[name] = (rng.standard_normal((co, ci, 3, 3)) * scale * np.sqrt(2.0 / (9 * ci)),
                   rng.standard_normal(co) * 0.1)
    p["head"] = (rng.standard_normal(16) * 0.25, 0.05)
    return unet.flatten(p)


def test_gradient_central_differences():
    """Every layer's weight and bias gradient against central differences of the loss."""
    rng = _rng(7)
    theta = _random_theta(8)
    r, U, V, e = _consistent_pair(2, 16, 16, 19)
    loss, g = unet.loss_grad(theta, r, U, V, e)
    assert 0 < loss < 1
    offsets, k = {}, 0
    for name, ci, co in unet.LAYERS:
        offsets[name] = (k, k + co * ci * 9)  # first weight, first bias
        k += co * ci * 9 + co
    offsets["head"] = (k, k + 16)
    picks = []
    for name, (w0, b0) in offsets.items():
        n_w = b0 - w0
        picks += [w0 + int(i) for i in rng.choice(n_w, 3, replace=False)] + [b0]
    h = 1e-6
    for i in picks:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (unet.loss_grad(tp, r, U, V, e)[0] - unet.loss_grad(tm, r, U, V, e)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_gradient_planted_mistake_is_caught(monkeypatch):
    """A wrong bias gradient planted in the conv backward must fail the
    central-difference pin."""
    theta = _random_theta(10)
    r, U, V, e = _consistent_pair(1, 16, 16, 20)
    k = sum(co * ci * 9 + co for _, ci, co in unet.LAYERS[:-1]) + 16 * 48 * 9  # first bias of d0
    h = 1e-6
    tp, tm = theta.copy(), theta.copy()
    tp[k] += h
    tm[k] -= h
    fd = (unet.loss_grad(tp, r, U, V, e)[0] - unet.loss_grad(tm, r, U, V, e)[0]) / (2 * h)
    real_backward = unet.conv3x3_backward

    def broken(x, W, dy):
        dx, dW, db = real_backward(x, W, dy)
        return dx, dW, db * 0.5
    monkeypatch.setattr(unet, "conv3x3_backward", broken)
    _, g_bad = unet.loss_grad(theta, r, U, V, e)
    assert abs(fd) > 1e-4
    assert abs(fd - g_bad[k]) > 1e-6 * max(abs(fd), 1e-3)
