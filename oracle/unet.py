"""FP64 CPU oracle of the learned preconditioner (a small U-Net used as M^-1
inside flexible CG) and of its training loss and gradient.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module; the product never
does.

The paper (Sec. 2) compares fixed algebraic preconditioners; a learned
preconditioner is an extension of its Algorithm 1 in which M^-1 r is replaced
by a network evaluated on the residual and the IRLS weights.  Definitions,
written out plainly in numpy FP64 (a matmul per 3x3 tap is the only library
step):

  network input   x = (r / rho, U, V) per pixel, rho = sqrt(mean(r^2)) over
                  the image (x = 0 when rho = 0)
  conv3x3(x)      y[i,j,o] = b[o] + sum_{ky,kx,c} W[o,c,ky,kx] x[i+ky-1, j+kx-1, c],
                  zero outside the image (stride 1, padding 1)
  levels          e0: 3->16 at H x W, e1: 16->32 at H/2, e2: 32->64 at H/4,
                  b3: 64->128 at H/8 (each input the 2x2 average pool of the
                  previous level's output); decoder d2: [a2, up(b3)] 192->64 at
                  H/4, d1: [a1, up(d2)] 96->32 at H/2, d0: [a0, up(d1)] 48->16 at
                  H x W (up = nearest-neighbour 2x); every conv followed by ReLU
  head            y = w_h . d0 + b_h  (1x1, 16 -> 1, linear)
  application     s = D^-1 r + rho * y (the Jacobi step plus the learned correction),
                  D the diagonal of A(U, V), D^-1 = 0 where D = 0; s = 0 on masked pixels
  training loss   per image, with x = r / rho and s~ = D^-1 x + y (the direction in
                  units of rho), the A-norm quality of s~ as a conjugate-gradient
                  search direction for the error e~ = e / rho (A e = r):
                      L = 1 - (s~^T x)^2 / ((s~^T A s~) (e~^T x))
                  i.e. 1 - cos^2 of the A-angle between s~ and e~, the fraction of
                  the error's energy norm that one exact line search along s~ leaves;
                  the batch loss is the mean over images.

Canonical parameter vector (FP32 on the device, FP64 here): for each conv in
the order e0 e1 e2 b3 d2 d1 d0 the weight [Cout][Cin][3][3] then the bias
[Cout]; then the head weight [16] and the head bias [1].

Parity status: conv3x3 and its adjoints are pinned by brute-force loops,
scipy.signal.correlate2d and the adjoint identities; the stencil by the CSR
matrix of the main oracle; the loss by its closed form on a direction
parallel to e (L = 0) and its bounds; the gradient by central finite
differences; the whole network by a hand-built exact identity network
(tests/test_oracle_unet.py).
"""
from __future__ import annotations

import numpy as np

LAYERS = (("e0", 3, 16), ("e1", 16, 32), ("e2", 32, 64), ("b3", 64, 128),
          ("d2", 192, 64), ("d1", 96, 32), ("d0", 48, 16))
HEAD_IN = 16


def param_count() -> int:
    n = sum(co * ci * 9 + co for _, ci, co in LAYERS)
    return n + HEAD_IN + 1


def unflatten(theta):
    """Canonical flat vector -> {name: (W [O,C,3,3], b [O])}, plus ('head', (w [16], b))."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (param_count(),)
    out, k = {}, 0
    for name, ci, co in LAYERS:
        W = theta[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = theta[k:k + co]
        k += co
        out[name] = (W, b)
    out["head"] = (theta[k:k + HEAD_IN], theta[k + HEAD_IN])
    return out


def flatten(p) -> np.ndarray:
    parts = []
    for name, _, _ in LAYERS:
        W, b = p[name]
        parts += [np.ravel(W), np.ravel(b)]
    w, b = p["head"]
    parts += [np.ravel(w), np.atleast_1d(b)]
    return np.concatenate(parts).astype(np.float64)


# ---------------------------------------------------------------- building blocks
def conv3x3(x, W, b):
    """x [B,H,W,C], W [O,C,3,3], b [O] -> [B,H,W,O]; zero padding 1, stride 1."""
    B, H, Wd, C = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (B, H, Wd, W.shape[0])).copy()
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + H, kx:kx + Wd, :] @ W[:, :, ky, kx].T
    return y


def conv3x3_backward(x, W, dy):
    """Gradients of sum(dy * conv3x3(x, W, b)): (dx, dW, db)."""
    B, H, Wd, C = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            win = xp[:, ky:ky + H, kx:kx + Wd, :]
            dW[:, :, ky, kx] = np.tensordot(dy, win, axes=([0, 1, 2], [0, 1, 2]))
            dxp[:, ky:ky + H, kx:kx + Wd, :] += dy @ W[:, :, ky, kx]
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, 1:-1, 1:-1, :], dW, db


def pool2(x):
    """2x2 average pool, [B,H,W,C] -> [B,H/2,W/2,C]."""
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def relu(x):
    return np.maximum(x, 0.0)


# ---------------------------------------------------------------- network
def forward(theta, x):
    """x [B,H,W,3] (H, W multiples of 8) -> (y [B,H,W], cache)."""
    p = unflatten(theta)
    c = {"x": x}
    c["a0"] = relu(conv3x3(x, *p["e0"]))
    c["p0"] = pool2(c["a0"])
    c["a1"] = relu(conv3x3(c["p0"], *p["e1"]))
    c["p1"] = pool2(c["a1"])
    c["a2"] = relu(conv3x3(c["p1"], *p["e2"]))
    c["p2"] = pool2(c["a2"])
    c["a3"] = relu(conv3x3(c["p2"], *p["b3"]))
    c["c2"] = np.concatenate([c["a2"], up2(c["a3"])], axis=3)
    c["g2"] = relu(conv3x3(c["c2"], *p["d2"]))
    c["c1"] = np.concatenate([c["a1"], up2(c["g2"])], axis=3)
    c["g1"] = relu(conv3x3(c["c1"], *p["d1"]))
    c["c0"] = np.concatenate([c["a0"], up2(c["g1"])], axis=3)
    c["g0"] = relu(conv3x3(c["c0"], *p["d0"]))
    w, b = p["head"]
    y = c["g0"] @ w + b
    return y, c


def _sum_up(d):
    """Adjoint of up2: sum over each 2x2 block."""
    B, H, W, C = d.shape
    return d.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def backward(theta, c, dy):
    """Gradient of sum(dy * y) with respect to theta (canonical layout)."""
    p = unflatten(theta)
    g = {}
    w, _ = p["head"]
    g["head"] = (np.tensordot(dy, c["g0"], axes=([0, 1, 2], [0, 1, 2])), dy.sum())
    d = dy[..., None] * w * (c["g0"] > 0)
    dc0, *g["d0"] = conv3x3_backward(c["c0"], p["d0"][0], d)
    d = _sum_up(dc0[..., 16:]) * (c["g1"] > 0)
    dc1, *g["d1"] = conv3x3_backward(c["c1"], p["d1"][0], d)
    d = _sum_up(dc1[..., 32:]) * (c["g2"] > 0)
    dc2, *g["d2"] = conv3x3_backward(c["c2"], p["d2"][0], d)
    d = _sum_up(dc2[..., 64:]) * (c["a3"] > 0)
    dp2, *g["b3"] = conv3x3_backward(c["p2"], p["b3"][0], d)
    d = (dc2[..., :64] + up2(dp2) / 4.0) * (c["a2"] > 0)
    dp1, *g["e2"] = conv3x3_backward(c["p1"], p["e2"][0], d)
    d = (dc1[..., :32] + up2(dp1) / 4.0) * (c["a1"] > 0)
    dp0, *g["e1"] = conv3x3_backward(c["p0"], p["e1"][0], d)
    d = (dc0[..., :16] + up2(dp0) / 4.0) * (c["a0"] > 0)
    _, *g["e0"] = conv3x3_backward(c["x"], p["e0"][0], d)
    return flatten({k: tuple(v) for k, v in g.items()})


# ---------------------------------------------------------------- preconditioner use
def diag(U, V):
    """D of Eq. (Axb): U_{i,j-1} + U_{i,j} + V_{i-1,j} + V_{i,j} (U, V [...,H,W])."""
    U, V = np.asarray(U, np.float64), np.asarray(V, np.float64)
    D = U + V
    D[..., :, 1:] += U[..., :, :-1]
    D[..., 1:, :] += V[..., :-1, :]
    return D


def stencil(U, V, x):
    """(A x)_{ij} = D x_{ij} - U_{ij} x_{i,j+1} - U_{i,j-1} x_{i,j-1} - V_{ij} x_{i+1,j} - V_{i-1,j} x_{i-1,j}."""
    U, V, x = (np.asarray(a, np.float64) for a in (U, V, x))
    y = diag(U, V) * x
    y[..., :, :-1] -= U[..., :, :-1] * x[..., :, 1:]
    y[..., :, 1:] -= U[..., :, :-1] * x[..., :, :-1]
    y[..., :-1, :] -= V[..., :-1, :] * x[..., 1:, :]
    y[..., 1:, :] -= V[..., :-1, :] * x[..., :-1, :]
    return y


def jacobi(U, V, x):
    D = diag(U, V)
    return np.where(D > 0, x / np.where(D > 0, D, 1.0), 0.0)


def network_input(r, U, V):
    """r, U, V [B,H,W] -> (x [B,H,W,3], rho [B]) with x = (r / rho, U, V)."""
    r = np.asarray(r, np.float64)
    if r.ndim == 2:
        r, U, V = r[None], np.asarray(U)[None], np.asarray(V)[None]
    rho = np.sqrt(np.mean(r * r, axis=(1, 2)))
    scale = np.where(rho > 0, 1.0 / np.where(rho > 0, rho, 1.0), 0.0)
    x = np.stack([r * scale[:, None, None], U, V], axis=3)
    return x, rho


def apply(theta, r, U, V, mask=None, pad=128):
    """One preconditioner application s = D^-1 r + rho * N_theta(r / rho, U, V)
    (0 on masked pixels).  rho is the RMS over the map itself; the network runs
    on the input zero-padded to multiples of ``pad`` rows and columns, and its
    output is cropped back."""
    x, rho = network_input(r, U, V)
    B, H, W, _ = x.shape
    Hn, Wn = -(-H // pad) * pad, -(-W // pad) * pad
    xp = np.zeros((B, Hn, Wn, 3))
    xp[:, :H, :W, :] = x
    y, _ = forward(theta, xp)
    s = jacobi(x[..., 1], x[..., 2], np.asarray(r, np.float64).reshape(B, H, W)) + rho[:, None, None] * y[:, :H, :W]
    if mask is not None:
        s = np.where(np.asarray(mask, bool), 0.0, s)
    return s[0] if np.ndim(r) == 2 else s


def direction_loss(x, U, V, e_scaled, y):
    """Per-image loss 1 - (s^T x)^2 / ((s^T A s)(e^T x)) with s = D^-1 x + y, and dL/dy."""
    s = jacobi(U, V, x) + y
    As = stencil(U, V, s)
    a = np.sum(s * x, axis=(1, 2))
    b = np.sum(s * As, axis=(1, 2))
    g = np.sum(e_scaled * x, axis=(1, 2))
    L = 1.0 - a * a / (b * g)
    # dL/ds = -(2 a / (b g)) x + (2 a^2 / (b^2 g)) A s  (A symmetric)
    dy = (-(2 * a / (b * g)))[:, None, None] * x + (2 * a * a / (b * b * g))[:, None, None] * As
    return L, dy


def loss_grad(theta, r, U, V, e):
    """Training loss (mean over the batch of the direction loss) and its gradient."""
    x, rho = network_input(r, U, V)
    U = np.asarray(U, np.float64).reshape(x.shape[:3])
    V = np.asarray(V, np.float64).reshape(x.shape[:3])
    e = np.asarray(e, np.float64).reshape(x.shape[:3])
    es = e / rho[:, None, None]
    y, c = forward(theta, x)
    L, dy = direction_loss(x[..., 0], U, V, es, y)
    B = x.shape[0]
    return float(np.mean(L)), backward(theta, c, dy / B)


def zero_params():
    """N = 0: the application is the Jacobi step."""
    return np.zeros(param_count())
def identity_params():
    """Parameters for which N(x) = x_r exactly: e0 splits r into relu(r) and
    relu(-r), d0 passes both through, the head takes their difference."""
    p = {name: (np.zeros((co, ci, 3, 3)), np.zeros(co)) for name, ci, co in LAYERS}
    p["e0"][0][0, 0, 1, 1] = 1.0
    p["e0"][0][1, 0, 1, 1] = -1.0
    p["d0"][0][0, 0, 1, 1] = 1.0
    p["d0"][0][1, 1, 1, 1] = 1.0
    w = np.zeros(HEAD_IN)
    w[0], w[1] = 1.0, -1.0
    p["head"] = (w, 0.0)
    return flatten(p)
