"""Pins of the network oracle (oracle/unet.py) to things other than itself:
library routines (scipy's 2-D correlation, numpy's dense solve, torch's
bfloat16 conversion), closed forms, exact adjoint identities of linear maps,
and central finite differences of the loss for every backward pass.
"""
import numpy as np
import pytest

from oracle import unet


def rnd(seed, *shape):
    return np.random.default_rng(seed).standard_normal(shape)


def small_params(seed, arch=unet.ARCH):
    """Random weights scaled by 1/sqrt(fan-in) so activations stay O(1)."""
    rng = np.random.default_rng(seed)
    parts = []
    for n, ws, bs in unet.param_shapes(arch):
        fan = ws[1] * ws[2] * ws[3]
        parts.append(rng.standard_normal(int(np.prod(ws))) / np.sqrt(fan))
        parts.append(0.1 * rng.standard_normal(bs[0]))
    return np.concatenate(parts)


def test_conv_is_scipy_correlation():
    from scipy.signal import correlate2d
    x = rnd(1, 2, 7, 9, 3)
    w = rnd(2, 4, 3, 3, 3)
    b = rnd(3, 4)
    y = unet.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(y[n, :, :, o], ref, atol=1e-12)
    # 1x1 kernel: a matrix product over channels
    w1 = rnd(4, 2, 1, 1, 3)
    assert np.allclose(unet.conv(x, w1, np.zeros(2)), np.einsum("nijc,oc->nijo", x, w1[:, 0, 0, :]))


def test_conv_backward_adjoint_identities():
    """conv is bilinear: <conv(x, w, 0), g> = <x, dx> = <w, dw>, and db = sum g."""
    x, w, g = rnd(5, 2, 6, 8, 3), rnd(6, 5, 3, 3, 3), rnd(7, 2, 6, 8, 5)
    y = unet.conv(x, w, np.zeros(5))
    dx, dw, db = unet.conv_backward(x, w, g)
    s = np.sum(y * g)
    assert abs(np.sum(x * dx) - s) < 1e-10 * abs(s) + 1e-10
    assert abs(np.sum(w * dw) - s) < 1e-10 * abs(s) + 1e-10
    assert np.allclose(db, g.sum(axis=(0, 1, 2)))


def test_pool_and_prolongation():
    x = rnd(8, 1, 4, 6, 2)
    # pooling a prolonged field gives it back; a constant stays constant
    assert np.allclose(unet.pool(unet.up(x)), x)
    assert np.allclose(unet.pool(np.full((1, 4, 4, 1), 3.5)), 3.5)
    # a bilinear field averages to its value at the coarse-cell centre
    i, j = np.meshgrid(np.arange(8), np.arange(6), indexing="ij")
    f = (2.0 * i + 3.0 * j + 1.0)[None, :, :, None]
    I, J = np.meshgrid(np.arange(4) * 2 + 0.5, np.arange(3) * 2 + 0.5, indexing="ij")
    assert np.allclose(unet.pool(f)[0, :, :, 0], 2.0 * I + 3.0 * J + 1.0)
    # adjoints
    y = rnd(9, 1, 2, 3, 2)
    assert abs(np.sum(unet.pool(x) * y) - np.sum(x * unet.pool_backward(y))) < 1e-12
    z = rnd(10, 1, 8, 12, 2)
    assert abs(np.sum(unet.up(x) * z) - np.sum(x * unet.up_backward(z))) < 1e-12


def test_param_count_and_pack():
    n = unet.n_params()
    assert 150_000 < n < 300_000          # "about 0.2M parameters"
    th = np.arange(n, dtype=np.float64)
    assert np.array_equal(unet.pack({k: v for k, v in unet.unpack(th).items()}), th)


@pytest.mark.parametrize("act", [True, False])
def test_network_gradient_finite_differences(act):
    """backward() against central differences of sum(g * N(x)) along random
    directions and along single parameters."""
    th = small_params(11)
    x = rnd(12, 2, 8, 16)
    g = rnd(13, 2, 8, 16)
    y, cache = unet.forward(th, x, act=act)
    gt, gx = unet.backward(cache, g)

    def f(t, xx=x):
        return np.sum(g * unet.forward(t, xx, act=act)[0])

    h = 1e-6
    rng = np.random.default_rng(14)
    for _ in range(3):
        d = rng.standard_normal(th.size)
        fd = (f(th + h * d) - f(th - h * d)) / (2 * h)
        assert abs(fd - gt @ d) <= 1e-6 * (abs(fd) + 1e-3), (fd, gt @ d)
    for idx in rng.choice(th.size, 12, replace=False):
        e = np.zeros(th.size)
        e[idx] = 1.0
        fd = (f(th + h * e) - f(th - h * e)) / (2 * h)
        assert abs(fd - gt[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, gt[idx])
    dxd = rng.standard_normal(x.shape)
    fd = (f(th, x + h * dxd) - f(th, x - h * dxd)) / (2 * h)
    assert abs(fd - np.sum(gx * dxd)) <= 1e-6 * (abs(fd) + 1e-3)


def dense_helmholtz(c, ax, az):
    """The matrix of A written from its definition: diagonal c_i + sum of the
    cell's interior face coefficients, -a_f to the neighbour across f."""
    H, W = c.shape
    M = np.zeros((H * W, H * W))
    for i in range(H):
        for j in range(W):
            k = i * W + j
            M[k, k] += c[i, j]
            for (ii, jj, a) in ((i, j - 1, ax[i, j]), (i, j + 1, ax[i, j + 1]),
                                (i - 1, j, az[i, j]), (i + 1, j, az[i + 1, j])):
                if 0 <= ii < H and 0 <= jj < W:
                    M[k, k] += a
                    M[k, ii * W + jj] -= a
    return M


def coeffs(seed, H, W):
    rng = np.random.default_rng(seed)
    c = 1.0 + rng.random((H, W))
    ax = 0.5 + rng.random((H, W + 1))
    az = 0.5 + rng.random((H + 1, W))
    ax[:, 0] = ax[:, -1] = 0.0
    az[0, :] = az[-1, :] = 0.0
    return c, ax, az


def test_helmholtz_apply_and_energy_minimiser():
    H, W = 4, 6
    c, ax, az = coeffs(15, H, W)
    M = dense_helmholtz(c, ax, az)
    e = rnd(16, H, W)
    assert np.allclose(unet.helmholtz_apply(e, c, ax, az).ravel(), M @ e.ravel())
    assert np.allclose(M, M.T) and np.linalg.eigvalsh(M).min() > 0
    # the energy loss is minimal at A_hat^-1 x, with zero gradient there
    x = rnd(17, 1, H, W)
    nstar = np.linalg.solve(M / c.mean(), x[0].ravel()).reshape(H, W)[None]
    l0, g0 = unet.energy_loss(nstar, x, c[None], ax[None], az[None])
    assert np.abs(g0).max() < 1e-12
    for s in range(3):
        d = rnd(18 + s, 1, H, W)
        l1, _ = unet.energy_loss(nstar + 1e-2 * d, x, c[None], ax[None], az[None])
        assert l1 > l0
    # and its gradient matches central differences
    n = rnd(21, 1, H, W)
    _, g = unet.energy_loss(n, x, c[None], ax[None], az[None])
    d = rnd(22, 1, H, W)
    h = 1e-6
    fd = (unet.energy_loss(n + h * d, x, c[None], ax[None], az[None])[0]
          - unet.energy_loss(n - h * d, x, c[None], ax[None], az[None])[0]) / (2 * h)
    assert abs(fd - np.sum(g * d)) < 1e-8


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([rnd(23, 1000) * 10.0 ** rnd(24, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 65504.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(unet.bf16_round(x), ref)
    assert unet.bf16_round(1.0 + 2 ** -8) == 1.0            # tie to even
    assert unet.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_bf16_backward_equals_fp64_backward_on_representable_data():
    """With operands already bfloat16 and every rounding point exact (a
    network of exactly representable integers), the bfloat16 path is the
    FP64 path."""
    arch = [("a", 1, 16, 3, True, "x"), ("b", 16, 16, 3, True, "a"), ("out", 16, 1, 1, False, "b")]
    rng = np.random.default_rng(25)
    th = np.concatenate([rng.integers(-2, 3, unet.param_shapes(arch)[0][1]).ravel(), np.zeros(16),
                         rng.integers(-1, 2, unet.param_shapes(arch)[1][1]).ravel(), np.zeros(16),
                         rng.integers(-1, 2, 16), [0.0]]).astype(np.float64)
    x = rng.integers(-2, 3, (1, 8, 8)).astype(np.float64)
    g = rng.integers(-2, 3, (1, 8, 8)).astype(np.float64)
    y0, c0 = unet.forward(th, x, arch=arch)
    y1, c1 = unet.forward(th, x, bf16=True, arch=arch)
    assert np.array_equal(y0, y1)
    assert np.array_equal(unet.backward(c0, g)[0], unet.backward(c1, g)[0])


def test_adam_first_step():
    """At t = 1 the bias-corrected moments are g and g^2: the step is
    lr g / (|g| + eps)."""
    th, g = rnd(26, 50), rnd(27, 50)
    t1, m, v = unet.adam(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
